// Measured peaks of the device: FP64 and FP32 fused multiply-add throughput with independent
// dependency chains in every thread of a grid that fills every SM (the denominators of the ALU
// rooflines), and the HBM bandwidth of a read-only stream (context for the read-dominated block
// products, whose roofline stays the copy bandwidth). The paper has no counterpart.
#include <algorithm>

#include "dg_internal.h"

namespace dg {
namespace {

constexpr int kPeakChains = 8;  // independent FMA chains per thread (hides the FMA latency)

template <class T>
__global__ void __launch_bounds__(256) fma_chain_kernel(int iters, T b, T c, T* sink) {
  T a[kPeakChains];
#pragma unroll
  for (int j = 0; j < kPeakChains; ++j) a[j] = T(threadIdx.x + j) * T(1e-3);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int j = 0; j < kPeakChains; ++j) a[j] = fma(a[j], b, c);
  }
  T s = T(0);
#pragma unroll
  for (int j = 0; j < kPeakChains; ++j) s += a[j];
  if (s == T(-12345.678)) sink[blockIdx.x] = s;  // keeps the chains alive; never true for these inputs
}

template <class T>
int measure(Handle* h, int nsm, double* tflops, cudaStream_t st) {
  T* sink = nullptr;
  DG_CUDA(h, cudaMalloc(&sink, sizeof(T) * 4096));
  const int blocks = nsm * 8, threads = 256;
  const int iters = sizeof(T) == 8 ? 2048 : 16384;
  cudaEvent_t e0, e1;
  DG_CUDA(h, cudaEventCreate(&e0));
  DG_CUDA(h, cudaEventCreate(&e1));
  const T b = T(0.999999), c = T(1e-7);
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {  // first launch warms up; best of the other three
    DG_CUDA(h, cudaEventRecord(e0, st));
    fma_chain_kernel<T><<<blocks, threads, 0, st>>>(iters, b, c, sink);
    DG_CUDA(h, cudaGetLastError());
    DG_CUDA(h, cudaEventRecord(e1, st));
    DG_CUDA(h, cudaEventSynchronize(e1));
    float ms = 0.f;
    DG_CUDA(h, cudaEventElapsedTime(&ms, e0, e1));
    if (rep > 0) best = std::min(best, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  const double flop = 2.0 * kPeakChains * 16.0 * iters * (double)blocks * threads;
  *tflops = flop / (best * 1e-3) / 1e12;
  return DG_OK;
}

// HBM read streaming: every thread sums 16-byte loads of a buffer far larger than L2 (grid-stride,
// four loads in flight per thread); one value per CTA is written
__global__ void __launch_bounds__(256) read_stream_kernel(long long n4, const float4* __restrict__ src, float* sink) {
  float s = 0.0f;
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  for (; i + 3 * stride < n4; i += 4 * stride) {
    const float4 a = src[i], b = src[i + stride], c = src[i + 2 * stride], d = src[i + 3 * stride];
    s += (a.x + a.y + a.z + a.w) + (b.x + b.y + b.z + b.w) + (c.x + c.y + c.z + c.w) + (d.x + d.y + d.z + d.w);
  }
  for (; i < n4; i += stride) {
    const float4 a = src[i];
    s += a.x + a.y + a.z + a.w;
  }
  if (s == -12345.678f) sink[blockIdx.x] = s;  // never true for the zero-filled buffer
}

int measure_read(Handle* h, int nsm, double* gbs, cudaStream_t st) {
  const size_t bytes = (size_t)2 << 30;  // 2 GiB, 16 x L2
  float4* buf = nullptr;
  float* sink = nullptr;
  DG_CUDA(h, cudaMalloc(&buf, bytes));
  DG_CUDA(h, cudaMalloc(&sink, sizeof(float) * 65536));
  DG_CUDA(h, cudaMemsetAsync(buf, 0, bytes, st));
  cudaEvent_t e0, e1;
  DG_CUDA(h, cudaEventCreate(&e0));
  DG_CUDA(h, cudaEventCreate(&e1));
  const long long n4 = (long long)(bytes / 16);
  const int blocks = nsm * 8;
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {
    DG_CUDA(h, cudaEventRecord(e0, st));
    read_stream_kernel<<<blocks, 256, 0, st>>>(n4, buf, sink);
    DG_CUDA(h, cudaGetLastError());
    DG_CUDA(h, cudaEventRecord(e1, st));
    DG_CUDA(h, cudaEventSynchronize(e1));
    float ms = 0.f;
    DG_CUDA(h, cudaEventElapsedTime(&ms, e0, e1));
    if (rep > 0) best = std::min(best, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  cudaFree(sink);
  *gbs = (double)bytes / (best * 1e-3) / 1e9;
  return DG_OK;
}

}  // namespace
}  // namespace dg

extern "C" int dg_measure_peak(int which, double* tflops, void* stream) {
  using namespace dg;
  if (!tflops || (which != DG_PEAK_FP64_FMA && which != DG_PEAK_FP32_FMA && which != DG_PEAK_HBM_READ))
    return DG_ERR_ARG;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return DG_ERR_CUDA;
  Handle tmp;  // error text holder only
  const cudaStream_t st = as_stream(stream);
  if (which == DG_PEAK_HBM_READ) return measure_read(&tmp, nsm, tflops, st);
  return which == DG_PEAK_FP64_FMA ? measure<double>(&tmp, nsm, tflops, st) : measure<float>(&tmp, nsm, tflops, st);
}
