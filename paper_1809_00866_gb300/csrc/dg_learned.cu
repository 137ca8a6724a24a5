// Learned coarse-level correction (no counterpart in the paper): a per-element network
// 112 -> 128 -> 128 -> 16 with GELU that maps the coarsest-level (P1) right-hand side of an
// element and of its six face neighbours to the element's correction. Inference and training
// run on the tensor cores with BF16 operands and FP32 accumulation (mma.sync m16n8k16); the
// packed BF16 weights reach shared memory by one bulk asynchronous copy (cp.async.bulk) that
// overlaps the gather of the features.
#include <cuda_bf16.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "dg_async.h"
#include "dg_internal.h"

namespace dg {

namespace {

constexpr int kIn = DG_MLP_IN, kHid = DG_MLP_HIDDEN, kOut = DG_MLP_OUT;
// offsets of the FP32 parameter vector theta
constexpr int oW1 = 0, ob1 = oW1 + kHid * kIn, oW2 = ob1 + kHid, ob2 = oW2 + kHid * kHid, oW3 = ob2 + kHid,
              ob3 = oW3 + kOut * kHid, kNP = ob3 + kOut;
static_assert(kNP == DG_MLP_NPARAM, "parameter count");

// Packed BF16 network (device and shared memory): rows padded to 120 / 136 entries so that
// the fragment loads of a warp hit 32 different banks; biases b1, b2, b3 in FP32 at the end.
constexpr int kLd1 = 120, kLd2 = 136;
constexpr int kPW1 = 0;
constexpr int kPW2 = kPW1 + kHid * kLd1 * 2;
constexpr int kPW3 = kPW2 + kHid * kLd2 * 2;
constexpr int kPB = kPW3 + kOut * kLd2 * 2;
constexpr int kPBytes = kPB + (2 * kHid + kOut) * 4;
static_assert(kPW2 % 16 == 0 && kPW3 % 16 == 0 && kPB % 16 == 0 && kPBytes % 16 == 0, "16-byte parts");

constexpr int kWarps = 4, kRows = 16 * kWarps;  // rows (elements or samples) per CTA

// ---------------------------------------------------------------- PTX helpers
// D += A B, m16n8k16, A row-major bf16, B column-major bf16, FP32 accumulators
__device__ __forceinline__ void mma16816(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// two floats -> packed bf16x2 (round to nearest even), the first in the low half
__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  uint32_t u;
  memcpy(&u, &v, 4);
  return u;
}
__device__ __forceinline__ uint16_t bf16_bits(float x) {
  __nv_bfloat16 v = __float2bfloat16_rn(x);
  uint16_t u;
  memcpy(&u, &v, 2);
  return u;
}
__device__ __forceinline__ float bf16_to_f(uint16_t u) {
  return __uint_as_float(static_cast<uint32_t>(u) << 16);
}

constexpr float kRsqrt2 = 0.70710678118654752f, kRsqrt2Pi = 0.39894228040143268f;
__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * kRsqrt2)); }
__device__ __forceinline__ float gelu_d(float z) {
  return 0.5f * (1.0f + erff(z * kRsqrt2)) + z * kRsqrt2Pi * expf(-0.5f * z * z);
}

// theta (FP32) -> packed BF16 network; one thread per packed slot
__global__ void pack_kernel(const float* __restrict__ theta, unsigned char* __restrict__ net) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  uint16_t* W1 = reinterpret_cast<uint16_t*>(net + kPW1);
  uint16_t* W2 = reinterpret_cast<uint16_t*>(net + kPW2);
  uint16_t* W3 = reinterpret_cast<uint16_t*>(net + kPW3);
  float* B = reinterpret_cast<float*>(net + kPB);
  if (i < kHid * kLd1) {
    const int r = i / kLd1, c = i % kLd1;
    W1[i] = c < kIn ? bf16_bits(theta[oW1 + r * kIn + c]) : 0;
    return;
  }
  i -= kHid * kLd1;
  if (i < kHid * kLd2) {
    const int r = i / kLd2, c = i % kLd2;
    W2[i] = c < kHid ? bf16_bits(theta[oW2 + r * kHid + c]) : 0;
    return;
  }
  i -= kHid * kLd2;
  if (i < kOut * kLd2) {
    const int r = i / kLd2, c = i % kLd2;
    W3[i] = c < kHid ? bf16_bits(theta[oW3 + r * kHid + c]) : 0;
    return;
  }
  i -= kOut * kLd2;
  if (i < kHid) B[i] = theta[ob1 + i];
  else if (i < 2 * kHid) B[i] = theta[ob2 + i - kHid];
  else if (i < 2 * kHid + kOut) B[i] = theta[ob3 + i - 2 * kHid];
}
constexpr int kPackSlots = kHid * kLd1 + kHid * kLd2 + kOut * kLd2 + 2 * kHid + kOut;

// Layers 2 and 3 and the bias/GELU epilogues of one warp's 16 rows, from the layer-1
// accumulators; out[j][.] holds the output columns 8j + 2t, 8j + 2t + 1 of rows g, g + 8.
__device__ __forceinline__ void mlp_tail(const unsigned char* sm, int g, int t, float (&acc)[16][4],
                                         float (&out)[2][4]) {
  const uint16_t* W2s = reinterpret_cast<const uint16_t*>(sm + kPW2);
  const uint16_t* W3s = reinterpret_cast<const uint16_t*>(sm + kPW3);
  const float* Bs = reinterpret_cast<const float*>(sm + kPB);
  uint32_t a[8][4];
#pragma unroll
  for (int kk = 0; kk < 8; ++kk) {
    a[kk][0] = pack2(gelu(acc[2 * kk][0]), gelu(acc[2 * kk][1]));
    a[kk][1] = pack2(gelu(acc[2 * kk][2]), gelu(acc[2 * kk][3]));
    a[kk][2] = pack2(gelu(acc[2 * kk + 1][0]), gelu(acc[2 * kk + 1][1]));
    a[kk][3] = pack2(gelu(acc[2 * kk + 1][2]), gelu(acc[2 * kk + 1][3]));
  }
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const float2 bb = *reinterpret_cast<const float2*>(Bs + kHid + 8 * j + 2 * t);
    acc[j][0] = bb.x; acc[j][1] = bb.y; acc[j][2] = bb.x; acc[j][3] = bb.y;
  }
#pragma unroll
  for (int kk = 0; kk < 8; ++kk)
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const uint32_t* w = reinterpret_cast<const uint32_t*>(W2s + (8 * j + g) * kLd2 + 16 * kk + 2 * t);
      mma16816(acc[j], a[kk], w[0], w[4]);
    }
#pragma unroll
  for (int kk = 0; kk < 8; ++kk) {
    a[kk][0] = pack2(gelu(acc[2 * kk][0]), gelu(acc[2 * kk][1]));
    a[kk][1] = pack2(gelu(acc[2 * kk][2]), gelu(acc[2 * kk][3]));
    a[kk][2] = pack2(gelu(acc[2 * kk + 1][0]), gelu(acc[2 * kk + 1][1]));
    a[kk][3] = pack2(gelu(acc[2 * kk + 1][2]), gelu(acc[2 * kk + 1][3]));
  }
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const float2 bb = *reinterpret_cast<const float2*>(Bs + 2 * kHid + 8 * j + 2 * t);
    out[j][0] = bb.x; out[j][1] = bb.y; out[j][2] = bb.x; out[j][3] = bb.y;
  }
#pragma unroll
  for (int kk = 0; kk < 8; ++kk)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const uint32_t* w = reinterpret_cast<const uint32_t*>(W3s + (8 * j + g) * kLd2 + 16 * kk + 2 * t);
      mma16816(out[j], a[kk], w[0], w[4]);
    }
}

__device__ __forceinline__ void layer1(const unsigned char* sm, int g, int t, const uint32_t (&a1)[7][4],
                                       float (&acc)[16][4]) {
  const uint16_t* W1s = reinterpret_cast<const uint16_t*>(sm + kPW1);
  const float* Bs = reinterpret_cast<const float*>(sm + kPB);
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const float2 bb = *reinterpret_cast<const float2*>(Bs + 8 * j + 2 * t);
    acc[j][0] = bb.x; acc[j][1] = bb.y; acc[j][2] = bb.x; acc[j][3] = bb.y;
  }
#pragma unroll
  for (int kk = 0; kk < 7; ++kk)
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const uint32_t* w = reinterpret_cast<const uint32_t*>(W1s + (8 * j + g) * kLd1 + 16 * kk + 2 * t);
      mma16816(acc[j], a1[kk], w[0], w[4]);
    }
}

// Start the bulk copy of the packed network into shared memory (thread 0) and return.
__device__ __forceinline__ void start_weights(unsigned char* sm, const unsigned char* net, uint64_t* bar) {
  if (threadIdx.x == 0) mbar_init(bar, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_expect_tx(bar, kPBytes);
    bulk_g2s(sm, net, kPBytes, bar);
  }
}

// ------------------------------------------------------------- inference
// Rows of 16 features-times-7 (FEAT: given features X [n][112] -> Y [n][16]) or the coarse
// correction (COARSE: gathered from the level vector d [ne][16] and neighbours nbr [ne][6],
// normalised, x = s N(X)). One warp per 16 rows, 4 warps per CTA.
enum { kModeFeat = 0, kModeCoarse = 1 };

template <int MODE, class R>
__global__ void __launch_bounds__(32 * kWarps) mlp_forward_kernel(const unsigned char* __restrict__ net, long long n,
                                                                  const float* __restrict__ X, float* __restrict__ Y,
                                                                  const R* __restrict__ d, const int* __restrict__ nbr,
                                                                  R* __restrict__ x, int accumulate, unsigned* status) {
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ uint64_t bar;
  start_weights(sm, net, &bar);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const long long ra = (long long)blockIdx.x * kRows + warp * 16 + g, rb = ra + 8;
  const bool va = ra < n, vb = rb < n;
  uint32_t a1[7][4];
  R sa = R(0), sb = R(0);  // output scales (COARSE)
  if constexpr (MODE == kModeFeat) {
#pragma unroll
    for (int kk = 0; kk < 7; ++kk) {
      float2 p0 = make_float2(0.f, 0.f), p1 = p0, p2 = p0, p3 = p0;
      if (va) {
        p0 = *reinterpret_cast<const float2*>(X + ra * kIn + 16 * kk + 2 * t);
        p2 = *reinterpret_cast<const float2*>(X + ra * kIn + 16 * kk + 8 + 2 * t);
      }
      if (vb) {
        p1 = *reinterpret_cast<const float2*>(X + rb * kIn + 16 * kk + 2 * t);
        p3 = *reinterpret_cast<const float2*>(X + rb * kIn + 16 * kk + 8 + 2 * t);
      }
      a1[kk][0] = pack2(p0.x, p0.y);
      a1[kk][1] = pack2(p1.x, p1.y);
      a1[kk][2] = pack2(p2.x, p2.y);
      a1[kk][3] = pack2(p3.x, p3.y);
    }
  } else {
    int ea[7], eb[7];
    ea[0] = va ? (int)ra : 0;
    eb[0] = vb ? (int)rb : 0;
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      ea[f + 1] = va ? nbr[ra * 6 + f] : 0;
      eb[f + 1] = vb ? nbr[rb * 6 + f] : 0;
    }
    // pass 1: squared norms of the 112 features of rows a and b (4 lanes per row)
    R qa = R(0), qb = R(0);
#pragma unroll
    for (int kk = 0; kk < 7; ++kk) {
      if (va && ea[kk] >= 0) {  // a missing neighbour (wall) contributes zero features
        const R* p = d + (size_t)ea[kk] * 16;
        const R u0 = p[2 * t], u1 = p[2 * t + 1], u2 = p[8 + 2 * t], u3 = p[9 + 2 * t];
        qa += u0 * u0 + u1 * u1 + u2 * u2 + u3 * u3;
      }
      if (vb && eb[kk] >= 0) {
        const R* p = d + (size_t)eb[kk] * 16;
        const R u0 = p[2 * t], u1 = p[2 * t + 1], u2 = p[8 + 2 * t], u3 = p[9 + 2 * t];
        qb += u0 * u0 + u1 * u1 + u2 * u2 + u3 * u3;
      }
    }
    qa += __shfl_xor_sync(0xffffffffu, qa, 1);
    qa += __shfl_xor_sync(0xffffffffu, qa, 2);
    qb += __shfl_xor_sync(0xffffffffu, qb, 1);
    qb += __shfl_xor_sync(0xffffffffu, qb, 2);
    sa = sqrt(qa);
    sb = sqrt(qb);
    const R ia = sa > R(0) ? R(1) / sa : R(0), ib = sb > R(0) ? R(1) / sb : R(0);
    // pass 2: normalised features -> BF16 A fragments (k-step kk = neighbour slot kk)
#pragma unroll
    for (int kk = 0; kk < 7; ++kk) {
      float f0 = 0.f, f1 = 0.f, f2 = 0.f, f3 = 0.f, h0 = 0.f, h1 = 0.f, h2 = 0.f, h3 = 0.f;
      if (va && ea[kk] >= 0) {
        const R* p = d + (size_t)ea[kk] * 16;
        f0 = (float)(p[2 * t] * ia); f1 = (float)(p[2 * t + 1] * ia);
        f2 = (float)(p[8 + 2 * t] * ia); f3 = (float)(p[9 + 2 * t] * ia);
      }
      if (vb && eb[kk] >= 0) {
        const R* p = d + (size_t)eb[kk] * 16;
        h0 = (float)(p[2 * t] * ib); h1 = (float)(p[2 * t + 1] * ib);
        h2 = (float)(p[8 + 2 * t] * ib); h3 = (float)(p[9 + 2 * t] * ib);
      }
      a1[kk][0] = pack2(f0, f1);
      a1[kk][1] = pack2(h0, h1);
      a1[kk][2] = pack2(f2, f3);
      a1[kk][3] = pack2(h2, h3);
    }
  }
  if (!mbar_wait(&bar, 0)) {
    // give up: report, and let the weights' copy land (a second bounded wait) before leaving,
    // so that it cannot write this CTA's shared memory after the CTA exits
    if (lane == 0) {
      atomicOr(status, DG_STATUS_WAIT);
      mbar_wait(&bar, 0);
    }
    __syncwarp();
    return;
  }
  float acc[16][4], out[2][4];
  layer1(sm, g, t, a1, acc);
  mlp_tail(sm, g, t, acc, out);
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int c = 8 * j + 2 * t;
    if constexpr (MODE == kModeFeat) {
      if (va) *reinterpret_cast<float2*>(Y + ra * kOut + c) = make_float2(out[j][0], out[j][1]);
      if (vb) *reinterpret_cast<float2*>(Y + rb * kOut + c) = make_float2(out[j][2], out[j][3]);
    } else {
      R* pa = x + ra * kOut + c;
      R* pb = x + rb * kOut + c;
      if (va) { pa[0] = (accumulate ? pa[0] : R(0)) + sa * (R)out[j][0]; pa[1] = (accumulate ? pa[1] : R(0)) + sa * (R)out[j][1]; }
      if (vb) { pb[0] = (accumulate ? pb[0] : R(0)) + sb * (R)out[j][2]; pb[1] = (accumulate ? pb[1] : R(0)) + sb * (R)out[j][3]; }
    }
  }
}

// -------------------------------------------------------------- training
// One CTA: forward and backward of 64 samples, then its share of the weight gradient
// dW = dZ^T H (a contraction over its samples) on the tensor cores, written as one
// partial row; grad_reduce_kernel sums the rows in a fixed order.
constexpr int kLdT = 72;  // feature-major tiles [feature][64 samples + 8] (bank-conflict-free fragments)
constexpr int sXT = kPBytes;
constexpr int sH1T = sXT + kIn * kLdT * 2;
constexpr int sH2T = sH1T + kHid * kLdT * 2;
constexpr int sDZ1T = sH2T + kHid * kLdT * 2;
constexpr int sDZ2T = sDZ1T + kHid * kLdT * 2;
constexpr int sDYT = sDZ2T + kHid * kLdT * 2;
constexpr int sG = sDYT + kOut * kLdT * 2;           // gelu' of layers 1, 2: [warp][2][64 regs][32 lanes] bf16
constexpr int sBsum = sG + kWarps * 2 * 64 * 32 * 2;  // [warp][128 + 128 + 16] column sums of dZ1, dZ2, dY
constexpr int sLoss = sBsum + kWarps * (2 * kHid + kOut) * 4;
constexpr int kTrainSmem = sLoss + 16 * 4;
constexpr int kPartLd = kNP + 16;  // partial row: gradient, then the loss sum
static_assert(kTrainSmem <= 227 * 1024, "training tile exceeds shared memory");
static_assert(sXT % 16 == 0 && sG % 16 == 0 && sBsum % 16 == 0, "alignment");

__device__ __forceinline__ long long sample_row(long long seed, long long step, long long s, long long npairs) {
  if (seed < 0) return s;
  unsigned long long z = (unsigned long long)seed * 0x9E3779B97F4A7C15ull +
                         (unsigned long long)step * 0xD1B54A32D192ED03ull + (unsigned long long)s * 0x8CB92BA72F3D8DD7ull;
  z ^= z >> 30;
  z *= 0xBF58476D1CE4E5B9ull;
  z ^= z >> 27;
  z *= 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (long long)(z % (unsigned long long)npairs);
}

// store a feature-major BF16 value T[col][s]
__device__ __forceinline__ void stT(unsigned char* sm, int off, int col, int s, uint16_t v) {
  reinterpret_cast<uint16_t*>(sm + off)[col * kLdT + s] = v;
}

// column sums over the 16 rows of a warp of C-fragment values v[j][4] (cols 8j+2t, +1)
template <int NB>
__device__ __forceinline__ void warp_colsum(const float (&v)[NB][4], float* dst, int lane) {
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    float c0 = v[j][0] + v[j][2], c1 = v[j][1] + v[j][3];
#pragma unroll
    for (int o = 4; o < 32; o <<= 1) {
      c0 += __shfl_xor_sync(0xffffffffu, c0, o);
      c1 += __shfl_xor_sync(0xffffffffu, c1, o);
    }
    if (lane < 4) {
      dst[8 * j + 2 * lane] = c0;
      dst[8 * j + 2 * lane + 1] = c1;
    }
  }
}

// one 16-row block of dW = A B^T over the CTA's 64 samples: A rows from the feature-major
// tile at offA (rows m0..m0+15), B rows nb = 0..NB-1 of the tile at offB; writes NB tiles.
template <int NB>
__device__ __forceinline__ void wgrad_block(const unsigned char* sm, int offA, int m0, int offB, int nb0, int g, int t,
                                            float* dst, int ldd) {
  const uint16_t* A = reinterpret_cast<const uint16_t*>(sm + offA);
  const uint16_t* B = reinterpret_cast<const uint16_t*>(sm + offB);
  float acc[NB][4];
#pragma unroll
  for (int j = 0; j < NB; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    uint32_t a[4];
    a[0] = *reinterpret_cast<const uint32_t*>(A + (m0 + g) * kLdT + 16 * kk + 2 * t);
    a[1] = *reinterpret_cast<const uint32_t*>(A + (m0 + g + 8) * kLdT + 16 * kk + 2 * t);
    a[2] = *reinterpret_cast<const uint32_t*>(A + (m0 + g) * kLdT + 16 * kk + 8 + 2 * t);
    a[3] = *reinterpret_cast<const uint32_t*>(A + (m0 + g + 8) * kLdT + 16 * kk + 8 + 2 * t);
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      const uint16_t* b = B + (8 * (nb0 + j) + g) * kLdT + 16 * kk + 2 * t;
      mma16816(acc[j], a, *reinterpret_cast<const uint32_t*>(b), *reinterpret_cast<const uint32_t*>(b + 8));
    }
  }
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    const int c = 8 * (nb0 + j) + 2 * t;
    *reinterpret_cast<float2*>(dst + (m0 + g) * ldd + c) = make_float2(acc[j][0], acc[j][1]);
    *reinterpret_cast<float2*>(dst + (m0 + g + 8) * ldd + c) = make_float2(acc[j][2], acc[j][3]);
  }
}

__global__ void __launch_bounds__(32 * kWarps) mlp_grad_kernel(const unsigned char* __restrict__ net,
                                                               const float* __restrict__ X, const float* __restrict__ T,
                                                               long long npairs, int batch, long long seed,
                                                               long long step, float* __restrict__ part,
                                                               unsigned* status) {
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ uint64_t bar;
  __shared__ int ok_all;
  start_weights(sm, net, &bar);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int la = warp * 16 + g, lb = la + 8;  // local sample slots
  const long long sa = (long long)blockIdx.x * kRows + la, sb = sa + 8;
  const bool va = sa < batch, vb = sb < batch;
  const long long ra = va ? sample_row(seed, step, sa, npairs) : 0, rb = vb ? sample_row(seed, step, sb, npairs) : 0;
  // inputs: A fragments and the feature-major copy XT
  uint32_t a1[7][4];
#pragma unroll
  for (int kk = 0; kk < 7; ++kk) {
    float2 p0 = make_float2(0.f, 0.f), p1 = p0, p2 = p0, p3 = p0;
    if (va) {
      p0 = *reinterpret_cast<const float2*>(X + ra * kIn + 16 * kk + 2 * t);
      p2 = *reinterpret_cast<const float2*>(X + ra * kIn + 16 * kk + 8 + 2 * t);
    }
    if (vb) {
      p1 = *reinterpret_cast<const float2*>(X + rb * kIn + 16 * kk + 2 * t);
      p3 = *reinterpret_cast<const float2*>(X + rb * kIn + 16 * kk + 8 + 2 * t);
    }
    a1[kk][0] = pack2(p0.x, p0.y);
    a1[kk][1] = pack2(p1.x, p1.y);
    a1[kk][2] = pack2(p2.x, p2.y);
    a1[kk][3] = pack2(p3.x, p3.y);
  }
  if (threadIdx.x == 0) ok_all = 1;
  const bool ok = mbar_wait(&bar, 0);
  __syncthreads();
  if (!ok) ok_all = 0;
  __syncthreads();
  if (!ok_all) {
    if (threadIdx.x == 0) {  // report; the copy in flight lands before the CTA leaves
      atomicOr(status, DG_STATUS_WAIT);
      mbar_wait(&bar, 0);
    }
    __syncthreads();
    return;
  }
  // XT (after the weights landed: the bulk copy only writes the network region)
#pragma unroll
  for (int kk = 0; kk < 7; ++kk) {
    const int c = 16 * kk + 2 * t;
    stT(sm, sXT, c, la, a1[kk][0] & 0xffff); stT(sm, sXT, c + 1, la, a1[kk][0] >> 16);
    stT(sm, sXT, c, lb, a1[kk][1] & 0xffff); stT(sm, sXT, c + 1, lb, a1[kk][1] >> 16);
    stT(sm, sXT, c + 8, la, a1[kk][2] & 0xffff); stT(sm, sXT, c + 9, la, a1[kk][2] >> 16);
    stT(sm, sXT, c + 8, lb, a1[kk][3] & 0xffff); stT(sm, sXT, c + 9, lb, a1[kk][3] >> 16);
  }
  uint16_t* Gs = reinterpret_cast<uint16_t*>(sm + sG) + warp * 2 * 64 * 32;
  const uint16_t* W2s = reinterpret_cast<const uint16_t*>(sm + kPW2);
  const uint16_t* W3s = reinterpret_cast<const uint16_t*>(sm + kPW3);
  const uint16_t* W1s = reinterpret_cast<const uint16_t*>(sm + kPW1);
  const float* Bs = reinterpret_cast<const float*>(sm + kPB);
  float* bsum = reinterpret_cast<float*>(sm + sBsum) + warp * (2 * kHid + kOut);
  float acc[16][4];
  uint32_t a[8][4];
  // ---- forward: layer 1
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const float2 bb = *reinterpret_cast<const float2*>(Bs + 8 * j + 2 * t);
    acc[j][0] = bb.x; acc[j][1] = bb.y; acc[j][2] = bb.x; acc[j][3] = bb.y;
  }
#pragma unroll
  for (int kk = 0; kk < 7; ++kk)
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const uint32_t* w = reinterpret_cast<const uint32_t*>(W1s + (8 * j + g) * kLd1 + 16 * kk + 2 * t);
      mma16816(acc[j], a1[kk], w[0], w[4]);
    }
  // H1 = gelu(Z1) (A fragments and H1T), G1 = gelu'(Z1)
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const int c = 8 * j + 2 * t;
#pragma unroll
    for (int q = 0; q < 4; ++q) Gs[(0 * 64 + 4 * j + q) * 32 + lane] = bf16_bits(gelu_d(acc[j][q]));
    const uint32_t lo = pack2(gelu(acc[j][0]), gelu(acc[j][1])), hi = pack2(gelu(acc[j][2]), gelu(acc[j][3]));
    a[j >> 1][(j & 1) * 2 + 0] = lo;
    a[j >> 1][(j & 1) * 2 + 1] = hi;
    stT(sm, sH1T, c, la, lo & 0xffff); stT(sm, sH1T, c + 1, la, lo >> 16);
    stT(sm, sH1T, c, lb, hi & 0xffff); stT(sm, sH1T, c + 1, lb, hi >> 16);
  }
  // ---- layer 2
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const float2 bb = *reinterpret_cast<const float2*>(Bs + kHid + 8 * j + 2 * t);
    acc[j][0] = bb.x; acc[j][1] = bb.y; acc[j][2] = bb.x; acc[j][3] = bb.y;
  }
#pragma unroll
  for (int kk = 0; kk < 8; ++kk)
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const uint32_t* w = reinterpret_cast<const uint32_t*>(W2s + (8 * j + g) * kLd2 + 16 * kk + 2 * t);
      mma16816(acc[j], a[kk], w[0], w[4]);
    }
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const int c = 8 * j + 2 * t;
#pragma unroll
    for (int q = 0; q < 4; ++q) Gs[(1 * 64 + 4 * j + q) * 32 + lane] = bf16_bits(gelu_d(acc[j][q]));
    const uint32_t lo = pack2(gelu(acc[j][0]), gelu(acc[j][1])), hi = pack2(gelu(acc[j][2]), gelu(acc[j][3]));
    a[j >> 1][(j & 1) * 2 + 0] = lo;
    a[j >> 1][(j & 1) * 2 + 1] = hi;
    stT(sm, sH2T, c, la, lo & 0xffff); stT(sm, sH2T, c + 1, la, lo >> 16);
    stT(sm, sH2T, c, lb, hi & 0xffff); stT(sm, sH2T, c + 1, lb, hi >> 16);
  }
  // ---- layer 3 and the loss
  float out[2][4];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const float2 bb = *reinterpret_cast<const float2*>(Bs + 2 * kHid + 8 * j + 2 * t);
    out[j][0] = bb.x; out[j][1] = bb.y; out[j][2] = bb.x; out[j][3] = bb.y;
  }
#pragma unroll
  for (int kk = 0; kk < 8; ++kk)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const uint32_t* w = reinterpret_cast<const uint32_t*>(W3s + (8 * j + g) * kLd2 + 16 * kk + 2 * t);
      mma16816(out[j], a[kk], w[0], w[4]);
    }
  const float sc = 2.0f / (float)batch;
  float lsum = 0.f;
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int c = 8 * j + 2 * t;
    float2 ta = make_float2(0.f, 0.f), tb = ta;
    if (va) ta = *reinterpret_cast<const float2*>(T + ra * kOut + c);
    if (vb) tb = *reinterpret_cast<const float2*>(T + rb * kOut + c);
    const float r0 = va ? out[j][0] - ta.x : 0.f, r1 = va ? out[j][1] - ta.y : 0.f;
    const float r2 = vb ? out[j][2] - tb.x : 0.f, r3 = vb ? out[j][3] - tb.y : 0.f;
    lsum += r0 * r0 + r1 * r1 + r2 * r2 + r3 * r3;
    out[j][0] = sc * r0; out[j][1] = sc * r1; out[j][2] = sc * r2; out[j][3] = sc * r3;  // dY
    stT(sm, sDYT, c, la, bf16_bits(out[j][0])); stT(sm, sDYT, c + 1, la, bf16_bits(out[j][1]));
    stT(sm, sDYT, c, lb, bf16_bits(out[j][2])); stT(sm, sDYT, c + 1, lb, bf16_bits(out[j][3]));
  }
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  if (lane == 0) reinterpret_cast<float*>(sm + sLoss)[warp] = lsum;
  warp_colsum<2>(out, bsum + 2 * kHid, lane);
  // ---- dH2 = dY W3 (one k-step over the 16 outputs), dZ2 = dH2 . G2
  {
    uint32_t ay[4] = {pack2(out[0][0], out[0][1]), pack2(out[0][2], out[0][3]), pack2(out[1][0], out[1][1]),
                      pack2(out[1][2], out[1][3])};
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
      const int col = 8 * j + g;
      const uint32_t b0 = (uint32_t)W3s[(2 * t) * kLd2 + col] | ((uint32_t)W3s[(2 * t + 1) * kLd2 + col] << 16);
      const uint32_t b1 =
          (uint32_t)W3s[(2 * t + 8) * kLd2 + col] | ((uint32_t)W3s[(2 * t + 9) * kLd2 + col] << 16);
      mma16816(acc[j], ay, b0, b1);
    }
  }
#pragma unroll
  for (int j = 0; j < 16; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[j][q] *= bf16_to_f(Gs[(1 * 64 + 4 * j + q) * 32 + lane]);
  warp_colsum<16>(acc, bsum + kHid, lane);
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const int c = 8 * j + 2 * t;
    const uint32_t lo = pack2(acc[j][0], acc[j][1]), hi = pack2(acc[j][2], acc[j][3]);
    a[j >> 1][(j & 1) * 2 + 0] = lo;
    a[j >> 1][(j & 1) * 2 + 1] = hi;
    stT(sm, sDZ2T, c, la, lo & 0xffff); stT(sm, sDZ2T, c + 1, la, lo >> 16);
    stT(sm, sDZ2T, c, lb, hi & 0xffff); stT(sm, sDZ2T, c + 1, lb, hi >> 16);
  }
  // ---- dH1 = dZ2 W2 (B fragments read down the columns of W2), dZ1 = dH1 . G1
#pragma unroll
  for (int j = 0; j < 16; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
#pragma unroll
  for (int kk = 0; kk < 8; ++kk)
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int col = 8 * j + g, k0 = 16 * kk + 2 * t;
      const uint32_t b0 = (uint32_t)W2s[k0 * kLd2 + col] | ((uint32_t)W2s[(k0 + 1) * kLd2 + col] << 16);
      const uint32_t b1 = (uint32_t)W2s[(k0 + 8) * kLd2 + col] | ((uint32_t)W2s[(k0 + 9) * kLd2 + col] << 16);
      mma16816(acc[j], a[kk], b0, b1);
    }
#pragma unroll
  for (int j = 0; j < 16; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[j][q] *= bf16_to_f(Gs[(0 * 64 + 4 * j + q) * 32 + lane]);
  warp_colsum<16>(acc, bsum, lane);
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const int c = 8 * j + 2 * t;
    stT(sm, sDZ1T, c, la, bf16_bits(acc[j][0])); stT(sm, sDZ1T, c + 1, la, bf16_bits(acc[j][1]));
    stT(sm, sDZ1T, c, lb, bf16_bits(acc[j][2])); stT(sm, sDZ1T, c + 1, lb, bf16_bits(acc[j][3]));
  }
  __syncthreads();
  // ---- weight gradients of this CTA: dW1 = dZ1^T X, dW2 = dZ2^T H1, dW3 = dY^T H2
  float* P = part + (size_t)blockIdx.x * kPartLd;
#pragma unroll 1
  for (int mb = 2 * warp; mb < 2 * warp + 2; ++mb) {
    wgrad_block<14>(sm, sDZ1T, 16 * mb, sXT, 0, g, t, P + oW1, kIn);
    wgrad_block<16>(sm, sDZ2T, 16 * mb, sH1T, 0, g, t, P + oW2, kHid);
  }
  wgrad_block<4>(sm, sDYT, 0, sH2T, 4 * warp, g, t, P + oW3, kHid);
  // bias gradients and the loss: sums over the warps in a fixed order
  const float* bs = reinterpret_cast<const float*>(sm + sBsum);
  for (int i = threadIdx.x; i < 2 * kHid + kOut; i += blockDim.x) {
    float s = 0.f;
    for (int w = 0; w < kWarps; ++w) s += bs[w * (2 * kHid + kOut) + i];
    const int dst = i < kHid ? ob1 + i : i < 2 * kHid ? ob2 + (i - kHid) : ob3 + (i - 2 * kHid);
    P[dst] = s;
  }
  if (threadIdx.x == 0) {
    const float* ls = reinterpret_cast<const float*>(sm + sLoss);
    float s = 0.f;
    for (int w = 0; w < kWarps; ++w) s += ls[w];
    P[kNP] = s;
  }
}

// grad[p] = sum_c part[c][p]; loss = sum_c part[c][kNP] / batch (fixed order)
__global__ void grad_reduce_kernel(const float* __restrict__ part, int nparts, int batch, float* __restrict__ grad,
                                   float* __restrict__ loss) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > kNP) return;
  float s = 0.f;
  for (int c = 0; c < nparts; ++c) s += part[(size_t)c * kPartLd + p];
  if (p < kNP) grad[p] = s;
  else if (loss) *loss = s / (float)batch;
}

__global__ void adam_kernel(float* __restrict__ theta, const float* __restrict__ grad, float* __restrict__ m,
                            float* __restrict__ v, float lr_t, float b1, float b2, float eps, float bc2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kNP) return;
  const float gr = grad[p];
  const float mm = b1 * m[p] + (1.0f - b1) * gr;
  const float vv = b2 * v[p] + (1.0f - b2) * gr * gr;
  m[p] = mm;
  v[p] = vv;
  theta[p] -= lr_t * mm / (sqrtf(vv / bc2) + eps);
}

// Training pairs of the coarsest level: one thread per element.
__global__ void pairs_kernel(int ne, const double* __restrict__ d, const double* __restrict__ x,
                             const double* __restrict__ q, const int* __restrict__ nbr, float* __restrict__ X,
                             float* __restrict__ T, float* __restrict__ s) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  int src[7];
  src[0] = e;
  for (int f = 0; f < 6; ++f) src[f + 1] = nbr[(size_t)e * 6 + f];
  double ss = 0.0;
  for (int k = 0; k < 7; ++k)
    for (int i = 0; i < 16; ++i) {
      const double u = src[k] >= 0 ? d[(size_t)src[k] * 16 + i] : 0.0;  // zero across a wall
      ss += u * u;
    }
  const double nrm = sqrt(ss);
  const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
  for (int k = 0; k < 7; ++k)
    for (int i = 0; i < 16; ++i)
      X[(size_t)e * kIn + 16 * k + i] = src[k] >= 0 ? (float)(d[(size_t)src[k] * 16 + i] * inv) : 0.0f;
  for (int i = 0; i < 16; ++i)
    T[(size_t)e * kOut + i] = (float)(x[(size_t)e * 16 + i] * inv + (q ? nrm * q[(size_t)e * 16 + i] : 0.0));
  s[e] = (float)nrm;
}

// opt-in, once per kernel, to more than 48 KB of dynamic shared memory
std::mutex g_optin_mu;
std::vector<const void*> g_optin_done;
template <class K>
int smem_opt_in(K kernel, int bytes) {
  std::lock_guard<std::mutex> lock(g_optin_mu);
  const void* key = reinterpret_cast<const void*>(kernel);
  for (const void* k : g_optin_done)
    if (k == key) return 0;
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess) return 1;
  g_optin_done.push_back(key);
  return 0;
}

long long grad_parts(long long batch) { return (batch + kRows - 1) / kRows; }

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// status word of the handle-less calls
__device__ unsigned g_mlp_status;

unsigned* mlp_status_ptr() {
  static std::mutex mu;
  static unsigned* p = nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!p) {
    void* a = nullptr;
    if (cudaGetSymbolAddress(&a, g_mlp_status) != cudaSuccess) return nullptr;
    p = static_cast<unsigned*>(a);
  }
  return p;
}

}  // namespace

int net_bytes() { return kPBytes; }

template <class R>
int learned_coarse(Handle* h, const R* g, R* x, bool accumulate, cudaStream_t st) {
  if (!h->net_ready) return fail(h, DG_ERR_STATE, "no coarse network set (dg_set_coarse_network)");
  const Level& C = h->lev[h->nlev - 1];
  if (C.k != 1) return fail(h, DG_ERR_ARG, "the learned coarse correction needs k = 1 on the coarsest level");
  if (smem_opt_in(mlp_forward_kernel<kModeCoarse, R>, kPBytes))
    return fail(h, DG_ERR_CUDA, "cannot opt in to the shared memory of the network kernel");
  const int grid = (int)((h->ne + kRows - 1) / kRows);
  mlp_forward_kernel<kModeCoarse, R><<<grid, 32 * kWarps, kPBytes, st>>>(h->net, h->ne, nullptr, nullptr, g, h->nbr,
                                                                         x, accumulate ? 1 : 0, h->status);
  DG_LAUNCH_CHECK(h);
  return DG_OK;
}
template int learned_coarse<double>(Handle*, const double*, double*, bool, cudaStream_t);
template int learned_coarse<float>(Handle*, const float*, float*, bool, cudaStream_t);

}  // namespace dg

using namespace dg;

#define MLP_CUDA(call)                                                                      \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) return fail(nullptr, DG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

extern "C" {

long long dg_mlp_workspace_bytes(long long rows) {
  if (rows < 1) rows = 1;
  return (long long)kPBytes + grad_parts(rows) * (long long)kPartLd * 4;
}

int dg_mlp_forward(const float* theta, const float* X, long long n, float* Y, void* ws, void* stream) {
  if (!theta || !X || !Y || !ws || n < 0) return fail(nullptr, DG_ERR_ARG, "dg_mlp_forward: bad argument");
  if (!aligned16(ws) || !aligned16(X) || !aligned16(Y)) return fail(nullptr, DG_ERR_ARG, "dg_mlp_forward: unaligned");
  if (n == 0) return DG_OK;
  cudaStream_t st = as_stream(stream);
  unsigned* status = mlp_status_ptr();
  if (!status) return fail(nullptr, DG_ERR_CUDA, "cannot look up the status word");
  unsigned char* net = static_cast<unsigned char*>(ws);
  pack_kernel<<<(kPackSlots + 255) / 256, 256, 0, st>>>(theta, net);
  MLP_CUDA(cudaGetLastError());
  if (smem_opt_in(mlp_forward_kernel<kModeFeat, float>, kPBytes))
    return fail(nullptr, DG_ERR_CUDA, "cannot opt in to the shared memory of the network kernel");
  const long long grid = (n + kRows - 1) / kRows;
  if (grid > 0x7fffffffLL) return fail(nullptr, DG_ERR_ARG, "dg_mlp_forward: too many rows");
  mlp_forward_kernel<kModeFeat, float><<<(unsigned)grid, 32 * kWarps, kPBytes, st>>>(net, n, X, Y, nullptr, nullptr,
                                                                                  nullptr, 0, status);
  MLP_CUDA(cudaGetLastError());
  return DG_OK;
}

int dg_mlp_grad(const float* theta, const float* X, const float* T, long long npairs, int batch, long long seed,
                long long step, float* grad, float* loss, void* ws, void* stream) {
  if (!theta || !X || !T || !grad || !ws || batch < 1 || npairs < 1)
    return fail(nullptr, DG_ERR_ARG, "dg_mlp_grad: bad argument");
  if (seed < 0 && batch > npairs) return fail(nullptr, DG_ERR_ARG, "dg_mlp_grad: batch > npairs without sampling");
  if (!aligned16(ws) || !aligned16(X) || !aligned16(T)) return fail(nullptr, DG_ERR_ARG, "dg_mlp_grad: unaligned");
  cudaStream_t st = as_stream(stream);
  unsigned* status = mlp_status_ptr();
  if (!status) return fail(nullptr, DG_ERR_CUDA, "cannot look up the status word");
  unsigned char* net = static_cast<unsigned char*>(ws);
  float* part = reinterpret_cast<float*>(net + kPBytes);
  pack_kernel<<<(kPackSlots + 255) / 256, 256, 0, st>>>(theta, net);
  MLP_CUDA(cudaGetLastError());
  if (smem_opt_in(mlp_grad_kernel, kTrainSmem))
    return fail(nullptr, DG_ERR_CUDA, "cannot opt in to the shared memory of the training kernel");
  const int nparts = (int)grad_parts(batch);
  mlp_grad_kernel<<<nparts, 32 * kWarps, kTrainSmem, st>>>(net, X, T, npairs, batch, seed, step, part, status);
  MLP_CUDA(cudaGetLastError());
  grad_reduce_kernel<<<(kNP + 1 + 255) / 256, 256, 0, st>>>(part, nparts, batch, grad, loss);
  MLP_CUDA(cudaGetLastError());
  return DG_OK;
}

int dg_mlp_adam(float* theta, const float* grad, float* m, float* v, long long t, double lr, double beta1, double beta2,
                double eps, void* stream) {
  if (!theta || !grad || !m || !v || t < 1 || !(lr > 0.0) || !(beta1 >= 0.0 && beta1 < 1.0) ||
      !(beta2 >= 0.0 && beta2 < 1.0) || !(eps > 0.0))
    return fail(nullptr, DG_ERR_ARG, "dg_mlp_adam: bad argument");
  const double bc1 = 1.0 - std::pow(beta1, (double)t), bc2 = 1.0 - std::pow(beta2, (double)t);
  adam_kernel<<<(kNP + 255) / 256, 256, 0, as_stream(stream)>>>(theta, grad, m, v, (float)(lr / bc1), (float)beta1,
                                                                 (float)beta2, (float)eps, (float)bc2);
  MLP_CUDA(cudaGetLastError());
  return DG_OK;
}

int dg_set_coarse_network(dg_handle* hh, const float* theta, void* stream) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return DG_ERR_ARG;
  if (!theta) {
    h->net_ready = false;
    return DG_OK;
  }
  if (h->lev[h->nlev - 1].k != 1)
    return fail(h, DG_ERR_ARG, "the learned coarse correction needs k = 1 on the coarsest level");
  if (!h->net) DG_CUDA(h, cudaMalloc((void**)&h->net, kPBytes));
  pack_kernel<<<(kPackSlots + 255) / 256, 256, 0, as_stream(stream)>>>(theta, h->net);
  DG_LAUNCH_CHECK(h);
  h->net_ready = true;
  return DG_OK;
}

int dg_coarse_pairs(dg_handle* hh, const double* d, const double* x, const double* q, float* X, float* T, float* s,
                    void* stream) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return DG_ERR_ARG;
  if (!d || !x || !X || !T || !s) return fail(h, DG_ERR_ARG, "dg_coarse_pairs: null pointer");
  if (h->lev[h->nlev - 1].k != 1) return fail(h, DG_ERR_ARG, "dg_coarse_pairs needs k = 1 on the coarsest level");
  pairs_kernel<<<(h->ne + 127) / 128, 128, 0, as_stream(stream)>>>(h->ne, d, x, q, h->nbr, X, T, s);
  DG_LAUNCH_CHECK(h);
  return DG_OK;
}

int dg_record_coarse(dg_handle* hh, double* buf, int capacity) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return DG_ERR_ARG;
  if (buf && capacity < 1) return fail(h, DG_ERR_ARG, "dg_record_coarse: capacity must be >= 1");
  h->rec_buf = buf;
  h->rec_cap = buf ? capacity : 0;
  h->rec_count = 0;
  return DG_OK;
}

int dg_recorded(const dg_handle* hh, int* count) {
  const Handle* h = reinterpret_cast<const Handle*>(hh);
  if (!h || !count) return DG_ERR_ARG;
  *count = h->rec_count;
  return DG_OK;
}

}  // extern "C"
