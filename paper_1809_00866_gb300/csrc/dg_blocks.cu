// Element-block products of the preconditioner, streamed through shared memory.
//
// The block-Jacobi smoother (Sec. 2.3, element-wise block Jacobi) and the block-sparse coarse
// operators (Sec. 2.4.3) multiply every element by b x b blocks read once per application:
// b^2 values per element and block against 2 b^2 flops, so they are bound by HBM bandwidth.
// Measured on GB300 at 16^3 P4, the two ways of streaming differ per product: the block-Jacobi
// apply (one 78 KB inverse per element at P4) is fastest with the inverses brought into shared
// memory by bulk asynchronous copies (two stages per CTA); the block-sparse rows (seven 40 x 40
// blocks per element at P2) are fastest read straight from global memory by many small CTAs.
// Both use one thread per output row. The smoother uses explicit inverses D^-1, formed once per
// assembly from the LU factors.
#include <algorithm>

#include "dg_async.h"
#include "dg_internal.h"

namespace dg {

namespace {

// In place: LU factors (unit L below the diagonal, U above it with 1/U_kk on the diagonal,
// column-major, row permutation pi: row i of P D is row pi[i] of D) -> D^-1, column-major.
// D^-1 = U^-1 L^-1 P, and column c of P^T-free W = U^-1 L^-1 is column pinv[c] of D^-1's
// source, so thread j computes column j of W by substitution with uniform loop bounds (the
// leading zeros of e_j make the extra terms vanish) and the store permutes the columns.
template <class R>
__global__ void lu_to_inverse_kernel(int ne, int b, R* __restrict__ M, const int* __restrict__ perm) {
  extern __shared__ __align__(16) unsigned char sraw_[];
  R* LU = reinterpret_cast<R*>(sraw_);  // [b][b] column-major
  R* X = LU + (size_t)b * b;             // [b][b] row-major: X[i*b + j] = W[i][j]
  int* pinv = reinterpret_cast<int*>(X + (size_t)b * b);
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = blockIdx.x; e < ne; e += gridDim.x) {
    R* Me = M + (size_t)e * b * b;
    for (int t = tid; t < b * b; t += nt) LU[t] = Me[t];
    for (int i = tid; i < b; i += nt) pinv[perm[(size_t)e * b + i]] = i;
    __syncthreads();
    for (int j = tid; j < b; j += nt) {
      // forward: y = L^-1 e_j
      for (int i = 0; i < b; ++i) {
        R acc = i == j ? R(1) : R(0);
        for (int k = 0; k < i; ++k) acc = fma(-LU[(size_t)k * b + i], X[(size_t)k * b + j], acc);
        X[(size_t)i * b + j] = acc;
      }
      // backward: x = U^-1 y (the diagonal holds 1/U_ii)
      for (int i = b - 1; i >= 0; --i) {
        R acc = X[(size_t)i * b + j];
        for (int k = i + 1; k < b; ++k) acc = fma(-LU[(size_t)k * b + i], X[(size_t)k * b + j], acc);
        X[(size_t)i * b + j] = acc * LU[(size_t)i * b + i];
      }
    }
    __syncthreads();
    // D^-1[:, c] = W[:, pinv[c]]
    for (int t = tid; t < b * b; t += nt) {
      const int c = t / b, i = t - c * b;
      Me[t] = X[(size_t)i * b + pinv[c]];
    }
    __syncthreads();
  }
}

// Block Jacobi with explicit inverses, x <- (x_zero ? 0 : x) + alpha D_e^-1 (g - Gx)_e (Gx may
// be null): stages of G consecutive elements, whose inverses (contiguous) arrive by one bulk
// asynchronous copy into one of two shared-memory buffers while the previous stage is
// multiplied; stages are dealt to the CTAs round-robin, so neighbouring CTAs stream
// neighbouring memory. One thread per output row, four independent accumulators.
template <class R>
__global__ void __launch_bounds__(256) staged_jacobi_kernel(int ne, int b, int G, const R* __restrict__ A,
                                                            const R* __restrict__ g, const R* __restrict__ Gx,
                                                            R alpha, int x_zero, R* __restrict__ x,
                                                            unsigned* status) {
  extern __shared__ __align__(128) unsigned char sraw_[];
  __shared__ uint64_t bar[2];
  const size_t per = (size_t)b * b;  // values per element
  R* const buf0 = reinterpret_cast<R*>(sraw_);
  R* const buf1 = buf0 + (size_t)G * per;
  R* const rv = buf1 + (size_t)G * per;  // [G][b] residuals of the stage
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nstages = (ne + G - 1) / G;
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
  }
  __syncthreads();
  auto issue = [&](int stg, int slot) {
    const int e0 = stg * G;
    const unsigned bytes = (unsigned)(min(G, ne - e0) * per * sizeof(R));
    mbar_expect_tx(&bar[slot], bytes);
    bulk_g2s(slot ? buf1 : buf0, A + (size_t)e0 * per, bytes, &bar[slot]);
  };
  if (tid == 0 && (int)blockIdx.x < nstages) issue(blockIdx.x, 0);
  int k = 0;
  for (int stg = blockIdx.x; stg < nstages; stg += gridDim.x, ++k) {
    const int slot = k & 1;
    const int nxt = stg + gridDim.x;
    if (tid == 0 && nxt < nstages) issue(nxt, slot ^ 1);  // its buffer was released at the end of k - 1
    const int e0 = stg * G;
    const int cnt = min(G, ne - e0);
    for (int t = tid; t < cnt * b; t += nt) {
      const size_t o = (size_t)e0 * b + t;
      rv[t] = g[o] - (Gx ? Gx[o] : R(0));
    }
    const bool got = mbar_wait(&bar[slot], (unsigned)((k >> 1) & 1));
    if (!__syncthreads_and(got)) {
      // give up: report, let the copy issued for the next stage land (bounded), leave
      if (tid == 0) {
        atomicOr(status, (unsigned)DG_STATUS_WAIT);
        if (nxt < nstages) mbar_wait(&bar[slot ^ 1], (unsigned)(((k + 1) >> 1) & 1));
      }
      return;
    }
    const R* Ab = slot ? buf1 : buf0;
    for (int t = tid; t < cnt * b; t += nt) {
      const int el = t / b, i = t - el * b;
      const R* Ae = Ab + (size_t)el * per + i;
      const R* re = rv + (size_t)el * b;
      R a0 = R(0), a1 = R(0), a2 = R(0), a3 = R(0);
      int j = 0;
      for (; j + 3 < b; j += 4) {
        a0 = fma(Ae[(size_t)j * b], re[j], a0);
        a1 = fma(Ae[(size_t)(j + 1) * b], re[j + 1], a1);
        a2 = fma(Ae[(size_t)(j + 2) * b], re[j + 2], a2);
        a3 = fma(Ae[(size_t)(j + 3) * b], re[j + 3], a3);
      }
      for (; j < b; ++j) a0 = fma(Ae[(size_t)j * b], re[j], a0);
      R* xe = x + (size_t)e0 * b + t;
      *xe = (x_zero ? R(0) : *xe) + alpha * ((a0 + a1) + (a2 + a3));
    }
    __syncthreads();  // both buffers and rv free for the next stage
  }
}

// The same row products read straight from global memory: one thread per output row, `epc`
// elements per CTA (b rows each), the input vectors in shared memory. Loads of one warp cover
// 32 consecutive rows of a column (coalesced); eight independent accumulators keep eight loads
// in flight per thread, and small CTAs keep many elements in flight per SM.
template <class R, int NBLK>
__global__ void __launch_bounds__(256) direct_apply_kernel(int ne, int b, int epc, const R* __restrict__ A,
                                                           const int* __restrict__ nbr, const R* __restrict__ v,
                                                           const R* __restrict__ w, R alpha, R beta, int x_zero,
                                                           R* __restrict__ y) {
  extern __shared__ __align__(16) unsigned char sraw_[];
  R* rv = reinterpret_cast<R*>(sraw_);  // [epc][ncol]
  const int ncol = NBLK * b;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e0 = blockIdx.x * epc; e0 < ne; e0 += gridDim.x * epc) {
    const int cnt = min(epc, ne - e0);
    for (int t = tid; t < cnt * ncol; t += nt) {
      const int el = t / ncol, q = t - el * ncol;
      const int e = e0 + el;
      const int s = q / b, c = q - s * b;
      if (NBLK == 1) {
        rv[t] = v[(size_t)e * b + c] - (w ? w[(size_t)e * b + c] : R(0));
      } else {
        const int src = s == 0 ? e : nbr[(size_t)e * 6 + s - 1];
        rv[t] = v[(size_t)src * b + c];
      }
    }
    __syncthreads();
    if (tid < cnt * b) {
      const int el = tid / b, i = tid - el * b;
      const R* Ae = A + (size_t)(e0 + el) * ncol * b + i;
      const R* re = rv + (size_t)el * ncol;
      R a[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) a[u] = R(0);
      int q = 0;
      for (; q + 7 < ncol; q += 8) {
#pragma unroll
        for (int u = 0; u < 8; ++u) a[u] = fma(__ldg(Ae + (size_t)(q + u) * b), re[q + u], a[u]);
      }
      for (; q < ncol; ++q) a[0] = fma(__ldg(Ae + (size_t)q * b), re[q], a[0]);
      const R acc = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
      R* ye = y + (size_t)(e0 + el) * b + i;
      if (NBLK == 1) *ye = (x_zero ? R(0) : *ye) + alpha * acc;
      else *ye = alpha * acc + (beta == R(0) ? R(0) : beta * *ye);
    }
    __syncthreads();
  }
}

template <class R, int NBLK>
int launch_direct(Handle* h, int b, const R* A, const R* v, const R* w, R alpha, R beta, int x_zero, R* y,
                  cudaStream_t st) {
  if (b > 256) return -1;
  const int epc = std::max(1, 256 / b);
  const int threads = 32 * ((epc * b + 31) / 32);
  const size_t smem = sizeof(R) * (size_t)epc * NBLK * b;
  const int grid = (h->ne + epc - 1) / epc;
  direct_apply_kernel<R, NBLK><<<grid, threads, smem, st>>>(h->ne, b, epc, A, h->nbr, v, w, alpha, beta, x_zero, y);
  DG_LAUNCH_CHECK(h);
  return DG_OK;
}

constexpr size_t kStageTarget = 96 * 1024;  // bytes of inverses per stage (one buffer)
constexpr size_t kSmemLimit = 220 * 1024;    // dynamic shared memory a kernel may take

template <class R>
int launch_staged_jacobi(Handle* h, int b, const R* A, const R* g, const R* Gx, R alpha, int x_zero, R* x,
                         cudaStream_t st) {
  const size_t per = (size_t)b * b * sizeof(R);
  int G = (int)std::max<size_t>(1, kStageTarget / per);
  G = std::max(1, std::min(G, (h->ne + 2 * h->nsm - 1) / (2 * h->nsm)));  // >= 2 stages per SM when possible
  const size_t smem = 2 * (size_t)G * per + (size_t)G * b * sizeof(R);
  if (smem > kSmemLimit || per % 16 != 0) return -1;
  static bool opted = false;  // per template instance; one device per process
  if (!opted) {
    DG_CUDA(h, cudaFuncSetAttribute(staged_jacobi_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kSmemLimit));
    opted = true;
  }
  const int nstages = (h->ne + G - 1) / G;
  const int per_sm = (int)std::max<size_t>(1, std::min<size_t>(4, (227 * 1024) / (smem + 1024)));
  const int grid = std::min(nstages, h->nsm * per_sm);
  staged_jacobi_kernel<R><<<grid, 256, smem, st>>>(h->ne, b, G, A, g, Gx, alpha, x_zero, x, h->status);
  DG_LAUNCH_CHECK(h);
  return DG_OK;
}

}  // namespace

int staged_jacobi_f(Handle* h, int lvl, const float* g, const float* Gx, float omega, bool x_zero, float* x,
                    cudaStream_t st) {
  const Level& L = h->lev[lvl];
  return launch_staged_jacobi<float>(h, L.b, L.LUf, g, Gx, omega, x_zero ? 1 : 0, x, st);
}

template <class R>
int staged_bsr(Handle* h, int lvl, const R* B, R alpha, const R* x, R beta, R* y, cudaStream_t st) {
  return launch_direct<R, 7>(h, h->lev[lvl].b, B, x, nullptr, alpha, beta, 0, y, st);
}
template int staged_bsr<float>(Handle*, int, const float*, float, const float*, float, float*, cudaStream_t);
template int staged_bsr<double>(Handle*, int, const double*, double, const double*, double, double*, cudaStream_t);

int invert_levels_f32(Handle* h, cudaStream_t st) {
  for (int l = 0; l < h->nlev; ++l) {
    const Level& L = h->lev[l];
    const size_t smem = 2 * sizeof(float) * (size_t)L.b * L.b + sizeof(int) * L.b;
    if (smem > kSmemLimit) return fail(h, DG_ERR_ARG, "element block too large for the FP32 inverse");
    DG_CUDA(h, cudaFuncSetAttribute(lu_to_inverse_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kSmemLimit));
    const int threads = 32 * ((L.b + 31) / 32);
    const int per_sm = (int)std::max<size_t>(1, std::min<size_t>(8, (227 * 1024) / (smem + 1024)));
    const int grid = std::min(h->ne, h->nsm * per_sm);
    lu_to_inverse_kernel<float><<<grid, threads, smem, st>>>(h->ne, L.b, L.LUf, L.perm);
    DG_LAUNCH_CHECK(h);
  }
  return DG_OK;
}

}  // namespace dg
