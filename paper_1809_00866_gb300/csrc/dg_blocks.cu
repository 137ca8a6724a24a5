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
// assembly by Gauss-Jordan elimination in shared memory.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstring>
#include <type_traits>

#include "dg_async.h"
#include "dg_internal.h"

namespace dg {

namespace {

// value of a stored block entry in the arithmetic type R (blocks may be stored narrower)
template <class R> __device__ __forceinline__ R wide(float v) { return R(v); }
template <class R> __device__ __forceinline__ R wide(double v) { return R(v); }
template <class R> __device__ __forceinline__ R wide(__half v) { return R(__half2float(v)); }
template <class R> __device__ __forceinline__ R wide(__nv_bfloat16 v) { return R(__bfloat162float(v)); }

// two adjacent stored entries (rows i, i + 1 of one column; i even) as R
template <class R> __device__ __forceinline__ void wide2(const float* p, R& a, R& b) {
  const float2 v = *reinterpret_cast<const float2*>(p);
  a = R(v.x); b = R(v.y);
}
template <class R> __device__ __forceinline__ void wide2(const double* p, R& a, R& b) {
  const double2 v = *reinterpret_cast<const double2*>(p);
  a = R(v.x); b = R(v.y);
}
template <class R> __device__ __forceinline__ void wide2(const __half* p, R& a, R& b) {
  const float2 v = __half22float2(*reinterpret_cast<const __half2*>(p));
  a = R(v.x); b = R(v.y);
}
template <class R> __device__ __forceinline__ void wide2(const __nv_bfloat16* p, R& a, R& b) {
  const float2 v = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p));
  a = R(v.x); b = R(v.y);
}

// The leading dimension of a block in shared memory: a multiple of 4 (float4 rows) that is 4 mod 8,
// so that a column (stride LD) spreads over 8 banks instead of 2 (LD = b + 4 would be 0 mod 8 at
// b = 140).
__host__ __device__ constexpr int gj_ld(int b) { return (b + 4) % 8 == 4 ? b + 4 : b + 8; }

constexpr int kGjSlots = 5;  // panel rows per lane of the factoring warp: b <= 160

__device__ __forceinline__ float f4get(const float4& v, int q) {
  return q == 0 ? v.x : (q == 1 ? v.y : (q == 2 ? v.z : v.w));
}
__device__ __forceinline__ void f4set(float4& v, int q, float x) {
  if (q == 0) v.x = x; else if (q == 1) v.y = x; else if (q == 2) v.z = x; else v.w = x;
}

// Four elimination steps of the panel whose pivot columns are k0..k0+3, on those columns alone,
// held in the registers of one warp (lane l holds rows l + 32 m, m < kGjSlots, b <= 160): pivot
// search over the rows not yet pivoted by one warp-wide maximum (ties to the lower row), row
// interchange by shuffles, in-place elimination. The pivots go to piv[] and pq[].
__device__ __forceinline__ void gj_factor_panel(float4 (&pv)[kGjSlots], int b, int k0, int lane, int* piv,
                                                int (&pq)[4], unsigned* status) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int k = k0 + q;
    // one warp-wide integer maximum over keys |v| (bit pattern, the low 8 mantissa bits
    // replaced by 255 - row): the largest |v|, ties and values within 2^-15 relative to the
    // lower row; rows not eligible have key 0
    unsigned key = 0u;
#pragma unroll
    for (int m = 0; m < kGjSlots; ++m) {
      const int i = lane + 32 * m;
      if (i >= k && i < b) {
        const unsigned kv = (__float_as_uint(fabsf(f4get(pv[m], q))) & 0xffffff00u) | (unsigned)(255 - i);
        key = kv > key ? kv : key;
      }
    }
    key = __reduce_max_sync(0xffffffffu, key);
    const int p = 255 - (int)(key & 0xffu);
    pq[q] = p;
    if (lane == 0) {
      piv[k] = p;
      // a zero (or NaN, whose key exceeds every finite one) pivot
      const float best = __uint_as_float(key & 0xffffff00u);
      if (!(best > 0.0f) && status) atomicOr(status, (unsigned)DG_STATUS_NONFINITE);
    }
    // interchange rows k and p: each lane offers its slot's value, the owners exchange
    const int sk = k >> 5, sp = p >> 5, lk = k & 31, lp = p & 31;
    float4 rowp, rowk, o = pv[0];
#pragma unroll
    for (int m = 1; m < kGjSlots; ++m)
      if (m == sp) o = pv[m];
    rowp.x = __shfl_sync(0xffffffffu, o.x, lp);
    rowp.y = __shfl_sync(0xffffffffu, o.y, lp);
    rowp.z = __shfl_sync(0xffffffffu, o.z, lp);
    rowp.w = __shfl_sync(0xffffffffu, o.w, lp);
    o = pv[0];
#pragma unroll
    for (int m = 1; m < kGjSlots; ++m)
      if (m == sk) o = pv[m];
    rowk.x = __shfl_sync(0xffffffffu, o.x, lk);
    rowk.y = __shfl_sync(0xffffffffu, o.y, lk);
    rowk.z = __shfl_sync(0xffffffffu, o.z, lk);
    rowk.w = __shfl_sync(0xffffffffu, o.w, lk);
#pragma unroll
    for (int m = 0; m < kGjSlots; ++m)
      if (m == sp && lane == lp) pv[m] = rowk;
    // the pivot row (old row p) is now row k: scale it, eliminate column k elsewhere
    const float inv = 1.0f / f4get(rowp, q);
    float4 r4 = make_float4(rowp.x * inv, rowp.y * inv, rowp.z * inv, rowp.w * inv);
    f4set(r4, q, inv);
#pragma unroll
    for (int m = 0; m < kGjSlots; ++m) {
      const int i = lane + 32 * m;
      if (i == k) {
        pv[m] = r4;
      } else {
        float4 v = pv[m];
        const float c = f4get(v, q);
        v.x = fmaf(-c, r4.x, v.x);
        v.y = fmaf(-c, r4.y, v.y);
        v.z = fmaf(-c, r4.z, v.z);
        v.w = fmaf(-c, r4.w, v.w);
        f4set(v, q, -c * inv);
        pv[m] = v;
      }
    }
  }
}

// The panel's four interchanges on every other column group (one lane per group), then its pivot
// rows of those groups to the buffer Rp, zeroed in A: the panel's update then writes
// A[P,J] = X A[P,J] into them with the same multiply-adds as every other row.
__device__ __forceinline__ void gj_interchange(float* A, float* Rp, int LD, int NG, int g, const int (&pq)[4],
                                               int lane) {
  const int k0 = 4 * g;
  for (int j = lane; j < NG; j += 32) {
    if (j == g) continue;
    for (int q = 0; q < 4; ++q) {
      const int k = k0 + q, p = pq[q];
      if (p != k) {
        float4* ak = reinterpret_cast<float4*>(A + (size_t)k * LD + 4 * j);
        float4* ap = reinterpret_cast<float4*>(A + (size_t)p * LD + 4 * j);
        const float4 t = *ak;
        *ak = *ap;
        *ap = t;
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float4* ak = reinterpret_cast<float4*>(A + (size_t)(k0 + q) * LD + 4 * j);
      *reinterpret_cast<float4*>(Rp + q * LD + 4 * j) = *ak;
      *ak = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
}

// The same for panel g with one thread per column (t < 4 NG, column t of group t / 4), the
// panel's pivots read from piv[]: the interchanges of a column in panel order, then its pivot
// rows to Rp and zero.
__device__ __forceinline__ void gj_interchange_cols(float* A, float* Rp, int LD, int NG, int g, const int* piv,
                                                    int t) {
  const int j = t >> 2, k0 = 4 * g;
  if (t >= 4 * NG || j == g) return;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int k = k0 + q, p = piv[k];
    if (p != k) {
      const float a = A[(size_t)k * LD + t], b2 = A[(size_t)p * LD + t];
      A[(size_t)k * LD + t] = b2;
      A[(size_t)p * LD + t] = a;
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float* ak = A + (size_t)(k0 + q) * LD + t;
    Rp[q * LD + t] = *ak;
    *ak = 0.0f;
  }
}

// v + t0 r0 + t1 r1 + t2 r2 + t3 r3 on four columns
__device__ __forceinline__ float4 gj_rank4(float4 v, const float4& t, const float4& r0, const float4& r1,
                                           const float4& r2, const float4& r3) {
  v.x = fmaf(t.x, r0.x, v.x);
  v.y = fmaf(t.x, r0.y, v.y);
  v.z = fmaf(t.x, r0.z, v.z);
  v.w = fmaf(t.x, r0.w, v.w);
  v.x = fmaf(t.y, r1.x, v.x);
  v.y = fmaf(t.y, r1.y, v.y);
  v.z = fmaf(t.y, r1.z, v.z);
  v.w = fmaf(t.y, r1.w, v.w);
  v.x = fmaf(t.z, r2.x, v.x);
  v.y = fmaf(t.z, r2.y, v.y);
  v.z = fmaf(t.z, r2.z, v.z);
  v.w = fmaf(t.z, r2.w, v.w);
  v.x = fmaf(t.w, r3.x, v.x);
  v.y = fmaf(t.w, r3.y, v.y);
  v.z = fmaf(t.w, r3.z, v.z);
  v.w = fmaf(t.w, r3.w, v.w);
  return v;
}

// In place D -> D^-1 (column-major FP32 blocks, b a multiple of 4) by Gauss-Jordan elimination
// with partial (row) pivoting, one block per CTA in shared memory (row-major, leading dimension
// gj_ld(b) so that rows are float4-aligned), in panels of four pivots. The four pivot columns K
// of a panel are one float4 column group. With P the panel's pivot rows, O the other rows and
// X = A[P,K]^-1, four elimination steps map
//   A[:,K] -> T = [X; -A[O,K] X],   A[P,J] -> X A[P,J],   A[O,J] -> A[O,J] + T[O,:] A[P,J]
// on every other column J (the in-place form of the inverse keeps T in the pivot columns).
// Warp 0 factors the panels: it runs a panel's four steps on its columns alone, in registers,
// which leaves T in place; the pivots are those of the unblocked elimination, since a step reads
// only its own column and the pivot rows' entries in the panel. It then applies the panel's
// interchanges to the other column groups and copies their pivot rows to a buffer. The other
// warps apply the rank-4 update: a thread owns one column group and every RG-th row, so a
// pivot-row float4 it loads serves all its rows, and four steps read and write the matrix once.
// Look-ahead: while the other warps apply panel g's update, warp 0 applies it to group g + 1
// alone and factors panel g + 1, so the factoring chain is off the critical path. Two barriers
// per panel. b^3 multiply-adds per block; the row interchanges are undone on the columns at the
// end, as one column permutation applied while the inverse is written out. BT > 0 fixes b = BT
// and 512 threads at compile time (the P4 fine level, b = 140): the update's rows are then an
// unrolled loop with constant shared-memory offsets.
template <int BT>
__global__ void __launch_bounds__(512, 2) gj_inverse_kernel(int nblk, int b_arg, float* __restrict__ M,
                                                            unsigned* status) {
  extern __shared__ __align__(16) unsigned char sraw_[];
  const int b = BT > 0 ? BT : b_arg;
  const int LD = gj_ld(b);
  float* A = reinterpret_cast<float*>(sraw_);  // [b][LD]
  float* Rp = A + (size_t)b * LD;             // [4][LD] the panel's pivot rows before the update
  int* piv = reinterpret_cast<int*>(Rp + 4 * LD);
  int* colsrc = piv + b;  // [b]
  const int tid = threadIdx.x, nt = BT > 0 ? 512 : (int)blockDim.x, lane = tid & 31;
  const int NG = b / 4;  // float4 column groups = panels
  const int RG = (nt - 32) / NG < b ? (nt - 32) / NG : b;  // row groups of the update, on warps 1..
  const int tu = tid - 32;
  const bool upd = tid >= 32 && tu < NG * RG;
  const int jg = upd ? tu % NG : 0, ig = upd ? tu / NG : 0;
  for (int blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    float* Mb = M + (size_t)blk * b * b;
    for (int t = tid; t < b * b; t += nt) {
      const int c = t / b, r = t - c * b;
      A[r * LD + c] = Mb[t];
    }
    __syncthreads();
    int pq[4] = {0, 0, 0, 0};
    if (tid < 32) {  // panel 0
      float4 pv[kGjSlots];
#pragma unroll
      for (int m = 0; m < kGjSlots; ++m) {
        const int i = lane + 32 * m;
        pv[m] = i < b ? *reinterpret_cast<const float4*>(A + (size_t)i * LD) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      gj_factor_panel(pv, b, 0, lane, piv, pq, status);
#pragma unroll
      for (int m = 0; m < kGjSlots; ++m) {
        const int i = lane + 32 * m;
        if (i < b) *reinterpret_cast<float4*>(A + (size_t)i * LD) = pv[m];
      }
      gj_interchange(A, Rp, LD, NG, 0, pq, lane);
    }
    __syncthreads();
    for (int g = 0; g < NG; ++g) {
      const int k0 = 4 * g;
      const bool next = g + 1 < NG;
      if (tid < 32) {
        if (next) {  // panel g's update of group g + 1, then panel g + 1's steps
          const int j = g + 1;
          const float4 r0 = *reinterpret_cast<const float4*>(Rp + 4 * j);
          const float4 r1 = *reinterpret_cast<const float4*>(Rp + LD + 4 * j);
          const float4 r2 = *reinterpret_cast<const float4*>(Rp + 2 * LD + 4 * j);
          const float4 r3 = *reinterpret_cast<const float4*>(Rp + 3 * LD + 4 * j);
          float4 pv[kGjSlots];
#pragma unroll
          for (int m = 0; m < kGjSlots; ++m) {
            const int i = lane + 32 * m;
            if (i < b) {
              const float4 t = *reinterpret_cast<const float4*>(A + (size_t)i * LD + k0);
              const float4 v = *reinterpret_cast<const float4*>(A + (size_t)i * LD + 4 * j);
              pv[m] = gj_rank4(v, t, r0, r1, r2, r3);
            } else {
              pv[m] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
          }
          gj_factor_panel(pv, b, 4 * j, lane, piv, pq, status);
#pragma unroll
          for (int m = 0; m < kGjSlots; ++m) {
            const int i = lane + 32 * m;
            if (i < b) *reinterpret_cast<float4*>(A + (size_t)i * LD + 4 * j) = pv[m];
          }
        }
      } else if (upd && jg != g && jg != g + 1) {  // panel g's update of the other groups
        const float4 r0 = *reinterpret_cast<const float4*>(Rp + 4 * jg);
        const float4 r1 = *reinterpret_cast<const float4*>(Rp + LD + 4 * jg);
        const float4 r2 = *reinterpret_cast<const float4*>(Rp + 2 * LD + 4 * jg);
        const float4 r3 = *reinterpret_cast<const float4*>(Rp + 3 * LD + 4 * jg);
        const float* At = A + ig * LD + k0;
        float* Av = A + ig * LD + 4 * jg;
        if constexpr (BT > 0) {
          constexpr int RGc = (512 - 32) / (BT / 4) < BT ? (512 - 32) / (BT / 4) : BT;
          constexpr int LDc = gj_ld(BT);
#pragma unroll
          for (int u = 0; u < (BT + RGc - 1) / RGc; ++u) {
            if (BT % RGc == 0 || ig + u * RGc < BT) {
              const float4 t = *reinterpret_cast<const float4*>(At + u * RGc * LDc);
              float4* ai = reinterpret_cast<float4*>(Av + u * RGc * LDc);
              *ai = gj_rank4(*ai, t, r0, r1, r2, r3);
            }
          }
        } else {
          for (int i = ig; i < b; i += RG, At += RG * LD, Av += RG * LD) {
            const float4 t = *reinterpret_cast<const float4*>(At);
            float4* ai = reinterpret_cast<float4*>(Av);
            *ai = gj_rank4(*ai, t, r0, r1, r2, r3);
          }
        }
      }
      __syncthreads();
      if (next) {  // the next panel's interchanges on the other groups, one thread per column
        gj_interchange_cols(A, Rp, LD, NG, g + 1, piv, tid);
        __syncthreads();
      }
    }
    // the row interchanges, undone on the columns in reverse order, composed into one column
    // permutation (column c of the inverse is column colsrc[c] of A) and applied while writing out
    if (tid == 0) {
      for (int c = 0; c < b; ++c) colsrc[c] = c;
      for (int k = b - 1; k >= 0; --k) {
        const int p = piv[k];
        if (p != k) {
          const int t = colsrc[k];
          colsrc[k] = colsrc[p];
          colsrc[p] = t;
        }
      }
    }
    __syncthreads();
    for (int t = tid; t < b * b; t += nt) {
      const int c = t / b, r = t - c * b;
      Mb[t] = A[r * LD + colsrc[c]];
    }
    __syncthreads();
  }
}

// In place D -> D^-1 for small blocks (b <= 64; the coarse levels at P4, b = 40 and 16), one
// warp per block in its own shared memory, column-major like the blocks in HBM. Gauss-Jordan
// with partial pivoting by row choice instead of row interchanges: step k takes as pivot row p_k
// the not yet pivoted row with the largest |A[i][k]| (ties, and values within 2^-15 relative,
// to the lower row), and updates every entry in place (pivot row scaled, column k replaced by
// -A[i][k] / pivot). That is the in-place inversion of the row-permuted block P A, stored with
// row k at row p_k, so D^-1[r][c] = X[p_r][j] with p_j = c, read so while writing out. The
// b^2 entries of a step are dealt to the lanes in order (conflict-free), b^3 multiply-adds in
// all; eight blocks per CTA.
constexpr int kGjwWarps = 8;

template <int B>
__global__ void __launch_bounds__(32 * kGjwWarps) gj_inverse_warp_kernel(int nblk, float* __restrict__ M,
                                                                         unsigned* status) {
  static_assert(B >= 1 && B <= 64, "one warp per block of at most 64 rows");
  constexpr int W = B * B + 2 * B + 2 * B;  // floats per warp: block, column k, pivot row, order (ints)
  extern __shared__ __align__(16) unsigned char sraw_[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* A = reinterpret_cast<float*>(sraw_) + (size_t)warp * W;
  float* colk = A + B * B;
  float* prow = colk + B;
  int* ord = reinterpret_cast<int*>(prow + B);  // [B] p_k
  int* inv_ord = ord + B;                        // [B] j with p_j = c
  for (int blk = blockIdx.x * kGjwWarps + warp; blk < nblk; blk += gridDim.x * kGjwWarps) {
    float* Mb = M + (size_t)blk * B * B;
    for (int t = lane; t < B * B; t += 32) A[t] = Mb[t];
    __syncwarp();
    unsigned long long used = 0ull;
    for (int k = 0; k < B; ++k) {
      // one warp-wide integer maximum over keys |A[i][k]| (bit pattern, the low 8 mantissa bits
      // replaced by 255 - i) of the rows not yet pivoted: the largest, ties and values within
      // 2^-15 relative to the lower row; a NaN's key exceeds every finite one
      unsigned key = 0u;
      for (int i = lane; i < B; i += 32)
        if (!((used >> i) & 1ull)) {
          const unsigned kv = (__float_as_uint(fabsf(A[k * B + i])) & 0xffffff00u) | (unsigned)(255 - i);
          key = kv > key ? kv : key;
        }
      key = __reduce_max_sync(0xffffffffu, key);
      const int p = key ? 255 - (int)(key & 0xffu) : __ffsll((long long)~used) - 1;
      used |= 1ull << p;
      if (lane == 0) {
        ord[k] = p;
        inv_ord[p] = k;
        const float best = __uint_as_float(key & 0xffffff00u);
        if (!(best > 0.0f) && status) atomicOr(status, (unsigned)DG_STATUS_NONFINITE);
      }
      const float inv = 1.0f / A[k * B + p];
      for (int i = lane; i < B; i += 32) colk[i] = A[k * B + i];
      for (int j = lane; j < B; j += 32) prow[j] = j == k ? inv : A[j * B + p] * inv;
      __syncwarp();
      // entry e = j B + i (column-major): i the row, j the column
      int i = lane % B, j = lane / B;
#pragma unroll 4
      for (int e = lane; e < B * B; e += 32) {
        float nv;
        if (i == p) nv = prow[j];
        else if (j == k) nv = -colk[i] * inv;
        else nv = fmaf(-colk[i], prow[j], A[e]);
        A[e] = nv;
        i += 32;
        j += i / B;
        i %= B;
      }
      __syncwarp();
    }
    // D^-1[r][c] = X[p_r][inv_ord[c]]: column-major output entry t = c B + r
    for (int t = lane; t < B * B; t += 32) {
      const int c = t / B, r = t - c * B;
      Mb[t] = A[inv_ord[c] * B + ord[r]];
    }
    __syncwarp();
  }
}

// Block Jacobi with explicit inverses, x <- (x_zero ? 0 : x) + alpha D_e^-1 (g - Gx)_e (Gx may
// be null): stages of G consecutive elements, whose inverses (contiguous) arrive by one bulk
// asynchronous copy into one of two shared-memory buffers while the previous stage is
// multiplied; stages are dealt to the CTAs round-robin, so neighbouring CTAs stream
// neighbouring memory. A task is two adjacent rows (one paired load per column) over every
// CS-th column; when a stage has few rows, CS > 1 column slices meet in shared memory.
constexpr int kJacobiThreads = 512;
constexpr int kJacobiSlots = 2;  // stage buffers in the ring (3 and 4 measured no faster at 16^3 P4)

template <class R, class S>
__global__ void __launch_bounds__(kJacobiThreads) staged_jacobi_kernel(int ne, int b, int G, int ns,
                                                                       const S* __restrict__ A,
                                                                       const R* __restrict__ g,
                                                                       const R* __restrict__ Gx, R alpha, int x_zero,
                                                                       R* __restrict__ x, unsigned* status,
                                                                       unsigned wait_polls, int withhold_first) {
  extern __shared__ __align__(128) unsigned char sraw_[];
  __shared__ uint64_t bar[kJacobiSlots];
  __shared__ R red[2 * kJacobiThreads];  // partial sums of the column slices
  const size_t per = (size_t)b * b;  // values per element
  // ns (2..4) stage buffers in a ring, each: the G element blocks, then the stage's slices of g,
  // Gx and the old x, all brought by bulk copies on the buffer's barrier (no global load on the
  // critical path); ns - 1 stages are in flight while one is multiplied
  const size_t blk_bytes = (size_t)G * per * sizeof(S), vec = (size_t)G * b;
  const size_t slot_bytes = blk_bytes + 3 * vec * sizeof(R);
  auto blocks_of = [&](int slot) { return reinterpret_cast<S*>(sraw_ + slot * slot_bytes); };
  auto vecs_of = [&](int slot) { return reinterpret_cast<R*>(sraw_ + slot * slot_bytes + blk_bytes); };
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nstages = (ne + G - 1) / G;
  const int hb = b / 2;  // row pairs per element
  const int CS = max(1, min(8, nt / (G * hb)));
  if (tid == 0)
    for (int i = 0; i < ns; ++i) mbar_init(&bar[i], 1);
  __syncthreads();
  auto issue = [&](int stg, int slot) {
    const int e0 = stg * G;
    const int cnt = min(G, ne - e0);
    const unsigned bytes = (unsigned)(cnt * per * sizeof(S));
    const unsigned vb = (unsigned)(cnt * b * sizeof(R));  // a multiple of 16 (b * 4 is)
    const unsigned total = bytes + vb * (1 + (Gx ? 1 : 0) + (x_zero ? 0 : 1));
    mbar_expect_tx(&bar[slot], total);
    bulk_g2s(blocks_of(slot), A + (size_t)e0 * per, bytes, &bar[slot]);
    R* v = vecs_of(slot);
    bulk_g2s(v, g + (size_t)e0 * b, vb, &bar[slot]);
    if (Gx) bulk_g2s(v + vec, Gx + (size_t)e0 * b, vb, &bar[slot]);
    if (!x_zero) bulk_g2s(v + 2 * vec, x + (size_t)e0 * b, vb, &bar[slot]);
  };
  // iteration k of this CTA handles stage blockIdx.x + k * gridDim.x in slot k % ns (use k / ns).
  // Thread 0 keeps a bit per slot whose copies are in flight. withhold_first != 0 (a test of the
  // bounded wait) leaves the first stage's copies unissued, so its barrier phase never completes.
  unsigned inflight = 0;
  if (tid == 0)
    for (int i = 0; i < ns - 1; ++i) {
      const int st0 = blockIdx.x + i * gridDim.x;
      if (st0 < nstages && !(withhold_first && i == 0)) {
        issue(st0, i);
        inflight |= 1u << i;
      }
    }
  int k = 0;
  for (int stg = blockIdx.x; stg < nstages; stg += gridDim.x, ++k) {
    const int slot = k % ns;
    const int ahead = stg + (ns - 1) * gridDim.x;  // into the slot released at the end of k - 1
    if (tid == 0 && ahead < nstages) {
      issue(ahead, (k + ns - 1) % ns);
      inflight |= 1u << ((k + ns - 1) % ns);
    }
    const int e0 = stg * G;
    const int cnt = min(G, ne - e0);
    const bool got = mbar_wait(&bar[slot], (unsigned)((k / ns) & 1), wait_polls);
    if (!__syncthreads_and(got)) {
      // give up: report, let every copy in flight land (the current slot's included; bounded
      // waits with the full limit), then leave, so that no copy writes this CTA's shared memory
      // after it exits
      if (tid == 0) {
        atomicOr(status, (unsigned)DG_STATUS_WAIT);
        for (int i = 0; i < ns; ++i) {
          const int sl = (k + i) % ns;
          if (inflight & (1u << sl)) mbar_wait(&bar[sl], (unsigned)(((k + i) / ns) & 1));
        }
      }
      return;
    }
    if (tid == 0) inflight &= ~(1u << slot);
    const S* Ab = blocks_of(slot);
    R* const rv = vecs_of(slot);  // g, turned into the residual g - Gx in place
    const R* const xo = rv + 2 * vec;
    if (Gx) {
      for (int t = tid; t < cnt * b; t += nt) rv[t] -= rv[vec + t];
      __syncthreads();
    }
    const int npairs = cnt * hb;
    for (int t = tid; t < npairs * CS; t += nt) {
      const int pr = t % npairs, cs = t / npairs;
      const int el = pr / hb, i0 = 2 * (pr - el * hb);
      const S* Ae = Ab + (size_t)el * per + i0;
      const R* re = rv + (size_t)el * b;
      R a0 = R(0), a1 = R(0), c0 = R(0), c1 = R(0);
      int j = cs;
      for (; j + CS < b; j += 2 * CS) {
        R u0, u1, v0, v1;
        wide2<R>(Ae + (size_t)j * b, u0, u1);
        wide2<R>(Ae + (size_t)(j + CS) * b, v0, v1);
        a0 = fma(u0, re[j], a0);
        a1 = fma(u1, re[j], a1);
        c0 = fma(v0, re[j + CS], c0);
        c1 = fma(v1, re[j + CS], c1);
      }
      if (j < b) {
        R u0, u1;
        wide2<R>(Ae + (size_t)j * b, u0, u1);
        a0 = fma(u0, re[j], a0);
        a1 = fma(u1, re[j], a1);
      }
      a0 += c0;
      a1 += c1;
      if (CS == 1) {
        R* xe = x + (size_t)(e0 + el) * b + i0;
        const R* xs = xo + (size_t)el * b + i0;
        xe[0] = (x_zero ? R(0) : xs[0]) + alpha * a0;
        xe[1] = (x_zero ? R(0) : xs[1]) + alpha * a1;
      } else {
        red[2 * t] = a0;
        red[2 * t + 1] = a1;
      }
    }
    if (CS > 1) {
      __syncthreads();
      for (int pr = tid; pr < npairs; pr += nt) {
        R a0 = R(0), a1 = R(0);
        for (int cs = 0; cs < CS; ++cs) {
          a0 += red[2 * (cs * npairs + pr)];
          a1 += red[2 * (cs * npairs + pr) + 1];
        }
        const int el = pr / hb, i0 = 2 * (pr - el * hb);
        R* xe = x + (size_t)(e0 + el) * b + i0;
        const R* xs = xo + (size_t)el * b + i0;
        xe[0] = (x_zero ? R(0) : xs[0]) + alpha * a0;
        xe[1] = (x_zero ? R(0) : xs[1]) + alpha * a1;
      }
    }
    // this slot, its residual and red are free for the copy issued next: the generic-proxy
    // writes above (the residual formed in place) are ordered before that async-proxy copy
    fence_proxy_async_smem();
    __syncthreads();
  }
}

// The 16-bit block-Jacobi apply for large blocks (b = 140 at P4: a 39.2 KB inverse per element),
// one element per stage and a ring of up to kPairSlots stages, so that four elements stream in
// while one is multiplied. Same update as staged_jacobi_kernel. A column pair of the
// column-major inverse (2 B entries) is B / 4 chunks of 16 bytes, and thread tid reads chunks
// tid, tid + T, tid + 2 T, ... (T = CS * B / 4): all of them hold the same eight rows (rows of
// column 2m, of column 2m + 1, or four of each where a chunk straddles the two), so the thread
// keeps eight row sums in registers, and consecutive threads read consecutive chunks (no bank
// conflicts). The sums over the even and the odd columns of the CS column slices meet in shared
// memory. The residual g - Gx is formed where it
// is used. Per element: one barrier after the stage's wait (it also frees the previous stage's
// buffer, refilled right after it) and one before the slice reduction.
constexpr int kPairSlots = 5;

template <class S> __device__ __forceinline__ float2 widen_word(unsigned w);
template <> __device__ __forceinline__ float2 widen_word<__half>(unsigned w) {
  __half2 h;
  memcpy(&h, &w, sizeof(h));
  return __half22float2(h);
}
template <> __device__ __forceinline__ float2 widen_word<__nv_bfloat16>(unsigned w) {
  return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));  // exact
}

template <int B, int NT, class S>
__global__ void __launch_bounds__(NT) pair_jacobi_kernel(int ne, int ns, const S* __restrict__ A,
                                                         const float* __restrict__ g, const float* __restrict__ Gx,
                                                         float alpha, int x_zero, float* __restrict__ x,
                                                         unsigned* status, unsigned wait_polls, int withhold_first) {
  static_assert(B % 4 == 0 && sizeof(S) == 2, "16-bit blocks of 4 n rows");
  constexpr int CP = B / 4;                  // 16-byte chunks per column pair
  constexpr int NP = B / 2;                  // column pairs
  constexpr int CS = NT / CP;                // column slices
  constexpr int PPS = (NP + CS - 1) / CS;    // column pairs per slice (the last ones ragged)
  constexpr size_t kBlk = (size_t)B * B * 2;
  constexpr size_t kSlot = kBlk + 3 * B * sizeof(float);  // inverse, then g, Gx, old x
  static_assert(CS >= 1 && kBlk % 16 == 0 && kSlot % 16 == 0, "stage layout");
  extern __shared__ __align__(128) unsigned char sraw_[];
  __shared__ uint64_t bar[kPairSlots];
  float* red = reinterpret_cast<float*>(sraw_ + (size_t)ns * kSlot);  // [CS][2][B] slice sums
  const int tid = threadIdx.x;
  const bool has_gx = Gx != nullptr;
  if (tid == 0)
    for (int i = 0; i < ns; ++i) mbar_init(&bar[i], 1);
  __syncthreads();
  auto issue = [&](int e, int slot) {
    unsigned char* sb = sraw_ + (size_t)slot * kSlot;
    float* v = reinterpret_cast<float*>(sb + kBlk);
    const unsigned vb = B * sizeof(float);
    mbar_expect_tx(&bar[slot], (unsigned)kBlk + vb * (1 + (has_gx ? 1 : 0) + (x_zero ? 0 : 1)));
    bulk_g2s(sb, A + (size_t)e * B * B, (unsigned)kBlk, &bar[slot]);
    bulk_g2s(v, g + (size_t)e * B, vb, &bar[slot]);
    if (has_gx) bulk_g2s(v + B, Gx + (size_t)e * B, vb, &bar[slot]);
    if (!x_zero) bulk_g2s(v + 2 * B, x + (size_t)e * B, vb, &bar[slot]);
  };
  // iteration k of this CTA takes element blockIdx.x + k * gridDim.x in slot k % ns (phase k / ns);
  // thread 0 keeps a bit per slot whose copies are in flight; withhold_first (a test of the
  // bounded wait) leaves the first element's copies unissued
  unsigned inflight = 0;
  if (tid == 0)
    for (int i = 0; i < ns - 1; ++i) {
      const int e = blockIdx.x + i * gridDim.x;
      if (e < ne && !(withhold_first && i == 0)) {
        issue(e, i);
        inflight |= 1u << i;
      }
    }
  // the thread's chunk within a column pair, its first column pair, and the rows of its chunk:
  // entries 0-3 at rows lo_r.. of column 2m + lo_c, entries 4-7 at rows up_r.. of column 2m + up_c
  const int t = tid % CP, s0 = tid / CP;
  const bool active = tid < CS * CP;
  const int lo_c = 8 * t < B ? 0 : 1, lo_r = 8 * t - lo_c * B;
  const int up_c = 8 * t + 4 < B ? 0 : 1, up_r = 8 * t + 4 - up_c * B;
  int k = 0;
  for (int e = blockIdx.x; e < ne; e += gridDim.x, ++k) {
    const int slot = k % ns;
    const bool got = mbar_wait(&bar[slot], (unsigned)((k / ns) & 1), wait_polls);
    if (!__syncthreads_and(got)) {
      // give up: report, let every copy in flight land (bounded waits with the full limit), then
      // leave, so that no copy writes this CTA's shared memory after it exits
      if (tid == 0) {
        atomicOr(status, (unsigned)DG_STATUS_WAIT);
        for (int i = 0; i < ns; ++i) {
          const int sl = (k + i) % ns;
          if (inflight & (1u << sl)) mbar_wait(&bar[sl], (unsigned)(((k + i) / ns) & 1));
        }
      }
      return;
    }
    if (tid == 0) {
      // every thread is past the previous element (its reads of that slot were fenced against
      // the async proxy): refill that slot with the element ns - 1 ahead
      inflight &= ~(1u << slot);
      const int ahead = e + (ns - 1) * gridDim.x;
      if (ahead < ne) {
        const int sl = (k + ns - 1) % ns;
        issue(ahead, sl);
        inflight |= 1u << sl;
      }
    }
    const unsigned char* sb = sraw_ + (size_t)slot * kSlot;
    const uint4* Ab = reinterpret_cast<const uint4*>(sb);
    const float* gv = reinterpret_cast<const float*>(sb + kBlk);
    if (active) {
      float acc[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[q] = 0.0f;
#pragma unroll
      for (int i = 0; i < PPS; ++i) {
        const int m = s0 + i * CS;
        if (NP % CS == 0 || m < NP) {
          const uint4 w = Ab[m * CP + t];
          float2 r = *reinterpret_cast<const float2*>(gv + 2 * m);
          if (has_gx) {
            const float2 q = *reinterpret_cast<const float2*>(gv + B + 2 * m);
            r.x -= q.x;
            r.y -= q.y;
          }
          const float rl = lo_c ? r.y : r.x, ru = up_c ? r.y : r.x;
          const float2 a0 = widen_word<S>(w.x), a1 = widen_word<S>(w.y);
          const float2 a2 = widen_word<S>(w.z), a3 = widen_word<S>(w.w);
          acc[0] = fmaf(a0.x, rl, acc[0]);
          acc[1] = fmaf(a0.y, rl, acc[1]);
          acc[2] = fmaf(a1.x, rl, acc[2]);
          acc[3] = fmaf(a1.y, rl, acc[3]);
          acc[4] = fmaf(a2.x, ru, acc[4]);
          acc[5] = fmaf(a2.y, ru, acc[5]);
          acc[6] = fmaf(a3.x, ru, acc[6]);
          acc[7] = fmaf(a3.y, ru, acc[7]);
        }
      }
      // every row has one sum over the slice's even columns and one over its odd columns
      *reinterpret_cast<float4*>(red + (2 * s0 + lo_c) * B + lo_r) = make_float4(acc[0], acc[1], acc[2], acc[3]);
      *reinterpret_cast<float4*>(red + (2 * s0 + up_c) * B + up_r) = make_float4(acc[4], acc[5], acc[6], acc[7]);
    }
    __syncthreads();
    const float* xo = gv + 2 * B;
    for (int r = tid; r < B; r += NT) {
      float sum = 0.0f;
#pragma unroll
      for (int s = 0; s < 2 * CS; ++s) sum += red[s * B + r];
      x[(size_t)e * B + r] = (x_zero ? 0.0f : xo[r]) + alpha * sum;
    }
    // this slot's reads (generic proxy) before the bulk copy that refills it (async proxy)
    fence_proxy_async_smem();
  }
}

// The same row products read straight from global memory: one thread per output row, `epc`
// elements per CTA (b rows each), the input vectors in shared memory. Loads of one warp cover
// 32 consecutive rows of a column (coalesced); eight independent accumulators keep eight loads
// in flight per thread, and small CTAs keep many elements in flight per SM. (One thread per
// pair of rows with paired loads halves the threads and was slower: 61 against 45 us at P2.)
template <class R, int NBLK, class S>
__global__ void __launch_bounds__(256) direct_apply_kernel(int ne, int b, int epc, const S* __restrict__ A,
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
        rv[t] = src >= 0 ? v[(size_t)src * b + c] : R(0);  // no neighbour across a wall (zero block)
      }
    }
    __syncthreads();
    if (tid < cnt * b) {
      const int el = tid / b, i = tid - el * b;
      const S* Ae = A + (size_t)(e0 + el) * ncol * b + i;
      const R* re = rv + (size_t)el * ncol;
      R a[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) a[u] = R(0);
      int q = 0;
      for (; q + 7 < ncol; q += 8) {
#pragma unroll
        for (int u = 0; u < 8; ++u) a[u] = fma(wide<R>(__ldg(Ae + (size_t)(q + u) * b)), re[q + u], a[u]);
      }
      for (; q < ncol; ++q) a[0] = fma(wide<R>(__ldg(Ae + (size_t)q * b)), re[q], a[0]);
      const R acc = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
      R* ye = y + (size_t)(e0 + el) * b + i;
      if (NBLK == 1) *ye = (x_zero ? R(0) : *ye) + alpha * acc;
      else *ye = alpha * acc + (beta == R(0) ? R(0) : beta * *ye);
    }
    __syncthreads();
  }
}

template <class R, int NBLK, class S>
int launch_direct(Handle* h, int b, const S* A, const R* v, const R* w, R alpha, R beta, int x_zero, R* y,
                  cudaStream_t st) {
  if (b > 256) return -1;  // -1, not a DG_ code: the caller falls back to bsr_kernel
  const int epc = std::max(1, 256 / b);
  const int threads = 32 * ((epc * b + 31) / 32);
  const size_t smem = sizeof(R) * (size_t)epc * NBLK * b;
  const int grid = (h->ne + epc - 1) / epc;
  direct_apply_kernel<R, NBLK, S><<<grid, threads, smem, st>>>(h->ne, b, epc, A, h->nbr, v, w, alpha, beta, x_zero,
                                                               y);
  DG_LAUNCH_CHECK(h);
  return DG_OK;
}

// Eight 16-bit entries (one 16-byte vector) widened to float.
__device__ __forceinline__ void wide8(const uint4& raw, const __half*, float* o) {
  const __half2* h2 = reinterpret_cast<const __half2*>(&raw);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float2 f = __half22float2(h2[j]);
    o[2 * j] = f.x;
    o[2 * j + 1] = f.y;
  }
}
__device__ __forceinline__ void wide8(const uint4& raw, const __nv_bfloat16*, float* o) {
  const __nv_bfloat162* h2 = reinterpret_cast<const __nv_bfloat162*>(&raw);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float2 f = __bfloat1622float2(h2[j]);
    o[2 * j] = f.x;
    o[2 * j + 1] = f.y;
  }
}

// y = alpha A x + beta y over rows of 7 blocks stored in 16 bits (b a multiple of 8), FP32
// accumulation. A task is eight consecutive rows of one block: per block column it loads one
// 16-byte vector, so a warp's load moves 512 bytes and a thread keeps eight loads (128 bytes)
// in flight. The seven block partial sums of a row meet in shared memory and are added in
// block order.
template <class S>
__global__ void __launch_bounds__(256) direct7_vec_kernel(int ne, int b, int epc, const S* __restrict__ A,
                                                          const int* __restrict__ nbr, const float* __restrict__ v,
                                                          float alpha, float beta, float* __restrict__ y) {
  extern __shared__ __align__(16) unsigned char sraw_[];
  const int ncol = 7 * b, rg = b / 8, tpe = 7 * rg;
  float* rv = reinterpret_cast<float*>(sraw_);  // [epc][ncol] the seven slices of v
  float* part = rv + (size_t)epc * ncol;       // [epc][7][b] block partial sums
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e0 = blockIdx.x * epc; e0 < ne; e0 += gridDim.x * epc) {
    const int cnt = min(epc, ne - e0);
    for (int t = tid; t < cnt * ncol; t += nt) {
      const int el = t / ncol, q = t - el * ncol;
      const int e = e0 + el;
      const int sb = q / b, c = q - sb * b;
      const int src = sb == 0 ? e : nbr[(size_t)e * 6 + sb - 1];
      rv[t] = src >= 0 ? v[(size_t)src * b + c] : 0.0f;  // no neighbour across a wall (zero block)
    }
    __syncthreads();
    if (tid < cnt * tpe) {
      const int el = tid / tpe, r = tid - el * tpe, sb = r / rg, r8 = r - sb * rg;
      const S* As = A + (size_t)(e0 + el) * ncol * b + (size_t)sb * b * b + 8 * r8;
      const float* re = rv + (size_t)el * ncol + sb * b;
      float acc[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) acc[u] = 0.0f;
#pragma unroll 8
      for (int c = 0; c < b; ++c) {
        const uint4 raw = __ldg(reinterpret_cast<const uint4*>(As + (size_t)c * b));
        float a8[8];
        wide8(raw, As, a8);
        const float xc = re[c];
#pragma unroll
        for (int u = 0; u < 8; ++u) acc[u] = fmaf(a8[u], xc, acc[u]);
      }
      float* ps = part + ((size_t)el * 7 + sb) * b + 8 * r8;
#pragma unroll
      for (int u = 0; u < 8; ++u) ps[u] = acc[u];
    }
    __syncthreads();
    for (int t = tid; t < cnt * b; t += nt) {
      const int el = t / b, i = t - el * b;
      const float* pe = part + (size_t)el * 7 * b + i;
      float acc = pe[0];
#pragma unroll
      for (int sb = 1; sb < 7; ++sb) acc += pe[sb * b];
      float* ye = y + (size_t)(e0 + el) * b + i;
      *ye = alpha * acc + (beta == 0.0f ? 0.0f : beta * *ye);
    }
    __syncthreads();
  }
}

template <class S>
int launch_direct7_vec(Handle* h, int b, const S* A, const float* v, float alpha, float beta, float* y,
                       cudaStream_t st) {
  const int tpe = 7 * (b / 8);
  if (b % 8 != 0 || tpe > 256) return -1;  // -1: unsuited; the caller reports it
  const int epc = std::max(1, 256 / tpe);
  const int threads = 32 * ((epc * tpe + 31) / 32);
  const size_t smem = sizeof(float) * (size_t)epc * 14 * b;  // slices of v and partial sums
  const int grid = (h->ne + epc - 1) / epc;
  direct7_vec_kernel<S><<<grid, threads, smem, st>>>(h->ne, b, epc, A, h->nbr, v, alpha, beta, y);
  DG_LAUNCH_CHECK(h);
  return DG_OK;
}

constexpr size_t kStageTarget = 96 * 1024;  // bytes of inverses per stage (one buffer)
constexpr size_t kSmemLimit = 220 * 1024;    // dynamic shared memory a kernel may take

// the 16-bit apply of large blocks, one element per stage (pair_jacobi_kernel); -1: unsuited
template <int B, class S>
int launch_pair_jacobi(Handle* h, const S* A, const float* g, const float* Gx, float alpha, int x_zero, float* x,
                       cudaStream_t st) {
  constexpr int NT = kJacobiThreads, CS = NT / (B / 4);
  constexpr size_t slot = (size_t)B * B * 2 + 3 * (size_t)B * sizeof(float);
  const size_t red = sizeof(float) * 2 * CS * B;
  const int ns = (int)std::min<size_t>(kPairSlots, (kSmemLimit - red) / slot);
  if (ns < 2) return -1;
  const size_t smem = (size_t)ns * slot + red;
  static bool opted = false;  // per template instance; one device per process
  if (!opted) {
    DG_CUDA(h, cudaFuncSetAttribute(pair_jacobi_kernel<B, NT, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kSmemLimit));
    opted = true;
  }
  const int cap = h->tune[1].jacobi_max_ctas;  // 0: one CTA per SM
  const int grid = std::min(h->ne, cap > 0 ? std::min(cap, h->nsm) : h->nsm);
  const unsigned polls = h->dbg.wait_polls > 0 ? (unsigned)h->dbg.wait_polls : kBulkWaitLimit;
  pair_jacobi_kernel<B, NT, S><<<grid, NT, smem, st>>>(h->ne, ns, A, g, Gx, alpha, x_zero, x, h->status, polls,
                                                      h->dbg.withhold_copy);
  DG_LAUNCH_CHECK(h);
  return DG_OK;
}

template <class R, class S>
int launch_staged_jacobi(Handle* h, int b, const S* A, const R* g, const R* Gx, R alpha, int x_zero, R* x,
                         cudaStream_t st) {
  if constexpr (std::is_same<R, float>::value && sizeof(S) == 2) {
    if (b == 140) return launch_pair_jacobi<140, S>(h, A, g, Gx, alpha, x_zero, x, st);
  }
  const size_t per = (size_t)b * b * sizeof(S);
  const size_t target = h->tune[1].jacobi_stage_kb > 0 ? (size_t)h->tune[1].jacobi_stage_kb * 1024 : kStageTarget;
  int G = (int)std::max<size_t>(1, target / per);
  const size_t per_slot = per + 3 * (size_t)b * sizeof(R);  // one buffer: block + g, Gx, x slices
  G = std::min(G, (int)std::max<size_t>(1, kSmemLimit / (2 * per_slot)));  // two buffers fit
  // at most this many CTAs (jacobi_max_ctas, 0: no cap; every CTA then walks the ring more often)
  const int cap = h->tune[1].jacobi_max_ctas;
  const int ctas = cap > 0 ? std::min(cap, h->nsm) : h->nsm;
  G = std::max(1, std::min(G, (h->ne + 2 * ctas - 1) / (2 * ctas)));  // >= 2 stages per CTA when possible
  // as many buffers as fit (2..4): the stages in flight while one is multiplied
  const int ns = (int)std::max<size_t>(2, std::min<size_t>(kJacobiSlots, kSmemLimit / ((size_t)G * per_slot)));
  const size_t smem = (size_t)ns * G * per_slot;
  // -1, not a DG_ code: the block does not fit the staged copies; the smoother and the autotuner
  // report it
  if (smem > kSmemLimit || per % 16 != 0 || (b * sizeof(R)) % 16 != 0) return -1;
  static bool opted = false;  // per template instance; one device per process
  if (!opted) {
    DG_CUDA(h, cudaFuncSetAttribute(staged_jacobi_kernel<R, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kSmemLimit));
    opted = true;
  }
  const int nstages = (h->ne + G - 1) / G;
  const int per_sm = (int)std::max<size_t>(1, std::min<size_t>(4, (227 * 1024) / (smem + 1024)));
  const int grid = std::min(nstages, cap > 0 ? ctas : h->nsm * per_sm);
  const unsigned polls = h->dbg.wait_polls > 0 ? (unsigned)h->dbg.wait_polls : kBulkWaitLimit;
  staged_jacobi_kernel<R, S><<<grid, kJacobiThreads, smem, st>>>(h->ne, b, G, ns, A, g, Gx, alpha, x_zero, x,
                                                                h->status, polls, h->dbg.withhold_copy);
  DG_LAUNCH_CHECK(h);
  return DG_OK;
}

}  // namespace

namespace {
__global__ void narrow_half_kernel(long long n, const float* __restrict__ x, __half* __restrict__ y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = __float2half_rn(x[i]);
}
__global__ void narrow_bf16_kernel(long long n, const float* __restrict__ x, __nv_bfloat16* __restrict__ y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16_rn(x[i]);
}
int narrow(Handle* h, int storage, long long n, const float* x, void* y, cudaStream_t st) {
  const int grid = (int)std::min<long long>((long long)h->nsm * 8, n / 256 + 1);
  if (storage == DG_PRECOND_FP32_H16)
    narrow_half_kernel<<<grid, 256, 0, st>>>(n, x, static_cast<__half*>(y));
  else
    narrow_bf16_kernel<<<grid, 256, 0, st>>>(n, x, static_cast<__nv_bfloat16*>(y));
  DG_LAUNCH_CHECK(h);
  return DG_OK;
}
size_t storage_size(int storage) { return storage == DG_PRECOND_FP32 ? sizeof(float) : 2; }
}  // namespace

int prepare_blocks16(Handle* h, int storage, cudaStream_t st) {
  if (h->asm16 == storage) return DG_OK;
  for (int l = 0; l < h->nlev; ++l) {
    Level& L = h->lev[l];
    const long long nbb = (long long)h->ne * L.b * L.b;
    if (!L.LU16) DG_CUDA(h, cudaMalloc(&L.LU16, 2 * (size_t)nbb));
    if (int rc = narrow(h, storage, nbb, L.LUf, L.LU16, st)) return rc;
    if (l >= 1) {
      if (!L.Bsr16) DG_CUDA(h, cudaMalloc(&L.Bsr16, 2 * (size_t)nbb * 7));
      if (int rc = narrow(h, storage, 7 * nbb, L.Bsrf, L.Bsr16, st)) return rc;
    }
  }
  h->asm16 = storage;
  return DG_OK;
}

int staged_jacobi_f(Handle* h, int lvl, const float* g, const float* Gx, float omega, bool x_zero, float* x,
                    int storage, cudaStream_t st) {
  const Level& L = h->lev[lvl];
  cudaEvent_t e0 = nullptr;
  int rc;
  if (lvl == 0 && (rc = prof_begin(h, st, &e0))) return rc;
  const int xz = x_zero ? 1 : 0;
  if (storage == DG_PRECOND_FP32_H16)
    rc = launch_staged_jacobi<float, __half>(h, L.b, static_cast<const __half*>(L.LU16), g, Gx, omega, xz, x, st);
  else if (storage == DG_PRECOND_FP32_BF16)
    rc = launch_staged_jacobi<float, __nv_bfloat16>(h, L.b, static_cast<const __nv_bfloat16*>(L.LU16), g, Gx, omega, xz,
                                                    x, st);
  else
    rc = launch_staged_jacobi<float, float>(h, L.b, L.LUf, g, Gx, omega, xz, x, st);
  if (rc) return rc;
  // algorithmic bytes: the inverses, g, Gx and the old x read once, x written once
  const double vec = (double)h->ne * L.b * sizeof(float);
  const double bytes = (double)h->ne * L.b * L.b * storage_size(storage) + vec * (2 + (Gx ? 1 : 0) + (x_zero ? 0 : 1));
  return lvl == 0 ? prof_end(h, DG_PROF_BJ32, st, e0, bytes) : DG_OK;
}

template <class R>
int staged_bsr(Handle* h, int lvl, const R* B, R alpha, const R* x, R beta, R* y, cudaStream_t st) {
  const int b = h->lev[lvl].b;
  cudaEvent_t e0 = nullptr;
  int rc;
  if (lvl == 1 && (rc = prof_begin(h, st, &e0))) return rc;
  rc = launch_direct<R, 7, R>(h, b, B, x, nullptr, alpha, beta, 0, y, st);
  if (rc) return rc;
  // algorithmic bytes: the 7 blocks of every row, x and the old y read once, y written once
  const double vec = (double)h->ne * b * sizeof(R);
  const double bytes = 7.0 * h->ne * b * b * sizeof(R) + vec * (2 + (beta != R(0) ? 1 : 0));
  return lvl == 1 ? prof_end(h, sizeof(R) == 4 ? DG_PROF_BSR32 : DG_PROF_BSR64, st, e0, bytes) : DG_OK;
}
template int staged_bsr<float>(Handle*, int, const float*, float, const float*, float, float*, cudaStream_t);
template int staged_bsr<double>(Handle*, int, const double*, double, const double*, double, double*, cudaStream_t);

int bsr16_f(Handle* h, int lvl, int storage, float alpha, const float* x, float beta, float* y, cudaStream_t st) {
  const Level& L = h->lev[lvl];
  cudaEvent_t e0 = nullptr;
  int rc;
  if (lvl == 1 && (rc = prof_begin(h, st, &e0))) return rc;
  if (L.b % 8 == 0) {  // 16-byte vectors of eight rows
    if (storage == DG_PRECOND_FP32_H16)
      rc = launch_direct7_vec<__half>(h, L.b, static_cast<const __half*>(L.Bsr16), x, alpha, beta, y, st);
    else
      rc = launch_direct7_vec<__nv_bfloat16>(h, L.b, static_cast<const __nv_bfloat16*>(L.Bsr16), x, alpha, beta, y,
                                             st);
  } else if (storage == DG_PRECOND_FP32_H16) {
    rc = launch_direct<float, 7, __half>(h, L.b, static_cast<const __half*>(L.Bsr16), x, nullptr, alpha, beta, 0, y, st);
  } else {
    rc = launch_direct<float, 7, __nv_bfloat16>(h, L.b, static_cast<const __nv_bfloat16*>(L.Bsr16), x, nullptr, alpha,
                                                beta, 0, y, st);
  }
  if (rc) return rc;
  const double vec = (double)h->ne * L.b * sizeof(float);
  const double bytes = 7.0 * h->ne * L.b * L.b * 2 + vec * (2 + (beta != 0.0f ? 1 : 0));
  return lvl == 1 ? prof_end(h, DG_PROF_BSR32, st, e0, bytes) : DG_OK;
}

int invert_levels_f32(Handle* h, cudaStream_t st, unsigned* status) {
  for (int l = 0; l < h->nlev; ++l) {
    const Level& L = h->lev[l];
    if (L.b == 40 || L.b == 16) {  // one warp per block
      const size_t smem = sizeof(float) * kGjwWarps * (size_t)(L.b * L.b + 4 * L.b);
      const int grid = std::min((h->ne + kGjwWarps - 1) / kGjwWarps, h->nsm * 4);
      if (L.b == 40) {
        DG_CUDA(h, cudaFuncSetAttribute(gj_inverse_warp_kernel<40>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem));
        gj_inverse_warp_kernel<40><<<grid, 32 * kGjwWarps, smem, st>>>(h->ne, L.LUf, status);
      } else {
        gj_inverse_warp_kernel<16><<<grid, 32 * kGjwWarps, smem, st>>>(h->ne, L.LUf, status);
      }
      DG_LAUNCH_CHECK(h);
      continue;
    }
    const size_t smem = sizeof(float) * ((size_t)(L.b + 4) * gj_ld(L.b)) + sizeof(int) * 2 * L.b;
    if (smem > kSmemLimit || L.b % 4 != 0 || L.b > 32 * kGjSlots)
      return fail(h, DG_ERR_ARG, "element block unsuited to the FP32 inverse");
    DG_CUDA(h, cudaFuncSetAttribute(gj_inverse_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kSmemLimit));
    DG_CUDA(h, cudaFuncSetAttribute(gj_inverse_kernel<140>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kSmemLimit));
    const int per_sm = (int)std::max<size_t>(1, std::min<size_t>(4, (227 * 1024) / (smem + 1024)));
    const int grid = std::min(h->ne, h->nsm * per_sm);
    // warp 0 factors; the (column group, row group) pairs of the update on the warps after it:
    // at most 512 threads, at most b row groups
    const int ng = L.b / 4, active = ng * std::min(L.b, 480 / ng);
    const int threads = std::min(512, 32 + 32 * ((active + 31) / 32));
    if (L.b == 140 && threads == 512)
      gj_inverse_kernel<140><<<grid, threads, smem, st>>>(h->ne, L.b, L.LUf, status);
    else
      gj_inverse_kernel<0><<<grid, threads, smem, st>>>(h->ne, L.b, L.LUf, status);
    DG_LAUNCH_CHECK(h);
  }
  return DG_OK;
}

}  // namespace dg
