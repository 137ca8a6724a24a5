// p-multigrid and Krylov parts of the hot path (Sec. 2.3-2.4, Algorithms 2-3):
// restriction / prolongation, block-sparse coarse products, element-block-Jacobi
// smoothing, MG_V / MG_full cycles and right-preconditioned flexible GMRES, with
// deterministic (fixed-order) FP64 reductions.
#include <algorithm>
#include <cmath>
#include <vector>

#include "dg_internal.h"

namespace dg {

constexpr int kRedBlocks = 512;  // fixed partial count: reductions are bitwise reproducible

// ------------------------------------------------------------ reductions
__global__ void __launch_bounds__(256) norm2_partial_kernel(long long n, const double* x, double* part) {
  __shared__ double s[256];
  double acc = 0.0;
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += (long long)gridDim.x * 256) acc += x[i] * x[i];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

// out[j] = sum_b part[b * stride + j] for j < nvec, in a fixed order.
__global__ void __launch_bounds__(256) reduce_partials_kernel(int nblk, int nvec, int stride, const double* part,
                                                              double* out) {
  __shared__ double s[256];
  for (int j = 0; j < nvec; ++j) {
    double acc = 0.0;
    for (int b = threadIdx.x; b < nblk; b += 256) acc += part[(size_t)b * stride + j];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
      if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[j] = s[0];
    __syncthreads();
  }
}

int vec_norm2(Handle* h, const double* x, long long n, double* dev_out, cudaStream_t st) {
  norm2_partial_kernel<<<kRedBlocks, 256, 0, st>>>(n, x, h->red);
  DG_LAUNCH_CHECK(h);
  reduce_partials_kernel<<<1, 256, 0, st>>>(kRedBlocks, 1, 1, h->red, dev_out);
  DG_LAUNCH_CHECK(h);
  return DG_OK;
}

// part[b][j] = sum over this block's slice of V[j][i] * w[i], j < nv (nv <= 8 per launch)
__global__ void __launch_bounds__(256) multidot_partial_kernel(long long n, int nv, const double* V, long long ldv,
                                                               const double* w, double* part, int stride) {
  __shared__ double s[8][256];
  double acc[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) acc[j] = 0.0;
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
    const double wi = w[i];
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (j < nv) acc[j] += V[j * ldv + i] * wi;
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) s[j][threadIdx.x] = acc[j];
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int j = 0; j < nv; ++j) s[j][threadIdx.x] += s[j][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x < nv) part[(size_t)blockIdx.x * stride + threadIdx.x] = s[threadIdx.x][0];
}

// w -= sum_j hcoef[j] * V[j], j < nv; also w is scaled by nothing
__global__ void multi_axpy_kernel(long long n, int nv, const double* V, long long ldv, const double* hcoef, double* w) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double acc = w[i];
    for (int j = 0; j < nv; ++j) acc -= hcoef[j] * V[j * ldv + i];
    w[i] = acc;
  }
}

template <class R>
__global__ void axpby_kernel(long long n, R a, const R* x, R b, R* y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = a * x[i] + (b == R(0) ? R(0) : b * y[i]);
}

// FP64 <-> FP32 copies at the boundary of the reduced-precision preconditioner
template <class A, class B>
__global__ void convert_kernel(long long n, const A* x, B* y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = (B)x[i];
}

__global__ void scale_by_dev_kernel(long long n, const double* x, const double* dnorm2, double* y) {
  const double nv = sqrt(*dnorm2);
  const double inv = nv > 0.0 ? 1.0 / nv : 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = x[i] * inv;
}

int launch_axpby(Handle* h, long long n, double a, const double* x, double b, double* y, cudaStream_t st) {
  axpby_kernel<double><<<h->nsm * 8, 256, 0, st>>>(n, a, x, b, y);
  DG_LAUNCH_CHECK(h);
  return DG_OK;
}

// ------------------------------------------------------ transfer operators
template <class R>
__global__ void restrict_kernel(int ne, int nbf, int nbc, const R* xf, R* xc) {
  const long long n = (long long)ne * 4 * nbc;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long ev = i / nbc;
    const int m = (int)(i - ev * nbc);
    xc[i] = xf[ev * nbf + m];
  }
}
template <class R>
__global__ void prolong_add_kernel(int ne, int nbf, int nbc, const R* xc, R* xf) {
  const long long n = (long long)ne * 4 * nbc;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long ev = i / nbc;
    const int m = (int)(i - ev * nbc);
    xf[ev * nbf + m] += xc[i];
  }
}

// ------------------------------------------------------- block operations
// y[e] = alpha * sum_s B[e][s] x[nbr(e,s)] + beta * y[e]; slot 0 is the element itself.
template <class R>
__global__ void __launch_bounds__(128) bsr_kernel(int ne, int b, const int* nbr, const R* B, R alpha,
                                                  const R* x, R beta, R* y) {
  extern __shared__ __align__(16) unsigned char sraw_[];
  R* sx = reinterpret_cast<R*>(sraw_);  // [7][b]
  for (int e = blockIdx.x; e < ne; e += gridDim.x) {
    for (int t = threadIdx.x; t < 7 * b; t += blockDim.x) {
      const int s = t / b, c = t - s * b;
      const int col = s == 0 ? e : nbr[e * 6 + s - 1];
      sx[t] = col >= 0 ? x[(size_t)col * b + c] : R(0);  // no neighbour across a wall (zero block)
    }
    __syncthreads();
    for (int r = threadIdx.x; r < b; r += blockDim.x) {
      R acc = R(0);
      const R* Be = B + (size_t)e * 7 * b * b;
      for (int s = 0; s < 7; ++s)
        for (int c = 0; c < b; ++c) acc += Be[((size_t)s * b + c) * b + r] * sx[s * b + c];
      y[(size_t)e * b + r] = alpha * acc + (beta == R(0) ? R(0) : beta * y[(size_t)e * b + r]);
    }
    __syncthreads();
  }
}

// y[e] = alpha * (G^T x)[e] + beta * y[e]: the blocks of column e are B[e][0] and, for each face
// slot s of e, B[nbr(e,s)][opposite(s)] (the neighbour's block pointing back across that face).
template <class R>
__global__ void __launch_bounds__(128) bsr_t_kernel(int ne, int b, const int* nbr, const R* B, R alpha,
                                                    const R* x, R beta, R* y) {
  extern __shared__ __align__(16) unsigned char sraw_[];
  R* sx = reinterpret_cast<R*>(sraw_);  // [7][b]
  __shared__ int src[7];
  for (int e = blockIdx.x; e < ne; e += gridDim.x) {
    if (threadIdx.x < 7) src[threadIdx.x] = threadIdx.x == 0 ? e : nbr[e * 6 + threadIdx.x - 1];
    __syncthreads();
    for (int t = threadIdx.x; t < 7 * b; t += blockDim.x) {
      const int s = t / b, c = t - s * b;
      sx[t] = src[s] >= 0 ? x[(size_t)src[s] * b + c] : R(0);
    }
    __syncthreads();
    for (int r = threadIdx.x; r < b; r += blockDim.x) {
      R acc = R(0);
      for (int s = 0; s < 7; ++s) {
        if (src[s] < 0) continue;  // a wall
        const int opp = s == 0 ? 0 : ((s & 1) ? s + 1 : s - 1);
        const R* blk = B + ((size_t)src[s] * 7 + opp) * b * b + (size_t)r * b;  // column r of that block
        for (int c = 0; c < b; ++c) acc += blk[c] * sx[s * b + c];
      }
      y[(size_t)e * b + r] = alpha * acc + (beta == R(0) ? R(0) : beta * y[(size_t)e * b + r]);
    }
    __syncthreads();
  }
}

// x[e] = x[e] + omega * D[e]^-1 (g[e] - Gx[e]) with the LU factors of D[e]
// (Gx == nullptr: Gx = 0; x_zero: the old x is 0). One warp per element: the
// residual is gathered in row order pi into shared memory, then forward substitution
// with the unit-lower L and backward substitution with U (1/U_kk stored on the
// diagonal), both along contiguous columns.
constexpr int kApplyWarps = 4;
template <class R>
__global__ void __launch_bounds__(32 * kApplyWarps) bj_update_kernel(int ne, int b, const R* LU, const int* perm,
                                                                    const R* g, const R* Gx, R omega, int x_zero,
                                                                    R* x) {
  extern __shared__ __align__(16) unsigned char sraw_[];
  R* sz = reinterpret_cast<R*>(sraw_);  // [warps][b]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  R* z = sz + warp * b;
  for (int e = blockIdx.x * kApplyWarps + warp; e < ne; e += gridDim.x * kApplyWarps) {
    const int* pi = perm + (size_t)e * b;
    const R* ge = g + (size_t)e * b;
    const R* gx = Gx ? Gx + (size_t)e * b : nullptr;
    for (int i = lane; i < b; i += 32) {
      const int r = pi[i];
      z[i] = ge[r] - (gx ? gx[r] : R(0));
    }
    __syncwarp();
    const R* M = LU + (size_t)e * b * b;
    for (int j = 0; j < b; ++j) {  // z <- L^-1 z
      const R zj = z[j];
      const R* col = M + (size_t)j * b;
      for (int i = j + 1 + lane; i < b; i += 32) z[i] = fma(-col[i], zj, z[i]);
      __syncwarp();
    }
    for (int j = b - 1; j >= 0; --j) {  // z <- U^-1 z
      const R* col = M + (size_t)j * b;
      const R zj = z[j] * col[j];
      __syncwarp();
      if (lane == 0) z[j] = zj;
      for (int i = lane; i < j; i += 32) z[i] = fma(-col[i], zj, z[i]);
      __syncwarp();
    }
    R* xe = x + (size_t)e * b;
    for (int i = lane; i < b; i += 32) xe[i] = (x_zero ? R(0) : xe[i]) + omega * z[i];
    __syncwarp();
  }
}

static int grid_for(const Handle* h, long long work) {
  long long g = (long long)h->nsm * 8;
  if (g > work) g = work;
  return g < 1 ? 1 : (int)g;
}

static int apply_grid(const Handle* h) {
  long long g = (h->ne + kApplyWarps - 1) / kApplyWarps;
  const long long cap = (long long)h->nsm * 16;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

static int run_bsr(Handle* h, int lvl, double alpha, const double* x, double beta, double* y, cudaStream_t st) {
  const Level& L = h->lev[lvl];
  const int rc = staged_bsr<double>(h, lvl, L.Bsr, alpha, x, beta, y, st);
  if (rc >= 0) return rc;  // -1: the blocks do not fit the staged kernel
  bsr_kernel<double><<<grid_for(h, h->ne), 128, sizeof(double) * 7 * L.b, st>>>(h->ne, L.b, h->nbr, L.Bsr, alpha, x, beta, y);
  DG_LAUNCH_CHECK(h);
  return DG_OK;
}

int level_matvec(Handle* h, int lvl, const double* x, double* y, cudaStream_t st) {
  if (lvl == 0) return op_tangent(h, x, y, st);
  return run_bsr(h, lvl, 1.0, x, 0.0, y, st);
}

// sweeps of x <- x + omega D^-1 (g - G x) on level lvl; x_zero: the initial x is 0
static int jacobi_sweeps(Handle* h, int lvl, const double* g, double* x, int sweeps, double omega, bool x_zero,
                         cudaStream_t st) {
  Level& L = h->lev[lvl];
  const size_t smem = sizeof(double) * L.b * kApplyWarps;
  for (int s = 0; s < sweeps; ++s) {
    const bool zero = x_zero && s == 0;
    if (!zero) {
      int rc = level_matvec(h, lvl, x, L.t2, st);
      if (rc) return rc;
    }
    cudaEvent_t e0 = nullptr;
    int rc;
    if (lvl == 0 && (rc = prof_begin(h, st, &e0))) return rc;
    bj_update_kernel<double><<<apply_grid(h), 32 * kApplyWarps, smem, st>>>(h->ne, L.b, L.Dinv, L.perm, g,
                                                                    zero ? nullptr : L.t2, omega, zero ? 1 : 0, x);
    DG_LAUNCH_CHECK(h);
    if (lvl == 0) {  // algorithmic bytes: LU factors and permutation, g, Gx, old x read; x written
      const double vec = (double)h->ne * L.b * sizeof(double);
      const double bytes = (double)h->ne * L.b * ((double)L.b * sizeof(double) + sizeof(int)) +
                           vec * (2 + (zero ? 0 : 2));
      if ((rc = prof_end(h, DG_PROF_BJ64, st, e0, bytes))) return rc;
    }
  }
  if (sweeps == 0 && x_zero) DG_CUDA(h, cudaMemsetAsync(x, 0, sizeof(double) * L.n, st));
  return DG_OK;
}

// small device arrays of the GMRES smoother (offsets into h->smSmall)
constexpr int kSmH = 0;                                                     // [(its+1) * its] column-major
constexpr int kSmTmp = kSmH + (DG_SMOOTH_MAX_ITS + 1) * DG_SMOOTH_MAX_ITS;  // [its+1] dot products
constexpr int kSmHn2 = kSmTmp + DG_SMOOTH_MAX_ITS + 1;                      // [its] squared norms
constexpr int kSmBeta2 = kSmHn2 + DG_SMOOTH_MAX_ITS;                        // [1]
constexpr int kSmNy = kSmBeta2 + 1;                                         // [its] -y
constexpr int kSmTotal = kSmNy + DG_SMOOTH_MAX_ITS;

// H[col j][0..nv) (+)= src[0..nv)
__global__ void hcol_accumulate_kernel(double* Hcol, const double* src, int nv, int first) {
  const int i = threadIdx.x;
  if (i < nv) Hcol[i] = first ? src[i] : Hcol[i] + src[i];
}

// v <- v / sqrt(n2[0]) (zero when the norm vanishes)
__global__ void normalize_kernel(long long n, double* v, const double* n2) {
  const double nv = sqrt(*n2);
  const double inv = nv > 0.0 ? 1.0 / nv : 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    v[i] *= inv;
}

// Least-squares step of GMRES(its): min || beta e1 - H y || with Givens rotations, H
// upper Hessenberg with subdiagonal sqrt(hn2); writes -y (for the update x -= (-y) V).
// Stops at the first breakdown (zero subdiagonal). One thread.
__global__ void gmres_lsq_kernel(int its, const double* Hc, const double* hn2, const double* beta2, double* ny) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double H[(DG_SMOOTH_MAX_ITS + 1) * DG_SMOOTH_MAX_ITS];
  double cs[DG_SMOOTH_MAX_ITS], sn[DG_SMOOTH_MAX_ITS], s[DG_SMOOTH_MAX_ITS + 1], y[DG_SMOOTH_MAX_ITS];
  const int ld = its + 1;
  const double beta = sqrt(*beta2);
  for (int j = 0; j < its; ++j) ny[j] = 0.0;
  if (!(beta > 0.0)) return;
  int k = its;
  for (int j = 0; j < its; ++j)
    if (!(hn2[j] > 0.0)) { k = j + 1; break; }
  for (int j = 0; j < k; ++j) {
    for (int i = 0; i <= j; ++i) H[j * ld + i] = Hc[j * ld + i];
    H[j * ld + j + 1] = sqrt(hn2[j]);
  }
  for (int i = 0; i <= k; ++i) s[i] = 0.0;
  s[0] = beta;
  for (int j = 0; j < k; ++j) {
    double* c = H + j * ld;
    for (int i = 0; i < j; ++i) {
      const double t = cs[i] * c[i] + sn[i] * c[i + 1];
      c[i + 1] = -sn[i] * c[i] + cs[i] * c[i + 1];
      c[i] = t;
    }
    const double den = hypot(c[j], c[j + 1]);
    cs[j] = den > 0.0 ? c[j] / den : 1.0;
    sn[j] = den > 0.0 ? c[j + 1] / den : 0.0;
    c[j] = den;
    c[j + 1] = 0.0;
    s[j + 1] = -sn[j] * s[j];
    s[j] = cs[j] * s[j];
  }
  for (int i = k - 1; i >= 0; --i) {
    double acc = s[i];
    for (int j = i + 1; j < k; ++j) acc -= H[j * ld + i] * y[j];
    y[i] = H[i * ld + i] != 0.0 ? acc / H[i * ld + i] : 0.0;
  }
  for (int j = 0; j < k; ++j) ny[j] = -y[j];
}

static int multidot(Handle* h, long long n, int nv, const double* V, const double* w, double* hout, cudaStream_t st);

// GMRES(its) on level lvl left-preconditioned by the element block inverses, from x
// (x_zero: from 0), no restart: min ||D^-1 (g - G y)|| over y in x + K_its (Sec. 2.4.3).
static int gmres_smooth(Handle* h, int lvl, const double* g, double* x, int its, bool x_zero, cudaStream_t st) {
  Level& L = h->lev[lvl];
  const long long n = L.n;
  if (its <= 0) {
    if (x_zero) DG_CUDA(h, cudaMemsetAsync(x, 0, sizeof(double) * n, st));
    return DG_OK;
  }
  if (its > DG_SMOOTH_MAX_ITS) return fail(h, DG_ERR_ARG, "too many GMRES smoother iterations");
  if (h->smV_its[lvl] < its) {
    if (h->smV[lvl]) cudaFree(h->smV[lvl]);
    h->smV[lvl] = nullptr;
    h->smV_its[lvl] = 0;
    DG_CUDA(h, cudaMalloc((void**)&h->smV[lvl], sizeof(double) * (size_t)(its + 1) * n));
    h->smV_its[lvl] = its;
  }
  if (!h->smSmall) DG_CUDA(h, cudaMalloc((void**)&h->smSmall, sizeof(double) * kSmTotal));
  double* V = h->smV[lvl];
  double* Hc = h->smSmall + kSmH;
  double* tmp = h->smSmall + kSmTmp;
  double* hn2 = h->smSmall + kSmHn2;
  double* beta2 = h->smSmall + kSmBeta2;
  double* ny = h->smSmall + kSmNy;
  const size_t smem = sizeof(double) * L.b * kApplyWarps;
  const int ld = its + 1;
  int rc;
  // v0 = D^-1 (g - G x)
  if (!x_zero && (rc = level_matvec(h, lvl, x, L.t2, st))) return rc;
  bj_update_kernel<double><<<apply_grid(h), 32 * kApplyWarps, smem, st>>>(h->ne, L.b, L.Dinv, L.perm, g,
                                                                  x_zero ? nullptr : L.t2, 1.0, 1, V);
  DG_LAUNCH_CHECK(h);
  if ((rc = vec_norm2(h, V, n, beta2, st))) return rc;
  normalize_kernel<<<grid_for(h, n / 256 + 1), 256, 0, st>>>(n, V, beta2);
  DG_LAUNCH_CHECK(h);
  for (int j = 0; j < its; ++j) {
    double* vj = V + (size_t)j * n;
    double* w = V + (size_t)(j + 1) * n;
    if ((rc = level_matvec(h, lvl, vj, L.t2, st))) return rc;
    bj_update_kernel<double><<<apply_grid(h), 32 * kApplyWarps, smem, st>>>(h->ne, L.b, L.Dinv, L.perm, L.t2, nullptr, 1.0,
                                                                    1, w);
    DG_LAUNCH_CHECK(h);
    for (int pass = 0; pass < 2; ++pass) {
      if ((rc = multidot(h, n, j + 1, V, w, tmp, st))) return rc;
      multi_axpy_kernel<<<grid_for(h, n / 256 + 1), 256, 0, st>>>(n, j + 1, V, n, tmp, w);
      DG_LAUNCH_CHECK(h);
      hcol_accumulate_kernel<<<1, 64, 0, st>>>(Hc + (size_t)j * ld, tmp, j + 1, pass == 0 ? 1 : 0);
      DG_LAUNCH_CHECK(h);
    }
    if ((rc = vec_norm2(h, w, n, hn2 + j, st))) return rc;
    normalize_kernel<<<grid_for(h, n / 256 + 1), 256, 0, st>>>(n, w, hn2 + j);
    DG_LAUNCH_CHECK(h);
  }
  gmres_lsq_kernel<<<1, 32, 0, st>>>(its, Hc, hn2, beta2, ny);
  DG_LAUNCH_CHECK(h);
  if (x_zero) DG_CUDA(h, cudaMemsetAsync(x, 0, sizeof(double) * n, st));
  multi_axpy_kernel<<<grid_for(h, n / 256 + 1), 256, 0, st>>>(n, its, V, n, ny, x);
  DG_LAUNCH_CHECK(h);
  return DG_OK;
}

static int smooth(Handle* h, int lvl, const double* g, double* x, int iters, double omega, bool x_zero, int kind,
                  cudaStream_t st) {
  if (kind == DG_SMOOTH_GMRES) return gmres_smooth(h, lvl, g, x, iters, x_zero, st);
  return jacobi_sweeps(h, lvl, g, x, iters, omega, x_zero, st);
}

static int restrict_to(Handle* h, int lvl, const double* xf, double* xc, cudaStream_t st) {
  const Level &F = h->lev[lvl], &C = h->lev[lvl + 1];
  restrict_kernel<double><<<grid_for(h, C.n / 64 + 1), 256, 0, st>>>(h->ne, F.nb, C.nb, xf, xc);
  DG_LAUNCH_CHECK(h);
  return DG_OK;
}
static int prolong_add(Handle* h, int lvl, const double* xc, double* xf, cudaStream_t st) {
  const Level &F = h->lev[lvl], &C = h->lev[lvl + 1];
  prolong_add_kernel<double><<<grid_for(h, C.n / 64 + 1), 256, 0, st>>>(h->ne, F.nb, C.nb, xc, xf);
  DG_LAUNCH_CHECK(h);
  return DG_OK;
}

// a = (c.x)/(c.c) for the constant-pressure vector c (c_e = sqrt|K_e| = sqrt(8) s_e on the
// pressure mode 0); one block, fixed summation order
__global__ void __launch_bounds__(1024) pressure_dot_kernel(int ne, int nb, const double* geo, const double* x,
                                                            double* a) {
  __shared__ double sn[1024], sd[1024];
  double num = 0.0, den = 0.0;
  for (int e = threadIdx.x; e < ne; e += blockDim.x) {
    const double c = sqrt(8.0) * geo[(size_t)e * kGeo + 3];
    num += c * x[(size_t)e * 4 * nb + 3 * nb];
    den += c * c;
  }
  sn[threadIdx.x] = num;
  sd[threadIdx.x] = den;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sn[threadIdx.x] += sn[threadIdx.x + o];
      sd[threadIdx.x] += sd[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *a = sd[0] > 0.0 ? sn[0] / sd[0] : 0.0;
}
__global__ void pressure_sub_kernel(int ne, int nb, const double* geo, const double* a, double* x) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < ne) x[(size_t)e * 4 * nb + 3 * nb] -= *a * sqrt(8.0) * geo[(size_t)e * kGeo + 3];
}

// copy the coarsest-level right-hand side into the recording buffer (dg_record_coarse)
static int record_coarse(Handle* h, const double* g, cudaStream_t st) {
  if (!h->rec_buf || h->rec_count >= h->rec_cap) return DG_OK;
  const long long n = h->lev[h->nlev - 1].n;
  DG_CUDA(h, cudaMemcpyAsync(h->rec_buf + (size_t)h->rec_count * n, g, sizeof(double) * n, cudaMemcpyDeviceToDevice,
                             st));
  ++h->rec_count;
  return DG_OK;
}
static int record_coarse_f(Handle* h, const float* g, cudaStream_t st) {
  if (!h->rec_buf || h->rec_count >= h->rec_cap) return DG_OK;
  const long long n = h->lev[h->nlev - 1].n;
  convert_kernel<float, double><<<grid_for(h, n / 256 + 1), 256, 0, st>>>(n, g, h->rec_buf + (size_t)h->rec_count * n);
  DG_LAUNCH_CHECK(h);
  ++h->rec_count;
  return DG_OK;
}

// The coarsest-level SOLVE of the cycles (Sec. 2.4.3): smoother iterations from zero, GMRES
// left-preconditioned by the element block inverses (restarted every DG_SMOOTH_MAX_ITS), or
// the learned correction followed by smoother iterations. x = 0 on entry is not assumed.
static int coarse_solve(Handle* h, const double* g, double* x, const dg_solve_opts& o, cudaStream_t st) {
  const int Lc = h->nlev - 1;
  int rc;
  if ((rc = record_coarse(h, g, st))) return rc;
  if (o.coarse_solver == DG_COARSE_LEARNED) {
    if ((rc = learned_coarse<double>(h, g, x, false, st))) return rc;
    return smooth(h, Lc, g, x, o.coarse_sweeps, o.omega, false, o.smoother, st);
  }
  if (o.coarse_solver == DG_COARSE_LEARNED_ITER) {  // x <- x + N(g - G x)
    Level& C = h->lev[Lc];
    if ((rc = learned_coarse<double>(h, g, x, false, st))) return rc;
    for (int it = 0; it < o.coarse_sweeps; ++it) {
      if ((rc = run_bsr(h, Lc, 1.0, x, 0.0, C.t2, st))) return rc;
      axpby_kernel<double><<<grid_for(h, C.n / 256 + 1), 256, 0, st>>>(C.n, 1.0, g, -1.0, C.t2);
      DG_LAUNCH_CHECK(h);
      if ((rc = learned_coarse<double>(h, C.t2, x, true, st))) return rc;
    }
    return DG_OK;
  }
  if (o.coarse_solver == DG_COARSE_GMRES) {
    if (o.coarse_sweeps == 0) return gmres_smooth(h, Lc, g, x, 0, true, st);
    for (int done = 0; done < o.coarse_sweeps; done += DG_SMOOTH_MAX_ITS) {
      const int c = std::min(DG_SMOOTH_MAX_ITS, o.coarse_sweeps - done);
      if ((rc = gmres_smooth(h, Lc, g, x, c, done == 0, st))) return rc;
    }
    return DG_OK;
  }
  return smooth(h, Lc, g, x, o.coarse_sweeps, o.omega, true, o.smoother, st);
}

// MG_V(l, g, x) of Algorithm 2 (x in/out; x_zero: the incoming x is 0).
// Level l >= 1 keeps its right-hand side in t0 and its iterate in t1; t2 is scratch.
static int mg_v(Handle* h, int l, const double* g, double* x, bool x_zero, const dg_solve_opts& o, cudaStream_t st) {
  int rc;
  const int Lc = h->nlev - 1;
  if (l == Lc) return coarse_solve(h, g, x, o, st);
  if ((rc = smooth(h, l, g, x, o.pre_sweeps, o.omega, x_zero, o.smoother, st))) return rc;
  Level& L = h->lev[l];
  Level& C = h->lev[l + 1];
  const bool xz = x_zero && o.pre_sweeps == 0;
  if (xz) {
    if ((rc = restrict_to(h, l, g, C.t0, st))) return rc;
  } else {
    if ((rc = level_matvec(h, l, x, L.t2, st))) return rc;
    axpby_kernel<double><<<grid_for(h, L.n / 256 + 1), 256, 0, st>>>(L.n, 1.0, g, -1.0, L.t2);  // t2 = g - G x
    DG_LAUNCH_CHECK(h);
    if ((rc = restrict_to(h, l, L.t2, C.t0, st))) return rc;
  }
  if ((rc = mg_v(h, l + 1, C.t0, C.t1, true, o, st))) return rc;
  if (xz) DG_CUDA(h, cudaMemsetAsync(x, 0, sizeof(double) * L.n, st));
  if ((rc = prolong_add(h, l, C.t1, x, st))) return rc;
  return smooth(h, l, g, x, o.post_sweeps, o.omega, false, o.smoother, st);
}

// MG_full(l, g, 0) of Algorithm 3 (x output).
static int mg_full(Handle* h, int l, const double* g, double* x, const dg_solve_opts& o, cudaStream_t st) {
  int rc;
  const int Lc = h->nlev - 1;
  if (l == Lc) return coarse_solve(h, g, x, o, st);
  Level& L = h->lev[l];
  Level& C = h->lev[l + 1];
  // g_{l+1} = I g_l; w_{l+1} = MG_full(l+1, g_{l+1}); keep them in the coarse level's t0/t1
  if ((rc = restrict_to(h, l, g, C.t0, st))) return rc;
  if ((rc = mg_full(h, l + 1, C.t0, C.t1, o, st))) return rc;
  DG_CUDA(h, cudaMemsetAsync(x, 0, sizeof(double) * L.n, st));
  if ((rc = prolong_add(h, l, C.t1, x, st))) return rc;  // w_hat_l = I w_{l+1}
  // d_l = g - G w_hat_l ; e_l = MG_V(l, d_l, 0) ; x = w_hat + e
  if ((rc = level_matvec(h, l, x, L.t2, st))) return rc;
  axpby_kernel<double><<<grid_for(h, L.n / 256 + 1), 256, 0, st>>>(L.n, 1.0, g, -1.0, L.t2);
  DG_LAUNCH_CHECK(h);
  // The V-cycle below uses t2 as scratch on this level, so d_l moves out of it. On the fine
  // level t0/t1 are free here; on coarse levels they hold this level's (g, x), so the fine
  // finite-difference scratch of the handle (not in use during a preconditioner cycle) serves.
  double* d = l == 0 ? L.t1 : h->fd_w;
  double* e = l == 0 ? L.t0 : h->fd_f;
  DG_CUDA(h, cudaMemcpyAsync(d, L.t2, sizeof(double) * L.n, cudaMemcpyDeviceToDevice, st));
  if ((rc = mg_v(h, l, d, e, true, o, st))) return rc;
  axpby_kernel<double><<<grid_for(h, L.n / 256 + 1), 256, 0, st>>>(L.n, 1.0, e, 1.0, x);
  DG_LAUNCH_CHECK(h);
  return DG_OK;
}

// ------------------------------------------------------ FP32 preconditioner cycle
// FP32 copies of the linearisation cache (for the FP32 operator), explicit FP32 inverses of the
// element blocks
// and block-sparse coarse operators; refreshed after every linearisation / assembly.
int prepare_lin_fp32(Handle* h, cudaStream_t st) {
  if (h->lin_f_ready) return DG_OK;
  const int ne = h->ne;
  const long long nu = (long long)ne * 3 * h->tab.nq, nf = (long long)(3 * ne + h->nbf) * h->tab.nqf * 32;
  convert_kernel<double, float><<<grid_for(h, nu / 256 + 1), 256, 0, st>>>(nu, h->ubar, h->ubar_f);
  DG_LAUNCH_CHECK(h);
  convert_kernel<double, float><<<grid_for(h, nf / 256 + 1), 256, 0, st>>>(nf, h->dFlux, h->dFlux_f);
  DG_LAUNCH_CHECK(h);
  if (int rc = tc_prepare_lin(h, st)) return rc;  // scales of the tensor-core volume pass
  h->lin_f_ready = true;
  return DG_OK;
}

static int prepare_fp32(Handle* h, cudaStream_t st) {
  const int ne = h->ne;
  int rc;
  if ((rc = prepare_lin_fp32(h, st))) return rc;
  if (!h->asm_f_ready) {
    if (!h->asm64_ready) return fail(h, DG_ERR_STATE, "no assembled preconditioner");
    for (int l = 0; l < h->nlev; ++l) {
      Level& L = h->lev[l];
      const long long nbb = (long long)ne * L.b * L.b;
      if (!L.LUf) DG_CUDA(h, cudaMalloc((void**)&L.LUf, sizeof(float) * nbb));
      if (!L.t0f) DG_CUDA(h, cudaMalloc((void**)&L.t0f, sizeof(float) * L.n));
      if (!L.t1f) DG_CUDA(h, cudaMalloc((void**)&L.t1f, sizeof(float) * L.n));
      if (!L.t2f) DG_CUDA(h, cudaMalloc((void**)&L.t2f, sizeof(float) * L.n));
      convert_kernel<double, float><<<grid_for(h, nbb / 256 + 1), 256, 0, st>>>(nbb, L.Dblk, L.LUf);
      DG_LAUNCH_CHECK(h);
      if (l >= 1) {
        if (!L.Bsrf) DG_CUDA(h, cudaMalloc((void**)&L.Bsrf, sizeof(float) * nbb * 7));
        convert_kernel<double, float><<<grid_for(h, 7 * nbb / 256 + 1), 256, 0, st>>>(7 * nbb, L.Bsr, L.Bsrf);
        DG_LAUNCH_CHECK(h);
      }
    }
    if (int rc2 = invert_levels_f32(h, st, h->status)) return rc2;  // the blocks (rounded) -> explicit inverses
    h->asm_f_ready = true;
  }
  return DG_OK;
}

// the FP32 cycles with tensor-core volume contractions store their blocks as the H16 / BF16 cycles do
static int storage_of(int precision) {
  return precision == DG_PRECOND_FP32_H16_TC ? DG_PRECOND_FP32_H16
         : precision == DG_PRECOND_FP32_BF16_TC ? DG_PRECOND_FP32_BF16 : precision;
}
static int tc_of(int precision) {
  return precision == DG_PRECOND_FP32_H16_TC ? 1 : precision == DG_PRECOND_FP32_BF16_TC ? 2 : 0;
}
static bool is16(int precision) {
  const int s = storage_of(precision);
  return s == DG_PRECOND_FP32_H16 || s == DG_PRECOND_FP32_BF16;
}

// y = G_lvl x in the FP32 cycle; `precision` (the cycle's) says how the blocks are stored and
// whether the fine level's volume contractions run on the tensor cores
static int level_matvec_f(Handle* h, int lvl, const float* x, float* y, int precision, cudaStream_t st) {
  if (lvl == 0) return op_tangent_f32(h, x, y, tc_of(precision), st);
  const Level& L = h->lev[lvl];
  const int storage = storage_of(precision);
  if (is16(storage)) {
    const int r16 = bsr16_f(h, lvl, storage, 1.0f, x, 0.0f, y, st);
    if (r16 >= 0) return r16;
    return fail(h, DG_ERR_ARG, "block size unsuited to the 16-bit block-sparse product");
  }
  const int rc = staged_bsr<float>(h, lvl, L.Bsrf, 1.0f, x, 0.0f, y, st);
  if (rc >= 0) return rc;
  bsr_kernel<float><<<grid_for(h, h->ne), 128, sizeof(float) * 7 * L.b, st>>>(h->ne, L.b, h->nbr, L.Bsrf, 1.0f, x,
                                                                               0.0f, y);
  DG_LAUNCH_CHECK(h);
  return DG_OK;
}

static int jacobi_sweeps_f(Handle* h, int lvl, const float* g, float* x, int sweeps, float omega, bool x_zero,
                           int storage,
                           cudaStream_t st) {
  Level& L = h->lev[lvl];
  for (int s = 0; s < sweeps; ++s) {
    const bool zero = x_zero && s == 0;
    int rc;
    if (!zero && (rc = level_matvec_f(h, lvl, x, L.t2f, storage, st))) return rc;
    rc = staged_jacobi_f(h, lvl, g, zero ? nullptr : L.t2f, omega, zero, x, storage_of(storage), st);
    if (rc < 0) return fail(h, DG_ERR_ARG, "element block too large for the FP32 smoother");
    if (rc) return rc;
  }
  if (sweeps == 0 && x_zero) DG_CUDA(h, cudaMemsetAsync(x, 0, sizeof(float) * L.n, st));
  return DG_OK;
}

// MG_V(l, g, x) of Algorithm 2 in FP32 (block-Jacobi smoothing); level l >= 1 keeps its
// right-hand side in t0f and its iterate in t1f, t2f is scratch.
static int mg_v_f(Handle* h, int l, const float* g, float* x, bool x_zero, const dg_solve_opts& o, cudaStream_t st) {
  int rc;
  const int Lc = h->nlev - 1;
  const float om = (float)o.omega;
  if (l == Lc) {
    if ((rc = record_coarse_f(h, g, st))) return rc;
    if (o.coarse_solver == DG_COARSE_LEARNED) {
      if ((rc = learned_coarse<float>(h, g, x, false, st))) return rc;
      return jacobi_sweeps_f(h, l, g, x, o.coarse_sweeps, om, false, o.precision, st);
    }
    if (o.coarse_solver == DG_COARSE_LEARNED_ITER) {  // x <- x + N(g - G x)
      Level& C = h->lev[l];
      if ((rc = learned_coarse<float>(h, g, x, false, st))) return rc;
      for (int it = 0; it < o.coarse_sweeps; ++it) {
        if ((rc = level_matvec_f(h, l, x, C.t2f, o.precision, st))) return rc;
        axpby_kernel<float><<<grid_for(h, C.n / 256 + 1), 256, 0, st>>>(C.n, 1.0f, g, -1.0f, C.t2f);
        DG_LAUNCH_CHECK(h);
        if ((rc = learned_coarse<float>(h, C.t2f, x, true, st))) return rc;
      }
      return DG_OK;
    }
    return jacobi_sweeps_f(h, l, g, x, o.coarse_sweeps, om, true, o.precision, st);
  }
  if ((rc = jacobi_sweeps_f(h, l, g, x, o.pre_sweeps, om, x_zero, o.precision, st))) return rc;
  Level& L = h->lev[l];
  Level& C = h->lev[l + 1];
  const bool xz = x_zero && o.pre_sweeps == 0;
  if (xz) {
    restrict_kernel<float><<<grid_for(h, C.n / 64 + 1), 256, 0, st>>>(h->ne, L.nb, C.nb, g, C.t0f);
    DG_LAUNCH_CHECK(h);
  } else {
    if ((rc = level_matvec_f(h, l, x, L.t2f, o.precision, st))) return rc;
    axpby_kernel<float><<<grid_for(h, L.n / 256 + 1), 256, 0, st>>>(L.n, 1.0f, g, -1.0f, L.t2f);
    DG_LAUNCH_CHECK(h);
    restrict_kernel<float><<<grid_for(h, C.n / 64 + 1), 256, 0, st>>>(h->ne, L.nb, C.nb, L.t2f, C.t0f);
    DG_LAUNCH_CHECK(h);
  }
  if ((rc = mg_v_f(h, l + 1, C.t0f, C.t1f, true, o, st))) return rc;
  if (xz) DG_CUDA(h, cudaMemsetAsync(x, 0, sizeof(float) * L.n, st));
  prolong_add_kernel<float><<<grid_for(h, C.n / 64 + 1), 256, 0, st>>>(h->ne, L.nb, C.nb, C.t1f, x);
  DG_LAUNCH_CHECK(h);
  return jacobi_sweeps_f(h, l, g, x, o.post_sweeps, om, false, o.precision, st);
}

// z = MG_V(v) with the cycle in FP32: v rounded to FP32, the result widened to FP64.
static int vcycle_fp32(Handle* h, const dg_solve_opts& o, const double* v, double* z, cudaStream_t st) {
  int rc;
  if ((rc = prepare_fp32(h, st))) return rc;
  if (is16(o.precision) && (rc = prepare_blocks16(h, storage_of(o.precision), st))) return rc;
  if (tc_of(o.precision) && (rc = tc_prepare_tables(h))) return rc;
  Level& L0 = h->lev[0];
  convert_kernel<double, float><<<grid_for(h, L0.n / 256 + 1), 256, 0, st>>>(L0.n, v, L0.t0f);
  DG_LAUNCH_CHECK(h);
  if ((rc = mg_v_f(h, 0, L0.t0f, L0.t1f, true, o, st))) return rc;
  convert_kernel<float, double><<<grid_for(h, L0.n / 256 + 1), 256, 0, st>>>(L0.n, L0.t1f, z);
  DG_LAUNCH_CHECK(h);
  return DG_OK;
}

static bool is_learned(int coarse_solver) {
  return coarse_solver == DG_COARSE_LEARNED || coarse_solver == DG_COARSE_LEARNED_ITER;
}

static int check_opts(Handle* h, const dg_solve_opts* o) {
  if (!o) return fail(h, DG_ERR_ARG, "null options");
  if (o->pre_sweeps < 0 || o->post_sweeps < 0 || o->coarse_sweeps < 0) return fail(h, DG_ERR_ARG, "negative sweeps");
  if (!(o->omega > 0.0 && o->omega <= 1.0)) return fail(h, DG_ERR_ARG, "omega must be in (0, 1]");
  if (o->smoother != DG_SMOOTH_JACOBI && o->smoother != DG_SMOOTH_GMRES) return fail(h, DG_ERR_ARG, "unknown smoother");
  if (o->precision != DG_PRECOND_FP64 && o->precision != DG_PRECOND_FP32 && !is16(o->precision))
    return fail(h, DG_ERR_ARG, "unknown preconditioner precision");
  if (o->precision != DG_PRECOND_FP64 && (o->smoother != DG_SMOOTH_JACOBI || o->precond == DG_PREC_FULLV))
    return fail(h, DG_ERR_ARG, "the FP32 preconditioner supports block-Jacobi smoothing in V-cycles only");
  if (o->coarse_solver != DG_COARSE_SMOOTHER && o->coarse_solver != DG_COARSE_GMRES &&
      o->coarse_solver != DG_COARSE_LEARNED && o->coarse_solver != DG_COARSE_LEARNED_ITER)
    return fail(h, DG_ERR_ARG, "unknown coarse solver");
  const bool learned = o->coarse_solver == DG_COARSE_LEARNED || o->coarse_solver == DG_COARSE_LEARNED_ITER;
  if (o->coarse_solver == DG_COARSE_GMRES && o->precision != DG_PRECOND_FP64)
    return fail(h, DG_ERR_ARG, "the GMRES coarse solver runs in the FP64 cycle only");
  if (learned) {
    if (h->nlev < 2) return fail(h, DG_ERR_ARG, "the learned coarse correction needs at least two levels");
    if (h->lev[h->nlev - 1].k != 1) return fail(h, DG_ERR_ARG, "the learned coarse correction needs k = 1 there");
    if (!h->net_ready) return fail(h, DG_ERR_STATE, "no coarse network set (dg_set_coarse_network)");
    if (o->fallback_its < 0 || (o->fallback_its > 0 && !(o->fallback_rho > 0.0 && o->fallback_rho < 1.0)))
      return fail(h, DG_ERR_ARG, "fallback_its >= 0 and fallback_rho in (0, 1) needed");
  }
  if (h->nprob > 1 && (o->smoother == DG_SMOOTH_GMRES || o->coarse_solver == DG_COARSE_GMRES || o->jvp_mode == DG_JVP_FD))
    return fail(h, DG_ERR_ARG, "GMRES smoothing, the GMRES coarse solve and FD products reduce over the whole "
                               "vector: not available on a handle of several problems");
  if (o->smoother == DG_SMOOTH_GMRES &&
      (o->pre_sweeps > DG_SMOOTH_MAX_ITS || o->post_sweeps > DG_SMOOTH_MAX_ITS || o->coarse_sweeps > DG_SMOOTH_MAX_ITS))
    return fail(h, DG_ERR_ARG, "GMRES smoother iterations above DG_SMOOTH_MAX_ITS");
  return DG_OK;
}

static int apply_prec(Handle* h, const dg_solve_opts& o, const double* v, double* z, cudaStream_t st) {
  if (o.precond == DG_PREC_NONE) {
    DG_CUDA(h, cudaMemcpyAsync(z, v, sizeof(double) * h->lev[0].n, cudaMemcpyDeviceToDevice, st));
    return DG_OK;
  }
  if (o.precision == DG_PRECOND_FP64 && !h->asm64_ready)
    return fail(h, DG_ERR_STATE, "the FP64 preconditioner needs an FP64 assembly");
  if (o.precond == DG_PREC_VCYCLE) {
    if (o.precision != DG_PRECOND_FP64) return vcycle_fp32(h, o, v, z, st);
    return mg_v(h, 0, v, z, true, o, st);
  }
  if (o.precond == DG_PREC_FULLV) {
    if (h->nlev > 1 && h->lev[1].n > h->lev[0].n) return fail(h, DG_ERR_ARG, "bad level sizes");
    return mg_full(h, 0, v, z, o, st);
  }
  return fail(h, DG_ERR_ARG, "unknown preconditioner");
}

static int outer_matvec(Handle* h, const dg_solve_opts& o, const double* x, double* y, cudaStream_t st) {
  return o.jvp_mode == DG_JVP_FD ? op_fd(h, x, y, st) : op_tangent(h, x, y, st);
}

// hcol[0..nv) = V[0..nv)^T w (device), in chunks of 8 vectors
static int multidot(Handle* h, long long n, int nv, const double* V, const double* w, double* hout, cudaStream_t st) {
  for (int j0 = 0; j0 < nv; j0 += 8) {
    const int c = nv - j0 < 8 ? nv - j0 : 8;
    multidot_partial_kernel<<<kRedBlocks, 256, 0, st>>>(n, c, V + (size_t)j0 * n, n, w, h->red, 8);
    DG_LAUNCH_CHECK(h);
    reduce_partials_kernel<<<1, 256, 0, st>>>(kRedBlocks, c, 8, h->red, hout + j0);
    DG_LAUNCH_CHECK(h);
  }
  return DG_OK;
}

static int ensure_krylov(Handle* h, int m) {
  if (h->kry_m >= m) return DG_OK;
  if (h->V) cudaFree(h->V);
  if (h->Z) cudaFree(h->Z);
  if (h->hcol) cudaFree(h->hcol);
  if (h->hcol_host) cudaFreeHost(h->hcol_host);
  h->V = h->Z = h->hcol = h->hcol_host = nullptr;
  h->kry_m = 0;
  const long long n0 = h->lev[0].n;
  DG_CUDA(h, cudaMalloc((void**)&h->V, sizeof(double) * (size_t)(m + 1) * n0));
  DG_CUDA(h, cudaMalloc((void**)&h->Z, sizeof(double) * (size_t)m * n0));
  DG_CUDA(h, cudaMalloc((void**)&h->hcol, sizeof(double) * (m + 8)));
  DG_CUDA(h, cudaMallocHost((void**)&h->hcol_host, sizeof(double) * (m + 8)));
  h->kry_m = m;
  return DG_OK;
}

static int fgmres(Handle* h, const double* g, double* x, const dg_solve_opts& o, dg_solve_info* info, cudaStream_t st) {
  const long long n = h->lev[0].n;
  const int m = o.restart;
  int rc;
  if ((rc = ensure_krylov(h, m))) return rc;
  double* V = h->V;
  double* Z = h->Z;
  double* r = h->lev[0].t0;  // t0/t1 of level 0 are free during the solve (the smoothers use t2)
  double* tmp = h->lev[0].t1;
  auto norm = [&](const double* v, double* out) -> int {
    int c = vec_norm2(h, v, n, h->red_out, st);
    if (c) return c;
    DG_CUDA(h, cudaMemcpyAsync(h->hcol_host, h->red_out, sizeof(double), cudaMemcpyDeviceToHost, st));
    DG_CUDA(h, cudaStreamSynchronize(st));
    *out = std::sqrt(h->hcol_host[0]);
    return DG_OK;
  };
  // r = g - G x0
  if (o.x0_is_zero) {
    DG_CUDA(h, cudaMemsetAsync(x, 0, sizeof(double) * n, st));
    DG_CUDA(h, cudaMemcpyAsync(r, g, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  } else {
    if ((rc = outer_matvec(h, o, x, tmp, st))) return rc;
    DG_CUDA(h, cudaMemcpyAsync(r, g, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    if ((rc = launch_axpby(h, n, -1.0, tmp, 1.0, r, st))) return rc;
  }
  double beta0;
  if ((rc = norm(r, &beta0))) return rc;
  if (!std::isfinite(beta0)) return fail(h, DG_ERR_NONFINITE, "non-finite right-hand side or initial residual");
  int its = 0;
  const int limit = o.fixed_its > 0 ? o.fixed_its : o.maxit;
  double est = beta0;
  bool converged = beta0 == 0.0;
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), s(m + 1), y(m);
  // the preconditioner in use: the learned coarse correction is dropped for the rest of the
  // solve when it stalls the residual or produces a non-finite vector
  dg_solve_opts cur = o;
  int fallback_at = -1;
  while (!converged && its < limit) {
    double beta;
    if ((rc = norm(r, &beta))) return rc;
    if (beta == 0.0) { converged = true; break; }
    if ((rc = launch_axpby(h, n, 1.0 / beta, r, 0.0, V, st))) return rc;
    std::fill(H.begin(), H.end(), 0.0);
    std::fill(s.begin(), s.end(), 0.0);
    s[0] = beta;
    const int mm = std::min(m, limit - its);
    int jdone = 0;
    for (int j = 0; j < mm; ++j) {
      double* vj = V + (size_t)j * n;
      double* zj = Z + (size_t)j * n;
      double* w = V + (size_t)(j + 1) * n;
      double hn = 0.0;
      for (int attempt = 0;; ++attempt) {
        if ((rc = apply_prec(h, cur, vj, zj, st))) return rc;
        if ((rc = outer_matvec(h, o, zj, w, st))) return rc;
        for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = 0.0;
        // classical Gram-Schmidt, twice
        for (int pass = 0; pass < 2; ++pass) {
          if ((rc = multidot(h, n, j + 1, V, w, h->hcol, st))) return rc;
          multi_axpy_kernel<<<grid_for(h, n / 256 + 1), 256, 0, st>>>(n, j + 1, V, n, h->hcol, w);
          DG_LAUNCH_CHECK(h);
          DG_CUDA(h, cudaMemcpyAsync(h->hcol_host, h->hcol, sizeof(double) * (j + 1), cudaMemcpyDeviceToHost, st));
          DG_CUDA(h, cudaStreamSynchronize(st));
          for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] += h->hcol_host[i];
        }
        if ((rc = norm(w, &hn))) return rc;
        bool finite = std::isfinite(hn);
        for (int i = 0; i <= j; ++i) finite = finite && std::isfinite(H[(size_t)i * m + j]);
        if (finite) break;
        if (attempt == 0 && is_learned(cur.coarse_solver)) {  // redo with the plain cycle
          cur.coarse_solver = DG_COARSE_SMOOTHER;
          fallback_at = its;
          continue;
        }
        return fail(h, DG_ERR_NONFINITE, "non-finite Arnoldi vector");
      }
      H[(size_t)(j + 1) * m + j] = hn;
      if (hn > 0.0 && (rc = launch_axpby(h, n, 1.0 / hn, w, 0.0, w, st))) return rc;
      for (int i = 0; i < j; ++i) {
        const double t = cs[i] * H[(size_t)i * m + j] + sn[i] * H[(size_t)(i + 1) * m + j];
        H[(size_t)(i + 1) * m + j] = -sn[i] * H[(size_t)i * m + j] + cs[i] * H[(size_t)(i + 1) * m + j];
        H[(size_t)i * m + j] = t;
      }
      const double den = std::hypot(H[(size_t)j * m + j], H[(size_t)(j + 1) * m + j]);
      cs[j] = H[(size_t)j * m + j] / den;
      sn[j] = H[(size_t)(j + 1) * m + j] / den;
      H[(size_t)j * m + j] = den;
      H[(size_t)(j + 1) * m + j] = 0.0;
      s[j + 1] = -sn[j] * s[j];
      s[j] = cs[j] * s[j];
      ++its;
      jdone = j + 1;
      est = std::fabs(s[j + 1]);
      if (is_learned(cur.coarse_solver) && o.fallback_its > 0 && its >= o.fallback_its &&
          est > std::pow(o.fallback_rho, (double)its) * beta0) {
        cur.coarse_solver = DG_COARSE_SMOOTHER;
        fallback_at = its;
      }
      if (o.fixed_its <= 0 && est <= o.rtol * beta0) break;
      if (hn == 0.0) break;
    }
    // y = H^-1 s (upper triangular), x += Z y
    for (int i = jdone - 1; i >= 0; --i) {
      double acc = s[i];
      for (int k = i + 1; k < jdone; ++k) acc -= H[(size_t)i * m + k] * y[k];
      y[i] = acc / H[(size_t)i * m + i];
    }
    for (int i = 0; i < jdone; ++i)
      if ((rc = launch_axpby(h, n, y[i], Z + (size_t)i * n, 1.0, x, st))) return rc;
    // true residual
    if ((rc = outer_matvec(h, o, x, tmp, st))) return rc;
    DG_CUDA(h, cudaMemcpyAsync(r, g, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    if ((rc = launch_axpby(h, n, -1.0, tmp, 1.0, r, st))) return rc;
    double rn;
    if ((rc = norm(r, &rn))) return rc;
    if (o.fixed_its <= 0 && rn <= o.rtol * beta0) converged = true;
    if (info) info->true_relres = beta0 > 0 ? rn / beta0 : 0.0;
  }
  if (info) {
    info->its = its;
    info->r0 = beta0;
    info->relres_est = beta0 > 0 ? est / beta0 : 0.0;
    if (beta0 == 0.0) info->true_relres = 0.0;
    info->rho = (its > 0 && info->true_relres > 0) ? std::exp(std::log(info->true_relres) / its) : 0.0;
    info->status = (converged || o.fixed_its > 0) ? DG_OK : DG_ERR_NOT_CONVERGED;
    info->fallback_at = fallback_at;
  }
  if (!converged && o.fixed_its <= 0) return fail(h, DG_ERR_NOT_CONVERGED, "FGMRES did not reach the tolerance");
  return DG_OK;
}

// Entry points of the preconditioner for the batched solver (dg_batch.cu).
int solve_opts_check(Handle* h, const dg_solve_opts* o) { return check_opts(h, o); }

int precond_prepare(Handle* h, const dg_solve_opts& o, cudaStream_t st) {
  if (o.precond == DG_PREC_NONE) return DG_OK;
  if (o.precision == DG_PRECOND_FP64) {
    if (!h->asm64_ready) return fail(h, DG_ERR_STATE, "the FP64 preconditioner needs an FP64 assembly");
    return DG_OK;
  }
  int rc;
  if ((rc = prepare_fp32(h, st))) return rc;
  if (is16(o.precision) && (rc = prepare_blocks16(h, storage_of(o.precision), st))) return rc;
  if (tc_of(o.precision) && (rc = tc_prepare_tables(h))) return rc;
  return DG_OK;
}

int precond_apply(Handle* h, const dg_solve_opts& o, const double* v, double* z, cudaStream_t st) {
  return apply_prec(h, o, v, z, st);
}

}  // namespace dg

using namespace dg;

extern "C" {

int pmg_restrict(dg_handle* hh, int lvl, const double* xf, double* xc, void* stream) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return DG_ERR_ARG;
  if (lvl < 0 || lvl + 1 >= h->nlev || !xf || !xc) return fail(h, DG_ERR_ARG, "bad level or pointer");
  return restrict_to(h, lvl, xf, xc, as_stream(stream));
}

int pmg_prolong(dg_handle* hh, int lvl, const double* xc, double* xf, void* stream) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return DG_ERR_ARG;
  if (lvl < 0 || lvl + 1 >= h->nlev || !xf || !xc) return fail(h, DG_ERR_ARG, "bad level or pointer");
  return prolong_add(h, lvl, xc, xf, as_stream(stream));
}

int block_jacobi_smooth(dg_handle* hh, int lvl, const double* g, double* x, int sweeps, double omega, void* stream) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return DG_ERR_ARG;
  if (lvl < 0 || lvl >= h->nlev || !g || !x || g == x) return fail(h, DG_ERR_ARG, "bad level or pointer");
  if (sweeps < 0 || !(omega > 0.0 && omega <= 1.0)) return fail(h, DG_ERR_ARG, "bad sweeps or omega");
  if (!h->asm64_ready) return fail(h, DG_ERR_STATE, "block_jacobi_smooth needs an FP64 dg_assemble first");
  return jacobi_sweeps(h, lvl, g, x, sweeps, omega, false, as_stream(stream));
}

int bsr_spmv(dg_handle* hh, int lvl, double alpha, const double* x, double beta, double* y, void* stream) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return DG_ERR_ARG;
  if (lvl < 1 || lvl >= h->nlev || !x || !y || x == y) return fail(h, DG_ERR_ARG, "bad level or pointer");
  if (!h->asm64_ready) return fail(h, DG_ERR_STATE, "bsr_spmv needs an FP64 dg_assemble first");
  return run_bsr(h, lvl, alpha, x, beta, y, as_stream(stream));
}

int bsr_spmv_t(dg_handle* hh, int lvl, double alpha, const double* x, double beta, double* y, void* stream) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return DG_ERR_ARG;
  if (lvl < 1 || lvl >= h->nlev || !x || !y || x == y) return fail(h, DG_ERR_ARG, "bad level or pointer");
  if (!h->asm64_ready) return fail(h, DG_ERR_STATE, "bsr_spmv_t needs an FP64 dg_assemble first");
  const Level& L = h->lev[lvl];
  bsr_t_kernel<double><<<grid_for(h, h->ne), 128, sizeof(double) * 7 * L.b, as_stream(stream)>>>(
      h->ne, L.b, h->nbr, L.Bsr, alpha, x, beta, y);
  DG_LAUNCH_CHECK(h);
  return DG_OK;
}

int dg_coarse_apply(dg_handle* hh, const double* d, double* x, int accumulate, void* stream) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return DG_ERR_ARG;
  if (!d || !x || d == x) return fail(h, DG_ERR_ARG, "bad pointer");
  if (h->nlev < 2 || h->lev[h->nlev - 1].k != 1)
    return fail(h, DG_ERR_ARG, "the learned coarse correction needs at least two levels and k = 1 on the last");
  return learned_coarse<double>(h, d, x, accumulate != 0, as_stream(stream));
}

int pmg_vcycle(dg_handle* hh, const double* g, double* x, const dg_solve_opts* opts, void* stream) {
  const dg::NvtxRange nvtx_range_("pmg_vcycle");
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return DG_ERR_ARG;
  int rc = check_opts(h, opts);
  if (rc) return rc;
  if (!g || !x || g == x) return fail(h, DG_ERR_ARG, "bad pointer");
  if (!h->assembled) return fail(h, DG_ERR_STATE, "pmg_vcycle needs dg_assemble first");
  if (opts->precision != DG_PRECOND_FP64) return vcycle_fp32(h, *opts, g, x, as_stream(stream));
  if (!h->asm64_ready) return fail(h, DG_ERR_STATE, "the FP64 cycle needs an FP64 assembly");
  return mg_v(h, 0, g, x, true, *opts, as_stream(stream));
}

int pmg_project_pressure(dg_handle* hh, int lvl, double* x, void* stream) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return DG_ERR_ARG;
  if (lvl < 0 || lvl >= h->nlev || !x) return fail(h, DG_ERR_ARG, "bad level or pointer");
  if (h->nprob > 1) return fail(h, DG_ERR_ARG, "one problem per handle only");
  cudaStream_t st = as_stream(stream);
  const Level& L = h->lev[lvl];
  pressure_dot_kernel<<<1, 1024, 0, st>>>(h->ne, L.nb, h->geo, x, h->red_out);
  DG_LAUNCH_CHECK(h);
  pressure_sub_kernel<<<(h->ne + 255) / 256, 256, 0, st>>>(h->ne, L.nb, h->geo, h->red_out, x);
  DG_LAUNCH_CHECK(h);
  return DG_OK;
}

int pmg_level_solve(dg_handle* hh, int lvl, const double* g, double* x, double rtol, int maxit, int x0_is_zero,
                    dg_solve_info* info, void* stream) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return DG_ERR_ARG;
  if (lvl < 1 || lvl >= h->nlev || !g || !x || g == x) return fail(h, DG_ERR_ARG, "bad level or pointer");
  if (h->nprob > 1) return fail(h, DG_ERR_ARG, "one problem per handle only");
  if (!(rtol > 0.0) || maxit < 1) return fail(h, DG_ERR_ARG, "bad rtol or maxit");
  if (!h->asm64_ready) return fail(h, DG_ERR_STATE, "pmg_level_solve needs an FP64 dg_assemble first");
  cudaStream_t st = as_stream(stream);
  Level& L = h->lev[lvl];
  int rc;
  // r = g - G x into t1 (t2 is the smoother's scratch); returns ||r||
  auto resnorm = [&](bool zero, double* out) -> int {
    if (zero) {
      if (int c = vec_norm2(h, g, L.n, h->red_out, st)) return c;
    } else {
      if (int c = run_bsr(h, lvl, 1.0, x, 0.0, L.t1, st)) return c;
      axpby_kernel<double><<<grid_for(h, L.n / 256 + 1), 256, 0, st>>>(L.n, 1.0, g, -1.0, L.t1);
      DG_LAUNCH_CHECK(h);
      if (int c = vec_norm2(h, L.t1, L.n, h->red_out, st)) return c;
    }
    double v = 0.0;
    DG_CUDA(h, cudaMemcpyAsync(&v, h->red_out, sizeof(double), cudaMemcpyDeviceToHost, st));
    DG_CUDA(h, cudaStreamSynchronize(st));
    *out = std::sqrt(v);
    return DG_OK;
  };
  double r0 = 0.0, rn = 0.0;
  if ((rc = resnorm(x0_is_zero != 0, &r0))) return rc;
  if (x0_is_zero) DG_CUDA(h, cudaMemsetAsync(x, 0, sizeof(double) * L.n, st));
  int its = 0;
  bool conv = r0 == 0.0;
  rn = r0;
  while (!conv && its < maxit) {
    const int c = std::min(DG_SMOOTH_MAX_ITS, maxit - its);
    if ((rc = gmres_smooth(h, lvl, g, x, c, false, st))) return rc;
    its += c;
    if ((rc = resnorm(false, &rn))) return rc;
    if (!std::isfinite(rn)) return fail(h, DG_ERR_NONFINITE, "non-finite residual in pmg_level_solve");
    conv = rn <= rtol * r0;
  }
  if (info) {
    *info = dg_solve_info{};
    info->its = its;
    info->r0 = r0;
    info->true_relres = r0 > 0.0 ? rn / r0 : 0.0;
    info->relres_est = info->true_relres;
    info->rho = (its > 0 && info->true_relres > 0) ? std::exp(std::log(info->true_relres) / its) : 0.0;
    info->status = conv ? DG_OK : DG_ERR_NOT_CONVERGED;
    info->fallback_at = -1;
  }
  return conv ? DG_OK : fail(h, DG_ERR_NOT_CONVERGED, "pmg_level_solve did not reach the tolerance");
}

int fgmres_solve(dg_handle* hh, const double* g, double* x, const dg_solve_opts* opts, dg_solve_info* info,
                 void* stream) {
  const dg::NvtxRange nvtx_range_("fgmres_solve");
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return DG_ERR_ARG;
  int rc = check_opts(h, opts);
  if (rc) return rc;
  if (!g || !x || g == x) return fail(h, DG_ERR_ARG, "bad pointer");
  if (h->nprob > 1) return fail(h, DG_ERR_ARG, "a handle of several problems is solved by dg_plan_solve");
  if (opts->restart < 1 || opts->restart > 64) return fail(h, DG_ERR_ARG, "restart must be in 1..64");
  if (opts->fixed_its <= 0 && (opts->maxit < 1 || !(opts->rtol > 0.0))) return fail(h, DG_ERR_ARG, "bad maxit/rtol");
  if (!h->linearized) return fail(h, DG_ERR_STATE, "fgmres_solve needs dg_set_linearization first");
  if (opts->precond != DG_PREC_NONE && !h->assembled) return fail(h, DG_ERR_STATE, "preconditioner needs dg_assemble");
  if (opts->jvp_mode != DG_JVP_TANGENT && opts->jvp_mode != DG_JVP_FD) return fail(h, DG_ERR_ARG, "bad jvp mode");
  if (info) *info = dg_solve_info{};
  return fgmres(h, g, x, *opts, info, as_stream(stream));
}

}  // extern "C"
