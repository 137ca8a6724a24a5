// Batched, device-driven flexible GMRES (Sec. 2.3, right-preconditioned by the p-multigrid
// cycles of Algorithms 2-3) for many independent problems at once, and its CUDA-graph form.
//
// A handle may hold several independent periodic boxes (dg_create_batch). Their element
// vectors are concatenated, so every element kernel of the operator and of the cycle acts on all
// of them in one launch; only the Krylov method needs to know the problems apart. Here each
// problem keeps its own Krylov space, Hessenberg matrix, Givens rotations and convergence test,
// while the problems advance in lockstep: one Arnoldi step of every still-active problem per
// step. The reductions are per problem, over fixed chunks in a fixed order, so a problem's
// numbers do not depend on the other problems of the batch. Everything that the host-driven
// solver does on the host (Givens rotations, the convergence test, the triangular solve) runs in
// small device kernels here, so that a restart cycle issues no host synchronisation. That makes
// the cycle capturable as a CUDA graph: the Arnoldi step is the body of a conditional WHILE node
// whose condition the step's last kernel sets (some problem still active and j < m). Several
// handles (for instance one per polynomial degree) become parallel branches of one graph, so a
// whole batch of uneven solves is one graph launch per restart cycle.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "dg_internal.h"

namespace dg {

constexpr int kSegThreads = 256;
// control words on the device
constexpr int kCtlJ = 0;      // Arnoldi step within the current cycle
constexpr int kCtlCond = 1;   // continue the cycle (some problem active and j < m)
constexpr int kCtlSteps = 2;  // steps executed in this solve
constexpr int kCtlDone = 3;   // every problem converged or at its iteration limit
constexpr int kCtlBad = 4;    // a non-finite Krylov quantity was met
constexpr int kCtlConv = 5;   // every problem converged
constexpr int kCtlN = 8;

struct BatchDev {
  double* H;       // [np][(m+1)*m] row i, column j at i*m + j
  double* cs;      // [np][m]
  double* sn;      // [np][m]
  double* s;       // [np][m+1]
  double* y;       // [np][m]
  double* hpass;   // [np][m+1] dots of one Gram-Schmidt pass
  double* hsum;    // [np][m+1] their sum over the two passes
  double* beta0;   // [np] initial residual norms
  double* nrm2;    // [np] squared norms (scratch)
  double* scale;   // [np] factor of the next basis vector (0 for an inactive problem)
  double* relres;  // [np] true relative residual after the last cycle
  int* jdone;      // [np] steps of the current cycle that count for the problem
  int* active;     // [np]
  int* its;        // [np] steps over the solve
  int* conv;       // [np]
  int* ctl;        // [kCtlN]
};

// ------------------------------------------------------- per-problem reductions
// part[c][v] = sum over chunk c of V_v . w for v < nv, nv = nv_fixed if > 0, else jdev[0] + 1.
__global__ void __launch_bounds__(kSegThreads) seg_dot_kernel(int nchunk, const int2* chunk, int per_e, const double* V,
                                                              long long ldv, int nv_fixed, const int* jdev,
                                                              const double* w, double* part, int ld) {
  __shared__ double red[kSegThreads / 32][8];
  const int nv = nv_fixed > 0 ? nv_fixed : jdev[0] + 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int c = blockIdx.x; c < nchunk; c += gridDim.x) {
    const long long i0 = (long long)chunk[c].x * per_e, i1 = (long long)chunk[c].y * per_e;
    for (int v0 = 0; v0 < nv; v0 += 8) {
      const int cnt = min(8, nv - v0);
      double acc[8];
#pragma unroll
      for (int v = 0; v < 8; ++v) acc[v] = 0.0;
      for (long long i = i0 + threadIdx.x; i < i1; i += kSegThreads) {
        const double wi = w[i];
#pragma unroll
        for (int v = 0; v < 8; ++v)
          if (v < cnt) acc[v] += V[(size_t)(v0 + v) * ldv + i] * wi;
      }
#pragma unroll
      for (int v = 0; v < 8; ++v) {
        double a = acc[v];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) red[warp][v] = a;
      }
      __syncthreads();
      if (threadIdx.x < cnt) {
        double t = 0.0;
        for (int q = 0; q < kSegThreads / 32; ++q) t += red[q][threadIdx.x];
        part[(size_t)c * ld + v0 + threadIdx.x] = t;
      }
      __syncthreads();
    }
  }
}

// pass[p][v] = sum of the chunk partials of problem p (fixed order); sum[p][v] = pass (first
// pass) or sum + pass. One block per problem.
__global__ void __launch_bounds__(kSegThreads) seg_reduce_kernel(const int* pchunk0, const double* part, int ld,
                                                                 int nv_fixed, const int* jdev, double* pass,
                                                                 double* sum, int accumulate, int pld) {
  const int p = blockIdx.x;
  const int c0 = pchunk0[p], c1 = pchunk0[p + 1];
  const int nv = nv_fixed > 0 ? nv_fixed : jdev[0] + 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int v = warp; v < nv; v += kSegThreads / 32) {
    double a = 0.0;
    for (int c = c0 + lane; c < c1; c += 32) a += part[(size_t)c * ld + v];
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) {
      pass[(size_t)p * pld + v] = a;
      if (sum) sum[(size_t)p * pld + v] = accumulate ? sum[(size_t)p * pld + v] + a : a;
    }
  }
}

// w <- w - sum_{v <= j} V_v coef[p][v], p the problem of the entry
__global__ void seg_axpy_kernel(long long n, int per_e, const int* elem_prob, const double* V, long long ldv,
                                const int* jdev, const double* coef, int pld, double* w) {
  const int nv = jdev[0] + 1;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double* cp = coef + (size_t)elem_prob[i / per_e] * pld;
    double acc = w[i];
    for (int v = 0; v < nv; ++v) acc -= V[(size_t)v * ldv + i] * cp[v];
    w[i] = acc;
  }
}

// ------------------------------------------------------------ Arnoldi kernels
// V_j <- src * scale[p] and vin <- the same, j = jdev[0]
__global__ void batch_normalize_kernel(long long n, int per_e, const int* elem_prob, const double* src,
                                       const double* scale, const int* jdev, double* V, double* vin) {
  double* vj = V + (size_t)jdev[0] * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double v = src[i] * scale[elem_prob[i / per_e]];
    vj[i] = v;
    vin[i] = v;
  }
}

// Z_j <- z, j = jdev[0]
__global__ void batch_store_kernel(long long n, const double* z, const int* jdev, double* Z) {
  double* zj = Z + (size_t)jdev[0] * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    zj[i] = z[i];
}

// Start of a restart cycle: beta_p = ||r_p|| (nrm2), s_p = beta_p e_1, which problems iterate.
__global__ void __launch_bounds__(1024) batch_cycle_init_kernel(int np, int m, int limit, int first, BatchDev d,
                                                                cudaGraphConditionalHandle hc, int use_cond) {
  int any = 0;
  for (int p = threadIdx.x; p < np; p += blockDim.x) {
    const double beta = sqrt(d.nrm2[p]);
    if (!isfinite(beta)) atomicOr(&d.ctl[kCtlBad], 1);
    if (first) {
      d.beta0[p] = beta;
      d.its[p] = 0;
      d.conv[p] = beta == 0.0;
      d.relres[p] = 0.0;
    }
    double* s = d.s + (size_t)p * (m + 1);
    s[0] = beta;
    for (int i = 1; i <= m; ++i) s[i] = 0.0;
    d.jdone[p] = 0;
    const int act = !d.conv[p] && beta > 0.0 && isfinite(beta) && d.its[p] < limit;
    d.active[p] = act;
    d.scale[p] = act ? 1.0 / beta : 0.0;
    any |= act;
  }
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) {
    d.ctl[kCtlJ] = 0;
    d.ctl[kCtlCond] = any && m > 0;
    if (use_cond) cudaGraphSetConditional(hc, (unsigned)(any && m > 0));
  }
}

// End of an Arnoldi step: new Hessenberg column of every active problem (hsum, ||w||^2 in
// nrm2), its Givens rotation, the residual estimate and the stopping test; j <- j + 1 and the
// loop condition.
__global__ void __launch_bounds__(1024) batch_givens_kernel(int np, int m, int limit, double rtol, BatchDev d,
                                                            cudaGraphConditionalHandle hc, int use_cond) {
  const int j = d.ctl[kCtlJ];
  int any = 0;
  for (int p = threadIdx.x; p < np; p += blockDim.x) {
    if (!d.active[p]) {
      d.scale[p] = 0.0;
      continue;
    }
    const double* hc_ = d.hsum + (size_t)p * (m + 1);
    const double hn = sqrt(d.nrm2[p]);
    bool finite = isfinite(hn);
    for (int i = 0; i <= j; ++i) finite = finite && isfinite(hc_[i]);
    if (!finite) {  // the step does not count; the host reports the failure
      atomicOr(&d.ctl[kCtlBad], 1);
      d.active[p] = 0;
      d.scale[p] = 0.0;
      continue;
    }
    double* H = d.H + (size_t)p * (m + 1) * m;
    double* cs = d.cs + (size_t)p * m;
    double* sn = d.sn + (size_t)p * m;
    double* s = d.s + (size_t)p * (m + 1);
    for (int i = 0; i <= j; ++i) H[i * m + j] = hc_[i];
    H[(j + 1) * m + j] = hn;
    for (int i = 0; i < j; ++i) {
      const double t = cs[i] * H[i * m + j] + sn[i] * H[(i + 1) * m + j];
      H[(i + 1) * m + j] = -sn[i] * H[i * m + j] + cs[i] * H[(i + 1) * m + j];
      H[i * m + j] = t;
    }
    const double den = hypot(H[j * m + j], H[(j + 1) * m + j]);
    cs[j] = den > 0.0 ? H[j * m + j] / den : 1.0;
    sn[j] = den > 0.0 ? H[(j + 1) * m + j] / den : 0.0;
    H[j * m + j] = den;
    H[(j + 1) * m + j] = 0.0;
    s[j + 1] = -sn[j] * s[j];
    s[j] = cs[j] * s[j];
    d.its[p] += 1;
    d.jdone[p] = j + 1;
    const bool stop = fabs(s[j + 1]) <= rtol * d.beta0[p] || hn == 0.0 || d.its[p] >= limit || den == 0.0;
    if (stop) d.active[p] = 0;
    d.scale[p] = stop ? 0.0 : 1.0 / hn;
    any |= !stop;
  }
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) {
    const int jn = j + 1;
    d.ctl[kCtlJ] = jn;
    d.ctl[kCtlSteps] += 1;
    const int cond = any && jn < m;
    d.ctl[kCtlCond] = cond;
    if (use_cond) cudaGraphSetConditional(hc, (unsigned)cond);
  }
}

// y_p = R_p^-1 s_p over the problem's own steps (upper-triangular back substitution)
__global__ void batch_backsub_kernel(int np, int m, BatchDev d) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x) {
    const int jd = d.jdone[p];
    const double* H = d.H + (size_t)p * (m + 1) * m;
    const double* s = d.s + (size_t)p * (m + 1);
    double* y = d.y + (size_t)p * m;
    for (int i = jd - 1; i >= 0; --i) {
      double acc = s[i];
      for (int k = i + 1; k < jd; ++k) acc -= H[i * m + k] * y[k];
      y[i] = acc / H[i * m + i];
    }
  }
}

// x <- x + sum_{k < jdone_p} Z_k y_p[k]
__global__ void batch_update_kernel(long long n, int per_e, const int* elem_prob, const double* Z, int m, BatchDev d,
                                    double* x) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int p = elem_prob[i / per_e];
    const int jd = d.jdone[p];
    const double* y = d.y + (size_t)p * m;
    double acc = x[i];
    for (int k = 0; k < jd; ++k) acc += Z[(size_t)k * n + i] * y[k];
    x[i] = acc;
  }
}

// After the true residual of a cycle (its squared norms in nrm2): convergence per problem.
__global__ void __launch_bounds__(1024) batch_cycle_end_kernel(int np, int limit, double rtol, int fixed, BatchDev d) {
  int undone = 0, missed = 0;
  for (int p = threadIdx.x; p < np; p += blockDim.x) {
    const double rn = sqrt(d.nrm2[p]);
    if (!isfinite(rn)) atomicOr(&d.ctl[kCtlBad], 1);
    d.relres[p] = d.beta0[p] > 0.0 ? rn / d.beta0[p] : 0.0;
    const int c = fixed ? d.its[p] >= limit : (d.beta0[p] == 0.0 || rn <= rtol * d.beta0[p]);
    d.conv[p] = c;
    undone |= !c && d.its[p] < limit && isfinite(rn);
    missed |= !c;
  }
  undone = __syncthreads_or(undone);
  missed = __syncthreads_or(missed);
  if (threadIdx.x == 0) {
    d.ctl[kCtlDone] = !undone;
    d.ctl[kCtlConv] = !missed;
  }
}

// ------------------------------------------------------------------ plan
struct BatchWs {
  Handle* h = nullptr;
  const double* g = nullptr;
  double* x = nullptr;
  int m = 0, np = 0;
  long long n = 0;
  int per_e = 0;
  double* V = nullptr;   // [(m+1)][n]
  double* Z = nullptr;   // [m][n]
  double* vin = nullptr;
  double* zf = nullptr;
  double* wf = nullptr;
  double* r = nullptr;
  double* tmp = nullptr;
  double* part = nullptr;  // [nchunk][m+1]
  BatchDev d{};
  void* small = nullptr;   // one allocation behind d
  int* host_ctl = nullptr;  // pinned [kCtlN]
  // launches / operator applications of the prologue, one step and the epilogue (graph replays)
  long long l_pro[2] = {0, 0}, l_body = 0, l_epi = 0, o_pro[2] = {0, 0}, o_body = 0, o_epi = 0;
};

struct Plan {
  std::vector<BatchWs> ws;
  dg_solve_opts o{};
  bool graph = false;
  bool captured = false;
  cudaGraphExec_t exec[2] = {nullptr, nullptr};  // [0] first cycle, [1] restart cycle
  cudaStream_t origin = nullptr;
  std::vector<cudaStream_t> side, body;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  int cycles = 0, steps = 0;
  long long graph_launches = 0;
  std::string err;
};

static int pfail(Plan* P, int code, const std::string& msg) {
  if (P) P->err = msg;
  return code;
}
#define PL_CUDA(P, call)                                                                          \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess) return pfail((P), DG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

static int seg_grid(const Handle* h, long long work) {
  long long g = (long long)h->nsm * 8;
  if (g > work) g = work;
  return g < 1 ? 1 : (int)g;
}

static int alloc_ws(Plan* P, BatchWs& b) {
  Handle* h = b.h;
  const long long n = b.n;
  const int m = b.m, np = b.np;
  PL_CUDA(P, cudaMalloc((void**)&b.V, sizeof(double) * (size_t)(m + 1) * n));
  PL_CUDA(P, cudaMalloc((void**)&b.Z, sizeof(double) * (size_t)m * n));
  double** vecs[5] = {&b.vin, &b.zf, &b.wf, &b.r, &b.tmp};
  for (double** v : vecs) PL_CUDA(P, cudaMalloc((void**)v, sizeof(double) * n));
  PL_CUDA(P, cudaMalloc((void**)&b.part, sizeof(double) * (size_t)h->nchunk * (m + 1)));
  const size_t nd = (size_t)np * ((m + 1) * m + 3 * m + 3 * (m + 1) + 5);
  const size_t bytes = nd * sizeof(double) + sizeof(int) * ((size_t)np * 4 + kCtlN);
  PL_CUDA(P, cudaMalloc(&b.small, bytes));
  PL_CUDA(P, cudaMemset(b.small, 0, bytes));
  double* q = reinterpret_cast<double*>(b.small);
  auto take = [&](size_t cnt) { double* r = q; q += cnt; return r; };
  b.d.H = take((size_t)np * (m + 1) * m);
  b.d.cs = take((size_t)np * m);
  b.d.sn = take((size_t)np * m);
  b.d.y = take((size_t)np * m);
  b.d.s = take((size_t)np * (m + 1));
  b.d.hpass = take((size_t)np * (m + 1));
  b.d.hsum = take((size_t)np * (m + 1));
  b.d.beta0 = take(np);
  b.d.nrm2 = take(np);
  b.d.scale = take(np);
  b.d.relres = take(np);
  take(np);  // spare
  int* qi = reinterpret_cast<int*>(q);
  b.d.jdone = qi; qi += np;
  b.d.active = qi; qi += np;
  b.d.its = qi; qi += np;
  b.d.conv = qi; qi += np;
  b.d.ctl = qi;
  PL_CUDA(P, cudaMallocHost((void**)&b.host_ctl, sizeof(int) * kCtlN));
  return DG_OK;
}

static void free_ws(BatchWs& b) {
  auto F = [](void* p) { if (p) cudaFree(p); };
  F(b.V); F(b.Z); F(b.vin); F(b.zf); F(b.wf); F(b.r); F(b.tmp); F(b.part); F(b.small);
  if (b.host_ctl) cudaFreeHost(b.host_ctl);
  b = BatchWs{};
}

// squared norms per problem of x into d.nrm2
static int seg_norm2(BatchWs& b, const double* x, cudaStream_t st) {
  Handle* h = b.h;
  seg_dot_kernel<<<seg_grid(h, h->nchunk), kSegThreads, 0, st>>>(h->nchunk, h->chunk, b.per_e, x, 0, 1, nullptr, x,
                                                                 b.part, b.m + 1);
  DG_LAUNCH_CHECK(h);
  seg_reduce_kernel<<<b.np, kSegThreads, 0, st>>>(h->pchunk0, b.part, b.m + 1, 1, nullptr, b.d.nrm2, nullptr, 0, 1);
  DG_LAUNCH_CHECK(h);
  return DG_OK;
}

// one Arnoldi step of every active problem (the body of the cycle's loop)
static int arnoldi_step(const Plan& P, BatchWs& b, cudaGraphConditionalHandle hc, int use_cond, cudaStream_t st) {
  Handle* h = b.h;
  const dg_solve_opts& o = P.o;
  const int m = b.m;
  const long long n = b.n;
  const int gv = seg_grid(h, n / 256 + 1);
  int rc;
  if ((rc = precond_apply(h, o, b.vin, b.zf, st))) return rc;
  batch_store_kernel<<<gv, 256, 0, st>>>(n, b.zf, b.d.ctl + kCtlJ, b.Z);
  DG_LAUNCH_CHECK(h);
  if ((rc = op_tangent(h, b.zf, b.wf, st))) return rc;
  for (int pass = 0; pass < 2; ++pass) {  // classical Gram-Schmidt, twice
    seg_dot_kernel<<<seg_grid(h, h->nchunk), kSegThreads, 0, st>>>(h->nchunk, h->chunk, b.per_e, b.V, n, 0,
                                                                   b.d.ctl + kCtlJ, b.wf, b.part, m + 1);
    DG_LAUNCH_CHECK(h);
    seg_reduce_kernel<<<b.np, kSegThreads, 0, st>>>(h->pchunk0, b.part, m + 1, 0, b.d.ctl + kCtlJ, b.d.hpass,
                                                    b.d.hsum, pass, m + 1);
    DG_LAUNCH_CHECK(h);
    seg_axpy_kernel<<<gv, 256, 0, st>>>(n, b.per_e, h->elem_prob, b.V, n, b.d.ctl + kCtlJ, b.d.hpass, m + 1, b.wf);
    DG_LAUNCH_CHECK(h);
  }
  if ((rc = seg_norm2(b, b.wf, st))) return rc;
  const int limit = o.fixed_its > 0 ? o.fixed_its : o.maxit;
  const double rtol = o.fixed_its > 0 ? -1.0 : o.rtol;
  batch_givens_kernel<<<1, 1024, 0, st>>>(b.np, m, limit, rtol, b.d, hc, use_cond);
  DG_LAUNCH_CHECK(h);
  batch_normalize_kernel<<<gv, 256, 0, st>>>(n, b.per_e, h->elem_prob, b.wf, b.d.scale, b.d.ctl + kCtlJ, b.V, b.vin);
  DG_LAUNCH_CHECK(h);
  return DG_OK;
}

static int read_ctl(Plan* P, BatchWs& b, cudaStream_t st) {
  PL_CUDA(P, cudaMemcpyAsync(b.host_ctl, b.d.ctl, sizeof(int) * kCtlN, cudaMemcpyDeviceToHost, st));
  PL_CUDA(P, cudaStreamSynchronize(st));
  return DG_OK;
}

// Prologue of a cycle. first: r = g - G x0 (or g), the solve's counters reset.
static int cycle_prologue(const Plan& P, BatchWs& b, bool first, cudaGraphConditionalHandle hc, int use_cond,
                          cudaStream_t st) {
  Handle* h = b.h;
  const dg_solve_opts& o = P.o;
  int rc;
  if (first) {
    DG_CUDA(h, cudaMemsetAsync(b.d.ctl, 0, sizeof(int) * kCtlN, st));
    if (o.x0_is_zero) {
      DG_CUDA(h, cudaMemsetAsync(b.x, 0, sizeof(double) * b.n, st));
      DG_CUDA(h, cudaMemcpyAsync(b.r, b.g, sizeof(double) * b.n, cudaMemcpyDeviceToDevice, st));
    } else {
      if ((rc = op_tangent(h, b.x, b.tmp, st))) return rc;
      DG_CUDA(h, cudaMemcpyAsync(b.r, b.g, sizeof(double) * b.n, cudaMemcpyDeviceToDevice, st));
      if ((rc = launch_axpby(h, b.n, -1.0, b.tmp, 1.0, b.r, st))) return rc;
    }
    if ((rc = seg_norm2(b, b.r, st))) return rc;
  }
  // later cycles start from the true residual r and its norms left by the previous epilogue
  const int limit = o.fixed_its > 0 ? o.fixed_its : o.maxit;
  batch_cycle_init_kernel<<<1, 1024, 0, st>>>(b.np, b.m, limit, first ? 1 : 0, b.d, hc, use_cond);
  DG_LAUNCH_CHECK(h);
  batch_normalize_kernel<<<seg_grid(h, b.n / 256 + 1), 256, 0, st>>>(b.n, b.per_e, h->elem_prob, b.r, b.d.scale,
                                                                    b.d.ctl + kCtlJ, b.V, b.vin);
  DG_LAUNCH_CHECK(h);
  return DG_OK;
}

// Epilogue: x += Z y per problem, true residual r = g - G x, convergence per problem.
static int cycle_epilogue(const Plan& P, BatchWs& b, cudaStream_t st) {
  Handle* h = b.h;
  const dg_solve_opts& o = P.o;
  int rc;
  batch_backsub_kernel<<<(b.np + 127) / 128, 128, 0, st>>>(b.np, b.m, b.d);
  DG_LAUNCH_CHECK(h);
  batch_update_kernel<<<seg_grid(h, b.n / 256 + 1), 256, 0, st>>>(b.n, b.per_e, h->elem_prob, b.Z, b.m, b.d, b.x);
  DG_LAUNCH_CHECK(h);
  if ((rc = op_tangent(h, b.x, b.tmp, st))) return rc;
  DG_CUDA(h, cudaMemcpyAsync(b.r, b.g, sizeof(double) * b.n, cudaMemcpyDeviceToDevice, st));
  if ((rc = launch_axpby(h, b.n, -1.0, b.tmp, 1.0, b.r, st))) return rc;
  if ((rc = seg_norm2(b, b.r, st))) return rc;
  const int limit = o.fixed_its > 0 ? o.fixed_its : o.maxit;
  batch_cycle_end_kernel<<<1, 1024, 0, st>>>(b.np, limit, o.rtol, o.fixed_its > 0 ? 1 : 0, b.d);
  DG_LAUNCH_CHECK(h);
  return DG_OK;
}

static int handle_error(Plan* P, BatchWs& b, int rc) {
  return pfail(P, rc, b.h->err);
}

// One restart cycle of one handle, launched eagerly: the loop condition is read on the host.
static int eager_cycle(Plan* P, BatchWs& b, bool first, cudaStream_t st) {
  int rc;
  if ((rc = cycle_prologue(*P, b, first, 0, 0, st))) return handle_error(P, b, rc);
  if ((rc = read_ctl(P, b, st))) return rc;
  for (int guard = 0; b.host_ctl[kCtlCond] && guard < b.m; ++guard) {
    if ((rc = arnoldi_step(*P, b, 0, 0, st))) return handle_error(P, b, rc);
    if ((rc = read_ctl(P, b, st))) return rc;
  }
  if ((rc = cycle_epilogue(*P, b, st))) return handle_error(P, b, rc);
  return read_ctl(P, b, st);
}

// Capture one restart cycle of b on stream st (already capturing): prologue, a conditional
// WHILE node whose body is one Arnoldi step (captured on the handle's body stream), epilogue.
static int capture_cycle(Plan* P, int i, bool first, cudaStream_t st) {
  BatchWs& b = P->ws[i];
  Handle* h = b.h;
  cudaStreamCaptureStatus cst;
  cudaGraph_t graph = nullptr;
  PL_CUDA(P, cudaStreamGetCaptureInfo(st, &cst, nullptr, &graph, nullptr, nullptr, nullptr));
  if (cst != cudaStreamCaptureStatusActive || !graph) return pfail(P, DG_ERR_CUDA, "stream is not capturing");
  cudaGraphConditionalHandle hc;
  PL_CUDA(P, cudaGraphConditionalHandleCreate(&hc, graph, 0, cudaGraphCondAssignDefault));
  int rc;
  const long long l0 = h->launches, o0 = h->op_apps;
  if ((rc = cycle_prologue(*P, b, first, hc, 1, st))) return handle_error(P, b, rc);
  b.l_pro[first ? 0 : 1] = h->launches - l0;
  b.o_pro[first ? 0 : 1] = h->op_apps - o0;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  PL_CUDA(P, cudaStreamGetCaptureInfo(st, &cst, nullptr, &graph, &deps, nullptr, &ndeps));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = hc;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  PL_CUDA(P, cudaGraphAddNode(&node, graph, deps, nullptr, ndeps, &cp));
  cudaGraph_t bodyg = cp.conditional.phGraph_out[0];
  cudaStream_t bs = P->body[i];
  PL_CUDA(P, cudaStreamBeginCaptureToGraph(bs, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  const long long l1 = h->launches, o1 = h->op_apps;
  rc = arnoldi_step(*P, b, hc, 1, bs);
  b.l_body = h->launches - l1;
  b.o_body = h->op_apps - o1;
  cudaGraph_t got = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(bs, &got);
  if (rc) return handle_error(P, b, rc);
  if (ec != cudaSuccess) return pfail(P, DG_ERR_CUDA, std::string("body capture: ") + cudaGetErrorString(ec));
  PL_CUDA(P, cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  const long long l2 = h->launches, o2 = h->op_apps;
  if ((rc = cycle_epilogue(*P, b, st))) return handle_error(P, b, rc);
  b.l_epi = h->launches - l2;
  b.o_epi = h->op_apps - o2;
  // captured launches are counted when the graph runs, not here
  h->launches = l0;
  h->op_apps = o0;
  return DG_OK;
}

static int capture_plan(Plan* P) {
  std::vector<bool> prof(P->ws.size());
  for (size_t i = 0; i < P->ws.size(); ++i) {  // no event nodes inside conditional bodies
    prof[i] = P->ws[i].h->prof;
    P->ws[i].h->prof = false;
  }
  int rc = DG_OK;
  for (int first = 1; first >= 0 && rc == DG_OK; --first) {
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(P->origin, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) { rc = pfail(P, DG_ERR_CUDA, cudaGetErrorString(e)); break; }
    e = cudaEventRecord(P->fork, P->origin);
    for (size_t i = 0; i < P->ws.size() && rc == DG_OK && e == cudaSuccess; ++i) {
      e = cudaStreamWaitEvent(P->side[i], P->fork, 0);
      if (e != cudaSuccess) break;
      rc = capture_cycle(P, (int)i, first == 1, P->side[i]);
      if (rc) break;
      e = cudaEventRecord(P->join[i], P->side[i]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(P->origin, P->join[i], 0);
    }
    const cudaError_t ee = cudaStreamEndCapture(P->origin, &graph);
    if (rc == DG_OK && e != cudaSuccess) rc = pfail(P, DG_ERR_CUDA, cudaGetErrorString(e));
    if (rc == DG_OK && ee != cudaSuccess) rc = pfail(P, DG_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(ee));
    if (rc == DG_OK) {
      e = cudaGraphInstantiate(&P->exec[first ? 0 : 1], graph, 0);
      if (e != cudaSuccess) rc = pfail(P, DG_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(e));
    }
    if (graph) cudaGraphDestroy(graph);
  }
  for (size_t i = 0; i < P->ws.size(); ++i) P->ws[i].h->prof = prof[i];
  if (rc == DG_OK) P->captured = true;
  return rc;
}

static void destroy_plan(Plan* P) {
  if (!P) return;
  cudaDeviceSynchronize();
  for (auto& e : P->exec)
    if (e) cudaGraphExecDestroy(e);
  for (auto& b : P->ws) free_ws(b);
  for (auto s : P->side) cudaStreamDestroy(s);
  for (auto s : P->body) cudaStreamDestroy(s);
  for (auto e : P->join) cudaEventDestroy(e);
  if (P->fork) cudaEventDestroy(P->fork);
  if (P->origin) cudaStreamDestroy(P->origin);
  delete P;
}

static thread_local std::string g_plan_error;

}  // namespace dg

using namespace dg;

extern "C" {

int dg_plan_create(int nh, dg_handle* const* hs, const double* const* g, double* const* x, const dg_solve_opts* o,
                   int use_graph, dg_plan** out) {
  if (!out) return DG_ERR_ARG;
  *out = nullptr;
  g_plan_error.clear();
  if (nh < 1 || !hs || !g || !x || !o) { g_plan_error = "null argument or nh < 1"; return DG_ERR_ARG; }
  for (int i = 0; i < nh; ++i) {
    Handle* h = reinterpret_cast<Handle*>(hs[i]);
    if (!h || !g[i] || !x[i] || g[i] == x[i]) { g_plan_error = "null handle or bad g/x pointer"; return DG_ERR_ARG; }
    for (int k = 0; k < i; ++k)
      if (hs[k] == hs[i]) { g_plan_error = "a handle appears twice"; return DG_ERR_ARG; }
    int rc = solve_opts_check(h, o);
    if (rc) { g_plan_error = h->err; return rc; }
  }
  if (o->restart < 1 || o->restart > 64) { g_plan_error = "restart must be in 1..64"; return DG_ERR_ARG; }
  if (o->fixed_its <= 0 && (o->maxit < 1 || !(o->rtol > 0.0))) { g_plan_error = "bad maxit/rtol"; return DG_ERR_ARG; }
  if (o->jvp_mode != DG_JVP_TANGENT) { g_plan_error = "the batched solver uses the exact products"; return DG_ERR_ARG; }
  if (o->coarse_solver != DG_COARSE_SMOOTHER && o->coarse_solver != DG_COARSE_LEARNED) {
    g_plan_error = "the batched solver takes the smoother or the learned coarse solve";
    return DG_ERR_ARG;
  }
  Plan* P = new (std::nothrow) Plan();
  if (!P) return DG_ERR_ARG;
  P->o = *o;
  P->graph = use_graph != 0;
  P->ws.resize(nh);
  int rc = DG_OK;
  for (int i = 0; i < nh && rc == DG_OK; ++i) {
    BatchWs& b = P->ws[i];
    b.h = reinterpret_cast<Handle*>(hs[i]);
    b.g = g[i];
    b.x = x[i];
    b.m = o->restart;
    b.np = b.h->nprob;
    b.n = b.h->lev[0].n;
    b.per_e = b.h->lev[0].b;
    rc = alloc_ws(P, b);
  }
  if (rc == DG_OK) {
    cudaError_t e = cudaStreamCreateWithFlags(&P->origin, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->fork, cudaEventDisableTiming);
    P->side.resize(nh, nullptr);
    P->body.resize(nh, nullptr);
    P->join.resize(nh, nullptr);
    for (int i = 0; i < nh && e == cudaSuccess; ++i) {
      e = cudaStreamCreateWithFlags(&P->side[i], cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&P->body[i], cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->join[i], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) rc = pfail(P, DG_ERR_CUDA, cudaGetErrorString(e));
  }
  if (rc != DG_OK) {
    g_plan_error = P->err;
    destroy_plan(P);
    return rc;
  }
  *out = reinterpret_cast<dg_plan*>(P);
  return DG_OK;
}

int dg_plan_destroy(dg_plan* pp) {
  destroy_plan(reinterpret_cast<Plan*>(pp));
  return DG_OK;
}

const char* dg_plan_error(const dg_plan* pp) {
  if (!pp) return g_plan_error.c_str();
  return reinterpret_cast<const Plan*>(pp)->err.c_str();
}

int dg_plan_solve(dg_plan* pp, void* stream) {
  const dg::NvtxRange nvtx_range_("dg_plan_solve");
  Plan* P = reinterpret_cast<Plan*>(pp);
  if (!P) return DG_ERR_ARG;
  P->err.clear();
  cudaStream_t st = as_stream(stream);
  int rc;
  for (auto& b : P->ws) {  // eager: FP32 / 16-bit copies of the current assembly
    if (!b.h->linearized) return pfail(P, DG_ERR_STATE, "every handle needs dg_set_linearization first");
    if ((rc = precond_prepare(b.h, P->o, st))) return handle_error(P, b, rc);
  }
  const int limit = P->o.fixed_its > 0 ? P->o.fixed_its : P->o.maxit;
  const int max_cycles = (limit + P->o.restart - 1) / P->o.restart + 1;
  P->cycles = 0;
  P->steps = 0;
  bool done = false;
  if (!P->graph) {
    for (int c = 0; c < max_cycles && !done; ++c) {
      done = true;
      for (auto& b : P->ws) {
        if (c > 0 && b.host_ctl[kCtlDone]) continue;
        if ((rc = eager_cycle(P, b, c == 0, st))) return rc;
        done = done && b.host_ctl[kCtlDone];
      }
      ++P->cycles;
    }
  } else {
    if (!P->captured) {
      PL_CUDA(P, cudaStreamSynchronize(st));
      if ((rc = capture_plan(P))) return rc;
    }
    std::vector<int> before(P->ws.size(), 0);
    for (int c = 0; c < max_cycles && !done; ++c) {
      for (size_t i = 0; i < P->ws.size(); ++i) before[i] = c == 0 ? 0 : P->ws[i].host_ctl[kCtlSteps];
      PL_CUDA(P, cudaGraphLaunch(P->exec[c == 0 ? 0 : 1], st));
      ++P->graph_launches;
      ++P->cycles;
      done = true;
      for (size_t i = 0; i < P->ws.size(); ++i) {
        BatchWs& b = P->ws[i];
        if ((rc = read_ctl(P, b, st))) return rc;
        const long long stepped = b.host_ctl[kCtlSteps] - before[i];
        b.h->launches += b.l_pro[c == 0 ? 0 : 1] + stepped * b.l_body + b.l_epi;
        b.h->op_apps += b.o_pro[c == 0 ? 0 : 1] + stepped * b.o_body + b.o_epi;
        done = done && b.host_ctl[kCtlDone];
      }
    }
  }
  int bad = 0, conv = 1;
  for (auto& b : P->ws) {
    bad |= b.host_ctl[kCtlBad];
    conv &= b.host_ctl[kCtlConv];
    P->steps = std::max(P->steps, b.host_ctl[kCtlSteps]);
  }
  if (bad) return pfail(P, DG_ERR_NONFINITE, "non-finite Krylov quantity in a problem of the batch");
  if (!done || !conv) return pfail(P, DG_ERR_NOT_CONVERGED, "some problem did not reach the tolerance");
  return DG_OK;
}

int dg_plan_result(const dg_plan* pp, int i, int* its, double* relres, int* converged) {
  const Plan* P = reinterpret_cast<const Plan*>(pp);
  if (!P || i < 0 || i >= (int)P->ws.size()) return DG_ERR_ARG;
  const BatchWs& b = P->ws[i];
  if (its && cudaMemcpy(its, b.d.its, sizeof(int) * b.np, cudaMemcpyDeviceToHost) != cudaSuccess) return DG_ERR_CUDA;
  if (relres && cudaMemcpy(relres, b.d.relres, sizeof(double) * b.np, cudaMemcpyDeviceToHost) != cudaSuccess)
    return DG_ERR_CUDA;
  if (converged && cudaMemcpy(converged, b.d.conv, sizeof(int) * b.np, cudaMemcpyDeviceToHost) != cudaSuccess)
    return DG_ERR_CUDA;
  return DG_OK;
}

int dg_plan_stats(const dg_plan* pp, int* cycles, int* steps, long long* graph_launches) {
  const Plan* P = reinterpret_cast<const Plan*>(pp);
  if (!P) return DG_ERR_ARG;
  if (cycles) *cycles = P->cycles;
  if (steps) *steps = P->steps;
  if (graph_launches) *graph_launches = P->graph_launches;
  return DG_OK;
}

}  // extern "C"
