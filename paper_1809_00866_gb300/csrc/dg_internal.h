// Internal declarations of the dgpmg CUDA library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdint>
#include <string>
#include <vector>

#include "dgpmg.h"

namespace dg {

constexpr int kMaxK = 4;

__host__ __device__ constexpr int nb_of(int k) { return (k + 1) * (k + 2) * (k + 3) / 6; }

// Tables of the fine level's reference basis phi_hat_m(xi) = prod_d sqrt((2n_d+1)/2) L_{n_d}(xi_d)
// on [-1,1]^3 (orthonormal), at the Gauss points of the level's rule (k+1 points per axis).
struct Tables {
  int k = 0, nb = 0, n1 = 0, nq = 0, nqf = 0, n2 = 0;
  double* Bvol = nullptr;   // [nq][nb]          phi_hat at volume points, q = (q0*n1 + q1)*n1 + q2
  double* wvol = nullptr;   // [nq]              reference volume weights
  double* xg = nullptr;     // [n1]              Gauss nodes on [-1,1]
  double* L1 = nullptr;     // [k+1][n1]         normalised Legendre P_hat_a(x_q)
  // 2D trace modes on a face: pairs (b, c), b + c <= k, b the exponent along the first
  // tangential axis t1 = (d+1)%3 and c along t2 = (d+2)%3; n2 = (k+1)(k+2)/2 of them.
  double* B2 = nullptr;     // [nqf][n2]         P_hat_b P_hat_c at the face points, q = q1*n1 + q2
  double* W2 = nullptr;     // [nqf]             reference face weights
  double* pv = nullptr;     // [2][k+1]          P_hat_a(+1), P_hat_a(-1)
  double* pd = nullptr;     // [2][k+1]          P_hat_a'(+1), P_hat_a'(-1)
  int* M3 = nullptr;        // [3][n2][k+1]      3D mode of (exponent a along d, 2D mode n2) or -1
  int* fmap = nullptr;      // [3][nb]           2D mode of 3D mode m seen from a face normal to d
  int* fa = nullptr;        // [3][nb]           exponent of m along d
  int* md3 = nullptr;       // [nb][3]           exponents of 3D mode m
  int* pidx = nullptr;      // [(k+1)][(k+1)]    index of the pair (a, b), a + b <= k (the 2D ordering)
  int* pab = nullptr;       // [n2][2]           the pair (a, b) of a pair index
  // Sparse reference derivative operator: d/dxi_b phi_hat_n = sum_m D_b[m][n] phi_hat_m.
  // Drow[b][m][j] / Dcol[b][n][j] hold at most kDw entries (index, value) of row m / column n.
  int* Drow_idx = nullptr;     // [3][nb][kDw]
  double* Drow_val = nullptr;  // [3][nb][kDw]
  int* Dcol_idx = nullptr;     // [3][nb][kDw]
  double* Dcol_val = nullptr;  // [3][nb][kDw]
  // the same for the 2D trace modes along t1 (dir 0) and t2 (dir 1), by rows
  int* D2_idx = nullptr;       // [2][n2][kDw]
  double* D2_val = nullptr;    // [2][n2][kDw]
  static constexpr int kDw = 3;
};

// FP32 copies of the real-valued tables (reduced-precision preconditioner)
struct TablesF {
  float* Bvol = nullptr;
  float* L1 = nullptr;
  float* wvol = nullptr;
  float* B2 = nullptr;
  float* W2 = nullptr;
  float* pv = nullptr;
  float* pd = nullptr;
  float* Drow_val = nullptr;
  float* Dcol_val = nullptr;
  float* D2_val = nullptr;
};

struct Level {
  int k = 0, nb = 0, b = 0;  // degree, modes per variable, block size 4*nb
  long long n = 0;           // vector length ne*4*nb
  double* Dblk = nullptr;    // [ne][b][b] diagonal blocks, column-major per block
  double* Dinv = nullptr;    // [ne][b][b] LU factors (unit L, U, 1/U_kk on the diagonal), column-major per block
  int* perm = nullptr;       // [ne][b] row permutation of the LU factors
  double* Bsr = nullptr;     // [ne][7][b][b] level >= 1: slot 0 diagonal, slots 1..6 faces -x,+x,-y,+y,-z,+z
  double* Dlin = nullptr;    // level 0: [ne][b][b] diagonal blocks of the state-independent linear part
  double* Blin = nullptr;    // level 1: [ne][7][b][b] off-diagonal blocks of the linear part (slot 0 unused)
  double* t0 = nullptr;      // work vectors of length n
  double* t1 = nullptr;
  double* t2 = nullptr;
  // FP32 copies for the reduced-precision preconditioner (allocated on first use)
  float* LUf = nullptr;      // [ne][b][b] explicit inverses D^-1 (column-major) once assembled
  float* Bsrf = nullptr;     // [ne][7][b][b] (level >= 1)
  float* t0f = nullptr;
  float* t1f = nullptr;
  float* t2f = nullptr;
  // 16-bit copies of LUf and Bsrf (FP16 or bfloat16, Handle::asm16 says which)
  void* LU16 = nullptr;
  void* Bsr16 = nullptr;
};

// Launch shapes of the tangent operator passes and of the staged block-Jacobi apply
// (dg_set_tuning / dg_autotune); every shape gives the same results.
struct OpTune {
  int face_warps = 4;         // faces per CTA of the face pass: 2, 4 or 8
  int vol_threads = 128;      // threads per CTA of the volume pass: 64, 128 or 256
  int face_per_sm = 0;        // cap on CTAs per SM (0: shared memory decides)
  int vol_per_sm = 0;
  int jacobi_stage_kb = 96;   // element blocks staged per bulk copy of the block-Jacobi apply (KB)
  int jacobi_max_ctas = 0;    // cap on the CTAs of that apply (0: one wave of the GPU)
};

// Test settings of the failure-detection paths (dg_set_test_knob); the defaults are the
// production values.
struct DebugKnobs {
  int riemann_its = 60;   // iteration cap of the star-state solve (Newton with bisection safeguard)
  int wait_polls = 0;     // polls of the staged block-Jacobi apply's bounded waits (0: kBulkWaitLimit)
  int withhold_copy = 0;  // != 0: that apply leaves each CTA's first stage uncopied (its wait gives up)
};

struct Handle {
  dg_params p{};
  OpTune tune[2];               // [0] FP64 products, [1] FP32 products (and the FP32 block-Jacobi apply)
  DebugKnobs dbg;
  int n[3] = {0, 0, 0};
  int ne = 0;
  int nlev = 0;
  std::vector<double> node[3];  // host node coordinates
  double* dnode[3] = {nullptr, nullptr, nullptr};
  double* geo = nullptr;        // [ne][kGeo] per-element geometry
  float* geof = nullptr;        // the same in FP32 (read by the FP32 passes)
  int* nbr = nullptr;           // [ne][6] face neighbours -x,+x,-y,+y,-z,+z; -1 across a wall
  std::vector<int> nbr_host;    // host copy of nbr
  // faces: 3 per element (its +x, +y, +z faces; a +y face on a wall has no neighbour), then the
  // nbf wall faces below the elements of the first row (bface[b] = that element); bslot[e] =
  // b for those elements, else -1
  int nbf = 0;
  int* bface = nullptr;
  int* bslot = nullptr;
  // independent problems (periodic boxes) sharing the handle: problem p owns the elements
  // [pe0[p], pe0[p+1]); every face neighbour of an element lies in its own problem
  int nprob = 1;
  std::vector<int> pe0;         // host [nprob+1]
  int* elem_prob = nullptr;     // device [ne] problem of each element
  double* dshift = nullptr;     // device [nprob] mass-shift multipliers (geo slot 11 holds them per element)
  // per-problem reduction chunks: chunk c covers the elements [chunk[c].x, chunk[c].y) of
  // problem chunk_prob[c]; the chunks of problem p are pchunk0[p] .. pchunk0[p+1]-1
  int nchunk = 0;
  int2* chunk = nullptr;
  int* chunk_prob = nullptr;
  int* pchunk0 = nullptr;
  int* colour = nullptr;        // [ne] element colouring used by the assembly probes
  Tables tab;                   // fine-level tables (the matrix-free level)
  TablesF tabf;                 // their FP32 copies
  Level lev[DG_MAX_LEVELS];
  int nsm = 0;
  int device = 0;               // the CUDA device that was current at dg_create (holds every buffer)

  // scratch of the matrix-free operator
  double* face_out = nullptr;  // [ne][6][4][n2] face-term contributions per element face slot (2D modes)
  double* face_lift = nullptr; // [ne][6][3][n2] BR2 local lifting (scaled 2D jump) per element face slot
  float* face_out_f = nullptr;   // FP32 scratch of the FP32 operator
  float* face_lift_f = nullptr;
  void* tc_tab[2] = {nullptr, nullptr};  // 16-bit basis tables of the tensor-core volume pass (FP16, BF16)
  float* ubar_scale = nullptr;            // [ne] power-of-two scale of the FP32 linearisation velocity
  float* ubar_f = nullptr;       // FP32 copies of the linearisation cache
  float* dFlux_f = nullptr;
  bool lin_f_ready = false;      // the FP32 copies match the current linearisation
  bool asm_f_ready = false;      // the FP32 factors / blocks match the current assembly
  bool asm64_ready = false;      // the FP64 factors / blocks match the current assembly
  int asm16 = 0;                 // storage type of the 16-bit block copies that match it (0: none)
  // linearisation cache
  bool linearized = false;
  bool assembled = false;
  bool linpart_ready = false;  // Dlin / Blin probed (they depend on the mesh only)
  // rescaled-inherited coarse operators (Appendix A): the stabilisation (BR2 penalty) part of
  // the level-1 block rows, [ne][7][b1][b1] with slot 0 the diagonal, probed once when enabled
  bool stb_rescale = false;
  bool stb_ready = false;
  double* stb1 = nullptr;
  float* stb1f = nullptr;       // the same in FP32, for the FP32 assembly
  double inv_gdt = 0.0;
  double* wlin = nullptr;   // [n0]
  double* flin = nullptr;   // [n0] f_h(wlin)
  double* ubar = nullptr;   // [ne][3][nq] velocity at the volume points
  double* dFlux = nullptr;  // [3*ne][nqf][4][8] Jacobian of the Riemann flux at the face points
  double* wnorm2 = nullptr; // device scalar ||wlin||^2
  // finite-difference scratch
  double* fd_w = nullptr;
  double* fd_f = nullptr;
  double* red = nullptr;    // reduction partials
  double* red_out = nullptr;
  unsigned* status = nullptr;  // device status words: [0] the handle's (dg_get_status), [1] the
                               // linearisation's, [2] the current assembly's
  // Krylov workspace
  int kry_m = 0;
  double* V = nullptr;  // [(m+1)][n0]
  double* Z = nullptr;  // [m][n0]
  double* hcol = nullptr;     // device [m+2]
  double* hcol_host = nullptr;  // pinned [m+2]
  // GMRES smoother workspace: per-level Krylov basis and small device arrays
  double* smV[DG_MAX_LEVELS] = {nullptr, nullptr, nullptr, nullptr};  // [(its+1)][n_l]
  int smV_its[DG_MAX_LEVELS] = {0, 0, 0, 0};
  double* smSmall = nullptr;  // H, dots, squared norms, beta^2, -y
  // learned coarse correction: packed BF16 network (dg_set_coarse_network)
  unsigned char* net = nullptr;
  bool net_ready = false;
  // recording of the coarsest-level right-hand sides (dg_record_coarse)
  double* rec_buf = nullptr;
  int rec_cap = 0;
  int rec_count = 0;
  std::string err;
  // instrumentation
  long long launches = 0;
  long long op_apps = 0;
  bool prof = false;
  struct ProfEv { int cls; cudaEvent_t a, b; double bytes; };
  std::vector<ProfEv> prof_pending;
  std::vector<cudaEvent_t> ev_pool;
  double prof_ms[DG_PROF_N] = {};
  long long prof_cnt[DG_PROF_N] = {};
  double prof_bytes[DG_PROF_N] = {};
};

// A named NVTX range for the span of one C-ABI call (visible in Nsight timelines; a no-op when no
// tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// error helpers
int fail(Handle* h, int code, const std::string& msg);
#define DG_CUDA(h, call)                                                                         \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess)                                                                       \
      return ::dg::fail((h), DG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));   \
  } while (0)
#define DG_LAUNCH_CHECK(h)    \
  do {                        \
    ++(h)->launches;          \
    DG_CUDA(h, cudaGetLastError()); \
  } while (0)

// CUDA events around the launches of one kernel class (when profiling is on)
cudaEvent_t prof_event(Handle* h);
int prof_begin(Handle* h, cudaStream_t st, cudaEvent_t* a);
int prof_end(Handle* h, int cls, cudaStream_t st, cudaEvent_t a, double bytes = 0.0);

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// mesh geometry on the device
// Per-element geometry, computed once on the host: h[3], s = sqrt(|K|/8) (phi = phi_hat/s),
// 1/s, J = 2/h[3] (reference-to-physical derivative factors), lower corner lo[3], and the
// multiplier of the handle's mass shift 1/(gamma dt) for the element's problem (1 by default).
constexpr int kGeo = 12;
struct MeshDev {
  int nx, ny, nz, ne;
  const double* geo;  // [ne][kGeo]
  const float* geof;  // the same in FP32
  const int* nbr;
  int nbf;            // wall faces below the first row (faces 3 ne .. 3 ne + nbf - 1)
  const int* bface;   // [nbf] element above each of them
  const int* bslot;   // [ne] index of the wall face below the element, or -1
};
inline MeshDev mesh_dev(const Handle* h) {
  return MeshDev{h->n[0], h->n[1], h->n[2], h->ne, h->geo, h->geof, h->nbr, h->nbf, h->bface, h->bslot};
}

struct ElemGeom {
  double h[3];   // box sizes
  double lo[3];  // lower corner
  double s;      // sqrt(|K|/8)
  double is;     // 1/s
  double J[3];   // 2/h
  double sh;     // multiplier of the mass shift
};
// the geometry row of element e in the arithmetic type R (FP32 passes read the FP32 copy, so
// that they convert nothing on GB300's narrow FP64 pipe): h[0..2] at 0, s at 3, 1/s at 4,
// 2/h[0..2] at 5, lower corner at 8, mass-shift multiplier at 11
template <class R> __device__ __forceinline__ const R* geo_row(const MeshDev& M, int e);
template <> __device__ __forceinline__ const double* geo_row<double>(const MeshDev& M, int e) {
  return M.geo + (size_t)e * kGeo;
}
template <> __device__ __forceinline__ const float* geo_row<float>(const MeshDev& M, int e) {
  return M.geof + (size_t)e * kGeo;
}
__device__ __forceinline__ ElemGeom elem_geom(const MeshDev& M, int e) {
  ElemGeom g;
  const double* G = M.geo + (size_t)e * kGeo;
  g.h[0] = G[0]; g.h[1] = G[1]; g.h[2] = G[2];
  g.s = G[3];
  g.is = G[4];
  g.J[0] = G[5]; g.J[1] = G[6]; g.J[2] = G[7];
  g.lo[0] = G[8]; g.lo[1] = G[9]; g.lo[2] = G[10];
  g.sh = G[11];
  return g;
}

// operator entry points (dg_operator.cu)
int op_residual(Handle* h, const double* w, double* f, bool store_lin, cudaStream_t st);
int op_tangent(Handle* h, const double* v, double* out, cudaStream_t st);
int op_linear_part(Handle* h, const double* v, double* out, cudaStream_t st);
// tc = 0: CUDA-core volume pass; 1 / 2: volume contractions on the tensor cores in FP16 / BF16
int op_tangent_f32(Handle* h, const float* v, float* out, int tc, cudaStream_t st);
int op_fd(Handle* h, const double* v, double* out, cudaStream_t st);
int op_project_tgv(Handle* h, double* w, cudaStream_t st);
int op_quad_points(Handle* h, double* xyz, cudaStream_t st);
int op_project_points(Handle* h, const double* vals, double* w, cudaStream_t st);

// tensor-core volume pass of the FP32 Jacobian action (dg_tc_volume.cu)
int tc_prepare_tables(Handle* h);                   // once per handle (allocates)
int tc_prepare_lin(Handle* h, cudaStream_t st);     // per linearisation, after the FP32 cache
int tc_volume_tangent(Handle* h, const float* in, float* out, int tc, cudaStream_t st);

// vector helpers (dg_solvers.cu)
int vec_norm2(Handle* h, const double* x, long long n, double* dev_out, cudaStream_t st);
int launch_axpby(Handle* h, long long n, double a, const double* x, double b, double* y, cudaStream_t st);

// assembly (dg_assemble.cu)
int assemble_all(Handle* h, int precision, cudaStream_t st);
int prepare_lin_fp32(Handle* h, cudaStream_t st);
int level_matvec(Handle* h, int lvl, const double* x, double* y, cudaStream_t st);  // y = G_lvl x

// element-block products streamed through shared memory (dg_blocks.cu). The FP32 cycle keeps
// explicit inverses in Level::LUf (invert_levels_f32 turns the FP32 blocks held there into them).
// status: the word the singular-block flags go to (the assembly's own word, or the handle's)
int invert_levels_f32(Handle* h, cudaStream_t st, unsigned* status);
int staged_jacobi_f(Handle* h, int lvl, const float* g, const float* Gx, float omega, bool x_zero, float* x,
                    int storage, cudaStream_t st);  // x <- (x_zero ? 0 : x) + omega D^-1 (g - Gx); Gx may be null
int prepare_blocks16(Handle* h, int storage, cudaStream_t st);  // LUf, Bsrf -> 16-bit copies
int bsr16_f(Handle* h, int lvl, int storage, float alpha, const float* x, float beta, float* y, cudaStream_t st);
template <class R>
int staged_bsr(Handle* h, int lvl, const R* B, R alpha, const R* x, R beta, R* y, cudaStream_t st);  // -1: n/a

// the preconditioner as the batched solver uses it (dg_solvers.cu)
int solve_opts_check(Handle* h, const dg_solve_opts* o);
int precond_prepare(Handle* h, const dg_solve_opts& o, cudaStream_t st);  // FP32 / 16-bit copies, eagerly
int precond_apply(Handle* h, const dg_solve_opts& o, const double* v, double* z, cudaStream_t st);

// learned coarse correction (dg_learned.cu): x <- s_e N(X_e) on the coarsest level
// (accumulate: x <- x + s_e N(X_e))
template <class R>
int learned_coarse(Handle* h, const R* g, R* x, bool accumulate, cudaStream_t st);
int net_bytes();

}  // namespace dg
