/*
 * dgpmg.h - C ABI of the GB300 (sm_103a) implementation of the matrix-free
 * p-multigrid discontinuous Galerkin hot path of
 *   Franciolini, Botti, Colombo, Crivellini, "p-Multigrid matrix-free
 *   discontinuous Galerkin solution strategies for the under-resolved
 *   simulation of incompressible turbulent flows", arXiv 1809.00866.
 *
 * The library applies the implicit-stage operator G = M/(gamma dt) + dR/dw
 * (Eq. (rosSysOp)) of the DG discretisation of the incompressible
 * Navier-Stokes equations (Eq. (NSdiscr), residual Eq. (NSdiscrRes)) on a
 * periodic box of hexahedra with an orthonormal modal P^k basis, and the
 * p-multigrid preconditioned FGMRES that solves G dw = g (Sec. 2.3-2.4).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - All vector arguments are DEVICE pointers owned by the caller: contiguous
 *    FP64 arrays laid out [element][variable u, v, w, p][mode] with
 *    element e = i + nx*(j + ny*k) and N_b(k) = (k+1)(k+2)(k+3)/6 modes per
 *    variable, ordered by total degree, then by the x exponent descending,
 *    then by the y exponent descending. A level-l vector has N_e*4*N_b(k_l)
 *    entries. Pointers must be 8-byte aligned.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream). Work is enqueued on it; a call returns before the GPU finishes
 *    unless its description says it synchronises.
 *  - The handle owns all internal workspaces (basis tables, linearisation
 *    caches, element block inverses, block-sparse coarse operators, Krylov
 *    bases) and frees them in dg_destroy. Calls on one handle must not
 *    overlap in time (one host thread, one stream at a time).
 *  - Every call returns DG_OK (0) or an error code; nothing aborts, throws
 *    or traps. dg_last_error() gives a text. Device-side conditions (a
 *    Riemann iteration that did not converge, a non-finite value) are
 *    recorded in a status word that dg_get_status() reads.
 */
#ifndef DGPMG_H
#define DGPMG_H

#ifdef __cplusplus
extern "C" {
#endif

#define DG_OK 0
#define DG_ERR_ARG 1            /* invalid argument (size, level, pointer, option) */
#define DG_ERR_CUDA 2           /* a CUDA runtime call failed */
#define DG_ERR_NOT_CONVERGED 3  /* FGMRES did not reach the tolerance within maxit */
#define DG_ERR_RIEMANN 4        /* the star-state iteration did not converge somewhere */
#define DG_ERR_NONFINITE 5      /* a non-finite value was produced */
#define DG_ERR_BOUNDS 6         /* an index check failed */
#define DG_ERR_STATE 7          /* a call was made before what it needs (linearisation, assembly) */

/* Status bits reported by dg_get_status. */
#define DG_STATUS_RIEMANN 1u
#define DG_STATUS_NONFINITE 2u
#define DG_STATUS_WAIT 4u       /* a bounded wait inside a kernel gave up (its work was skipped) */

#define DG_JVP_TANGENT 0 /* exact Jacobian action, Eqs. (jacTrilFnotNU), (jacTrilnu) */
#define DG_JVP_FD 1      /* finite-difference action, Eqs. (matrix-free), (epsdef) */

#define DG_MAX_LEVELS 4

typedef struct dg_params {
  int nx, ny, nz;        /* cells per axis of the periodic box, each >= 2 */
  const double* xn;      /* HOST arrays of nx+1, ny+1, nz+1 increasing node coordinates; copied */
  const double* yn;
  const double* zn;
  int nlevels;           /* p-multigrid levels, 1..DG_MAX_LEVELS */
  int k[DG_MAX_LEVELS];  /* polynomial degree per level: 1 <= k[l] <= 4, strictly decreasing */
  double nu;             /* kinematic viscosity (> 0) */
  double ac_c;           /* artificial-compressibility constant c of the Riemann flux (> 0) */
  double eta;            /* BR2 penalty eta_sigma (> 6 for hexahedra, Sec. 2.1) */
  int walls;             /* DG_WALLS_NONE: periodic in y; DG_WALLS_Y: no-slip walls (data f = 0) at
                            y = yn[0] and y = yn[ny] (Sec. 2.1: Dirichlet viscous flux with the
                            one-sided lifting of [u] = u_K - f, inviscid flux against the ghost
                            state (f, p_K)); x and z stay periodic. ny >= 2 with walls. */
} dg_params;
#define DG_WALLS_NONE 0
#define DG_WALLS_Y 1

typedef struct dg_handle dg_handle;

/* Solver options of fgmres_solve. */
#define DG_PREC_NONE 0
#define DG_PREC_VCYCLE 1  /* one MG_V cycle (Algorithm 2) per outer iteration */
#define DG_PREC_FULLV 2   /* one MG_full cycle (Algorithm 3) per outer iteration */

/* Smoothers of the p-multigrid cycles (Sec. 2.4.3). */
#define DG_SMOOTH_JACOBI 0 /* damped element-block-Jacobi sweeps x <- x + omega D^-1 (g - G x) */
#define DG_SMOOTH_GMRES 1  /* GMRES iterations left-preconditioned by the element block inverses
                              (EWBJ), restarted at every call, from the current iterate; at most
                              DG_SMOOTH_MAX_ITS iterations per call */
#define DG_SMOOTH_MAX_ITS 32

/* Precision of the preconditioner cycle (and of its assembly, dg_assemble_precision). */
#define DG_PRECOND_FP64 0
#define DG_PRECOND_FP32 1 /* block-Jacobi smoothing only */
#define DG_PRECOND_FP32_H16 2  /* the FP32 cycle with its element-block inverses and block-sparse coarse
                                  operators stored in FP16 (IEEE half), products accumulated in FP32 */
#define DG_PRECOND_FP32_BF16 3 /* the same with bfloat16 storage */
#define DG_PRECOND_FP32_H16_TC 4  /* DG_PRECOND_FP32_H16 whose fine-level operator runs the quadrature
                                     contractions of its convective volume term (interpolation of the
                                     velocity variation to the Gauss points, integration of the
                                     weighted products against the basis; Sec. 2.1, Eq. (NSdiscrRes))
                                     as dense per-element GEMMs on the tensor cores: FP16 operands
                                     with per-element power-of-two scaling, FP32 accumulation */
#define DG_PRECOND_FP32_BF16_TC 5 /* the same with bfloat16 block storage and BF16 operands */

/* Coarsest-level SOLVE of the cycles (Sec. 2.4.3 uses a preconditioned GMRES there). */
#define DG_COARSE_SMOOTHER 0 /* coarse_sweeps iterations of the level smoother from zero */
#define DG_COARSE_GMRES 1    /* coarse_sweeps GMRES iterations left-preconditioned by the element
                                block inverses (restarted every DG_SMOOTH_MAX_ITS), from zero; FP64 cycle */
#define DG_COARSE_LEARNED 2  /* the learned per-element correction (dg_set_coarse_network) as the
                                initial iterate, then coarse_sweeps smoother iterations; needs
                                k = 1 on the coarsest level */
#define DG_COARSE_LEARNED_ITER 3 /* x = N(g), then coarse_sweeps iterations x <- x + N(g - G x):
                                    the network as the approximate inverse of a Richardson iteration */

typedef struct dg_solve_opts {
  int restart;       /* Krylov subspace size m before a restart (1..64) */
  int maxit;         /* maximum number of outer iterations */
  double rtol;       /* stop when ||g - G x||_2 <= rtol * ||g - G x0||_2 (recurrence estimate, then checked) */
  int fixed_its;     /* > 0: run exactly this many iterations, no early exit */
  int precond;       /* DG_PREC_* */
  int pre_sweeps;    /* block-Jacobi sweeps before the coarse correction on every non-coarsest level */
  int post_sweeps;   /* ... after it */
  int coarse_sweeps; /* block-Jacobi sweeps from zero that make the coarsest-level SOLVE */
  double omega;      /* block-Jacobi damping (0, 1] */
  int jvp_mode;      /* DG_JVP_TANGENT or DG_JVP_FD for the fine-level G products of the outer solve */
  int x0_is_zero;    /* 1: x holds no initial guess (treated as 0, not read) */
  int smoother;      /* DG_SMOOTH_JACOBI or DG_SMOOTH_GMRES: what the sweep counts above count */
  int precision;     /* DG_PRECOND_FP64, or DG_PRECOND_FP32: the preconditioner cycle (its operator
                        products, block-Jacobi factors, block-sparse coarse operators and vectors) in
                        FP32; FGMRES, its products with G and the true residual stay FP64 */
  int coarse_solver; /* DG_COARSE_SMOOTHER, DG_COARSE_GMRES or DG_COARSE_LEARNED */
  int fallback_its;  /* DG_COARSE_LEARNED(_ITER) only, > 0: from this outer iteration on, if the residual
                        estimate is above fallback_rho^its * r0, the rest of the solve uses
                        DG_COARSE_SMOOTHER. A non-finite Arnoldi vector under the learned
                        correction always redoes that iteration with DG_COARSE_SMOOTHER and keeps it */
  double fallback_rho;
} dg_solve_opts;

typedef struct dg_solve_info {
  int its;              /* outer iterations performed */
  int status;           /* DG_OK or DG_ERR_NOT_CONVERGED */
  double r0;            /* ||g - G x0||_2 */
  double relres_est;    /* recurrence estimate at exit / r0 */
  double true_relres;   /* ||g - G x||_2 / r0 recomputed with the exact G at exit */
  double rho;           /* convergence factor exp(ln(true_relres)/its), Appendix B */
  int fallback_at;      /* outer iteration at which the learned coarse correction was dropped, or -1 */
} dg_solve_info;

/* ---------------------------------------------------------------- handle */

/* Create a handle: copies the mesh, builds the basis/quadrature tables of every
 * level (Gauss-Legendre with k+1 points per direction, Sec. 2.1), and
 * allocates all workspaces on the current device. Synchronises. */
int dg_create(const dg_params* p, dg_handle** out);

/* Free everything the handle owns. Synchronises the device. h may be NULL. */
int dg_destroy(dg_handle* h);

/* Text of the last error on h (or of the last failed dg_create when h is NULL). */
const char* dg_last_error(const dg_handle* h);

/* Size of level lvl: modes per variable and vector length N_e*4*N_b. */
int dg_level_size(const dg_handle* h, int lvl, int* nb, long long* n);

/* Read and clear the device status word (DG_STATUS_* bits). Synchronises `stream`. */
int dg_get_status(dg_handle* h, unsigned* status, void* stream);

/* Test settings of the failure-detection paths. The production values are the defaults;
 * a test changes one, makes the condition happen on the host side of the GPU (no fault, no
 * trap, no endless wait), checks the status or the error code, and restores it.
 *  - DG_KNOB_RIEMANN_ITS (default 60, 0..1000): iteration cap of the star-state solve of the
 *    exact Riemann flux (Sec. 2.1). A face whose iteration does not meet its stopping test
 *    within the cap sets DG_STATUS_RIEMANN; dg_set_linearization then returns DG_ERR_RIEMANN.
 *  - DG_KNOB_WAIT_POLLS (default 0 = 2^22, 0..2^30): polls of each bounded wait of the FP32
 *    cycle's staged block-Jacobi apply before it gives up (DG_STATUS_WAIT).
 *  - DG_KNOB_WITHHOLD_COPY (default 0): != 0 makes that apply leave the first stage of every
 *    CTA uncopied, so that its first wait runs out; the CTA then waits (with the full limit)
 *    for its other copies in flight, sets DG_STATUS_WAIT and skips its work. */
#define DG_KNOB_RIEMANN_ITS 1
#define DG_KNOB_WAIT_POLLS 2
#define DG_KNOB_WITHHOLD_COPY 3
int dg_set_test_knob(dg_handle* h, int knob, long long value);

/* ------------------------------------------------------------- operators */

/* w <- L2 projection (Gauss rule) of the Taylor-Green vortex
 * u = sin x cos y cos z, v = -cos x sin y cos z, w = 0,
 * p = (cos 2x + cos 2y)(cos 2z + 2)/16 onto the fine level. */
int dg_project_tgv(dg_handle* h, double* w, void* stream);

/* Coordinates of the fine level's volume Gauss points: xyz [N_e][(k+1)^3][3] (device), point
 * q = (q0 (k+1) + q1)(k+1) + q2 with q0, q1, q2 the Gauss-node indices along x, y, z. */
int dg_quad_points(dg_handle* h, double* xyz, void* stream);

/* w <- the L2 projection (Gauss rule) onto the fine level of a field given by its values at the
 * points of dg_quad_points: vals [N_e][4][(k+1)^3] (device; u, v, w, p). */
int dg_project_points(dg_handle* h, const double* vals, double* w, void* stream);

/* f <- f_h(w; phi_m e_i) for every test function (Eq. (NSdiscrRes)): volume
 * terms with the BR2 corrected gradient grad u - R^K(u), face terms with the
 * exact artificial-compressibility Riemann flux and the BR2 viscous flux
 * F^nu({grad u - eta r^s([u])}) (Eq. (vflux), Sec. 2.1). Fine level. w and f
 * must not alias. Asynchronous: a non-finite output entry sets DG_STATUS_NONFINITE and a
 * star-state iteration that missed its stopping test sets DG_STATUS_RIEMANN (dg_get_status). */
int dg_residual(dg_handle* h, const double* w, double* f, void* stream);

/* Fix the linearisation state of G: caches w, f_h(w), ||w||_2, the velocity
 * at the volume quadrature points and the Jacobian of the Riemann flux at the
 * face points, and sets 1/(gamma dt) (>= 0). Synchronises (reads ||w||). Returns
 * DG_ERR_NONFINITE if w or f_h(w) has a non-finite entry and DG_ERR_RIEMANN if the star-state
 * iteration missed its stopping test on some face; the handle is then not linearised, and the
 * condition's bit is also left in the status word. */
int dg_set_linearization(dg_handle* h, const double* w, double inv_gamma_dt, void* stream);

/* dg_set_linearization that also writes the right-hand side of the stage started from w,
 * g <- -f_h(w) (Eq. (rosSysOp) with no earlier stages), from the residual it evaluates anyway:
 * one nonlinear face pass (exact Riemann solves) per stage instead of two. g must not alias w. */
int dg_set_linearization_rhs(dg_handle* h, const double* w, double inv_gamma_dt, double* g, void* stream);

/* out <- G v = J(w) v + (1/(gamma dt)) M v on the fine level, M the
 * velocity-only mass form (Eq. (massBil)). mode DG_JVP_TANGENT: exact
 * linearisation (Eqs. (jacTrilFnotNU), (jacTrilnu)); DG_JVP_FD:
 * (f(w + D v) - f(w))/D with D = 1e-9 sqrt(1 + ||w||)/||v|| (Eqs.
 * (matrix-free), (epsdef)). Needs dg_set_linearization. v and out must not alias. */
int dg_jvp(dg_handle* h, const double* v, double* out, int mode, void* stream);

/* Assemble the preconditioner at the current linearisation: the element
 * diagonal blocks of G on every level and their inverses (element-wise block
 * Jacobi, Sec. 2.3), and the inherited block-sparse coarse operators of levels
 * >= 1 (Galerkin projection = sub-block extraction with a hierarchical
 * orthonormal basis, Eq. (GalProj)); off-diagonal blocks are built at the
 * degree of level 1 only (Sec. 2.4.3). Synchronises. */
int dg_assemble(dg_handle* h, void* stream);

/* dg_assemble in the precision of the preconditioner that will use it (DG_PRECOND_FP32_H16 and
 * _BF16 assemble as DG_PRECOND_FP32; their 16-bit block copies are rounded from it at first use):
 * DG_PRECOND_FP64 (= dg_assemble; also usable by the FP32 cycle after rounding), or
 * DG_PRECOND_FP32: the state-dependent blocks, the inherited coarse blocks and the LU
 * factors are computed in FP32 (the mesh-only linear part is probed once in FP64), for
 * the FP32 preconditioner cycle only. Synchronises. */
int dg_assemble_precision(dg_handle* h, int precision, void* stream);

/* Rescaled-inherited coarse operators (Appendix A): enable != 0 makes every later assembly
 * weight the viscous stabilisation part (the BR2 penalty terms, the part of G proportional to
 * eta) of each inherited coarse operator by S_0^l = k_l (k_l + 3) / (k_0 (k_0 + 3)):
 * G_l = M (G_0 - G_stb) M^T + S_0^l M G_stb M^T. The fine level is unchanged. The first
 * assembly after enabling probes G_stb's level-1 block rows once (G(eta) - G(0), FP64).
 * Off by default (plain Galerkin inheritance). Invalidates the current assembly. */
int dg_set_stb_rescaling(dg_handle* h, int enable);

/* Preconditioner lagging (Sec. 4.1, T3L1 case): keep the element blocks, their factors and the
 * coarse block-sparse operators assembled at an earlier linearisation for the current one (the
 * paper freezes them for several time steps). The matrix-free fine-level products of the cycle
 * and of FGMRES still use the current linearisation. DG_ERR_STATE if nothing has been assembled. */
int dg_reuse_assembly(dg_handle* h);

/* ------------------------------------------------------------ p-multigrid */

/* xc <- restriction of level-lvl vector xf to level lvl+1 (L2 projection =
 * keep the leading modes, Sec. 2.4.1). */
int pmg_restrict(dg_handle* h, int lvl, const double* xf, double* xc, void* stream);

/* xf <- xf + prolongation of level-(lvl+1) vector xc (injection = zero-pad, Sec. 2.4.1). */
int pmg_prolong(dg_handle* h, int lvl, const double* xc, double* xf, void* stream);

/* `sweeps` damped element-block-Jacobi iterations x <- x + omega D^{-1}(g - G x)
 * on level lvl (lvl 0: G v matrix-free, exact mode; lvl >= 1: block-sparse G).
 * Needs dg_assemble. x is read and updated in place. */
int block_jacobi_smooth(dg_handle* h, int lvl, const double* g, double* x, int sweeps, double omega,
                        void* stream);

/* y <- alpha G_lvl x + beta y with the assembled block-sparse coarse operator
 * of level lvl >= 1 (diagonal + one block per face). */
int bsr_spmv(dg_handle* h, int lvl, double alpha, const double* x, double beta, double* y, void* stream);

/* y <- alpha G_lvl^T x + beta y with the transpose of the assembled block-sparse coarse operator
 * of level lvl >= 1 (used to train the learned coarse correction on the coarse residual). */
int bsr_spmv_t(dg_handle* h, int lvl, double alpha, const double* x, double beta, double* y, void* stream);

/* x <- MG_V(0, g, 0) (Algorithm 2) with the smoothing options of opts; the
 * coarsest-level SOLVE is opts->coarse_sweeps iterations of the smoother from zero. */
int pmg_vcycle(dg_handle* h, const double* g, double* x, const dg_solve_opts* opts, void* stream);

/* Solve G x = g with right-preconditioned flexible GMRES(restart) (Sec.
 * 2.4.3, Saad 1993), classical Gram-Schmidt with one re-orthogonalisation,
 * FP64 throughout. x holds the initial guess unless opts->x0_is_zero.
 * Synchronises. info may be NULL. Returns DG_ERR_NOT_CONVERGED (with x the
 * last iterate) if the tolerance was not met. */
int fgmres_solve(dg_handle* h, const double* g, double* x, const dg_solve_opts* opts, dg_solve_info* info,
                 void* stream);

/* Solve G_lvl x = g on a coarse level lvl >= 1 with its assembled block-sparse operator by
 * GMRES(DG_SMOOTH_MAX_ITS) left-preconditioned by the element block inverses, restarted,
 * until ||g - G x||_2 <= rtol ||g - G x0||_2 or maxit iterations (the coarse solver of Sec.
 * 2.4.3 run to a tolerance). x0 = 0 when x0_is_zero. FP64; needs an FP64 dg_assemble.
 * Synchronises once per restart. info (may be NULL): its, r0, true_relres, status. */
int pmg_level_solve(dg_handle* h, int lvl, const double* g, double* x, double rtol, int maxit, int x0_is_zero,
                    dg_solve_info* info, void* stream);

/* x <- x - (c.x / c.c) c on level lvl, with c the constant-pressure vector (coefficient
 * sqrt|K_e| on the pressure mode 0 of every element, zero elsewhere). On a periodic box c spans
 * the null space of G (a constant pressure has no gradient and no jump) and, read as test-function
 * integrals, its left null space (the continuity residuals integrate to zero), so this projection
 * makes a right-hand side consistent and removes the arbitrary constant from a solution. */
int pmg_project_pressure(dg_handle* h, int lvl, double* x, void* stream);

/* --------------------------------------------------- learned coarse correction
 * The paper has no learned component. These calls add a per-element network that
 * stands in for the coarsest (P1) SOLVE of the cycles:
 *   x_e = s_e * N(X_e),  X_e = F_e / s_e,  s_e = ||F_e||_2  (x_e = 0 where s_e = 0),
 * F_e = the coarsest-level right-hand side of element e followed by that of its six face
 * neighbours (order -x, +x, -y, +y, -z, +z), 7 x 4 variables x 4 modes = 112 values;
 * N(X) = W3 gelu(W2 gelu(W1 X + b1) + b2) + b3 with gelu(t) = t (1 + erf(t/sqrt 2))/2.
 * Parameters: one FP32 vector theta of DG_MLP_NPARAM entries, in the order W1 [128][112],
 * b1 [128], W2 [128][128], b2 [128], W3 [16][128], b3 [16] (row-major, [out][in]).
 * Every evaluation uses BF16 weights and layer inputs (round to nearest even) on the tensor
 * cores with FP32 accumulation; biases and activations are FP32. */
#define DG_MLP_IN 112
#define DG_MLP_HIDDEN 128
#define DG_MLP_OUT 16
#define DG_MLP_NPARAM 33040

/* Bytes of the device workspace that dg_mlp_forward / dg_mlp_grad need for `rows` rows. */
long long dg_mlp_workspace_bytes(long long rows);

/* Y [n][16] <- N(X [n][112]) (features used as given). theta, X, Y, ws: device pointers, ws of
 * dg_mlp_workspace_bytes(n) bytes, 16-byte aligned. */
int dg_mlp_forward(const float* theta, const float* X, long long n, float* Y, void* ws, void* stream);

/* Loss L = (1/B) sum_s ||N(X_r(s)) - T_r(s)||_2^2 over a batch of B rows and its gradient
 * grad [DG_MLP_NPARAM] = dL/dtheta (BF16 operands, FP32 accumulation, fixed reduction order).
 * Rows: seed < 0: r(s) = s (B <= npairs); seed >= 0: r(s) drawn uniformly from [0, npairs)
 * by a counter-based hash of (seed, step, s). X [npairs][112], T [npairs][16]. loss: device
 * scalar (may be NULL). ws of dg_mlp_workspace_bytes(B) bytes. */
int dg_mlp_grad(const float* theta, const float* X, const float* T, long long npairs, int batch, long long seed,
                long long step, float* grad, float* loss, void* ws, void* stream);

/* One Adam step (Kingma & Ba 2015) on theta with moments m, v (all DG_MLP_NPARAM FP32,
 * device): t >= 1 is the step number used in the bias corrections. */
int dg_mlp_adam(float* theta, const float* grad, float* m, float* v, long long t, double lr, double beta1,
                double beta2, double eps, void* stream);

/* Set (copy, rounded to BF16) the network of DG_COARSE_LEARNED from device theta; NULL unsets it. */
int dg_set_coarse_network(dg_handle* h, const float* theta, void* stream);

/* x <- s_e N(X_e(d)) (accumulate = 0) or x + s_e N(X_e(d)) on the coarsest level (FP64 vectors;
 * the network of dg_set_coarse_network). */
int dg_coarse_apply(dg_handle* h, const double* d, double* x, int accumulate, void* stream);

/* Training pairs of the coarsest level from a right-hand side d and a coarsest-level vector x:
 * X [ne][112] the normalised features of d, s [ne] their norms and T [ne][16] = x_e / s_e +
 * s_e q_e (FP32, device; q may be NULL = 0; rows with s_e = 0 are zero). Needs k = 1 there.
 *  - supervised targets: x = the solution of G x = d, q = NULL;
 *  - residual targets: x = s N(X) (dg_coarse_apply) and q = G^T (d - G x) (bsr_spmv_t): then the
 *    gradient of the squared error ||N(X) - T||^2 with respect to N(X) is the gradient of the
 *    coarse residual ||d - G x||^2 (times a constant), so dg_mlp_grad trains N as a local
 *    approximate inverse of the coarse operator. */
int dg_coarse_pairs(dg_handle* h, const double* d, const double* x, const double* q, float* X, float* T, float* s,
                    void* stream);

/* Record the right-hand sides that the cycles pass to the coarsest-level SOLVE: each one
 * is copied (as FP64) into buf [capacity][n_coarsest] in call order until capacity is
 * reached; buf = NULL stops recording. dg_recorded reads how many were stored. */
int dg_record_coarse(dg_handle* h, double* buf, int capacity);
int dg_recorded(const dg_handle* h, int* count);

/* ------------------------------------------------- residual without allocation
 * The paper has no counterpart of this call; it serves callers that must not
 * allocate device memory at the point where they evaluate the residual: a host
 * application or framework that owns the whole device memory budget and forbids
 * its plugins to call cudaMalloc, or code running where an allocation would
 * synchronise the device or fail because the memory is already committed.
 *
 * dg_residual_noalloc computes exactly what dg_residual computes (same kernels)
 * but keeps the face-pass scratch (N_e * 6 * 7 * N_2 doubles, N_2 = (k_0+1)(k_0+2)/2) in a
 * file-scope device array of DG_NOALLOC_SCRATCH_DOUBLES doubles (8 MiB) instead of
 * the handle's buffers. It calls no cudaMalloc, cudaFree or allocating routine.
 *  - Meshes needing more scratch than that return DG_ERR_ARG with the sizes in
 *    the error text (at k = 4: up to 1664 elements; at k = 2: up to 4161).
 *  - The first call on a device looks the array's device address up
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture.
 *  - Every call on a device shares the one array, which keeps the last call's
 *    contents (nothing in it needs to start at zero: every entry is written
 *    before it is read). Calls that overlap on the GPU, from any handle or
 *    stream, race on it.
 *  - Every GPU that loads the library holds the array until the process exits.
 *  - The handle's device (current at its dg_create) must be current at the call, else
 *    DG_ERR_ARG; the address is looked up for that device.
 *  - The looked-up address belongs to the device's context: after cudaDeviceReset (which also
 *    frees every handle's buffers) the entry point must not be called again in this process.
 * The handle must come from dg_create as usual; w and f as for dg_residual. */
#define DG_NOALLOC_SCRATCH_DOUBLES (1 << 20)
int dg_residual_noalloc(dg_handle* h, const double* w, double* f, void* stream);

/* w <- w + b dw on the fine level: the state update of a linearly implicit stage (Sec. 2.2,
 * w^{n+1} = w^n + sum_i b_i dw_i; one stage with b = 1 here). w and dw must not alias. */
int dg_stage_update(dg_handle* h, double* w, const double* dw, double b, void* stream);

/* ---------------------------------------------------------- measured peaks
 * The paper has no counterpart. Throughput of the device's FP64 or FP32 fused multiply-add
 * pipe (TFLOP/s, FMA = 2 FLOP), measured with eight independent FMA chains per thread in a grid
 * of 8 x 256-thread CTAs per SM on the current device: the best of three timed launches after a
 * warm-up one (CUDA events on `stream`). The denominators of the ALU rooflines.
 * DG_PEAK_HBM_READ: the bandwidth (GB/s, written to *tflops) of a read-only stream of 16-byte
 * loads over a 2 GiB buffer (allocated and freed by the call). Synchronises. */
#define DG_PEAK_FP64_FMA 0
#define DG_PEAK_FP32_FMA 1
#define DG_PEAK_HBM_READ 2
int dg_measure_peak(int which, double* tflops, void* stream);

/* ----------------------------------------------------------------- batching
 * Many independent implicit-stage solves at once. The paper solves one system per process
 * group (Sec. 2.3); on one GPU, small problems leave most of the device idle, so a handle can
 * hold several independent periodic boxes and a plan solves all of them together. */

/* Create a handle holding nprob independent periodic boxes with the degrees, viscosity,
 * constant and penalty of p (p->nx, ny, nz, xn, yn, zn are ignored).
 *  - dims: HOST [nprob][3] cells per axis of each box, each >= 2.
 *  - nodes: HOST array with, box after box, the nx+1, then ny+1, then nz+1 increasing node
 *    coordinates of that box; copied.
 * Elements are numbered box after box (x fastest within a box), so every vector of the handle
 * is the concatenation of the boxes' vectors; dg_problems gives the offsets. Face neighbours
 * stay within a box. Every element kernel acts on all boxes in one launch. Calls that reduce
 * over the whole vector (fgmres_solve, DG_JVP_FD, the GMRES smoother or coarse solve,
 * pmg_level_solve, pmg_project_pressure) return DG_ERR_ARG on a handle of nprob > 1; it is
 * solved by dg_plan_solve. Synchronises. */
int dg_create_batch(const dg_params* p, int nprob, const int* dims, const double* nodes, dg_handle** out);

/* Number of problems of h and, if elem_start is not NULL, the HOST array [nprob + 1] of their
 * first elements (elem_start[nprob] = N_e). */
int dg_problems(const dg_handle* h, int* nprob, int* elem_start);

/* Per-problem multipliers of the mass shift: problem q solves with 1/(gamma dt_q) =
 * mult[q] * inv_gamma_dt of dg_set_linearization (default 1). mult: HOST [nprob], finite and
 * >= 0. The assembled preconditioner holds the shift: assemble again after this call. */
int dg_set_problem_shifts(dg_handle* h, const double* mult, void* stream);

/* A plan: FGMRES(m) right-preconditioned by the options' cycle for every problem of nh
 * handles, each problem with its own Krylov space, Hessenberg matrix, Givens rotations and
 * stopping test ||g_q - G_q x_q|| <= rtol ||g_q - G_q x0_q|| (Sec. 2.3). All problems of a
 * handle advance in lockstep (a converged problem stops contributing); the reductions are per
 * problem in a fixed order. The Givens rotations, the tests and the triangular solves run on
 * the device, so a restart cycle needs no host synchronisation.
 *  - hs[i], g[i], x[i]: distinct handles and their device vectors (g[i] != x[i]); kept by the
 *    plan, which must be destroyed before them.
 *  - opts: as for fgmres_solve, with DG_JVP_TANGENT, block-Jacobi smoothing and the smoother
 *    (or learned, no fallback) coarse solve.
 *  - use_graph != 0: the first dg_plan_solve captures the restart cycle of every handle as one
 *    CUDA graph: the handles become parallel branches, and the Arnoldi step is the body of a
 *    conditional WHILE node (continue while some problem of the handle is active and j < m).
 *    Every later solve replays it: one graph launch per restart cycle for the whole batch.
 *    The graph keeps the pointers of g, x and the handles' buffers; the state, the assembly
 *    and the vectors' contents may change between solves.
 *  - use_graph == 0: the same kernels launched one by one, with the loop condition read on
 *    the host after every step.
 * Allocates the Krylov workspaces ((2m+6) vectors per handle plus small arrays). */
typedef struct dg_plan dg_plan;
int dg_plan_create(int nh, dg_handle* const* hs, const double* const* g, double* const* x,
                   const dg_solve_opts* opts, int use_graph, dg_plan** out);

/* Solve with the current linearisation and assembly of every handle (x[i] is the initial guess
 * unless opts.x0_is_zero). Synchronises. DG_ERR_NOT_CONVERGED when some problem missed the
 * tolerance within opts.maxit steps, DG_ERR_NONFINITE when a Krylov quantity was not finite. */
int dg_plan_solve(dg_plan* plan, void* stream);

/* Per-problem outcome of handle i's problems after the last solve (HOST arrays of nprob
 * entries, each may be NULL): Arnoldi steps, true relative residual, converged flag. */
int dg_plan_result(const dg_plan* plan, int i, int* its, double* relres, int* converged);

/* Restart cycles and maximal Arnoldi steps of the last solve; graph launches so far. */
int dg_plan_stats(const dg_plan* plan, int* cycles, int* steps, long long* graph_launches);

/* Text of the last error of plan (or of the last failed dg_plan_create when plan is NULL). */
const char* dg_plan_error(const dg_plan* plan);

int dg_plan_destroy(dg_plan* plan);

/* ------------------------------------------------------------ launch shapes
 * The paper's kernels are CPU loops; here the launch shapes of the hot GPU kernels are chosen per
 * (degree k, quadrature size N_q = (k+1)^3) and mesh size. None of them changes a result: every
 * output entry is computed by the same arithmetic in the same order for every shape. */
#define DG_TUNE_FP64 0  /* the FP64 Jacobian action (outer FGMRES products, FP64 cycle) */
#define DG_TUNE_FP32 1  /* the FP32 Jacobian action and block-Jacobi apply of the FP32 cycle */
typedef struct dg_tuning {
  int face_warps;        /* faces per CTA of the face pass (one warp each): 2, 4 or 8 (default 4) */
  int vol_threads;       /* threads per CTA of the volume pass (one element per CTA): 64, 128, 160, 192
                            or 256 (128) */
  int face_ctas_per_sm;  /* cap on resident CTAs per SM of the face pass, 0..32 (0: shared memory decides) */
  int vol_ctas_per_sm;   /* the same for the volume pass */
  int jacobi_stage_kb;   /* FP32 cycle: KB of element inverses per bulk-copy stage of the fine-level
                            block-Jacobi apply, 8..224 (96); capped by shared memory */
  int jacobi_max_ctas;   /* cap on the CTAs of that apply, 0..4096 (0: no cap, one wave of the GPU). A
                            small cap makes every CTA take many stages through its ring of stage
                            buffers (the stage size then also shrinks to keep >= 2 stages per CTA);
                            the autotuner leaves it as set */
} dg_tuning;

int dg_get_tuning(const dg_handle* h, int which, dg_tuning* t);

/* Set the shapes of class `which`. A plan captured as a graph keeps the shapes it was captured
 * with. DG_ERR_ARG outside the listed values. */
int dg_set_tuning(dg_handle* h, int which, const dg_tuning* t);

/* Measure the candidate shapes on h (CUDA events around the real kernels at h's current
 * linearisation; for DG_TUNE_FP32 the block-Jacobi stages too when an FP32 assembly exists) and
 * keep the fastest per kernel. The candidates: face_warps 2/4/8; vol_threads 64/128/160/192/256 with no
 * CTA cap and with 4 CTAs per SM; jacobi_stage_kb 48/96/144/200. use_cache != 0: reuse the result
 * of an earlier call in this process on the same (which, k, N_q, SM count, log2 N_e, block
 * storage). report: NULL or HOST [6] = device ms per launch of the default and of the chosen face
 * pass, volume pass and block-Jacobi apply (0 where not measured or taken from the cache).
 * Overwrites the level-0 work vectors; keeps the profiler's accumulated counts. Synchronises. */
int dg_autotune(dg_handle* h, int which, int use_cache, double* report, void* stream);

/* --------------------------------------------------------- instrumentation
 * The paper profiles its solver per linear system (Sec. 3.1: code profiling
 * over 10 time steps); these calls expose the same information per kernel. */

/* Kernel classes timed by the profiler. */
#define DG_PROF_FACE_RES 0  /* face pass of f_h (and of the linearisation) */
#define DG_PROF_VOL_RES 1   /* volume pass of f_h */
#define DG_PROF_FACE_TAN 2  /* face pass of the exact Jacobian action */
#define DG_PROF_VOL_TAN 3   /* volume pass of the exact Jacobian action */
#define DG_PROF_FACE_TAN32 4 /* face pass of the FP32 Jacobian action (reduced-precision preconditioner) */
#define DG_PROF_VOL_TAN32 5  /* volume pass of the FP32 Jacobian action */
#define DG_PROF_BJ32 6       /* fine-level block-Jacobi apply of the FP32 cycle (explicit inverses) */
#define DG_PROF_BSR32 7      /* level-1 block-sparse product of the FP32 cycle */
#define DG_PROF_BJ64 8       /* fine-level block-Jacobi apply of the FP64 cycle (LU factors) */
#define DG_PROF_BSR64 9      /* level-1 block-sparse product of the FP64 cycle */
#define DG_PROF_VOL_TC32 10  /* volume pass of the FP32 Jacobian action with tensor-core contractions */
#define DG_PROF_N 11

/* Counters since dg_create: kernels launched by the library, and applications
 * of the fine-level operator (residual or Jacobian action). Host-only, no sync. */
int dg_counters(const dg_handle* h, long long* kernel_launches, long long* operator_applications);

/* enable != 0: bracket every launch of the timed kernel classes with CUDA
 * events recorded on the launching stream. Costs two event records per launch. */
int dg_profile(dg_handle* h, int enable);

/* Accumulated device time (ms) and launch count per kernel class since the
 * last read (arrays of DG_PROF_N entries); resets them. Synchronises the
 * device. */
int dg_profile_read(dg_handle* h, double* ms, long long* counts);

/* dg_profile_read plus the algorithmic HBM bytes of the timed launches per class (each value
 * read and each value written once: the blocks, the input and output vectors; for the operator
 * classes 0-5 nothing is counted and 0 is returned). bytes: DG_PROF_N entries. */
int dg_profile_read_bytes(dg_handle* h, double* ms, long long* counts, double* bytes);

#ifdef __cplusplus
}
#endif
#endif /* DGPMG_H */
