"""GB300 (sm_103a) implementation of the matrix-free p-multigrid DG hot path of arXiv 1809.00866.

The compute path is the C-ABI CUDA library ``libdgpmg.so`` (``include/dgpmg.h``);
this package only builds it, loads it with ctypes and marshals torch tensors
(device memory) and CUDA streams into its plain-pointer calls. Every step of
the path runs in the library's kernels. There is no CPU fallback: loading
fails loudly when the library is missing or no GPU is present.
"""
import ctypes
import os

from ._build_lib import LIB, build  # noqa: F401

DG_OK = 0
DG_ERR_ARG = 1
DG_ERR_CUDA = 2
DG_ERR_NOT_CONVERGED = 3
DG_ERR_RIEMANN = 4
DG_ERR_NONFINITE = 5
DG_ERR_BOUNDS = 6
DG_ERR_STATE = 7
DG_STATUS_RIEMANN = 1
DG_STATUS_NONFINITE = 2
DG_JVP_TANGENT = 0
DG_JVP_FD = 1
DG_PREC_NONE = 0
DG_PREC_VCYCLE = 1
DG_PREC_FULLV = 2
DG_SMOOTH_JACOBI = 0
DG_SMOOTH_GMRES = 1
DG_PRECOND_FP64 = 0
DG_PRECOND_FP32 = 1
DG_PRECOND_FP32_H16 = 2
DG_PRECOND_FP32_BF16 = 3
DG_PRECOND_FP32_H16_TC = 4
DG_PRECOND_FP32_BF16_TC = 5
DG_COARSE_SMOOTHER = 0
DG_COARSE_GMRES = 1
DG_COARSE_LEARNED = 2
DG_COARSE_LEARNED_ITER = 3
DG_STATUS_WAIT = 4
DG_KNOB_RIEMANN_ITS = 1
DG_KNOB_WAIT_POLLS = 2
DG_KNOB_WITHHOLD_COPY = 3
DG_PEAK_FP64_FMA = 0
DG_PEAK_FP32_FMA = 1
DG_PEAK_HBM_READ = 2
DG_MAX_LEVELS = 4
DG_SMOOTH_MAX_ITS = 32
DG_MLP_IN = 112
DG_MLP_HIDDEN = 128
DG_MLP_OUT = 16
DG_MLP_NPARAM = 33040

# Every exported symbol of include/dgpmg.h
EXPORTS = ("dg_create", "dg_destroy", "dg_last_error", "dg_level_size", "dg_get_status", "dg_project_tgv",
           "dg_residual", "dg_set_linearization", "dg_jvp", "dg_assemble", "pmg_restrict", "pmg_prolong",
           "block_jacobi_smooth", "bsr_spmv", "pmg_vcycle", "fgmres_solve", "dg_counters", "dg_profile",
           "dg_profile_read", "dg_residual_noalloc", "dg_assemble_precision", "pmg_level_solve",
           "dg_mlp_workspace_bytes", "dg_mlp_forward", "dg_mlp_grad", "dg_mlp_adam", "dg_set_coarse_network",
           "dg_coarse_pairs", "dg_record_coarse", "dg_recorded", "pmg_project_pressure",
           "bsr_spmv_t", "dg_coarse_apply", "dg_profile_read_bytes",
           "dg_reuse_assembly", "dg_set_linearization_rhs", "dg_set_stb_rescaling",
           "dg_create_batch", "dg_problems", "dg_set_problem_shifts", "dg_plan_create", "dg_plan_solve",
           "dg_plan_result", "dg_plan_stats", "dg_plan_error", "dg_plan_destroy",
           "dg_get_tuning", "dg_set_tuning", "dg_autotune", "dg_quad_points", "dg_project_points",
           "dg_set_test_knob", "dg_stage_update", "dg_measure_peak")
DG_WALLS_NONE = 0
DG_WALLS_Y = 1
DG_TUNE_FP64 = 0
DG_TUNE_FP32 = 1
DG_PROF_N = 11
PROF_NAMES = ("face_res", "vol_res", "face_tan", "vol_tan", "face_tan32", "vol_tan32", "bj32_fine", "bsr32_l1",
              "bj64_fine", "bsr64_l1", "vol_tc32")


class DgParams(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("xn", ctypes.POINTER(ctypes.c_double)), ("yn", ctypes.POINTER(ctypes.c_double)),
                ("zn", ctypes.POINTER(ctypes.c_double)), ("nlevels", ctypes.c_int),
                ("k", ctypes.c_int * DG_MAX_LEVELS), ("nu", ctypes.c_double), ("ac_c", ctypes.c_double),
                ("eta", ctypes.c_double), ("walls", ctypes.c_int)]


class DgSolveOpts(ctypes.Structure):
    _fields_ = [("restart", ctypes.c_int), ("maxit", ctypes.c_int), ("rtol", ctypes.c_double),
                ("fixed_its", ctypes.c_int), ("precond", ctypes.c_int), ("pre_sweeps", ctypes.c_int),
                ("post_sweeps", ctypes.c_int), ("coarse_sweeps", ctypes.c_int), ("omega", ctypes.c_double),
                ("jvp_mode", ctypes.c_int), ("x0_is_zero", ctypes.c_int), ("smoother", ctypes.c_int),
                ("precision", ctypes.c_int), ("coarse_solver", ctypes.c_int), ("fallback_its", ctypes.c_int),
                ("fallback_rho", ctypes.c_double)]


class DgTuning(ctypes.Structure):
    _fields_ = [("face_warps", ctypes.c_int), ("vol_threads", ctypes.c_int), ("face_ctas_per_sm", ctypes.c_int),
                ("vol_ctas_per_sm", ctypes.c_int), ("jacobi_stage_kb", ctypes.c_int), ("jacobi_max_ctas", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class DgSolveInfo(ctypes.Structure):
    _fields_ = [("its", ctypes.c_int), ("status", ctypes.c_int), ("r0", ctypes.c_double),
                ("relres_est", ctypes.c_double), ("true_relres", ctypes.c_double), ("rho", ctypes.c_double),
                ("fallback_at", ctypes.c_int)]


_lib = None


def load(path=None):
    """Load libdgpmg.so (build it first with ``build()``); raises if it is missing."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    path = path or LIB
    if not os.path.exists(path):
        raise RuntimeError("dgpmg CUDA library not built (%s); run paper_1809_00866_gb300.build()" % path)
    L = ctypes.CDLL(path)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    L.dg_create.argtypes = [ctypes.POINTER(DgParams), ctypes.POINTER(vp)]
    L.dg_destroy.argtypes = [vp]
    L.dg_last_error.argtypes = [vp]
    L.dg_last_error.restype = ctypes.c_char_p
    L.dg_level_size.argtypes = [vp, i, ctypes.POINTER(i), ctypes.POINTER(ctypes.c_longlong)]
    L.dg_get_status.argtypes = [vp, ctypes.POINTER(ctypes.c_uint), vp]
    L.dg_project_tgv.argtypes = [vp, vp, vp]
    L.dg_residual.argtypes = [vp, vp, vp, vp]
    L.dg_set_linearization.argtypes = [vp, vp, d, vp]
    L.dg_jvp.argtypes = [vp, vp, vp, i, vp]
    L.dg_assemble.argtypes = [vp, vp]
    L.pmg_restrict.argtypes = [vp, i, vp, vp, vp]
    L.pmg_prolong.argtypes = [vp, i, vp, vp, vp]
    L.block_jacobi_smooth.argtypes = [vp, i, vp, vp, i, d, vp]
    L.bsr_spmv.argtypes = [vp, i, d, vp, d, vp, vp]
    L.pmg_vcycle.argtypes = [vp, vp, vp, ctypes.POINTER(DgSolveOpts), vp]
    L.fgmres_solve.argtypes = [vp, vp, vp, ctypes.POINTER(DgSolveOpts), ctypes.POINTER(DgSolveInfo), vp]
    L.dg_residual_noalloc.argtypes = [vp, vp, vp, vp]
    L.dg_assemble_precision.argtypes = [vp, i, vp]
    ll, f32p = ctypes.c_longlong, ctypes.c_void_p
    L.pmg_level_solve.argtypes = [vp, i, vp, vp, d, i, i, ctypes.POINTER(DgSolveInfo), vp]
    L.dg_mlp_workspace_bytes.argtypes = [ll]
    L.dg_mlp_forward.argtypes = [vp, vp, ll, vp, vp, vp]
    L.dg_mlp_grad.argtypes = [vp, vp, vp, ll, i, ll, ll, vp, vp, vp, vp]
    L.dg_mlp_adam.argtypes = [vp, vp, vp, vp, ll, d, d, d, d, vp]
    L.dg_set_coarse_network.argtypes = [vp, vp, vp]
    L.dg_coarse_pairs.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
    L.bsr_spmv_t.argtypes = [vp, i, d, vp, d, vp, vp]
    L.dg_coarse_apply.argtypes = [vp, vp, vp, i, vp]
    L.dg_record_coarse.argtypes = [vp, vp, i]
    L.dg_recorded.argtypes = [vp, ctypes.POINTER(i)]
    L.pmg_project_pressure.argtypes = [vp, i, vp, vp]
    L.dg_counters.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]
    L.dg_profile.argtypes = [vp, i]
    L.dg_profile_read.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)]
    L.dg_profile_read_bytes.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong),
                                        ctypes.POINTER(ctypes.c_double)]
    L.dg_reuse_assembly.argtypes = [vp]
    L.dg_set_stb_rescaling.argtypes = [vp, i]
    L.dg_set_linearization_rhs.argtypes = [vp, vp, d, vp, vp]
    L.dg_create_batch.argtypes = [ctypes.POINTER(DgParams), i, ctypes.POINTER(i), ctypes.POINTER(d),
                                  ctypes.POINTER(vp)]
    L.dg_problems.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(i)]
    L.dg_set_problem_shifts.argtypes = [vp, ctypes.POINTER(d), vp]
    L.dg_plan_create.argtypes = [i, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                 ctypes.POINTER(DgSolveOpts), i, ctypes.POINTER(vp)]
    L.dg_plan_solve.argtypes = [vp, vp]
    L.dg_plan_result.argtypes = [vp, i, ctypes.POINTER(i), ctypes.POINTER(d), ctypes.POINTER(i)]
    L.dg_plan_stats.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(ctypes.c_longlong)]
    L.dg_plan_error.argtypes = [vp]
    L.dg_plan_error.restype = ctypes.c_char_p
    L.dg_plan_destroy.argtypes = [vp]
    L.dg_quad_points.argtypes = [vp, vp, vp]
    L.dg_project_points.argtypes = [vp, vp, vp, vp]
    L.dg_get_tuning.argtypes = [vp, i, ctypes.POINTER(DgTuning)]
    L.dg_set_tuning.argtypes = [vp, i, ctypes.POINTER(DgTuning)]
    L.dg_autotune.argtypes = [vp, i, i, ctypes.POINTER(d), vp]
    L.dg_set_test_knob.argtypes = [vp, i, ctypes.c_longlong]
    L.dg_stage_update.argtypes = [vp, vp, vp, d, vp]
    L.dg_measure_peak.argtypes = [i, ctypes.POINTER(d), vp]
    for name in EXPORTS:
        if name not in ("dg_last_error", "dg_plan_error"):
            getattr(L, name).restype = ctypes.c_int
    L.dg_mlp_workspace_bytes.restype = ctypes.c_longlong
    _lib = L
    return L


class DgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("dgpmg error %d: %s" % (code, msg))
        self.code = code


def solve_opts(restart=30, maxit=200, rtol=1e-8, fixed_its=0, precond=DG_PREC_VCYCLE, pre_sweeps=2,
               post_sweeps=2, coarse_sweeps=2, omega=1.0, jvp_mode=DG_JVP_TANGENT, x0_is_zero=1,
               smoother=DG_SMOOTH_JACOBI, precision=DG_PRECOND_FP64, coarse_solver=DG_COARSE_SMOOTHER,
               fallback_its=0, fallback_rho=0.9):
    return DgSolveOpts(restart, maxit, rtol, fixed_its, precond, pre_sweeps, post_sweeps, coarse_sweeps, omega,
                       jvp_mode, x0_is_zero, smoother, precision, coarse_solver, fallback_its, fallback_rho)


def _tptr(t, dtype, numel=None):
    import torch
    if not isinstance(t, torch.Tensor) or t.dtype != dtype or not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous %s CUDA tensor" % dtype)
    if numel is not None and t.numel() != numel:
        raise ValueError("expected %d entries, got %d" % (numel, t.numel()))
    return ctypes.c_void_p(t.data_ptr())


def _mchk(rc):
    if rc != DG_OK:
        raise DgError(rc, load().dg_last_error(None).decode())


def _cur_stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def dg_measure_peak(which, stream=None):
    """Measured FMA throughput (TFLOP/s) of the current device (DG_PEAK_FP64_FMA, DG_PEAK_FP32_FMA) or its
    read-only HBM streaming bandwidth in GB/s (DG_PEAK_HBM_READ)."""
    t = ctypes.c_double()
    _mchk(load().dg_measure_peak(int(which), ctypes.byref(t), _cur_stream(stream)))
    return t.value


def dg_mlp_workspace_bytes(rows):
    return int(load().dg_mlp_workspace_bytes(int(rows)))


def mlp_workspace(rows):
    """A device workspace (uint8 tensor) for dg_mlp_forward / dg_mlp_grad on `rows` rows."""
    import torch
    return torch.empty(dg_mlp_workspace_bytes(rows), dtype=torch.uint8, device="cuda")


def dg_mlp_forward(theta, X, Y, ws=None, stream=None):
    import torch
    n = X.shape[0]
    ws = mlp_workspace(n) if ws is None else ws
    _mchk(load().dg_mlp_forward(_tptr(theta, torch.float32, DG_MLP_NPARAM), _tptr(X, torch.float32, n * DG_MLP_IN),
                                n, _tptr(Y, torch.float32, n * DG_MLP_OUT), _tptr(ws, torch.uint8),
                                _cur_stream(stream)))


def dg_mlp_grad(theta, X, T, batch, grad, loss=None, seed=-1, step=0, ws=None, stream=None):
    import torch
    npairs = X.shape[0]
    ws = mlp_workspace(batch) if ws is None else ws
    lp = _tptr(loss, torch.float32, 1) if loss is not None else None
    _mchk(load().dg_mlp_grad(_tptr(theta, torch.float32, DG_MLP_NPARAM), _tptr(X, torch.float32, npairs * DG_MLP_IN),
                             _tptr(T, torch.float32, npairs * DG_MLP_OUT), npairs, int(batch), int(seed), int(step),
                             _tptr(grad, torch.float32, DG_MLP_NPARAM), lp, _tptr(ws, torch.uint8),
                             _cur_stream(stream)))


def dg_mlp_adam(theta, grad, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    import torch
    f = lambda a: _tptr(a, torch.float32, DG_MLP_NPARAM)
    _mchk(load().dg_mlp_adam(f(theta), f(grad), f(m), f(v), int(t), float(lr), float(beta1), float(beta2),
                             float(eps), _cur_stream(stream)))


class DG:
    """One solver handle (mesh, levels, workspaces) on the current CUDA device.

    Methods mirror the C ABI (same names, same order of arguments) and take
    contiguous float64 CUDA tensors laid out [element][u, v, w, p][mode].
    """

    def __init__(self, xn, yn, zn, levels, nu, ac_c=1.0, eta=7.0, boxes=None, walls=False):
        """One box with node coordinates xn, yn, zn, periodic, or with no-slip walls at
        y = yn[0] and y = yn[-1] (``walls``); or, with ``boxes`` (a list of (xn, yn, zn) triples,
        xn etc. None), a handle of several independent boxes (``dg_create_batch``)."""
        import numpy as np
        self._L = load()
        P = ctypes.POINTER(ctypes.c_double)
        ks = (ctypes.c_int * DG_MAX_LEVELS)(*(list(levels) + [0] * (DG_MAX_LEVELS - len(levels))))
        h = ctypes.c_void_p()
        if boxes is None:
            self._nodes = [np.ascontiguousarray(a, dtype=np.float64) for a in (xn, yn, zn)]
            self.params = DgParams(len(xn) - 1, len(yn) - 1, len(zn) - 1,
                                   self._nodes[0].ctypes.data_as(P), self._nodes[1].ctypes.data_as(P),
                                   self._nodes[2].ctypes.data_as(P), len(levels), ks, nu, ac_c, eta,
                                   DG_WALLS_Y if walls else DG_WALLS_NONE)
            rc = self._L.dg_create(ctypes.byref(self.params), ctypes.byref(h))
            self.ne = self.params.nx * self.params.ny * self.params.nz
        else:
            dims = np.array([[len(a) - 1 for a in b] for b in boxes], dtype=np.int32).ravel()
            nodes = np.ascontiguousarray(np.concatenate([np.asarray(a, dtype=np.float64) for b in boxes for a in b]))
            self._nodes = [nodes, dims]
            self.params = DgParams(0, 0, 0, None, None, None, len(levels), ks, nu, ac_c, eta,
                                   DG_WALLS_Y if walls else DG_WALLS_NONE)
            rc = self._L.dg_create_batch(ctypes.byref(self.params), len(boxes),
                                         dims.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), nodes.ctypes.data_as(P),
                                         ctypes.byref(h))
            self.ne = int(sum(int(np.prod([len(a) - 1 for a in b])) for b in boxes))
        if rc != DG_OK:
            raise DgError(rc, self._L.dg_last_error(None).decode())
        self.h = h
        self.levels = list(levels)
        self.nprob, self.elem_start = self.dg_problems()
        self.nb = []
        self.n = []
        for lvl in range(len(levels)):
            nb = ctypes.c_int()
            n = ctypes.c_longlong()
            self._chk(self._L.dg_level_size(self.h, lvl, ctypes.byref(nb), ctypes.byref(n)))
            self.nb.append(nb.value)
            self.n.append(n.value)

    # -- helpers
    def _chk(self, rc):
        if rc != DG_OK:
            raise DgError(rc, self._L.dg_last_error(self.h).decode())
        return rc

    @staticmethod
    def _stream(stream):
        import torch
        s = torch.cuda.current_stream() if stream is None else stream
        return ctypes.c_void_p(s.cuda_stream)

    def _ptr(self, t, lvl=0):
        import torch
        if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous():
            raise ValueError("expected a contiguous float64 CUDA tensor")
        if t.numel() != self.n[lvl]:
            raise ValueError("expected %d entries on level %d, got %d" % (self.n[lvl], lvl, t.numel()))
        return ctypes.c_void_p(t.data_ptr())

    def empty(self, lvl=0):
        import torch
        return torch.empty((self.ne, 4, self.nb[lvl]), dtype=torch.float64, device="cuda")

    def close(self):
        if getattr(self, "h", None):
            self._L.dg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- C ABI, one method per entry point
    def dg_problems(self):
        n = ctypes.c_int()
        self._chk(self._L.dg_problems(self.h, ctypes.byref(n), None))
        es = (ctypes.c_int * (n.value + 1))()
        self._chk(self._L.dg_problems(self.h, ctypes.byref(n), es))
        return n.value, list(es)

    def dg_set_problem_shifts(self, mult, stream=None):
        arr = (ctypes.c_double * self.nprob)(*[float(v) for v in mult])
        self._chk(self._L.dg_set_problem_shifts(self.h, arr, self._stream(stream)))

    def dg_get_tuning(self, which):
        t = DgTuning()
        self._chk(self._L.dg_get_tuning(self.h, int(which), ctypes.byref(t)))
        return t

    def dg_set_tuning(self, which, t=None, **kw):
        t = t if t is not None else self.dg_get_tuning(which)
        for key, val in kw.items():
            setattr(t, key, int(val))
        self._chk(self._L.dg_set_tuning(self.h, int(which), ctypes.byref(t)))

    def dg_autotune(self, which, use_cache=True, stream=None):
        """Returns the report: device ms of the default and chosen face pass, volume pass and
        block-Jacobi apply."""
        rep = (ctypes.c_double * 6)()
        self._chk(self._L.dg_autotune(self.h, int(which), 1 if use_cache else 0, rep, self._stream(stream)))
        keys = ("face_default_ms", "face_chosen_ms", "vol_default_ms", "vol_chosen_ms", "jacobi_default_ms",
                "jacobi_chosen_ms")
        return dict(zip(keys, list(rep)))

    def dg_set_test_knob(self, knob, value):
        self._chk(self._L.dg_set_test_knob(self.h, int(knob), int(value)))

    def dg_get_status(self, stream=None):
        s = ctypes.c_uint()
        self._chk(self._L.dg_get_status(self.h, ctypes.byref(s), self._stream(stream)))
        return s.value

    def dg_project_tgv(self, w, stream=None):
        self._chk(self._L.dg_project_tgv(self.h, self._ptr(w), self._stream(stream)))

    def dg_quad_points(self, stream=None):
        """[N_e, (k+1)^3, 3] float64 CUDA tensor of the volume Gauss points."""
        import torch
        nq = (self.levels[0] + 1) ** 3
        xyz = torch.empty((self.ne, nq, 3), dtype=torch.float64, device="cuda")
        self._chk(self._L.dg_quad_points(self.h, ctypes.c_void_p(xyz.data_ptr()), self._stream(stream)))
        return xyz

    def dg_project_points(self, vals, w, stream=None):
        import torch
        nq = (self.levels[0] + 1) ** 3
        v = _tptr(vals, torch.float64, self.ne * 4 * nq)
        self._chk(self._L.dg_project_points(self.h, v, self._ptr(w), self._stream(stream)))

    def dg_residual(self, w, f, stream=None):
        self._chk(self._L.dg_residual(self.h, self._ptr(w), self._ptr(f), self._stream(stream)))

    def dg_set_linearization(self, w, inv_gamma_dt, stream=None):
        self._chk(self._L.dg_set_linearization(self.h, self._ptr(w), float(inv_gamma_dt), self._stream(stream)))

    def dg_set_linearization_rhs(self, w, inv_gamma_dt, g, stream=None):
        self._chk(self._L.dg_set_linearization_rhs(self.h, self._ptr(w), float(inv_gamma_dt), self._ptr(g),
                                                   self._stream(stream)))

    def dg_stage_update(self, w, dw, b=1.0, stream=None):
        self._chk(self._L.dg_stage_update(self.h, self._ptr(w), self._ptr(dw), float(b), self._stream(stream)))

    def dg_jvp(self, v, out, mode=DG_JVP_TANGENT, stream=None):
        self._chk(self._L.dg_jvp(self.h, self._ptr(v), self._ptr(out), int(mode), self._stream(stream)))

    def dg_assemble(self, stream=None, precision=None):
        if precision is None:
            self._chk(self._L.dg_assemble(self.h, self._stream(stream)))
        else:
            self._chk(self._L.dg_assemble_precision(self.h, int(precision), self._stream(stream)))

    def dg_assemble_precision(self, precision, stream=None):
        self._chk(self._L.dg_assemble_precision(self.h, int(precision), self._stream(stream)))

    def pmg_restrict(self, lvl, xf, xc, stream=None):
        self._chk(self._L.pmg_restrict(self.h, lvl, self._ptr(xf, lvl), self._ptr(xc, lvl + 1), self._stream(stream)))

    def pmg_prolong(self, lvl, xc, xf, stream=None):
        self._chk(self._L.pmg_prolong(self.h, lvl, self._ptr(xc, lvl + 1), self._ptr(xf, lvl), self._stream(stream)))

    def block_jacobi_smooth(self, lvl, g, x, sweeps, omega=1.0, stream=None):
        self._chk(self._L.block_jacobi_smooth(self.h, lvl, self._ptr(g, lvl), self._ptr(x, lvl), int(sweeps),
                                              float(omega), self._stream(stream)))

    def bsr_spmv(self, lvl, alpha, x, beta, y, stream=None):
        self._chk(self._L.bsr_spmv(self.h, lvl, float(alpha), self._ptr(x, lvl), float(beta), self._ptr(y, lvl),
                                   self._stream(stream)))

    def pmg_vcycle(self, g, x, opts=None, stream=None):
        o = opts or solve_opts()
        self._chk(self._L.pmg_vcycle(self.h, self._ptr(g), self._ptr(x), ctypes.byref(o), self._stream(stream)))

    def dg_counters(self):
        a, b = ctypes.c_longlong(), ctypes.c_longlong()
        self._chk(self._L.dg_counters(self.h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def dg_profile(self, enable=True):
        self._chk(self._L.dg_profile(self.h, 1 if enable else 0))

    def dg_profile_read(self):
        ms = (ctypes.c_double * DG_PROF_N)()
        cnt = (ctypes.c_longlong * DG_PROF_N)()
        self._chk(self._L.dg_profile_read(self.h, ms, cnt))
        return {PROF_NAMES[i]: (ms[i], cnt[i]) for i in range(DG_PROF_N)}

    def dg_profile_read_bytes(self):
        """{class: (ms, launches, algorithmic bytes)} since the last read."""
        ms = (ctypes.c_double * DG_PROF_N)()
        cnt = (ctypes.c_longlong * DG_PROF_N)()
        by = (ctypes.c_double * DG_PROF_N)()
        self._chk(self._L.dg_profile_read_bytes(self.h, ms, cnt, by))
        return {PROF_NAMES[i]: (ms[i], cnt[i], by[i]) for i in range(DG_PROF_N)}

    def dg_reuse_assembly(self):
        self._chk(self._L.dg_reuse_assembly(self.h))

    def dg_set_stb_rescaling(self, enable=True):
        self._chk(self._L.dg_set_stb_rescaling(self.h, 1 if enable else 0))

    def pmg_level_solve(self, lvl, g, x, rtol=1e-8, maxit=1000, x0_is_zero=True, stream=None, check=True):
        info = DgSolveInfo()
        rc = self._L.pmg_level_solve(self.h, int(lvl), self._ptr(g, lvl), self._ptr(x, lvl), float(rtol), int(maxit),
                                     1 if x0_is_zero else 0, ctypes.byref(info), self._stream(stream))
        if check and rc not in (DG_OK, DG_ERR_NOT_CONVERGED):
            self._chk(rc)
        return info, rc

    def pmg_project_pressure(self, lvl, x, stream=None):
        self._chk(self._L.pmg_project_pressure(self.h, int(lvl), self._ptr(x, lvl), self._stream(stream)))

    def dg_set_coarse_network(self, theta, stream=None):
        import torch
        p = None if theta is None else _tptr(theta, torch.float32, DG_MLP_NPARAM)
        self._chk(self._L.dg_set_coarse_network(self.h, p, self._stream(stream)))

    def bsr_spmv_t(self, lvl, alpha, x, beta, y, stream=None):
        self._chk(self._L.bsr_spmv_t(self.h, lvl, float(alpha), self._ptr(x, lvl), float(beta), self._ptr(y, lvl),
                                     self._stream(stream)))

    def dg_coarse_apply(self, d, x, accumulate=False, stream=None):
        lc = len(self.levels) - 1
        self._chk(self._L.dg_coarse_apply(self.h, self._ptr(d, lc), self._ptr(x, lc), 1 if accumulate else 0,
                                          self._stream(stream)))

    def dg_coarse_pairs(self, d, x, X, T, s, q=None, stream=None):
        import torch
        lc = len(self.levels) - 1
        qp = None if q is None else self._ptr(q, lc)
        self._chk(self._L.dg_coarse_pairs(self.h, self._ptr(d, lc), self._ptr(x, lc), qp,
                                          _tptr(X, torch.float32, self.ne * DG_MLP_IN),
                                          _tptr(T, torch.float32, self.ne * DG_MLP_OUT),
                                          _tptr(s, torch.float32, self.ne), self._stream(stream)))

    def dg_record_coarse(self, buf, capacity=None):
        import torch
        if buf is None:
            self._chk(self._L.dg_record_coarse(self.h, None, 0))
            self._rec = None
            return
        lc = len(self.levels) - 1
        cap = buf.numel() // self.n[lc] if capacity is None else int(capacity)
        if cap < 1 or cap * self.n[lc] > buf.numel():
            raise ValueError("recording buffer too small")
        self._chk(self._L.dg_record_coarse(self.h, _tptr(buf, torch.float64), cap))
        self._rec = buf  # keep it alive while recording

    def dg_recorded(self):
        c = ctypes.c_int()
        self._chk(self._L.dg_recorded(self.h, ctypes.byref(c)))
        return c.value

    def fgmres_solve(self, g, x, opts=None, stream=None, check=True, log=None, **log_fields):
        """``log``: a path; one JSON line per solve (iterations, residuals, rho, status) is appended."""
        o = opts or solve_opts()
        info = DgSolveInfo()
        rc = self._L.fgmres_solve(self.h, self._ptr(g), self._ptr(x), ctypes.byref(o), ctypes.byref(info),
                                  self._stream(stream))
        if log is not None:
            from .checkpoint import log_solve
            log_solve(log, info, rc, precision=int(o.precision), **log_fields)
        if check and rc not in (DG_OK, DG_ERR_NOT_CONVERGED):
            self._chk(rc)
        return info, rc


class Plan:
    """``dg_plan_*``: FGMRES over every problem of several handles, optionally as one CUDA
    graph. ``dgs``, ``gs``, ``xs``: handles and their right-hand sides / solutions (kept alive
    by the plan)."""

    def __init__(self, dgs, gs, xs, opts, use_graph=True):
        self._L = load()
        self._keep = (list(dgs), list(gs), list(xs))
        nh = len(dgs)
        V = ctypes.c_void_p * nh
        hs = V(*[d.h.value for d in dgs])
        gp = V(*[d._ptr(g).value for d, g in zip(dgs, gs)])
        xp = V(*[d._ptr(x).value for d, x in zip(dgs, xs)])
        self.opts = opts
        p = ctypes.c_void_p()
        rc = self._L.dg_plan_create(nh, hs, gp, xp, ctypes.byref(opts), 1 if use_graph else 0, ctypes.byref(p))
        if rc != DG_OK:
            raise DgError(rc, self._L.dg_plan_error(None).decode())
        self.p = p
        self.nh = nh

    def _chk(self, rc):
        if rc != DG_OK:
            raise DgError(rc, self._L.dg_plan_error(self.p).decode())
        return rc

    def dg_plan_solve(self, stream=None, check=True):
        rc = self._L.dg_plan_solve(self.p, DG._stream(stream))
        if check:
            self._chk(rc)
        return rc

    def dg_plan_result(self, i):
        """(its, relres, converged) lists for handle i's problems."""
        n = self._keep[0][i].nprob
        its, rr, cv = (ctypes.c_int * n)(), (ctypes.c_double * n)(), (ctypes.c_int * n)()
        self._chk(self._L.dg_plan_result(self.p, i, its, rr, cv))
        return list(its), list(rr), [bool(c) for c in cv]

    def dg_plan_stats(self):
        c, s, g = ctypes.c_int(), ctypes.c_int(), ctypes.c_longlong()
        self._chk(self._L.dg_plan_stats(self.p, ctypes.byref(c), ctypes.byref(s), ctypes.byref(g)))
        return {"cycles": c.value, "steps": s.value, "graph_launches": g.value}

    def close(self):
        if getattr(self, "p", None):
            self._L.dg_plan_destroy(self.p)
            self.p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
