"""GPU parity at the benchmark's sizes, in the launch shapes the benchmark uses (through the C ABI).

The benchmark runs Taylor-Green stages on 16^3 and 32^3 periodic hexahedra at P4, where the
launch shapes of the operator passes are autotuned per mesh size. Here the FP64 residual
(Eq. (NSdiscrRes)) and the exact Jacobian action (Eqs. (jacTrilFnotNU), (jacTrilnu)) on those
meshes are compared with the oracle's, entry by entry: relative 2-norm <= 1e-12 and
max |a - b| <= 1e-12 max |b|, for the autotuned shapes and for the extreme candidate shapes.
The oracle runs its element loops on all host cores (its results do not depend on the count).

For the Jacobian action on the generic 32^3 state the bound also allows for the problem's own
rounding sensitivity: the entries of G v grow like 1/h (up to ~3e4 there) and come from sums
that cancel, so a one-ulp relative perturbation of w and v already moves the oracle's own result
by up to ~5e-12 of its largest entry (2e-12 in the 2-norm). No FP64 evaluation in another
summation order can do better; the test measures that sensitivity with the oracle and asserts
max(1e-12, 4 x sensitivity), element-wise and in the 2-norm.

The FP32 preconditioner cycle at 16^3 (the staged block-Jacobi apply walks its ring several
times per CTA there) is compared with the FP64 cycle on the same assembly, at the bounds the
small-mesh tests state: 1e-5 for FP32 blocks, 5e-3 for FP16 blocks.
"""
import numpy as np
import pytest

import oracle as O
import synthetic as S
from _gpu_common import dev, host, maxrel, pair, rel

pytestmark = pytest.mark.gpu


def _mesh(n):
    un = S.uniform_nodes(n)
    return pair(un, un, un, [4, 2, 1])


@pytest.mark.parametrize("n", [16, 32])
def test_residual_and_exact_jvp_at_benchmark_size(n):
    import paper_1809_00866_gb300 as P
    dg, m = _mesh(n)
    inv = 1.0 / S.acoustic_dt(n, 4)
    w_tgv = O.project_tgv(m)
    w_gen = w_tgv + S.perturbation(m.ne, 4, 0.1, 1600 + n)
    f = dg.empty()
    for w in (w_tgv, w_gen):  # the benchmark's first state, and a generic one
        dg.dg_residual(dev(w), f)
        ref = O.residual(m, w)
        got = host(f)
        assert rel(got, ref) < 1e-12
        assert maxrel(got, ref) < 1e-12
    assert dg.dg_get_status() == 0
    dg.dg_set_linearization(dev(w_gen), inv)
    dg.dg_autotune(P.DG_TUNE_FP64, use_cache=False)
    tuned = dg.dg_get_tuning(P.DG_TUNE_FP64).as_dict()
    v = S.direction(m.ne, 4, S.SEED_V)
    ref = O.jvp(m, w_gen, v, inv)
    # the oracle's own sensitivity to one-ulp relative perturbations of its inputs
    rng = np.random.default_rng(n)
    eps = np.finfo(np.float64).eps
    ref_p = O.jvp(m, w_gen * (1 + eps * rng.standard_normal(w_gen.shape)),
                  v * (1 + eps * rng.standard_normal(v.shape)), inv)
    tol2 = max(1e-12, 4 * rel(ref_p, ref))
    tolmax = max(1e-12, 4 * maxrel(ref_p, ref))
    out = dg.empty()
    shapes = [tuned, dict(tuned, face_warps=2, vol_threads=64, vol_ctas_per_sm=0),
              dict(tuned, face_warps=8, vol_threads=256, vol_ctas_per_sm=4)]
    for sh in shapes:
        dg.dg_set_tuning(P.DG_TUNE_FP64, **sh)
        dg.dg_jvp(dev(v), out)
        got = host(out)
        assert rel(got, ref) < tol2, (sh, tol2)
        assert maxrel(got, ref) < tolmax, (sh, tolmax)
    assert dg.dg_get_status() == 0


@pytest.mark.parametrize("storage,bound", [("FP32", 1e-5), ("FP32_H16", 5e-3), ("FP32_BF16", 4e-2)])
def test_fp32_cycle_at_benchmark_size(storage, bound):
    import paper_1809_00866_gb300 as P
    dg, m = _mesh(16)
    inv = 1.0 / S.acoustic_dt(16, 4)
    g = dg.empty()
    dg.dg_set_linearization_rhs(dev(O.project_tgv(m)), inv, g)
    dg.dg_assemble()
    x64 = dg.empty()
    dg.pmg_vcycle(g, x64, P.solve_opts(omega=0.9))
    prec = getattr(P, "DG_PRECOND_" + storage)
    x32 = dg.empty()
    opts = P.solve_opts(omega=0.9, precision=prec)
    dg.pmg_vcycle(g, x32, opts)  # makes the FP32 (and 16-bit) copies of the FP64 assembly
    dg.dg_autotune(P.DG_TUNE_FP32, use_cache=False)  # the shapes the benchmark measures, Jacobi stages included
    dg.pmg_vcycle(g, x32, opts)
    a, b = host(x32), host(x64)
    assert rel(a, b) < bound
    assert maxrel(a, b) < bound
    assert dg.dg_get_status() == 0
