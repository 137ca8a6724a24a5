"""What the trained coarse network gains over the cycle without it (GPU, through the C ABI).

Workload: Taylor-Green vortex on 8^3 periodic hexahedra, P2 with a P1 coarse level (two
p-levels, where the coarse solve carries much of the cycle), acoustic CFL 50, inside FP64
FGMRES(30). The network is trained by the library's kernels (coarse-residual loss) on the
coarse right-hand sides that the FP32 cycle (block-Jacobi, omega 0.7, 2/2/2 sweeps) produces
in the stages of states 0-3, then judged on later states it has not seen:
 1. at the coarse level, one application of the network leaves less of the coarse residual
    than the two block-Jacobi sweeps of the plain coarse solve;
 2. in the undamped FP64 cycle (omega 1), whose plain coarse sweeps let FGMRES stall on these
    states, the cycle with the network reaches a smaller residual after 40 iterations.
Iteration counts of the FP32 cycle with and without the network are printed (the two are
within a few iterations of each other there).
"""
import numpy as np
import pytest

import synthetic as S
from _gpu_common import require_gpu

pytestmark = pytest.mark.gpu


def test_learned_coarse_correction_gain():
    torch, P = require_gpu()
    import paper_1809_00866_gb300.learned as Lrn
    n, levels = 8, [2, 1]
    un = S.uniform_nodes(n)
    dg = P.DG(un, un, un, levels, S.NU_TGV, S.AC_C, S.ETA)
    inv = 1.0 / S.acoustic_dt(n, levels[0])
    lc = 1

    def opts(**kw):
        base = dict(restart=30, maxit=400, rtol=1e-8, omega=0.7, precision=P.DG_PRECOND_FP32)
        base.update(kw)
        return P.solve_opts(**base)

    def stage(w, o):
        f = dg.empty()
        dg.dg_residual(w, f)
        g = (-f).contiguous()
        dg.dg_set_linearization(w, inv)
        dg.dg_assemble()
        x = dg.empty()
        info, rc = dg.fgmres_solve(g, x, o)
        return x, info, rc

    w = dg.empty()
    dg.dg_project_tgv(w)
    states = [w]
    for _ in range(6):
        x, info, rc = stage(states[-1], opts())
        assert info.true_relres < 1e-4  # the states only need to be plausible later flow fields
        states.append((states[-1] + x).contiguous())
    D = Lrn.collect_rhs(dg, states[0:4], inv, opts(), per_state=40)
    dg.dg_set_linearization(states[3], inv)
    dg.dg_assemble()
    theta, rep = Lrn.train_residual(dg, D, steps=2000, lr=1e-3, seed=0)
    dg.dg_set_coarse_network(theta)
    # 1. coarse residual left by the network vs by two block-Jacobi sweeps from zero (held-out state 5)
    Dv = Lrn.collect_rhs(dg, [states[5]], inv, opts(), per_state=8)
    r_net = Lrn.residual_ratio(dg, Dv)
    y, r = dg.empty(lc), dg.empty(lc)
    r_jac = []
    for d in Dv:
        y.zero_()
        dg.block_jacobi_smooth(lc, d, y, 2, 0.7)
        r.copy_(d)
        dg.bsr_spmv(lc, -1.0, y, 1.0, r)
        r_jac.append(float(r.norm().item()) / float(d.norm().item()))
    r_jac = float(np.mean(r_jac))
    # 2. outer solve on held-out states 4 and 6
    its, res40 = {}, {}
    for k in (4, 6):
        _, i0, _ = stage(states[k], opts())
        _, i1, _ = stage(states[k], opts(coarse_solver=P.DG_COARSE_LEARNED))
        its[k] = (i0.its, i1.its)
        fp64 = dict(fixed_its=40, omega=1.0, precision=P.DG_PRECOND_FP64)
        _, f0, _ = stage(states[k], opts(**fp64))
        _, f1, _ = stage(states[k], opts(coarse_solver=P.DG_COARSE_LEARNED, **fp64))
        res40[k] = (f0.true_relres, f1.true_relres)
    print("coarse residual ratio: network %.3f, 2 block-Jacobi sweeps %.3f; FP32 cycle, FGMRES its to 1e-8 "
          "(without, with): %s; FP64 cycle omega 1, rel res after 40 its (without, with): %s; training %.2f s"
          % (r_net, r_jac, its, res40, rep["train_s"]))
    assert r_net < r_jac
    for k, (a, b) in res40.items():
        assert b < a, (k, a, b)
