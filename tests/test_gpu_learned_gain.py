"""What the trained coarse network gains over the cycle without it (GPU, through the C ABI).

The network is trained by the library's kernels (coarse-residual loss) on the coarse
right-hand sides that the cycle produces in the stages of Taylor-Green states 0-3 (acoustic
CFL 50), then judged on later states it has not seen.

1. 8^3 P2 with a P1 coarse level (two p-levels), FP32 cycle: at the coarse level one
   application of the network leaves less of the coarse residual than the two block-Jacobi
   sweeps of the plain coarse solve it replaces. The outer FGMRES solve with it converges
   without falling back (iteration counts printed; on this small mesh the fine-level smoothing
   decides the outer count, and the network's cycle is within a few iterations either way).
2. 32^3 P4, levels 4-2-1, the benchmark's chosen cycle (FP32 with FP16 block storage and
   tensor-core volume contractions, omega 0.95, 4/4/2 sweeps), network trained on the first
   stages of the Taylor-Green run and judged on states from seeds training never saw (the field
   plus a seeded smooth divergence-free perturbation): the network leaves less of the coarse
   residual than the two
   block-Jacobi sweeps it replaces, and the outer solves converge without falling back. The
   outer FGMRES iterations and wall times with and without it are printed, not asserted: with
   this cycle the fine-level smoothing decides the outer count, and no wall-time gain exists
   (the benchmark's learned form reports the same on the 24^3 mesh).
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
    # 2. outer solve on held-out states 4 and 6: converges with the network, no fallback
    its = {}
    for k in (4, 6):
        _, i0, rc0 = stage(states[k], opts())
        _, i1, rc1 = stage(states[k], opts(coarse_solver=P.DG_COARSE_LEARNED, fallback_its=5, fallback_rho=0.8))
        assert rc0 == P.DG_OK and rc1 == P.DG_OK and i1.fallback_at == -1
        its[k] = (i0.its, i1.its)
    print("coarse residual ratio: network %.3f, 2 block-Jacobi sweeps %.3f; FGMRES its to 1e-8 (without, with): "
          "%s; training %.2f s" % (r_net, r_jac, its, rep["train_s"]))
    assert r_net < 0.9 * r_jac


def test_learned_coarse_correction_held_out_32():
    torch, P = require_gpu()
    import paper_1809_00866_gb300.learned as Lrn
    n, levels = 32, [4, 2, 1]
    un = S.uniform_nodes(n)
    dg = P.DG(un, un, un, levels, S.NU_TGV, S.AC_C, S.ETA)
    dg.dg_set_stb_rescaling(True)
    inv = 1.0 / S.acoustic_dt(n, levels[0])
    lc = len(levels) - 1
    prec = P.DG_PRECOND_FP32_H16_TC

    def opts(**kw):
        base = dict(restart=30, maxit=300, rtol=1e-8, omega=0.95, pre_sweeps=4, post_sweeps=4, coarse_sweeps=2,
                    precision=prec)
        base.update(kw)
        return P.solve_opts(**base)

    def stage(w, o):
        g = dg.empty()
        dg.dg_set_linearization_rhs(w, inv, g)
        dg.dg_assemble(precision=o.precision)
        x = dg.empty()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        info, rc = dg.fgmres_solve(g, x, o)
        e1.record()
        torch.cuda.synchronize()
        return x, info, rc, e0.elapsed_time(e1) / 1e3

    w = dg.empty()
    dg.dg_project_tgv(w)
    states = [w]
    for _ in range(3):
        x, info, rc, _ = stage(states[-1], opts())
        assert rc == P.DG_OK
        states.append((states[-1] + x).contiguous())
    D = Lrn.collect_rhs(dg, states, inv, opts(), per_state=40)
    dg.dg_set_linearization(states[-1], inv)
    dg.dg_assemble()
    theta, rep = Lrn.train_residual(dg, D, steps=2000, lr=1e-3, seed=0)
    dg.dg_set_coarse_network(theta)
    # held out: the field plus a seeded smooth divergence-free perturbation (seeds 11 and 12,
    # 5 % of the field's peak speed), projected on the handle's Gauss points. (Seeded noise on
    # every modal coefficient is no stand-in at this mesh: with amplitude 0.005 or more no form
    # of the solver reaches 1e-8 in 100 iterations, the plain FP64 one included.)
    xyz = dg.dg_quad_points().cpu().numpy()
    held = []
    for seed in (11, 12):
        vals = np.ascontiguousarray(np.stack(S.box_noise_field(xyz[..., 0], xyz[..., 1], xyz[..., 2], seed),
                                             axis=1))
        dw = dg.empty()
        dg.dg_project_points(torch.from_numpy(vals).cuda(), dw)
        held.append((w + dw).contiguous())
    # coarse level: the network against the two block-Jacobi sweeps it replaces, on held-out data
    Dv = Lrn.collect_rhs(dg, held, inv, opts(), per_state=8)
    dg.dg_set_coarse_network(theta)
    r_net = Lrn.residual_ratio(dg, Dv)
    y, r = dg.empty(lc), dg.empty(lc)
    r_jac = []
    for d in Dv:
        y.zero_()
        dg.block_jacobi_smooth(lc, d, y, 2, 0.95)
        r.copy_(d)
        dg.bsr_spmv(lc, -1.0, y, 1.0, r)
        r_jac.append(float(r.norm().item()) / float(d.norm().item()))
    r_jac = float(np.mean(r_jac))
    its, secs = {}, {}
    for k, wh in enumerate(held):
        _, i0, rc0, t0 = stage(wh, opts())
        _, i1, rc1, t1 = stage(wh, opts(coarse_solver=P.DG_COARSE_LEARNED, fallback_its=5, fallback_rho=0.8))
        assert rc0 == P.DG_OK and rc1 == P.DG_OK and i1.fallback_at == -1
        its[k], secs[k] = (i0.its, i1.its), (round(t0, 4), round(t1, 4))
    print("32^3 P4, held-out seeded states: coarse residual ratio network %.3f vs 2 block-Jacobi sweeps %.3f; "
          "FGMRES its (without, with) %s; solve seconds (without, with) %s; training %.2f s"
          % (r_net, r_jac, its, secs, rep["train_s"]))
    assert r_net < 0.9 * r_jac
