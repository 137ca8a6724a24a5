"""GPU parity of the batched handle (several independent periodic boxes in one element set) and
of the batched FGMRES plans, eager and as one CUDA graph (through the C ABI).

Every problem of a batch is checked against the oracle on its own box, with its own mass shift
1/(gamma dt_q): the operator and the assembled preconditioner at 1e-12, a fixed number of FGMRES
iterations at 1e-10, converged solves by their true residual under the oracle's exact operator.
The batch must also equal the same boxes solved by one-box handles (no coupling between
problems), and the graph form must equal the eager form bit for bit (same kernels, same order).
"""
import numpy as np
import pytest

import oracle as O
import oracle.solvers as SV
import synthetic as S
from _gpu_common import dev, host, meshes, rel, require_gpu

pytestmark = pytest.mark.gpu


def boxes_of(names):
    u = S.uniform_nodes
    extra = {"u345": (u(3), u(4), u(5))}
    return [extra[n] if n in extra else meshes()[n] for n in names]


def make_batch(names, levels, mults, seed=1, amp=0.2):
    torch, P = require_gpu()
    boxes = boxes_of(names)
    dg = P.DG(None, None, None, levels, S.NU_TGV, S.AC_C, S.ETA, boxes=boxes)
    ms = [O.Mesh(*b, levels[0], S.NU_TGV, S.AC_C, S.ETA) for b in boxes]
    ws = [O.project_tgv(m) + S.perturbation(m.ne, m.k, amp, seed + q) for q, m in enumerate(ms)]
    inv = 1.0 / S.acoustic_dt(ms[0].nx, ms[0].k)
    dg.dg_set_problem_shifts(mults)
    return P, dg, ms, ws, inv


def cat(arrs):
    return np.concatenate([np.asarray(a).reshape(-1) for a in arrs])


def split(dg, ms, t, nb=None):
    """Per-problem pieces of a batch vector (element ranges from dg_problems)."""
    a = host(t).reshape(dg.ne, -1)
    es = dg.elem_start
    return [a[es[q]:es[q + 1]].reshape(-1) for q in range(len(ms))]


def oracle_levels(m, w, inv, levels):
    G0 = O.dense_G(m, w, inv)
    Gs = [G0] + [SV.inherited_operator(G0, m.ne, m.nb, O.nb(k)) for k in levels[1:]]
    nbs = [O.nb(k) for k in levels]
    Ds = [SV.block_inverses(G, m.ne, nb) for G, nb in zip(Gs, nbs)]
    return Gs, Ds, nbs


NAMES = ["u2", "box233", "u3", "box345"]
MULTS = [1.0, 0.5, 2.0, 1.3]
# boxes whose stage systems restarted FGMRES solves in the oracle too (the 2-cell and
# perturbed-node boxes above stall at these time steps: their operators are close to the
# singular constant-pressure mode of the periodic box)
CONV = ["u3", "u345", "u3"]
CONV_MULTS = [2.0, 2.5, 3.0]


def test_batch_layout():
    P, dg, ms, ws, inv = make_batch(NAMES, [2, 1], MULTS)
    assert dg.nprob == len(NAMES)
    assert dg.elem_start == list(np.cumsum([0] + [m.ne for m in ms]))
    assert dg.ne == sum(m.ne for m in ms)


@pytest.mark.parametrize("levels", [[2, 1], [3, 2, 1]])
def test_batch_operator(levels):
    # residual (Eq. (NSdiscrRes)) and exact Jacobian action with the per-problem shift (Eq. (rosSysOp))
    P, dg, ms, ws, inv = make_batch(NAMES, levels, MULTS)
    wd = dev(cat(ws).reshape(dg.ne, 4, -1))
    f = dg.empty()
    dg.dg_residual(wd, f)
    for q, (m, fq) in enumerate(zip(ms, split(dg, ms, f))):
        assert rel(fq, O.residual(m, ws[q]).reshape(-1)) < 1e-12, q
    dg.dg_set_linearization(wd, inv)
    vs = [S.direction(m.ne, m.k, seed=7 + q) for q, m in enumerate(ms)]
    out = dg.empty()
    dg.dg_jvp(dev(cat(vs).reshape(dg.ne, 4, -1)), out)
    for q, (m, oq) in enumerate(zip(ms, split(dg, ms, out))):
        assert rel(oq, O.jvp(m, ws[q], vs[q], inv * MULTS[q]).reshape(-1)) < 1e-12, q


def test_batch_equals_one_box_handles():
    # the same kernels on the concatenated element set: every problem's numbers are those of a
    # handle holding that box alone (with 1/(gamma dt) scaled by its multiplier)
    P, dg, ms, ws, inv = make_batch(NAMES, [3, 2, 1], MULTS)
    wd = dev(cat(ws).reshape(dg.ne, 4, -1))
    dg.dg_set_linearization(wd, inv)
    dg.dg_assemble()
    vs = [S.direction(m.ne, m.k, seed=3 + q) for q, m in enumerate(ms)]
    out = dg.empty()
    dg.dg_jvp(dev(cat(vs).reshape(dg.ne, 4, -1)), out)
    rng = np.random.default_rng(4)
    xs = [rng.standard_normal(m.ne * 4 * O.nb(1)) for m in ms]
    yb = dg.empty(2)
    dg.bsr_spmv(2, 1.0, dev(cat(xs).reshape(dg.ne, 4, -1)), 0.0, yb)
    gs = [rng.standard_normal(m.n) for m in ms]
    xb = dg.empty()
    xb.zero_()
    dg.block_jacobi_smooth(0, dev(cat(gs).reshape(dg.ne, 4, -1)), xb, 2, 0.8)
    for q, (name, m) in enumerate(zip(NAMES, ms)):
        one = P.DG(*meshes()[name], [3, 2, 1], S.NU_TGV, S.AC_C, S.ETA)
        one.dg_set_linearization(dev(ws[q]), inv * MULTS[q])
        one.dg_assemble()
        o = one.empty()
        one.dg_jvp(dev(vs[q]), o)
        assert np.array_equal(split(dg, ms, out)[q], host(o).reshape(-1)), q
        y = one.empty(2)
        one.bsr_spmv(2, 1.0, dev(xs[q].reshape(m.ne, 4, -1)), 0.0, y)
        assert rel(split(dg, ms, yb)[q], host(y).reshape(-1)) < 1e-13, q
        x1 = one.empty()
        x1.zero_()
        one.block_jacobi_smooth(0, dev(gs[q]), x1, 2, 0.8)
        assert rel(split(dg, ms, xb)[q], host(x1).reshape(-1)) < 1e-13, q


def test_batch_assembly_vs_oracle():
    levels = [2, 1]
    P, dg, ms, ws, inv = make_batch(NAMES, levels, MULTS)
    dg.dg_set_linearization(dev(cat(ws).reshape(dg.ne, 4, -1)), inv)
    dg.dg_assemble()
    rng = np.random.default_rng(5)
    refs = [oracle_levels(m, ws[q], inv * MULTS[q], levels) for q, m in enumerate(ms)]
    for lvl in range(len(levels)):
        x = [rng.standard_normal(r[0][lvl].shape[0]) for r in refs]
        g = [rng.standard_normal(r[0][lvl].shape[0]) for r in refs]
        xd = dev(cat(x).reshape(dg.ne, 4, -1))
        dg.block_jacobi_smooth(lvl, dev(cat(g).reshape(dg.ne, 4, -1)), xd, 2, 0.8)
        for q, (Gs, Ds, nbs) in enumerate(refs):
            ref = SV.block_jacobi(lambda v, G=Gs[lvl]: G @ v, Ds[lvl], g[q], x[q], 2, 0.8)
            assert rel(split(dg, ms, xd)[q], ref) < 1e-12, (lvl, q)
        if lvl >= 1:
            yd = dg.empty(lvl)
            dg.bsr_spmv(lvl, 1.0, dev(cat(x).reshape(dg.ne, 4, -1)), 0.0, yd)
            for q, (Gs, Ds, nbs) in enumerate(refs):
                assert rel(split(dg, ms, yd)[q], Gs[lvl] @ x[q]) < 1e-12, (lvl, q)


def rhs(dg, ms, ws):
    return dev(cat([-O.residual(m, w) for m, w in zip(ms, ws)]).reshape(dg.ne, 4, -1))


@pytest.mark.parametrize("use_graph", [False, True])
def test_plan_fixed_iterations_vs_oracle(use_graph):
    levels = [2, 1]
    P, dg, ms, ws, inv = make_batch(NAMES, levels, MULTS)
    dg.dg_set_linearization(dev(cat(ws).reshape(dg.ne, 4, -1)), inv)
    dg.dg_assemble()
    g = rhs(dg, ms, ws)
    x = dg.empty()
    its = 6
    plan = P.Plan([dg], [g], [x], P.solve_opts(fixed_its=its), use_graph=use_graph)
    plan.dg_plan_solve()
    got_its, relres, conv = plan.dg_plan_result(0)
    assert got_its == [its] * len(ms) and all(conv)
    for q, m in enumerate(ms):
        Gs, Ds, nbs = oracle_levels(m, ws[q], inv * MULTS[q], levels)
        lv = [SV.Level(lambda v, G=G: G @ v, D, m.ne, nb) for G, D, nb in zip(Gs, Ds, nbs)]
        gq = -O.residual(m, ws[q]).reshape(-1)
        xr, _, _ = SV.fgmres(lambda v: Gs[0] @ v, lambda v: SV.mg_v(lv, 0, v, np.zeros_like(v)), gq, restart=30,
                             fixed_its=its)
        vol = m.vol()
        a = SV.remove_mean_pressure(split(dg, ms, x)[q], m.ne, m.nb, vol)
        b = SV.remove_mean_pressure(xr, m.ne, m.nb, vol)
        assert rel(a, b) < 1e-10, q


@pytest.mark.parametrize("use_graph", [False, True])
def test_plan_converges_vs_oracle(use_graph):
    levels = [3, 2, 1]
    P, dg, ms, ws, inv = make_batch(CONV, levels, CONV_MULTS, amp=0.05)
    dg.dg_set_linearization(dev(cat(ws).reshape(dg.ne, 4, -1)), inv)
    dg.dg_assemble()
    g = rhs(dg, ms, ws)
    x = dg.empty()
    plan = P.Plan([dg], [g], [x], P.solve_opts(rtol=1e-10, maxit=300, restart=8), use_graph=use_graph)
    plan.dg_plan_solve()  # restart 8: several restart cycles
    its, relres, conv = plan.dg_plan_result(0)
    assert all(conv) and max(relres) <= 1e-10
    assert plan.dg_plan_stats()["cycles"] >= 2
    for q, m in enumerate(ms):
        G0 = O.dense_G(m, ws[q], inv * CONV_MULTS[q])
        gq = -O.residual(m, ws[q]).reshape(-1)
        assert np.linalg.norm(gq - G0 @ split(dg, ms, x)[q]) / np.linalg.norm(gq) < 1e-9, q


def test_plan_graph_equals_eager():
    levels = [3, 2, 1]
    P, dg, ms, ws, inv = make_batch(CONV, levels, CONV_MULTS, amp=0.05)
    dg.dg_set_linearization(dev(cat(ws).reshape(dg.ne, 4, -1)), inv)
    dg.dg_assemble()
    g = rhs(dg, ms, ws)
    xe, xg = dg.empty(), dg.empty()
    opts = P.solve_opts(rtol=1e-9, maxit=100, restart=10, omega=0.9)
    pe = P.Plan([dg], [g], [xe], opts, use_graph=False)
    pg = P.Plan([dg], [g], [xg], opts, use_graph=True)
    pe.dg_plan_solve()
    pg.dg_plan_solve()
    assert np.array_equal(host(xe), host(xg))
    assert pe.dg_plan_result(0) == pg.dg_plan_result(0)
    # a second solve replays the captured graph with new right-hand-side values (the stage
    # right-hand sides of other states: consistent with the operator's range)
    ws2 = [w + S.perturbation(m.ne, m.k, 0.02, 40 + q) for q, (m, w) in enumerate(zip(ms, ws))]
    g.copy_(rhs(dg, ms, ws2))
    pe.dg_plan_solve()
    pg.dg_plan_solve()
    assert np.array_equal(host(xe), host(xg))
    assert pg.dg_plan_stats()["graph_launches"] >= 2


@pytest.mark.parametrize("precision", ["fp64", "h16"])
def test_plan_two_handles_one_graph(precision):
    # a k = 2 batch and a k = 3 batch as parallel branches of one graph equal their eager solves
    torch, P = require_gpu()
    prec = P.DG_PRECOND_FP64 if precision == "fp64" else P.DG_PRECOND_FP32_H16
    sets = [(["u345", "u3"], [2, 1], [2.5, 3.0]), (["u3", "u345", "u345"], [3, 2, 1], [2.0, 2.5, 3.5])]
    dgs, gs, ms_all, ws_all = [], [], [], []
    for names, levels, mults in sets:
        P, dg, ms, ws, inv = make_batch(names, levels, mults, seed=11, amp=0.05)
        dg.dg_set_linearization(dev(cat(ws).reshape(dg.ne, 4, -1)), inv)
        dg.dg_assemble_precision(P.DG_PRECOND_FP64 if prec == P.DG_PRECOND_FP64 else P.DG_PRECOND_FP32)
        dgs.append(dg)
        gs.append(rhs(dg, ms, ws))
        ms_all.append(ms)
        ws_all.append(ws)
    opts = P.solve_opts(rtol=1e-8, maxit=200, precision=prec, omega=0.9 if precision != "fp64" else 1.0)
    xg = [d.empty() for d in dgs]
    pg = P.Plan(dgs, gs, xg, opts, use_graph=True)
    pg.dg_plan_solve()
    for i, d in enumerate(dgs):
        xe = d.empty()
        pe = P.Plan([d], [gs[i]], [xe], opts, use_graph=False)
        pe.dg_plan_solve()
        assert np.array_equal(host(xe), host(xg[i])), i
        its, relres, conv = pg.dg_plan_result(i)
        assert all(conv) and max(relres) <= 1e-8
        assert pe.dg_plan_result(0) == (its, relres, conv)
        pe.close()


def test_plan_single_problem_matches_fgmres():
    # one box: the device-driven solver and the host-driven fgmres_solve run the same method
    torch, P = require_gpu()
    from _gpu_common import pair
    dg, m = pair(*meshes()["u4"], [2, 1])
    w = O.project_tgv(m) + S.perturbation(m.ne, m.k, 0.1, 3)
    inv = 1.0 / S.acoustic_dt(4, 2)
    dg.dg_set_linearization(dev(w), inv)
    dg.dg_assemble()
    g = dev(-O.residual(m, w))
    for its in (5, 12):
        x1, x2 = dg.empty(), dg.empty()
        dg.fgmres_solve(g, x1, P.solve_opts(fixed_its=its))
        plan = P.Plan([dg], [g], [x2], P.solve_opts(fixed_its=its), use_graph=True)
        plan.dg_plan_solve()
        vol = m.vol()
        a = SV.remove_mean_pressure(host(x1).reshape(-1), m.ne, m.nb, vol)
        b = SV.remove_mean_pressure(host(x2).reshape(-1), m.ne, m.nb, vol)
        assert rel(b, a) < 1e-10, its
        plan.close()


def test_plan_reports_missed_tolerance():
    # a problem that exhausts maxit is reported, with the converged flags per problem
    P, dg, ms, ws, inv = make_batch(NAMES, [2, 1], MULTS)
    dg.dg_set_linearization(dev(cat(ws).reshape(dg.ne, 4, -1)), inv)
    dg.dg_assemble()
    g = rhs(dg, ms, ws)
    x = dg.empty()
    plan = P.Plan([dg], [g], [x], P.solve_opts(rtol=1e-12, maxit=3, restart=30), use_graph=True)
    assert plan.dg_plan_solve(check=False) == P.DG_ERR_NOT_CONVERGED
    its, relres, conv = plan.dg_plan_result(0)
    assert its == [3] * len(ms) and not any(conv)
    assert all(r > 1e-12 for r in relres)


def test_batch_rejects_whole_vector_reductions():
    P, dg, ms, ws, inv = make_batch(NAMES[:2], [2, 1], MULTS[:2])
    dg.dg_set_linearization(dev(cat(ws).reshape(dg.ne, 4, -1)), inv)
    dg.dg_assemble()
    g, x = dg.empty(), dg.empty()
    g.normal_()
    with pytest.raises(P.DgError):
        dg.fgmres_solve(g, x, P.solve_opts())
    with pytest.raises(P.DgError):
        dg.dg_jvp(g, x, mode=P.DG_JVP_FD)
    with pytest.raises(P.DgError):
        P.Plan([dg], [g], [x], P.solve_opts(smoother=P.DG_SMOOTH_GMRES))


def test_batch_of_channels():
    # boxes with no-slip walls (the walls flag applies to every box of a batch): the operator
    # equals one-box handles bit for bit, and the graph-captured solve of each problem passes the
    # oracle's exact operator
    torch, P = require_gpu()
    boxes = [(S.uniform_nodes(3), S.tanh_nodes(4, 1.15), S.uniform_nodes(2, np.pi)),
             (S.uniform_nodes(2), S.tanh_nodes(5, 1.15), S.uniform_nodes(3, np.pi))]
    mults = [1.5, 2.5]
    nu = S.NU_TGV * 20
    dg = P.DG(None, None, None, [2, 1], nu, S.AC_C, S.ETA, boxes=boxes, walls=True)
    dg.dg_set_problem_shifts(mults)
    ms = [O.Mesh(*b, 2, nu, S.AC_C, S.ETA, walls=True) for b in boxes]
    ws = []
    for q, m in enumerate(ms):
        x, _ = O.quad_points(m)
        y = x[..., 1]
        ws.append(O.project_points(m, np.stack([1 - y * y, 0 * y, 0 * y, 0 * y], axis=1))
                  + S.perturbation(m.ne, 2, 0.05, 30 + q))
    inv = 2.0
    dg.dg_set_linearization(dev(cat(ws).reshape(dg.ne, 4, -1)), inv)
    dg.dg_assemble()
    vs = [S.direction(m.ne, 2, 40 + q) for q, m in enumerate(ms)]
    out = dg.empty()
    dg.dg_jvp(dev(cat(vs).reshape(dg.ne, 4, -1)), out)
    for q, m in enumerate(ms):
        one = P.DG(*boxes[q], [2, 1], nu, S.AC_C, S.ETA, walls=True)
        one.dg_set_linearization(dev(ws[q]), inv * mults[q])
        o = one.empty()
        one.dg_jvp(dev(vs[q]), o)
        assert np.array_equal(split(dg, ms, out)[q], host(o).reshape(-1)), q
    g = rhs(dg, ms, ws)
    x = dg.empty()
    plan = P.Plan([dg], [g], [x], P.solve_opts(rtol=1e-10, maxit=200), use_graph=True)
    plan.dg_plan_solve()
    its, relres, conv = plan.dg_plan_result(0)
    assert all(conv)
    for q, m in enumerate(ms):
        G0 = O.dense_G(m, ws[q], inv * mults[q])
        gq = -O.residual(m, ws[q]).reshape(-1)
        assert np.linalg.norm(gq - G0 @ split(dg, ms, x)[q]) / np.linalg.norm(gq) < 1e-9, q
