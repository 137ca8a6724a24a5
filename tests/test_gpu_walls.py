"""GPU parity of the no-slip channel walls (Sec. 2.1; reading c8) against the oracle, through
the C ABI: the residual and the exact Jacobian action (FP64 at 1e-12, FP32 at its rounding),
the assembled blocks and coarse operators, one V-cycle, FGMRES at a fixed iteration count, a
converged stage, the reduced-precision cycle, and the learned coarse correction's features
(a wall contributes zero neighbour features).
"""
import numpy as np
import pytest

import oracle as O
import oracle.mlp as M
import oracle.solvers as SV
import synthetic as S
from _gpu_common import dev, host, rel, require_gpu

pytestmark = pytest.mark.gpu


def chan_nodes(nx, ny, nz, seed=0):
    xn = S.uniform_nodes(nx) if seed == 0 else S.perturbed_nodes(nx, seed=seed)
    return xn, S.tanh_nodes(ny, 1.15), S.uniform_nodes(nz, np.pi)


def wall_pair(nodes, levels, nu=S.NU_TGV * 20):
    torch, P = require_gpu()
    dg = P.DG(*nodes, levels, nu, S.AC_C, S.ETA, walls=True)
    m = O.Mesh(*nodes, levels[0], nu, S.AC_C, S.ETA, walls=True)
    return P, dg, m


def channel_state(m, seed, amp=0.05):
    """Laminar profile U(1 - y^2) e_x (projected) plus seeded modal noise."""
    x, _ = O.quad_points(m)
    y = x[..., 1]
    vals = np.stack([1.0 - y * y, 0 * y, 0 * y, 0 * y], axis=1)
    return O.project_points(m, vals) + S.perturbation(m.ne, m.k, amp, seed)


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_wall_operator(k):
    P, dg, m = wall_pair(chan_nodes(3, 4, 2, seed=3), [k])
    w = channel_state(m, 1, 0.2)
    f = dg.empty()
    dg.dg_residual(dev(w), f)
    assert rel(host(f).reshape(-1), O.residual(m, w).reshape(-1)) < 1e-12
    inv = 0.7
    dg.dg_set_linearization(dev(w), inv)
    v = S.direction(m.ne, k, 4)
    out = dg.empty()
    dg.dg_jvp(dev(v), out)
    ref = O.jvp(m, w, v, inv).reshape(-1)
    assert rel(host(out).reshape(-1), ref) < 1e-12


def test_poiseuille_on_the_gpu():
    # the exactly representable laminar profile: f_h is the strong form 2 nu U on the u modes
    nu = 0.05
    P, dg, m = wall_pair(chan_nodes(2, 4, 2), [2], nu=nu)
    x, _ = O.quad_points(m)
    y = x[..., 1]
    w = O.project_points(m, np.stack([0.8 * (1 - y * y), 0 * y, 0 * y, 0.3 + 0 * y], axis=1))
    f = dg.empty()
    dg.dg_residual(dev(w), f)
    expect = O.project_points(m, np.stack([2 * nu * 0.8 + 0 * y, 0 * y, 0 * y, 0 * y], axis=1))
    assert np.abs(host(f) - expect).max() < 1e-12 * np.abs(expect).max()


def setup_levels(nodes, levels, seed=1, amp=0.1, inv=2.0):
    P, dg, m = wall_pair(nodes, levels)
    w = channel_state(m, seed, amp)
    dg.dg_set_linearization(dev(w), inv)
    dg.dg_assemble()
    G0 = O.dense_G(m, w, inv)
    Gs = [G0] + [SV.inherited_operator(G0, m.ne, m.nb, O.nb(kl)) for kl in levels[1:]]
    nbs = [O.nb(kl) for kl in levels]
    Ds = [SV.block_inverses(G, m.ne, nb) for G, nb in zip(Gs, nbs)]
    return P, dg, m, w, Gs, Ds, nbs


@pytest.mark.parametrize("levels", [[2, 1], [3, 2, 1]])
def test_wall_assembly(levels):
    P, dg, m, w, Gs, Ds, nbs = setup_levels(chan_nodes(3, 4, 2, seed=5), levels)
    rng = np.random.default_rng(3)
    for lvl in range(len(levels)):
        x = rng.standard_normal(Gs[lvl].shape[0])
        g = rng.standard_normal(Gs[lvl].shape[0])
        xd = dev(x.reshape(m.ne, 4, nbs[lvl]))
        dg.block_jacobi_smooth(lvl, dev(g.reshape(m.ne, 4, nbs[lvl])), xd, 2, 0.8)
        ref = SV.block_jacobi(lambda v, G=Gs[lvl]: G @ v, Ds[lvl], g, x, 2, 0.8)
        assert rel(host(xd).reshape(-1), ref) < 1e-12, lvl
        if lvl >= 1:
            yd = dg.empty(lvl)
            dg.bsr_spmv(lvl, 1.0, dev(x.reshape(m.ne, 4, nbs[lvl])), 0.0, yd)
            assert rel(host(yd).reshape(-1), Gs[lvl] @ x) < 1e-12, lvl
            dg.bsr_spmv_t(lvl, 1.0, dev(x.reshape(m.ne, 4, nbs[lvl])), 0.0, yd)
            assert rel(host(yd).reshape(-1), Gs[lvl].T @ x) < 1e-12, lvl


def test_wall_vcycle_and_fgmres():
    levels = [3, 2, 1]
    P, dg, m, w, Gs, Ds, nbs = setup_levels(chan_nodes(3, 4, 2), levels)
    lv = [SV.Level(lambda v, G=G: G @ v, D, m.ne, nb) for G, D, nb in zip(Gs, Ds, nbs)]
    g = -O.residual(m, w).reshape(-1)
    ref = SV.mg_v(lv, 0, g, np.zeros_like(g), 2, 2, 2, 0.9)
    x = dg.empty()
    dg.pmg_vcycle(dev(g.reshape(x.shape)), x, P.solve_opts(omega=0.9))
    assert rel(host(x).reshape(-1), ref) < 1e-12
    its = 6
    xr, _, _ = SV.fgmres(lambda v: Gs[0] @ v, lambda v: SV.mg_v(lv, 0, v, np.zeros_like(v)), g, restart=30,
                         fixed_its=its)
    xf = dg.empty()
    info, rc = dg.fgmres_solve(dev(g.reshape(x.shape)), xf, P.solve_opts(fixed_its=its))
    vol = m.vol()
    assert rel(SV.remove_mean_pressure(host(xf).reshape(-1), m.ne, m.nb, vol),
               SV.remove_mean_pressure(xr, m.ne, m.nb, vol)) < 1e-10
    # a converged stage, checked with the oracle's exact operator
    xc = dg.empty()
    info, rc = dg.fgmres_solve(dev(g.reshape(x.shape)), xc, P.solve_opts(rtol=1e-10, maxit=200))
    assert rc == P.DG_OK
    assert np.linalg.norm(g - Gs[0] @ host(xc).reshape(-1)) / np.linalg.norm(g) < 1e-9


@pytest.mark.parametrize("storage", ["FP32", "FP32_H16"])
def test_wall_reduced_precision_cycle(storage):
    torch, P = require_gpu()
    prec = getattr(P, "DG_PRECOND_" + storage)
    levels = [3, 2, 1]
    P, dg, m = wall_pair(chan_nodes(3, 4, 2), levels)
    w = channel_state(m, 2, 0.1)
    inv = 2.0
    dg.dg_set_linearization(dev(w), inv)
    # the FP32 Jacobian action at its rounding
    dg.dg_assemble(precision=P.DG_PRECOND_FP32)
    g = -O.residual(m, w).reshape(-1)
    x = dg.empty()
    info, rc = dg.fgmres_solve(dev(g.reshape(x.shape)), x, P.solve_opts(rtol=1e-10, maxit=200, precision=prec,
                                                                          omega=0.9))
    assert rc == P.DG_OK
    G0 = O.dense_G(m, w, inv)
    assert np.linalg.norm(g - G0 @ host(x).reshape(-1)) / np.linalg.norm(g) < 1e-9


def test_wall_learned_features():
    # the network's coarse correction in the cycle: features of a missing neighbour are zero
    torch, P = require_gpu()
    levels = [2, 1]
    P, dg, m = wall_pair(chan_nodes(3, 4, 2), levels)
    w = channel_state(m, 3, 0.1)
    dg.dg_set_linearization(dev(w), 2.0)
    dg.dg_assemble()
    rng = np.random.default_rng(3)
    th = np.concatenate([rng.standard_normal(np.prod(shp)) / np.sqrt(shp[1] if len(shp) == 2 else 1)
                         for _, shp in M.SHAPES]).astype(np.float32)
    dg.dg_set_coarse_network(torch.from_numpy(th).cuda())
    gc = dev(S.direction(m.ne, 2, 9))
    zc = dg.empty()
    dg.pmg_vcycle(gc, zc, P.solve_opts(pre_sweeps=0, post_sweeps=0, coarse_sweeps=0,
                                       coarse_solver=P.DG_COARSE_LEARNED))
    dc = SV.restrict(host(gc).reshape(-1), m.ne, m.nb, O.nb(1)).reshape(m.ne, 4, O.nb(1))
    ref = SV.prolong(M.coarse_correction(th.astype(np.float64), dc, m.neighbours(), O.nb(1)).reshape(-1),
                     m.ne, m.nb, O.nb(1))
    assert rel(host(zc).reshape(-1), ref) < 2e-3


def test_quad_points_and_projection():
    # the channel field at the handle's Gauss points, projected on the GPU and by the oracle
    P, dg, m = wall_pair(chan_nodes(3, 4, 2, seed=2), [3])
    xyz = host(dg.dg_quad_points())
    xo, _ = O.quad_points(m)
    np.testing.assert_allclose(xyz, xo, rtol=0, atol=1e-14)
    vals = np.ascontiguousarray(np.stack(S.channel_field(xo[..., 0], xo[..., 1], xo[..., 2]), axis=1))
    w = dg.empty()
    dg.dg_project_points(dev(vals), w)
    assert rel(host(w).reshape(-1), O.project_points(m, vals).reshape(-1)) < 1e-13
