"""GPU parity of the p-multigrid and FGMRES parts against the oracle's dense counterparts (through the C ABI).

Operators and one V-cycle application agree to rounding (relative 1e-12).
Krylov solves are compared at a fixed iteration count (no early exit), where
rounding differences of two Gram-Schmidt variants are amplified by the
conditioning, with a 1e-10 bound; converged solves are checked by their true
residual under the oracle's exact operator.
"""
import numpy as np
import pytest

import oracle as O
import oracle.solvers as SV
import synthetic as S
from _gpu_common import dev, host, meshes, pair, rel

pytestmark = pytest.mark.gpu


def setup(name, levels, seed=1, amp=0.2, dt=None):
    import paper_1809_00866_gb300 as P
    dg, m = pair(*meshes()[name], levels)
    w = O.project_tgv(m) + S.perturbation(m.ne, m.k, amp, seed)
    inv = 1.0 / (dt if dt else S.acoustic_dt(m.nx, m.k))
    dg.dg_set_linearization(dev(w), inv)
    dg.dg_assemble()
    G0 = O.dense_G(m, w, inv)
    Gs = [G0]
    for kl in levels[1:]:
        Gs.append(SV.inherited_operator(G0, m.ne, m.nb, O.nb(kl)))
    nbs = [O.nb(k) for k in levels]
    Ds = [SV.block_inverses(G, m.ne, nb) for G, nb in zip(Gs, nbs)]
    return P, dg, m, w, inv, Gs, Ds, nbs


def test_restrict_prolong():
    dg, m = pair(*meshes()["box233"], [3, 2, 1])
    rng = np.random.default_rng(0)
    xf = rng.standard_normal(m.shape())
    xc = dg.empty(1)
    dg.pmg_restrict(0, dev(xf), xc)
    np.testing.assert_array_equal(host(xc), SV.restrict(xf, m.ne, m.nb, O.nb(2)).reshape(xc.shape))
    y = rng.standard_normal(m.shape())
    yd = dev(y)
    dg.pmg_prolong(0, xc, yd)
    np.testing.assert_allclose(host(yd), y + SV.prolong(host(xc), m.ne, m.nb, O.nb(2)).reshape(y.shape),
                               rtol=0, atol=0)


@pytest.mark.parametrize("name,levels", [("u2", [3, 2, 1]), ("u3", [2, 1]), ("box233", [3, 1])])
def test_bsr_and_block_jacobi(name, levels):
    P, dg, m, w, inv, Gs, Ds, nbs = setup(name, levels)
    rng = np.random.default_rng(5)
    for lvl in range(len(levels)):
        x = rng.standard_normal(Gs[lvl].shape[0])
        g = rng.standard_normal(Gs[lvl].shape[0])
        if lvl >= 1:
            y0 = rng.standard_normal(Gs[lvl].shape[0])
            yd = dev(y0.reshape(m.ne, 4, nbs[lvl]))
            dg.bsr_spmv(lvl, 0.7, dev(x.reshape(m.ne, 4, nbs[lvl])), -0.3, yd)
            assert rel(host(yd).reshape(-1), 0.7 * Gs[lvl] @ x - 0.3 * y0) < 1e-12
        xd = dev(x.reshape(m.ne, 4, nbs[lvl]))
        dg.block_jacobi_smooth(lvl, dev(g.reshape(m.ne, 4, nbs[lvl])), xd, 2, 0.8)
        ref = SV.block_jacobi(lambda v, G=Gs[lvl]: G @ v, Ds[lvl], g, x, 2, 0.8)
        assert rel(host(xd).reshape(-1), ref) < 1e-12, lvl


@pytest.mark.parametrize("name,levels,sweeps", [("u3", [2, 1], (2, 2, 2)), ("u2", [3, 2, 1], (1, 2, 3)),
                                                ("box233", [4, 2, 1], (2, 1, 4))])
def test_vcycle(name, levels, sweeps):
    P, dg, m, w, inv, Gs, Ds, nbs = setup(name, levels)
    lv = [SV.Level(lambda v, G=G: G @ v, D, m.ne, nb) for G, D, nb in zip(Gs, Ds, nbs)]
    g = np.random.default_rng(9).standard_normal(Gs[0].shape[0])
    pre, post, cs = sweeps
    ref = SV.mg_v(lv, 0, g, np.zeros_like(g), pre, post, cs, 0.9)
    opts = P.solve_opts(pre_sweeps=pre, post_sweeps=post, coarse_sweeps=cs, omega=0.9)
    x = dg.empty()
    dg.pmg_vcycle(dev(g.reshape(x.shape)), x, opts)
    assert rel(host(x).reshape(-1), ref) < 1e-12
    ref_f = SV.mg_full(lv, 0, g, pre, post, cs, 0.9)
    # MG_full as the preconditioner of one fixed FGMRES iteration equals a scaled MG_full application
    opts_f = P.solve_opts(restart=1, fixed_its=1, precond=P.DG_PREC_FULLV, pre_sweeps=pre, post_sweeps=post,
                          coarse_sweeps=cs, omega=0.9)
    xf = dg.empty()
    dg.fgmres_solve(dev(g.reshape(x.shape)), xf, opts_f)
    z = ref_f
    Gz = Gs[0] @ z
    alpha = np.dot(Gz, g) / np.dot(Gz, Gz)
    assert rel(host(xf).reshape(-1), alpha * z) < 1e-11


@pytest.mark.parametrize("name,levels", [("u3", [2, 1]), ("u2", [3, 2, 1])])
def test_fgmres_fixed_iterations(name, levels):
    P, dg, m, w, inv, Gs, Ds, nbs = setup(name, levels)
    lv = [SV.Level(lambda v, G=G: G @ v, D, m.ne, nb) for G, D, nb in zip(Gs, Ds, nbs)]
    g = -O.residual(m, w).reshape(-1)
    its = 6
    xr, _, _ = SV.fgmres(lambda v: Gs[0] @ v, lambda v: SV.mg_v(lv, 0, v, np.zeros_like(v)), g, restart=30,
                         fixed_its=its)
    x = dg.empty()
    info, rc = dg.fgmres_solve(dev(g.reshape(x.shape)), x, P.solve_opts(fixed_its=its))
    assert info.its == its
    vol = m.vol()
    a = SV.remove_mean_pressure(host(x).reshape(-1), m.ne, m.nb, vol)
    b = SV.remove_mean_pressure(xr, m.ne, m.nb, vol)
    assert rel(a, b) < 1e-10


def test_fgmres_converges_tgv4_p2():
    # one linearly implicit stage of the 4^3 P2 Taylor-Green workload, 2-level V-cycle, rel-tol 1e-10
    import paper_1809_00866_gb300 as P
    dg, m = pair(*meshes()["u4"], [2, 1])
    w = O.project_tgv(m)
    inv = 1.0 / S.acoustic_dt(4, 2)
    wd = dev(w)
    f = dg.empty()
    dg.dg_residual(wd, f)
    g = -f
    dg.dg_set_linearization(wd, inv)
    dg.dg_assemble()
    x = dg.empty()
    info, rc = dg.fgmres_solve(g.contiguous(), x, P.solve_opts(rtol=1e-10, maxit=200))
    assert rc == P.DG_OK and info.true_relres <= 1e-10
    G0 = O.dense_G(m, w, inv)
    gr = host(g).reshape(-1)
    assert np.linalg.norm(gr - G0 @ host(x).reshape(-1)) / np.linalg.norm(gr) < 1e-9


def test_fgmres_fd_mode_generic_state():
    # Finite-difference outer products (Eqs. (matrix-free), (epsdef)). The pure Taylor-Green
    # state lies on a kink of the upwinded tangential flux (u* = 0 with u_t,L = -u_t,R on faces
    # where cos z is odd), where a one-sided difference sees only one side; a generic state is
    # differentiable, and the FD action then serves tolerances above its ~1e-7 noise (Sec. 2.3).
    # A small time step (acoustic CFL 2) and no preconditioner keep the solve well posed there.
    import paper_1809_00866_gb300 as P
    dg, m = pair(*meshes()["u4"], [2, 1])
    w = O.project_tgv(m) + S.perturbation(m.ne, 2, 0.01, 21)
    inv = 1.0 / S.acoustic_dt(4, 2, cfl=2.0)
    wd = dev(w)
    f = dg.empty()
    dg.dg_residual(wd, f)
    g = (-f).contiguous()
    dg.dg_set_linearization(wd, inv)
    dg.dg_assemble()
    xf = dg.empty()
    info, rc = dg.fgmres_solve(g, xf, P.solve_opts(rtol=1e-5, maxit=300, jvp_mode=P.DG_JVP_FD,
                                                   precond=P.DG_PREC_NONE))
    assert rc == P.DG_OK and info.true_relres <= 1e-5
    G0 = O.dense_G(m, w, inv)
    gr = host(g).reshape(-1)
    assert np.linalg.norm(gr - G0 @ host(xf).reshape(-1)) / np.linalg.norm(gr) < 1e-4


@pytest.mark.parametrize("name,levels,its", [("u3", [2, 1], (2, 2, 6)), ("u2", [3, 2, 1], (3, 2, 8))])
def test_vcycle_gmres_smoother(name, levels, its):
    # GMRES[EWBJ] smoothers (Sec. 2.4.3); the device version orthogonalises with classical
    # Gram-Schmidt twice, the oracle with modified Gram-Schmidt: equal up to rounding of the
    # small least-squares problems.
    P, dg, m, w, inv, Gs, Ds, nbs = setup(name, levels)
    lv = [SV.Level(lambda v, G=G: G @ v, D, m.ne, nb) for G, D, nb in zip(Gs, Ds, nbs)]
    g = np.random.default_rng(17).standard_normal(Gs[0].shape[0])
    pre, post, cs = its
    ref = SV.mg_v(lv, 0, g, np.zeros_like(g), pre, post, cs, 1.0, "gmres")
    opts = P.solve_opts(pre_sweeps=pre, post_sweeps=post, coarse_sweeps=cs, smoother=P.DG_SMOOTH_GMRES)
    x = dg.empty()
    dg.pmg_vcycle(dev(g.reshape(x.shape)), x, opts)
    assert rel(host(x).reshape(-1), ref) < 1e-10
    # FGMRES at a fixed iteration count with this preconditioner
    gg = -O.residual(m, w).reshape(-1)
    xr, _, _ = SV.fgmres(lambda v: Gs[0] @ v, lambda v: SV.mg_v(lv, 0, v, np.zeros_like(v), pre, post, cs, 1.0,
                                                               "gmres"), gg, restart=30, fixed_its=4)
    xg = dg.empty()
    info, rc = dg.fgmres_solve(dev(gg.reshape(x.shape)), xg, P.solve_opts(fixed_its=4, pre_sweeps=pre,
                                                                            post_sweeps=post, coarse_sweeps=cs,
                                                                            smoother=P.DG_SMOOTH_GMRES))
    vol = m.vol()
    a = SV.remove_mean_pressure(host(xg).reshape(-1), m.ne, m.nb, vol)
    b = SV.remove_mean_pressure(xr, m.ne, m.nb, vol)
    assert rel(a, b) < 1e-9


@pytest.mark.parametrize("name,levels", [("u3", [2, 1]), ("u2", [3, 2, 1]), ("box233", [4, 2, 1])])
def test_fp32_preconditioner_cycle(name, levels):
    # Reduced-precision preconditioner: the same V-cycle with FP32 operator products,
    # LU factors, coarse blocks and vectors. Its deviation from the FP64 cycle is rounding of
    # FP32 arithmetic (unit roundoff 6e-8) amplified through the cycle: stated bound 1e-5.
    P, dg, m, w, inv, Gs, Ds, nbs = setup(name, levels)
    lv = [SV.Level(lambda v, G=G: G @ v, D, m.ne, nb) for G, D, nb in zip(Gs, Ds, nbs)]
    g = -O.residual(m, w).reshape(-1)
    ref = SV.mg_v(lv, 0, g, np.zeros_like(g))
    x64, x32 = dg.empty(), dg.empty()
    gd = dev(g.reshape(x64.shape))
    dg.pmg_vcycle(gd, x64, P.solve_opts())
    dg.pmg_vcycle(gd, x32, P.solve_opts(precision=P.DG_PRECOND_FP32))
    assert rel(host(x64).reshape(-1), ref) < 1e-12
    assert rel(host(x32).reshape(-1), ref) < 1e-5


def test_fp32_preconditioner_reaches_fp64_accuracy():
    # FGMRES and its products with G stay FP64, so the FP32 preconditioner does not limit the
    # attainable accuracy: one implicit stage of the 4^3 P2 Taylor-Green workload to 1e-10.
    import paper_1809_00866_gb300 as P
    dg, m = pair(*meshes()["u4"], [2, 1])
    w = O.project_tgv(m)
    inv = 1.0 / S.acoustic_dt(4, 2)
    wd = dev(w)
    f = dg.empty()
    dg.dg_residual(wd, f)
    g = (-f).contiguous()
    dg.dg_set_linearization(wd, inv)
    dg.dg_assemble()
    # damped block Jacobi (omega 0.7): the FP32 rounding noise leaves the symmetric subspace of the
    # Taylor-Green right-hand side, where undamped block Jacobi is not a convergent smoother
    x64, x32 = dg.empty(), dg.empty()
    i64, rc64 = dg.fgmres_solve(g, x64, P.solve_opts(rtol=1e-10, maxit=300, omega=0.7))
    i32, rc32 = dg.fgmres_solve(g, x32, P.solve_opts(rtol=1e-10, maxit=300, omega=0.7,
                                                     precision=P.DG_PRECOND_FP32))
    assert rc64 == P.DG_OK and rc32 == P.DG_OK
    G0 = O.dense_G(m, w, inv)
    gr = host(g).reshape(-1)
    assert np.linalg.norm(gr - G0 @ host(x32).reshape(-1)) / np.linalg.norm(gr) < 1e-9
    vol = m.vol()
    a = SV.remove_mean_pressure(host(x32).reshape(-1), m.ne, m.nb, vol)
    b = SV.remove_mean_pressure(host(x64).reshape(-1), m.ne, m.nb, vol)
    assert rel(a, b) < 1e-8


@pytest.mark.parametrize("name,levels", [("u3", [2, 1]), ("box233", [4, 2, 1])])
def test_fp32_assembly(name, levels):
    # assembly in FP32 (state blocks, inherited coarse blocks, LU factors): the cycle built on it
    # stays within the FP32 bound of the FP64 cycle; the FP64 cycle then refuses to run
    P, dg, m, w, inv, Gs, Ds, nbs = setup(name, levels)
    lv = [SV.Level(lambda v, G=G: G @ v, D, m.ne, nb) for G, D, nb in zip(Gs, Ds, nbs)]
    g = -O.residual(m, w).reshape(-1)
    ref = SV.mg_v(lv, 0, g, np.zeros_like(g), 2, 2, 2, 0.7)
    dg.dg_assemble(precision=P.DG_PRECOND_FP32)
    x = dg.empty()
    gd = dev(g.reshape(x.shape))
    dg.pmg_vcycle(gd, x, P.solve_opts(omega=0.7, precision=P.DG_PRECOND_FP32))
    assert rel(host(x).reshape(-1), ref) < 1e-5
    with pytest.raises(P.DgError) as e:
        dg.pmg_vcycle(gd, x, P.solve_opts(omega=0.7))
    assert e.value.code == P.DG_ERR_STATE


def test_lagged_preconditioner():
    # the blocks assembled at state A precondition the solve linearised at state B (Sec. 4.1 lags
    # them over time steps); the solution is judged by B's exact operator
    import paper_1809_00866_gb300 as P
    dg, m = pair(*meshes()["u4"], [2, 1])
    wa = O.project_tgv(m)
    wb = 0.8 * wa  # another Taylor-Green state (weaker flow), on which the block-Jacobi cycle converges
    inv = 1.0 / S.acoustic_dt(m.nx, m.k)
    dg.dg_set_linearization(dev(wa), inv)
    dg.dg_assemble()
    g = dg.empty()
    dg.dg_set_linearization_rhs(dev(wb), inv, g)
    x = dg.empty()
    o = P.solve_opts(rtol=1e-9, maxit=300)
    with pytest.raises(P.DgError):
        dg.fgmres_solve(g, x, o)  # the assembly belongs to another linearisation
    dg.dg_reuse_assembly()
    info, rc = dg.fgmres_solve(g, x, o)
    assert rc == P.DG_OK
    Gb = O.dense_G(m, wb, inv)
    gr = host(g).reshape(-1)
    assert np.linalg.norm(gr - Gb @ host(x).reshape(-1)) <= 2e-9 * np.linalg.norm(gr)


@pytest.mark.parametrize("name,levels", [("u3", [2, 1]), ("box233", [4, 2, 1])])
@pytest.mark.parametrize("storage,bound", [("H16", 5e-3), ("BF16", 4e-2)])
def test_16bit_block_storage(name, levels, storage, bound):
    # the FP32 cycle with its block inverses and block-sparse operators stored in 16 bits and
    # multiplied with FP32 accumulation: each stored entry carries a relative rounding error of
    # at most 2^-11 (FP16) or 2^-8 (bfloat16), which the cycle passes on to its result; the
    # bounds are 10x those unit roundoffs
    P, dg, m, w, inv, Gs, Ds, nbs = setup(name, levels)
    lv = [SV.Level(lambda v, G=G: G @ v, D, m.ne, nb) for G, D, nb in zip(Gs, Ds, nbs)]
    g = -O.residual(m, w).reshape(-1)
    ref = SV.mg_v(lv, 0, g, np.zeros_like(g))
    prec = getattr(P, "DG_PRECOND_FP32_" + storage)
    x16 = dg.empty()
    dg.pmg_vcycle(dev(g.reshape(x16.shape)), x16, P.solve_opts(precision=prec))
    assert rel(host(x16).reshape(-1), ref) < bound


def test_16bit_block_storage_reaches_fp64_accuracy():
    # FGMRES stays FP64: with FP16 block storage in the cycle one implicit stage of the 4^3 P2
    # Taylor-Green workload still reaches 1e-10, checked with the oracle's exact operator
    import paper_1809_00866_gb300 as P
    dg, m = pair(*meshes()["u4"], [2, 1])
    w = O.project_tgv(m)
    inv = 1.0 / S.acoustic_dt(4, 2)
    g = dg.empty()
    dg.dg_set_linearization_rhs(dev(w), inv, g)
    dg.dg_assemble(precision=P.DG_PRECOND_FP32_H16)
    x = dg.empty()
    info, rc = dg.fgmres_solve(g, x, P.solve_opts(rtol=1e-10, maxit=300, omega=0.7,
                                                   precision=P.DG_PRECOND_FP32_H16))
    assert rc == P.DG_OK
    G0 = O.dense_G(m, w, inv)
    gr = host(g).reshape(-1)
    assert np.linalg.norm(gr - G0 @ host(x).reshape(-1)) / np.linalg.norm(gr) < 1e-9


@pytest.mark.parametrize("name,levels", [("u3", [2, 1]), ("box233", [4, 2, 1]), ("u2", [3, 2, 1])])
def test_rescaled_inherited_coarse_operators(name, levels):
    # Appendix A: coarse operators with the stabilisation part weighted by S_0^l, against the
    # oracle's M (G0 + (S - 1) Gstb) M^T with Gstb = G(eta) - G(0); and one V-cycle on them
    P, dg, m, w, inv, Gs, Ds, nbs = setup(name, levels)
    dg.dg_set_stb_rescaling(True)
    dg.dg_assemble()
    m0 = O.Mesh(m.xn, m.yn, m.zn, m.k, S.NU_TGV, S.AC_C, 0.0)
    stb = Gs[0] - O.dense_G(m0, w, inv)
    rng = np.random.default_rng(23)
    Gr = [Gs[0]]
    for lvl in range(1, len(levels)):
        G = SV.rescaled_inherited_operator(Gs[0], stb, m.ne, m.nb, nbs[lvl], levels[0], levels[lvl])
        Gr.append(G)
        x = rng.standard_normal(G.shape[0])
        y = dg.empty(lvl)
        dg.bsr_spmv(lvl, 1.0, dev(x.reshape(y.shape)), 0.0, y)
        np.testing.assert_allclose(host(y).reshape(-1), G @ x, rtol=0, atol=1e-12 * np.abs(G).max() * np.abs(x).max() * 40)
        # the rescaling changed the operator (S < 1 for every coarse level here)
        assert np.abs(G - SV.inherited_operator(Gs[0], m.ne, m.nb, nbs[lvl])).max() > 1e-6 * np.abs(G).max()
    lv = [SV.Level(lambda v, G=G: G @ v, SV.block_inverses(G, m.ne, nb), m.ne, nb) for G, nb in zip(Gr, nbs)]
    g = -O.residual(m, w).reshape(-1)
    ref = SV.mg_v(lv, 0, g, np.zeros_like(g))
    x = dg.empty()
    dg.pmg_vcycle(dev(g.reshape(x.shape)), x, P.solve_opts())
    assert rel(host(x).reshape(-1), ref) < 1e-12
