"""Pins of the oracle's p-multigrid and FGMRES algorithms (Sec. 2.4, Algorithms 2-3).

Checks against closed forms and direct solves: restriction/prolongation are a
left inverse pair and the restriction is the L2 projection; the block-sparse
coarse storage reproduces the inherited operator; FGMRES converges to the
dense direct solution (modulo the constant-pressure null space); one V-cycle
equals the product of its explicit iteration matrices.
"""
import numpy as np
import pytest

import oracle as O
import oracle.solvers as SV
import synthetic as S


@pytest.fixture(scope="module")
def setup3():
    n, k = 3, 2
    m = O.Mesh(S.uniform_nodes(n), S.uniform_nodes(n), S.uniform_nodes(n), k, S.NU_TGV, S.AC_C, S.ETA)
    w = O.project_tgv(m)
    dt = S.acoustic_dt(n, k)
    G0 = O.dense_G(m, w, 1.0 / dt)
    return m, w, dt, G0


def test_restrict_prolong():
    ne, nbf, nbc = 5, 20, 10
    rng = np.random.default_rng(0)
    xc = rng.standard_normal(ne * 4 * nbc)
    np.testing.assert_array_equal(SV.restrict(SV.prolong(xc, ne, nbf, nbc), ne, nbf, nbc), xc)
    xf = rng.standard_normal(ne * 4 * nbf)
    pr = SV.prolong(SV.restrict(xf, ne, nbf, nbc), ne, nbf, nbc)
    np.testing.assert_array_equal(SV.prolong(SV.restrict(pr, ne, nbf, nbc), ne, nbf, nbc), pr)
    # the restriction is the adjoint of the injection (L2 projection, orthonormal basis)
    assert abs(np.dot(SV.restrict(xf, ne, nbf, nbc), xc) - np.dot(xf, SV.prolong(xc, ne, nbf, nbc))) < 1e-12


@pytest.mark.parametrize("n", [2, 3])
def test_bsr_reproduces_inherited_operator(n):
    m = O.Mesh(S.uniform_nodes(n), S.uniform_nodes(n), S.uniform_nodes(n), 2, S.NU_TGV, S.AC_C, S.ETA)
    w = O.project_tgv(m) + S.perturbation(m.ne, 2, 0.1, 1)
    G0 = O.dense_G(m, w, 0.8)
    nbc = O.nb(1)
    G1 = SV.inherited_operator(G0, m.ne, m.nb, nbc)
    cols, vals = SV.bsr_from_dense(G1, m.ne, nbc, m.neighbours())
    x = np.random.default_rng(2).standard_normal(G1.shape[0])
    np.testing.assert_allclose(SV.bsr_matvec(cols, vals, x), G1 @ x, atol=1e-12 * np.abs(G1).max())
    # the sparsity is exactly diagonal + face neighbours: everything else in G1 is zero
    mask = np.zeros_like(G1, dtype=bool)
    b = 4 * nbc
    for e in range(m.ne):
        for c in cols[e]:
            mask[e * b:(e + 1) * b, c * b:(c + 1) * b] = True
    assert np.abs(G1[~mask]).max() == 0.0


def test_fgmres_converges_to_direct_solution(setup3):
    m, w, dt, G0 = setup3
    g = -O.residual(m, w).reshape(-1)
    Dinv = SV.block_inverses(G0, m.ne, m.nb)
    x, its, hist = SV.fgmres(lambda v: G0 @ v, lambda v: SV.apply_block_inverse(Dinv, v), g,
                             restart=30, maxit=400, rtol=1e-12)
    xd = np.linalg.lstsq(G0, g, rcond=None)[0]
    vol = m.vol()
    a = SV.remove_mean_pressure(x, m.ne, m.nb, vol)
    b = SV.remove_mean_pressure(xd, m.ne, m.nb, vol)
    assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-10
    assert np.linalg.norm(g - G0 @ x) / np.linalg.norm(g) < 1e-11
    assert hist[-1] <= 1e-12 * hist[0] and its < 400


def test_vcycle_is_product_of_iteration_matrices(setup3):
    m, w, dt, G0 = setup3
    nbc = O.nb(1)
    G1 = SV.inherited_operator(G0, m.ne, m.nb, nbc)
    D0 = SV.block_inverses(G0, m.ne, m.nb)
    D1 = SV.block_inverses(G1, m.ne, nbc)
    levels = [SV.Level(lambda v: G0 @ v, D0, m.ne, m.nb), SV.Level(lambda v: G1 @ v, D1, m.ne, nbc)]
    pre, post, cs, om = 2, 2, 3, 0.9
    n0, n1 = G0.shape[0], G1.shape[0]
    Bd0 = np.zeros((n0, n0))
    Bd1 = np.zeros((n1, n1))
    b0, b1 = 4 * m.nb, 4 * nbc
    for e in range(m.ne):
        Bd0[e * b0:(e + 1) * b0, e * b0:(e + 1) * b0] = D0[e]
        Bd1[e * b1:(e + 1) * b1, e * b1:(e + 1) * b1] = D1[e]

    def sweeps(G, Dm, nu):
        # nu Jacobi sweeps: x_nu = T^nu x_0 + A g with T = I - om D^-1 G
        T = np.eye(G.shape[0]) - om * Dm @ G
        A = np.zeros_like(G)
        P = np.eye(G.shape[0])
        for _ in range(nu):
            A = A + P @ (om * Dm)
            P = T @ P
        return P, A

    T0post, Apost = sweeps(G0, Bd0, post)
    _, Apre = sweeps(G0, Bd0, pre)
    _, C = sweeps(G1, Bd1, cs)
    idx = SV.coarse_index(m.ne, m.nb, nbc)
    R = np.zeros((n1, n0))
    R[np.arange(n1), idx] = 1.0
    B = T0post @ (Apre + R.T @ C @ R @ (np.eye(n0) - G0 @ Apre)) + Apost
    g = np.random.default_rng(3).standard_normal(n0)
    v = SV.mg_v(levels, 0, g, np.zeros(n0), pre, post, cs, om)
    np.testing.assert_allclose(v, B @ g, atol=1e-11 * np.abs(B @ g).max())
    # MG_full with these parts is linear too: check it against its own unit-vector matrix on a sample
    f1 = SV.mg_full(levels, 0, g, pre, post, cs, om)
    f2 = SV.mg_full(levels, 0, 2.0 * g, pre, post, cs, om)
    np.testing.assert_allclose(f2, 2.0 * f1, atol=1e-11 * np.abs(f1).max())


def test_convergence_factor():
    assert abs(SV.convergence_factor(1.0, 1e-8, 4) - 1e-2) < 1e-15


@pytest.mark.parametrize("iters", [1, 3, 6])
def test_gmres_smoother_is_the_krylov_minimiser(setup3, iters):
    # GMRES(iters) left-preconditioned by EWBJ minimises ||D^-1 (g - G y)|| over
    # x0 + span{r, (D^-1 G) r, ...}: compare with a least-squares solve on that explicit basis
    m, w, dt, G0 = setup3
    D = SV.block_inverses(G0, m.ne, m.nb)
    rng = np.random.default_rng(11)
    g = rng.standard_normal(G0.shape[0])
    x0 = rng.standard_normal(G0.shape[0]) * 0.1
    got = SV.gmres_smooth(lambda v: G0 @ v, D, g, x0, iters)
    A = lambda v: SV.apply_block_inverse(D, G0 @ v)
    r0 = SV.apply_block_inverse(D, g - G0 @ x0)
    K = [r0]
    for _ in range(iters - 1):
        K.append(A(K[-1]))
    K = np.array(K).T
    K, _ = np.linalg.qr(K)  # orthonormal basis of the same space
    AK = np.stack([A(K[:, i]) for i in range(K.shape[1])], 1)
    c = np.linalg.lstsq(AK, r0, rcond=None)[0]
    ref = x0 + K @ c
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-9
    # the preconditioned residual never grows
    res = lambda y: np.linalg.norm(SV.apply_block_inverse(D, g - G0 @ y))
    assert res(got) <= res(x0) * (1 + 1e-12)



def test_stabilisation_part_and_its_rescaling():
    # The viscous stabilisation (BR2 penalty) part of G is G(eta) - G(0): linear in eta, and a
    # symmetric positive semidefinite form (eta times the lifted jumps' inner product, Sec. 2.1,
    # Appendix A). The rescaled inherited operator reduces to the inherited one for S = 1 and
    # scales exactly that part by S_0^l = k_l (k_l + 3) / (k_0 (k_0 + 3)).
    n, k = 2, 2
    xs = S.uniform_nodes(n)
    w = None
    Gs = {}
    for eta in (0.0, 7.0, 14.0):
        m = O.Mesh(xs, xs, xs, k, S.NU_TGV, S.AC_C, eta)
        if w is None:
            w = O.project_tgv(m) + S.perturbation(m.ne, k, 0.1, 4)
        Gs[eta] = O.dense_G(m, w, 0.5)
    stb = Gs[7.0] - Gs[0.0]
    np.testing.assert_allclose(Gs[14.0] - Gs[0.0], 2.0 * stb, atol=1e-11 * np.abs(stb).max())
    np.testing.assert_allclose(stb, stb.T, atol=1e-12 * np.abs(stb).max())
    assert np.linalg.eigvalsh(0.5 * (stb + stb.T)).min() > -1e-10 * np.abs(stb).max()
    # only the velocity rows and columns carry it (the penalty acts on the velocity jumps)
    nb = O.nb(k)
    p_idx = [e * 4 * nb + 3 * nb + j for e in range(m.ne) for j in range(nb)]
    assert np.abs(stb[p_idx]).max() == 0.0 and np.abs(stb[:, p_idx]).max() == 0.0
    assert abs(SV.stb_scaling(4, 2) - 10.0 / 28.0) < 1e-15 and SV.stb_scaling(3, 3) == 1.0
    G = Gs[7.0]
    nbc = O.nb(1)
    np.testing.assert_array_equal(SV.rescaled_inherited_operator(G, stb, m.ne, nb, nb, k, k),
                                  SV.inherited_operator(G, m.ne, nb, nb))
    Gr = SV.rescaled_inherited_operator(G, stb, m.ne, nb, nbc, k, 1)
    Gi = SV.inherited_operator(G, m.ne, nb, nbc)
    Si = SV.inherited_operator(stb, m.ne, nb, nbc)
    np.testing.assert_allclose(Gr - Gi, (SV.stb_scaling(k, 1) - 1.0) * Si, atol=1e-14 * np.abs(G).max())
