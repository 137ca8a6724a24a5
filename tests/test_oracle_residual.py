"""Pins of the oracle's residual f_h (Eq. (NSdiscrRes)) and Jacobian action (Eqs. (jacTrilFnotNU), (jacTrilnu)).

Each check rests on something the paper or the mathematics fixes, not on the
oracle's own formulas: free-stream preservation and conservation (consistent,
conservative DG fluxes), equivariance under a 90-degree rotation, symmetry and
positivity of the BR2 viscous form, the strong form for continuous fields,
central finite differences, the paper's matrix-free formula, and the equality
of inherited and non-inherited inviscid coarse operators (Sec. 2.4.2).
"""
import itertools
import math

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

import oracle as O
import synthetic as S


def cube(n, k, nu=0.02, nodes=None):
    xn = S.uniform_nodes(n) if nodes is None else nodes
    return O.Mesh(xn, xn, xn, k, nu, S.AC_C, S.ETA)


def box(n, k, nu=0.02):
    return O.Mesh(S.perturbed_nodes(n, seed=1), S.perturbed_nodes(n + 1, seed=2), S.perturbed_nodes(n, seed=3),
                  k, nu, S.AC_C, S.ETA)


def random_state(m, seed, amp=0.3):
    return O.project_tgv(m) + S.perturbation(m.ne, m.k, amp, seed)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_free_stream_preserved(k):
    m = box(2, k)
    x, _ = O.quad_points(m)
    vals = np.zeros((m.ne, 4, x.shape[1]))
    for v, c in enumerate((0.3, -0.7, 0.45, 1.3)):
        vals[:, v] = c
    w = O.project_points(m, vals)
    assert np.abs(O.residual(m, w)).max() < 1e-13


@pytest.mark.parametrize("k", [1, 2])
def test_global_conservation(k):
    # test function z = e_i (constant 1) = sqrt(|K|) phi_0 in every element: the volume term
    # has grad z = 0 and the face term [z] = 0 on a periodic mesh, so sum_K sqrt|K| f[K][i][0] = 0
    m = box(2, k)
    w = random_state(m, 5)
    f = O.residual(m, w)
    s = np.sqrt(m.vol())
    scale = np.abs(f).max()
    for i in range(4):
        assert abs(np.dot(s, f[:, i, 0])) < 1e-12 * scale * m.ne


def rotate_z(w, n, k):
    """Coefficients of R u(R^-1 x) for a 90-degree rotation about the z axis through the centre
    of the periodic cube (uniform n^3 cells). R(x, y, z) = (-y, x, z)."""
    md = [tuple(r) for r in O.modes(k)]
    pos = {m: i for i, m in enumerate(md)}
    W = np.asarray(w).reshape(n, n, n, 4, len(md))  # [k][j][i]
    out = np.zeros_like(W)
    for kk, jj, ii in itertools.product(range(n), repeat=3):
        src = W[kk, n - 1 - ii, jj]  # source cell (i_s, j_s) = (j', n-1-i')
        for j, (a, b, c) in enumerate(md):
            t = pos[(b, a, c)]
            sg = (-1.0) ** b
            out[kk, jj, ii, 0, t] = -sg * src[1, j]
            out[kk, jj, ii, 1, t] = sg * src[0, j]
            out[kk, jj, ii, 2, t] = sg * src[2, j]
            out[kk, jj, ii, 3, t] = sg * src[3, j]
    return out.reshape(-1, 4, len(md))


@pytest.mark.parametrize("n,k", [(2, 2), (3, 1), (3, 2)])
def test_rotation_equivariance(n, k):
    m = cube(n, k)
    w = random_state(m, 11)
    f = O.residual(m, w)
    fr = O.residual(m, rotate_z(w, n, k))
    np.testing.assert_allclose(fr, rotate_z(f, n, k), atol=1e-12 * np.abs(f).max())
    v = S.direction(m.ne, k, 3)
    jv = O.jvp(m, w, v, 0.7)
    jvr = O.jvp(m, rotate_z(w, n, k), rotate_z(v, n, k), 0.7)
    np.testing.assert_allclose(jvr, rotate_z(jv, n, k), atol=1e-12 * np.abs(jv).max())


@pytest.mark.parametrize("n,k", [(2, 1), (2, 2), (3, 1)])
def test_br2_viscous_form_symmetric_psd(n, k):
    # F^nu is linear and self-adjoint, so the BR2 viscous Jacobian is a symmetric,
    # positive semi-definite bilinear form on the velocity (Sec. 2.4.2, Eq. (jacTrilFNURef))
    nu = 0.05
    m = box(n, k, nu)
    w = random_state(m, 2)
    Gv = O.dense_G(m, w, 0.0) - O.dense_G(m.with_nu(0.0), w, 0.0)
    nbk = m.nb
    idx = np.array([i for i in range(m.n) if (i // nbk) % 4 < 3])
    pidx = np.array([i for i in range(m.n) if (i // nbk) % 4 == 3])
    A = Gv[np.ix_(idx, idx)]
    scale = np.abs(A).max()
    assert np.abs(Gv[pidx]).max() < 1e-12 * scale and np.abs(Gv[:, pidx]).max() < 1e-12 * scale
    assert np.abs(A - A.T).max() < 1e-11 * scale
    ev = np.linalg.eigvalsh(0.5 * (A + A.T))
    assert ev.min() > -1e-10 * scale
    # constant velocities are in the kernel; nothing else is small for the penalised form
    assert ev[3] > 1e-6 * scale


def test_tangent_vs_central_fd_on_2cube():
    # on 2^3 each element's -x and +x neighbours are the same element
    for k in (1, 2):
        m = box(2, k)
        w = random_state(m, 7)
        v = S.direction(m.ne, k, 8)
        jv = O.jvp(m, w, v, 0.0)
        h = 1e-6
        fd = (O.residual(m, w + h * v) - O.residual(m, w - h * v)) / (2 * h)
        assert np.abs(jv - fd).max() / np.abs(jv).max() < 1e-7


def test_matrix_free_fd_vs_tangent():
    # Eqs. (matrix-free), (epsdef) with eps = 1e-9 agree with the exact action well above eps
    for k in (1, 2, 3):
        m = box(2, k)
        w = random_state(m, 9)
        v = S.direction(m.ne, k, 10)
        ex = O.jvp(m, w, v, 0.3)
        fd = O.jvp_fd(m, w, v, 0.3, 1e-9)
        assert np.linalg.norm(fd - ex) / np.linalg.norm(ex) < 1e-5


def test_dense_G_is_the_action():
    m = box(2, 1)
    w = random_state(m, 4)
    G = O.dense_G(m, w, 1.7)
    v = S.direction(m.ne, 1, 5)
    np.testing.assert_allclose(G @ v.reshape(-1), O.jvp(m, w, v, 1.7).reshape(-1), atol=1e-13 * np.abs(G).max())
    # the mass form is the identity on velocity modes and zero on pressure
    Gm = O.dense_G(m, w, 0.0)
    d = np.diag(G - Gm)
    var = (np.arange(m.n) // m.nb) % 4
    np.testing.assert_allclose(d, np.where(var < 3, 1.7, 0.0), atol=1e-12)


@pytest.mark.parametrize("k0,kl", [(2, 1), (3, 1), (3, 2)])
def test_inherited_inviscid_equals_non_inherited(k0, kl):
    # Sec. 2.4.2: the inherited (sub-block) and re-discretised inviscid coarse Jacobians coincide
    # when both use the same quadrature and the state lies in the coarse space.
    m0 = box(2, k0, nu=0.0)
    ml = m0.with_k(kl, nq=m0.nq)
    wl = random_state(ml, 3)
    w0 = np.zeros(m0.shape())
    w0[:, :, :ml.nb] = wl
    from oracle.solvers import inherited_operator
    Ginh = inherited_operator(O.dense_G(m0, w0, 0.5), m0.ne, m0.nb, ml.nb)
    Gnon = O.dense_G(ml, wl, 0.5)
    np.testing.assert_allclose(Ginh, Gnon, atol=1e-12 * np.abs(Gnon).max())
    # the viscous parts differ (the inherited lifting lives in P^{k_0})
    m0v, mlv = m0.with_nu(0.05), ml.with_nu(0.05)
    Ginh = inherited_operator(O.dense_G(m0v, w0, 0.5), m0.ne, m0.nb, ml.nb)
    Gnon = O.dense_G(mlv, wl, 0.5)
    assert np.abs(Ginh - Gnon).max() > 1e-6 * np.abs(Gnon).max()


def _hat(nodes_vals, xn, x):
    """Periodic continuous piecewise-linear function with nodal values, and its derivative."""
    L = xn[-1] - xn[0]
    x = np.mod(x - xn[0], L) + xn[0]
    i = np.clip(np.searchsorted(xn, x, side="right") - 1, 0, len(xn) - 2)
    h = xn[i + 1] - xn[i]
    a, b = nodes_vals[i], nodes_vals[(i + 1) % (len(xn) - 1)]
    t = (x - xn[i]) / h
    return a + (b - a) * t, (b - a) / h


def test_inviscid_strong_form_for_continuous_fields():
    # For a continuous field the Riemann flux is the physical flux, so (nu = 0)
    # f_h(w; z) = sum_K int_K div(F^c(w)) z, the element-wise integrated strong form.
    n, k = 3, 2
    m = box(n, k, nu=0.0)
    rng = np.random.default_rng(12)
    gA, gB, gC, gD, gE = (0.4 * rng.standard_normal(n) for _ in range(5))
    gB = 0.4 * rng.standard_normal(n + 1)
    gE = 0.4 * rng.standard_normal(n + 1)

    def fields(X):
        A, dA = _hat(gA, m.xn, X[:, 0])
        B, dB = _hat(gB, m.yn, X[:, 1])
        Cz, dC = _hat(gC, m.zn, X[:, 2])
        D, dD = _hat(gD, m.xn, X[:, 0])
        E, dE = _hat(gE, m.yn, X[:, 1])
        u = np.stack([A + 0.5, B - 0.2, Cz + 0.1], 1)
        p = D + E
        gu = np.zeros((X.shape[0], 3, 3))
        gu[:, 0, 0], gu[:, 1, 1], gu[:, 2, 2] = dA, dB, dC
        gp = np.stack([dD, dE, 0 * dD], 1)
        return u, p, gu, gp

    x, _ = O.quad_points(m)
    vals = np.zeros((m.ne, 4, x.shape[1]))
    for e in range(m.ne):
        # evaluate inside the element (avoid the nodal kinks exactly on faces)
        u, p, _, _ = fields(x[e])
        vals[e, :3] = u.T
        vals[e, 3] = p
    w = O.project_points(m, vals)
    f = O.residual(m, w)
    # reference: element-wise Gauss rule with k+2 points of div F^c times the basis
    g, gw = npleg.leggauss(k + 2)
    xi = np.array(list(itertools.product(g, g, g)))
    wr = np.array([a * b * c for a, b, c in itertools.product(gw, gw, gw)])
    ref = np.zeros_like(f)
    for e in range(m.ne):
        I = [e % m.nx, (e // m.nx) % m.ny, e // (m.nx * m.ny)]
        lo = np.array([m.xn[I[0]], m.yn[I[1]], m.zn[I[2]]])
        h = np.array([m.xn[I[0] + 1] - lo[0], m.yn[I[1] + 1] - lo[1], m.zn[I[2] + 1] - lo[2]])
        X = lo + 0.5 * h * (xi + 1.0)
        u, p, gu, gp = fields(X)
        div = np.einsum("qjj->q", gu)
        mom = np.einsum("qj,qij->qi", u, gu) + u * div[:, None] + gp  # d_j(u_i u_j) + d_i p
        phi, _ = O.basis(m, e, xi)
        W = wr * np.prod(h) / 8.0
        ref[e, :3] = np.einsum("q,qi,qm->im", W, mom, phi)
        ref[e, 3] = np.einsum("q,q,qm->m", W, div, phi)
    np.testing.assert_allclose(f, ref, atol=1e-12 * np.abs(ref).max())


def test_tgv_projection_and_kinetic_energy():
    # mean kinetic energy of the Taylor-Green field is 1/8; the L2 projection approaches it as k grows
    errs = []
    for k in (1, 2, 3, 4):
        m = cube(4, k)
        w = O.project_tgv(m)
        ke = 0.5 * np.sum(w[:, :3, :] ** 2) / (2 * math.pi) ** 3
        errs.append(abs(ke - 0.125))
        assert ke <= 0.125 + 1e-12
    assert all(errs[i + 1] < errs[i] for i in range(3)) and errs[-1] < 1e-4
    # independent projection with numpy's Legendre series and the same Gauss rule
    m = cube(2, 2)
    w = O.project_tgv(m)
    g, gw = npleg.leggauss(3)
    xi = np.array(list(itertools.product(g, g, g)))
    wr = np.array([a * b * c for a, b, c in itertools.product(gw, gw, gw)])
    md = O.modes(2)
    h = math.pi
    for e in range(m.ne):
        I = [e % 2, (e // 2) % 2, e // 4]
        X = np.array(I) * h + 0.5 * h * (xi + 1.0)
        tg = np.stack([np.sin(X[:, 0]) * np.cos(X[:, 1]) * np.cos(X[:, 2]),
                       -np.cos(X[:, 0]) * np.sin(X[:, 1]) * np.cos(X[:, 2]), 0 * X[:, 0],
                       (np.cos(2 * X[:, 0]) + np.cos(2 * X[:, 1])) * (np.cos(2 * X[:, 2]) + 2) / 16], 0)
        phi = np.ones((len(xi), len(md)))
        for j, ab in enumerate(md):
            for d in range(3):
                c = np.zeros(ab[d] + 1)
                c[-1] = 1
                phi[:, j] *= math.sqrt((2 * ab[d] + 1) / 2) * npleg.legval(xi[:, d], c)
        phi /= math.sqrt(h ** 3 / 8)
        ref = np.einsum("q,vq,qm->vm", wr * h ** 3 / 8, tg, phi)
        np.testing.assert_allclose(w[e], ref, atol=1e-14)


def test_results_do_not_depend_on_the_thread_count():
    # the OpenMP loops over elements write disjoint entries in a fixed order: the residual and the
    # exact Jacobian action are bitwise the same on one thread and on all of them
    xn, yn, zn = S.perturbed_nodes(3, seed=2), S.uniform_nodes(4), S.perturbed_nodes(3, seed=5)
    m = O.Mesh(xn, yn, zn, 3, S.NU_TGV, S.AC_C, S.ETA)
    w = O.project_tgv(m) + S.perturbation(m.ne, 3, 0.3, 4)
    v = S.direction(m.ne, 3, 6)
    n0 = O.threads()
    try:
        O.threads(1)
        f1, j1 = O.residual(m, w), O.jvp(m, w, v, 0.7)
        O.threads(max(2, n0))
        f2, j2 = O.residual(m, w), O.jvp(m, w, v, 0.7)
    finally:
        O.threads(n0)
    assert np.array_equal(f1, f2) and np.array_equal(j1, j2)
