"""Pins of the oracle's basis and quadrature (Sec. 2.1 broken P^k space, Sec. 2.4 hierarchical orthonormal basis)."""
import itertools
import json
import math
import os

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

import oracle as O
import synthetic as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7])
def test_gauss_matches_numpy(n):
    x, w = O.gauss(n)
    xr, wr = npleg.leggauss(n)
    np.testing.assert_allclose(x, xr, atol=1e-15)
    np.testing.assert_allclose(w, wr, atol=1e-15)


@pytest.mark.parametrize("n", [0, 1, 2, 3, 4, 5, 6])
def test_legendre_matches_numpy(n):
    import ctypes
    for x in np.linspace(-1, 1, 11):
        v = ctypes.c_double()
        d = ctypes.c_double()
        O.lib().orc_legendre(n, float(x), ctypes.byref(v), ctypes.byref(d))
        c = np.zeros(n + 1)
        c[n] = 1.0
        assert abs(v.value - npleg.legval(x, c)) < 1e-14
        assert abs(d.value - npleg.legval(x, npleg.legder(c))) < 1e-13


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6])
def test_mode_count_is_total_degree(k):
    # dim P^k in 3D = C(k+3, 3): 4, 10, 20, 35, 56, 84
    assert O.nb(k) == math.comb(k + 3, 3) == S.nb(k)
    md = O.modes(k)
    assert len({tuple(r) for r in md}) == len(md)
    deg = md.sum(axis=1)
    assert (np.diff(deg) >= 0).all() and deg.max() == k
    np.testing.assert_array_equal(deg, S.mode_degrees(k))


def test_paper_nonzero_ratios():
    # Sec. 2.5: G_2 and G_1 have 440 and 70 times fewer non-zeros than G_0 for k = 6, 2, 1
    g = json.load(open(os.path.join(GOLDEN, "paper_counts.json")))
    k0, k1, k2 = g["k_levels"]           # levels l = 0, 1, 2
    r2 = (O.nb(k0) / O.nb(k2)) ** 2      # (84/4)^2 = 441
    r1 = (O.nb(k0) / O.nb(k1)) ** 2      # (84/10)^2 = 70.56
    assert round(r2) in (g["nnz_ratio_G0_over_G2"], g["nnz_ratio_G0_over_G2"] + 1)
    assert int(r1) == g["nnz_ratio_G0_over_G1"]
    # EWBJ keeps 1 of the 2d+1 blocks of a block row in 3D
    assert abs(1.0 / 7.0 - g["ewbj_block_fraction_3d"]) < 1e-15


def _mesh(n=2, k=2, nodes=None, nu=0.01):
    xn = S.uniform_nodes(n) if nodes is None else nodes
    return O.Mesh(xn, S.perturbed_nodes(n, seed=3), S.uniform_nodes(n), k, nu)


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_mass_matrix_is_identity(k):
    m = _mesh(3, k, nodes=S.perturbed_nodes(3, seed=7))
    x, wq = O.quad_points(m)
    gx, _ = O.gauss(m.nq)
    xi = np.array(list(itertools.product(gx, gx, gx)))
    for e in (0, 5, m.ne - 1):
        phi, _ = O.basis(m, e, xi)
        M = phi.T @ (wq[e][:, None] * phi)
        assert np.abs(M - np.eye(m.nb)).max() < 1e-13


def _numpy_basis(k, xi, h):
    """Independent evaluation of the orthonormal box basis with numpy's Legendre series."""
    md = O.modes(k)
    vol = np.prod(h)
    out = np.zeros((xi.shape[0], len(md)))
    for j, (a, b, c) in enumerate(md):
        val = np.ones(xi.shape[0])
        for d, n in enumerate((a, b, c)):
            cc = np.zeros(n + 1)
            cc[n] = 1.0
            val *= math.sqrt((2 * n + 1) / 2.0) * npleg.legval(xi[:, d], cc)
        out[:, j] = val / math.sqrt(vol / 8.0)
    return out


@pytest.mark.parametrize("k", [1, 3])
def test_basis_matches_independent_evaluation(k):
    m = _mesh(2, k)
    rng = np.random.default_rng(0)
    xi = rng.uniform(-1, 1, (20, 3))
    for e in range(m.ne):
        phi, dphi = O.basis(m, e, xi)
        I = [e % m.nx, (e // m.nx) % m.ny, e // (m.nx * m.ny)]
        h = np.array([np.diff(m.xn)[I[0]], np.diff(m.yn)[I[1]], np.diff(m.zn)[I[2]]])
        np.testing.assert_allclose(phi, _numpy_basis(k, xi, h), atol=1e-13)
        # gradient by central differences in reference coordinates
        for d in range(3):
            dx = np.zeros(3)
            dx[d] = 1e-6
            fd = (_numpy_basis(k, xi + dx, h) - _numpy_basis(k, xi - dx, h)) / 2e-6 * (2.0 / h[d])
            np.testing.assert_allclose(dphi[:, :, d], fd, atol=1e-7 * max(1.0, np.abs(fd).max()))


@pytest.mark.parametrize("k", [2, 3])
def test_polynomials_reproduced_and_hierarchy(k):
    # Any polynomial of total degree <= k is reproduced exactly by the L2 projection,
    # and truncating a P^k field to P^k' equals its L2 projection onto P^k'.
    m = _mesh(2, k)
    x, wq = O.quad_points(m)
    rng = np.random.default_rng(1)
    coeffs = {(a, b, c): rng.standard_normal() for a in range(k + 1) for b in range(k + 1) for c in range(k + 1)
              if a + b + c <= k}
    poly = lambda X: sum(v * X[..., 0] ** a * X[..., 1] ** b * X[..., 2] ** c for (a, b, c), v in coeffs.items())
    vals = np.zeros((m.ne, 4, x.shape[1]))
    for v in range(4):
        vals[:, v] = poly(x) * (v + 1)
    w = O.project_points(m, vals)
    gx, _ = O.gauss(m.nq)
    xi = np.array(list(itertools.product(gx, gx, gx)))
    for e in range(m.ne):
        got = O.eval_field(m, w, e, xi)
        for v in range(4):
            np.testing.assert_allclose(got[:, v], vals[e, v], rtol=1e-10, atol=1e-9)
    # hierarchy: projection onto P^{k-1} with the fine rule == truncation
    kc = k - 1
    nbc = O.nb(kc)
    mc = m.with_k(kc, nq=m.nq)
    wf = rng.standard_normal(m.shape())
    for e in range(m.ne):
        phif, _ = O.basis(m, e, xi)
        phic, _ = O.basis(mc, e, xi)
        for v in range(4):
            fvals = phif @ wf[e, v]
            proj = phic.T @ (wq[e] * fvals)
            np.testing.assert_allclose(proj, wf[e, v, :nbc], atol=1e-12)
