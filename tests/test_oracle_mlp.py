"""Pins of the oracle's learned-correction network: its gradient against central differences,
the GELU derivative against its definition, the bfloat16 rounding against exact cases, and the
homogeneity of the feature normalisation."""
import numpy as np
import pytest

from oracle import mlp as M


def _theta(seed):
    rng = np.random.default_rng(seed)
    p = {}
    for name, shp in M.SHAPES:
        fan = shp[1] if len(shp) == 2 else 1
        p[name] = rng.standard_normal(shp) / np.sqrt(fan) * (0.5 if name.startswith("b") else 1.0)
    return M.pack(p)


def test_gelu_derivative():
    t = np.linspace(-4, 4, 41)
    h = 1e-6
    np.testing.assert_allclose(M.gelu_prime(t), (M.gelu(t + h) - M.gelu(t - h)) / (2 * h), atol=1e-9)
    assert abs(M.gelu(np.array([0.0]))[0]) == 0.0 and abs(M.gelu(np.array([10.0]))[0] - 10.0) < 1e-12


def test_gradient_central_differences():
    theta = _theta(1)
    rng = np.random.default_rng(2)
    X = rng.standard_normal((6, M.N_IN))
    T = rng.standard_normal((6, M.N_OUT))
    loss, g = M.loss_and_grad(theta, X, T)
    idx = rng.choice(theta.size, 60, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(theta)
        e[i] = h
        fd = (M.loss_and_grad(theta + e, X, T)[0] - M.loss_and_grad(theta - e, X, T)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_bf16_rounding():
    vals = np.array([1.0, 1.0 + 2.0 ** -7, 1.0 + 2.0 ** -9, 1.0 + 3 * 2.0 ** -9, -2.5, 1e-3])
    r = M.bf16_round(vals)
    assert r[0] == 1.0 and r[1] == 1.0 + 2.0 ** -7
    assert r[2] == 1.0                      # tie -> even mantissa
    assert r[3] == 1.0 + 2.0 ** -7          # above half -> up
    assert r[4] == -2.5
    assert abs(r[5] - 1e-3) / 1e-3 < 2.0 ** -8


def test_feature_normalisation_is_homogeneous():
    rng = np.random.default_rng(3)
    ne, nb1 = 8, 4
    nbr = rng.integers(0, ne, (ne, 6))
    d = rng.standard_normal((ne, 4, nb1))
    X1, s1 = M.features(d, nbr, nb1)
    X2, s2 = M.features(3.0 * d, nbr, nb1)
    np.testing.assert_allclose(X1, X2, atol=1e-15)
    np.testing.assert_allclose(s2, 3.0 * s1, rtol=1e-15)
    np.testing.assert_allclose(np.linalg.norm(X1, axis=1), 1.0, atol=1e-15)


def test_coarse_correction_structure():
    # the features of element e are its own P1 block followed by its face neighbours'
    # blocks in the order -x, +x, -y, +y, -z, +z; the map is positively homogeneous
    import oracle as O
    import synthetic as S
    n = 3
    m = O.Mesh(S.uniform_nodes(n), S.uniform_nodes(n), S.uniform_nodes(n), 1, S.NU_TGV, S.AC_C, S.ETA)
    nbr = m.neighbours()
    rng = np.random.default_rng(4)
    d = rng.standard_normal((m.ne, 4, 4))
    X, s = M.features(d, nbr, 4)
    e = 13  # the centre cell (1, 1, 1)
    i, j, k = 1, 1, 1
    cells = [(i, j, k), (i - 1, j, k), (i + 1, j, k), (i, j - 1, k), (i, j + 1, k), (i, j, k - 1), (i, j, k + 1)]
    F = np.concatenate([d[a + n * (b + n * c)].reshape(-1) for a, b, c in cells])
    np.testing.assert_allclose(X[e] * s[e], F, rtol=1e-15, atol=0)
    theta = _theta(5)
    x1 = M.coarse_correction(theta, d, nbr, 4)
    x2 = M.coarse_correction(theta, 2.5 * d, nbr, 4)
    np.testing.assert_allclose(x2, 2.5 * x1, rtol=1e-12, atol=1e-14)
    z = d.copy()
    z[:] = 0.0
    assert np.all(M.coarse_correction(theta, z, nbr, 4) == 0.0)


def test_bf16_forward_close_to_fp64():
    theta = _theta(6)
    X = np.random.default_rng(7).standard_normal((32, M.N_IN)) / np.sqrt(M.N_IN)
    y64 = M.forward(theta, X)[0]
    y16 = M.forward_bf16(theta, X)
    rel = np.linalg.norm(y16 - y64) / np.linalg.norm(y64)
    assert 1e-5 < rel < 3e-2
