"""Pins of the oracle's no-slip walls (Sec. 2.1: Dirichlet viscous flux with the one-sided
lifting, inviscid flux against the ghost boundary state (2f - u_K, p_K); the reading of the
ghost state and of the boundary lifting is c8).

Each check rests on the mathematics, not on the oracle's formulas:
* plane Poiseuille flow u = U(1 - y^2) e_x with constant pressure lies in the discrete space for
  k >= 2 and vanishes on the walls, so a consistent discretisation returns exactly the strong
  form, f_h = (-nu Laplacian u, 0, 0, 0) projected = 2 nu U on the u modes, on a stretched mesh;
* a fluid at rest under a constant pressure has zero residual;
* the channel is symmetric under y -> -y (v -> -v), so the residual and its Jacobian action
  commute with that mirror: this ties the lower wall to the upper one;
* the BR2 viscous form stays symmetric, and the walls make it positive definite on the
  velocity (no constant velocity is in the kernel any more);
* the exact Jacobian action equals central finite differences of the residual;
* the ghost state makes the interface velocity the wall's, so no mass crosses a wall: the
  continuity residuals of any state sum to zero, and the constant pressure is a left as well as
  a right null vector of G (the stage systems of a closed channel are consistent).
"""
import numpy as np
import pytest

import oracle as O
import synthetic as S


def channel(nx, ny, nz, k, nu=0.02):
    return O.Mesh(S.uniform_nodes(nx), S.tanh_nodes(ny, 1.15), S.uniform_nodes(nz, np.pi), k, nu, S.AC_C, S.ETA,
                  walls=True)


def project(m, fn):
    x, _ = O.quad_points(m)
    vals = np.stack(fn(x[..., 0], x[..., 1], x[..., 2]), axis=1)  # [ne][4][npt]
    return O.project_points(m, vals)


@pytest.mark.parametrize("k", [2, 3])
def test_poiseuille_residual_is_the_strong_form(k):
    nu, U, p0 = 0.05, 0.8, 0.3
    m = channel(2, 4, 2, k, nu)
    w = project(m, lambda x, y, z: (U * (1 - y * y), 0 * y, 0 * y, p0 + 0 * y))
    f = O.residual(m, w)
    expect = project(m, lambda x, y, z: (2 * nu * U + 0 * y, 0 * y, 0 * y, 0 * y))
    np.testing.assert_allclose(f, expect, atol=1e-12 * np.abs(expect).max())


def test_rest_under_constant_pressure():
    m = channel(2, 3, 2, 2)
    w = project(m, lambda x, y, z: (0 * y, 0 * y, 0 * y, 0.7 + 0 * y))
    assert np.abs(O.residual(m, w)).max() < 1e-13


def mirror_y(a, m):
    """y -> -y on a mesh with symmetric y nodes: element row j -> ny-1-j, mode sign (-1)^(y exponent),
    v -> -v."""
    a = np.asarray(a).reshape(m.nz, m.ny, m.nx, 4, m.nb)
    sgn = (-1.0) ** O.modes(m.k)[:, 1]
    out = a[:, ::-1] * sgn[None, None, None, None, :]
    out = out.copy()
    out[:, :, :, 1] *= -1.0
    return out.reshape(m.shape())


@pytest.mark.parametrize("k", [1, 2])
def test_mirror_equivariance(k):
    m = channel(2, 4, 3, k)
    w = O.project_tgv(m) + S.perturbation(m.ne, k, 0.3, 4)
    f = O.residual(m, w)
    np.testing.assert_allclose(O.residual(m, mirror_y(w, m)), mirror_y(f, m), atol=1e-12 * np.abs(f).max())
    v = S.direction(m.ne, k, 5)
    jv = O.jvp(m, w, v, 0.9)
    np.testing.assert_allclose(O.jvp(m, mirror_y(w, m), mirror_y(v, m), 0.9), mirror_y(jv, m),
                               atol=1e-12 * np.abs(jv).max())


@pytest.mark.parametrize("k", [1, 2])
def test_br2_wall_form_symmetric_positive_definite(k):
    nu = 0.05
    m = channel(2, 3, 2, k, nu)
    w = O.project_tgv(m) + S.perturbation(m.ne, k, 0.3, 6)
    Gv = O.dense_G(m, w, 0.0) - O.dense_G(m.with_nu(0.0), w, 0.0)
    idx = np.array([i for i in range(m.n) if (i // m.nb) % 4 < 3])
    A = Gv[np.ix_(idx, idx)]
    scale = np.abs(A).max()
    assert np.abs(A - A.T).max() < 1e-11 * scale
    ev = np.linalg.eigvalsh(0.5 * (A + A.T))
    assert ev.min() > 1e-6 * scale


def test_tangent_vs_central_fd_with_walls():
    for k in (1, 2):
        m = channel(2, 3, 2, k)
        w = O.project_tgv(m) + S.perturbation(m.ne, k, 0.3, 7)
        v = S.direction(m.ne, k, 8)
        jv = O.jvp(m, w, v, 0.0)
        h = 1e-6
        fd = (O.residual(m, w + h * v) - O.residual(m, w - h * v)) / (2 * h)
        assert np.abs(jv - fd).max() / np.abs(jv).max() < 1e-7


def test_wall_neighbours():
    m = channel(3, 4, 2, 1)
    nbr = m.neighbours()
    j = (np.arange(m.ne) // m.nx) % m.ny
    assert (nbr[j == 0, 2] == -1).all() and (nbr[j == m.ny - 1, 3] == -1).all()
    assert (nbr[(j > 0), 2] >= 0).all() and (nbr[(j < m.ny - 1), 3] >= 0).all()


def test_tanh_nodes():
    y = S.tanh_nodes(12, 1.15)
    h = np.diff(y)
    assert abs(y[0] + 1) < 1e-15 and abs(y[-1] - 1) < 1e-15
    assert abs(h[1] / h[0] - 1.15) < 1e-9 and abs(h[-2] / h[-1] - 1.15) < 1e-9
    np.testing.assert_allclose(y, -y[::-1], atol=1e-15)


def test_no_mass_crosses_a_wall():
    m = channel(2, 3, 2, 2)
    w = O.project_tgv(m) + S.perturbation(m.ne, 2, 0.3, 9)
    f = O.residual(m, w).reshape(m.ne, 4, m.nb)
    vol = m.vol()
    # test function q = 1 on the pressure: mode 0 of every element, phi_0 = 1 / sqrt(|K|)
    total = np.sum(f[:, 3, 0] * np.sqrt(vol))
    assert abs(total) < 1e-13 * np.abs(f).max()
    G = O.dense_G(m, w, 1.3)
    z = np.zeros(m.shape())
    z[:, 3, 0] = np.sqrt(vol)
    z = z.reshape(-1)
    assert np.abs(G @ z).max() < 1e-12 * np.abs(G).max()
    assert np.abs(z @ G).max() < 1e-12 * np.abs(G).max()
