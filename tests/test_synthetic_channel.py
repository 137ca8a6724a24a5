"""Input recipes (input generation only; the discretisation never reads them):
* the channel workload: tanh nodes and an initial field that is the laminar profile plus a
  perturbation that is divergence-free, vanishes on the walls and has the stated amplitude;
* the held-out flow states of the learned correction: a seeded smooth perturbation of the
  periodic box, divergence-free, periodic and of the stated amplitude."""
import numpy as np

import synthetic as S


def field(x, y, z):
    return np.array(S.channel_field(x, y, z)[:3])


def test_perturbation_is_solenoidal_and_vanishes_on_the_walls():
    rng = np.random.default_rng(0)
    x, y, z = rng.uniform(0, 2 * np.pi, 50), rng.uniform(-0.99, 0.99, 50), rng.uniform(0, np.pi, 50)
    h = 1e-5
    div = ((field(x + h, y, z)[0] - field(x - h, y, z)[0]) + (field(x, y + h, z)[1] - field(x, y - h, z)[1])
           + (field(x, y, z + h)[2] - field(x, y, z - h)[2])) / (2 * h)
    assert np.abs(div).max() < 1e-8
    for yw in (-1.0, 1.0):
        assert np.abs(field(x, np.full(50, yw), z)).max() < 1e-14


def test_perturbation_amplitude_and_periodicity():
    gx = np.linspace(0.0, 2 * np.pi, 33)[:-1]
    gy = np.linspace(-1.0, 1.0, 33)
    gz = np.linspace(0.0, np.pi, 17)[:-1]
    X, Y, Z = np.meshgrid(gx, gy, gz, indexing="ij")
    u = field(X, Y, Z)
    u[0] -= 1.0 - Y * Y
    rms = np.sqrt(np.mean(np.sum(u * u, axis=0)))
    assert 0.04 < rms < 0.06
    rng = np.random.default_rng(1)
    x, y, z = rng.uniform(0, 2 * np.pi, 10), rng.uniform(-1, 1, 10), rng.uniform(0, np.pi, 10)
    np.testing.assert_allclose(field(x + 2 * np.pi, y, z), field(x, y, z), atol=1e-12)
    np.testing.assert_allclose(field(x, y, z + np.pi), field(x, y, z), atol=1e-12)


def test_channel_viscosity():
    nu = S.channel_nu(180.0)
    u_tau = np.sqrt(nu * 2.0)  # wall shear of 1 - y^2
    assert abs(u_tau / nu - 180.0) < 1e-9


def test_box_noise_is_solenoidal_periodic_and_has_the_stated_amplitude():
    # the held-out flow states of the learned correction: divergence-free, periodic on the box,
    # rms 0.05 over a uniform sampling, different for different seeds
    def f(x, y, z, seed=11):
        return np.array(S.box_noise_field(x, y, z, seed)[:3])

    rng = np.random.default_rng(2)
    x, y, z = (rng.uniform(0, 2 * np.pi, 40) for _ in range(3))
    h = 1e-5
    div = ((f(x + h, y, z)[0] - f(x - h, y, z)[0]) + (f(x, y + h, z)[1] - f(x, y - h, z)[1])
           + (f(x, y, z + h)[2] - f(x, y, z - h)[2])) / (2 * h)
    assert np.abs(div).max() < 1e-8
    for sh in ((2 * np.pi, 0, 0), (0, 2 * np.pi, 0), (0, 0, 2 * np.pi)):
        np.testing.assert_allclose(f(x + sh[0], y + sh[1], z + sh[2]), f(x, y, z), atol=1e-12)
    g = np.linspace(0.0, 2 * np.pi, 25)[:-1]
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    u = f(X, Y, Z)
    assert 0.045 < np.sqrt(np.mean(np.sum(u * u, axis=0))) < 0.055
    assert np.abs(f(x, y, z, 12) - f(x, y, z, 11)).max() > 1e-3
    assert np.all(np.asarray(S.box_noise_field(x, y, z, 11)[3]) == 0.0)
