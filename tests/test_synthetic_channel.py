"""The channel workload's input recipe: tanh nodes and an initial field that is the laminar
profile plus a perturbation that is divergence-free, vanishes on the walls and has the stated
amplitude. (The recipe is input generation; the discretisation never reads it.)"""
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
