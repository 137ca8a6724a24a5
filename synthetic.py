"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module holds no arithmetic of the method: it only produces meshes (node
coordinates), random coefficient vectors and random face states from seeds,
with the shapes and value ranges of the workloads. The Taylor-Green field and
every operator are computed separately by each implementation.

Workloads (they stand in for the paper's cylinder / sphere / T3L1 / landing-gear
meshes, which are not available): Taylor-Green vortex at Re = 1600 on the
triply periodic cube [0, 2 pi]^3 with uniform hexahedra, modal P^k, k <= 4.
"""
import math

import numpy as np

TWO_PI = 2.0 * math.pi
RE_TGV = 1600.0
NU_TGV = 1.0 / RE_TGV
AC_C = 1.0        # artificial-compressibility constant
ETA = 7.0         # BR2 penalty, greater than the 6 faces of a hexahedron
SEED_V = 1809     # Jacobian-action direction


def nb(k):
    """Number of modes of the total-degree-k space in 3D, C(k+3, 3)."""
    return (k + 1) * (k + 2) * (k + 3) // 6


def mode_degrees(k):
    """Total degree of every mode in the hierarchical ordering (degree 0, then 1, ...)."""
    out = []
    for t in range(k + 1):
        out += [t] * ((t + 1) * (t + 2) // 2)
    return np.array(out)


def uniform_nodes(n, length=TWO_PI):
    return np.linspace(0.0, length, n + 1)


def perturbed_nodes(n, length=TWO_PI, amp=0.25, seed=0):
    """Node coordinates with each cell size scaled by a seeded factor in [1-amp, 1+amp]."""
    rng = np.random.default_rng(seed)
    h = 1.0 + amp * (2.0 * rng.random(n) - 1.0)
    h *= length / h.sum()
    return np.concatenate([[0.0], np.cumsum(h)])


def direction(ne, k, seed=SEED_V):
    """Seeded Jacobian-action direction: N(0,1) modal coefficients scaled by 1/(1+degree)."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((ne, 4, nb(k)))
    return v / (1.0 + mode_degrees(k))[None, None, :]


def perturbation(ne, k, amp, seed):
    """Seeded state perturbation amp * N(0,1)/(1+degree) on every coefficient."""
    return amp * direction(ne, k, seed)


def face_states(n, seed, umax=0.9, pmax=1.0):
    """Random left/right states (u[3], p) for Riemann-solver tests."""
    rng = np.random.default_rng(seed)
    uL = rng.uniform(-umax, umax, (n, 3))
    uR = rng.uniform(-umax, umax, (n, 3))
    pL = rng.uniform(-pmax, pmax, n)
    pR = rng.uniform(-pmax, pmax, n)
    return uL, pL, uR, pR


# Benchmark / parity workloads: name -> (cells per axis, fine degree, p-levels)
CONFIGS = {
    "tgv4_p2": dict(n=4, k=2, levels=(2, 1)),
    "tgv16_p4": dict(n=16, k=4, levels=(4, 2, 1)),
    "tgv32_p4": dict(n=32, k=4, levels=(4, 2, 1)),
    "tgv24_p4": dict(n=24, k=4, levels=(4, 2, 1)),
}


def acoustic_dt(n, k, cfl=50.0, c=AC_C, umax=1.0, length=TWO_PI):
    """Time step for an acoustic CFL: cfl * h / ((2k+1) * (|u| + sqrt(|u|^2 + c^2)))."""
    h = length / n
    return cfl * h / ((2 * k + 1) * (umax + math.sqrt(umax * umax + c * c)))


# Batch of independent periodic Taylor-Green boxes of uneven size and degree: n^3 cells with
# n drawn uniformly from 4..12, k uniformly from {2, 3, 4}; p-levels per degree.
BATCH_LEVELS = {2: (2, 1), 3: (3, 2, 1), 4: (4, 2, 1)}


def batch_boxes(count=64, seed=64, n_min=4, n_max=12, degrees=(2, 3, 4)):
    """List of (n, k) for the batch workload (seeded)."""
    rng = np.random.default_rng(seed)
    ns = rng.integers(n_min, n_max + 1, size=count)
    ks = rng.choice(np.asarray(degrees), size=count)
    return [(int(n), int(k)) for n, k in zip(ns, ks)]


# Channel of the batching configuration: box 2pi x 2 x pi, walls at y = -1 and y = 1, tanh
# wall-normal stretching whose second cell is 1.15 times the first; laminar parabolic profile
# plus 5% seeded noise.
CHANNEL = dict(nx=24, ny=12, nz=12, k=3, levels=(3, 2, 1), lx=TWO_PI, ly=2.0, lz=math.pi, ratio=1.15,
               re_tau=180.0)


def tanh_nodes(n, ratio, lo=-1.0, hi=1.0):
    """n+1 nodes on [lo, hi], y = tanh(g s)/tanh(g) on s uniform in [-1, 1], with g chosen so
    that the second cell from either wall is `ratio` times the first."""
    s = np.linspace(-1.0, 1.0, n + 1)

    def growth(g):
        y = np.tanh(g * s) / np.tanh(g)
        h = np.diff(y)
        return h[1] / h[0]

    a, b = 1e-6, 10.0
    if growth(b) < ratio:
        b = 50.0
    for _ in range(200):
        mid = 0.5 * (a + b)
        if growth(mid) < ratio:
            a = mid
        else:
            b = mid
    y = np.tanh(0.5 * (a + b) * s) / np.tanh(0.5 * (a + b))
    return lo + (hi - lo) * 0.5 * (y + 1.0)


def channel_nodes(cfg=None):
    c = CHANNEL if cfg is None else cfg
    return (uniform_nodes(c["nx"], c["lx"]), tanh_nodes(c["ny"], c["ratio"], -0.5 * c["ly"], 0.5 * c["ly"]),
            uniform_nodes(c["nz"], c["lz"]))


def channel_noise_modes(seed, modes=8):
    """Seeded modes of the vector potential of the channel's perturbation: per component of psi
    and per mode, (kx, kz, ky, phase_xz, phase_y, amplitude); kx, kz integer multiples of the
    box's wavenumbers 2pi/lx = 1 and 2pi/lz = 2."""
    rng = np.random.default_rng(seed)
    out = np.zeros((3, modes, 6))
    out[..., 0] = rng.integers(1, 4, size=(3, modes))
    out[..., 1] = 2.0 * rng.integers(1, 3, size=(3, modes))
    out[..., 2] = rng.uniform(0.5, 3.0, size=(3, modes))
    out[..., 3] = rng.uniform(0.0, TWO_PI, size=(3, modes))
    out[..., 4] = rng.uniform(0.0, TWO_PI, size=(3, modes))
    out[..., 5] = rng.standard_normal((3, modes))
    return out


def channel_field(x, y, z, seed=180, amp=0.05, modes=8):
    """Channel initial field at points (arrays of equal shape): the laminar profile
    u = 1 - y^2 (walls at y = -1, 1) plus amp times a unit-rms divergence-free perturbation,
    the curl of psi = (1 - y^2)^2 sum_m a cos(kx x + kz z + t1) cos(ky y + t2), which vanishes
    with its first derivatives on the walls. Returns (u, v, w, p)."""
    md = channel_noise_modes(seed, modes)
    up = _channel_curl(md, x, y, z)
    # unit rms over a fixed sampling of the box, independent of the points asked for
    gx = np.linspace(0.0, TWO_PI, 17)[:-1]
    gy = np.linspace(-1.0, 1.0, 17)
    gz = np.linspace(0.0, math.pi, 9)[:-1]
    X, Y, Z = np.meshgrid(gx, gy, gz, indexing="ij")
    rms = math.sqrt(np.mean(np.sum(_channel_curl(md, X, Y, Z) ** 2, axis=0)))
    up = up * (amp / rms)
    return 1.0 - y * y + up[0], up[1], up[2], 0.0 * y


def _channel_curl(md, x, y, z):
    g = (1.0 - y * y) ** 2
    dg = -4.0 * y * (1.0 - y * y)
    d = np.zeros((3, 3) + np.shape(x))
    for i in range(3):
        for kx, kz, ky, t1, t2, a in md[i]:
            A = kx * x + kz * z + t1
            B = ky * y + t2
            ca, sa, cb, sb = np.cos(A), np.sin(A), np.cos(B), np.sin(B)
            d[i, 0] += -a * kx * sa * cb * g
            d[i, 1] += a * ca * (cb * dg - ky * sb * g)
            d[i, 2] += -a * kz * sa * cb * g
    return np.stack([d[2, 1] - d[1, 2], d[0, 2] - d[2, 0], d[1, 0] - d[0, 1]])


def box_noise_field(x, y, z, seed, amp=0.05, modes=8):
    """Seeded smooth perturbation of the periodic box [0, 2 pi]^3 at points (arrays of equal
    shape): amp times a unit-rms divergence-free velocity, the curl of a vector potential with
    `modes` seeded Fourier modes per component (integer wavenumbers 1..3 per axis, seeded
    phases and amplitudes); zero pressure. Returns (u, v, w, p)."""
    rng = np.random.default_rng(seed)
    kk = rng.integers(1, 4, size=(3, modes, 3)).astype(float)
    ph = rng.uniform(0.0, TWO_PI, size=(3, modes))
    aa = rng.standard_normal((3, modes))

    def curl(X, Y, Z):
        d = np.zeros((3, 3) + np.shape(X))  # d[i, j] = d psi_i / d x_j
        for i in range(3):
            for m in range(modes):
                kx, ky, kz = kk[i, m]
                sn = np.sin(kx * X + ky * Y + kz * Z + ph[i, m]) * aa[i, m]
                d[i, 0] += kx * sn
                d[i, 1] += ky * sn
                d[i, 2] += kz * sn
        return np.stack([d[2, 1] - d[1, 2], d[0, 2] - d[2, 0], d[1, 0] - d[0, 1]])

    g = np.linspace(0.0, TWO_PI, 17)[:-1]
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    rms = math.sqrt(np.mean(np.sum(curl(X, Y, Z) ** 2, axis=0)))
    up = curl(x, y, z) * (amp / rms)
    return up[0], up[1], up[2], 0.0 * np.asarray(x)


def channel_nu(re_tau=180.0, u_center=1.0):
    """Viscosity for which the laminar profile u_c (1 - y^2) has friction Reynolds number re_tau
    (half-height 1): u_tau^2 = nu |du/dy|_wall = 2 nu u_c, re_tau = u_tau / nu."""
    return 2.0 * u_center / (re_tau * re_tau)
