"""Plain FP64 CPU oracle for the DG incompressible-flow operator of arXiv 1809.00866.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package. It shares
no code with the CUDA path (``paper_1809_00866_gb300``) and imports nothing from
it; the product fails loudly when its CUDA library is missing instead of
falling back here.

The discretisation (basis, quadrature, residual, exact Jacobian action,
finite-difference action, Taylor-Green projection) lives in ``dg_oracle.cpp``
and is loaded through ctypes; the solver algorithms (restriction/prolongation,
inherited coarse operators, block-Jacobi smoothing, V-cycle, FGMRES) are plain
numpy in ``oracle.solvers``.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dg_oracle.cpp")
_LIB = os.path.join(_HERE, "_build", "liborc.so")
_lock = threading.Lock()
_lib = None


def build(force=False):
    """Compile the C++ oracle into oracle/_build/liborc.so (g++, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp.%d" % os.getpid()
    cmd = ["g++", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c++17", "-o", tmp, _SRC]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


class _Mesh(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("k", ctypes.c_int),
                ("nq", ctypes.c_int), ("nu", ctypes.c_double), ("c", ctypes.c_double), ("eta", ctypes.c_double),
                ("xn", ctypes.POINTER(ctypes.c_double)), ("yn", ctypes.POINTER(ctypes.c_double)),
                ("zn", ctypes.POINTER(ctypes.c_double)), ("wall_y", ctypes.c_int)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            P = ctypes.POINTER(ctypes.c_double)
            M = ctypes.POINTER(_Mesh)
            L.orc_nb.restype = ctypes.c_int
            L.orc_threads.restype = ctypes.c_int
            L.orc_threads.argtypes = [ctypes.c_int]
            L.orc_p_wave1.restype = ctypes.c_double
            L.orc_p_wave3.restype = ctypes.c_double
            L.orc_tang1.restype = ctypes.c_double
            L.orc_tang3.restype = ctypes.c_double
            for name in ("orc_p_wave1", "orc_p_wave3"):
                getattr(L, name).argtypes = [ctypes.c_double] * 4
            for name in ("orc_tang1", "orc_tang3"):
                getattr(L, name).argtypes = [ctypes.c_double] * 3
            L.orc_residual.argtypes = [M, P, P]
            L.orc_jvp.argtypes = [M, P, P, ctypes.c_double, P]
            L.orc_jvp_fd.argtypes = [M, P, P, ctypes.c_double, ctypes.c_double, P]
            L.orc_dense_G.argtypes = [M, P, ctypes.c_double, P]
            L.orc_project_tgv.argtypes = [M, P]
            L.orc_quad_points.argtypes = [M, P, P]
            L.orc_project_points.argtypes = [M, P, P]
            L.orc_basis.argtypes = [M, ctypes.c_int, ctypes.c_int, P, P, P]
            L.orc_eval_field.argtypes = [M, P, ctypes.c_int, ctypes.c_int, P, P]
            L.orc_riemann.argtypes = [P, ctypes.c_double, P, ctypes.c_double, ctypes.c_int, ctypes.c_double, P, P, P]
            L.orc_riemann_tangent.argtypes = [P, ctypes.c_double, P, ctypes.c_double, P, ctypes.c_double, P,
                                              ctypes.c_double, ctypes.c_int, ctypes.c_double, P]
            L.orc_gauss.argtypes = [ctypes.c_int, P, P]
            L.orc_legendre.argtypes = [ctypes.c_int, ctypes.c_double, P, P]
            L.orc_modes.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
            _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def nb(k):
    """Number of modes of P^k in 3D, C(k+3, 3)."""
    return lib().orc_nb(k)


def threads(n=0):
    """Threads of the oracle's OpenMP loops over elements (n > 0 sets them); returns the count in
    use. Results do not depend on it."""
    return int(lib().orc_threads(int(n)))


def modes(k):
    n = nb(k)
    out = np.zeros((n, 3), dtype=np.int32)
    lib().orc_modes(k, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return out


def gauss(n):
    x = np.zeros(n)
    w = np.zeros(n)
    lib().orc_gauss(n, _p(x), _p(w))
    return x, w


class Mesh:
    """Box mesh of nx*ny*nz hexahedra with node coordinates per axis, periodic in every
    direction, or with no-slip walls at y = yn[0] and y = yn[-1] (``walls=True``).

    Elements are numbered e = i + nx*(j + ny*k); unknowns are laid out
    [element][u, v, w, p][mode].
    """

    def __init__(self, xn, yn, zn, k, nu, c=1.0, eta=7.0, nq=0, walls=False):
        self.xn = np.ascontiguousarray(xn, dtype=np.float64)
        self.yn = np.ascontiguousarray(yn, dtype=np.float64)
        self.zn = np.ascontiguousarray(zn, dtype=np.float64)
        self.nx, self.ny, self.nz = len(self.xn) - 1, len(self.yn) - 1, len(self.zn) - 1
        self.k, self.nu, self.c, self.eta = int(k), float(nu), float(c), float(eta)
        self.nq = int(nq) if nq else self.k + 1
        self.walls = bool(walls)
        self.ne = self.nx * self.ny * self.nz
        self.nb = nb(self.k)
        self.n = self.ne * 4 * self.nb

    def with_k(self, k, nq=0):
        return Mesh(self.xn, self.yn, self.zn, k, self.nu, self.c, self.eta, nq, self.walls)

    def with_nu(self, nu):
        return Mesh(self.xn, self.yn, self.zn, self.k, nu, self.c, self.eta, self.nq, self.walls)

    def vol(self):
        hx, hy, hz = np.diff(self.xn), np.diff(self.yn), np.diff(self.zn)
        return (hx[None, None, :] * hy[None, :, None] * hz[:, None, None]).reshape(-1)

    def neighbours(self):
        """Face neighbours of every element in the order -x, +x, -y, +y, -z, +z."""
        e = np.arange(self.ne)
        i, j, k = e % self.nx, (e // self.nx) % self.ny, e // (self.nx * self.ny)
        idx = lambda a, b, c: (a % self.nx) + self.nx * ((b % self.ny) + self.ny * (c % self.nz))
        nbr = np.stack([idx(i - 1, j, k), idx(i + 1, j, k), idx(i, j - 1, k), idx(i, j + 1, k),
                        idx(i, j, k - 1), idx(i, j, k + 1)], axis=1)
        if self.walls:  # no neighbour across a wall
            nbr[j == 0, 2] = -1
            nbr[j == self.ny - 1, 3] = -1
        return nbr

    def _c(self):
        m = _Mesh(self.nx, self.ny, self.nz, self.k, self.nq if self.nq != self.k + 1 else 0,
                  self.nu, self.c, self.eta,
                  _p(self.xn), _p(self.yn), _p(self.zn), 1 if self.walls else 0)
        self._keep = m
        return ctypes.byref(m)

    def shape(self):
        return (self.ne, 4, self.nb)


def _arr(x, m):
    a = np.ascontiguousarray(x, dtype=np.float64)
    assert a.size == m.n, (a.shape, m.shape())
    return a


def residual(m, w):
    """f_h(w; phi_m e_i), Eq. (NSdiscrRes)."""
    w = _arr(w, m)
    f = np.zeros(m.shape())
    lib().orc_residual(m._c(), _p(w), _p(f))
    return f


def jvp(m, w, v, inv_gdt):
    """G v = J(w) v + M v/(gamma dt): exact derivative of the residual + mass form."""
    w, v = _arr(w, m), _arr(v, m)
    out = np.zeros(m.shape())
    lib().orc_jvp(m._c(), _p(w), _p(v), float(inv_gdt), _p(out))
    return out


def jvp_fd(m, w, v, inv_gdt, eps=1e-9):
    """Finite-difference G v of Eqs. (matrix-free), (epsdef)."""
    w, v = _arr(w, m), _arr(v, m)
    out = np.zeros(m.shape())
    lib().orc_jvp_fd(m._c(), _p(w), _p(v), float(inv_gdt), float(eps), _p(out))
    return out


def dense_G(m, w, inv_gdt):
    """Dense G = J(w) + M/(gamma dt), column by column of the exact Jacobian action."""
    w = _arr(w, m)
    G = np.zeros((m.n, m.n))
    lib().orc_dense_G(m._c(), _p(w), float(inv_gdt), _p(G))
    return G


def project_tgv(m):
    """L2 projection (Gauss rule) of the Taylor-Green vortex field."""
    w = np.zeros(m.shape())
    lib().orc_project_tgv(m._c(), _p(w))
    return w


def quad_points(m):
    npt = m.nq ** 3
    x = np.zeros((m.ne, npt, 3))
    wq = np.zeros((m.ne, npt))
    lib().orc_quad_points(m._c(), _p(x), _p(wq))
    return x, wq


def project_points(m, vals):
    """L2 projection of values at the volume Gauss points, vals[ne][4][nq^3]."""
    vals = np.ascontiguousarray(vals, dtype=np.float64)
    w = np.zeros(m.shape())
    lib().orc_project_points(m._c(), _p(vals), _p(w))
    return w


def basis(m, e, xi):
    xi = np.ascontiguousarray(np.atleast_2d(xi), dtype=np.float64)
    npt = xi.shape[0]
    phi = np.zeros((npt, m.nb))
    dphi = np.zeros((npt, m.nb, 3))
    lib().orc_basis(m._c(), int(e), npt, _p(xi), _p(phi), _p(dphi))
    return phi, dphi


def eval_field(m, w, e, xi):
    w = _arr(w, m)
    xi = np.ascontiguousarray(np.atleast_2d(xi), dtype=np.float64)
    out = np.zeros((xi.shape[0], 4))
    lib().orc_eval_field(m._c(), _p(w), int(e), xi.shape[0], _p(xi), _p(out))
    return out


def riemann(uL, pL, uR, pR, d, c):
    """Exact AC Riemann interface flux along e_d: (flux[4], u*, p*, u_face[3])."""
    uL = np.ascontiguousarray(uL, dtype=np.float64)
    uR = np.ascontiguousarray(uR, dtype=np.float64)
    flux = np.zeros(4)
    star = np.zeros(3)
    uf = np.zeros(3)
    lib().orc_riemann(_p(uL), float(pL), _p(uR), float(pR), int(d), float(c), _p(flux), _p(star), _p(uf))
    return flux, star[0], star[1], uf


def riemann_tangent(uL, pL, uR, pR, duL, dpL, duR, dpR, d, c):
    a = [np.ascontiguousarray(x, dtype=np.float64) for x in (uL, uR, duL, duR)]
    out = np.zeros(4)
    lib().orc_riemann_tangent(_p(a[0]), float(pL), _p(a[1]), float(pR), _p(a[2]), float(dpL), _p(a[3]),
                              float(dpR), int(d), float(c), _p(out))
    return out


def p_wave1(u, uL, pL, c):
    return lib().orc_p_wave1(u, uL, pL, c)


def p_wave3(u, uR, pR, c):
    return lib().orc_p_wave3(u, uR, pR, c)


def tang1(u, uL, c):
    return lib().orc_tang1(u, uL, c)


def tang3(u, uR, c):
    return lib().orc_tang3(u, uR, c)
