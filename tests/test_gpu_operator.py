"""GPU parity of the matrix-free operator against the FP64 oracle (called through the C ABI).

Tolerance: the FP64 kernels and the oracle evaluate the same discrete operator
with different summation orders, Newton vs bisection for the Riemann star state
and different table generators, so they agree to rounding: relative 2-norm
difference <= 1e-12 for the residual and the exact Jacobian action. The
finite-difference action amplifies rounding by 1/Delta ~ 1e9, so it is compared
with a 1e-5 bound (Sec. 2.3: FD is accurate to tolerances above eps = 1e-9).
"""
import numpy as np
import pytest

import oracle as O
import synthetic as S
from _gpu_common import dev, host, meshes, pair, rel

pytestmark = pytest.mark.gpu

CASES = [("u2", 1), ("u2", 2), ("u2", 3), ("u2", 4), ("u3", 2), ("box233", 2), ("box345", 3), ("u4", 4)]


def state(m, seed, amp=0.3):
    return O.project_tgv(m) + S.perturbation(m.ne, m.k, amp, seed)


@pytest.mark.parametrize("name,k", CASES)
def test_tgv_projection(name, k):
    dg, m = pair(*meshes()[name], [k])
    w = dg.empty()
    dg.dg_project_tgv(w)
    assert rel(host(w), O.project_tgv(m)) < 1e-13


@pytest.mark.parametrize("name,k", CASES)
def test_residual(name, k):
    dg, m = pair(*meshes()[name], [k])
    w = state(m, 10 + k)
    f = dg.empty()
    dg.dg_residual(dev(w), f)
    ref = O.residual(m, w)
    assert rel(host(f), ref) < 1e-12
    assert dg.dg_get_status() == 0


@pytest.mark.parametrize("name,k", CASES)
def test_tangent_jvp(name, k):
    dg, m = pair(*meshes()[name], [k])
    w = state(m, 20 + k)
    v = S.direction(m.ne, k, 30 + k)
    inv_gdt = 1.0 / S.acoustic_dt(m.nx, k)
    dg.dg_set_linearization(dev(w), inv_gdt)
    out = dg.empty()
    dg.dg_jvp(dev(v), out, mode=0)
    ref = O.jvp(m, w, v, inv_gdt)
    assert rel(host(out), ref) < 1e-12


@pytest.mark.parametrize("name,k", [("u2", 2), ("box233", 3), ("u4", 4)])
def test_fd_jvp(name, k):
    dg, m = pair(*meshes()[name], [k])
    w = state(m, 40 + k)
    v = S.direction(m.ne, k, 50 + k)
    dg.dg_set_linearization(dev(w), 0.25)
    out = dg.empty()
    dg.dg_jvp(dev(v), out, mode=1)
    assert rel(host(out), O.jvp_fd(m, w, v, 0.25)) < 1e-5
    assert rel(host(out), O.jvp(m, w, v, 0.25)) < 1e-5
    # zero direction gives exactly the zero action
    z = dg.empty().zero_()
    dg.dg_jvp(z, out, mode=1)
    assert float(out.abs().max()) == 0.0


def test_tgv_symmetric_state_and_free_stream():
    # the pure Taylor-Green state has faces where u* is zero up to rounding (tie band)
    dg, m = pair(*meshes()["u4"], [3])
    w = O.project_tgv(m)
    f = dg.empty()
    dg.dg_residual(dev(w), f)
    assert rel(host(f), O.residual(m, w)) < 1e-12
    v = S.direction(m.ne, 3, 7)
    dg.dg_set_linearization(dev(w), 0.5)
    out = dg.empty()
    dg.dg_jvp(dev(v), out)
    assert rel(host(out), O.jvp(m, w, v, 0.5)) < 1e-12
    # free stream: the residual of a constant state vanishes
    wc = np.zeros(m.shape())
    for var, cval in enumerate((0.3, -0.7, 0.45, 1.3)):
        wc[:, var, 0] = cval * np.sqrt(m.vol())
    dg.dg_residual(dev(wc), f)
    assert float(f.abs().max()) < 1e-12
    assert dg.dg_get_status() == 0


def test_deterministic():
    dg, m = pair(*meshes()["box345"], [2])
    w = dev(state(m, 3))
    a, b = dg.empty(), dg.empty()
    dg.dg_residual(w, a)
    dg.dg_residual(w, b)
    assert bool((a == b).all())


def test_argument_errors_do_not_launch():
    import paper_1809_00866_gb300 as P
    dg, m = pair(*meshes()["u2"], [2])
    w = dg.empty()
    with pytest.raises(P.DgError) as e:
        dg.dg_jvp(w, dg.empty())  # no linearisation yet
    assert e.value.code == P.DG_ERR_STATE
    with pytest.raises(P.DgError) as e:
        dg.dg_residual(w, w)  # aliasing
    assert e.value.code == P.DG_ERR_ARG


def test_linearization_rhs_is_minus_residual():
    # one nonlinear face pass gives both the linearisation and the stage right-hand side -f(w)
    dg, m = pair(*meshes()["box233"], [3, 1])
    w = O.project_tgv(m) + S.perturbation(m.ne, m.k, 0.2, 21)
    g = dg.empty()
    inv = 1.0 / S.acoustic_dt(m.nx, m.k)
    dg.dg_set_linearization_rhs(dev(w), inv, g)
    assert rel(host(g), -O.residual(m, w)) < 1e-12
    v = S.direction(m.ne, m.k, 22)
    out = dg.empty()
    dg.dg_jvp(dev(v), out)
    assert rel(host(out), O.jvp(m, w, v, inv)) < 1e-12
