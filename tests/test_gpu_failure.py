"""Failure detection of the kernels, exercised without any GPU fault (through the C ABI).

Each condition is made on the host side: a test setting (dg_set_test_knob) or a non-finite
value planted in a host buffer before it is copied to the device. Nothing here faults, traps
or waits without bound: the waits that run out are bounded by a few thousand polls.

* Riemann: the star-state iteration of the exact artificial-compressibility Riemann flux
  (Sec. 2.1) capped at 0 or 1 iterations misses its stopping test on generic faces; the kernels
  set DG_STATUS_RIEMANN and dg_set_linearization returns DG_ERR_RIEMANN.
* Non-finite values: a NaN in the state sets DG_STATUS_NONFINITE from the operator's output
  scan; dg_set_linearization returns DG_ERR_NONFINITE; fgmres_solve rejects a NaN right-hand side.
* Bounded waits: the FP32 cycle's staged block-Jacobi apply, told to withhold every CTA's first
  stage copy, gives up after its poll limit, drains its other copies, sets DG_STATUS_WAIT and
  leaves the context usable (the next apply is correct).
"""
import numpy as np
import pytest

import oracle as O
import oracle.solvers as SV
import synthetic as S
from _gpu_common import dev, host, maxrel, meshes, pair, rel

pytestmark = pytest.mark.gpu


def generic_state(m, seed):
    return O.project_tgv(m) + S.perturbation(m.ne, m.k, 0.3, seed)


@pytest.mark.parametrize("cap", [0, 1])
def test_riemann_iteration_cap_is_reported(cap):
    import paper_1809_00866_gb300 as P
    dg, m = pair(*meshes()["box233"], [2])
    w = generic_state(m, 7)
    inv = 1.0 / S.acoustic_dt(m.nx, m.k)
    dg.dg_set_test_knob(P.DG_KNOB_RIEMANN_ITS, cap)
    with pytest.raises(P.DgError) as e:
        dg.dg_set_linearization(dev(w), inv)
    assert e.value.code == P.DG_ERR_RIEMANN
    assert dg.dg_get_status() & P.DG_STATUS_RIEMANN
    with pytest.raises(P.DgError) as e:  # not linearised after the failure
        dg.dg_jvp(dev(S.direction(m.ne, m.k, 3)), dg.empty())
    assert e.value.code == P.DG_ERR_STATE
    f = dg.empty()
    dg.dg_residual(dev(w), f)  # asynchronous: reported through the status word
    assert dg.dg_get_status() & P.DG_STATUS_RIEMANN
    # the production cap: no condition, and the operator is the oracle's again
    dg.dg_set_test_knob(P.DG_KNOB_RIEMANN_ITS, 60)
    dg.dg_set_linearization(dev(w), inv)
    assert dg.dg_get_status() == 0
    dg.dg_residual(dev(w), f)
    assert dg.dg_get_status() == 0
    assert rel(host(f), O.residual(m, w)) < 1e-12


def test_nonfinite_state_is_reported():
    import paper_1809_00866_gb300 as P
    dg, m = pair(*meshes()["u3"], [3, 1])
    w = generic_state(m, 8)
    bad = w.copy()
    bad[5, 1, 3] = np.nan  # planted in the host buffer
    inv = 1.0 / S.acoustic_dt(m.nx, m.k)
    f = dg.empty()
    dg.dg_residual(dev(bad), f)
    assert dg.dg_get_status() & P.DG_STATUS_NONFINITE
    with pytest.raises(P.DgError) as e:
        dg.dg_set_linearization(dev(bad), inv)
    assert e.value.code == P.DG_ERR_NONFINITE
    assert dg.dg_get_status() & P.DG_STATUS_NONFINITE
    # a clean state afterwards: no condition; FGMRES refuses a right-hand side with a NaN
    g = dg.empty()
    dg.dg_set_linearization_rhs(dev(w), inv, g)
    dg.dg_assemble()
    assert dg.dg_get_status() == 0
    # a flag left unread by an earlier call is not the assembly's: it succeeds, the flag stays
    dg.dg_residual(dev(bad), f)
    dg.dg_set_linearization_rhs(dev(w), inv, g)
    dg.dg_assemble()
    assert dg.dg_get_status() & P.DG_STATUS_NONFINITE
    assert dg.dg_get_status() == 0
    gh = host(g).copy()
    gh[2, 0, 1] = np.inf
    x = dg.empty()
    info, rc = dg.fgmres_solve(dev(gh), x, P.solve_opts(rtol=1e-8, maxit=50), check=False)
    assert rc == P.DG_ERR_NONFINITE
    # the finite right-hand side is accepted again (a few iterations, whatever their outcome)
    info, rc = dg.fgmres_solve(g, x, P.solve_opts(rtol=1e-8, maxit=5, omega=0.9), check=False)
    assert rc in (P.DG_OK, P.DG_ERR_NOT_CONVERGED) and info.its > 0 and np.isfinite(info.true_relres)
    assert dg.dg_get_status() == 0


@pytest.mark.parametrize("levels,storage", [([2, 1], "FP32_H16"), ([2, 1], "FP32"), ([4, 2, 1], "FP32_H16"),
                                            ([4, 2, 1], "FP32_BF16")])
def test_staged_jacobi_wait_gives_up_and_recovers(levels, storage):
    # the FP32 cycle's fine-level block-Jacobi apply inside one V-cycle: with the first stage of
    # every CTA withheld, each CTA's first wait runs out after 2000 polls (at P4 with 16-bit
    # blocks, the one-element-per-stage apply of 140 x 140 inverses)
    import paper_1809_00866_gb300 as P
    dg, m = pair(*meshes()["u4"], levels)
    w = O.project_tgv(m)
    inv = 1.0 / S.acoustic_dt(m.nx, m.k)
    g = dg.empty()
    dg.dg_set_linearization_rhs(dev(w), inv, g)
    prec = getattr(P, "DG_PRECOND_" + storage)
    dg.dg_assemble(precision=prec)
    opts = P.solve_opts(precision=prec, omega=0.9)
    ref = dg.empty()
    dg.pmg_vcycle(g, ref, opts)
    assert dg.dg_get_status() == 0
    dg.dg_set_test_knob(P.DG_KNOB_WAIT_POLLS, 2000)
    dg.dg_set_test_knob(P.DG_KNOB_WITHHOLD_COPY, 1)
    x = dg.empty()
    dg.pmg_vcycle(g, x, opts)
    assert dg.dg_get_status() & P.DG_STATUS_WAIT
    # back to the production settings: the context is usable and the cycle is what it was
    dg.dg_set_test_knob(P.DG_KNOB_WITHHOLD_COPY, 0)
    dg.dg_set_test_knob(P.DG_KNOB_WAIT_POLLS, 0)
    dg.pmg_vcycle(g, x, opts)
    assert dg.dg_get_status() == 0
    assert rel(host(x), host(ref)) == 0.0
