"""Checkpoint / resume of a solver state and the per-solve JSONL log (host I/O).

CPU: a state written and read back is bit-for-bit the same, the header describes the
discretisation, and a checkpoint of another discretisation is refused. GPU: a stage resumed from
a reloaded state on a new handle equals the stage continued in memory, bit for bit.
"""
import json
import types

import numpy as np
import pytest

import synthetic as S


def _stub(levels=(3, 2, 1), n=(3, 4, 5), nu=S.NU_TGV):
    nodes = [S.uniform_nodes(m) for m in n]
    params = types.SimpleNamespace(nx=n[0], ny=n[1], nz=n[2], nu=nu, ac_c=S.AC_C, eta=S.ETA, walls=0)
    ne, nb = int(np.prod(n)), S.nb(levels[0])
    return types.SimpleNamespace(params=params, levels=list(levels), ne=ne, nb=[nb], n=[ne * 4 * nb], nprob=1,
                                 _nodes=nodes, elem_start=[0, ne])


def test_state_roundtrip_is_bitwise(tmp_path):
    pytest.importorskip("torch")
    from paper_1809_00866_gb300.checkpoint import load_state, save_state
    dg = _stub()
    w = np.random.default_rng(4).standard_normal((dg.ne, 4, dg.nb[0]))
    w[0, 0, 0] = np.nextafter(1.0, 2.0)  # a value that any rounding on the way would change
    path = str(tmp_path / "state")
    save_state(path, w, dg, t=1.25, step=7, inv_gamma_dt=0.5, extra={"case": "box345"})
    got, hdr = load_state(path, dg, device=None)
    assert np.array_equal(got.numpy(), w)
    assert hdr["t"] == 1.25 and hdr["step"] == 7 and hdr["inv_gamma_dt"] == 0.5 and hdr["levels"] == [3, 2, 1]
    assert hdr["cells"] == [3, 4, 5] and hdr["extra"] == {"case": "box345"}
    with pytest.raises(ValueError):
        load_state(path, _stub(levels=(3, 1)), device=None)  # another p-level hierarchy
    with pytest.raises(ValueError):
        load_state(path, _stub(nu=2e-3), device=None)  # another viscosity


def test_solve_log_lines(tmp_path):
    from paper_1809_00866_gb300.checkpoint import log_solve
    info = types.SimpleNamespace(its=12, status=0, r0=3.0, relres_est=9e-9, true_relres=9.5e-9, rho=0.2, fallback_at=-1)
    path = str(tmp_path / "solves.jsonl")
    log_solve(path, info, 0, stage=1)
    log_solve(path, info, 3, stage=2)
    lines = [json.loads(x) for x in open(path)]
    assert [x["stage"] for x in lines] == [1, 2] and lines[1]["rc"] == 3 and lines[0]["its"] == 12


@pytest.mark.gpu
def test_resume_from_checkpoint_equals_continuing(tmp_path):
    from _gpu_common import pair, require_gpu
    torch, P = require_gpu()
    from paper_1809_00866_gb300.checkpoint import load_state, save_state
    un = S.uniform_nodes(4)
    levels = [3, 2, 1]
    inv = 1.0 / S.acoustic_dt(4, 3, cfl=5.0)  # a time step at which consecutive stages converge quickly
    opts = P.solve_opts(rtol=1e-8, maxit=200, omega=0.9, precision=P.DG_PRECOND_FP32_H16)

    def stage(dg, w, log=None):
        g, x = dg.empty(), dg.empty()
        dg.dg_set_linearization_rhs(w, inv, g)
        dg.dg_assemble(precision=opts.precision)
        info, rc = dg.fgmres_solve(g, x, opts, log=log)
        assert rc == P.DG_OK
        dg.dg_stage_update(w, x)

    dg, _ = pair(un, un, un, levels)
    w = dg.empty()
    dg.dg_project_tgv(w)
    stage(dg, w)
    path = str(tmp_path / "tgv4")
    save_state(path, w, dg, step=1, inv_gamma_dt=inv)
    stage(dg, w, log=str(tmp_path / "solves.jsonl"))  # continued in memory
    dg2, _ = pair(un, un, un, levels)
    w2, hdr = load_state(path, dg2)
    assert hdr["step"] == 1
    stage(dg2, w2)  # resumed on a new handle
    assert torch.equal(w, w2)
    assert json.loads(open(str(tmp_path / "solves.jsonl")).readline())["true_relres"] <= 1e-8
