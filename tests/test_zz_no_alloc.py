"""dg_residual_noalloc: the residual for callers that must not allocate device memory.

Some callers own the whole device memory budget (a host application that forbids
its plugins to call cudaMalloc) or run where an allocation is not allowed; they
use this entry point, whose scratch lives in a fixed static device array. It must
return what dg_residual returns, call after call (the shared array keeps the last
call's contents), and refuse meshes that do not fit the array. This file is
collected last so that a failure here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
import synthetic as S
from _gpu_common import dev, host, meshes, pair, rel

pytestmark = pytest.mark.gpu


def _noalloc(dg, w, f):
    import torch
    L = dg._L
    return L.dg_residual_noalloc(dg.h, ctypes.c_void_p(w.data_ptr()), ctypes.c_void_p(f.data_ptr()),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def _free_bytes():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


@pytest.mark.parametrize("name,k", [("box345", 3), ("u4", 4)])
def test_noalloc_residual_matches_dg_residual_twice(name, k):
    import paper_1809_00866_gb300 as P
    dg, m = pair(*meshes()[name], [k])
    outs = []
    for seed in (1, 2):  # two calls in a row with different states
        wh = O.project_tgv(m) + S.perturbation(m.ne, k, 0.3, seed)
        w = dev(wh)
        ref = dg.empty()
        dg.dg_residual(w, ref)  # the existing entry point (its kernels' module is loaded by now)
        got = dg.empty().fill_(np.nan)
        free0 = _free_bytes()
        assert _noalloc(dg, w, got) == P.DG_OK
        # the call allocated nothing: the device's free memory is unchanged across it
        assert _free_bytes() == free0
        assert rel(host(got), host(ref)) < 1e-12
        # and both equal the oracle's residual, element by element as well as in norm
        orc = O.residual(m, wh)
        assert rel(host(got), orc) < 1e-12
        assert np.abs(host(got) - orc).max() <= 1e-12 * np.abs(orc).max()
        outs.append(host(got))
    assert rel(outs[0], outs[1]) > 1e-6  # the second call really recomputed
    assert dg.dg_get_status() == 0


def test_noalloc_rejects_meshes_beyond_the_static_scratch():
    import paper_1809_00866_gb300 as P
    un = S.uniform_nodes(16)
    dg, _ = pair(un, un, un, [4])  # 4096 elements at P4 need 6.0e6 doubles > 2^20
    w = dg.empty().zero_()
    f = dg.empty()
    assert _noalloc(dg, w, f) == P.DG_ERR_ARG
    assert b"too large for the static scratch" in dg._L.dg_last_error(dg.h)
