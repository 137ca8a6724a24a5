"""The FP32 cycle with its fine-level volume contractions on the tensor cores (through the C ABI).

DG_PRECOND_FP32_H16_TC / _BF16_TC run the quadrature contractions of the convective volume term of
the linearised residual (Sec. 2.1, Eq. (NSdiscrRes)) -- interpolation of the velocity variation to
the Gauss points, integration of the weighted products against the basis -- as dense per-element
tcgen05 GEMMs with 16-bit operands and FP32 accumulation; everything else is the FP32 cycle with
16-bit block storage.

Stated errors (derivation): every operand of the two contractions is rounded once to 16 bits (the
basis table, the scaled velocity coefficients, the weighted products): unit roundoff u = 2^-11
(FP16) or 2^-8 (bfloat16). The interpolated values carry at most 2u relative error per term and
the projections another 2u; the convective contribution, a part of the operator's output,
therefore changes by a few u of its own size. One cycle is compared with the oracle's cycle at
10 x (2 + 2) u on top of the 16-bit block-storage bound of the same cycle without tensor cores
(5e-3 FP16, 4e-2 bfloat16): 2.5e-2 for FP16, 2e-1 for bfloat16; and with that cycle without
tensor cores at 10 x 4u: 2e-2 (FP16), 1.6e-1 (bfloat16). FGMRES stays FP64, so a stage solved with
the FP16 form still reaches 1e-10, checked with the oracle's exact operator.
"""
import numpy as np
import pytest

import oracle as O
import oracle.solvers as SV
import synthetic as S
from _gpu_common import dev, host, maxrel, meshes, pair, rel

pytestmark = pytest.mark.gpu

BOUND_ORACLE = {"H16": 2.5e-2, "BF16": 2e-1}
BOUND_NO_TC = {"H16": 2e-2, "BF16": 1.6e-1}


@pytest.mark.parametrize("name,levels", [("u3", [2, 1]), ("box233", [4, 2, 1]), ("u4", [4, 2, 1]),
                                         ("box345", [3, 1])])
@pytest.mark.parametrize("storage", ["H16", "BF16"])
def test_tensor_core_cycle_matches_oracle(name, levels, storage):
    import paper_1809_00866_gb300 as P
    dg, m = pair(*meshes()[name], levels)
    w = O.project_tgv(m) + S.perturbation(m.ne, m.k, 0.2, 1)
    inv = 1.0 / S.acoustic_dt(m.nx, m.k)
    dg.dg_set_linearization(dev(w), inv)
    dg.dg_assemble()
    G0 = O.dense_G(m, w, inv)
    Gs = [G0] + [SV.inherited_operator(G0, m.ne, m.nb, O.nb(kl)) for kl in levels[1:]]
    nbs = [O.nb(k) for k in levels]
    lv = [SV.Level(lambda v, G=G: G @ v, SV.block_inverses(G, m.ne, nb), m.ne, nb) for G, nb in zip(Gs, nbs)]
    g = -O.residual(m, w).reshape(-1)
    ref = SV.mg_v(lv, 0, g, np.zeros_like(g))
    gd = dev(g.reshape(dg.empty().shape))
    x_tc, x_16 = dg.empty(), dg.empty()
    dg.pmg_vcycle(gd, x_tc, P.solve_opts(precision=getattr(P, "DG_PRECOND_FP32_%s_TC" % storage)))
    dg.pmg_vcycle(gd, x_16, P.solve_opts(precision=getattr(P, "DG_PRECOND_FP32_%s" % storage)))
    assert dg.dg_get_status() == 0
    a, b = host(x_tc).reshape(-1), host(x_16).reshape(-1)
    print("%s %s: vs oracle %.2e (max %.2e), vs the cycle without tensor cores %.2e, that cycle vs oracle %.2e"
          % (name, storage, rel(a, ref), maxrel(a, ref), rel(a, b), rel(b, ref)))
    assert rel(a, ref) < BOUND_ORACLE[storage]
    assert maxrel(a, ref) < BOUND_ORACLE[storage]
    assert rel(a, b) < BOUND_NO_TC[storage]
    assert rel(a, b) > 0.0  # the tensor-core path really ran a different contraction


def test_tensor_core_cycle_reaches_fp64_accuracy():
    import paper_1809_00866_gb300 as P
    un = S.uniform_nodes(4)
    dg, m = pair(un, un, un, [4, 2, 1])
    w = O.project_tgv(m)
    inv = 1.0 / S.acoustic_dt(4, 4)
    g = dg.empty()
    dg.dg_set_linearization_rhs(dev(w), inv, g)
    dg.dg_assemble(precision=P.DG_PRECOND_FP32_H16_TC)
    x = dg.empty()
    info, rc = dg.fgmres_solve(g, x, P.solve_opts(rtol=1e-10, maxit=300, omega=0.95, pre_sweeps=4, post_sweeps=4,
                                                   precision=P.DG_PRECOND_FP32_H16_TC))
    assert rc == P.DG_OK
    G0 = O.dense_G(m, w, inv)
    gr = host(g).reshape(-1)
    assert np.linalg.norm(gr - G0 @ host(x).reshape(-1)) / np.linalg.norm(gr) < 1e-9


def test_tensor_core_cycle_at_benchmark_size():
    # 16^3 P4: 196 tiles of 21 elements over two CTAs per SM; against the cycle without tensor cores
    import paper_1809_00866_gb300 as P
    un = S.uniform_nodes(16)
    dg, m = pair(un, un, un, [4, 2, 1])
    g = dg.empty()
    dg.dg_set_linearization_rhs(dev(O.project_tgv(m)), 1.0 / S.acoustic_dt(16, 4), g)
    dg.dg_assemble(precision=P.DG_PRECOND_FP32)
    xs = {}
    for st in ("H16", "H16_TC", "BF16", "BF16_TC"):
        xs[st] = dg.empty()
        dg.pmg_vcycle(g, xs[st], P.solve_opts(omega=0.95, pre_sweeps=4, post_sweeps=4,
                                              precision=getattr(P, "DG_PRECOND_FP32_" + st)))
    assert dg.dg_get_status() == 0
    e16 = rel(host(xs["H16_TC"]), host(xs["H16"]))
    ebf = rel(host(xs["BF16_TC"]), host(xs["BF16"]))
    print("16^3 P4 cycle, tensor cores vs CUDA cores: FP16 %.2e, BF16 %.2e" % (e16, ebf))
    assert 0.0 < e16 < BOUND_NO_TC["H16"]
    assert 0.0 < ebf < BOUND_NO_TC["BF16"]


def test_tensor_core_wait_gives_up_and_recovers():
    # the volume pass's bounded MMA waits: with a limit of one poll the wait for the first MMA gives
    # up (DG_STATUS_WAIT) unless the MMA already landed; the next cycle at the production limit is
    # the same as before
    import paper_1809_00866_gb300 as P
    dg, m = pair(*meshes()["u4"], [4, 2, 1])
    g = dg.empty()
    dg.dg_set_linearization_rhs(dev(O.project_tgv(m)), 1.0 / S.acoustic_dt(4, 4), g)
    dg.dg_assemble(precision=P.DG_PRECOND_FP32)
    opts = P.solve_opts(precision=P.DG_PRECOND_FP32_H16_TC)
    x0, x1 = dg.empty(), dg.empty()
    dg.pmg_vcycle(g, x0, opts)
    assert dg.dg_get_status() == 0
    dg.dg_set_test_knob(P.DG_KNOB_WAIT_POLLS, 1)
    dg.pmg_vcycle(g, x1, opts)
    st = dg.dg_get_status()
    dg.dg_set_test_knob(P.DG_KNOB_WAIT_POLLS, 0)
    assert st & ~P.DG_STATUS_WAIT == 0
    dg.pmg_vcycle(g, x1, opts)
    assert dg.dg_get_status() == 0
    assert rel(host(x1), host(x0)) == 0.0
