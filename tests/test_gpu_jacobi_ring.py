"""The staged block-Jacobi apply of the FP32 cycle when every CTA walks its ring of stage
buffers many times (through the C ABI, against the oracle).

The apply (Sec. 2.3, element-wise block Jacobi, x <- x + omega D^-1 (g - G x)) deals stages of
G consecutive elements to its CTAs round-robin; a CTA reuses a stage buffer once it has taken
more stages than the ring has buffers, which on the benchmark's 16^3 mesh happens about seven
times per CTA, but never on small meshes at the default launch shape. A cap on the CTAs
(dg_tuning.jacobi_max_ctas) makes one or a few CTAs take every stage here, with several stage
sizes (jacobi_stage_kb): G = 1, 2, 15, 16 and 30 elements, ragged last stages, and the
column-slice reduction (stages of few rows) as well as the direct path. With 16-bit blocks of
140 rows (the P4 fine level of box233) the apply takes one element per stage in a ring of five
buffers, whatever the stage size asked for; the cap still applies.

Reference: the oracle's V-cycle (Algorithm 2) on its dense operators. The cycle runs its
fine-level and coarse-level smoothing through this apply. Bounds per block storage, as for the
uncapped cycle: FP32 1e-5, FP16 5e-3, bfloat16 4e-2 (ten times the storage unit roundoff),
in the 2-norm and element by element relative to the largest entry.
"""
import numpy as np
import pytest

import oracle as O
import oracle.solvers as SV
import synthetic as S
from _gpu_common import dev, host, maxrel, meshes, pair, rel

pytestmark = pytest.mark.gpu

BOUND = {"FP32": 1e-5, "FP32_H16": 5e-3, "FP32_BF16": 4e-2}
_cache = {}


def _setup(name, levels):
    key = (name, tuple(levels))
    if key not in _cache:
        dg, m = pair(*meshes()[name], levels)
        w = O.project_tgv(m) + S.perturbation(m.ne, m.k, 0.2, 3)
        inv = 1.0 / S.acoustic_dt(m.nx, m.k)
        G0 = O.dense_G(m, w, inv)
        Gs = [G0] + [SV.inherited_operator(G0, m.ne, m.nb, O.nb(kl)) for kl in levels[1:]]
        nbs = [O.nb(k) for k in levels]
        lv = [SV.Level(lambda v, G=G: G @ v, SV.block_inverses(G, m.ne, nb), m.ne, nb) for G, nb in zip(Gs, nbs)]
        g = -O.residual(m, w).reshape(-1)
        ref = SV.mg_v(lv, 0, g, np.zeros_like(g), 2, 2, 2, 0.9)
        _cache[key] = (dg, m, w, inv, g, ref)
    return _cache[key]


@pytest.mark.parametrize("name,levels", [("u4", [2, 1]), ("box233", [4, 2, 1])])
@pytest.mark.parametrize("storage", ["FP32", "FP32_H16", "FP32_BF16"])
@pytest.mark.parametrize("max_ctas,stage_kb", [(1, 8), (1, 48), (2, 96), (3, 8), (1, 224)])
def test_ring_reuse_matches_oracle_cycle(name, levels, storage, max_ctas, stage_kb):
    import paper_1809_00866_gb300 as P
    dg, m, w, inv, g, ref = _setup(name, levels)
    prec = getattr(P, "DG_PRECOND_" + storage)
    dg.dg_set_linearization(dev(w), inv)
    dg.dg_assemble(precision=prec)
    dg.dg_set_tuning(P.DG_TUNE_FP32, jacobi_max_ctas=max_ctas, jacobi_stage_kb=stage_kb)
    x = dg.empty()
    dg.pmg_vcycle(dev(g.reshape(x.shape)), x, P.solve_opts(precision=prec, omega=0.9))
    assert dg.dg_get_status() == 0
    got = host(x).reshape(-1)
    assert rel(got, ref) < BOUND[storage]
    assert maxrel(got, ref) < BOUND[storage]
    # the uncapped launch agrees with the capped one to the same bound
    dg.dg_set_tuning(P.DG_TUNE_FP32, jacobi_max_ctas=0, jacobi_stage_kb=96)
    x0 = dg.empty()
    dg.pmg_vcycle(dev(g.reshape(x.shape)), x0, P.solve_opts(precision=prec, omega=0.9))
    assert maxrel(host(x0).reshape(-1), ref) < BOUND[storage]
