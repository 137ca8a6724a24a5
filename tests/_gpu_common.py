"""Shared helpers of the GPU parity tests: build the CUDA library, mirror a mesh in the oracle."""
import numpy as np
import pytest

import oracle as O
import synthetic as S


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1809_00866_gb300 as P
    P.build()  # fails loudly if nvcc or the sources are broken; there is no fallback
    P.load()
    return torch, P


def pair(xn, yn, zn, levels, nu=S.NU_TGV, c=S.AC_C, eta=S.ETA):
    torch, P = require_gpu()
    dg = P.DG(xn, yn, zn, levels, nu, c, eta)
    m = O.Mesh(xn, yn, zn, levels[0], nu, c, eta)
    return dg, m


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / (nb if nb > 0 else 1.0)


# meshes: (name, xn, yn, zn)
def meshes():
    u = S.uniform_nodes
    p = S.perturbed_nodes
    return {
        "u2": (u(2), u(2), u(2)),
        "u3": (u(3), u(3), u(3)),
        "u4": (u(4), u(4), u(4)),
        "box233": (p(2, seed=1), p(3, seed=2), p(3, seed=3)),
        "box345": (p(3, seed=4), p(4, seed=5), p(5, seed=6)),
    }


def maxrel(a, b):
    """Element-wise difference relative to the largest entry: max |a - b| / max |b|."""
    a, b = np.asarray(a).reshape(-1), np.asarray(b).reshape(-1)
    mb = np.abs(b).max()
    return float(np.abs(a - b).max() / (mb if mb > 0 else 1.0))
