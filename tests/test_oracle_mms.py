"""h/p convergence of the oracle's discretisation on a manufactured solution.

The manufactured problem is sigma u + div(F^c - F^nu) = s (momentum) and
div u = s_p (continuity) on the periodic cube, with s computed symbolically from
a smooth (u, p). The reaction term sigma*M is the implicit-stage mass term of
Eq. (rosSysOp) with 1/(gamma dt) = sigma; it removes the near-null space of
constant velocities of the steady periodic problem. The discrete problem
f_h(w) + sigma M w = s_h is solved by a chord-Newton iteration on the dense
oracle Jacobian. The L2 velocity error must fall under h- and p-refinement
at the rates of a consistent, stable DG method (order k+1 in h).
"""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
import synthetic as S

sp = pytest.importorskip("sympy")

NU = 0.1
SIG = 1.0


def _problem():
    x, y, z = sp.symbols("x y z")
    X = [x, y, z]
    A = 0.5
    u = [A * (sp.sin(x + y) + 0.4 * sp.cos(z)), A * (0.8 * sp.cos(x - z) + 0.2), A * 0.6 * sp.sin(y) * sp.cos(x)]
    p = A * (0.4 * sp.cos(x) * sp.sin(z) + 0.2 * sp.sin(y))
    div = sum(sp.diff(u[j], X[j]) for j in range(3))
    src = []
    for i in range(3):
        s = SIG * u[i]
        for j in range(3):
            fv = NU * (sp.diff(u[i], X[j]) + sp.diff(u[j], X[i]) - (sp.Rational(2, 3) * div if i == j else 0))
            s += sp.diff(u[i] * u[j] + (p if i == j else 0) - fv, X[j])
        src.append(s)
    src.append(div)
    lam = lambda es: [sp.lambdify((x, y, z), e, "numpy") for e in es]
    return lam(src), lam(u + [p])


def _project(m, funcs):
    xq, _ = O.quad_points(m)
    vals = np.zeros((m.ne, 4, xq.shape[1]))
    for v in range(4):
        vals[:, v] = funcs[v](xq[..., 0], xq[..., 1], xq[..., 2]) + 0.0 * xq[..., 0]
    return O.project_points(m, vals)


def _solve_error(n, k, fs, fe):
    m = O.Mesh(S.uniform_nodes(n), S.uniform_nodes(n), S.uniform_nodes(n), k, NU, S.AC_C, S.ETA)
    sh = _project(m, fs)
    we = _project(m, fe)
    w = we.copy()
    G = O.dense_G(m, w, SIG)
    # constant pressure is the null vector of G on the periodic mesh; border it away
    nvec = np.zeros(m.shape())
    nvec[:, 3, 0] = np.sqrt(m.vol())
    nvec = nvec.reshape(-1) / np.linalg.norm(nvec)
    lu = sla.lu_factor(G + np.outer(nvec, nvec))
    for _ in range(10):
        r = O.residual(m, w) + SIG * np.concatenate([w[:, :3], 0 * w[:, 3:]], 1) - sh
        w = w + sla.lu_solve(lu, -r.reshape(-1)).reshape(w.shape)
    r = O.residual(m, w) + SIG * np.concatenate([w[:, :3], 0 * w[:, 3:]], 1) - sh
    assert np.abs(r).max() < 1e-7
    return np.sqrt(np.sum((w - we)[:, :3] ** 2))


@pytest.mark.slow
def test_h_convergence_p2():
    fs, fe = _problem()
    errs = [_solve_error(n, 2, fs, fe) for n in (2, 3, 4)]
    hs = [2 * np.pi / n for n in (2, 3, 4)]
    rates = [np.log(errs[i] / errs[i + 1]) / np.log(hs[i] / hs[i + 1]) for i in range(2)]
    assert errs[0] > errs[1] > errs[2]
    assert rates[-1] > 2.5, (errs, rates)


@pytest.mark.slow
def test_p_convergence_n2():
    fs, fe = _problem()
    errs = [_solve_error(2, k, fs, fe) for k in (1, 2, 3, 4)]
    assert all(errs[i + 1] < errs[i] for i in range(3)), errs
    assert errs[3] < 0.2 * errs[1], errs
