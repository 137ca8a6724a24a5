"""GPU parity of the learned coarse correction (BF16 network kernels) against the FP64 oracle.

Tolerances come from the arithmetic: the kernels round the weights and every layer input to
bfloat16 (unit roundoff u = 2^-9) and accumulate in FP32. Against the oracle evaluated with the
same operand rounding (``forward_bf16``) the outputs differ only by FP32 accumulation order and
by the rare input whose rounding flips between neighbouring bfloat16 values (relative 2^-8 on
that input): 2e-3 normwise. The gradient kernel also rounds the backward operands (dY, dZ, the
activations of the weight-gradient products), so it is held to the FP64 gradient at 4e-2
normwise per parameter block, with cosine similarity above 0.999.
"""
import numpy as np
import pytest

import oracle as O
import oracle.mlp as M
import oracle.solvers as SV
import synthetic as S
from _gpu_common import dev, host, meshes, pair, rel, require_gpu

pytestmark = pytest.mark.gpu


def theta_np(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    parts = []
    for name, shp in M.SHAPES:
        fan = shp[1] if len(shp) == 2 else 1
        parts.append(rng.standard_normal(shp).ravel() * (0.3 if name.startswith("b") else scale / np.sqrt(fan)))
    return np.concatenate(parts)


def f32(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("n", [1, 63, 200])
def test_forward_matches_oracle(n):
    torch, P = require_gpu()
    th = theta_np(1)
    X = np.random.default_rng(2).standard_normal((n, M.N_IN)) / np.sqrt(M.N_IN)
    X32 = X.astype(np.float32).astype(np.float64)
    Y = torch.empty((n, M.N_OUT), dtype=torch.float32, device="cuda")
    P.dg_mlp_forward(f32(th), f32(X), Y)
    y = host(Y).astype(np.float64)
    th32 = th.astype(np.float32).astype(np.float64)
    assert rel(y, M.forward_bf16(th32, X32)) < 2e-3
    assert rel(y, M.forward(th32, X32)[0]) < 3e-2


@pytest.mark.parametrize("batch", [16, 130, 300])
def test_gradient_matches_oracle(batch):
    torch, P = require_gpu()
    th = theta_np(3)
    rng = np.random.default_rng(4)
    X = rng.standard_normal((batch, M.N_IN)) / np.sqrt(M.N_IN)
    T = rng.standard_normal((batch, M.N_OUT)) * 0.5
    th32, X32, T32 = (a.astype(np.float32).astype(np.float64) for a in (th, X, T))
    loss_o, g_o = M.loss_and_grad(th32, X32, T32)
    grad = torch.empty(M.n_params(), dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    P.dg_mlp_grad(f32(th), f32(X), f32(T), batch, grad, loss)
    g = host(grad).astype(np.float64)
    assert abs(float(host(loss)[0]) - loss_o) / loss_o < 1e-2
    go, gg = M.unpack(g_o), M.unpack(g)
    for name, _ in M.SHAPES:
        assert rel(gg[name], go[name]) < 4e-2, name
    cos = float(np.dot(g, g_o) / (np.linalg.norm(g) * np.linalg.norm(g_o)))
    assert cos > 0.999
    # determinism: the fixed-order reduction gives the same bits twice
    grad2 = torch.empty_like(grad)
    P.dg_mlp_grad(f32(th), f32(X), f32(T), batch, grad2)
    assert torch.equal(grad, grad2)


def test_adam_step_formula():
    torch, P = require_gpu()
    rng = np.random.default_rng(5)
    n = M.n_params()
    th, g, m, v = (rng.standard_normal(n).astype(np.float32) for _ in range(4))
    v = np.abs(v)
    t, lr, b1, b2, eps = 3, 1e-2, 0.9, 0.999, 1e-8
    T_, G_, M_, V_ = f32(th), f32(g), f32(m), f32(v)
    P.dg_mlp_adam(T_, G_, M_, V_, t, lr, b1, b2, eps)
    # Adam (Kingma & Ba 2015, Algorithm 1) in FP64, with the decay rates as the kernel holds them (FP32)
    b1, b2 = float(np.float32(b1)), float(np.float32(b2))
    m1 = b1 * m + (1 - b1) * g.astype(np.float64)
    v1 = b2 * v + (1 - b2) * g.astype(np.float64) ** 2
    ref = th - lr * (m1 / (1 - b1 ** t)) / (np.sqrt(v1 / (1 - b2 ** t)) + eps)
    np.testing.assert_allclose(host(M_), m1, rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(host(V_), v1, rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(host(T_), ref, rtol=1e-5, atol=1e-6)


def test_training_fits_a_teacher():
    # a student trained by the kernels on a teacher network's outputs lowers its error 4-fold
    torch, P = require_gpu()
    import paper_1809_00866_gb300.learned as Lrn
    teacher = theta_np(6)
    X = np.random.default_rng(7).standard_normal((8192, M.N_IN))
    X /= np.linalg.norm(X, axis=1, keepdims=True)
    T = M.forward(teacher, X)[0]
    th0 = Lrn.init_theta(8)
    Xd, Td = f32(X), f32(T)
    e0 = Lrn.validation_error(th0, Xd, Td)
    th, rep = Lrn.train(Xd, Td, steps=600, batch=1024, lr=3e-3, lr_final=3e-4, seed=9, theta=th0)
    print("teacher fit: rel err %.3e -> %.3e" % (e0, rep["val_rel_err"]))
    assert rep["val_rel_err"] < 0.25 * e0, (e0, rep["val_rel_err"])


def _two_level(name="u3", levels=(2, 1), amp=0.2):
    # amp = 0: the Taylor-Green state itself, on which the block-Jacobi cycle converges
    dg, m = pair(*meshes()[name], list(levels))
    w = O.project_tgv(m) + S.perturbation(m.ne, m.k, amp, 3)
    inv = 1.0 / S.acoustic_dt(m.nx, m.k)
    dg.dg_set_linearization(dev(w), inv)
    dg.dg_assemble()
    return dg, m, w, inv


def test_coarse_pairs_match_oracle():
    torch, P = require_gpu()
    dg, m, w, inv = _two_level("box345", (2, 1))
    rng = np.random.default_rng(10)
    d = rng.standard_normal((m.ne, 4, 4))
    x = rng.standard_normal((m.ne, 4, 4))
    X = torch.empty((m.ne, M.N_IN), dtype=torch.float32, device="cuda")
    T = torch.empty((m.ne, M.N_OUT), dtype=torch.float32, device="cuda")
    s = torch.empty(m.ne, dtype=torch.float32, device="cuda")
    dg.dg_coarse_pairs(dev(d), dev(x), X, T, s)
    Xo, so = M.features(d, m.neighbours(), 4)
    np.testing.assert_allclose(host(X), Xo, rtol=2e-7, atol=1e-7)
    np.testing.assert_allclose(host(s), so, rtol=2e-7)
    np.testing.assert_allclose(host(T), x.reshape(m.ne, 16) / so[:, None], rtol=2e-7, atol=1e-7)
    # residual targets: T = x / s + s q
    q = rng.standard_normal((m.ne, 4, 4))
    dg.dg_coarse_pairs(dev(d), dev(x), X, T, s, q=dev(q))
    ref = x.reshape(m.ne, 16) / so[:, None] + so[:, None] * q.reshape(m.ne, 16)
    np.testing.assert_allclose(host(T), ref, rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("name", ["u2", "box345"])
def test_bsr_transpose(name):
    torch, P = require_gpu()
    dg, m, w, inv = _two_level(name, (2, 1))
    G0 = O.dense_G(m, w, inv)
    G1 = SV.inherited_operator(G0, m.ne, m.nb, O.nb(1))
    rng = np.random.default_rng(17)
    x = rng.standard_normal(G1.shape[0])
    y0 = rng.standard_normal(G1.shape[0])
    yd = dev(y0.reshape(m.ne, 4, 4))
    dg.bsr_spmv_t(1, 0.6, dev(x.reshape(m.ne, 4, 4)), -0.4, yd)
    np.testing.assert_allclose(host(yd).reshape(-1), 0.6 * G1.T @ x - 0.4 * y0, rtol=0,
                               atol=1e-12 * np.abs(G1).max() * np.abs(x).max() * 7 * 16)


def test_coarse_apply():
    torch, P = require_gpu()
    dg, m, w, inv = _two_level("box345", (2, 1))
    th = theta_np(18)
    dg.dg_set_coarse_network(f32(th))
    rng = np.random.default_rng(19)
    d = rng.standard_normal((m.ne, 4, 4))
    d[7] = 0.0
    x0 = rng.standard_normal((m.ne, 4, 4))
    xd = dev(x0)
    dg.dg_coarse_apply(dev(d), xd, accumulate=True)
    ref = M.coarse_correction(th.astype(np.float32).astype(np.float64), d, m.neighbours(), 4)
    assert rel(host(xd) - x0, ref) < 2e-3
    dg.dg_coarse_apply(dev(d), xd)
    assert rel(host(xd), ref) < 2e-3


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name,levels", [("box345", (2, 1)), ("u4", (3, 2, 1))])
def test_learned_coarse_correction_in_the_cycle(name, levels, precision):
    # with no smoothing the V-cycle is P N(R g): the learned correction alone
    torch, P = require_gpu()
    dg, m, w, inv = _two_level(name, levels)
    th = theta_np(11)
    dg.dg_set_coarse_network(f32(th))
    g = np.random.default_rng(12).standard_normal(m.shape())
    x = dg.empty()
    o = P.solve_opts(pre_sweeps=0, post_sweeps=0, coarse_sweeps=0, coarse_solver=P.DG_COARSE_LEARNED,
                     precision=precision)
    dg.pmg_vcycle(dev(g), x, o)
    nbc = O.nb(1)
    dc = SV.restrict(g.reshape(-1), m.ne, m.nb, nbc).reshape(m.ne, 4, nbc)
    if precision == 1:
        dc = dc.astype(np.float32).astype(np.float64)
    xc = M.coarse_correction(th.astype(np.float32).astype(np.float64), dc, m.neighbours(), nbc)
    ref = SV.prolong(xc.reshape(-1), m.ne, m.nb, nbc).reshape(m.shape())
    assert rel(host(x), ref) < 2e-3
    assert dg.dg_get_status() == 0


def test_level_solve_reaches_tolerance():
    torch, P = require_gpu()
    dg, m, w, inv = _two_level("u3", (2, 1))
    G0 = O.dense_G(m, w, inv)
    G1 = SV.inherited_operator(G0, m.ne, m.nb, O.nb(1))
    xt = np.random.default_rng(13).standard_normal(G1.shape[0])
    d = G1 @ xt  # in the range of the (pressure-singular) coarse operator
    x = dg.empty(1)
    info, rc = dg.pmg_level_solve(1, dev(d.reshape(m.ne, 4, 4)), x, rtol=1e-10, maxit=3000)
    assert rc == P.DG_OK and info.true_relres <= 1e-10
    assert np.linalg.norm(d - G1 @ host(x).reshape(-1)) <= 2e-10 * np.linalg.norm(d)


def test_record_and_gmres_coarse_solver():
    torch, P = require_gpu()
    dg, m, w, inv = _two_level("u4", (2, 1), amp=0.0)
    f = dg.empty()
    dg.dg_residual(dev(w), f)
    g = (-f).contiguous()
    buf = torch.zeros(5 * dg.n[1], dtype=torch.float64, device="cuda")
    dg.dg_record_coarse(buf, 5)
    x = dg.empty()
    o = P.solve_opts(rtol=1e-10, maxit=60, pre_sweeps=0, coarse_solver=P.DG_COARSE_GMRES, coarse_sweeps=40)
    info, rc = dg.fgmres_solve(g, x, o)
    n = dg.dg_recorded()
    dg.dg_record_coarse(None)
    assert rc == P.DG_OK and n == min(5, info.its)
    # the first recorded right-hand side is the restriction of the first Krylov vector g/||g||
    g0 = host(g).reshape(-1) / np.linalg.norm(host(g))
    r0 = SV.restrict(g0, m.ne, m.nb, O.nb(1))
    np.testing.assert_allclose(host(buf[:dg.n[1]]), r0, rtol=0, atol=1e-15)
    # the oracle's exact operator confirms the converged solution
    G0 = O.dense_G(m, w, inv)
    gr = host(g).reshape(-1)
    assert np.linalg.norm(gr - G0 @ host(x).reshape(-1)) <= 2e-10 * np.linalg.norm(gr)


def test_fallback_on_nonfinite_and_on_stall():
    torch, P = require_gpu()
    dg, m, w, inv = _two_level("u4", (2, 1), amp=0.0)
    f = dg.empty()
    dg.dg_residual(dev(w), f)
    g = (-f).contiguous()
    G0 = O.dense_G(m, w, inv)
    gr = host(g).reshape(-1)
    # a network whose weights are not finite: the first Arnoldi vector is redone with the plain cycle
    th = theta_np(14)
    th[5] = np.inf
    dg.dg_set_coarse_network(f32(th))
    x = dg.empty()
    o = P.solve_opts(rtol=1e-10, maxit=80, coarse_solver=P.DG_COARSE_LEARNED, coarse_sweeps=2)
    info, rc = dg.fgmres_solve(g, x, o)
    assert rc == P.DG_OK and info.fallback_at == 0
    assert np.linalg.norm(gr - G0 @ host(x).reshape(-1)) <= 2e-10 * np.linalg.norm(gr)
    # an untrained network judged by the outer residual: dropped once it stalls (the GMRES
    # smoother keeps the cycle convergent after the network has left the symmetric subspace)
    dg.dg_set_coarse_network(f32(theta_np(15, scale=30.0)))
    o = P.solve_opts(rtol=1e-8, maxit=300, coarse_solver=P.DG_COARSE_LEARNED, coarse_sweeps=2, fallback_its=2,
                     fallback_rho=0.05, smoother=P.DG_SMOOTH_GMRES, pre_sweeps=3, post_sweeps=3)
    info, rc = dg.fgmres_solve(g, x, o)
    print("stall fallback: its %d, fallback at %d, rel res %.2e" % (info.its, info.fallback_at, info.true_relres))
    assert info.fallback_at >= 2
    assert rc == P.DG_OK
    assert np.linalg.norm(gr - G0 @ host(x).reshape(-1)) <= 2e-8 * np.linalg.norm(gr)
    # without a network the learned solver is refused
    dg.dg_set_coarse_network(None)
    with pytest.raises(P.DgError):
        dg.fgmres_solve(g, x, o)


def test_project_pressure():
    torch, P = require_gpu()
    dg, m, w, inv = _two_level("box345", (2, 1))
    rng = np.random.default_rng(16)
    for lvl, nb in ((0, O.nb(2)), (1, O.nb(1))):
        x = rng.standard_normal((m.ne, 4, nb))
        xd = dev(x)
        dg.pmg_project_pressure(lvl, xd)
        c = np.zeros_like(x)
        c[:, 3, 0] = np.sqrt(m.vol())  # the constant pressure 1 in the orthonormal basis
        ref = x - (np.sum(c * x) / np.sum(c * c)) * c
        np.testing.assert_allclose(host(xd), ref, rtol=0, atol=1e-13)
    # c is a null vector of the fine operator: G c = 0
    c = np.zeros(m.shape())
    c[:, 3, 0] = np.sqrt(m.vol())
    out = dg.empty()
    dg.dg_jvp(dev(c), out)
    assert np.abs(host(out)).max() < 1e-12 * np.abs(c).max() * inv + 1e-12
