"""Training of the learned coarse-level correction from pairs the solver itself generates.

Host-side orchestration over the C ABI: the arithmetic of every step runs in the library's
kernels; torch only holds the buffers and does the bookkeeping (indexing, scaling a recorded
vector to unit norm, reporting norms).

1. ``collect_pairs``: for each linearisation state, one implicit-stage solve with the plain
   cycle records the right-hand sides that reach the coarsest (P1) level
   (``dg_record_coarse``); each is then solved to a tight tolerance on that level
   (``pmg_level_solve``: GMRES with element-block-Jacobi preconditioning, the coarse solver of
   Sec. 2.4.3) and turned into per-element pairs (``dg_coarse_pairs``): normalised features of
   the element and its six face neighbours, and the element's solution scaled alike. Every
   pair also enters with both signs (the coarse problem is linear).
2. ``train``: Adam on the mean squared error with the BF16 forward/backward kernels
   (``dg_mlp_grad``, ``dg_mlp_adam``), mini-batches drawn on the device by a counter hash.
3. ``dg_set_coarse_network`` installs the result for ``DG_COARSE_LEARNED``.
"""
import math
import time

import numpy as np

from . import (DG_MLP_HIDDEN, DG_MLP_IN, DG_MLP_NPARAM, DG_MLP_OUT, dg_mlp_adam, dg_mlp_grad, mlp_workspace)


def init_theta(seed=0, out_scale=0.1):
    """He-normal hidden layers, a small output layer, zero biases (FP32 CUDA tensor)."""
    import torch
    rng = np.random.default_rng(seed)
    W1 = rng.standard_normal((DG_MLP_HIDDEN, DG_MLP_IN)) * math.sqrt(2.0 / DG_MLP_IN)
    W2 = rng.standard_normal((DG_MLP_HIDDEN, DG_MLP_HIDDEN)) * math.sqrt(2.0 / DG_MLP_HIDDEN)
    W3 = rng.standard_normal((DG_MLP_OUT, DG_MLP_HIDDEN)) * math.sqrt(1.0 / DG_MLP_HIDDEN) * out_scale
    th = np.concatenate([W1.ravel(), np.zeros(DG_MLP_HIDDEN), W2.ravel(), np.zeros(DG_MLP_HIDDEN), W3.ravel(),
                         np.zeros(DG_MLP_OUT)]).astype(np.float32)
    assert th.size == DG_MLP_NPARAM
    return torch.from_numpy(th).cuda()


def collect_rhs(dg, states, inv_gamma_dt, opts, per_state=32):
    """Run one plain solve per state (opts with the plain coarse solve) and return the recorded
    coarsest-level right-hand sides, each made consistent (``pmg_project_pressure``) and scaled
    to unit norm: a float64 tensor [N, ne, 4, nb1]. The FP64 assembly is left in place."""
    import torch
    lc = len(dg.levels) - 1
    nc = dg.n[lc]
    out = []
    for w in states:
        g = dg.empty()
        dg.dg_set_linearization_rhs(w, inv_gamma_dt, g)
        dg.dg_assemble()
        buf = torch.empty(per_state * nc, dtype=torch.float64, device="cuda")
        dg.dg_record_coarse(buf, per_state)
        x = dg.empty()
        dg.fgmres_solve(g, x, opts)
        cnt = dg.dg_recorded()
        dg.dg_record_coarse(None)
        for r in range(cnt):
            d = buf[r * nc:(r + 1) * nc].view(dg.ne, 4, dg.nb[lc])
            dg.pmg_project_pressure(lc, d)
            nrm = float(d.norm().item())  # bookkeeping: scale each vector to unit norm
            if nrm > 0:
                out.append((d / nrm).contiguous())
    return torch.stack(out)


def train_residual(dg, D, steps=2000, lr=1e-3, lr_final=5e-5, seed=0, theta=None, iterate_every=2, val=None,
                   extra=None):
    """Train N as a local approximate inverse of the coarsest-level operator G of the handle's
    current assembly: minimise ||d - G s N(X(d))||^2 over recorded right-hand sides d (whole
    coarse vectors, all elements form the batch). Each step: x = s N(X) (``dg_coarse_apply``),
    r = d - G x (``bsr_spmv``), q = G^T r (``bsr_spmv_t``), residual targets
    (``dg_coarse_pairs`` with q), BF16 gradient (``dg_mlp_grad``) and Adam. Every
    ``iterate_every``-th step trains on the residual d - G x of the current network instead, the
    input that the next iteration of ``DG_COARSE_LEARNED_ITER`` sees. ``extra``: more
    (handle, vectors) sets, for instance of another mesh; the steps cycle through the sets, each
    with its own handle's operator. The network ends installed on every handle. Returns
    (theta, report)."""
    import torch
    sets = [(dg, D)] + list(extra or [])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    th = init_theta(seed, out_scale=0.01) if theta is None else theta.clone()
    m = torch.zeros_like(th)
    v = torch.zeros_like(th)
    grad = torch.empty_like(th)
    bufs = []
    for h, _ in sets:
        lc = len(h.levels) - 1
        bufs.append({"X": torch.empty((h.ne, DG_MLP_IN), dtype=torch.float32, device="cuda"),
                     "T": torch.empty((h.ne, DG_MLP_OUT), dtype=torch.float32, device="cuda"),
                     "s": torch.empty(h.ne, dtype=torch.float32, device="cuda"),
                     "vec": [h.empty(lc) for _ in range(4)], "ws": mlp_workspace(h.ne), "lc": lc})
    rng = np.random.default_rng(seed)

    for it in range(1, steps + 1):
        si = (it - 1) % len(sets)
        h, Dh = sets[si]
        b = bufs[si]
        lc = b["lc"]
        y, r, q, d2 = b["vec"]

        def residual(d):
            h.dg_coarse_apply(d, y)
            r.copy_(d)
            h.bsr_spmv(lc, -1.0, y, 1.0, r)

        h.dg_set_coarse_network(th)
        d = Dh[int(rng.integers(len(Dh)))]
        if iterate_every and it % iterate_every == 0:
            residual(d)
            d2.copy_(r)
            d = d2
        residual(d)
        h.bsr_spmv_t(lc, 1.0, r, 0.0, q)
        h.dg_coarse_pairs(d, y, b["X"], b["T"], b["s"], q=q)
        dg_mlp_grad(th, b["X"], b["T"], h.ne, grad, ws=b["ws"])
        c = 0.5 * (1.0 + math.cos(math.pi * (it - 1) / max(1, steps - 1)))
        dg_mlp_adam(th, grad, m, v, it, lr=lr_final + (lr - lr_final) * c)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    for h, _ in sets:
        h.dg_set_coarse_network(th)
    rep = {"steps": steps, "train_s": t_train, "vectors": int(sum(len(Dh) for _, Dh in sets)),
           "vectors_per_set": [int(len(Dh)) for _, Dh in sets]}
    if val is not None:
        rep["val_residual_ratio"] = residual_ratio(dg, val)
    return th, rep


def residual_ratio(dg, D):
    """Mean over the vectors d of ||d - G s N(X(d))|| / ||d|| with the handle's network."""
    lc = len(dg.levels) - 1
    y, r = dg.empty(lc), dg.empty(lc)
    vals = []
    for d in D:
        dg.dg_coarse_apply(d, y)
        r.copy_(d)
        dg.bsr_spmv(lc, -1.0, y, 1.0, r)
        vals.append(float(r.norm().item()) / max(float(d.norm().item()), 1e-300))
    return float(np.mean(vals))


def collect_pairs(dg, states, inv_gamma_dt, opts, per_state=32, level_rtol=1e-6, level_maxit=2000,
                  both_signs=True):
    """Run one plain solve per state (opts must use the plain coarse solve) and return the
    per-element pairs (X [N, 112], T [N, 16]) of the recorded coarsest-level problems, plus
    statistics. ``states``: iterable of fine-level state tensors."""
    import torch
    lc = len(dg.levels) - 1
    nc = dg.n[lc]
    Xs, Ts = [], []
    its_level, nrec = [], 0
    for w in states:
        g = dg.empty()
        dg.dg_set_linearization_rhs(w, inv_gamma_dt, g)
        dg.dg_assemble()  # FP64: the level solves below need it (the FP32 cycle rounds it)
        buf = torch.empty(per_state * nc, dtype=torch.float64, device="cuda")
        dg.dg_record_coarse(buf, per_state)
        x = dg.empty()
        dg.fgmres_solve(g, x, opts)
        cnt = dg.dg_recorded()
        dg.dg_record_coarse(None)
        for r in range(cnt):
            d = buf[r * nc:(r + 1) * nc].view(dg.ne, 4, dg.nb[lc])
            # the coarse operator is singular along the constant pressure: make d consistent
            # (its rounding leaves a small inconsistent part) and take the solution without it
            dg.pmg_project_pressure(lc, d)
            xs = dg.empty(lc)
            info, _ = dg.pmg_level_solve(lc, d, xs, rtol=level_rtol, maxit=level_maxit)
            dg.pmg_project_pressure(lc, xs)
            its_level.append(info.its)
            X = torch.empty((dg.ne, DG_MLP_IN), dtype=torch.float32, device="cuda")
            T = torch.empty((dg.ne, DG_MLP_OUT), dtype=torch.float32, device="cuda")
            s = torch.empty(dg.ne, dtype=torch.float32, device="cuda")
            dg.dg_coarse_pairs(d, xs, X, T, s)
            keep = s > 0
            Xs.append(X[keep])
            Ts.append(T[keep])
        nrec += cnt
    X = torch.cat(Xs)
    T = torch.cat(Ts)
    if both_signs:
        X = torch.cat([X, -X])
        T = torch.cat([T, -T])
    stats = {"recorded": nrec, "pairs": int(X.shape[0]),
             "level_solve_its_mean": float(np.mean(its_level)) if its_level else 0.0}
    return X.contiguous(), T.contiguous(), stats


def train(X, T, steps=3000, batch=4096, lr=2e-3, lr_final=1e-4, seed=0, theta=None, val_frac=0.05, log_every=0):
    """Adam with a cosine learning-rate decay; returns (theta, report). The last ``val_frac`` of
    a seeded permutation of the pairs is held out for the validation error."""
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    n = X.shape[0]
    perm = torch.from_numpy(np.random.default_rng(seed).permutation(n)).cuda()
    nval = max(1, int(n * val_frac))
    Xtr, Ttr = X[perm[nval:]].contiguous(), T[perm[nval:]].contiguous()
    Xva, Tva = X[perm[:nval]].contiguous(), T[perm[:nval]].contiguous()
    th = init_theta(seed) if theta is None else theta.clone()
    m = torch.zeros_like(th)
    v = torch.zeros_like(th)
    grad = torch.empty_like(th)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    ws = mlp_workspace(batch)
    hist = []
    for it in range(1, steps + 1):
        dg_mlp_grad(th, Xtr, Ttr, batch, grad, loss, seed=seed, step=it, ws=ws)
        c = 0.5 * (1.0 + math.cos(math.pi * (it - 1) / max(1, steps - 1)))
        dg_mlp_adam(th, grad, m, v, it, lr=lr_final + (lr - lr_final) * c)
        if log_every and (it % log_every == 0 or it == 1):
            hist.append((it, float(loss.item())))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    return th, {"steps": steps, "batch": batch, "train_s": t_train, "history": hist,
                "val_rel_err": validation_error(th, Xva, Tva), "train_pairs": int(Xtr.shape[0]),
                "val_pairs": int(nval)}


def validation_error(theta, X, T, chunk=1 << 16):
    """||N(X) - T|| / ||T|| over the rows of X (BF16 forward kernel)."""
    import torch
    from . import dg_mlp_forward
    num = den = 0.0
    ws = mlp_workspace(min(chunk, X.shape[0]))
    for a in range(0, X.shape[0], chunk):
        xb = X[a:a + chunk].contiguous()
        yb = torch.empty((xb.shape[0], DG_MLP_OUT), dtype=torch.float32, device="cuda")
        dg_mlp_forward(theta, xb, yb, ws=ws)
        num += float(((yb - T[a:a + chunk]) ** 2).sum().item())
        den += float((T[a:a + chunk] ** 2).sum().item())
    return math.sqrt(num / den) if den > 0 else 0.0
