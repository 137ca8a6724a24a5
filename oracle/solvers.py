"""Plain numpy solver algorithms of the p-multigrid preconditioned FGMRES (oracle).

TEST INFRASTRUCTURE (see ``oracle/__init__.py``). Follows the paper's
statements directly, on dense matrices of tiny meshes:

* restriction / prolongation (Sec. 2.4.1): with a hierarchical orthonormal
  basis the L2 restriction keeps the modes of degree <= k_{l+1} and the
  injection zero-pads;
* inherited coarse operators (Eq. (GalProj)): M J M^T with a unit-diagonal
  rectangular M, i.e. the sub-matrix of G_0 on the coarse modes;
* element-wise block Jacobi (Sec. 2.3, EWBJ): inverse of the diagonal element
  blocks; smoothing x <- x + omega D^{-1} (g - G x);
* MG_V (Algorithm 2) and MG_full (Algorithm 3);
* right-preconditioned flexible GMRES (Sec. 2.4.3, Saad 1993), restarted;
* convergence factor rho (Appendix B).

Vectors are numpy arrays laid out [element][u, v, w, p][mode] (flattened).
"""
import numpy as np


def coarse_index(ne, nb_fine, nb_coarse):
    """Global indices (into a fine vector) of the coarse modes, in coarse layout order."""
    e = np.arange(ne)[:, None, None]
    v = np.arange(4)[None, :, None]
    m = np.arange(nb_coarse)[None, None, :]
    return ((e * 4 + v) * nb_fine + m).reshape(-1)


def restrict(x, ne, nb_fine, nb_coarse):
    """L2 restriction P^{k_l} -> P^{k_{l+1}}: keep the leading modes."""
    return np.asarray(x).reshape(ne, 4, nb_fine)[:, :, :nb_coarse].reshape(-1).copy()


def prolong(xc, ne, nb_fine, nb_coarse):
    """Injection P^{k_{l+1}} -> P^{k_l}: zero-pad the missing modes."""
    out = np.zeros((ne, 4, nb_fine))
    out[:, :, :nb_coarse] = np.asarray(xc).reshape(ne, 4, nb_coarse)
    return out.reshape(-1)


def inherited_operator(G0, ne, nb0, nbl):
    """G_l = M G_0 M^T: sub-matrix of the fine operator on the coarse modes."""
    idx = coarse_index(ne, nb0, nbl)
    return G0[np.ix_(idx, idx)].copy()


def stb_scaling(k0, kl, d=3):
    """Scaling factor S_0^l = k_l (k_l + d) / (k_0 (k_0 + d)) of the stabilisation term on level l
    (Appendix A: the trace-inequality constant grows like k (k + d))."""
    return kl * (kl + d) / (k0 * (k0 + d))


def rescaled_inherited_operator(G0, Gstb, ne, nb0, nbl, k0, kl, d=3):
    """Rescaled inherited coarse operator of Appendix A: the Galerkin projection of the fine
    operator with its viscous stabilisation part Gstb (the BR2 penalty terms) weighted by S_0^l:
    M (G0 - Gstb) M^T + S_0^l M Gstb M^T."""
    idx = coarse_index(ne, nb0, nbl)
    S = stb_scaling(k0, kl, d)
    return G0[np.ix_(idx, idx)] + (S - 1.0) * Gstb[np.ix_(idx, idx)]


def diag_blocks(G, ne, nb):
    """Element diagonal blocks of G (block size 4*nb)."""
    b = 4 * nb
    return np.stack([G[e * b:(e + 1) * b, e * b:(e + 1) * b] for e in range(ne)])


def block_inverses(G, ne, nb):
    """Inverses of the element diagonal blocks (EWBJ)."""
    return np.stack([np.linalg.inv(B) for B in diag_blocks(G, ne, nb)])


def apply_block_inverse(Dinv, r):
    ne, b, _ = Dinv.shape
    return np.einsum("eij,ej->ei", Dinv, np.asarray(r).reshape(ne, b)).reshape(-1)


def bsr_from_dense(G, ne, nb, nbr):
    """Block rows with (diagonal + one block per face) in the order of ``nbr``.

    nbr[e] lists the 6 face neighbours (-x, +x, -y, +y, -z, +z). When a
    neighbour appears on two faces (two elements along an axis) its coupling
    block is stored at the first of those faces and a zero block at the other,
    so the sum over the row's blocks reproduces G.
    """
    b = 4 * nb
    cols = np.zeros((ne, 7), dtype=np.int64)
    vals = np.zeros((ne, 7, b, b))
    for e in range(ne):
        cols[e, 0] = e
        vals[e, 0] = G[e * b:(e + 1) * b, e * b:(e + 1) * b]
        for f in range(6):
            p = int(nbr[e][f])
            cols[e, f + 1] = p
            if p not in [int(q) for q in nbr[e][:f]]:
                vals[e, f + 1] = G[e * b:(e + 1) * b, p * b:(p + 1) * b]
    return cols, vals


def bsr_matvec(cols, vals, x):
    ne, nblk, b, _ = vals.shape
    X = np.asarray(x).reshape(ne, b)
    y = np.zeros((ne, b))
    for j in range(nblk):
        y += np.einsum("eij,ej->ei", vals[:, j], X[cols[:, j]])
    return y.reshape(-1)


def block_jacobi(matvec, Dinv, g, x, sweeps, omega=1.0):
    """``sweeps`` damped element-block-Jacobi iterations x <- x + omega D^{-1}(g - G x)."""
    x = np.array(x, dtype=np.float64, copy=True)
    for _ in range(sweeps):
        x = x + omega * apply_block_inverse(Dinv, g - matvec(x))
    return x


def gmres_smooth(matvec, Dinv, g, x, iters):
    """``iters`` iterations of GMRES left-preconditioned by the element block inverses (EWBJ).

    The smoother of Sec. 2.4.3 ("all the smoothers of the multigrid strategy are
    GMRES"): from x, minimise ||D^{-1}(g - G y)||_2 over y in x + K_iters(D^{-1}G, D^{-1}(g - G x)),
    built by modified Gram-Schmidt Arnoldi with Givens rotations; no restart.
    """
    x = np.array(x, dtype=np.float64, copy=True)
    r = apply_block_inverse(Dinv, g - matvec(x))
    beta = np.linalg.norm(r)
    if iters <= 0 or beta == 0.0:
        return x
    n = g.size
    V = np.zeros((iters + 1, n))
    H = np.zeros((iters + 1, iters))
    V[0] = r / beta
    cs = np.zeros(iters)
    sn = np.zeros(iters)
    s = np.zeros(iters + 1)
    s[0] = beta
    k = 0
    for j in range(iters):
        w = apply_block_inverse(Dinv, matvec(V[j]))
        for i in range(j + 1):
            H[i, j] = np.dot(w, V[i])
            w = w - H[i, j] * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] != 0.0:
            V[j + 1] = w / H[j + 1, j]
        for i in range(j):
            t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
            H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
            H[i, j] = t
        den = np.hypot(H[j, j], H[j + 1, j])
        cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
        H[j, j] = den
        H[j + 1, j] = 0.0
        s[j + 1] = -sn[j] * s[j]
        s[j] = cs[j] * s[j]
        k = j + 1
        if H[j + 1, j] == 0.0 and den == 0.0:
            break
    y = np.linalg.solve(np.triu(H[:k, :k]), s[:k])
    return x + V[:k].T @ y


def smooth(smoother, matvec, Dinv, g, x, iters, omega):
    if smoother == "gmres":
        return gmres_smooth(matvec, Dinv, g, x, iters)
    return block_jacobi(matvec, Dinv, g, x, iters, omega)


class Level:
    """One p-multigrid level: operator (callable), block inverses, sizes."""

    def __init__(self, matvec, Dinv, ne, nb):
        self.matvec, self.Dinv, self.ne, self.nb = matvec, Dinv, ne, nb


def mg_v(levels, l, g, x, pre=2, post=2, coarse_sweeps=2, omega=1.0, smoother="jacobi"):
    """MG_V(l, g_l, w_l) of Algorithm 2.

    SMOOTH is ``pre`` / ``post`` iterations of the chosen smoother (damped element-block
    Jacobi sweeps, or GMRES left-preconditioned by the element block inverses); the
    coarsest SOLVE is ``coarse_sweeps`` iterations of the same smoother from 0.
    """
    L = len(levels) - 1
    lv = levels[l]
    if l == L:
        return smooth(smoother, lv.matvec, lv.Dinv, g, np.zeros_like(g), coarse_sweeps, omega)
    xb = smooth(smoother, lv.matvec, lv.Dinv, g, x, pre, omega)       # pre-smoothing
    d = g - lv.matvec(xb)                                              # defect
    dc = restrict(d, lv.ne, lv.nb, levels[l + 1].nb)                   # restriction
    e = mg_v(levels, l + 1, dc, np.zeros_like(dc), pre, post, coarse_sweeps, omega, smoother)
    xh = xb + prolong(e, lv.ne, lv.nb, levels[l + 1].nb)               # coarse-grid correction
    return smooth(smoother, lv.matvec, lv.Dinv, g, xh, post, omega)   # post-smoothing


def mg_full(levels, l, g, pre=2, post=2, coarse_sweeps=2, omega=1.0, smoother="jacobi"):
    """MG_full(l, g_l, 0) of Algorithm 3."""
    L = len(levels) - 1
    lv = levels[l]
    if l == L:
        return smooth(smoother, lv.matvec, lv.Dinv, g, np.zeros_like(g), coarse_sweeps, omega)
    gc = restrict(g, lv.ne, lv.nb, levels[l + 1].nb)
    wc = mg_full(levels, l + 1, gc, pre, post, coarse_sweeps, omega, smoother)
    wh = prolong(wc, lv.ne, lv.nb, levels[l + 1].nb)
    d = g - lv.matvec(wh)
    e = mg_v(levels, l, d, np.zeros_like(d), pre, post, coarse_sweeps, omega, smoother)
    return wh + e


def fgmres(matvec, precond, g, x0=None, restart=30, maxit=200, rtol=1e-8, fixed_its=None):
    """Right-preconditioned flexible GMRES(restart) (Saad 1993), modified Gram-Schmidt.

    Stops when the recurrence residual falls below rtol * ||g - G x0||, or after
    exactly ``fixed_its`` iterations when given. Returns (x, its, history of
    recurrence residual norms).
    """
    n = g.size
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    r = g - matvec(x)
    beta0 = np.linalg.norm(r)
    hist = [beta0]
    its = 0
    limit = fixed_its if fixed_its is not None else maxit
    if beta0 == 0.0:
        return x, 0, hist
    while its < limit:
        beta = np.linalg.norm(r)
        m = min(restart, limit - its)
        V = np.zeros((m + 1, n))
        Z = np.zeros((m, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        s = np.zeros(m + 1)
        s[0] = beta
        V[0] = r / beta
        j_done = 0
        for j in range(m):
            Z[j] = precond(V[j])
            wv = matvec(Z[j])
            for i in range(j + 1):
                H[i, j] = np.dot(wv, V[i])
                wv = wv - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(wv)
            if H[j + 1, j] != 0.0:
                V[j + 1] = wv / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            s[j + 1] = -sn[j] * s[j]
            s[j] = cs[j] * s[j]
            its += 1
            j_done = j + 1
            hist.append(abs(s[j + 1]))
            if fixed_its is None and abs(s[j + 1]) <= rtol * beta0:
                break
        y = np.linalg.solve(np.triu(H[:j_done, :j_done]), s[:j_done])
        x = x + Z[:j_done].T @ y
        r = g - matvec(x)
        if fixed_its is None and np.linalg.norm(r) <= rtol * beta0:
            break
    return x, its, hist


def convergence_factor(d0, dN, its):
    """rho = exp((1/N_it) ln(||d_N|| / ||d_0||)) (Appendix B)."""
    if its <= 0:
        return 0.0
    return float(np.exp(np.log(dN / d0) / its))


def remove_mean_pressure(x, ne, nb, vol):
    """Remove the global constant-pressure component (null space of G on periodic meshes).

    The constant pressure p = 1 has mode-0 coefficients sqrt(|K|) in every element.
    """
    X = np.array(x, dtype=np.float64).reshape(ne, 4, nb)
    s = np.sqrt(np.asarray(vol, dtype=np.float64))
    alpha = np.dot(X[:, 3, 0], s) / np.dot(s, s)
    X[:, 3, 0] -= alpha * s
    return X.reshape(-1)


def implicit_stage(m, w, inv_gdt, levels, rtol=1e-8, restart=30, maxit=300, pre=2, post=2, coarse_sweeps=2,
                   omega=1.0):
    """One linearly implicit stage from the state w (Sec. 2.2 with one stage and gamma = 1):
    g = -f_h(w), G = dense assembled J(w) + M/(gamma dt), the inherited coarse operators and
    their element block inverses (Sec. 2.4), and FGMRES(restart) right-preconditioned by one
    MG_V cycle (Algorithm 2) per iteration to rtol. Dense: for meshes of a few thousand unknowns.
    Returns (w + dw, FGMRES iterations, true relative residual)."""
    import oracle as O
    g = -O.residual(m, w).reshape(-1)
    G0 = O.dense_G(m, w, inv_gdt)
    nbs = [O.nb(k) for k in levels]
    Gs = [G0] + [inherited_operator(G0, m.ne, m.nb, nb) for nb in nbs[1:]]
    lv = [Level(lambda v, G=G: G @ v, block_inverses(G, m.ne, nb), m.ne, nb) for G, nb in zip(Gs, nbs)]
    x, its, _ = fgmres(lambda v: G0 @ v,
                       lambda v: mg_v(lv, 0, v, np.zeros_like(v), pre, post, coarse_sweeps, omega),
                       g, restart=restart, maxit=maxit, rtol=rtol)
    relres = float(np.linalg.norm(g - G0 @ x) / np.linalg.norm(g))
    return np.asarray(w).reshape(-1) + x, its, relres
