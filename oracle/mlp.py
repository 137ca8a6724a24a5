"""FP64 reference of the learned coarse-level correction network (test infrastructure).

The network replaces the coarsest p-multigrid SOLVE by a per-element map from the
P1 coarse right-hand side of an element and of its 6 face neighbours (7 x 16 =
112 values) to the element's 16 P1 correction coefficients:
    z1 = W1 x + b1, h1 = gelu(z1), z2 = W2 h1 + b2, h2 = gelu(z2), y = W3 h2 + b3,
gelu(t) = t/2 (1 + erf(t / sqrt 2)). The features are divided by their Euclidean
norm s and the output multiplied by s, which makes the map homogeneous of degree
one like the linear coarse problem it approximates. Loss: mean over the batch of
the squared error summed over the 16 outputs.

Plain numpy FP64; only the tests use it (against the GPU kernels' gradients).
"""
import math

import numpy as np
from scipy.special import erf

N_IN, N_HID, N_OUT = 112, 128, 16
SHAPES = [("W1", (N_HID, N_IN)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
          ("W3", (N_OUT, N_HID)), ("b3", (N_OUT,))]


def n_params():
    return sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta):
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = np.asarray(theta[o:o + n], dtype=np.float64).reshape(shp)
        o += n
    return out


def pack(p):
    return np.concatenate([np.asarray(p[name], dtype=np.float64).reshape(-1) for name, _ in SHAPES])


def gelu(t):
    return 0.5 * t * (1.0 + erf(t / math.sqrt(2.0)))


def gelu_prime(t):
    return 0.5 * (1.0 + erf(t / math.sqrt(2.0))) + t * np.exp(-0.5 * t * t) / math.sqrt(2.0 * math.pi)


def forward(theta, X):
    """X: [B, 112] -> (y [B, 16], cache)."""
    p = unpack(theta)
    z1 = X @ p["W1"].T + p["b1"]
    h1 = gelu(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = gelu(z2)
    y = h2 @ p["W3"].T + p["b3"]
    return y, (X, z1, h1, z2, h2)


def loss_and_grad(theta, X, T):
    """Mean squared error (summed over outputs, averaged over samples) and its gradient."""
    p = unpack(theta)
    y, (X, z1, h1, z2, h2) = forward(theta, X)
    B = X.shape[0]
    r = y - T
    loss = float(np.sum(r * r) / B)
    dy = 2.0 * r / B
    g = {"W3": dy.T @ h2, "b3": dy.sum(0)}
    dz2 = (dy @ p["W3"]) * gelu_prime(z2)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ p["W2"]) * gelu_prime(z1)
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(0)
    return loss, pack(g)


def bf16_round(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    a32 = np.ascontiguousarray(a, dtype=np.float32)
    u = a32.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def features(dL, nbr, nb1):
    """Per-element features: the element's and its 6 neighbours' P1 coefficients (4 variables x nb1),
    divided by their norm. dL: [ne, 4, nb1]; nbr: [ne, 6]. Returns (X [ne, 7*4*nb1], s [ne])."""
    D = np.asarray(dL).reshape(-1, 4 * nb1)
    # a missing neighbour (index -1, across a wall) contributes zeros
    F = np.concatenate([D] + [np.where((nbr[:, f] >= 0)[:, None], D[nbr[:, f]], 0.0) for f in range(6)], axis=1)
    s = np.linalg.norm(F, axis=1)
    s = np.where(s > 0.0, s, 1.0)
    return F / s[:, None], s


def forward_bf16(theta, X):
    """The network with the operand rounding of a BF16 tensor-core evaluation: the weights and
    the input of every layer rounded to bfloat16, products accumulated exactly (here FP64),
    biases and activations kept wide. Returns y [B, 16]."""
    p = unpack(theta)
    W1, W2, W3 = (bf16_round(p[k]) for k in ("W1", "W2", "W3"))
    z1 = bf16_round(X) @ W1.T + p["b1"]
    z2 = bf16_round(gelu(z1)) @ W2.T + p["b2"]
    return bf16_round(gelu(z2)) @ W3.T + p["b3"]


def coarse_correction(theta, dL, nbr, nb1, bf16=True):
    """Learned coarse correction of a coarsest-level right-hand side dL [ne, 4, nb1]:
    x_e = s_e * net(X_e) with X_e the normalised features of the element and its face
    neighbours and s_e their norm (x_e = 0 where s_e = 0). Returns x [ne, 4, nb1]."""
    D = np.asarray(dL).reshape(-1, 4 * nb1)
    # a missing neighbour (index -1, across a wall) contributes zeros
    F = np.concatenate([D] + [np.where((nbr[:, f] >= 0)[:, None], D[nbr[:, f]], 0.0) for f in range(6)], axis=1)
    s = np.linalg.norm(F, axis=1)
    X = F / np.where(s > 0.0, s, 1.0)[:, None]
    y = forward_bf16(theta, X) if bf16 else forward(theta, X)[0]
    return (s[:, None] * y).reshape(np.shape(dL))
