"""FP64 oracle of the warm-start network (not part of the paper: an addition
that learns the subject-side dual f(x) of a fixed atlas from potentials the
solver produced, used only to initialise the solve at the finest scale).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Network: f(x) = out_mean + out_scale * (W4 s(W3 s(W2 s(W1 u + b1) + b2) + b3) + b4),
u = (x - in_mean) / in_scale, s(z) = z * sigmoid(z) (SiLU), layers
D -> H -> H -> H -> 1.  Loss: L = (1/2n) sum_i (f(x_i) - y_i)^2 / out_scale^2
(the mean squared error in normalised units).  Parameters are one flat vector
in the order W1, b1, W2, b2, W3, b3, W4, b4 (row-major W, rows = outputs).
Plain numpy in double precision; gradients by the chain rule, pinned against
central finite differences in the tests.
"""
from __future__ import annotations

import numpy as np


def shapes(D: int, H: int):
    return [(H, D), (H,), (H, H), (H,), (H, H), (H,), (1, H), (1,)]


def unflatten(theta, D, H):
    out, k = [], 0
    for s in shapes(D, H):
        n = int(np.prod(s))
        out.append(np.asarray(theta[k:k + n], np.float64).reshape(s))
        k += n
    return out


def n_params(D, H):
    return sum(int(np.prod(s)) for s in shapes(D, H))


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(theta, x, D, H, norm):
    """Returns (prediction in data units, cache)."""
    W1, b1, W2, b2, W3, b3, W4, b4 = unflatten(theta, D, H)
    in_mean, in_scale, out_mean, out_scale = norm
    u = (np.asarray(x, np.float64) - in_mean) / in_scale
    z1 = u @ W1.T + b1
    a1 = silu(z1)
    z2 = a1 @ W2.T + b2
    a2 = silu(z2)
    z3 = a2 @ W3.T + b3
    a3 = silu(z3)
    o = (a3 @ W4.T + b4)[:, 0]
    return out_mean + out_scale * o, (u, z1, a1, z2, a2, z3, a3, o)


def loss_and_grad(theta, x, y, D, H, norm):
    """L = (1/2n) sum ((o - (y - out_mean)/out_scale))^2 and dL/dtheta (flat)."""
    W1, b1, W2, b2, W3, b3, W4, b4 = unflatten(theta, D, H)
    _, (u, z1, a1, z2, a2, z3, a3, o) = forward(theta, x, D, H, norm)
    n = u.shape[0]
    t = (np.asarray(y, np.float64) - norm[2]) / norm[3]
    r = o - t
    L = 0.5 * float(np.mean(r * r))
    do = r / n                                 # dL/do
    gW4 = do[None, :] @ a3                     # (1, H)
    gb4 = np.array([do.sum()])
    da3 = do[:, None] @ W4                     # (n, H)
    dz3 = da3 * dsilu(z3)
    gW3 = dz3.T @ a2
    gb3 = dz3.sum(0)
    dz2 = (dz3 @ W3) * dsilu(z2)
    gW2 = dz2.T @ a1
    gb2 = dz2.sum(0)
    dz1 = (dz2 @ W2) * dsilu(z1)
    gW1 = dz1.T @ u
    gb1 = dz1.sum(0)
    g = np.concatenate([v.ravel() for v in (gW1, gb1, gW2, gb2, gW3, gb3, gW4, gb4)])
    return L, g


def init_params(D, H, seed):
    """He-style uniform initialisation (only used by tests that need a point)."""
    r = np.random.default_rng(seed)
    parts = []
    for s in shapes(D, H):
        if len(s) == 2:
            lim = np.sqrt(3.0 / s[1])
            parts.append(r.uniform(-lim, lim, size=s).ravel())
        else:
            parts.append(np.zeros(s))
    return np.concatenate(parts)


def adam_step(theta, m, v, g, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1) in double precision.

    t is the 1-based index of this update.  Returns (theta, m, v) new arrays.
    """
    g = np.asarray(g, np.float64)
    m = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return np.asarray(theta, np.float64) - lr * mh / (np.sqrt(vh) + eps), m, v
