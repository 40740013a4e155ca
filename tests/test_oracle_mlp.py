"""Pins of the FP64 warm-start network oracle (oracle/mlp.py) against things
other than itself: central finite differences of the loss, closed forms of the
activation, a hand-built network, and the constant-gradient behaviour of Adam.
CPU only."""
import numpy as np
import pytest

from oracle import mlp as om


def _problem(D, H, n, seed):
    r = np.random.default_rng(seed)
    theta = om.init_params(D, H, seed)
    # non-zero biases so that every bias gradient is exercised
    k = 0
    for s in om.shapes(D, H):
        sz = int(np.prod(s))
        if len(s) == 1:
            theta[k:k + sz] = r.normal(0, 0.3, sz)
        k += sz
    x = r.normal(1.5, 2.0, (n, D))
    y = r.normal(-3.0, 5.0, n)
    norm = (r.normal(1.5, 0.1, D), r.uniform(1.5, 2.5, D), -2.5, 4.0)
    return theta, x, y, norm


def test_silu_closed_forms():
    z = np.array([0.0, 1.0, -1.0, 30.0, -30.0])
    s = om.silu(z)
    assert s[0] == 0.0
    assert abs(s[1] - 1.0 / (1.0 + np.exp(-1.0))) < 1e-15
    assert abs(s[1] - s[2] - 1.0) < 1e-15          # silu(z) - silu(-z) = z
    assert abs(s[3] - 30.0) < 1e-9 and abs(s[4]) < 1e-9
    # derivative against a central difference
    zz = np.linspace(-6, 6, 25)
    h = 1e-6
    fd = (om.silu(zz + h) - om.silu(zz - h)) / (2 * h)
    assert np.max(np.abs(fd - om.dsilu(zz))) < 1e-8


def test_hand_built_network():
    # one active unit per layer: f = out_mean + out_scale * (w4 * s(w3 * s(w2 * s(w1 * u + b1) + b2) + b3) + b4)
    D, H = 3, 4
    theta = np.zeros(om.n_params(D, H))
    parts = [np.zeros(s) for s in om.shapes(D, H)]
    parts[0][0, 1] = 2.0      # W1: unit 0 reads u_1
    parts[1][0] = 0.5
    parts[2][0, 0] = -1.5     # W2
    parts[3][0] = 0.25
    parts[4][0, 0] = 0.75     # W3
    parts[5][0] = -0.1
    parts[6][0, 0] = 3.0      # W4
    parts[7][0] = 0.2
    theta = np.concatenate([p.ravel() for p in parts])
    x = np.array([[7.0, 2.0, -1.0]])
    norm = (np.array([0.0, 1.0, 0.0]), np.array([1.0, 0.5, 1.0]), 10.0, 2.0)
    u1 = (2.0 - 1.0) / 0.5
    sil = lambda z: z / (1 + np.exp(-z))
    h1 = sil(2.0 * u1 + 0.5)
    h2 = sil(-1.5 * h1 + 0.25)
    h3 = sil(0.75 * h2 - 0.1)
    # units 1..3 of every layer are silu(0) = 0 and carry nothing
    expect = 10.0 + 2.0 * (3.0 * h3 + 0.2)
    pred, _ = om.forward(theta, x, D, H, norm)
    assert abs(pred[0] - expect) < 1e-12


@pytest.mark.parametrize("D,H,n", [(5, 8, 7), (60, 32, 5)])
def test_gradient_matches_central_differences(D, H, n):
    theta, x, y, norm = _problem(D, H, n, seed=D + H)
    L, g = om.loss_and_grad(theta, x, y, D, H, norm)
    assert np.isfinite(L) and L > 0
    r = np.random.default_rng(7)
    idx = r.choice(theta.size, size=min(theta.size, 200), replace=False)
    # every block contributes at least one coordinate
    starts = np.cumsum([0] + [int(np.prod(s)) for s in om.shapes(D, H)])
    idx = np.unique(np.concatenate([idx, starts[:-1], starts[1:] - 1]))
    h = 1e-5
    for k in idx:
        tp = theta.copy(); tp[k] += h
        tm = theta.copy(); tm[k] -= h
        fd = (om.loss_and_grad(tp, x, y, D, H, norm)[0] - om.loss_and_grad(tm, x, y, D, H, norm)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(g[k])) + 1e-9, (k, fd, g[k])


def test_loss_is_half_mean_square_in_normalised_units():
    D, H, n = 4, 8, 9
    theta, x, y, norm = _problem(D, H, n, seed=3)
    pred, _ = om.forward(theta, x, D, H, norm)
    L, _ = om.loss_and_grad(theta, x, y, D, H, norm)
    assert abs(L - 0.5 * np.mean(((pred - y) / norm[3]) ** 2)) < 1e-12


def test_adam_constant_gradient_moves_linearly():
    # with a constant gradient the bias-corrected moments are exactly g and g^2,
    # so every step moves each coordinate by lr * g / (|g| + eps)
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    theta = np.array([1.0, 2.0, 3.0, 4.0])
    m = np.zeros(4)
    v = np.zeros(4)
    lr, eps = 1e-2, 1e-8
    for t in range(1, 6):
        theta, m, v = om.adam_step(theta, m, v, g, t, lr, eps=eps)
        expect = np.array([1.0, 2.0, 3.0, 4.0]) - t * lr * g / (np.abs(g) + eps)
        assert np.max(np.abs(theta - expect)) < 1e-12


def test_adam_first_moment_decay():
    # gradient g then 0: m_2 = beta1 (1 - beta1) g, corrected by 1 - beta1^2
    g = np.array([1.0])
    th, m, v = om.adam_step(np.zeros(1), np.zeros(1), np.zeros(1), g, 1, 1.0, eps=0.0)
    th2, m2, v2 = om.adam_step(th, m, v, np.zeros(1), 2, 1.0, eps=0.0)
    mh = 0.9 * 0.1 / (1 - 0.81)
    vh = 0.999 * 0.001 / (1 - 0.999 ** 2)
    assert abs((th - th2)[0] - mh / np.sqrt(vh)) < 1e-12
