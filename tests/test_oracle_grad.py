"""The oracle's gradient of the debiased divergence in the points (Section 2:
the gradients of S are expressions of the four dual vectors; they drive the
barycenter of the track-density atlas).  Pinned by central finite differences
of the oracle's own converged S (balanced and unbalanced, in x and in y), by
translation invariance (moving both clouds together leaves S unchanged, so the
two gradients sum to zero) and by the shift identity S(alpha, alpha + t) =
|t|^2 / 2, whose derivative in t is t."""
import numpy as np
import pytest

import oracle


def _on_grid(rng, n, D):
    # multiples of 2^-8, so that x +- 2^-8 is exact in float32
    return (rng.integers(0, 256, size=(n, D)) / 256.0).astype(np.float32)


def _solve(x, a, y, b, blur, reach):
    r = oracle.sinkhorn(x, a, y, b, blur, reach, scaling=0.5)
    assert r["converged"]
    return r


@pytest.mark.parametrize("reach", [0.0, 0.7])
def test_gradient_in_the_points_matches_finite_differences(reach):
    rng = np.random.default_rng(3)
    N, M, D = 9, 7, 2
    x, y = _on_grid(rng, N, D), _on_grid(rng, M, D)
    # weights k / 64 with the k summing to 64: both masses exactly 1 in float32 (balanced OT needs equal masses)
    def weights(n):
        k = np.ones(n, np.int64) + np.bincount(rng.integers(0, n, 64 - n), minlength=n)
        return (k / 64.0).astype(np.float32)

    a, b = weights(N), weights(M)
    if reach > 0.0:
        b = (b * 1.25).astype(np.float32)
    blur = 0.25
    eps = blur ** 2
    r = _solve(x, a, y, b, blur, reach)
    gx = oracle.grad_x(x, a, y, b, eps, r["a"], r["f"], r["g"])
    gy = oracle.grad_x(y, b, x, a, eps, r["b"], r["g"], r["f"])
    scale = max(np.abs(gx).max(), np.abs(gy).max())
    h = 2.0 ** -8
    for side, g in (("x", gx), ("y", gy)):
        pts = x if side == "x" else y
        for i, d in ((0, 0), (3, 1), (6, 0)):
            p_, m_ = pts.copy(), pts.copy()
            p_[i, d] += h
            m_[i, d] -= h
            Sp = _solve(p_, a, y, b, blur, reach)["S"] if side == "x" else _solve(x, a, p_, b, blur, reach)["S"]
            Sm = _solve(m_, a, y, b, blur, reach)["S"] if side == "x" else _solve(x, a, m_, b, blur, reach)["S"]
            # Richardson: central differences at h and h/2 (points on multiples of 2^-8 stay exact in float32)
            p2, m2 = pts.copy(), pts.copy()
            p2[i, d] += h / 2
            m2[i, d] -= h / 2
            Sp2 = _solve(p2, a, y, b, blur, reach)["S"] if side == "x" else _solve(x, a, p2, b, blur, reach)["S"]
            Sm2 = _solve(m2, a, y, b, blur, reach)["S"] if side == "x" else _solve(x, a, m2, b, blur, reach)["S"]
            fd = (4.0 * (Sp2 - Sm2) / h - (Sp - Sm) / (2 * h)) / 3.0
            assert abs(fd - g[i, d]) <= 1e-6 * scale, (side, i, d, fd, g[i, d])
    # translation invariance
    assert np.allclose(gx.sum(0) + gy.sum(0), 0.0, atol=1e-10 * scale)


def test_gradient_of_the_shift_identity():
    rng = np.random.default_rng(4)
    N, D = 12, 3
    x = _on_grid(rng, N, D)
    a = np.full(N, 1.0 / N, np.float32)
    t = np.array([0.25, -0.125, 0.0625], np.float32)
    y = x + t
    blur = 0.2
    r = _solve(x, a, y, a, blur, 0.0)
    assert r["S"] == pytest.approx(0.5 * float(t.astype(np.float64) @ t), rel=1e-7)
    gx = oracle.grad_x(x, a, y, a, blur ** 2, r["a"], r["f"], r["g"])
    gy = oracle.grad_x(y, a, x, a, blur ** 2, r["b"], r["g"], r["f"])
    assert np.allclose(gy.sum(0), t, atol=1e-7)
    assert np.allclose(gx.sum(0), -t, atol=1e-7)
