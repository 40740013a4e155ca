"""Gradient of the debiased divergence in the points, and the free-support
barycenter (Section 2: "Unbiased Sinkhorn divergences" -- gradients of S are
expressions of the four duals -- and "Track density atlas").

* The kernel, on the oracle's own converged duals, against oracle.grad_x
  (dS/dx and, with the measures exchanged, dS/dy), at 1e-5 of the largest
  gradient entry, in 3-D and in 60-D, balanced and unbalanced.
* End to end from the GPU's converged duals (float32 duals carry ~1e-6 of
  error, which the exponentials amplify by |C|/eps), at 1e-4.
* One barycenter step on three small track-density maps equals the step the
  oracle takes from the same points (its solves and its gradient), single-scale
  and coarse-to-fine, and the objective decreases over the iterations.
* In 60-D (fiber bundles, k-means clusters), a barycenter step -- its gradient
  over the kept cluster pairs of the solve -- equals the step built from the
  every-pair gradient kernel on the same solve's duals."""
import numpy as np
import pytest
import torch

import oracle
from paper_2107_02010_gb300 import synth

pytestmark = pytest.mark.gpu


def T(v):
    return torch.from_numpy(np.ascontiguousarray(v, dtype=np.float32)).cuda()


@pytest.fixture(scope="module")
def ctx():
    from paper_2107_02010_gb300 import otgb

    c = otgb.Context()
    yield c
    c.close()


def _exact(w, units=1 << 20):
    """Weights of total mass exactly 1 in float32 and double alike (multiples of
    2^-20, largest remainders rounded up): balanced OT needs equal masses."""
    w = np.asarray(w, np.float64)
    q = w / w.sum() * units
    k = np.maximum(np.floor(q), 1).astype(np.int64)
    rest = units - k.sum()
    order = np.argsort(-(q - np.floor(q)))
    k[order[:rest]] += 1
    assert k.sum() == units
    return (k / units).astype(np.float32)


def _cases():
    x3, a3, y3, b3 = synth.rotated_cloud(256, 256, seed=5)
    ctrl = synth.bundle_centrelines()
    xf, af, _ = synth.fiber_bundles(256, seed=14, ctrl=ctrl, perturb=3.0)
    yf, bf, _ = synth.fiber_bundles(256, seed=15, ctrl=ctrl)
    return {"3d": (x3, a3, y3, b3, 0.1), "60d": (xf, af, yf, bf, 2.0)}


# balanced 60-D fibers (20 nearly separate bundles, no damping) converge too
# slowly for the plain FP64 loop; the 60-D case is unbalanced
@pytest.mark.parametrize("name,reach_mult", [("3d", 0.0), ("3d", 5.0), ("60d", 5.0)])
def test_gradient_kernel_matches_oracle_on_oracle_duals(ctx, name, reach_mult):
    from paper_2107_02010_gb300 import otgb

    x, a, y, b, blur = _cases()[name]  # uniform weights 1/256: equal masses, exactly
    if reach_mult > 0.0:
        b = (b * 1.2).astype(np.float32)
    reach = reach_mult * blur
    eps = blur ** 2
    r = oracle.sinkhorn(x, a, y, b, blur=blur, reach=reach, scaling=0.5, tol=1e-12, max_iters=100000)
    assert r["converged"]
    want_x = oracle.grad_x(x, a, y, b, eps, r["a"], r["f"], r["g"])
    want_y = oracle.grad_x(y, b, x, a, eps, r["b"], r["g"], r["f"])
    got_x = otgb.sinkhorn_grad_x(ctx, T(x), T(a), T(y), T(b), eps, T(r["f"]), T(r["g"]), T(r["a"]))
    got_y = otgb.sinkhorn_grad_x(ctx, T(y), T(b), T(x), T(a), eps, T(r["g"]), T(r["f"]), T(r["b"]))
    for got, want in ((got_x, want_x), (got_y, want_y)):
        got = got.cpu().numpy().astype(np.float64)
        err = np.max(np.abs(got - want)) / np.max(np.abs(want))
        assert err < 1e-5, (name, reach, err)


def test_gradient_from_gpu_duals(ctx):
    from paper_2107_02010_gb300 import otgb

    x, a, y, b, blur = _cases()["3d"]
    reach, eps = 0.5, blur ** 2
    p = otgb.default_params(blur=blur, reach=reach, tol=1e-10, max_iters=20000)
    out = otgb.sinkhorn_divergence(ctx, T(x), T(a), T(y), T(b), p, want_self=True)
    got = otgb.sinkhorn_grad_x(ctx, T(x), T(a), T(y), T(b), eps, out["f"], out["g"], out["a_self"])
    r = oracle.sinkhorn(x, a, y, b, blur=blur, reach=reach, scaling=0.5, tol=1e-12, max_iters=100000)
    want = oracle.grad_x(x, a, y, b, eps, r["a"], r["f"], r["g"])
    err = np.max(np.abs(got.cpu().numpy() - want)) / np.max(np.abs(want))
    assert err < 1e-4, err


def _maps(K=3, n_keep=256):
    ys, bs = [], []
    for k in range(K):
        y, b, _, _ = synth.density_maps(grid=16, n_tubes=3, n_keep=n_keep, seeds=(60 + k, 61 + k), masses=(1.0, 1.0))
        ys.append(y)
        bs.append(_exact(b))
    # initial support: the voxels of the first map shifted by a quarter voxel, uniform weights
    x0 = ys[0].copy() + 0.25
    a0 = _exact(np.ones(x0.shape[0]))
    return x0, a0, ys, bs


# the barycenter takes its gradients from inside each solve, over the pairs the solve kept: every pair for a
# single-scale solve, the kept grid-cell pairs for a coarse-to-fine one (each dropped term below e^-27.6 of its row)
@pytest.mark.parametrize("multiscale", [0, 1])
def test_barycenter_step_matches_oracle_step(ctx, multiscale):
    from paper_2107_02010_gb300 import otgb

    x0, a0, ys, bs = _maps()
    blur, lr = 1.0, 1.0
    eps = blur ** 2
    p = otgb.default_params(blur=blur, reach=0.0, tol=1e-10, max_iters=20000, multiscale=multiscale, cluster=0,
                            cell=4.0)
    X = T(x0)
    hist = otgb.sinkhorn_barycenter(ctx, X, T(a0), [T(y) for y in ys], [T(b) for b in bs], p, iters=1, lr=lr)
    G = np.zeros(x0.shape)
    S0 = 0.0
    for y, b in zip(ys, bs):
        r = oracle.sinkhorn(x0, a0, y, b, blur=blur, reach=0.0, scaling=0.5, tol=1e-12, max_iters=100000)
        assert r["converged"]
        S0 += r["S"] / len(ys)
        G += oracle.grad_x(x0, a0, y, b, eps, r["a"], r["f"], r["g"]) / len(ys)
    x1 = x0.astype(np.float64) - lr * G / a0[:, None].astype(np.float64)
    step = np.max(np.abs(x1 - x0))
    got = X.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - x1)) <= 1e-4 * step + 1e-6, (np.max(np.abs(got - x1)), step)
    assert abs(hist[0] - S0) <= 1e-5 * abs(S0)


def test_barycenter_objective_decreases(ctx):
    from paper_2107_02010_gb300 import otgb

    x0, a0, ys, bs = _maps()
    p = otgb.default_params(blur=1.0, reach=0.0, tol=1e-8, max_iters=20000)
    hist = otgb.sinkhorn_barycenter(ctx, T(x0), T(a0), [T(y) for y in ys], [T(b) for b in bs], p, iters=4, lr=1.0)
    print("objective", hist)
    assert all(h1 < h0 for h0, h1 in zip(hist, hist[1:])), hist


def test_barycenter_step_60d_kept_pairs_match_every_pair(ctx):
    from paper_2107_02010_gb300 import otgb

    ctrl = synth.bundle_centrelines()
    x, a, _ = synth.fiber_bundles(3000, seed=21, ctrl=ctrl, perturb=3.0)
    y, b, _ = synth.fiber_bundles(2500, seed=22, ctrl=ctrl)
    blur, reach = 2.0, 20.0
    p = otgb.default_params(blur=blur, reach=reach, scaling=0.5, multiscale=1, cluster=1, k_clusters=40,
                            kmeans_iters=10, tol=1e-8, max_iters=5000)
    X, A, Y, B = T(x), T(a), T(y), T(b)
    r = otgb.sinkhorn_divergence(ctx, X, A, Y, B, p, want_self=True)
    stats = r["stats"]
    assert stats["kept_fraction"] < 0.9, stats["kept_fraction"]  # the truncation drops pairs here
    G = otgb.sinkhorn_grad_x(ctx, X, A, Y, B, blur ** 2, r["f"], r["g"], r["a_self"])
    want = (X.double() - G.double() / A.double()[:, None])
    Xb = X.clone()
    otgb.sinkhorn_barycenter(ctx, Xb, A, [Y], [B], p, iters=1, lr=1.0)
    step = float((want - X.double()).abs().max())
    err = float((Xb.double() - want).abs().max())
    assert err <= 1e-4 * step + 1e-6, (err, step)
