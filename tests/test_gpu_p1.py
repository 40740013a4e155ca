"""The cost C(x, y) = |x - y| (p = 1 in the cost |x - y|^p / p of Section 2;
eps = blur, rho = reach): dense and coarse-to-fine solves against the
converged FP64 oracle at 1e-5 (S and the four duals), in 3-D and in 60-D,
and the gradient in the points (x - y) / |x - y| against oracle.grad_x."""
import numpy as np
import pytest
import torch

import oracle
from paper_2107_02010_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = 1e-5


def T(v):
    return torch.from_numpy(np.ascontiguousarray(v, dtype=np.float32)).cuda()


@pytest.fixture(scope="module")
def ctx():
    from paper_2107_02010_gb300 import otgb

    c = otgb.Context()
    yield c
    c.close()


def _check(out, ref, eps, a=None, b=None):
    """S and the four duals within TOL; balanced problems (a, b given) compare
    (f, g) in the gauge <a, f> = <b, g>, since (f + c, g - c) is also a fixed
    point there."""
    assert abs(out["S"] - ref["S"]) <= TOL * abs(ref["S"]), (out["S"], ref["S"])
    got = {k: out[k].cpu().numpy().astype(np.float64) for k in ("f", "g", "a_self", "b_self")}
    want = {"f": ref["f"], "g": ref["g"], "a_self": ref["a"], "b_self": ref["b"]}
    if a is not None:
        for d in (got, want):
            c = (np.dot(a, d["f"]) - np.dot(b, d["g"])) / (a.sum() + b.sum())
            d["f"], d["g"] = d["f"] - c, d["g"] + c
    for k in ("f", "g", "a_self", "b_self"):
        err = np.max(np.abs(got[k] - want[k])) / (np.max(np.abs(want[k])) + eps)
        assert err < TOL, (k, err)


@pytest.mark.parametrize("reach", [0.0, 0.5])
def test_p1_dense_3d_matches_oracle(ctx, reach):
    from paper_2107_02010_gb300 import otgb

    x, a, y, b = synth.rotated_cloud(400, 400, seed=11)
    blur = 0.05
    ref = oracle.sinkhorn(x, a, y, b, blur=blur, reach=reach, scaling=0.5, p=1, tol=1e-12, max_iters=100000)
    assert ref["converged"]
    p = otgb.default_params(p=1, blur=blur, reach=reach, scaling=0.5, tol=1e-10, max_iters=20000)
    out = otgb.sinkhorn_divergence(ctx, T(x), T(a), T(y), T(b), p, want_self=True)
    _check(out, ref, blur, *((a.astype(np.float64), b.astype(np.float64)) if reach == 0.0 else ()))


def test_p1_multiscale_grid_matches_oracle(ctx):
    from paper_2107_02010_gb300 import otgb

    # the kernel of |x - y| decays slowly: at eps = 0.5 the truncation drops
    # pairs more than about 14 voxels apart
    x, a, y, b = synth.density_maps(grid=24, n_tubes=6, n_keep=1500, seeds=(21, 22))
    blur, reach = 0.5, 6.0
    ref = oracle.sinkhorn(x, a, y, b, blur=blur, reach=reach, scaling=0.5, p=1, tol=1e-12, max_iters=100000)
    assert ref["converged"]
    p = otgb.default_params(p=1, blur=blur, reach=reach, scaling=0.5, multiscale=1, cluster=0, cell=4.0,
                            tol=1e-10, max_iters=20000)
    out = otgb.sinkhorn_divergence(ctx, T(x), T(a), T(y), T(b), p, want_self=True)
    assert out["stats"]["iters_coarse"] > 0 and out["stats"]["kept_fraction"] < 1.0
    _check(out, ref, blur)


def test_p1_multiscale_kmeans_fibers_matches_oracle(ctx):
    from paper_2107_02010_gb300 import otgb

    ctrl = synth.bundle_centrelines()
    x, a, _ = synth.fiber_bundles(600, seed=24, ctrl=ctrl, perturb=3.0)
    y, b, _ = synth.fiber_bundles(500, seed=25, ctrl=ctrl)
    blur, reach = 2.0, 20.0
    ref = oracle.sinkhorn(x, a, y, b, blur=blur, reach=reach, scaling=0.5, p=1, tol=1e-12, max_iters=100000)
    assert ref["converged"]
    p = otgb.default_params(p=1, blur=blur, reach=reach, scaling=0.5, multiscale=1, cluster=1, k_clusters=20,
                            tol=1e-10, max_iters=20000)
    out = otgb.sinkhorn_divergence(ctx, T(x), T(a), T(y), T(b), p, want_self=True)
    _check(out, ref, blur)


def test_p1_gradient_matches_oracle(ctx):
    from paper_2107_02010_gb300 import otgb

    x, a, y, b = synth.rotated_cloud(256, 256, seed=12)
    blur, reach = 0.05, 0.5
    r = oracle.sinkhorn(x, a, y, b, blur=blur, reach=reach, scaling=0.5, p=1, tol=1e-12, max_iters=100000)
    assert r["converged"]
    want = oracle.grad_x(x, a, y, b, blur, r["a"], r["f"], r["g"], p=1)
    got = otgb.sinkhorn_grad_x(ctx, T(x), T(a), T(y), T(b), blur, T(r["f"]), T(r["g"]), T(r["a"]), p=1)
    err = np.max(np.abs(got.cpu().numpy() - want)) / np.max(np.abs(want))
    assert err < TOL, err


def test_p1_rejects_tensor_core_precision_and_label_transfer(ctx):
    from paper_2107_02010_gb300 import otgb

    ctrl = synth.bundle_centrelines()
    x, a, lab = synth.fiber_bundles(300, seed=26, ctrl=ctrl)
    X, A = T(x), T(a)
    p = otgb.default_params(p=1, blur=2.0, reach=20.0, precision=1)
    with pytest.raises(otgb.OtgbError) as e:
        otgb.sinkhorn_divergence(ctx, X, A, X, A, p)
    assert e.value.code == -1
    p = otgb.default_params(p=1, blur=2.0, reach=20.0)
    out = otgb.sinkhorn_divergence(ctx, X, A, X, A, p, want_plan=True)
    with pytest.raises(otgb.OtgbError) as e:
        otgb.transport_apply(ctx, out["plan"], out["f"], out["g"], torch.from_numpy(lab).cuda(), 20)
    assert e.value.code == -1
