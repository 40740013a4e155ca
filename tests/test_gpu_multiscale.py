"""Coarse-to-fine parity: the multiscale solve (clustering, coarse phase,
extrapolation, kernel truncation, block-sparse fine steps) reaches the same
fixed point as the plain single-scale definition (Section 2: truncation is an
acceleration, not an approximation of a different problem)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2107_02010_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = 1e-5
# GPU against GPU: each run is within TOL of the exact fixed point (the dense
# solve is parity-checked against the oracle), so two runs differ by <= 2 TOL
TOL2 = 2e-5


@pytest.fixture(scope="module")
def ctx():
    from paper_2107_02010_gb300 import otgb

    c = otgb.Context()
    yield c
    c.close()


def T(v):
    return torch.from_numpy(np.ascontiguousarray(v)).cuda()


def rel(got, want, eps):
    got = got.detach().cpu().numpy().astype(np.float64) if torch.is_tensor(got) else np.asarray(got, np.float64)
    return float(np.max(np.abs(got - want)) / (np.max(np.abs(want)) + eps))


# precision 0 (tensor-core exponent, float32 accuracy) and 2 (CUDA-core float32)
ENGINES = [0, 2]


@pytest.mark.parametrize("precision", ENGINES)
def test_multiscale_grid_matches_converged_oracle(ctx, precision):
    from paper_2107_02010_gb300 import otgb

    x, a, y, b = synth.density_maps(grid=24, n_tubes=6, n_keep=1500, seeds=(21, 22))
    blur, reach = 1.5, 4.0
    ref = oracle.sinkhorn(x, a, y, b, blur=blur, reach=reach, scaling=0.5, tol=1e-12, max_iters=5000)
    assert ref["converged"]
    p = otgb.default_params(blur=blur, reach=reach, scaling=0.5, multiscale=1, cluster=0, cell=4.0, tol=1e-8,
                            precision=precision)
    out = otgb.sinkhorn_divergence(ctx, T(x), T(a), T(y), T(b), p, want_self=True)
    st = out["stats"]
    print("stats", st)
    assert st["n_clusters_x"] > 1 and st["iters_coarse"] > 0
    eps = blur ** 2
    assert abs(out["S"] - ref["S"]) <= TOL * abs(ref["S"]), (out["S"], ref["S"])
    for k, key in (("f", "f"), ("g", "g"), ("a_self", "a"), ("b_self", "b")):
        assert rel(out[k], ref[key], eps) < TOL, (k, rel(out[k], ref[key], eps))


@pytest.mark.parametrize("precision", ENGINES)
@pytest.mark.parametrize("n_keep", [20_000])
def test_multiscale_grid_matches_dense_gpu(ctx, n_keep, precision):
    # larger problem: the dense GPU solve (itself parity-checked against the
    # oracle) is the reference; both run to a tight stopping rule
    from paper_2107_02010_gb300 import otgb

    x, a, y, b = synth.density_maps(grid=40, n_tubes=15, n_keep=n_keep, seeds=(31, 32))
    blur, reach = 1.0, 10.0
    common = dict(blur=blur, reach=reach, scaling=0.5, tol=1e-8, max_iters=20000, precision=precision)
    dense = otgb.sinkhorn_divergence(ctx, T(x), T(a), T(y), T(b), otgb.default_params(**common), want_self=True)
    ms = otgb.sinkhorn_divergence(ctx, T(x), T(a), T(y), T(b),
                                  otgb.default_params(multiscale=1, cluster=0, cell=4.0, **common), want_self=True)
    st = ms["stats"]
    print("dense", dense["stats"], "\nmultiscale", st)
    assert st["kept_fraction"] < 0.5
    eps = blur ** 2
    assert abs(ms["S"] - dense["S"]) <= TOL2 * abs(dense["S"]), (ms["S"], dense["S"])
    for k in ("f", "g", "a_self", "b_self"):
        assert rel(ms[k], dense[k].cpu().numpy().astype(np.float64), eps) < TOL2, k


def test_multiscale_kmeans_fibers_matches_dense_gpu(ctx):
    from paper_2107_02010_gb300 import otgb

    ctrl = synth.bundle_centrelines()
    x, a, _ = synth.fiber_bundles(3000, seed=4, ctrl=ctrl, perturb=3.0)
    y, b, _ = synth.fiber_bundles(2500, seed=5, ctrl=ctrl)
    blur, reach = 2.0, 20.0
    # both polished (params.polish): the duals then meet the float32 bar
    common = dict(blur=blur, reach=reach, scaling=0.5, tol=1e-8, max_iters=20000, polish=1)
    dense = otgb.sinkhorn_divergence(ctx, T(x), T(a), T(y), T(b), otgb.default_params(**common), want_self=True)
    ms = otgb.sinkhorn_divergence(ctx, T(x), T(a), T(y), T(b),
                                  otgb.default_params(multiscale=1, cluster=1, k_clusters=40, kmeans_iters=10,
                                                      **common), want_self=True)
    print("dense", dense["stats"], "\nmultiscale", ms["stats"])
    eps = blur ** 2
    assert abs(ms["S"] - dense["S"]) <= TOL2 * abs(dense["S"]), (ms["S"], dense["S"])
    for k in ("f", "g", "a_self", "b_self"):
        err = rel(ms[k], dense[k].cpu().numpy().astype(np.float64), eps)
        print(k, err)
        assert err < TOL2, k
