"""The tensor-core form (tcgen05 BF16 hi/lo cross term, FP32 accumulation and
log-sum-exp) against the FP64 oracle, to the reduced-precision bar of 1e-3
relative on S and the duals, with identical transferred labels on rows whose
top class is clear."""
import numpy as np
import pytest
import torch

import oracle
from paper_2107_02010_gb300 import synth

pytestmark = pytest.mark.gpu
TOL_TC = 1e-3


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


def test_tensorcore_fixed_steps_match_oracle(ctx):
    from paper_2107_02010_gb300 import otgb

    ctrl = synth.bundle_centrelines()
    x, a, _ = synth.fiber_bundles(700, seed=4, ctrl=ctrl, perturb=3.0)
    y, b, _ = synth.fiber_bundles(650, seed=5, ctrl=ctrl)
    blur, reach, q, extra = 2.0, 20.0, 0.5, 8
    d = oracle.diameter(x, y)
    n_sched = len(oracle.schedule(d, blur, q))
    p = otgb.default_params(blur=blur, reach=reach, scaling=q, diameter=d, fixed_iters=extra, translation=0,
                            anderson=0, precision=1)
    out = otgb.sinkhorn_divergence(ctx, T(x), T(a), T(y), T(b), p, want_self=True)
    ref = oracle.sinkhorn(x, a, y, b, blur=blur, reach=reach, scaling=q, diameter=d, tol=0.0,
                          max_iters=n_sched + extra)
    eps = blur ** 2
    errs = {k: rel(out[k], ref[key], eps) for k, key in (("f", "f"), ("g", "g"), ("a_self", "a"), ("b_self", "b"))}
    print("tensor-core errors", errs, "S", out["S"], ref["S"])
    for k, v in errs.items():
        assert v < TOL_TC, (k, errs)
    assert abs(out["S"] - ref["S"]) <= TOL_TC * abs(ref["S"])


def test_tensorcore_converged_labels(ctx):
    from paper_2107_02010_gb300 import otgb

    ctrl = synth.bundle_centrelines()
    x, a, _ = synth.fiber_bundles(900, seed=6, ctrl=ctrl, perturb=3.0)
    y, b, lab = synth.fiber_bundles(800, seed=7, ctrl=ctrl)
    blur, reach, L = 2.0, 20.0, 20
    fp32 = otgb.sinkhorn_divergence(ctx, T(x), T(a), T(y), T(b), otgb.default_params(blur=blur, reach=reach,
                                                                                     tol=1e-7))
    tc = otgb.sinkhorn_divergence(ctx, T(x), T(a), T(y), T(b),
                                  otgb.default_params(blur=blur, reach=reach, tol=1e-7, precision=1), want_plan=True)
    print("fp32", fp32["stats"], "\ntc", tc["stats"])
    assert abs(tc["S"] - fp32["S"]) <= TOL_TC * abs(fp32["S"])
    f64 = tc["f"].cpu().numpy().astype(np.float64)
    g64 = tc["g"].cpu().numpy().astype(np.float64)
    sc, am, rm = otgb.transport_apply(ctx, tc["plan"], tc["f"], tc["g"], T(lab), L)
    rsc, ram, rrm = oracle.transport_apply(x, y, b, blur ** 2, f64, g64, lab, L)
    top2 = np.sort(rsc, axis=1)[:, -2:]
    clear = top2[:, 1] - top2[:, 0] >= 1e-4 * top2[:, 1]
    assert np.all(am.cpu().numpy()[clear] == ram[clear])


@pytest.mark.parametrize("P", [20, 7])
def test_tensorcore_cluster_tiles_match_fp32_and_oracle_rows(ctx, P):
    """The cluster-tiled form of the coarse-to-fine solve (the column operand centred at its k-means
    cluster's centre, split once per solve, H_j refreshed every step; P = 20 gives D = 60, P = 7 gives
    D = 21, D4 = 24): S and the duals against the float32 solve of the same problem to the reduced-precision
    bar, sampled rows of the duals against the FP64 oracle's dense softmin (the fixed point, up to the last
    step and the truncation), S against the oracle's FP64 sums of the same duals."""
    from paper_2107_02010_gb300 import otgb

    ctrl = synth.bundle_centrelines(P=P)
    x, a, _ = synth.fiber_bundles(6000, seed=4, ctrl=ctrl, P=P, perturb=3.0)
    y, b, _ = synth.fiber_bundles(5000, seed=5, ctrl=ctrl, P=P)
    blur, reach = 2.0, 20.0
    common = dict(blur=blur, reach=reach, scaling=0.5, multiscale=1, cluster=1, k_clusters=30, kmeans_iters=10,
                  tol=1e-7, max_iters=20000)
    r32 = otgb.sinkhorn_divergence(ctx, T(x), T(a), T(y), T(b), otgb.default_params(precision=0, **common),
                                   want_self=True)
    rtc = otgb.sinkhorn_divergence(ctx, T(x), T(a), T(y), T(b), otgb.default_params(precision=1, **common),
                                   want_self=True)
    print("fp32", r32["stats"], "\ntc", rtc["stats"])
    assert rtc["status"] == 0 and rtc["stats"]["kept_fraction"] < 0.9
    eps = blur ** 2
    assert abs(rtc["S"] - r32["S"]) <= TOL_TC * abs(r32["S"]), (rtc["S"], r32["S"])
    for k in ("f", "g", "a_self", "b_self"):
        err = rel(rtc[k], r32[k].cpu().numpy().astype(np.float64), eps)
        print(k, err)
        assert err < TOL_TC, k
    d = [rtc[k].cpu().numpy().astype(np.float64) for k in ("a_self", "b_self", "f", "g")]
    S_ref = oracle.divergence(a, b, eps, oracle.rho(reach), *d)
    assert abs(rtc["S"] - S_ref) <= 1e-9 * abs(S_ref)
    f, g = d[2], d[3]
    lam = oracle.lam(blur, reach)
    delta = rtc["stats"]["last_delta"]
    rng = np.random.default_rng(9)
    ix = np.sort(rng.choice(len(x), 64, replace=False))
    iy = np.sort(rng.choice(len(y), 64, replace=False))
    for name, q, pts, w, pot, got in (("f", x[ix], y, b, g, f[ix]), ("g", y[iy], x, a, f, g[iy])):
        ref = oracle.softmin(q, pts, w, pot, eps, lam)
        err = np.abs(got - ref)
        assert np.all(err <= 3.0 * delta * eps + TOL_TC * (np.abs(ref) + eps)), (name, float(err.max()))
