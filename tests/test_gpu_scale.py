"""The scale workload: 60-D fiber bundles with N = M = 1,000,000 per side,
multiscale with k-means of 1000 clusters per side, coarse-plan truncation,
eps annealed 0.5 per step to blur = 2 mm, reach = 20 mm; FP32 and tensor-core
forms, FP64 final sums.

Checked on outputs the FP64 oracle computes one by one: sampled rows of the
converged duals against the dense softmin over all 1M columns (the fixed-point
identity, up to the last step size), S against the oracle's FP64 sums of the
GPU's duals, the tensor-core form against the FP32 form (1e-3 relative, the
reduced-precision bar), and transferred labels (Eq. (7), dense over all 1M
atlas fibers) on sampled rows against the oracle's scores: identical argmax
wherever the top class is clear."""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu

N = 1_000_000
BLUR, REACH, L = 2.0, 20.0, 20


def _solve(otgb, ctx, X, A, Y, B, precision):
    p = otgb.default_params(blur=BLUR, reach=REACH, scaling=0.5, multiscale=1, cluster=1, k_clusters=1000,
                            kmeans_iters=10, tol=1e-6, max_iters=3000, precision=precision)
    return otgb.sinkhorn_divergence(ctx, X, A, Y, B, p, want_self=True, want_plan=True)


@pytest.fixture(scope="module")
def scale():
    from paper_2107_02010_gb300 import otgb, synth
    oracle.build()
    ctx = otgb.Context()
    ctrl = synth.bundle_centrelines()
    x, a, _ = synth.fiber_bundles(N, seed=4, ctrl=ctrl, perturb=3.0)
    y, b, lab = synth.fiber_bundles(N, seed=5, ctrl=ctrl)
    X, A, Y, B = (torch.from_numpy(v).cuda() for v in (x, a, y, b))
    fp32 = _solve(otgb, ctx, X, A, Y, B, 0)
    tc = _solve(otgb, ctx, X, A, Y, B, 1)
    return dict(otgb=otgb, ctx=ctx, x=x, a=a, y=y, b=b, lab=lab, Y=Y, B=B, fp32=fp32, tc=tc)


def test_scale_solves_converge(scale):
    for key in ("fp32", "tc"):
        r = scale[key]
        assert r["status"] == 0, key
        st = r["stats"]
        print("\n%s: S %.10f, %d steps, %.1f ms, kept %.4f, pairs %.3e" % (
            key, r["S"], st["iters_total"], st["total_ms"], st["kept_fraction"], st["pairs_evaluated"]))


def test_scale_sampled_rows_are_dense_fixed_points(scale):
    x, a, y, b = scale["x"], scale["a"], scale["y"], scale["b"]
    r = scale["fp32"]
    f = r["f"].cpu().numpy().astype(np.float64)
    g = r["g"].cpu().numpy().astype(np.float64)
    eps = BLUR ** 2
    lam = oracle.lam(BLUR, REACH)
    delta = r["stats"]["last_delta"]
    rng = np.random.default_rng(7)
    ix = np.sort(rng.choice(N, 96, replace=False))
    iy = np.sort(rng.choice(N, 96, replace=False))
    for name, q, pts, w, pot, got in (("f", x[ix], y, b, g, f[ix]), ("g", y[iy], x, a, f, g[iy])):
        ref = oracle.softmin(q, pts, w, pot, eps, lam)
        bound = 3.0 * delta * eps + 2e-5 * (np.abs(ref) + eps)
        err = np.abs(got - ref)
        assert np.all(err <= bound), (name, float(err.max()))


def test_scale_divergence_fp64_sums_and_tensor_core_form(scale):
    a, b = scale["a"], scale["b"]
    eps = BLUR ** 2
    for key in ("fp32", "tc"):
        r = scale[key]
        d = [r[k].cpu().numpy().astype(np.float64) for k in ("a_self", "b_self", "f", "g")]
        S_ref = oracle.divergence(a, b, eps, oracle.rho(REACH), *d)
        assert abs(r["S"] - S_ref) <= 1e-9 * abs(S_ref), key
    S32, Stc = scale["fp32"]["S"], scale["tc"]["S"]
    assert abs(Stc - S32) <= 1e-3 * abs(S32), (Stc, S32)


def test_scale_label_transfer_sampled_rows(scale):
    otgb, ctx = scale["otgb"], scale["ctx"]
    x, y, b, lab = scale["x"], scale["y"], scale["b"], scale["lab"]
    r = scale["fp32"]
    _, am, _ = otgb.transport_apply(ctx, r["plan"], r["f"], r["g"], torch.from_numpy(lab).cuda(), L,
                                    want_scores=False)
    am = am.cpu().numpy()
    f = r["f"].cpu().numpy().astype(np.float64)
    g = r["g"].cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(8)
    ix = np.sort(rng.choice(N, 128, replace=False))
    rsc, ram, _ = oracle.transport_apply(x[ix], y, b, BLUR ** 2, f[ix], g, lab, L)
    top2 = np.sort(rsc, axis=1)[:, -2:]
    clear = top2[:, 1] - top2[:, 0] >= 1e-4 * top2[:, 1]
    assert clear.sum() >= 0.9 * len(ix)
    assert np.all(am[ix][clear] == ram[clear])
    # the tensor-core form transfers the same labels on the clear rows
    rt = scale["tc"]
    _, amt, _ = otgb.transport_apply(ctx, rt["plan"], rt["f"], rt["g"], torch.from_numpy(lab).cuda(), L,
                                     want_scores=False)
    assert np.all(amt.cpu().numpy()[ix][clear] == ram[clear])
