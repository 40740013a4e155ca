"""GPU parity of the softmin kernels and of the dense (single-scale) solve
against the FP64 oracle, through the C ABI.

Tolerance (potentials): max |gpu - oracle| <= 1e-5 (max |oracle| + eps), the
FP32 bar; divergence: |S - S*| <= 1e-5 |S*| + 1e-9 eps (mass).  Sizes span
several row blocks and ragged tails."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2107_02010_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def ctx():
    from paper_2107_02010_gb300 import otgb

    c = otgb.Context()
    yield c
    c.close()


def T(v):
    return torch.from_numpy(np.ascontiguousarray(v)).cuda()


def pot_err(got, want, eps):
    got = got.detach().cpu().numpy().astype(np.float64) if torch.is_tensor(got) else got
    return float(np.max(np.abs(got - want)) / (np.max(np.abs(want)) + eps))


def gauge_fixed(f, g, a, b):
    """Balanced OT leaves (f + c, g - c) free; pick c with <alpha, f> = <beta, g>."""
    f = f.detach().cpu().numpy().astype(np.float64) if torch.is_tensor(f) else np.asarray(f, np.float64)
    g = g.detach().cpu().numpy().astype(np.float64) if torch.is_tensor(g) else np.asarray(g, np.float64)
    A, B = a.astype(np.float64), b.astype(np.float64)
    c = (A @ f - B @ g) / (A.sum() + B.sum())
    return f - c, g + c


def check_pots(out, ref, a, b, eps, reach, tol=TOL):
    f, g = out["f"], out["g"]
    rf, rg = ref["f"], ref["g"]
    if not (reach > 0):
        f, g = gauge_fixed(f, g, a, b)
        rf, rg = gauge_fixed(rf, rg, a, b)
    errs = {"f": pot_err(f, rf, eps), "g": pot_err(g, rg, eps)}
    if "a_self" in out:
        errs["a"] = pot_err(out["a_self"], ref["a"], eps)
        errs["b"] = pot_err(out["b_self"], ref["b"], eps)
    print("potential errors", errs)
    for k, v in errs.items():
        assert v < tol, (k, errs)


# ------------------------------------------------------------- softmin ---
@pytest.mark.parametrize("D", [1, 2, 3, 5, 60])
@pytest.mark.parametrize("n_out,n_in", [(1, 1), (7, 129), (333, 1000), (1300, 517)])
def test_softmin_matches_oracle(ctx, D, n_out, n_in):
    from paper_2107_02010_gb300 import otgb

    r = np.random.default_rng(1000 + D * 7 + n_out)
    q = r.uniform(0, 1, size=(n_out, D)).astype(np.float32)
    p = r.uniform(0, 1, size=(n_in, D)).astype(np.float32)
    w = r.uniform(0.2, 1.0, size=n_in).astype(np.float32)
    w /= w.sum()
    pot = (0.01 * r.normal(size=n_in)).astype(np.float32)
    for eps, lam in ((0.01 * D, 1.0), (0.002 * D, 0.9)):
        got = otgb.softmin(ctx, T(q), T(p), T(w), T(pot), eps, lam)
        want = oracle.softmin(q, p, w, pot.astype(np.float64), eps, lam)
        assert pot_err(got, want, eps) < TOL, (eps, pot_err(got, want, eps))


@pytest.mark.parametrize("n_out", [80_000, 200_000])
def test_softmin_packed_rows_sampled(ctx, n_out):
    # enough rows for 2 or 4 rows per thread (packed f32x2 path); sampled rows
    # are checked against the oracle one by one
    from paper_2107_02010_gb300 import otgb

    r = np.random.default_rng(n_out)
    q = r.uniform(0, 10, size=(n_out, 3)).astype(np.float32)
    p = r.uniform(0, 10, size=(3001, 3)).astype(np.float32)
    w = r.uniform(0.2, 1.0, size=3001).astype(np.float32)
    pot = (0.1 * r.normal(size=3001)).astype(np.float32)
    old = (0.1 * r.normal(size=n_out)).astype(np.float32)
    eps = 0.05
    got = otgb.softmin(ctx, T(q), T(p), T(w), T(pot), eps, 0.95, old=T(old), omega=0.5).cpu().numpy()
    idx = np.unique(np.concatenate([np.arange(0, 700), r.integers(0, n_out, 600), np.arange(n_out - 300, n_out)]))
    want = 0.5 * (old[idx].astype(np.float64) + oracle.softmin(q[idx], p, w, pot.astype(np.float64), eps, 0.95))
    assert pot_err(got[idx].astype(np.float64), want, eps) < TOL


def test_softmin_blend_and_zero_weights(ctx):
    from paper_2107_02010_gb300 import otgb

    r = np.random.default_rng(7)
    q = r.uniform(0, 1, size=(500, 3)).astype(np.float32)
    p = r.uniform(0, 1, size=(400, 3)).astype(np.float32)
    w = r.uniform(0.2, 1.0, size=400).astype(np.float32)
    w[::3] = 0.0
    pot = (0.01 * r.normal(size=400)).astype(np.float32)
    old = (0.01 * r.normal(size=500)).astype(np.float32)
    eps = 0.005
    got = otgb.softmin(ctx, T(q), T(p), T(w), T(pot), eps, 1.0, old=T(old), omega=0.5)
    want = 0.5 * (old.astype(np.float64) + oracle.softmin(q, p, w, pot.astype(np.float64), eps, 1.0))
    assert pot_err(got, want, eps) < TOL


def test_softmin_far_rows_take_the_safe_path(ctx):
    # rows far from every column have sums far below the CTA's offset and are
    # finished by the two-pass kernel: values must still match.
    from paper_2107_02010_gb300 import otgb

    r = np.random.default_rng(8)
    q = np.concatenate([r.uniform(0, 1, size=(200, 3)), r.uniform(40, 41, size=(56, 3))]).astype(np.float32)
    p = r.uniform(0, 1, size=(300, 3)).astype(np.float32)
    w = np.full(300, 1 / 300, np.float32)
    pot = np.zeros(300, np.float32)
    eps = 0.01
    got = otgb.softmin(ctx, T(q), T(p), T(w), T(pot), eps, 1.0)
    want = oracle.softmin(q, p, w, pot.astype(np.float64), eps, 1.0)
    assert pot_err(got, want, eps) < TOL


@pytest.mark.parametrize("D", [3, 60])
def test_softmin_rows_with_a_wrong_shift_take_the_safe_path(ctx, D):
    # With old values given, the one-pass kernels shift each row by its old value;
    # for rows 40 units away from every column an old value of 0 misses the
    # row's log-sum by far more than 60 binades, so those rows are recomputed by
    # the two-pass fallback (direct differences).  Every row must equal the
    # oracle's blended value.
    from paper_2107_02010_gb300 import otgb

    r = np.random.default_rng(11)
    q = np.concatenate([r.uniform(0, 1, size=(200, D)), r.uniform(40, 41, size=(56, D))]).astype(np.float32)
    p = r.uniform(0, 1, size=(300, D)).astype(np.float32)
    w = r.uniform(0.5, 1.5, size=300).astype(np.float32)
    w /= w.sum()
    pot = r.uniform(-0.1, 0.1, size=300).astype(np.float32)
    old = np.zeros(len(q), np.float32)
    eps = 0.05
    got = otgb.softmin(ctx, T(q), T(p), T(w), T(pot), eps, 1.0, old=T(old), omega=0.5)
    want = 0.5 * oracle.softmin(q, p, w, pot.astype(np.float64), eps, 1.0)
    assert pot_err(got, want, eps) < TOL


# -------------------------------------------------------- dense solve ---
def _run_pair(ctx, x, a, y, b, blur, reach, q, extra, precision=0):
    from paper_2107_02010_gb300 import otgb

    d = oracle.diameter(x, y)
    n_sched = len(oracle.schedule(d, blur, q))
    # the paper's loop step for step (no translation step), as the oracle runs it
    p = otgb.default_params(blur=blur, reach=reach, scaling=q, diameter=d, fixed_iters=extra, translation=0,
                            precision=precision)
    out = otgb.sinkhorn_divergence(ctx, T(x), T(a), T(y), T(b), p, want_self=True)
    ref = oracle.sinkhorn(x, a, y, b, blur=blur, reach=reach, scaling=q, diameter=d, tol=0.0,
                          max_iters=n_sched + extra)
    assert out["stats"]["iters_total"] == ref["iters"] == n_sched + extra
    return out, ref


# precision 0: the D <= 3 exponent on the tensor cores (three-piece BF16, float32
# accuracy); 2: the CUDA-core float32 kernel -- both must meet the float32 bar
ENGINES = [0, 2]


@pytest.mark.parametrize("precision", ENGINES)
@pytest.mark.parametrize("reach", [0.0, 0.3])
def test_dense_solve_same_steps_as_oracle_3d(ctx, reach, precision):
    x, a, y, b = synth.rotated_cloud(700, 530, seed=3)
    blur = 0.05
    out, ref = _run_pair(ctx, x, a, y, b, blur, reach, 0.5, 12, precision)
    eps = blur ** 2
    check_pots(out, ref, a, b, eps, reach)
    assert abs(out["S"] - ref["S"]) <= TOL * abs(ref["S"]) + 1e-9 * eps, (out["S"], ref["S"])


def test_dense_solve_same_steps_as_oracle_fibers(ctx):
    ctrl = synth.bundle_centrelines()
    x, a, _ = synth.fiber_bundles(300, seed=4, ctrl=ctrl, perturb=3.0)
    y, b, _ = synth.fiber_bundles(257, seed=5, ctrl=ctrl)
    blur, reach = 2.0, 20.0
    out, ref = _run_pair(ctx, x, a, y, b, blur, reach, 0.5, 6)
    eps = blur ** 2
    check_pots(out, ref, a, b, eps, reach)
    assert abs(out["S"] - ref["S"]) <= TOL * abs(ref["S"]), (out["S"], ref["S"])


def test_single_dirac_closed_form_on_gpu(ctx):
    # N = M = 1: the converged S has the closed form of Eq. (2) in the plan mass.
    from paper_2107_02010_gb300 import otgb

    x = np.array([[0.1, 0.2, 0.3]], np.float32)
    y = np.array([[1.1, -0.4, 0.9]], np.float32)
    ma, mb, eps, reach = 1.0, 1.2, 1.0, 10.0
    rho = reach ** 2
    c = 0.5 * float(np.sum((x.astype(np.float64) - y) ** 2))

    def ot(m1, m2, cc):
        L = math.log(m1 * m2)
        pi = math.exp(((eps + rho) * L - cc) / (eps + 2 * rho))
        kl = lambda u, v: u * math.log(u / v) - u + v
        return pi * cc + eps * kl(pi, m1 * m2) + rho * kl(pi, m1) + rho * kl(pi, m2)

    ma32, mb32 = float(np.float32(ma)), float(np.float32(mb))
    S_ref = ot(ma32, mb32, c) - 0.5 * ot(ma32, ma32, 0) - 0.5 * ot(mb32, mb32, 0) + 0.5 * eps * (ma32 - mb32) ** 2
    p = otgb.default_params(blur=math.sqrt(eps), reach=reach, tol=1e-9, max_iters=20000)
    out = otgb.sinkhorn_divergence(ctx, T(x), T(np.array([ma], np.float32)), T(y), T(np.array([mb], np.float32)), p)
    assert out["S"] == pytest.approx(S_ref, rel=1e-5)


@pytest.mark.parametrize("precision", ENGINES)
def test_converged_solve_matches_converged_oracle(ctx, precision):
    from paper_2107_02010_gb300 import otgb

    x, a, y, b = synth.rotated_cloud(400, 300, seed=9)
    blur, reach = 0.15, 0.5
    ref = oracle.sinkhorn(x, a, y, b, blur=blur, reach=reach, scaling=0.5, tol=1e-12, max_iters=20000)
    assert ref["converged"]
    p = otgb.default_params(blur=blur, reach=reach, scaling=0.5, tol=1e-7, precision=precision)
    out = otgb.sinkhorn_divergence(ctx, T(x), T(a), T(y), T(b), p, want_self=True)
    eps = blur ** 2
    assert abs(out["S"] - ref["S"]) <= TOL * abs(ref["S"]), (out["S"], ref["S"])
    check_pots(out, ref, a, b, eps, reach)


@pytest.mark.parametrize("translation,anderson", [(0, 0), (1, 0), (0, 5), (1, 5)])
def test_accelerations_keep_the_fixed_point(ctx, translation, anderson):
    # unbalanced, slow (lambda close to 1): the translation step and Anderson
    # mixing change the number of steps, not the converged result.  The plain
    # averaged loop (0, 0) cannot resolve its slowest mode below the float32
    # step noise, so only S is required of it.
    from paper_2107_02010_gb300 import otgb

    x, a, y, b = synth.rotated_cloud(300, 250, seed=21)
    b = (b * 1.3).astype(np.float32)
    blur, reach = 0.1, 0.5
    ref = oracle.sinkhorn(x, a, y, b, blur=blur, reach=reach, scaling=0.5, tol=1e-12, max_iters=100000)
    assert ref["converged"]
    p = otgb.default_params(blur=blur, reach=reach, scaling=0.5, tol=1e-8, max_iters=50000,
                            translation=translation, anderson=anderson)
    out = otgb.sinkhorn_divergence(ctx, T(x), T(a), T(y), T(b), p, want_self=True)
    print("translation", translation, "anderson", anderson, "steps", out["stats"]["iters_total"],
          "oracle steps", ref["iters"])
    assert abs(out["S"] - ref["S"]) <= TOL * abs(ref["S"]), (out["S"], ref["S"])
    if translation or anderson:
        check_pots(out, ref, a, b, blur ** 2, reach)


def test_self_divergence_is_zero_on_gpu(ctx):
    from paper_2107_02010_gb300 import otgb

    x, a, _, _ = synth.rotated_cloud(600, seed=11)
    p = otgb.default_params(blur=0.1, reach=0.0, fixed_iters=20)
    out = otgb.sinkhorn_divergence(ctx, T(x), T(a), T(x), T(a), p)
    assert abs(out["S"]) < 1e-7
    np.testing.assert_array_equal(out["f"].cpu().numpy(), out["g"].cpu().numpy())


def test_invalid_arguments_are_rejected(ctx):
    from paper_2107_02010_gb300 import otgb

    x, a, y, b = synth.rotated_cloud(50, seed=1)
    X, A, Y, B = T(x), T(a), T(y), T(b)
    for kw in (dict(p=3), dict(blur=0.0), dict(blur=-1.0), dict(scaling=1.0), dict(scaling=0.0)):
        with pytest.raises(otgb.OtgbError) as e:
            otgb.sinkhorn_divergence(ctx, X, A, Y, B, otgb.default_params(**kw))
        assert e.value.code == -1
    bad = a.copy()
    bad[3] = -1.0
    with pytest.raises(otgb.OtgbError):
        otgb.sinkhorn_divergence(ctx, X, T(bad), Y, B, otgb.default_params())
    nanx = x.copy()
    nanx[5, 1] = np.nan
    with pytest.raises(otgb.OtgbError):
        otgb.sinkhorn_divergence(ctx, T(nanx), A, Y, B, otgb.default_params())
    with pytest.raises(otgb.OtgbError):
        otgb.sinkhorn_divergence(ctx, X, T(np.zeros_like(a)), Y, B, otgb.default_params())
    # the context stays usable after errors
    out = otgb.sinkhorn_divergence(ctx, X, A, Y, B, otgb.default_params(blur=0.2, fixed_iters=2))
    assert math.isfinite(out["S"])


# ----------------------------------------------------------- clustering ---
@pytest.mark.parametrize("n,cell", [(1, 1.0), (1000, 4.0), (50_000, 2.5)])
def test_cluster_grid_bit_exact(ctx, n, cell):
    from paper_2107_02010_gb300 import otgb

    r = np.random.default_rng(n)
    x = r.uniform(-3, 40, size=(n, 3)).astype(np.float32)
    w = r.uniform(0.1, 1.0, size=n).astype(np.float32)
    lab, perm, off, cent = otgb.cluster_grid(ctx, T(x), cell, w=T(w))
    rl, rp, ro, _ = oracle.cluster_grid(x, cell)
    np.testing.assert_array_equal(lab.cpu().numpy(), rl)
    np.testing.assert_array_equal(perm.cpu().numpy(), rp)
    np.testing.assert_array_equal(off.cpu().numpy(), ro)
    # centroids: weighted means of the clusters (float32 accumulation order differs)
    c = cent.cpu().numpy()
    for k in range(0, len(ro) - 1, max(1, (len(ro) - 1) // 50)):
        idx = rp[ro[k]:ro[k + 1]]
        ref = (w[idx, None].astype(np.float64) * x[idx]).sum(0) / w[idx].astype(np.float64).sum()
        np.testing.assert_allclose(c[k], ref, rtol=1e-5, atol=1e-5)


def test_cluster_kmeans_invariants(ctx):
    from paper_2107_02010_gb300 import otgb

    r = np.random.default_rng(5)
    centers = r.uniform(0, 10, size=(6, 60))
    x = (centers[r.integers(0, 6, 3000)] + r.normal(0, 0.2, size=(3000, 60))).astype(np.float32)
    lab, cent, perm, off = otgb.cluster_kmeans(ctx, T(x), 6, iters=15, seed=3)
    lab, cent, perm, off = lab.cpu().numpy(), cent.cpu().numpy().astype(np.float64), perm.cpu().numpy(), off.cpu().numpy()
    X = x.astype(np.float64)
    d2 = ((X[:, None] - cent[None]) ** 2).sum(-1)
    best = d2.min(1)
    assert np.all(d2[np.arange(3000), lab] <= best + 1e-3 * (1 + best))  # nearest up to fp32 ties
    assert sorted(perm) == list(range(3000))
    assert off[0] == 0 and off[-1] == 3000 and np.all(np.diff(off) >= 0)
    for k in range(6):
        idx = perm[off[k]:off[k + 1]]
        assert np.all(lab[idx] == k) and np.all(np.diff(idx) > 0)
    # same initial centroids -> same result as the oracle's Lloyd iterations
    init = x[[0, 500, 1000, 1500, 2000, 2500]]
    lab2, cent2, _, _ = otgb.cluster_kmeans(ctx, T(x), 6, iters=15, init=T(init))
    rl, rc = oracle.kmeans(x, None, 6, 15, init)
    assert np.mean(lab2.cpu().numpy() == rl) > 0.999
    np.testing.assert_allclose(cent2.cpu().numpy(), rc, rtol=1e-4, atol=1e-4)


# ----------------------------------------------------- transport_apply ---
def test_transport_apply_matches_oracle(ctx):
    from paper_2107_02010_gb300 import otgb

    x, a, y, b = synth.rotated_cloud(900, 700, seed=12)
    r = np.random.default_rng(12)
    labels = (np.floor(y[:, 0] * 4).clip(0, 3) + 4 * (y[:, 1] > 0.5)).astype(np.int32)
    blur, reach, L = 0.08, 0.5, 8
    p = otgb.default_params(blur=blur, reach=reach, tol=1e-7)
    out = otgb.sinkhorn_divergence(ctx, T(x), T(a), T(y), T(b), p, want_plan=True)
    f64 = out["f"].cpu().numpy().astype(np.float64)
    g64 = out["g"].cpu().numpy().astype(np.float64)
    sc, am, rm = otgb.transport_apply(ctx, out["plan"], out["f"], out["g"], T(labels), L)
    rsc, ram, rrm = oracle.transport_apply(x, y, b, blur ** 2, f64, g64, labels, L)
    np.testing.assert_allclose(sc.cpu().numpy(), rsc, rtol=1e-5, atol=1e-5 * rsc.max())
    np.testing.assert_allclose(rm.cpu().numpy(), rrm, rtol=1e-5)
    top2 = np.sort(rsc, axis=1)[:, -2:]
    clear = top2[:, 1] - top2[:, 0] >= 1e-4 * top2[:, 1]
    assert np.all(am.cpu().numpy()[clear] == ram[clear])


def test_transport_apply_fibers_identical_argmax(ctx):
    # 60-D label transfer by the smooth plan (Eq. (7)): scores against the
    # oracle and identical argmax labels on rows with a clear top class
    from paper_2107_02010_gb300 import otgb

    ctrl = synth.bundle_centrelines()
    x, a, _ = synth.fiber_bundles(600, seed=4, ctrl=ctrl, perturb=3.0)
    y, b, lab = synth.fiber_bundles(500, seed=5, ctrl=ctrl)
    blur, reach, L = 2.0, 20.0, 20
    out = otgb.sinkhorn_divergence(ctx, T(x), T(a), T(y), T(b), otgb.default_params(blur=blur, reach=reach, tol=1e-7),
                                   want_plan=True)
    f64 = out["f"].cpu().numpy().astype(np.float64)
    g64 = out["g"].cpu().numpy().astype(np.float64)
    sc, am, rm = otgb.transport_apply(ctx, out["plan"], out["f"], out["g"], T(lab), L)
    rsc, ram, rrm = oracle.transport_apply(x, y, b, blur ** 2, f64, g64, lab, L)
    np.testing.assert_allclose(sc.cpu().numpy(), rsc, rtol=1e-4, atol=1e-5 * rsc.max())
    np.testing.assert_allclose(rm.cpu().numpy(), rrm, rtol=1e-4)
    top2 = np.sort(rsc, axis=1)[:, -2:]
    clear = top2[:, 1] - top2[:, 0] >= 1e-4 * top2[:, 1]
    print("rows with a clear top class:", int(clear.sum()), "of", len(clear))
    assert np.all(am.cpu().numpy()[clear] == ram[clear])
