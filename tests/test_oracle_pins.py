"""Pins of the FP64 oracle against facts fixed by the paper and by the
mathematics, independent of the oracle's own code path.

Each test names the passage it rests on.  Together they are chosen so that a
plausible slip in the oracle (a dropped damping factor, a wrong sign in the
averaging, swapped weights, a wrong mass term, an off-by-one schedule) makes
at least one of them fail.
"""
import itertools
import math

import numpy as np
import pytest

import oracle

RNG = np.random.default_rng(12345)


def _cloud(n, d=3, seed=0, scale=1.0):
    r = np.random.default_rng(seed)
    return (r.uniform(0, scale, size=(n, d))).astype(np.float32)


def _weights(n, seed=0, total=1.0):
    """Positive weights of the given total.  Total 1.0 is met EXACTLY: the
    weights are multiples of 2^-14, so that balanced problems (equal masses,
    Eq. (1)) have equal masses in float32 and in double alike."""
    r = np.random.default_rng(seed)
    if total == 1.0:
        units = 1 << 14
        p = r.uniform(0.5, 1.5, size=n)
        c = r.multinomial(units - n, p / p.sum()) + 1  # each weight >= 2^-14
        w = c.astype(np.float64) / units
        assert w.sum() == 1.0
        return w.astype(np.float32)
    w = r.uniform(0.5, 1.5, size=n)
    return (w / w.sum() * total).astype(np.float32)


# ---------------------------------------------------------------- schedule --
def test_schedule_endpoints_and_length():
    # Algorithm (Section 2): sigma runs d, dq, dq^2, ... down to blur, in
    # ceil(log(d/blur)/log(1/q)) scaled steps.
    s = oracle.schedule(2.0, 0.05, 0.5)
    assert len(s) == math.ceil(math.log(40) / math.log(2)) + 1 == 7
    np.testing.assert_allclose(s[:-1], 2.0 * 0.5 ** np.arange(6))
    assert s[-1] == 0.05 and s[-2] > 0.05 and s[-2] * 0.5 < 0.05
    assert list(oracle.schedule(0.01, 0.05, 0.5)) == [0.05]
    assert len(oracle.schedule(111.0, 1.0, 0.9)) == math.ceil(math.log(111) / math.log(1 / 0.9)) + 1


def test_diameter_is_the_joint_bounding_box_diagonal():
    # Algorithm (Section 2): the schedule starts at a diameter d >= max |x_i - y_j|;
    # the documented reading is the diagonal of the bounding box of x and y
    # together.  Here x spans the first axis only and y the second and third,
    # so the box of x alone, the box of y alone, a missing square root or a
    # missing axis all give another number than sqrt(1 + 4 + 9).
    x = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0]], np.float32)
    y = np.array([[0.0, 2.0, 0.0], [0.0, 0.0, -3.0]], np.float32)
    assert oracle.diameter(x, y) == pytest.approx(math.sqrt(14.0), rel=1e-15)
    assert oracle.diameter(y, x) == pytest.approx(math.sqrt(14.0), rel=1e-15)
    # one point: no extent
    assert oracle.diameter(x[:1], x[:1]) == 0.0


@pytest.mark.parametrize("D", [1, 3, 7])
def test_diameter_bounds_every_pair_distance(D):
    # an upper bound of the paper's max_ij |x_i - y_j|, and equal to the largest
    # distance between corners of the joint box (brute force over the corners)
    r = np.random.default_rng(40 + D)
    x = r.normal(0.0, 2.0, size=(50, D)).astype(np.float32)
    y = (r.normal(0.0, 1.0, size=(40, D)) + 3.0).astype(np.float32)
    d = oracle.diameter(x, y)
    xd, yd = x.astype(np.float64), y.astype(np.float64)
    pair_max = np.sqrt(((xd[:, None, :] - yd[None, :, :]) ** 2).sum(-1)).max()
    assert d >= pair_max
    both = np.concatenate([xd, yd])
    lo, hi = both.min(0), both.max(0)
    corners = np.array(list(itertools.product(*zip(lo, hi))))
    corner_max = np.sqrt(((corners[:, None, :] - corners[None, :, :]) ** 2).sum(-1)).max()
    assert d == pytest.approx(corner_max, rel=1e-14)


def test_damping_and_rho():
    # lambda = 1/(1+(sigma/reach)^p), rho = reach^p; reach = inf -> balanced.
    assert oracle.lam(1.0, 10.0) == pytest.approx(1.0 / 1.01, rel=1e-15)
    assert oracle.lam(3.0, 0.0) == 1.0 and oracle.lam(3.0, math.inf) == 1.0
    assert oracle.rho(20.0) == 400.0 and math.isinf(oracle.rho(0.0))


# ----------------------------------------------------------------- softmin --
def test_softmin_single_column_closed_form():
    # One column: -lam eps log(w exp((pot - C)/eps)) = -lam (eps log w + pot - C).
    q = _cloud(5, seed=1)
    p = _cloud(1, seed=2)
    w, pot, eps, lam = 0.3, 0.7, 0.05, 0.9
    out = oracle.softmin(q, p, np.array([w], np.float32), np.array([pot]), eps, lam)
    C = 0.5 * np.sum((q.astype(np.float64) - p.astype(np.float64)) ** 2, axis=1)
    np.testing.assert_allclose(out, -lam * (eps * np.log(float(np.float32(w))) + pot - C), rtol=1e-13, atol=1e-15)


def test_softmin_reduces_to_library_logsumexp():
    from scipy.special import logsumexp

    q, p = _cloud(7, seed=3), _cloud(40, seed=4)
    w, pot = _weights(40, seed=5), RNG.normal(size=40)
    eps, lam = 0.02, 0.8
    C = 0.5 * ((q[:, None, :].astype(np.float64) - p[None, :, :].astype(np.float64)) ** 2).sum(-1)
    ref = -lam * eps * logsumexp((pot[None, :] - C) / eps, b=w.astype(np.float64)[None, :], axis=1)
    np.testing.assert_allclose(oracle.softmin(q, p, w, pot, eps, lam), ref, rtol=1e-12)
    # a zero-weight column is ignored
    w0 = w.copy(); w0[3] = 0
    ref0 = -lam * eps * logsumexp(np.delete((pot[None, :] - C) / eps, 3, 1),
                                  b=np.delete(w0.astype(np.float64), 3)[None, :], axis=1)
    np.testing.assert_allclose(oracle.softmin(q, p, w0, pot, eps, lam), ref0, rtol=1e-12)


# ------------------------------------------------------ single Dirac masses --
@pytest.mark.parametrize("p,ma,mb,eps,reach", [(2, 1.0, 1.2, 1.0, 10.0), (2, 0.3, 2.0, 0.5, 1.5),
                                               (2, 1.0, 1.0, 4.0, 20.0), (1, 1.0, 1.2, 0.5, 3.0),
                                               (1, 0.3, 2.0, 0.2, 1.5)])
def test_single_dirac_unbalanced_closed_form(p, ma, mb, eps, reach):
    # Eq. (2) with one Dirac on each side is a 1-D convex problem in the plan
    # mass pi: stationarity c + eps log(pi/(ma mb)) + rho log(pi/ma)
    # + rho log(pi/mb) = 0 gives log pi = ((eps + rho) log(ma mb) - c)/(eps + 2 rho).
    # OT, both self terms and S of Eq. (5) then follow in closed form; the
    # oracle reaches them through its fixed-point iteration and Eq. (6).
    # p = 1: C = |x - y|, eps = blur, rho = reach (Section 2: C = |x - y|^p / p, eps = blur^p).
    x = np.array([[0.1, 0.2, 0.3]], np.float32)
    y = np.array([[1.1, -0.4, 0.9]], np.float32)
    rho = reach ** p
    d2 = float(np.sum((x.astype(np.float64) - y.astype(np.float64)) ** 2))
    c = 0.5 * d2 if p == 2 else math.sqrt(d2)
    ma32, mb32 = float(np.float32(ma)), float(np.float32(mb))

    def ot_primal(m1, m2, cc):
        L = math.log(m1 * m2)
        pi = math.exp(((eps + rho) * L - cc) / (eps + 2 * rho))
        kl = lambda u, v: u * math.log(u / v) - u + v
        return pi * cc + eps * kl(pi, m1 * m2) + rho * kl(pi, m1) + rho * kl(pi, m2), pi

    ot_ab, pi_ab = ot_primal(ma32, mb32, c)
    ot_aa, _ = ot_primal(ma32, ma32, 0.0)
    ot_bb, _ = ot_primal(mb32, mb32, 0.0)
    S_ref = ot_ab - 0.5 * ot_aa - 0.5 * ot_bb + 0.5 * eps * (ma32 - mb32) ** 2
    r = oracle.sinkhorn(x, np.array([ma], np.float32), y, np.array([mb], np.float32), blur=eps ** (1.0 / p),
                        reach=reach, scaling=0.5, p=p)
    assert r["converged"]
    assert r["S"] == pytest.approx(S_ref, rel=1e-10, abs=1e-13)
    # plan mass of Eq. (4) from the oracle's duals
    pi = ma32 * mb32 * math.exp((r["f"][0] + r["g"][0] - c) / eps)
    assert pi == pytest.approx(pi_ab, rel=1e-10)


@pytest.mark.parametrize("t", [0.3, 1.7])
def test_single_dirac_balanced_p1_is_the_distance(t):
    # p = 1, balanced, one Dirac of mass 1 on each side: the only coupling is
    # the product, whose entropy term vanishes, so OT = C = |t| and both self
    # terms are 0: S = |t| for every eps (Eqs. (2) and (5)).
    x = np.array([[0.0, 0.0]], np.float32)
    y = np.array([[0.6 * t, 0.8 * t]], np.float32)
    one = np.array([1.0], np.float32)
    for blur in (0.05, 0.5):
        r = oracle.sinkhorn(x, one, y, one, blur=blur, reach=0.0, scaling=0.5, p=1)
        assert r["converged"]
        assert r["S"] == pytest.approx(float(np.linalg.norm(y.astype(np.float64))), rel=1e-12)


# --------------------------------------------------- balanced invariances --
@pytest.mark.parametrize("blur", [0.2, 0.4, 1.0])
def test_shift_identity_balanced(blur):
    # p = 2, balanced: C(x, x' + t) = C(x, x') - <x - x', t> + |t|^2/2 and the
    # linear term integrates to a constant under fixed marginals (Eq. (1)), so
    # S(alpha, alpha shifted by t) = |t|^2/2 * mass for every eps.
    x = _cloud(40, seed=7)
    w = _weights(40, seed=8)
    t = np.array([0.3, -0.1, 0.2])
    y = (x.astype(np.float64) + t).astype(np.float32)
    tt = (y.astype(np.float64) - x.astype(np.float64))  # exact float32 shift per point
    assert np.allclose(tt, tt[0], atol=1e-7)
    r = oracle.sinkhorn(x, w, y, w, blur=blur, reach=0.0, scaling=0.5)
    assert r["converged"]
    expect = 0.5 * float(np.sum(w.astype(np.float64) * np.sum(tt ** 2, axis=1)))
    assert r["S"] == pytest.approx(expect, rel=1e-7)


@pytest.mark.parametrize("reach", [0.0, 0.5])
def test_self_divergence_is_zero(reach):
    # Section 2: S is definite, S(alpha, alpha) = 0.
    x = _cloud(50, seed=9)
    w = _weights(50, seed=10, total=1.3)
    r = oracle.sinkhorn(x, w, x, w, blur=0.1, reach=reach, scaling=0.5)
    assert r["converged"]
    assert abs(r["S"]) < 1e-14


@pytest.mark.parametrize("reach", [0.0, 0.7])
def test_symmetry_and_positivity(reach):
    # Section 2: S is symmetric and positive.
    x, y = _cloud(30, seed=11), _cloud(45, seed=12, scale=1.3)
    a, b = _weights(30, seed=13), _weights(45, seed=14, total=1.0 if reach == 0.0 else 1.4)
    r1 = oracle.sinkhorn(x, a, y, b, blur=0.1, reach=reach, scaling=0.5)
    r2 = oracle.sinkhorn(y, b, x, a, blur=0.1, reach=reach, scaling=0.5)
    assert r1["converged"] and r2["converged"]
    assert r1["S"] > 0
    assert r1["S"] == pytest.approx(r2["S"], rel=1e-11)
    np.testing.assert_allclose(r1["a"], r2["b"], rtol=1e-11, atol=1e-14)


# ------------------------------------------------------ duality and Eq. (6) --
@pytest.mark.parametrize("reach", [0.0, 0.6])
def test_strong_duality_and_marginals(reach):
    # Eq. (2) evaluated at the plan of Eq. (4) equals Eq. (3) at the optimum
    # (strong duality); in the balanced case the plan has marginals alpha, beta.
    x, y = _cloud(12, seed=15), _cloud(9, seed=16)
    a, b = _weights(12, seed=17), _weights(9, seed=18, total=1.0 if reach == 0.0 else 0.7)
    blur = 0.25
    r = oracle.sinkhorn(x, a, y, b, blur=blur, reach=reach, scaling=0.5)
    assert r["converged"]
    eps, rho = blur ** 2, oracle.rho(reach)
    dual = oracle.ot_dual(x, a, y, b, eps, rho, r["f"], r["g"])
    primal, merr = oracle.ot_primal(x, a, y, b, eps, rho, r["f"], r["g"])
    assert primal == pytest.approx(dual, rel=1e-10, abs=1e-13)
    if reach == 0.0:
        assert merr < 1e-12
    # a perturbed dual pair is strictly worse (the optimum is a maximum)
    assert oracle.ot_dual(x, a, y, b, eps, rho, r["f"] + 1e-3 * np.sin(np.arange(12)), r["g"]) < dual


@pytest.mark.parametrize("reach", [0.0, 0.4, 2.0])
def test_dual_form_eq6_equals_definition_eq5(reach):
    # Eq. (5): S = OT(a,b) - OT(a,a)/2 - OT(b,b)/2 + eps/2 (sum a - sum b)^2,
    # each OT evaluated through Eq. (3) at its own optimum, equals the dual
    # shortcut Eq. (6) used by the solver.
    x, y = _cloud(10, seed=19), _cloud(13, seed=20, scale=1.5)
    a = _weights(10, seed=21, total=1.0)
    b = _weights(13, seed=22, total=1.0 if reach == 0.0 else 1.3)
    blur = 0.3
    r = oracle.sinkhorn(x, a, y, b, blur=blur, reach=reach, scaling=0.5)
    assert r["converged"]
    eps, rho = blur ** 2, oracle.rho(reach)
    ot_ab = oracle.ot_dual(x, a, y, b, eps, rho, r["f"], r["g"])
    ot_aa = oracle.ot_dual(x, a, x, a, eps, rho, r["a"], r["a"])
    ot_bb = oracle.ot_dual(y, b, y, b, eps, rho, r["b"], r["b"])
    ma, mb = float(a.astype(np.float64).sum()), float(b.astype(np.float64).sum())
    S5 = ot_ab - 0.5 * ot_aa - 0.5 * ot_bb + 0.5 * eps * (ma - mb) ** 2
    assert r["S"] == pytest.approx(S5, rel=1e-10, abs=1e-14)


def test_unbalanced_plan_masses_agree_at_the_fixed_point():
    # At the unbalanced fixed point sum_j b_j exp((f_i + g_j - C_ij)/eps) = e^{-f_i/rho}
    # (damped softmin), so the plan mass is <alpha, e^{-f/rho}> = <beta, e^{-g/rho}>:
    # the translation (f + c, g - c) with c = (rho/2) log of their ratio is 0 there.
    x, y = _cloud(30, seed=27), _cloud(22, seed=28)
    a, b = _weights(30, seed=29), _weights(22, seed=30, total=1.4)
    blur, reach = 0.2, 0.7
    r = oracle.sinkhorn(x, a, y, b, blur=blur, reach=reach, scaling=0.5)
    rho = oracle.rho(reach)
    A = float(a.astype(np.float64) @ np.exp(-r["f"] / rho))
    B = float(b.astype(np.float64) @ np.exp(-r["g"] / rho))
    assert A == pytest.approx(B, rel=1e-11)
    eps = blur ** 2
    C = 0.5 * ((x[:, None].astype(np.float64) - y[None]) ** 2).sum(-1)
    plan = a[:, None].astype(np.float64) * b[None] * np.exp((r["f"][:, None] + r["g"][None] - C) / eps)
    assert plan.sum() == pytest.approx(A, rel=1e-10)


def test_fixed_point_of_plain_update():
    # At convergence each vector is a fixed point of its own (undamped-average)
    # softmin update of the Algorithm, Section 2.
    x, y = _cloud(25, seed=23), _cloud(31, seed=24)
    a, b = _weights(25, seed=25), _weights(31, seed=26, total=1.2)
    blur, reach = 0.15, 0.8
    r = oracle.sinkhorn(x, a, y, b, blur=blur, reach=reach, scaling=0.5)
    eps, lam = blur ** 2, oracle.lam(blur, reach)
    np.testing.assert_allclose(oracle.softmin(x, y, b, r["g"], eps, lam), r["f"], atol=1e-12 * eps)
    np.testing.assert_allclose(oracle.softmin(y, x, a, r["f"], eps, lam), r["g"], atol=1e-12 * eps)
    np.testing.assert_allclose(oracle.softmin(x, x, a, r["a"], eps, lam), r["a"], atol=1e-12 * eps)
    np.testing.assert_allclose(oracle.softmin(y, y, b, r["b"], eps, lam), r["b"], atol=1e-12 * eps)


# ---------------------------------------------------------- blur -> 0 limit --
def test_small_blur_matches_assignment_brute_force():
    # Eq. (1) with N = M and uniform weights is an assignment problem; as
    # blur -> 0 the entropic terms eps log N of OT(a,b) and of the self terms
    # cancel in Eq. (5), so S -> min over permutations of (1/N) sum C.  Label
    # transfer (Eq. (7)) then gives each x_i the label of its matched y.
    r = np.random.default_rng(31)
    n = 6
    while True:
        x = r.uniform(0, 1, size=(n, 3)).astype(np.float32)
        y = (x[r.permutation(n)] + r.normal(0, 0.15, size=(n, 3))).astype(np.float32)
        X, Y = x.astype(np.float64), y.astype(np.float64)
        C = 0.5 * ((X[:, None] - Y[None]) ** 2).sum(-1)
        costs = sorted((sum(C[i, s[i]] for i in range(n)) / n, s) for s in itertools.permutations(range(n)))
        gap = costs[1][0] - costs[0][0]
        sep = min(min(0.5 * np.sum((X[i] - X[k]) ** 2), 0.5 * np.sum((Y[i] - Y[k]) ** 2))
                  for i in range(n) for k in range(n) if i != k)
        if gap > 2e-3 and sep > 2e-3:
            break
    W, sigma = costs[0]
    eps = min(gap * n, sep) / 40.0  # per-pair gap (x n) and self separation
    w = np.full(n, 1.0 / n, np.float32)
    # Near-permutation plans make the averaged iteration slow in the duals
    # (each matched pair is almost its own component), so run a fixed, large
    # number of steps rather than to a dual tolerance.
    res = oracle.sinkhorn(x, w, y, w, blur=math.sqrt(eps), reach=0.0, scaling=0.5, max_iters=100_000)
    assert abs(res["S"] - W) <= 1e-6 * W
    sc, am, mass = oracle.transport_apply(x, y, w, eps, res["f"], res["g"], np.arange(n, dtype=np.int32), n)
    assert list(am) == list(sigma)
    np.testing.assert_allclose(mass, 1.0, atol=1e-3)


# ------------------------------------------------------- transport_apply --
@pytest.mark.parametrize("reach", [0.0, 0.5])
def test_transport_apply_row_mass_is_marginal(reach):
    # Eq. (7) with a single class sums the plan row: (1/alpha_i)(pi 1)_i, which
    # is 1 at the balanced optimum and e^{-f_i/rho} at the unbalanced one
    # (fixed point of the damped update).
    x, y = _cloud(20, seed=40), _cloud(17, seed=41)
    a, b = _weights(20, seed=42), _weights(17, seed=43, total=1.0 if reach == 0.0 else 1.5)
    blur = 0.2
    r = oracle.sinkhorn(x, a, y, b, blur=blur, reach=reach, scaling=0.5)
    eps, rho = blur ** 2, oracle.rho(reach)
    labels = np.zeros(17, np.int32)
    sc, am, mass = oracle.transport_apply(x, y, b, eps, r["f"], r["g"], labels, 1)
    expect = np.ones(20) if reach == 0.0 else np.exp(-r["f"] / rho)
    np.testing.assert_allclose(mass, expect, rtol=1e-10)
    # several classes partition the row
    labels3 = (np.arange(17) % 3).astype(np.int32)
    sc3, am3, mass3 = oracle.transport_apply(x, y, b, eps, r["f"], r["g"], labels3, 3)
    np.testing.assert_allclose(sc3.sum(1), mass, rtol=1e-12)
    assert np.all(am3 == np.argmax(sc3, axis=1))


# ------------------------------------------------------------- clustering --
def _morton_less(ca, cb):
    """Order of two cell coordinates in bit-interleaved (Z) order, decided by
    the axis holding the most significant differing bit (x lowest in a bit
    triple, so ties between axes at the same bit go to the higher axis)."""
    best_axis, best_msb = -1, -1
    for d in range(len(ca)):
        xo = int(ca[d]) ^ int(cb[d])
        msb = xo.bit_length() - 1
        if xo and (msb > best_msb or (msb == best_msb and d > best_axis)):
            best_axis, best_msb = d, msb
    if best_axis < 0:
        return False
    return ca[best_axis] < cb[best_axis]


def test_grid_clustering_invariants():
    r = np.random.default_rng(50)
    x = r.uniform(0, 37.0, size=(3000, 3)).astype(np.float32)
    cell = 4.0
    labels, perm, offsets, keys = oracle.cluster_grid(x, cell)
    n = len(offsets) - 1
    assert sorted(perm) == list(range(3000))
    o = x.min(0)
    cells = []
    for c in range(n):
        idx = perm[offsets[c]:offsets[c + 1]]
        assert np.all(np.diff(idx) > 0)  # stable: original order inside a cluster
        assert np.all(labels[idx] == c)
        lo = np.floor((x[idx].astype(np.float64) - o) / cell).min(0)
        hi = np.floor((x[idx].astype(np.float64) - o) / cell).max(0)
        assert np.all(lo == hi)  # one cell per cluster
        cells.append(tuple(lo.astype(int)))
    assert len(set(cells)) == n  # distinct cells
    for c in range(n - 1):
        assert _morton_less(cells[c], cells[c + 1])
    # every occupied cell of the lattice is a cluster
    occ = {tuple(v) for v in np.floor((x.astype(np.float64) - o) / cell).astype(int)}
    assert occ == set(cells)


def test_kmeans_matches_library_lloyd():
    sk = pytest.importorskip("sklearn.cluster")
    r = np.random.default_rng(60)
    centers = r.uniform(0, 10, size=(5, 4))
    x = (centers[r.integers(0, 5, 600)] + r.normal(0, 0.3, size=(600, 4))).astype(np.float32)
    init = x[r.choice(600, 5, replace=False)]
    labels, cent = oracle.kmeans(x, None, 5, 20, init)
    km = sk.KMeans(n_clusters=5, init=init.astype(np.float64), n_init=1, max_iter=20, tol=0.0,
                   algorithm="lloyd").fit(x.astype(np.float64))
    np.testing.assert_allclose(cent, km.cluster_centers_, rtol=1e-9, atol=1e-9)
    assert np.all(labels == km.labels_)


def test_kmeans_weighted_invariants():
    r = np.random.default_rng(61)
    x = r.normal(size=(400, 3)).astype(np.float32)
    w = r.uniform(0.1, 2.0, 400).astype(np.float32)
    init = x[:8]
    labels, cent = oracle.kmeans(x, w, 8, 60, init)
    X = x.astype(np.float64)
    d2 = ((X[:, None] - cent[None]) ** 2).sum(-1)
    assert np.all(labels == np.argmin(d2, axis=1))  # nearest centroid
    for k in range(8):
        m = labels == k
        if m.any():  # converged: centroid is the weighted mean of its points
            np.testing.assert_allclose(cent[k], (w[m, None] * X[m]).sum(0) / w[m].astype(np.float64).sum(),
                                       rtol=1e-9, atol=1e-9)


# ------------------------------------------------------- flip augmentation --
def test_flip_augmentation_is_an_involution_on_the_points():
    # Section 2 (fiber encoding): a fiber and its mirror flip are the same
    # curve with the P points in reverse order
    r = np.random.default_rng(70)
    P = 20
    x = r.normal(size=(7, 3 * P)).astype(np.float32)
    aug = oracle.flip_fibers(x, P)
    assert aug.shape == (14, 3 * P)
    np.testing.assert_array_equal(aug[:7], x)
    back = oracle.flip_fibers(aug[7:], P)[7:]
    np.testing.assert_array_equal(back, x)
    pts = lambda v: np.sort(v.reshape(-1, P, 3), axis=1)
    np.testing.assert_array_equal(pts(aug[7:]), pts(x))
    np.testing.assert_array_equal(aug[7:].reshape(7, P, 3)[:, 0], x.reshape(7, P, 3)[:, -1])
    # a palindromic fiber is its own flip
    half = r.normal(size=(P // 2, 3))
    pal = np.concatenate([half, half[::-1]]).reshape(1, -1).astype(np.float32)
    np.testing.assert_array_equal(oracle.flip_fibers(pal, P)[1], pal[0])


def test_select_flips_keeps_the_version_with_the_larger_row_mass():
    mass = np.array([0.9, 0.1, 0.5, 1e-9, 0.8, 0.5])
    am = np.array([3, 4, 5, 6, 7, 8], np.int32)
    lab, ver, m = oracle.select_flips(mass, am, 3)
    assert list(ver) == [0, 1, 0] and list(lab) == [3, 7, 5]  # fiber 2: a tie keeps the original
    np.testing.assert_array_equal(m, [0.9, 0.8, 0.5])


def test_flip_augmented_label_transfer_matches_each_fiber_once():
    # Section 2 (label transfer on augmented data): with the subject in random
    # orientation and augmented by its flips, the unbalanced plan matches the
    # version that runs like the atlas fibers and leaves the other one as an
    # outlier, so every fiber gets its bundle's label from the kept version
    from paper_2107_02010_gb300 import synth

    ctrl = synth.bundle_centrelines(n_bundles=3)
    x, a, lab_x = synth.fiber_bundles(24, seed=71, ctrl=ctrl, canonical=False)
    y, b, lab_y = synth.fiber_bundles(24, seed=72, ctrl=ctrl)
    aug = oracle.flip_fibers(x)
    w = np.concatenate([a, a])
    blur, reach = 2.0, 20.0
    r = oracle.sinkhorn(aug, w, y, b, blur=blur, reach=reach, scaling=0.5)
    assert r["converged"]
    _, am, rm = oracle.transport_apply(aug, y, b, blur ** 2, r["f"], r["g"], lab_y, 3)
    lab, ver, m = oracle.select_flips(rm, am, 24)
    assert np.all(lab == lab_x)
    # the kept version carries clearly more mass (at reach 20 mm moving the
    # reversed version some way still costs less than destroying all of it)
    other = rm[np.where(ver == 0, np.arange(24) + 24, np.arange(24))]
    assert np.all(m > 0.5) and np.all(other < 0.5 * m)
    # the kept version runs like the canonical atlas: first point before last
    fib = aug[np.where(ver == 0, np.arange(24), np.arange(24) + 24)].reshape(24, 20, 3)
    first, last = fib[:, 0], fib[:, -1]
    ref = y.reshape(24, 20, 3)
    for i in range(24):
        j = np.where(lab_y == lab_x[i])[0][0]
        assert np.linalg.norm(first[i] - ref[j, 0]) < np.linalg.norm(last[i] - ref[j, 0])
