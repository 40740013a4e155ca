"""Parity at the benchmark's full size and launch configuration, on sampled
outputs the FP64 oracle computes one by one.

The benchmark solves the track-density workload (two 64^3 volumes, 100,000
voxels per side, masses 1.0 / 1.2, blur 1, reach 10, q = 0.5, multiscale with
4-voxel grid cells, truncation, stopping rule at 1e-6).  At the fixed point of
the averaged update every dual equals its own softmin over ALL columns (the
dense definition, no truncation), so for sampled rows the oracle's dense FP64
softmin of the GPU's final duals must reproduce the GPU's values up to the
size of the last step (the loop stops when max |new - old| / eps = delta; the
distance to the softmin is at most about 2 delta eps, one more delta eps for
the duals the softmin reads) plus float32 rounding.  S is recomputed from the
GPU's duals with the oracle's FP64 sums of Eq. (6)."""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu

BLUR, REACH, CELL = 1.0, 10.0, 4.0


@pytest.fixture(scope="module")
def solved():
    from paper_2107_02010_gb300 import otgb, synth
    oracle.build()
    ctx = otgb.Context()
    x, a, y, b = synth.density_maps(grid=64, n_keep=100_000)
    X, A, Y, B = (torch.from_numpy(v).cuda() for v in (x, a, y, b))
    p = otgb.default_params(blur=BLUR, reach=REACH, scaling=0.5, multiscale=1, cluster=0, cell=CELL, tol=1e-6,
                            max_iters=20000, check_every=10)
    r = otgb.sinkhorn_divergence(ctx, X, A, Y, B, p, want_self=True)
    duals = {k: r[k].cpu().numpy().astype(np.float64) for k in ("f", "g", "a_self", "b_self")}
    return dict(x=x, a=a, y=y, b=b, r=r, duals=duals)


def test_full_size_sampled_rows_are_dense_fixed_points(solved):
    x, a, y, b = solved["x"], solved["a"], solved["y"], solved["b"]
    d = solved["duals"]
    st = solved["r"]["stats"]
    eps = BLUR ** 2
    lam = oracle.lam(BLUR, REACH)
    delta = st["last_delta"]
    rng = np.random.default_rng(123)
    ix = np.sort(rng.choice(x.shape[0], 192, replace=False))
    iy = np.sort(rng.choice(y.shape[0], 192, replace=False))
    # (rows, columns, weights, the potential the softmin reads, the dual it must equal)
    cases = [
        ("f: beta -> alpha", x[ix], y, b, d["g"], d["f"][ix]),
        ("g: alpha -> beta", y[iy], x, a, d["f"], d["g"][iy]),
        ("a: alpha <-> alpha", x[ix], x, a, d["a_self"], d["a_self"][ix]),
        ("b: beta <-> beta", y[iy], y, b, d["b_self"], d["b_self"][iy]),
    ]
    for name, q, pts, w, pot, got in cases:
        ref = oracle.softmin(q, pts, w, pot, eps, lam)
        bound = 3.0 * delta * eps + 2e-5 * (np.abs(ref) + eps)
        err = np.abs(got - ref)
        assert np.all(err <= bound), (name, float(err.max()), float(bound[np.argmax(err - bound)]))


def test_full_size_divergence_from_fp64_sums(solved):
    x, a, y, b = solved["x"], solved["a"], solved["y"], solved["b"]
    d = solved["duals"]
    eps = BLUR ** 2
    S_ref = oracle.divergence(a, b, eps, oracle.rho(REACH), d["a_self"], d["b_self"], d["f"], d["g"])
    S = solved["r"]["S"]
    assert abs(S - S_ref) <= 1e-9 * abs(S_ref) + 1e-12, (S, S_ref)
    assert solved["r"]["status"] == 0
