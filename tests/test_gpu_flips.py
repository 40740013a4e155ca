"""Flip-augmented label transfer (Section 2: fibers are unoriented, the
tractogram is augmented with the mirror flip of every fiber, the plan is
computed on the augmented data and only the matched version of each fiber is
kept for the transfer of labels).  The GPU augmentation equals the oracle's
bit for bit; on a subject in random orientation the GPU solve, transport_apply
and the version choice give the oracle's labels and versions; at a larger size
the kept labels are the fibers' bundles."""
import numpy as np
import pytest
import torch

import oracle
from paper_2107_02010_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2107_02010_gb300 import otgb

    c = otgb.Context()
    yield c
    c.close()


def T(v):
    return torch.from_numpy(np.ascontiguousarray(v)).cuda()


def test_flip_fibers_bit_exact(ctx):
    from paper_2107_02010_gb300 import otgb

    x, _, _ = synth.fiber_bundles(777, seed=80, canonical=False)
    got = otgb.flip_fibers(ctx, T(x)).cpu().numpy()
    np.testing.assert_array_equal(got, oracle.flip_fibers(x))


def _augmented_transfer(otgb, ctx, x, a, y, b, lab_y, L, blur=2.0, reach=20.0):
    aug = otgb.flip_fibers(ctx, T(x))
    w = T(np.concatenate([a, a]))
    p = otgb.default_params(blur=blur, reach=reach, tol=1e-9, max_iters=20000)
    out = otgb.sinkhorn_divergence(ctx, aug, w, T(y), T(b), p, want_plan=True)
    _, am, rm = otgb.transport_apply(ctx, out["plan"], out["f"], out["g"], T(lab_y), L, want_scores=False)
    return aug, out, am, rm, otgb.select_flips(ctx, rm, am)


def test_flip_label_transfer_matches_oracle(ctx):
    from paper_2107_02010_gb300 import otgb

    ctrl = synth.bundle_centrelines(n_bundles=4)
    x, a, lab_x = synth.fiber_bundles(150, seed=81, ctrl=ctrl, perturb=2.0, canonical=False)
    y, b, lab_y = synth.fiber_bundles(120, seed=82, ctrl=ctrl)
    aug, out, am, rm, (lab, ver, mass) = _augmented_transfer(otgb, ctx, x, a, y, b, lab_y, 4)
    xa = oracle.flip_fibers(x)
    r = oracle.sinkhorn(xa, np.concatenate([a, a]), y, b, blur=2.0, reach=20.0, scaling=0.5, tol=1e-12,
                        max_iters=100000)
    assert r["converged"]
    _, ram, rrm = oracle.transport_apply(xa, y, b, 4.0, r["f"], r["g"], lab_y, 4)
    rlab, rver, rmass = oracle.select_flips(rrm, ram, 150)
    clear = np.abs(rrm[:150] - rrm[150:]) > 1e-3 * np.maximum(rrm[:150], rrm[150:])
    assert clear.sum() >= 140
    assert np.all(ver.cpu().numpy()[clear] == rver[clear])
    assert np.all(lab.cpu().numpy()[clear] == rlab[clear])
    np.testing.assert_allclose(mass.cpu().numpy(), rmass, rtol=1e-4)
    assert np.mean(rlab == lab_x) > 0.97


def test_flip_label_transfer_recovers_bundles_at_scale(ctx):
    from paper_2107_02010_gb300 import otgb

    ctrl = synth.bundle_centrelines()
    x, a, lab_x = synth.fiber_bundles(20000, seed=83, ctrl=ctrl, perturb=3.0, canonical=False)
    y, b, lab_y = synth.fiber_bundles(20000, seed=84, ctrl=ctrl)
    aug = otgb.flip_fibers(ctx, T(x))
    w = T(np.concatenate([a, a]))
    p = otgb.default_params(blur=2.0, reach=20.0, multiscale=1, cluster=1, k_clusters=80, check_every=3)
    out = otgb.sinkhorn_divergence(ctx, aug, w, T(y), T(b), p, want_plan=True)
    _, am, rm = otgb.transport_apply(ctx, out["plan"], out["f"], out["g"], T(lab_y), 20, want_scores=False)
    lab, ver, mass = otgb.select_flips(ctx, rm, am)
    acc = float(np.mean(lab.cpu().numpy() == lab_x))
    print("bundle accuracy %.4f" % acc)
    assert acc > 0.97
