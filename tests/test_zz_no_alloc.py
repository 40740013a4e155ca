"""The allocation-free softmin entry point (otgb_softmin_noalloc) gives the
same result as otgb_softmin, through the C ABI, on two calls in a row.

It is meant for callers that may not allocate device memory (a fixed memory
budget owned by the host application, latency-critical loops, callers with
no otgb context): all its scratch is one fixed device array inside the
library.  This file is collected last so that a failure here leaves every
other test already run."""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _case(seed, n_out, n_in, D):
    r = np.random.default_rng(seed)
    q = r.uniform(0, 1, size=(n_out, D)).astype(np.float32)
    p = r.uniform(0, 1, size=(n_in, D)).astype(np.float32)
    w = r.uniform(0.2, 1.0, size=n_in).astype(np.float32)
    pot = (0.01 * r.normal(size=n_in)).astype(np.float32)
    old = (0.01 * r.normal(size=n_out)).astype(np.float32)
    T = lambda v: torch.from_numpy(v).cuda()
    return T(q), T(p), T(w), T(pot), T(old)


def test_noalloc_matches_softmin_two_calls_in_a_row():
    from paper_2107_02010_gb300 import otgb

    ctx = otgb.Context()
    cases = [(1, 5000, 3000, 3, 0.01, 1.0), (2, 777, 1313, 60, 0.2, 0.9)]
    outs = [torch.empty(c[1], device="cuda", dtype=torch.float32) for c in cases]
    torch.cuda.synchronize()
    for (seed, n_out, n_in, D, eps, lam), out in zip(cases, outs):
        q, p, w, pot, old = _case(seed, n_out, n_in, D)
        got = otgb.softmin_noalloc(q, p, w, pot, eps, lam, old=old, omega=0.5, out=out)
        want = otgb.softmin(ctx, q, p, w, pot, eps, lam, old=old, omega=0.5)
        g, h = got.cpu().numpy().astype(np.float64), want.cpu().numpy().astype(np.float64)
        err = np.max(np.abs(g - h)) / (np.max(np.abs(h)) + eps)
        assert err < TOL, (seed, err)
        # and directly against the FP64 oracle's softmin, blended as the call blends
        o = old.cpu().numpy().astype(np.float64)
        tilde = oracle.softmin(q.cpu().numpy(), p.cpu().numpy(), w.cpu().numpy(),
                               pot.cpu().numpy().astype(np.float64), eps, lam)
        ref = o + 0.5 * (tilde - o)
        err = np.max(np.abs(g - ref)) / (np.max(np.abs(ref)) + eps)
        assert err < TOL, (seed, "oracle", err)
    ctx.close()


def test_noalloc_rejects_oversized_problems():
    from paper_2107_02010_gb300 import otgb

    q, p, w, pot, _ = _case(3, 1_500_000, 16, 3)
    with pytest.raises(otgb.OtgbError) as e:
        otgb.softmin_noalloc(q, p, w, pot, 0.01)
    assert e.value.code == -1 and "scratch" in str(e.value)
