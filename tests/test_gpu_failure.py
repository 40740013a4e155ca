"""Failure detection without a GPU fault: a bounded device wait that runs out.

Every spin-wait of the kernels (tensor-core completions, tile barriers) has an
iteration limit after which the kernel flags an error word and returns, and
the solve reports OTGB_ETIMEOUT instead of hanging.  The test hook
params.debug_wait_probe makes one such wait run out on purpose (a device word
that nothing writes; about a millisecond of polling): the call must come back
with ETIMEOUT, and the same context must then solve normally."""
import numpy as np
import pytest
import torch

import oracle
from paper_2107_02010_gb300 import synth

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_etimeout_and_context_stays_usable():
    from paper_2107_02010_gb300 import otgb

    x, a, y, b = synth.rotated_cloud(300, 260, seed=1)
    T = lambda v: torch.from_numpy(v).cuda()
    X, A, Y, B = T(x), T(a), T(y), T(b)
    ctx = otgb.Context()
    p = otgb.default_params(blur=0.1, reach=0.5, debug_wait_probe=1)
    with pytest.raises(otgb.OtgbError) as e:
        otgb.sinkhorn_divergence(ctx, X, A, Y, B, p)
    assert e.value.code == -6 and "wait" in str(e.value)
    # the context is still usable: the same problem without the probe converges
    # to the oracle's divergence
    p = otgb.default_params(blur=0.1, reach=0.5, tol=1e-9)
    out = otgb.sinkhorn_divergence(ctx, X, A, Y, B, p)
    assert out["status"] == 0
    ref = oracle.sinkhorn(x, a, y, b, blur=0.1, reach=0.5, scaling=0.5, tol=1e-12, max_iters=20000)
    assert abs(out["S"] - ref["S"]) <= 1e-5 * abs(ref["S"])
    ctx.close()
