"""Writes tests/golden/fibers_60d_2000x1800.npz: the FP64 oracle's converged
solve of one seeded 60-D fiber problem (the fiber-bundle generator of the
package's synthetic inputs, 20 bundles, subject of 2000 fibers perturbed by
3 mm against an atlas of 1800 fibers; p = 2, blur 2 mm, reach 20 mm, q 0.5).

The oracle iterates the plain averaged loop of the Algorithm (Section 2) until
max |new - old| / eps < 1e-12.  Twenty nearly separate bundles under the
unbalanced damping lambda = 1/(1 + (2/20)^2) contract at about 0.995 per step,
so the solve takes thousands of steps: too slow to repeat inside a test, hence
this stored result.  Only oracle/ and the seeded input generator are called.

    OMP_NUM_THREADS=8 python tests/golden/make_fibers_60d.py
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2107_02010_gb300 import synth  # noqa: E402

N, M = 2000, 1800
BLUR, REACH, Q = 2.0, 20.0, 0.5
TOL = 1e-12
OUT = os.path.join(HERE, "fibers_60d_2000x1800.npz")


def inputs():
    ctrl = synth.bundle_centrelines()
    x, a, _ = synth.fiber_bundles(N, seed=4, ctrl=ctrl, perturb=3.0)
    y, b, lab = synth.fiber_bundles(M, seed=5, ctrl=ctrl)
    return x, a, y, b, lab


def main():
    x, a, y, b, _ = inputs()
    t0 = time.time()
    r = oracle.sinkhorn(x, a, y, b, blur=BLUR, reach=REACH, scaling=Q, tol=TOL, max_iters=200000)
    dt = time.time() - t0
    assert r["converged"], r["delta"]
    np.savez_compressed(OUT, f=r["f"], g=r["g"], a=r["a"], b=r["b"], S=np.float64(r["S"]),
                        iters=np.int64(r["iters"]), delta=np.float64(r["delta"]),
                        recipe=np.array("fiber_bundles(%d, seed=4, perturb=3) vs fiber_bundles(%d, seed=5); "
                                        "blur %g, reach %g, q %g, oracle tol %g" % (N, M, BLUR, REACH, Q, TOL)))
    print("S = %.15g, %d steps, %.0f s, %d threads -> %s" % (r["S"], r["iters"], dt, oracle.threads(), OUT))


if __name__ == "__main__":
    main()
