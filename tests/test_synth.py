"""The seeded input generators against the recipe they state: shapes, dtypes,
masses, determinism, and the geometry each one promises (a rigid motion plus
noise for the rotated cloud, lattice voxels with normalised densities for the
track-density maps, canonically oriented fibers scaled by 1/sqrt(P) for the
fiber bundles)."""
import numpy as np
import pytest

from paper_2107_02010_gb300 import synth


def test_rotated_cloud_is_a_rigid_motion_plus_noise():
    x, a, y, b = synth.rotated_cloud(2000, seed=0)
    assert x.shape == y.shape == (2000, 3) and x.dtype == y.dtype == np.float32
    assert abs(a.sum() - 1.0) < 1e-5 and abs(b.sum() - 1.0) < 1e-5
    assert x.min() >= 0.0 and x.max() <= 1.0
    # Kabsch: the best rotation and shift between x and y leave a residual at the noise level
    X = x.astype(np.float64) - x.mean(0)
    Y = y.astype(np.float64) - y.mean(0)
    U, _, Vt = np.linalg.svd(X.T @ Y)
    d = np.sign(np.linalg.det(U @ Vt))
    R = (U @ np.diag([1.0, 1.0, d]) @ Vt).T
    res = Y - X @ R.T
    assert np.sqrt((res ** 2).sum(1).mean()) < 0.01 * np.sqrt(3) * 1.1  # N(0, 0.01^2) per coordinate
    assert np.linalg.det(R) > 0.99
    angle = np.degrees(np.arccos(np.clip((np.trace(R) - 1.0) / 2.0, -1.0, 1.0)))
    assert angle <= 15.0 + 0.5
    # the motion is about the cube centre, then shifted by (0.1, 0, 0)
    c = np.full(3, 0.5)
    shift = y.astype(np.float64).mean(0) - ((x.astype(np.float64).mean(0) - c) @ R.T + c)
    assert np.allclose(shift, [0.1, 0.0, 0.0], atol=2e-3)
    x2, _, y2, _ = synth.rotated_cloud(2000, seed=0)
    assert np.array_equal(x, x2) and np.array_equal(y, y2)


def test_density_maps_voxels_and_masses():
    x, a, y, b = synth.density_maps(grid=24, n_tubes=5, n_keep=500)
    for pts, w, mass in ((x, a, 1.0), (y, b, 1.2)):
        assert pts.shape == (500, 3) and pts.dtype == np.float32 and w.dtype == np.float32
        assert np.all(w > 0) and abs(float(w.sum(dtype=np.float64)) - mass) < 1e-5 * mass
        # voxel centres of the 24^3 lattice, no voxel twice
        assert np.allclose(pts - np.floor(pts), 0.5) and pts.min() > 0 and pts.max() < 24
        assert len(np.unique(pts, axis=0)) == 500
    assert not np.array_equal(x, y)  # two volumes (seeds 1 and 2)
    x2, a2, _, _ = synth.density_maps(grid=24, n_tubes=5, n_keep=500)
    assert np.array_equal(x, x2) and np.array_equal(a, a2)


@pytest.mark.parametrize("P", [20, 7])
def test_fiber_bundles_layout_orientation_and_labels(P):
    ctrl = synth.bundle_centrelines(P=P)
    x, w, lab = synth.fiber_bundles(3000, seed=4, ctrl=ctrl, P=P, perturb=3.0)
    assert x.shape == (3000, 3 * P) and x.dtype == np.float32
    assert np.allclose(w, 1.0 / 3000) and lab.dtype == np.int32
    assert lab.min() >= 0 and lab.max() < ctrl.shape[0] and len(np.unique(lab)) == ctrl.shape[0]
    fib = x.astype(np.float64).reshape(3000, P, 3) * np.sqrt(P)  # back to millimetres
    # inside the 140 mm box up to the perturbation and the per-fiber noise
    assert fib.min() > -40.0 and fib.max() < 180.0
    # canonical orientation: the first point is not lexicographically greater than the last
    first, last = fib[:, 0], fib[:, -1]
    for i in range(3000):
        assert tuple(first[i]) <= tuple(last[i]), i
    # fibers of one bundle follow one centreline: their points are near the bundle's mean fiber
    for k in range(3):
        f = fib[lab == k]
        spread = np.sqrt(((f - f.mean(0)) ** 2).sum(-1).mean())
        assert spread < 4.0, (k, spread)
    x2, _, lab2 = synth.fiber_bundles(3000, seed=4, ctrl=ctrl, P=P, perturb=3.0)
    assert np.array_equal(x, x2) and np.array_equal(lab, lab2)


def test_unit_mass_is_exact_in_float32():
    r = np.random.default_rng(5)
    for n in (1, 7, 1000, 300_000):
        w = synth.unit_mass(r.uniform(0.1, 2.0, n))
        assert w.dtype == np.float32 and np.all(w > 0)
        assert w.astype(np.float64).sum() == 1.0


def test_barycenter_maps_recipe():
    # K unit-mass maps of n_keep voxels; the initial support is every voxel of
    # the union, up-sampled, with the average density as weight
    x0, a0, ys, bs = synth.barycenter_maps(K=3, grid=24, n_keep=400, upsample=4)
    assert len(ys) == 3 and all(y.shape == (400, 3) for y in ys)
    assert all(b.astype(np.float64).sum() == 1.0 for b in bs)
    assert a0.astype(np.float64).sum() == 1.0
    assert x0.shape[0] % 4 == 0
    union = np.unique(np.concatenate([np.floor(y) for y in ys]), axis=0)
    assert x0.shape[0] == 4 * union.shape[0]
    cells = np.unique(np.floor(x0), axis=0)
    np.testing.assert_array_equal(cells, union)
