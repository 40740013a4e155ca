"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws data: it holds none of the transport arithmetic, and
both the CUDA path and the CPU oracle read exactly the float32 arrays it
returns.  The paper's own data (HCP tractograms, the fiber atlas of Zhang et
al. 2018, MRtrix3 track-density maps) is not available, so these generators
stand in for it with the same shapes:

* ``rotated_cloud``   -- N points uniform in the unit cube and a rigidly moved,
  noisy copy (a small balanced 3-D problem).
* ``density_maps``    -- two track-density volumes, each a sum of Gaussian
  tubes around random cubic Bezier curves, thresholded to the strongest
  voxels; voxels become weighted Diracs (Section 2: track density maps).
* ``fiber_bundles``   -- fibers resampled to P=20 points drawn around bundle
  centrelines, flattened to R^{3P} and scaled by 1/sqrt(P) (Section 2: fiber
  encoding), with a bundle label per fiber.

Every generator takes explicit sizes so that tests can draw small instances
of the same families.
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _rotation(rng: np.random.Generator, max_deg: float) -> np.ndarray:
    axis = rng.normal(size=3)
    axis /= np.linalg.norm(axis)
    ang = np.deg2rad(rng.uniform(0.0, max_deg))
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + np.sin(ang) * K + (1 - np.cos(ang)) * (K @ K)


def rotated_cloud(n: int = 2000, m: int | None = None, seed: int = 0, max_deg: float = 15.0,
                  shift=(0.1, 0.0, 0.0), noise: float = 0.01):
    """x ~ U[0,1]^3 (n points); y = R (x - c) + c + shift + N(0, noise^2), c the
    cube centre, R a rotation about a uniform random axis by an angle drawn
    uniformly in [0, max_deg] degrees.  When m differs from n, y uses the first
    m points of a second uniform draw of size m moved the same way.  Uniform
    weights 1/n, 1/m.  Returns (x, a, y, b) as float32."""
    rng = _rng(seed)
    m = n if m is None else m
    x = rng.uniform(0.0, 1.0, size=(n, 3))
    R = _rotation(rng, max_deg)
    base = x if m == n else rng.uniform(0.0, 1.0, size=(m, 3))
    c = np.full(3, 0.5)
    y = (base - c) @ R.T + c + np.asarray(shift) + rng.normal(0.0, noise, size=(m, 3))
    a = np.full(n, 1.0 / n)
    b = np.full(m, 1.0 / m)
    return x.astype(np.float32), a.astype(np.float32), y.astype(np.float32), b.astype(np.float32)


def _bezier(ctrl: np.ndarray, t: np.ndarray) -> np.ndarray:
    """Cubic Bezier curve with 4 control points (4 x 3) at parameters t."""
    t = t[:, None]
    s = 1.0 - t
    return s ** 3 * ctrl[0] + 3 * s * s * t * ctrl[1] + 3 * s * t * t * ctrl[2] + t ** 3 * ctrl[3]


def _density_volume(rng, grid: int, n_tubes: int, tube_sigma: float, samples: int = 256):
    from scipy.spatial import cKDTree

    ax = np.arange(grid, dtype=np.float64) + 0.5
    vox = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), axis=-1).reshape(-1, 3)
    lo, hi = grid / 8.0, grid * 7.0 / 8.0
    dens = np.zeros(vox.shape[0])
    t = np.linspace(0.0, 1.0, samples)
    for _ in range(n_tubes):
        ctrl = rng.uniform(lo, hi, size=(4, 3))
        curve = _bezier(ctrl, t)
        dist, _ = cKDTree(curve).query(vox, k=1, distance_upper_bound=6.0 * tube_sigma)
        near = np.isfinite(dist)
        dens[near] += np.exp(-dist[near] ** 2 / (2.0 * tube_sigma ** 2))
    return vox, dens


def density_maps(grid: int = 64, n_tubes: int = 30, tube_sigma: float = 1.5, n_keep: int = 100_000,
                 seeds=(1, 2), masses=(1.0, 1.2)):
    """Two track-density volumes on a grid^3 lattice (voxel units).  Each is the
    sum over n_tubes Gaussian tubes exp(-dist(v, curve)^2 / (2 tube_sigma^2)),
    curves being cubic Beziers with control points uniform in the central
    [grid/8, 7 grid/8]^3 box.  The n_keep strongest voxels are kept; their
    centres become the Dirac locations and their densities, normalised to the
    given total masses, the weights.  Returns (x, a, y, b) float32."""
    out = []
    for seed, mass in zip(seeds, masses):
        out += list(density_map(grid, n_tubes, tube_sigma, n_keep, seed, mass))
    return tuple(out)


def density_map(grid: int = 64, n_tubes: int = 30, tube_sigma: float = 1.5, n_keep: int = 100_000, seed: int = 1,
                mass: float = 1.0):
    """One track-density volume of `density_maps` (same recipe, one seed).
    Returns (points float32 n x 3, weights float32)."""
    rng = _rng(seed)
    vox, dens = _density_volume(rng, grid, n_tubes, tube_sigma)
    k = min(n_keep, int(np.count_nonzero(dens > 0)))
    idx = np.argpartition(-dens, k - 1)[:k]
    idx.sort()
    w = dens[idx]
    w = w / w.sum() * mass
    return vox[idx].astype(np.float32), w.astype(np.float32)


def _resample_arclength(curve: np.ndarray, P: int) -> np.ndarray:
    seg = np.linalg.norm(np.diff(curve, axis=0), axis=1)
    s = np.concatenate([[0.0], np.cumsum(seg)])
    u = np.linspace(0.0, s[-1], P)
    return np.stack([np.interp(u, s, curve[:, d]) for d in range(3)], axis=1)


def bundle_centrelines(n_bundles: int = 20, box: float = 140.0, P: int = 20, seed: int = 3):
    """Centrelines of the bundles: cubic Beziers with control points uniform in
    [0, box]^3 (mm), resampled to P points equally spaced in arc length.
    Returns the control points (n_bundles x 4 x 3) used by fiber_bundles."""
    rng = _rng(seed)
    return rng.uniform(0.0, box, size=(n_bundles, 4, 3))


def fiber_bundles(n: int, seed: int, ctrl: np.ndarray | None = None, P: int = 20, perturb: float = 0.0,
                  offset_sigma: float = 2.0, point_sigma: float = 0.5, canonical: bool = True):
    """n fibers, each of P points, drawn from the bundles whose control points are
    `ctrl` (default: bundle_centrelines()).  Per tractogram the control points are
    perturbed by N(0, perturb^2) mm.  Each fiber picks a bundle uniformly, follows
    its centreline (P points equally spaced in arc length) moved by one per-fiber
    offset N(0, offset_sigma^2 I) plus per-point noise N(0, point_sigma^2 I); it is
    reversed at random and then canonicalised (reversed iff its first point is
    lexicographically greater than its last); canonical=False keeps the random
    orientation (the input of flip augmentation).  Features are the flattened 3P
    coordinates times 1/sqrt(P).  Returns (x float32 n x 3P, w float32 uniform
    1/n, labels int32)."""
    rng = _rng(seed)
    ctrl = bundle_centrelines(P=P) if ctrl is None else np.asarray(ctrl, np.float64)
    nb = ctrl.shape[0]
    if perturb > 0:
        ctrl = ctrl + rng.normal(0.0, perturb, size=ctrl.shape)
    t = np.linspace(0.0, 1.0, 512)
    lines = np.stack([_resample_arclength(_bezier(ctrl[k], t), P) for k in range(nb)])  # nb x P x 3
    lab = rng.integers(0, nb, size=n).astype(np.int32)
    fib = lines[lab] + rng.normal(0.0, offset_sigma, size=(n, 1, 3)) + rng.normal(0.0, point_sigma, size=(n, P, 3))
    flip = rng.random(n) < 0.5
    fib[flip] = fib[flip, ::-1]
    if not canonical:
        x = (fib.reshape(n, 3 * P) / np.sqrt(P)).astype(np.float32)
        return x, np.full(n, 1.0 / n, np.float32), lab
    first, last = fib[:, 0, :], fib[:, -1, :]
    gt = np.zeros(n, bool)
    decided = np.zeros(n, bool)
    for d in range(3):
        gt |= (~decided) & (first[:, d] > last[:, d])
        decided |= first[:, d] != last[:, d]
    fib[gt] = fib[gt, ::-1]
    x = (fib.reshape(n, 3 * P) / np.sqrt(P)).astype(np.float32)
    w = np.full(n, 1.0 / n, np.float32)
    return x, w, lab


def unit_mass(w: np.ndarray, bits: int = 30) -> np.ndarray:
    """Positive weights of total mass exactly 1 in float32 and in double: each
    weight a multiple of 2^-b (at least one unit), the units summing to 2^b
    (largest remainders rounded up), b <= bits the finest resolution at which
    every weight is exact in float32.  Balanced transport needs equal masses
    on both sides, which float32 rounding of w / sum(w) breaks."""
    w = np.asarray(w, np.float64)
    # a multiple of 2^-b below 2^(24 - b) is exact in float32
    wmax = w.max() / w.sum()
    while bits > 1 and wmax * 2.0 >= 2.0 ** (24 - bits):
        bits -= 1
    units = 1 << bits
    q = w / w.sum() * units
    k = np.maximum(np.floor(q), 1).astype(np.int64)
    rest = units - int(k.sum())
    order = np.argsort(-(q - np.floor(q)), kind="stable")
    if rest >= 0:
        k[order[:rest]] += 1
    else:  # too many rounded-up ones: take units back from the largest weights
        big = np.argsort(-k, kind="stable")
        k[big[:-rest]] -= 1
    assert k.sum() == units and k.min() >= 1
    out = (k / units).astype(np.float32)
    assert np.all(out.astype(np.float64) * units == k)  # exact in float32
    return out


def barycenter_maps(K: int = 5, grid: int = 64, n_keep: int = 20_000, upsample: int = 6, seed: int = 40):
    """Inputs of the track-density atlas (Section 2, "Track density atlas"; the
    Results section uses 5 maps of ~20,000 voxels and a barycenter initialised
    with their average density, up-sampled by a factor of 6): K maps from
    `density_maps` (30 tubes each, seeds seed..seed+K-1) with unit mass, and
    the initial barycenter: the union of their voxels weighted by the average
    density, each voxel replaced by `upsample` points drawn uniformly inside it.
    Returns (x0, a0, ys, bs); all weights have total mass exactly 1."""
    ys, bs = [], []
    for k in range(K):
        y, b = density_map(grid=grid, n_keep=n_keep, seed=seed + k)
        ys.append(y)
        bs.append(unit_mass(b))
    keys = np.concatenate([np.floor(y).astype(np.int64) @ np.array([grid * grid, grid, 1]) for y in ys])
    wts = np.concatenate(bs).astype(np.float64) / K
    uniq, inv = np.unique(keys, return_inverse=True)
    dens = np.bincount(inv, weights=wts)
    vox = np.stack([uniq // (grid * grid), (uniq // grid) % grid, uniq % grid], axis=1).astype(np.float64)
    rng = _rng(seed + 2 * K)
    x0 = (np.repeat(vox, upsample, axis=0) + rng.uniform(0.0, 1.0, size=(vox.shape[0] * upsample, 3)))
    a0 = unit_mass(np.repeat(dens, upsample))
    return x0.astype(np.float32), a0, ys, bs
