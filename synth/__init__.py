"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only builds inputs: images shaped like the paper's data (Sec. IV-A: cardiac CT,
blood-cell, thigh MR volumes, which are not available here), seed sets, regions of interest,
edge lists and a generic orthonormal basis.  It holds none of the random walker's arithmetic
(no edge weights, no Laplacian, no solves), so both the CUDA path and the oracle can consume
its outputs without sharing any computation.

Conventions
-----------
* ``dims`` is ``(X, Y)`` or ``(X, Y, Z)``; a voxel (x, y, z) has linear index
  ``x + X * (y + Y * z)``.  Images are flat ``float64`` arrays of length ``N = prod(dims)``.
* An edge id is ``axis * N + i``: the edge from voxel ``i`` to ``i + stride[axis]``
  (``stride = (1, X, X*Y)``); it exists when voxel ``i`` is not on the last slice along ``axis``.
* Seeds are two int32 arrays: voxel indices and labels in ``[0, n_labels)``.
"""
from __future__ import annotations

import numpy as np
from scipy import ndimage

BASE_SEED = 160704174  # + config index, for every generator below


def strides(dims):
    s = [1]
    for k in dims[:-1]:
        s.append(s[-1] * int(k))
    return tuple(s)


def grid_coords(dims):
    """Per-axis integer coordinates of every voxel, in linear-index order."""
    N = int(np.prod(dims))
    i = np.arange(N, dtype=np.int64)
    out = []
    for k in dims:
        out.append(i % k)
        i = i // k
    return out


def _as_grid(a, dims):
    # numpy C-order array indexed [z, y, x] (or [y, x]) whose flattening matches the linear index
    return a.reshape(tuple(reversed(dims)))


# ----------------------------------------------------------------------------- images


def closed_curve_image(size=64, seed=BASE_SEED + 0, inside=0.7, outside=0.3, sigma=0.05):
    """Two piecewise-constant regions split by a random smooth closed curve, plus noise.

    r(theta) = R0 (1 + sum_{k=2..4} a_k cos(k theta + phi_k)), R0 = 0.3 size, centre
    (size/2, size/2) + U(-3, 3)^2, a_k ~ U(-0.1, 0.1), phi_k ~ U(0, 2 pi).  Inside ``inside``,
    outside ``outside``, Gaussian noise ``sigma``, clipped to [0, 1].
    Returns (J, dims, truth) with truth = 1 inside, 0 outside (int32).
    """
    rng = np.random.default_rng(seed)
    dims = (size, size)
    x, y = grid_coords(dims)
    c = size / 2.0 + rng.uniform(-3, 3, size=2)
    a = rng.uniform(-0.1, 0.1, size=3)
    phi = rng.uniform(0, 2 * np.pi, size=3)
    R0 = 0.3 * size
    dx, dy = x - c[0], y - c[1]
    th = np.arctan2(dy, dx)
    r = R0 * (1 + sum(a[k] * np.cos((k + 2) * th + phi[k]) for k in range(3)))
    truth = (np.hypot(dx, dy) < r).astype(np.int32)
    J = np.where(truth == 1, inside, outside) + sigma * rng.standard_normal(truth.size)
    return np.clip(J, 0.0, 1.0), dims, truth


def voronoi_image(X=512, Y=512, n_regions=4, sigma=0.05, seed=BASE_SEED + 1):
    """Voronoi regions around U([0,X)x[0,Y)) sites (ties -> lowest index), region means U(0,1),
    Gaussian noise ``sigma``, clipped to [0, 1].  Returns (J, dims, truth)."""
    rng = np.random.default_rng(seed)
    dims = (X, Y)
    sites = rng.uniform(0, 1, size=(n_regions, 2)) * np.array([X, Y])
    means = rng.uniform(0, 1, size=n_regions)
    x, y = grid_coords(dims)
    d2 = (x[:, None] - sites[None, :, 0]) ** 2 + (y[:, None] - sites[None, :, 1]) ** 2
    truth = np.argmin(d2, axis=1).astype(np.int32)  # argmin returns the lowest index on ties
    J = means[truth] + sigma * rng.standard_normal(truth.size)
    return np.clip(J, 0.0, 1.0), dims, truth


def ellipsoid_volume(n=128, seed=BASE_SEED + 2, inside=0.65, outside=0.25, sigma=0.08):
    """Randomly rotated ellipsoid in a background: centre ~ U([3n/8, 5n/8]^3), semi-axes
    ~ U(3n/16, 11n/32), inside 0.65 / background 0.25, noise 0.08, clipped to [0, 1]."""
    rng = np.random.default_rng(seed)
    dims = (n, n, n)
    c = rng.uniform(3 * n / 8, 5 * n / 8, size=3)
    ax = rng.uniform(3 * n / 16, 11 * n / 32, size=3)
    # random rotation from the QR of a Gaussian matrix (sign-fixed)
    A = rng.standard_normal((3, 3))
    Rq, Rr = np.linalg.qr(A)
    Rq = Rq * np.sign(np.diag(Rr))[None, :]
    x, y, z = grid_coords(dims)
    p = np.stack([x - c[0], y - c[1], z - c[2]], axis=1).astype(np.float64)
    p = p @ Rq
    truth = (((p / ax) ** 2).sum(axis=1) < 1.0).astype(np.int32)
    J = np.where(truth == 1, inside, outside) + sigma * rng.standard_normal(truth.size)
    return np.clip(J, 0.0, 1.0), dims, truth


def smooth_random_image(dims, seed, smooth=2.0, sigma=0.0):
    """Smoothed random field in [0,1] plus optional noise (a generic test image)."""
    rng = np.random.default_rng(seed)
    g = ndimage.gaussian_filter(rng.standard_normal(tuple(reversed(dims))), smooth)
    g = (g - g.min()) / max(g.max() - g.min(), 1e-12)
    J = g.ravel() + sigma * rng.standard_normal(g.size)
    return np.clip(J, 0.0, 1.0)


# ----------------------------------------------------------------------------- seeds


def sample_seeds(truth, dims, per_label, min_dist=2, seed=BASE_SEED, n_labels=None):
    """``per_label`` seeds per label, drawn without replacement from voxels whose Chebyshev
    distance to every voxel of another label is >= ``min_dist``.  Returns (idx, lab) int32,
    ordered label by label."""
    rng = np.random.default_rng(seed)
    n_labels = int(truth.max()) + 1 if n_labels is None else n_labels
    g = _as_grid(truth, dims)
    size = 2 * (min_dist - 1) + 1
    same = (ndimage.maximum_filter(g, size=size, mode="nearest") == g) & (
        ndimage.minimum_filter(g, size=size, mode="nearest") == g)
    ok = same.ravel()
    idx, lab = [], []
    for k in range(n_labels):
        cand = np.nonzero(ok & (truth == k))[0]
        if cand.size < per_label:
            raise ValueError(f"label {k}: only {cand.size} eligible voxels")
        pick = rng.choice(cand, size=per_label, replace=False)
        idx.append(pick)
        lab.append(np.full(per_label, k))
    return np.concatenate(idx).astype(np.int32), np.concatenate(lab).astype(np.int32)


# ----------------------------------------------------------------------------- basis


def dct_basis(dims, m, dtype=np.float64):
    """First ``m`` orthonormal DCT-II product vectors on the grid, ordered by increasing
    sum_axis (k_axis / n_axis)^2 (ties by linear order of the frequency tuple).

    A generic orthonormal N x m basis of smooth grid functions, node-major (row i = voxel i).
    It is an input for tests of the online solve at sizes where a dense eigensolver is out of
    reach: the fast random walker is defined for any orthonormal Q.
    """
    dims = tuple(int(k) for k in dims)
    # candidate frequency tuples: enough along each axis to contain the m lowest
    kmax = [min(n, int(np.ceil(np.sqrt(m) * 2)) + 2) for n in dims]
    grids = np.meshgrid(*[np.arange(k) for k in kmax], indexing="ij")
    freq = np.stack([g.ravel() for g in grids], axis=1)
    key = sum((freq[:, a] / dims[a]) ** 2 for a in range(len(dims)))
    order = np.lexsort(tuple(freq[:, a] for a in reversed(range(len(dims)))) + (key,))
    freq = freq[order[:m]]
    coords = grid_coords(dims)
    N = int(np.prod(dims))
    Q = np.ones((N, m), dtype=dtype)
    for a, n in enumerate(dims):
        k = freq[:, a][None, :]
        c = np.cos(np.pi * (coords[a][:, None] + 0.5) * k / n)
        scale = np.where(k == 0, np.sqrt(1.0 / n), np.sqrt(2.0 / n))
        Q *= (c * scale).astype(dtype)
    return Q


def random_orthonormal(N, m, seed, dtype=np.float64):
    rng = np.random.default_rng(seed)
    q, r = np.linalg.qr(rng.standard_normal((N, m)))
    return (q * np.sign(np.diag(r))[None, :]).astype(dtype)


# ----------------------------------------------------------------------------- edges / ROI


def roi_box(center, size, dims):
    """Half-open box [lo, hi) per axis of edge length ``size`` centred on ``center``, clipped."""
    lo = [max(0, int(c) - size // 2) for c in center]
    hi = [min(int(n), l + size) for l, n in zip(lo, dims)]
    lo = [h - size if h - l < size and h - size >= 0 else l for l, h in zip(lo, hi)]
    return tuple(lo), tuple(hi)


def roi_edge_ids(dims, lo, hi):
    """Ids of all forward edges with both end voxels inside the box [lo, hi)."""
    N = int(np.prod(dims))
    st = strides(dims)
    coords = grid_coords(dims)
    inside = np.ones(N, dtype=bool)
    for a in range(len(dims)):
        inside &= (coords[a] >= lo[a]) & (coords[a] < hi[a])
    ids = []
    for a in range(len(dims)):
        ok = inside & (coords[a] < hi[a] - 1)
        ids.append(a * N + np.nonzero(ok)[0])
    return np.concatenate(ids).astype(np.int64)


def boundary_voxel(truth, dims, seed):
    """A random voxel of label 1 that has a 6/4-neighbour of another label."""
    rng = np.random.default_rng(seed)
    g = _as_grid(truth, dims)
    edge = (ndimage.maximum_filter(g, size=3) != ndimage.minimum_filter(g, size=3)) & (g == 1)
    cand = np.nonzero(edge.ravel())[0]
    i = int(rng.choice(cand))
    return tuple(int(c[i]) for c in grid_coords(dims))


def pick_edges(ids, fraction, seed):
    rng = np.random.default_rng(seed)
    k = int(round(fraction * ids.size))
    return np.sort(rng.choice(ids, size=k, replace=False)).astype(np.int64)


# ----------------------------------------------------------------------------- registration


def registration_pair(n=96, seed=BASE_SEED + 5, max_disp=2.0, smooth=3.0, sigma=0.03,
                      field_smooth=8.0):
    """Fixed / moving volumes of side n: fixed is a smoothed random field in [0, 1] plus noise
    sigma; the displacement u (N x 3, components x, y, z) is a Gaussian-smoothed random vector
    field scaled so that max |u| = max_disp voxels; moving(x) = fixed(x + u(x)) by trilinear
    interpolation (nearest voxel outside), plus its own noise.  Returns (fixed, moving, dims, u)
    as flat float64 arrays, x fastest."""
    rng = np.random.default_rng(seed)
    dims = (n, n, n)
    base = ndimage.gaussian_filter(rng.standard_normal((n, n, n)), smooth)
    base = (base - base.min()) / max(base.max() - base.min(), 1e-12)
    comp = [ndimage.gaussian_filter(rng.standard_normal((n, n, n)), field_smooth)
            for _ in range(3)]                      # x, y, z components, arrays indexed [z, y, x]
    mag = np.sqrt(sum(c * c for c in comp))
    scale = max_disp / max(mag.max(), 1e-12)
    comp = [c * scale for c in comp]
    z, y, x = np.indices((n, n, n), dtype=np.float64)
    coords = [z + comp[2], y + comp[1], x + comp[0]]
    moving = ndimage.map_coordinates(base, coords, order=1, mode="nearest")
    fixed = np.clip(base + sigma * rng.standard_normal(base.shape), 0.0, 1.0)
    moving = np.clip(moving + sigma * rng.standard_normal(base.shape), 0.0, 1.0)
    u = np.stack([c.ravel() for c in comp], axis=1)
    return fixed.ravel(), moving.ravel(), dims, u
