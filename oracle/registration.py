"""Random-walker registration (RWIR) pieces of the paper (oracle, FP64).  Test infrastructure
only.

Labels are displacement vectors (Sec. II-A: in RWIR the K probabilities of a voxel belong to K
potential displacements).  The graph is the image available offline (the fixed image; the
eigenvectors are precomputed on it).  With no landmark seeds, Eq. (rw_eq) reduces to
(L + gamma D) U = gamma D P in the normalized form, and the fast RW of Eq. (U_lin_comb) to
U-hat = Q Lambda_gamma (gamma Q^T P-hat): ``fastrw.fast_rw`` and ``exact.exact_rw`` with empty seed
arrays compute exactly that.

* ``displacement_labels``: the 3 x 3 x 3 displacement grid {-1, 0, 1}^3 (x fastest).
* ``patch_sad``: local dissimilarity of Sec. IV-B, the sum of absolute intensity differences
  between the fixed image at x and the moving image at x + d over a 5 x 5 x 5 patch; patch
  voxels outside the volume take the nearest voxel inside (reading: the paper is silent on
  borders).
* ``registration_priors``: P for the displacements, the negative exponential of the squared patch
  difference normalized to sum to 1 at each voxel (Sec. IV-B), by the log-sum-exp shift.
* ``expected_displacement``: the registration's displacement field, the expected displacement
  sum_k U_k d_k at each voxel (Sec. IV).
* ``registration_solve``: m from the priors by Eq. (g) (all labels evaluated: K = 27 is below
  r^d = 64, so the paper's one-in-r^d sampling keeps every label), the fast RW with no seeds,
  damped-Jacobi refinement.
"""
from __future__ import annotations

import numpy as np

from .adaptive import choose_m_from_priors
from .fastrw import fast_rw
from .refine import refine


def displacement_labels(radius=1, ndim=3):
    r = np.arange(-radius, radius + 1)
    grids = np.meshgrid(*([r] * ndim), indexing="ij")   # grids[0] slowest
    # x fastest: column 0 is dx
    return np.stack([g.ravel() for g in reversed(grids)], axis=1).astype(np.int64)


def _clamped(a, dims):
    return np.clip(a, 0, np.asarray(dims)[None, :] - 1)


def patch_sad(I_f, I_m, dims, disp, half=2, voxels=None):
    """SAD_k(x) over the (2 half + 1)^d patch, N x K (or len(voxels) x K for the listed flat
    voxel indices only).  I_f, I_m: flat arrays (x fastest)."""
    dims = tuple(int(k) for k in dims)
    F = np.asarray(I_f, dtype=np.float64).reshape(tuple(reversed(dims)))
    M = np.asarray(I_m, dtype=np.float64).reshape(tuple(reversed(dims)))
    idx = np.indices(tuple(reversed(dims))).reshape(len(dims), -1)[::-1].T   # (x, y, z) rows
    if voxels is not None:
        idx = idx[np.asarray(voxels)]
    N = idx.shape[0]
    out = np.zeros((N, len(disp)))
    offs = np.stack(np.meshgrid(*([np.arange(-half, half + 1)] * len(dims)), indexing="ij"),
                    axis=-1).reshape(-1, len(dims))
    for k, d in enumerate(disp):
        acc = np.zeros(N)
        for o in offs:
            y = _clamped(idx + o[None, :], dims)
            yd = _clamped(idx + o[None, :] + np.asarray(d)[None, :], dims)
            fv = F[tuple(y[:, j] for j in reversed(range(len(dims))))]
            mv = M[tuple(yd[:, j] for j in reversed(range(len(dims))))]
            acc += np.abs(fv - mv)
        out[:, k] = acc
    return out


def registration_priors(I_f, I_m, dims, disp, half=2, voxels=None):
    s = patch_sad(I_f, I_m, dims, disp, half, voxels)
    logp = -s * s
    logp -= logp.max(axis=1, keepdims=True)
    P = np.exp(logp)
    return P / P.sum(axis=1, keepdims=True)


def expected_displacement(U, disp):
    return np.asarray(U) @ np.asarray(disp, dtype=np.float64)


def registration_solve(g, Q, lam, P, gamma=1.0, m=0, m_step=10, eps=0.1, refine_steps=3,
                       omega=0.8):
    """Returns dict(U, m, g)."""
    none = np.zeros(0, dtype=np.int64)
    K = P.shape[1]
    gv = None
    if m == 0:
        m, gv, _, _ = choose_m_from_priors(g, Q, P, Q.shape[1], m_step, eps)
    U = fast_rw(g, Q[:, :m], lam[:m], none, none, K, P, gamma)
    if refine_steps > 0:
        U, _ = refine(g, U, none, none, K, P, gamma, refine_steps, omega=omega)
    return dict(U=U, m=m, g=gv)
