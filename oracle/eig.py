"""Smallest eigenpairs of the (normalized) Laplacian, Eq. (L_eigs) of Sec. II-B (oracle, FP64).

The paper names no eigensolver.  The oracle uses LAPACK's dense symmetric solver (``eigh``) for
small graphs and ARPACK in shift-invert mode around a small negative shift for larger ones.
Columns are returned in ascending eigenvalue order, each of unit norm.
Test infrastructure only.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla


def smallest_eigpairs(op, m, dense_max=6000, sigma=-1e-3, tol=1e-13, seed=0):
    N = op.shape[0]
    if N <= dense_max:
        lam, Q = np.linalg.eigh(op.toarray())
        return lam[:m].copy(), np.ascontiguousarray(Q[:, :m])
    v0 = np.random.default_rng(seed).standard_normal(N)
    lam, Q = spla.eigsh(op.tocsc(), k=m, sigma=sigma, which="LM", tol=tol, v0=v0)
    order = np.argsort(lam)
    return lam[order], np.ascontiguousarray(Q[:, order])
