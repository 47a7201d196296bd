"""Basic random walker: the linear system Eq. (rw_eq) of Sec. II-A (oracle, FP64).

Unnormalized (Eq. rw_eq as printed):   (L_n + gamma I) U_n = gamma P_n - B^T U_s
Normalized (Sec. II-C): substituting U-hat = D^{1/2} U and P-hat = D^{1/2} P into Eq. (rw_eq)
written with L-hat gives (L-hat_n + gamma I) U-hat_n = gamma P-hat_n - B-hat^T U-hat_s; multiplying
by D_n^{1/2} on the left turns it into the equivalent system in U,
                                       (L_n + gamma D_n) U_n = gamma D_n P_n - B^T U_s,
which is what is solved here.  U_s is the one-hot label matrix of the seeds (Eq. U_block).
Block notation as in Eq. (LP_block): s = seeded rows, n = the others.
Test infrastructure only.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def onehot(labels, n_labels):
    U = np.zeros((len(labels), n_labels))
    U[np.arange(len(labels)), labels] = 1.0
    return U


def split(N, seed_idx):
    mask = np.zeros(N, dtype=bool)
    mask[seed_idx] = True
    return np.nonzero(~mask)[0]


def system(g, seed_idx, seed_lab, n_labels, P, gamma, normalized=True):
    """Returns (A, rhs, n): A = L_n + gamma D~_n, rhs = gamma D~_n P_n - B^T U_s."""
    n = split(g.N, seed_idx)
    L = g.L
    Ln = L[n][:, n]
    B = L[seed_idx][:, n]  # S x (N - S), Eq. (LP_block)
    Us = onehot(seed_lab, n_labels)
    Dt = g.d[n] if normalized else np.ones(n.size)
    A = (Ln + gamma * sp.diags(Dt)).tocsc()
    rhs = -(B.T @ Us)
    if gamma > 0:
        rhs = rhs + gamma * Dt[:, None] * P[n]
    return A, np.asarray(rhs), n


def exact_rw(g, seed_idx, seed_lab, n_labels, P, gamma, normalized=True, method="splu",
             tol=1e-12, maxiter=200000):
    """U (N x n_labels): seeds one-hot, the rest from Eq. (rw_eq) by a sparse direct solve
    (SuperLU) or by FP64 conjugate gradients to ||r|| <= tol ||b||."""
    A, rhs, n = system(g, seed_idx, seed_lab, n_labels, P, gamma, normalized)
    if method == "splu":
        lu = spla.splu(A)
        Un = lu.solve(rhs)
    elif method == "cg":
        Un = np.zeros_like(rhs)
        for k in range(rhs.shape[1]):
            x, info = spla.cg(A, rhs[:, k], rtol=tol, atol=0.0, maxiter=maxiter)
            if info != 0:
                raise RuntimeError("CG did not converge")
            Un[:, k] = x
    else:
        raise ValueError(method)
    U = np.zeros((g.N, n_labels))
    U[seed_idx] = onehot(seed_lab, n_labels)
    U[n] = Un
    return U
