"""Refinement of an approximate solution of Eq. (rw_eq) (oracle, FP64).  The paper has no
refinement step; it recovers accuracy lost to low-precision storage of the basis.
Test infrastructure only.

Two refiners are restated:
* ``jacobi``: k damped-Jacobi steps on the residual, x <- x + omega diag(A)^{-1} (b - A x).
  Linear in the starting point, and its iteration matrix has max-norm
  |1 - omega| + omega / (1 + gamma) <= 1 for 0 < omega <= 1 (rows of diag(A)^{-1} A), so a
  perturbation of the start never grows in max-norm.  This is the default.
* ``pcg``: k steps of Jacobi-preconditioned conjugate gradients (each column its own
  recurrence).  Its step lengths depend on the start, so a small perturbation of the start can
  grow; it is used to refine to a tolerance against the exact solve.

The system is the one the fast RW approximates: with the normalized Laplacian (Sec. II-C)
    (L-hat_n + gamma I) U-hat_n = gamma P-hat_n - B-hat^T U-hat_s,   U = D^{-1/2} U-hat,
otherwise Eq. (rw_eq) itself.  The preconditioner is diag(A) (constant 1 + gamma in the
normalized form, where Jacobi-PCG reduces to plain CG).  Every label column runs its own CG
recurrence (its own step lengths), starting from the given U_n.
"""
from __future__ import annotations

import numpy as np

from .exact import onehot, split


def hat_system(g, seed_idx, seed_lab, n_labels, P, gamma, normalized=True):
    op = g.operator(normalized)
    sc = np.sqrt(g.d) if normalized else np.ones(g.N)
    n = split(g.N, seed_idx)
    s = np.asarray(seed_idx)
    A = (op[n][:, n] + gamma * _eye(n.size)).tocsr()
    B = op[s][:, n]
    Us_hat = sc[s, None] * onehot(seed_lab, n_labels)
    b = -np.asarray(B.T @ Us_hat)
    if gamma > 0:
        b = b + gamma * sc[n, None] * P[n]
    return A, b, n, sc


def _eye(k):
    import scipy.sparse as sp
    return sp.identity(k, format="csr")


def pcg_steps(A, b, x0, steps):
    """k Jacobi-PCG steps for every column; returns x_k and the residual norms per step."""
    x = np.array(x0, dtype=np.float64, copy=True)
    Minv = 1.0 / A.diagonal()
    r = b - A @ x
    z = Minv[:, None] * r
    p = z.copy()
    rz = np.einsum("ij,ij->j", r, z)
    hist = [np.linalg.norm(r, axis=0)]
    for _ in range(steps):
        Ap = A @ p
        pAp = np.einsum("ij,ij->j", p, Ap)
        a = np.where(pAp > 0, rz / np.where(pAp > 0, pAp, 1.0), 0.0)
        x += a[None, :] * p
        r -= a[None, :] * Ap
        z = Minv[:, None] * r
        rz_new = np.einsum("ij,ij->j", r, z)
        beta = np.where(rz > 0, rz_new / np.where(rz > 0, rz, 1.0), 0.0)
        p = z + beta[None, :] * p
        rz = rz_new
        hist.append(np.linalg.norm(r, axis=0))
    return x, hist


def jacobi_steps(A, b, x0, steps, omega=0.8):
    """k damped-Jacobi steps; returns x_k and the residual norms per step."""
    x = np.array(x0, dtype=np.float64, copy=True)
    Dinv = 1.0 / A.diagonal()
    hist = []
    for _ in range(steps):
        r = b - A @ x
        hist.append(np.linalg.norm(r, axis=0))
        x += omega * Dinv[:, None] * r
    hist.append(np.linalg.norm(b - A @ x, axis=0))
    return x, hist


def refine(g, U0, seed_idx, seed_lab, n_labels, P, gamma, steps, normalized=True,
           method="jacobi", omega=0.8):
    """Start from U0 (N x l, e.g. the fast RW), run ``steps`` refinement steps on the hat
    system, return (U, residual-norm history)."""
    A, b, n, sc = hat_system(g, seed_idx, seed_lab, n_labels, P, gamma, normalized)
    x0 = sc[n, None] * U0[n]
    if method == "jacobi":
        x, hist = jacobi_steps(A, b, x0, steps, omega)
    elif method == "pcg":
        x, hist = pcg_steps(A, b, x0, steps)
    else:
        raise ValueError(method)
    U = np.array(U0, dtype=np.float64, copy=True)
    U[seed_idx] = onehot(seed_lab, n_labels)
    U[n] = x / sc[n, None]
    return U, hist
