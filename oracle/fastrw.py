"""Fast random walker by eigenvector precomputation, Sec. II-B (oracle, FP64).

Given m orthonormal columns Q (N x m) and values lam (m) — eigenpairs of L or L-hat, or the
Rayleigh-quotient values of Sec. III-B — with Lambda_gamma = (Lambda + gamma I)^{-1}:

  E   = Q Lambda_gamma Q^T                                    Eq. (E_def)
  E_s = Q_s Lambda_gamma Q_s^T, R = Q_s Lambda_gamma Q_n^T, E_n = Q_n Lambda_gamma Q_n^T
                                                               Eq. (E_block)
  (I - B R^T) F_s = L_s U_s + gamma (U_s + B E_n P_n)          Eq. (Fs)
  U_n = R^T F_s + gamma E_n P_n                                Eq. (Fs_2)
      = Q_n Lambda_gamma (Q_s^T F_s + gamma Q_n^T P_n)         Eq. (U_lin_comb)

In the normalized formulation (Sec. II-C, the default) L is replaced by L-hat, U_s by
U-hat_s = D_s^{1/2} U_s and P by P-hat = D^{1/2} P; the result is U-hat and U = D^{-1/2} U-hat.

``fast_rw`` is the factored form (X = B Q_n, Z = Q_n^T P_n; never forms an N x N matrix).
``fast_rw_dense`` is a second, independent restatement for small N that forms E explicitly and
takes its blocks literally.  Test infrastructure only.

Parity note: at m < N the result is an approximation.  Its pins are m = N (equality with the
exact solve, from E F = U, Eq. pseudo_E), the agreement of the two restatements, the row-sum
property when D^{1/2} 1 lies in span(Q), and two closed forms at m < N: exactness whenever the
exact solution lies in span(Q) (a graph of two components with consistent seeds and priors),
and, without seeds, the spectral filter sum_i gamma / (lambda_i + gamma) q_i q_i^T P of priors
inside span(Q) on the unweighted grid, whose eigenvectors are DCT-II products.  Parity
unpinned: the value at m < N when the exact solution lies outside span(Q) (the paper judges
that approximation only by segmentation quality).

gamma = 0 (no priors; Sec. II-B, the paragraph after Eq. Fs).  L-hat is singular: its null vector
is g = D^{1/2} 1 / ||D^{1/2} 1|| (g = 1 / sqrt(N) with L), E becomes the pseudo-inverse and
E L-hat = I - g g^T, so E F = U - g c with c = g^T U-hat (the column sums the paper names).
Reading: the basis column with the smallest value (column 0) is taken as the null direction and
replaced by the exact g; the other columns are projected orthogonal to g,
Q' = (I - g g^T) Q[:, 1:m], Lambda' = diag(lam[1:m]), E = Q' Lambda'^{-1} Q'^T, R, E_s, E_n its
blocks.  With F_n = 0 (gamma = 0), the unseeded rows of E F = U - g c and Eq. (Fs_1) give
  U-hat_n = R^T F_s + g_n c,
  (I - B R^T) F_s - (B g_n) c = L-hat_s U-hat_s,
and c = g_s^T U-hat_s + g_n^T U-hat_n gives the border row
  -(g_n^T R^T) F_s + (1 - g_n^T g_n) c = g_s^T U-hat_s.
``fast_rw_gamma0`` solves this (S + 1) x (S + 1) system in factored form,
``fast_rw_gamma0_dense`` from the explicit E; ``gamma0_basis`` is the basis [g, Q'] they use
(and on which m is chosen by Eq. alpha_1 at gamma = 0).  Pins: exact at m = N, constants
reproduced exactly at any m, rows summing to 1, the two restatements, invariance to g-components
added to the stored columns.
"""
from __future__ import annotations

import numpy as np

from .exact import onehot, split


def _hat(g, normalized):
    op = g.operator(normalized)
    sc = np.sqrt(g.d) if normalized else np.ones(g.N)
    return op, sc


def fast_rw(g, Q, lam, seed_idx, seed_lab, n_labels, P, gamma, normalized=True,
            return_parts=False):
    """Factored Eqs. (Fs), (U_lin_comb).  P may be None when gamma == 0 (not recommended:
    the gamma = 0 correction of Sec. II-B is not applied here)."""
    op, sc = _hat(g, normalized)
    n = split(g.N, seed_idx)
    s = np.asarray(seed_idx)
    Q = np.asarray(Q, dtype=np.float64)
    lg = 1.0 / (np.asarray(lam, dtype=np.float64) + gamma)        # diag of Lambda_gamma
    Qs, Qn = Q[s], Q[n]
    Us_hat = sc[s, None] * onehot(seed_lab, n_labels)
    Ls = op[s][:, s]
    B = op[s][:, n]
    X = np.asarray(B @ Qn)                                          # S x m
    if gamma > 0:
        Z = Qn.T @ (sc[n, None] * P[n])                             # m x l  (Q_n^T P-hat_n)
    else:
        Z = np.zeros((Q.shape[1], n_labels))
    rhs = np.asarray(Ls @ Us_hat) + gamma * (Us_hat + X @ (lg[:, None] * Z))
    M = np.eye(s.size) - X @ (lg[:, None] * Qs.T)                  # I - B R^T
    Fs = np.linalg.solve(M, rhs)
    C = lg[:, None] * (Qs.T @ Fs + gamma * Z)                       # m x l
    U = np.zeros((g.N, n_labels))
    U[s] = onehot(seed_lab, n_labels)
    U[n] = (Qn @ C) / sc[n, None]
    if return_parts:
        return U, dict(X=X, Z=Z, Fs=Fs, C=C, rhs=rhs, M=M)
    return U


def fast_rw_dense(g, Q, lam, seed_idx, seed_lab, n_labels, P, gamma, normalized=True):
    """Same result from the N x N matrix E and its literal blocks (small N only)."""
    op, sc = _hat(g, normalized)
    op = op.toarray()
    n = split(g.N, seed_idx)
    s = np.asarray(seed_idx)
    Q = np.asarray(Q, dtype=np.float64)
    E = Q @ np.diag(1.0 / (np.asarray(lam) + gamma)) @ Q.T        # Eq. (E_def)
    Es, R, En = E[np.ix_(s, s)], E[np.ix_(s, n)], E[np.ix_(n, n)]   # Eq. (E_block)
    Ls, B = op[np.ix_(s, s)], op[np.ix_(s, n)]
    Us = sc[s, None] * onehot(seed_lab, n_labels)
    Pn = sc[n, None] * P[n] if gamma > 0 else np.zeros((n.size, n_labels))
    Fs = np.linalg.solve(np.eye(s.size) - B @ R.T, Ls @ Us + gamma * (Us + B @ En @ Pn))
    Un = R.T @ Fs + gamma * En @ Pn                                  # Eq. (Fs_2)
    del Es
    U = np.zeros((g.N, n_labels))
    U[s] = onehot(seed_lab, n_labels)
    U[n] = Un / sc[n, None]
    return U


def null_vector(g, normalized=True):
    """Unit null vector of L-hat (D^{1/2} 1 normalized) or of L (1 / sqrt(N))."""
    sc = np.sqrt(g.d) if normalized else np.ones(g.N)
    return sc / np.linalg.norm(sc)


def gamma0_basis(g, Q, normalized=True):
    """[g, (I - g g^T) Q[:, 1:]]: the basis of the gamma = 0 solve (see the module notes)."""
    gv = null_vector(g, normalized)
    Q = np.asarray(Q, dtype=np.float64)
    rest = Q[:, 1:] - np.outer(gv, gv @ Q[:, 1:])
    return np.concatenate([gv[:, None], rest], axis=1)


def fast_rw_gamma0(g, Q, lam, seed_idx, seed_lab, n_labels, normalized=True, return_parts=False):
    """gamma = 0 fast RW with the first m = Q.shape[1] stored columns (column 0 the null
    direction).  Returns U (N x n_labels)."""
    op, sc = _hat(g, normalized)
    n = split(g.N, seed_idx)
    s = np.asarray(seed_idx)
    S = s.size
    gv = null_vector(g, normalized)
    Qt = gamma0_basis(g, Q, normalized)
    Qp = Qt[:, 1:]                                                  # Q'
    li = 1.0 / np.asarray(lam, dtype=np.float64)[1:]               # diag of Lambda'^{-1}
    Qs, Qn = Qp[s], Qp[n]
    gs, gn = gv[s], gv[n]
    Us_hat = sc[s, None] * onehot(seed_lab, n_labels)
    Ls = op[s][:, s]
    B = op[s][:, n]
    X = np.asarray(B @ Qn)                                          # S x (m - 1)
    bg = np.asarray(B @ gn)                                         # B g_n
    Rt_row = (gn @ Qn) * li                                         # g_n^T Q_n' Lambda'^{-1}
    A = np.zeros((S + 1, S + 1))
    A[:S, :S] = np.eye(S) - X @ (li[:, None] * Qs.T)               # I - B R^T
    A[:S, S] = -bg
    A[S, :S] = -(Rt_row @ Qs.T)                                     # -g_n^T R^T
    A[S, S] = 1.0 - gn @ gn
    rhs = np.vstack([np.asarray(Ls @ Us_hat), (gs @ Us_hat)[None, :]])
    sol = np.linalg.solve(A, rhs)
    Fs, c = sol[:S], sol[S]
    Cp = li[:, None] * (Qs.T @ Fs)                                  # Lambda'^{-1} Q_s'^T F_s
    U = np.zeros((g.N, n_labels))
    U[s] = onehot(seed_lab, n_labels)
    U[n] = (Qn @ Cp + np.outer(gn, c)) / sc[n, None]
    if return_parts:
        return U, dict(Fs=Fs, c=c, C=Cp, X=X, bg=bg, Qt=Qt)
    return U


def fast_rw_gamma0_dense(g, Q, lam, seed_idx, seed_lab, n_labels, normalized=True):
    """Same result from the explicit pseudo-inverse E = Q' Lambda'^{-1} Q'^T and its blocks."""
    op, sc = _hat(g, normalized)
    op = op.toarray()
    n = split(g.N, seed_idx)
    s = np.asarray(seed_idx)
    S = s.size
    gv = null_vector(g, normalized)
    Qp = gamma0_basis(g, Q, normalized)[:, 1:]
    E = Qp @ np.diag(1.0 / np.asarray(lam, dtype=np.float64)[1:]) @ Qp.T
    R = E[np.ix_(s, n)]
    Ls, B = op[np.ix_(s, s)], op[np.ix_(s, n)]
    gs, gn = gv[s], gv[n]
    Us = sc[s, None] * onehot(seed_lab, n_labels)
    A = np.block([[np.eye(S) - B @ R.T, -(B @ gn)[:, None]],
                  [-(gn @ R.T)[None, :], np.array([[1.0 - gn @ gn]])]])
    sol = np.linalg.solve(A, np.vstack([Ls @ Us, (gs @ Us)[None, :]]))
    Fs, c = sol[:S], sol[S]
    U = np.zeros((g.N, n_labels))
    U[s] = onehot(seed_lab, n_labels)
    U[n] = (R.T @ Fs + np.outer(gn, c)) / sc[n, None]
    return U
