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

Parity note: at m < N the result is an approximation whose only pins are m = N (equality with
the exact solve, from E F = U, Eq. pseudo_E), the agreement of the two restatements, and the
row-sum property when D^{1/2} 1 lies in span(Q).
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
