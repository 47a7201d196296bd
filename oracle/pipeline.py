"""The online solve composed from the oracle's pieces, in the paper's order (Sec. II-B, III-A):
priors from the seeds (Sec. IV-A) -> number of eigenvectors m from the seeds (Eq. alpha_1),
unless fixed -> fast RW with the first m columns (Eqs. Fs, U_lin_comb) -> k damped-Jacobi
refinement steps on Eq. (rw_eq) -> hard labels by the largest probability (ties to the lowest label, Sec. IV-A's
conversion of a probabilistic segmentation).  With gamma = 0 there are no priors: m is chosen on
the gamma = 0 basis [g, Q'] and the fast RW is the bordered form of ``fastrw.fast_rw_gamma0``.
Test infrastructure only.
"""
from __future__ import annotations

import numpy as np

from .adaptive import choose_m_from_seeds
from .fastrw import fast_rw, fast_rw_gamma0, gamma0_basis
from .priors import gaussian_priors
from .refine import refine


def hard_labels(U):
    return np.argmax(U, axis=1).astype(np.uint8)   # argmax returns the first maximum


def online_solve(g, Q, lam, seed_idx, seed_lab, n_labels, gamma=1e-3, m=0, m_step=10, eps=0.1,
                 refine_steps=3, normalized=True, P=None,
                 refine_method="jacobi", omega=0.8):
    """Returns dict(U, labels, m, f, capped, P)."""
    if P is None and gamma > 0:
        P = gaussian_priors(g.J, seed_idx, seed_lab, n_labels)
    info = dict(f=None, capped=False)
    if m == 0:
        Qm = gamma0_basis(g, Q, normalized) if gamma == 0 else Q
        m, f, capped, _ = choose_m_from_seeds(g, Qm, seed_idx, seed_lab, n_labels, Q.shape[1],
                                              m_step, eps, normalized)
        info.update(f=f, capped=capped)
    if gamma == 0:
        U = fast_rw_gamma0(g, Q[:, :m], lam[:m], seed_idx, seed_lab, n_labels, normalized)
    else:
        U = fast_rw(g, Q[:, :m], lam[:m], seed_idx, seed_lab, n_labels, P, gamma, normalized)
    if refine_steps > 0:
        U, _ = refine(g, U, seed_idx, seed_lab, n_labels, P, gamma, refine_steps, normalized,
                      refine_method, omega)
    return dict(U=U, labels=hard_labels(U), m=m, P=P, **info)
