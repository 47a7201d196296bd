"""Choosing the number of eigenvectors online, Sec. III-A (oracle, FP64).

From the seeds (Sec. III-A-1, Eq. alpha_1): for each label k,
    f(u_s^k) = min_{||alpha|| <= rho} || Q_s alpha - u_s^k ||^2,
with rho = sqrt(N), replaced by sqrt(1^T D 1) with the normalized Laplacian, where the target is
u-hat_s^k = D_s^{1/2} u_s^k.  If any label has f > f_max = S eps^2 (eps = 1/10 in the paper,
S = the number of seeds) more eigenvectors are added and f is evaluated again.  Here the
candidates are m = m_step, 2 m_step, ..., m_max (m_max last if it is not a multiple) and the
first m whose worst label passes is returned; if none passes, m_max is returned with
``capped = True``.

The norm-constrained least squares problem is solved through the SVD Q_s = U S V^T: if the
minimum-norm least-squares solution satisfies the constraint it is the minimizer; otherwise the
minimizer is alpha(mu) = V diag(s / (s^2 + mu)) U^T u with the unique mu > 0 where
||alpha(mu)|| = rho (the secular equation; a root exists because ||alpha(mu)|| falls
continuously from the min-norm value to 0), found by safeguarded Newton on
1/||alpha(mu)|| - 1/rho.  f is then evaluated directly as ||Q_s alpha - u||^2.

From priors (Sec. III-A-2, Eq. g): g(p^k) = ||p^k - Q Q^T p^k||^2 for orthonormal Q, evaluated
for one label in every r^d (r = 4), with g_max = n eps^2 (1^T D 1 eps^2 and P-hat = D^{1/2} P
with the normalized Laplacian, by analogy with the seed criterion).
Test infrastructure only.
"""
from __future__ import annotations

import numpy as np


def trust_region_ls(A, u, rho, tol=None):
    """Returns (f, alpha, mu) for min_{||alpha|| <= rho} ||A alpha - u||^2."""
    A = np.asarray(A, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    Uu, s, Vt = np.linalg.svd(A, full_matrices=False)
    if tol is None:
        tol = (s.max() if s.size else 0.0) * max(A.shape) * np.finfo(np.float64).eps
    keep = s > tol
    s, Uu, Vt = s[keep], Uu[:, keep], Vt[keep]
    c = Uu.T @ u
    alpha_ls = Vt.T @ (c / s)
    if np.linalg.norm(alpha_ls) <= rho:
        r = A @ alpha_ls - u
        return float(r @ r), alpha_ls, 0.0

    def norm_alpha(mu):
        return np.linalg.norm(s * c / (s * s + mu))

    # bracket: ||alpha(0)|| > rho; ||alpha(mu_hi)|| <= ||c|| / (s_min... ) -> choose mu_hi large
    lo, hi = 0.0, max(np.linalg.norm(c) * s.max() / rho, 1e-300)
    while norm_alpha(hi) > rho:
        hi *= 2.0
    mu = hi
    for _ in range(200):
        na = norm_alpha(mu)
        phi = 1.0 / na - 1.0 / rho
        if abs(phi) * rho < 1e-15:
            break
        if phi < 0:
            lo = mu
        else:
            hi = mu
        # d/dmu ||alpha||^2 = -2 sum s^2 c^2 / (s^2 + mu)^3
        dn2 = -2.0 * np.sum((s * c) ** 2 / (s * s + mu) ** 3)
        dphi = -0.5 * na ** -3 * dn2
        step = mu - phi / dphi if dphi != 0 else 0.5 * (lo + hi)
        mu = step if lo < step < hi else 0.5 * (lo + hi)
        if hi - lo <= 1e-15 * hi:
            break
    alpha = Vt.T @ (s * c / (s * s + mu))
    r = A @ alpha - u
    return float(r @ r), alpha, mu


def m_grid(m_max, m_step):
    g = list(range(m_step, m_max + 1, m_step))
    if not g or g[-1] != m_max:
        g.append(m_max)
    return g


def seed_targets(g, seed_idx, seed_lab, n_labels, normalized=True):
    """u-hat_s^k (S x l) and rho (Sec. III-A-1)."""
    S = len(seed_idx)
    U = np.zeros((S, n_labels))
    U[np.arange(S), seed_lab] = 1.0
    if normalized:
        return np.sqrt(g.d[seed_idx])[:, None] * U, float(np.sqrt(g.d.sum()))
    return U, float(np.sqrt(g.N))


def f_values(Q, seed_idx, targets, rho, m):
    Qs = np.asarray(Q[seed_idx, :m], dtype=np.float64)
    return np.array([trust_region_ls(Qs, targets[:, k], rho)[0] for k in range(targets.shape[1])])


def choose_m_from_seeds(g, Q, seed_idx, seed_lab, n_labels, m_max, m_step=10, eps=0.1,
                        normalized=True):
    """Returns (m, f_at_m, capped, table) with table = {m: f-vector} for the evaluated m."""
    targets, rho = seed_targets(g, seed_idx, seed_lab, n_labels, normalized)
    fmax = len(seed_idx) * eps ** 2
    table = {}
    for m in m_grid(m_max, m_step):
        f = f_values(Q, seed_idx, targets, rho, m)
        table[m] = f
        if f.max() <= fmax:
            return m, f, False, table
    return m_max, table[m_max], True, table


def g_values(Q, Phat, m):
    """Eq. (g): ||p - Q Q^T p||^2 per column of P-hat, with the first m columns of Q."""
    Qm = np.asarray(Q[:, :m], dtype=np.float64)
    R = Phat - Qm @ (Qm.T @ Phat)
    return np.einsum("ij,ij->j", R, R)


def sampled_labels(label_grid_shape, r=4):
    """One label in every r^d of a d-dimensional displacement-label grid, uniformly spaced
    (centred stride-r sub-grid, Sec. III-A-2).  Returns flat label indices."""
    axes = []
    for n in label_grid_shape:
        start = (n - 1 - ((n - 1) // r) * r) // 2
        axes.append(np.arange(start, n, r))
    mesh = np.meshgrid(*axes, indexing="ij")
    flat = np.ravel_multi_index([m.ravel() for m in mesh], label_grid_shape)
    return np.sort(flat)


def choose_m_from_priors(g, Q, P, m_max, m_step=10, eps=0.1, normalized=True, labels=None):
    sc = np.sqrt(g.d) if normalized else np.ones(g.N)
    Phat = sc[:, None] * P
    if labels is not None:
        Phat = Phat[:, labels]
    gmax = (g.d.sum() if normalized else g.N) * eps ** 2
    table = {}
    for m in m_grid(m_max, m_step):
        gv = g_values(Q, Phat, m)
        table[m] = gv
        if gv.max() <= gmax:
            return m, gv, False, table
    return m_max, table[m_max], True, table
