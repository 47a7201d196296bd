"""The m x m forms of Eq. (Fs) that the GPU path solves, checked on the CPU against the oracle's
literal S x S solve (Eqs. Fs, Fs_2, U_lin_comb).

With Lambda_gamma = (Lambda + gamma I)^{-1}, K = Q_s^T X (X = B-hat Q_n), h = Q_s^T (L-hat_s
U-hat_s + gamma U-hat_s) and M = Lambda_gamma^{-1} - K, the seeded system is equivalent to
M y = h + gamma K Lambda_gamma Z, C = y + gamma Lambda_gamma Z; and since K Lambda_gamma Z =
Z - M Lambda_gamma Z, also to C = M^{-1} (h + gamma Z).  Both must give the coefficient matrix C
of Eq. (U_lin_comb) that the oracle computes from F_s.

gamma = 0 (Sec. II-B, after Eq. Fs): the GPU path solves the bordered system of the oracle's
``fast_rw_gamma0`` in m x m form.  It works on the stored columns: w^n = Q_n^T g_n, p = Q_s^T g_s,
w = w^n + p; the seed rows become Q_s' = [g_s, Q_s - g_s w^T], X' = [B g_n, X - (B g_n) w^T], so
the seed Gram gives K, G, h, b on the basis [g, Q'] directly; row 0 is then replaced by the
column-sum equation (M_00 = s = g_s^T g_s, M_0j = -(w^n_j - w_j (1 - s)), h_0 = g_s^T U-hat_s);
C = M^{-1} h, and U-hat_n = Q_n C (row 0 of C zeroed) + g_n (c - w^T C')."""
import numpy as np
import pytest

import synth
from oracle import eig, fastrw, graph, priors
from oracle.exact import onehot


def _case(gamma, m, n_labels, seed):
    dims = (26, 21)
    J = synth.smooth_random_image(dims, seed=seed, smooth=2.5, sigma=0.02)
    truth = np.minimum((J * n_labels).astype(np.int32), n_labels - 1)
    si, sl = synth.sample_seeds(truth, dims, 5, 1, seed=seed, n_labels=n_labels)
    g = graph.build_graph(J, dims, 80.0)
    lam, Q = eig.smallest_eigpairs(g.Lhat, m)
    P = priors.gaussian_priors(J, si, sl, n_labels)
    return g, Q, lam, si, sl, P


@pytest.mark.parametrize("gamma,m,n_labels,seed", [(1e-3, 30, 2, 1), (0.05, 45, 3, 2),
                                                   (0.5, 12, 4, 3)])
def test_m_by_m_forms_match_the_seeded_system(gamma, m, n_labels, seed):
    g, Q, lam, si, sl, P = _case(gamma, m, n_labels, seed)
    U_ref, parts = fastrw.fast_rw(g, Q, lam, si, sl, n_labels, P, gamma, return_parts=True)
    X, Z, C_ref = parts["X"], parts["Z"], parts["C"]
    op = g.operator(True)
    sc = np.sqrt(g.d)
    Qs = Q[np.asarray(si)]
    Us_hat = sc[si, None] * onehot(sl, n_labels)
    lgam = lam + gamma                                   # diag of Lambda_gamma^{-1}
    K = Qs.T @ X
    h = Qs.T @ (np.asarray(op[si][:, si] @ Us_hat) + gamma * Us_hat)
    M = np.diag(lgam) - K
    W = Z / lgam[:, None]                                # Lambda_gamma Z
    y = np.linalg.solve(M, h + gamma * K @ W)
    C_a = y + gamma * W                                  # the y-then-C form
    C_b = np.linalg.solve(M, h + gamma * Z)              # the collapsed form
    scale = np.abs(C_ref).max()
    assert np.abs(C_a - C_ref).max() <= 1e-9 * scale
    assert np.abs(C_b - C_ref).max() <= 1e-9 * scale
    # and the back-projection of either gives the oracle's probabilities
    n = np.setdiff1d(np.arange(g.N), si)
    U = np.zeros_like(U_ref)
    U[si] = onehot(sl, n_labels)
    U[n] = (Q[n] @ C_b) / sc[n, None]
    assert np.abs(U - U_ref).max() <= 1e-9


def test_a_planted_sign_error_is_caught():
    """Flipping the sign of gamma Z in the collapsed form must break the match."""
    g, Q, lam, si, sl, P = _case(0.05, 30, 2, 4)
    _, parts = fastrw.fast_rw(g, Q, lam, si, sl, 2, P, 0.05, return_parts=True)
    X, Z, C_ref = parts["X"], parts["Z"], parts["C"]
    sc = np.sqrt(g.d)
    Qs = Q[np.asarray(si)]
    Us_hat = sc[si, None] * onehot(sl, 2)
    op = g.operator(True)
    h = Qs.T @ (np.asarray(op[si][:, si] @ Us_hat) + 0.05 * Us_hat)
    M = np.diag(lam + 0.05) - Qs.T @ X
    C_bad = np.linalg.solve(M, h - 0.05 * Z)
    assert np.abs(C_bad - C_ref).max() > 1e-3 * np.abs(C_ref).max()


@pytest.mark.parametrize("m,n_labels,seed", [(1, 2, 1), (12, 3, 2), (40, 4, 3)])
def test_gamma0_m_by_m_bordered_form_matches_the_oracle(m, n_labels, seed):
    g, Q, lam, si, sl, _ = _case(0.0, m, n_labels, seed)
    U_ref = fastrw.fast_rw_gamma0(g, Q, lam, si, sl, n_labels)
    op = g.operator(True)
    sc = np.sqrt(g.d)
    si = np.asarray(si)
    n = np.setdiff1d(np.arange(g.N), si)
    gv = sc / np.linalg.norm(sc)
    gs, gn = gv[si], gv[n]
    B = op[si][:, n]
    Us_hat = sc[si, None] * onehot(sl, n_labels)
    Qs = Q[si].copy()
    X = np.asarray(B @ Q[n])
    bg = np.asarray(B @ gn)
    wn = Q[n].T @ gn
    w = wn + Qs.T @ gs
    w[0] = 0.0
    Qs2 = Qs - np.outer(gs, w)
    Qs2[:, 0] = gs
    X2 = X - np.outer(bg, w)
    X2[:, 0] = bg
    r0 = np.asarray(op[si][:, si] @ Us_hat)
    K = Qs2.T @ X2
    G = Qs2.T @ Qs2
    h = Qs2.T @ r0
    bv = Qs2.T @ Us_hat
    s0 = G[0, 0]
    lam0 = lam.copy()
    lam0[0] = s0
    K[0, 0] = 0.0
    K[0, 1:] = wn[1:] - w[1:] * (1.0 - s0)
    h[0] = bv[0]
    C = np.linalg.solve(np.diag(lam0) - K, h)
    c_eff = C[0] - w[1:] @ C[1:]
    C[0] = 0.0
    U = np.zeros_like(U_ref)
    U[si] = onehot(sl, n_labels)
    U[n] = (Q[n] @ C + np.outer(sc[n], c_eff / np.linalg.norm(sc))) / sc[n, None]
    assert np.abs(U - U_ref).max() <= 1e-9
