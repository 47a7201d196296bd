"""The m x m forms of Eq. (Fs) that the GPU path solves, checked on the CPU against the oracle's
literal S x S solve (Eqs. Fs, Fs_2, U_lin_comb).

With Lambda_gamma = (Lambda + gamma I)^{-1}, K = Q_s^T X (X = B-hat Q_n), h = Q_s^T (L-hat_s
U-hat_s + gamma U-hat_s) and M = Lambda_gamma^{-1} - K, the seeded system is equivalent to
M y = h + gamma K Lambda_gamma Z, C = y + gamma Lambda_gamma Z; and since K Lambda_gamma Z =
Z - M Lambda_gamma Z, also to C = M^{-1} (h + gamma Z).  Both must give the coefficient matrix C
of Eq. (U_lin_comb) that the oracle computes from F_s."""
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
