"""Pins for the oracle's fast RW (Sec. II-B, Eqs. E_def - Fs; normalized form Sec. II-C)."""
import numpy as np
import pytest

import synth
from oracle import eig, exact, fastrw, graph, priors


def _case(seed, dims=(12, 10), n_labels=3, per=3, beta=40.0):
    J = synth.smooth_random_image(dims, seed=seed, smooth=2.0, sigma=0.03)
    truth = np.minimum((J * n_labels).astype(np.int32), n_labels - 1)
    si, sl = synth.sample_seeds(truth, dims, per, 1, seed=seed, n_labels=n_labels)
    g = graph.build_graph(J, dims, beta)
    P = priors.gaussian_priors(J, si, sl, n_labels)
    return g, si, sl, n_labels, P


@pytest.mark.parametrize("normalized", [True, False])
@pytest.mark.parametrize("gamma", [1e-3, 0.3])
def test_full_basis_equals_exact(normalized, gamma):
    """m = N: E = (L + gamma I)^{-1} exactly, so E F = U (Eq. pseudo_E) makes the fast RW equal
    the basic RW."""
    g, si, sl, nl, P = _case(0)
    lam, Q = eig.smallest_eigpairs(g.operator(normalized), g.N)
    Uf = fastrw.fast_rw(g, Q, lam, si, sl, nl, P, gamma, normalized)
    Ue = exact.exact_rw(g, si, sl, nl, P, gamma, normalized)
    np.testing.assert_allclose(Uf, Ue, atol=1e-10)


@pytest.mark.parametrize("normalized", [True, False])
def test_two_restatements_agree(normalized):
    g, si, sl, nl, P = _case(1)
    lam, Q = eig.smallest_eigpairs(g.operator(normalized), 30)
    U1 = fastrw.fast_rw(g, Q, lam, si, sl, nl, P, 1e-3, normalized)
    U2 = fastrw.fast_rw_dense(g, Q, lam, si, sl, nl, P, 1e-3, normalized)
    np.testing.assert_allclose(U1, U2, atol=1e-12)


def test_rowsums_one_when_null_vector_in_span():
    g, si, sl, nl, P = _case(2)
    lam, Q = eig.smallest_eigpairs(g.Lhat, 25)
    U = fastrw.fast_rw(g, Q, lam, si, sl, nl, P, 1e-3)
    np.testing.assert_allclose(U.sum(axis=1), 1.0, atol=1e-11)
    np.testing.assert_array_equal(U[si], exact.onehot(sl, nl))


def test_error_shrinks_toward_full_basis():
    g, si, sl, nl, P = _case(3, dims=(16, 16))
    lam, Q = eig.smallest_eigpairs(g.Lhat, g.N)
    Ue = exact.exact_rw(g, si, sl, nl, P, 1e-3)
    err = {m: np.abs(fastrw.fast_rw(g, Q[:, :m], lam[:m], si, sl, nl, P, 1e-3) - Ue).max()
           for m in (16, 64, 192, 256)}
    assert err[256] < 1e-10
    assert err[192] < err[16]
    assert err[64] < err[16]


def test_planted_transpose_is_caught(monkeypatch):
    """Using R where R^T belongs in Eq. (Fs_2) must break the m = N pin."""
    g, si, sl, nl, P = _case(0)
    lam, Q = eig.smallest_eigpairs(g.Lhat, g.N)
    Ue = exact.exact_rw(g, si, sl, nl, P, 1e-3)
    real_solve = np.linalg.solve

    def wrong(M, rhs):
        return real_solve(M.T, rhs)   # I - R B^T instead of I - B R^T
    monkeypatch.setattr(fastrw.np.linalg, "solve", wrong)
    Uf = fastrw.fast_rw(g, Q, lam, si, sl, nl, P, 1e-3)
    monkeypatch.setattr(fastrw.np.linalg, "solve", real_solve)
    assert np.abs(Uf - Ue).max() > 1e-6


def _two_components(seed=5, dims=(14, 11)):
    """A graph cut into a left and a right half (the crossing edges set to 0), seeds of label 0
    on the left and of label 1 on the right, priors equal to those halves."""
    X = dims[0]
    J = synth.smooth_random_image(dims, seed=seed, smooth=1.5, sigma=0.05)
    g0 = graph.build_graph(J, dims, 60.0)
    left = np.arange(g0.N) % X < X // 2
    cut = g0.ids[left[g0.a] & ~left[g0.b]]
    g = graph.set_edge_weights(g0, cut, np.zeros(cut.size))
    rng = np.random.default_rng(seed)
    si = np.concatenate([rng.choice(np.nonzero(left)[0], 4, replace=False),
                         rng.choice(np.nonzero(~left)[0], 3, replace=False)])
    sl = np.array([0] * 4 + [1] * 3)
    return g, si, sl, left, np.stack([left, ~left], 1).astype(np.float64)


@pytest.mark.parametrize("normalized", [True, False])
def test_exact_at_small_m_when_the_solution_lies_in_the_span(normalized):
    """m < N.  On a graph of two components with consistent seeds and priors the basic RW is the
    indicator of each half (it satisfies every row of Eq. rw_eq), and that indicator lies in the
    span of the two null vectors D^{1/2} 1_c.  The eigenvector form E = Q Lambda_gamma Q^T then
    reproduces it exactly: with the two null vectors alone (written from the degrees, value 0)
    and with the 2, 3, 7 and 20 lowest eigenvectors of a dense symmetric eigensolver."""
    g, si, sl, left, P = _two_components()
    gamma = 1e-2
    np.testing.assert_allclose(exact.exact_rw(g, si, sl, 2, P, gamma, normalized), P, atol=1e-12)
    sc = np.sqrt(g.d) if normalized else np.ones(g.N)
    nulls = np.stack([sc * left, sc * ~left], 1)
    nulls /= np.linalg.norm(nulls, axis=0)
    U = fastrw.fast_rw(g, nulls, np.zeros(2), si, sl, 2, P, gamma, normalized)
    np.testing.assert_allclose(U, P, atol=1e-12)
    lam, V = np.linalg.eigh(g.operator(normalized).toarray())
    for m in (2, 3, 7, 20):
        U = fastrw.fast_rw(g, V[:, :m], lam[:m], si, sl, 2, P, gamma, normalized)
        np.testing.assert_allclose(U, P, atol=1e-11)


def test_small_m_pin_catches_a_dropped_degree_scaling(monkeypatch):
    """The normalized form without its D^{1/2} scalings (U-hat_s, P-hat, U = D^{-1/2} U-hat)
    must fail the pin above."""
    g, si, sl, left, P = _two_components()
    lam, V = np.linalg.eigh(g.Lhat.toarray())
    real = fastrw._hat
    monkeypatch.setattr(fastrw, "_hat", lambda g_, normalized: (real(g_, normalized)[0],
                                                                 np.ones(g_.N)))
    U = fastrw.fast_rw(g, V[:, :7], lam[:7], si, sl, 2, P, 1e-2)
    monkeypatch.setattr(fastrw, "_hat", real)
    assert np.abs(U - P).max() > 1e-3


def _dct_grid_modes(dims, count):
    """Orthonormal eigenvectors of the unweighted 4-neighbour grid Laplacian L (free
    boundaries): products of DCT-II cosines, eigenvalue 4 sin^2(pi a / 2X) + 4 sin^2(pi b / 2Y),
    the ``count`` smallest (x fastest, as the graph numbers its nodes)."""
    X, Y = dims

    def cos_basis(n, k):
        c = np.cos(np.pi * k * (np.arange(n) + 0.5) / n)
        return c / np.linalg.norm(c)
    modes = sorted((4 * np.sin(np.pi * a / (2 * X)) ** 2 + 4 * np.sin(np.pi * b / (2 * Y)) ** 2,
                    a, b) for a in range(X) for b in range(Y))[:count]
    lam = np.array([v for v, _, _ in modes])
    Q = np.stack([np.outer(cos_basis(Y, b), cos_basis(X, a)).ravel() for _, a, b in modes], 1)
    return lam, Q


def test_unseeded_form_is_the_spectral_filter_of_priors_in_the_span():
    """No seeds (Eq. U_lin_comb with S = 0, as in registration), unnormalized Laplacian of the
    unweighted grid, priors inside the span of its first m eigenvectors: the basic RW
    (L + gamma I) U = gamma P has the closed form U = sum_i gamma / (lambda_i + gamma) q_i q_i^T P,
    and the fast solve with those m eigenvectors (m < N) must equal it."""
    dims = (9, 7)
    g = graph.build_graph(np.zeros(63), dims, 0.0)
    lam, Q = _dct_grid_modes(dims, 12)
    np.testing.assert_allclose(g.L @ Q, Q * lam, atol=1e-12)   # the modes are eigenvectors
    rng = np.random.default_rng(3)
    A = rng.normal(size=(12, 3))
    P = Q @ A
    gamma = 0.2
    want = Q @ ((gamma / (lam + gamma))[:, None] * A)
    none = np.zeros(0, dtype=np.int64)
    U = fastrw.fast_rw(g, Q, lam, none, none, 3, P, gamma, normalized=False)
    np.testing.assert_allclose(U, want, atol=1e-12)
    np.testing.assert_allclose(exact.exact_rw(g, none, none, 3, P, gamma, normalized=False),
                               want, atol=1e-10)
