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
