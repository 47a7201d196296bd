"""Pins for the oracle's eigenpairs, Eq. (L_eigs) (Sec. II-B) / Eq. (z_eig) (Sec. II-C)."""
import numpy as np
import pytest

import synth
from oracle import eig, graph


def _grid_closed_form(dims):
    """beta = 0, unnormalized: the grid Laplacian is a Kronecker sum of path Laplacians whose
    eigenvalues are 4 sin^2(pi k / (2 n)), k = 0..n-1."""
    vals = [4 * np.sin(np.pi * np.arange(n) / (2 * n)) ** 2 for n in dims]
    tot = vals[0]
    for v in vals[1:]:
        tot = (tot[:, None] + v[None, :]).ravel()
    return np.sort(tot)


@pytest.mark.parametrize("dims", [(6, 5), (4, 3, 3)])
def test_beta0_unnormalized_closed_form(dims):
    J = synth.smooth_random_image(dims, seed=0)
    g = graph.build_graph(J, dims, 0.0)
    lam, Q = eig.smallest_eigpairs(g.L, 12)
    np.testing.assert_allclose(lam, _grid_closed_form(dims)[:12], atol=1e-12)
    np.testing.assert_allclose(Q.T @ Q, np.eye(12), atol=1e-12)


def test_normalized_null_vector():
    dims = (9, 8)
    J = synth.smooth_random_image(dims, seed=1, sigma=0.05)
    g = graph.build_graph(J, dims, 50.0)
    lam, Q = eig.smallest_eigpairs(g.Lhat, 5)
    assert abs(lam[0]) < 1e-12
    v = np.sqrt(g.d) / np.linalg.norm(np.sqrt(g.d))
    assert abs(abs(Q[:, 0] @ v) - 1) < 1e-12


def test_shift_invert_matches_dense():
    dims = (40, 30)
    J = synth.smooth_random_image(dims, seed=2, sigma=0.05)
    g = graph.build_graph(J, dims, 50.0)
    lam_d, Qd = eig.smallest_eigpairs(g.Lhat, 20)
    lam_s, Qs = eig.smallest_eigpairs(g.Lhat, 20, dense_max=100)
    np.testing.assert_allclose(lam_s, lam_d, atol=1e-11)
    R = g.Lhat @ Qs - Qs * lam_s
    assert np.abs(R).max() < 1e-9
