"""Pins for the oracle's refinement steps and the eigenvalue update of Sec. III-B."""
import numpy as np
import pytest

import synth
from oracle import eig, exact, fastrw, graph, priors, refine, update


def _case(seed=0, dims=(14, 12), n_labels=3):
    J = synth.smooth_random_image(dims, seed=seed, smooth=2.0, sigma=0.03)
    truth = np.minimum((J * n_labels).astype(np.int32), n_labels - 1)
    si, sl = synth.sample_seeds(truth, dims, 3, 1, seed=seed, n_labels=n_labels)
    g = graph.build_graph(J, dims, 40.0)
    P = priors.gaussian_priors(J, si, sl, n_labels)
    return g, si, sl, n_labels, P


def test_cg_error_monotone_and_converges():
    g, si, sl, nl, P = _case()
    gamma = 1e-2
    lam, Q = eig.smallest_eigpairs(g.Lhat, 20)
    U0 = fastrw.fast_rw(g, Q, lam, si, sl, nl, P, gamma)
    Ue = exact.exact_rw(g, si, sl, nl, P, gamma)
    A, b, n, sc = refine.hat_system(g, si, sl, nl, P, gamma)
    xe = sc[n, None] * Ue[n]
    errs = []
    for k in range(0, 6):
        U, _ = refine.refine(g, U0, si, sl, nl, P, gamma, k, method="pcg")
        e = sc[n, None] * U[n] - xe
        errs.append(np.einsum("ij,ij->j", e, A @ e))     # A-norm error per column
    errs = np.array(errs)
    assert np.all(np.diff(errs, axis=0) <= 1e-14)        # CG: A-norm error never increases
    U, _ = refine.refine(g, U0, si, sl, nl, P, gamma, 400, method="pcg")
    np.testing.assert_allclose(U, Ue, atol=1e-9)
    U, _ = refine.refine(g, U0, si, sl, nl, P, gamma, 0, method="pcg")
    np.testing.assert_array_equal(U, U0)


def test_jacobi_fixed_point_contraction_and_convergence():
    """The exact solution is a fixed point; the max-norm distance between two runs from
    different starts never grows (iteration-matrix max-norm <= 1); many steps converge."""
    g, si, sl, nl, P = _case(seed=5)
    gamma = 0.05
    Ue = exact.exact_rw(g, si, sl, nl, P, gamma)
    U, _ = refine.refine(g, Ue, si, sl, nl, P, gamma, 3)
    np.testing.assert_allclose(U, Ue, atol=1e-13)
    rng = np.random.default_rng(1)
    n = exact.split(g.N, si)
    A0 = Ue.copy(); A0[n] += 0.1 * rng.standard_normal((n.size, nl))
    B0 = A0.copy(); B0[n] += 1e-3 * rng.standard_normal((n.size, nl))
    prev = np.abs(A0 - B0).max()
    for k in range(1, 6):
        a, _ = refine.refine(g, A0, si, sl, nl, P, gamma, k)
        b, _ = refine.refine(g, B0, si, sl, nl, P, gamma, k)
        cur = np.abs(a - b).max()
        assert cur <= prev * (1 + 1e-12)
        prev = cur
    U, _ = refine.refine(g, A0, si, sl, nl, P, gamma, 3000)
    np.testing.assert_allclose(U, Ue, atol=1e-8)


def test_values_unchanged_when_beta_unchanged():
    g, *_ = _case(1)
    lam, Q = eig.smallest_eigpairs(g.Lhat, 15)
    lh = update.updated_values(update.update_beta(g, g.beta), Q)
    np.testing.assert_allclose(lh, lam, atol=1e-12)


def test_rayleigh_edge_sum_form_and_ky_fan_bound():
    """Eq. (z_ray) through an explicit edge sum sum_e w_e (q_a/sqrt(d_a) - q_b/sqrt(d_b))^2,
    and the Ky Fan bound: the k smallest updated values sum to at least the k smallest true
    eigenvalues of the new L-hat."""
    g, *_ = _case(2)
    lam, Q = eig.smallest_eigpairs(g.Lhat, 12)
    g2 = update.update_beta(g, 2.5 * g.beta)
    lh = update.updated_values(g2, Q)
    for i in range(12):
        q = Q[:, i]
        s = sum(w * (q[a] / np.sqrt(g2.d[a]) - q[b] / np.sqrt(g2.d[b])) ** 2
                for a, b, w in zip(g2.a, g2.b, g2.w))
        np.testing.assert_allclose(lh[i], s, rtol=1e-12)
    lam2 = np.linalg.eigvalsh(g2.Lhat.toarray())
    for k in range(1, 13):
        assert lh[:k].sum() >= lam2[:k].sum() - 1e-12


def test_roi_update_equals_edge_list_update():
    dims = (10, 9, 8)
    J = synth.smooth_random_image(dims, seed=3, sigma=0.05)
    g = graph.build_graph(J, dims, 50.0)
    lo, hi = (2, 3, 1), (7, 8, 5)
    ids = synth.roi_edge_ids(dims, lo, hi)
    g1 = update.update_roi(g, lo, hi, 100.0)
    pos = np.searchsorted(g.ids, ids)
    w_new = graph.edge_weights(J, g.a[pos], g.b[pos], 100.0)
    g2 = update.update_edges(g, ids, w_new)
    np.testing.assert_array_equal(g1.w, g2.w)
    g3 = update.update_roi(g, lo, hi, 50.0)                # same beta: no change
    np.testing.assert_array_equal(g3.w, g.w)
    # edges outside the box keep their weights
    mask = np.ones(g.ids.size, bool)
    mask[pos] = False
    np.testing.assert_array_equal(g1.w[mask], g.w[mask])


def test_edge_removal_is_zero_weight_update():
    g, *_ = _case(4)
    lam, Q = eig.smallest_eigpairs(g.Lhat, 10)
    ids = g.ids[[3, 17, 40]]
    a = update.updated_values(update.remove_edges(g, ids), Q)
    b = update.updated_values(update.update_edges(g, ids, np.zeros(3)), Q)
    np.testing.assert_array_equal(a, b)
