"""Pins for the oracle's choice of m (Sec. III-A, Eqs. alpha_1 and g)."""
import numpy as np
import pytest

import synth
from oracle import adaptive, eig, graph


def _brute_force(A, u, rho, iters=20000):
    """Projected gradient descent on ||A a - u||^2 over the ball ||a|| <= rho."""
    L = 2 * np.linalg.norm(A, 2) ** 2
    a = np.zeros(A.shape[1])
    for _ in range(iters):
        a = a - (2 * A.T @ (A @ a - u)) / L
        na = np.linalg.norm(a)
        if na > rho:
            a *= rho / na
    r = A @ a - u
    return r @ r


@pytest.mark.parametrize("rho", [0.3, 1.0, 100.0])
@pytest.mark.parametrize("shape", [(20, 8), (6, 12)])
def test_trust_region_matches_projected_gradient(rho, shape):
    rng = np.random.default_rng(1)
    A = rng.standard_normal(shape) * np.linspace(1, 0.05, shape[1])[None, :]
    u = rng.standard_normal(shape[0])
    f, a, mu = adaptive.trust_region_ls(A, u, rho)
    assert np.linalg.norm(a) <= rho * (1 + 1e-9)
    fb = _brute_force(A, u, rho)
    assert f <= fb + 1e-9 and f >= fb - 1e-6 * max(1, fb)


def test_kkt_conditions():
    rng = np.random.default_rng(2)
    A = rng.standard_normal((15, 10))
    u = rng.standard_normal(15) * 10
    for rho in (0.2, 50.0):
        f, a, mu = adaptive.trust_region_ls(A, u, rho)
        grad = A.T @ (A @ a - u)
        if mu == 0:
            assert np.linalg.norm(a) <= rho and np.abs(grad).max() < 1e-9
        else:
            assert mu > 0 and abs(np.linalg.norm(a) - rho) < 1e-9 * rho
            np.testing.assert_allclose(grad, -mu * a, atol=1e-8 * max(1, mu))


def test_zero_when_target_in_range_with_small_norm():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((12, 5))
    a0 = rng.standard_normal(5)
    f, a, mu = adaptive.trust_region_ls(A, A @ a0, 10 * np.linalg.norm(a0))
    assert f < 1e-20


def _seeded_case():
    dims = (14, 12)
    J = synth.smooth_random_image(dims, seed=4, smooth=2.0, sigma=0.03)
    truth = np.minimum((J * 3).astype(np.int32), 2)
    si, sl = synth.sample_seeds(truth, dims, 5, 1, seed=4, n_labels=3)
    g = graph.build_graph(J, dims, 40.0)
    lam, Q = eig.smallest_eigpairs(g.Lhat, 60)
    return g, Q, si, sl


def test_f_non_increasing_in_m():
    """Nested feasible sets: adding columns can only lower the constrained minimum."""
    g, Q, si, sl = _seeded_case()
    targets, rho = adaptive.seed_targets(g, si, sl, 3)
    prev = None
    for m in adaptive.m_grid(60, 5):
        f = adaptive.f_values(Q, si, targets, rho, m)
        if prev is not None:
            assert np.all(f <= prev + 1e-9)
        prev = f


def test_choose_m_returns_first_passing_grid_point():
    g, Q, si, sl = _seeded_case()
    m, f, capped, table = adaptive.choose_m_from_seeds(g, Q, si, sl, 3, 60, 5, eps=0.1)
    fmax = len(si) * 0.01
    assert f.max() <= fmax or capped
    for mm, ff in table.items():
        if mm < m:
            assert ff.max() > fmax
    # a stricter accuracy never picks fewer eigenvectors
    m2, _, _, _ = adaptive.choose_m_from_seeds(g, Q, si, sl, 3, 60, 5, eps=0.03)
    assert m2 >= m


def test_g_residual_and_sampling():
    rng = np.random.default_rng(5)
    N, m = 50, 7
    Q = np.linalg.qr(rng.standard_normal((N, m)))[0]
    p = Q @ rng.standard_normal(m)
    assert adaptive.g_values(Q, p[:, None], m)[0] < 1e-24        # p in span(Q)
    q = rng.standard_normal(N)
    gq = adaptive.g_values(Q, q[:, None], m)[0]
    np.testing.assert_allclose(gq, q @ q - np.sum((Q.T @ q) ** 2), rtol=1e-12)
    # one label in every r^d on the paper's 31 x 31 x 13 displacement grid
    lab = adaptive.sampled_labels((31, 31, 13), r=4)
    assert lab.size == 8 * 8 * 4
    assert adaptive.sampled_labels((3, 3, 3), r=4).tolist() == [13]   # the centre label


def test_dual_bound_is_below_the_constrained_minimum():
    """The GPU's adaptive choice rejects a candidate m as soon as one label's Lagrangian dual
    bound g(mu) = ||u||^2 - b^T (G + mu I)^{-1} b - mu rho^2 (G = A^T A, b = A^T u) exceeds
    f_max.  Weak duality makes g(mu) a lower bound of the constrained minimum f for every
    mu >= 0, reaching it at the optimal multiplier; checked here against the oracle's
    trust-region solve on underdetermined fits (more columns than rows, the active case)."""
    rng = np.random.default_rng(17)
    for trial in range(20):
        S, m = int(rng.integers(4, 12)), int(rng.integers(12, 30))
        A = rng.standard_normal((S, m))
        u = rng.standard_normal(S)
        G, b = A.T @ A, A.T @ u
        _, alpha_ls, _ = adaptive.trust_region_ls(A, u, 1e30)
        rho = 0.3 * np.linalg.norm(alpha_ls)          # the constraint is active
        f, alpha, mu_star = adaptive.trust_region_ls(A, u, rho)
        assert mu_star > 0
        for mu in np.concatenate([np.geomspace(1e-6, 1e3, 25), [mu_star]]):
            a = np.linalg.solve(G + mu * np.eye(m), b)
            g = u @ u - a @ b - mu * rho ** 2
            assert g <= f + 1e-9 * max(1.0, f), (trial, mu, g, f)
        a = np.linalg.solve(G + mu_star * np.eye(m), b)
        assert abs((u @ u - a @ b - mu_star * rho ** 2) - f) <= 1e-7 * max(1.0, f)
