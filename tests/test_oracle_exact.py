"""Pins for the oracle's basic RW solve, Eq. (rw_eq) (Sec. II-A) and its normalized form
(Sec. II-C)."""
import json
import os

import numpy as np
import pytest

import synth
from oracle import exact, graph, priors

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_resistor_divider_closed_form():
    with open(os.path.join(GOLD, "chain_divider.json")) as f:
        fx = json.load(f)
    g = graph.build_graph(np.array(fx["J"]), fx["dims"], fx["beta"], fx["form"])
    for normalized in (False, True):   # with gamma = 0 both forms reduce to L_n U_n = -B^T U_s
        U = exact.exact_rw(g, np.array(fx["seed_idx"]), np.array(fx["seed_lab"]), 2, None, 0.0,
                           normalized=normalized)
        np.testing.assert_allclose(U[:, 1], fx["expected_u_label1"], atol=1e-14)


def _case(seed=0, dims=(16, 12), n_labels=3, per=4):
    J = synth.smooth_random_image(dims, seed=seed, smooth=2.0, sigma=0.03)
    truth = np.minimum((J * n_labels).astype(np.int32), n_labels - 1)
    si, sl = synth.sample_seeds(truth, dims, per, 1, seed=seed, n_labels=n_labels)
    g = graph.build_graph(J, dims, 40.0)
    P = priors.gaussian_priors(J, si, sl, n_labels)
    return g, si, sl, n_labels, P


@pytest.mark.parametrize("normalized", [True, False])
@pytest.mark.parametrize("gamma", [0.0, 1e-3, 0.5])
def test_max_principle_rowsums_and_seeds(normalized, gamma):
    g, si, sl, nl, P = _case()
    U = exact.exact_rw(g, si, sl, nl, P, gamma, normalized)
    assert U.min() >= -1e-12 and U.max() <= 1 + 1e-12
    np.testing.assert_allclose(U.sum(axis=1), 1.0, atol=1e-12)
    np.testing.assert_array_equal(U[si], exact.onehot(sl, nl))


def _energy(g, U, P, gamma, normalized):
    """Eq. (rw_energy) summed over labels, written with explicit edge sums; in the normalized
    formulation u-hat = D^{1/2} u, p-hat = D^{1/2} P and L-hat, which gives
    u^T L u + gamma (u - p)^T D (u - p)."""
    e = 0.0
    for k in range(U.shape[1]):
        u = U[:, k]
        e += sum(w * (u[a] - u[b]) ** 2 for a, b, w in zip(g.a, g.b, g.w))
        wgt = g.d if normalized else np.ones(g.N)
        if gamma > 0:
            e += gamma * np.sum(wgt * (u - P[:, k]) ** 2)
    return e


@pytest.mark.parametrize("normalized", [True, False])
def test_solution_minimizes_the_energy(normalized):
    g, si, sl, nl, P = _case(seed=1, dims=(9, 7))
    gamma = 0.05
    U = exact.exact_rw(g, si, sl, nl, P, gamma, normalized)
    rng = np.random.default_rng(5)
    n = exact.split(g.N, si)
    e0 = _energy(g, U, P, gamma, normalized)
    for _ in range(4):
        d = np.zeros_like(U)
        d[n] = rng.standard_normal((n.size, nl))
        t = 1e-3
        ep, em = _energy(g, U + t * d, P, gamma, normalized), _energy(g, U - t * d, P, gamma, normalized)
        assert ep > e0 and em > e0
        assert abs(ep - em) / (2 * t) < 1e-8 * max(1.0, e0)       # first variation vanishes


def test_splu_and_cg_agree():
    g, si, sl, nl, P = _case(seed=2, dims=(20, 20))
    U1 = exact.exact_rw(g, si, sl, nl, P, 1e-2, True, method="splu")
    U2 = exact.exact_rw(g, si, sl, nl, P, 1e-2, True, method="cg", tol=1e-13)
    np.testing.assert_allclose(U1, U2, atol=1e-9)


def test_planted_mistake_is_caught(monkeypatch):
    """A dropped prior term in the oracle's system must break the energy pin."""
    g, si, sl, nl, P = _case(seed=1, dims=(9, 7))
    real = exact.system

    def broken(*a, **k):
        A, rhs, n = real(*a, **k)
        return A, rhs - 0.05 * a[4][n] * 0.5, n        # wrong prior scaling
    monkeypatch.setattr(exact, "system", broken)
    U = exact.exact_rw(g, si, sl, nl, P, 0.05, True)
    d = np.zeros_like(U)
    d[exact.split(g.N, si)] = 1.0
    t = 1e-3
    slope = (_energy(g, U + t * d, P, 0.05, True) - _energy(g, U - t * d, P, 0.05, True)) / (2 * t)
    assert abs(slope) > 1e-4
