"""Pins for the oracle's image graph (Sec. II-A, Eq. W; Sec. II-C normalized Laplacian)."""
import json
import os

import numpy as np
import pytest

import synth
from oracle import graph

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def test_hand_worked_2x2_weights_and_degrees():
    fx = _load("grid_2x2_weights.json")
    g = graph.build_graph(np.array(fx["J"]), fx["dims"], fx["beta"], fx["form"])
    np.testing.assert_array_equal(g.ids, fx["expected_ids"])
    np.testing.assert_allclose(g.w, fx["expected_w"], rtol=1e-15)
    np.testing.assert_allclose(g.d, fx["expected_d"], rtol=1e-15)


def test_paper_abs_form_chain_weights():
    fx = _load("chain_divider.json")
    g = graph.build_graph(np.array(fx["J"]), fx["dims"], fx["beta"], fx["form"])
    np.testing.assert_allclose(g.w, fx["expected_weights"], rtol=1e-14)


@pytest.mark.parametrize("dims", [(7, 5), (4, 3, 5)])
@pytest.mark.parametrize("form", ["sq", "abs"])
def test_laplacian_identities(dims, form):
    J = synth.smooth_random_image(dims, seed=3, smooth=1.0, sigma=0.1)
    g = graph.build_graph(J, dims, 30.0, form)
    N = g.N
    # edge count of the 4-/6-neighbour grid
    ne = sum(int(np.prod(dims)) // dims[a] * (dims[a] - 1) for a in range(len(dims)))
    assert g.ids.size == ne
    L = g.L.toarray()
    Lh = g.Lhat.toarray()
    assert np.abs(L - L.T).max() == 0
    np.testing.assert_allclose(L @ np.ones(N), 0, atol=1e-14)               # L 1 = 0
    np.testing.assert_allclose(Lh @ np.sqrt(g.d), 0, atol=1e-14)            # L-hat D^1/2 1 = 0
    np.testing.assert_allclose(np.diag(Lh), 1.0, atol=1e-15)
    ev = np.linalg.eigvalsh(Lh)
    assert ev.min() > -1e-12 and ev.max() < 2 + 1e-12                       # spectrum in [0, 2]
    # quadratic form as an explicit sum over edges: u^T L u = sum_e w_e (u_a - u_b)^2
    u = np.random.default_rng(0).standard_normal(N)
    q = sum(w * (u[a] - u[b]) ** 2 for a, b, w in zip(g.a, g.b, g.w))
    np.testing.assert_allclose(u @ L @ u, q, rtol=1e-12)


def test_edge_layout_matches_ids():
    dims = (3, 2, 2)
    ids, a, b = graph.forward_edges(dims)
    N = 12
    for e, i, j in zip(ids, a, b):
        ax, src = divmod(int(e), N)
        assert src == i
        assert j - i == (1, 3, 6)[ax]


def test_isolated_node_rejected_in_normalized_mode():
    J = np.array([0.0, 0.0, 1.0, 1.0])
    g = graph.build_graph(J, (4, 1), 1.0)
    g2 = graph.set_edge_weights(g, np.array([0]), 0.0)   # voxel 0 loses its only edge
    with pytest.raises(ValueError):
        g2.Lhat
