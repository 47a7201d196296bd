"""Pins of the oracle's gamma = 0 fast RW (Sec. II-B, the paragraph after Eq. Fs: L-hat has the
null vector g, E is its pseudo-inverse, E L-hat = I - g g^T, and the column sums g^T U-hat enter
the seeded system).

* With all N eigenvectors (m = N) the bordered system is exact: equal to the basic RW of
  Eq. (rw_eq) at gamma = 0, normalized and unnormalized.
* At any m a constant labelling is reproduced exactly (one label seeded everywhere gives U = 1),
  and the rows of U sum to 1.
* The factored and the explicit-E restatements agree.
* The result does not change when g-components are added to the stored columns or column 0 is
  replaced: the basis is [g, (I - g g^T) Q[:, 1:]].
* A planted mistake (the border dropped, c = 0) breaks the row sums."""
import numpy as np
import pytest

import synth
from oracle import exact, fastrw, graph, pipeline


def _graph(dims=(7, 6), seed=3):
    J = synth.smooth_random_image(dims, seed=seed, smooth=1.5, sigma=0.05)
    return graph.build_graph(J, dims, 60.0), J


def _seeds(N, n_labels, seed, S=8):
    rng = np.random.default_rng(seed)
    si = np.sort(rng.choice(N, size=S, replace=False))
    sl = np.arange(S) % n_labels
    rng.shuffle(sl)
    return si, sl


def _eig(g, normalized):
    A = (g.Lhat if normalized else g.L).toarray()
    lam, Q = np.linalg.eigh(A)
    return lam, Q


@pytest.mark.parametrize("normalized", [True, False])
def test_full_rank_equals_exact(normalized):
    g, _ = _graph()
    lam, Q = _eig(g, normalized)
    assert abs(lam[0]) < 1e-10 and lam[1] > 1e-6
    si, sl = _seeds(g.N, 3, 1)
    U = fastrw.fast_rw_gamma0(g, Q, lam, si, sl, 3, normalized)
    Ue = exact.exact_rw(g, si, sl, 3, None, 0.0, normalized)
    assert np.abs(U - Ue).max() < 1e-10


def test_constant_labelling_reproduced_at_any_m():
    g, _ = _graph((9, 8), seed=5)
    lam, Q = _eig(g, True)
    si, _ = _seeds(g.N, 1, 2, S=6)
    sl = np.ones(si.size, dtype=np.int64)
    for m in (1, 2, 7, 20):
        U = fastrw.fast_rw_gamma0(g, Q[:, :m], lam[:m], si, sl, 3)
        np.testing.assert_allclose(U[:, 1], 1.0, atol=1e-12)
        np.testing.assert_allclose(U[:, [0, 2]], 0.0, atol=1e-12)


@pytest.mark.parametrize("m", [5, 12, 30])
def test_rows_sum_to_one_and_restatements_agree(m):
    g, _ = _graph((9, 8), seed=6)
    lam, Q = _eig(g, True)
    si, sl = _seeds(g.N, 3, 4, S=9)
    U = fastrw.fast_rw_gamma0(g, Q[:, :m], lam[:m], si, sl, 3)
    Ud = fastrw.fast_rw_gamma0_dense(g, Q[:, :m], lam[:m], si, sl, 3)
    np.testing.assert_allclose(U.sum(axis=1), 1.0, atol=1e-10)
    assert np.abs(U - Ud).max() < 1e-10


def test_invariant_to_null_components_of_the_stored_columns():
    g, _ = _graph((9, 8), seed=7)
    lam, Q = _eig(g, True)
    m = 15
    si, sl = _seeds(g.N, 2, 5, S=7)
    U = fastrw.fast_rw_gamma0(g, Q[:, :m], lam[:m], si, sl, 2)
    gv = fastrw.null_vector(g)
    rng = np.random.default_rng(9)
    Q2 = Q[:, :m].copy()
    Q2[:, 1:] += np.outer(gv, 0.3 * rng.standard_normal(m - 1))
    Q2[:, 0] = rng.standard_normal(g.N)          # column 0 is replaced by g
    U2 = fastrw.fast_rw_gamma0(g, Q2, lam[:m], si, sl, 2)
    assert np.abs(U - U2).max() < 1e-10


def test_unnormalized_null_vector_is_constant():
    g, _ = _graph()
    np.testing.assert_allclose(fastrw.null_vector(g, normalized=False), 1.0 / np.sqrt(g.N))
    gv = fastrw.null_vector(g)
    assert np.abs(g.Lhat @ gv).max() < 1e-12
    np.testing.assert_allclose(np.linalg.norm(gv), 1.0)


def test_pipeline_gamma0_chooses_m_on_the_gamma0_basis():
    g, _ = _graph((10, 9), seed=8)
    lam, Q = _eig(g, True)
    si, sl = _seeds(g.N, 2, 6, S=10)
    r = pipeline.online_solve(g, Q[:, :40], lam[:40], si, sl, 2, gamma=0.0, m=0, m_step=5,
                              refine_steps=0)
    U = fastrw.fast_rw_gamma0(g, Q[:, :r["m"]], lam[:r["m"]], si, sl, 2)
    assert np.abs(r["U"] - U).max() < 1e-12
    assert r["P"] is None
    # refinement at gamma = 0 moves toward the exact solve
    Ue = exact.exact_rw(g, si, sl, 2, None, 0.0)
    r5 = pipeline.online_solve(g, Q[:, :40], lam[:40], si, sl, 2, gamma=0.0, m=r["m"],
                               refine_steps=200)
    assert np.abs(r5["U"] - Ue).max() < np.abs(r["U"] - Ue).max()


def test_a_dropped_border_is_caught(monkeypatch):
    """With c forced to 0 (the column sums ignored) the rows no longer sum to 1."""
    g, _ = _graph((9, 8), seed=6)
    lam, Q = _eig(g, True)
    si, sl = _seeds(g.N, 3, 4, S=9)
    real = np.linalg.solve

    def no_border(A, b):
        x = real(A, b)
        if A.shape[0] == si.size + 1:
            x[-1] = 0.0
        return x
    monkeypatch.setattr(fastrw.np.linalg, "solve", no_border)
    U = fastrw.fast_rw_gamma0(g, Q[:, :12], lam[:12], si, sl, 3)
    assert np.abs(U.sum(axis=1) - 1.0).max() > 1e-3
