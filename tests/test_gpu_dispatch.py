"""GPU parity at the largest online sizes: m = 224 with 4 labels and m = 200 with 16 labels (the
two-CTA cluster holds the adaptive choice and the m x m LU in shared memory; 16 labels take the
16-wide projection kernel), fixed m and adaptive m, caller priors, against the oracle (Eqs. Fs,
U_lin_comb, alpha_1); m = 224 with 16 labels exceeds one CTA's shared memory and is refused."""
import numpy as np
import pytest

import synth
from oracle import eig, graph, pipeline
from tests.gpu_common import TOL_PROB, dev, f32, gap_mask, to_dev

pytestmark = pytest.mark.gpu

rw = pytest.importorskip("paper_1607_04174_gb300")
torch = pytest.importorskip("torch")

M = 224


@pytest.fixture(scope="module")
def case():
    from paper_1607_04174_gb300 import build
    build.build()
    dims = (48, 48)
    J = f32(synth.smooth_random_image(dims, seed=11, smooth=3.0, sigma=0.02))
    go = graph.build_graph(J, dims, 60.0)
    lam, Q = eig.smallest_eigpairs(go.Lhat, M)
    return dict(J=J, dims=dims, g=go, lam=lam, Q=f32(Q))


def _setup(case, n_labels):
    go, J, dims = case["g"], case["J"], case["dims"]
    truth = np.minimum((J * n_labels).astype(np.int32), n_labels - 1)
    si, sl = synth.sample_seeds(truth, dims, 4, 1, seed=7, n_labels=n_labels)
    rng = np.random.default_rng(1)
    P = rng.uniform(0.1, 1.0, size=(go.N, n_labels))
    return si, sl, f32(P / P.sum(axis=1, keepdims=True))


def test_m224_with_16_labels_is_refused(case):
    si, sl, P = _setup(case, 16)
    g = rw.rw_build_graph(to_dev(case["J"], torch.float32), case["dims"], 60.0)
    b = rw.rw_basis_create(g, to_dev(case["Q"], torch.float32), case["lam"])
    try:
        prob = torch.empty(case["g"].N, 16, device=dev())
        with pytest.raises(rw.RWError) as e:
            rw.rw_solve(g, b, to_dev(si), to_dev(sl), 16, prob, priors=to_dev(P, torch.float32),
                        prior_mode=1, gamma=0.05, m=M)
        assert e.value.status == rw.RW_ERR_UNSUPPORTED
    finally:
        rw.rw_basis_free(b)
        rw.rw_graph_free(g)


@pytest.mark.parametrize("n_labels,m_max", [(4, M), (16, 200)])
@pytest.mark.parametrize("adaptive", [False, True])
def test_largest_m_matches_oracle(case, n_labels, m_max, adaptive):
    go, J, dims = case["g"], case["J"], case["dims"]
    si, sl, P = _setup(case, n_labels)
    Qm = np.ascontiguousarray(case["Q"][:, :m_max])
    lam = case["lam"][:m_max]
    g = rw.rw_build_graph(to_dev(J, torch.float32), dims, 60.0)
    b = rw.rw_basis_create(g, to_dev(Qm, torch.float32), lam)
    try:
        prob = torch.empty(go.N, n_labels, device=dev())
        lab = torch.empty(go.N, dtype=torch.uint8, device=dev())
        _, info = rw.rw_solve(g, b, to_dev(si), to_dev(sl), n_labels, prob, lab,
                              priors=to_dev(P, torch.float32), prior_mode=1, gamma=0.05,
                              m=0 if adaptive else m_max,
                              m_step=16, eps=0.05, refine_steps=3)
    finally:
        rw.rw_basis_free(b)
        rw.rw_graph_free(g)
    m_used = info["m_used"]
    assert (16 <= m_used <= m_max) if adaptive else m_used == m_max
    ref = pipeline.online_solve(go, Qm, lam, si, sl, n_labels, gamma=0.05, m=m_used,
                                refine_steps=3, P=P)
    U = prob.cpu().numpy().astype(np.float64)
    assert np.abs(U - ref["U"]).max() <= TOL_PROB
    mask = gap_mask(ref["U"])
    assert np.array_equal(lab.cpu().numpy()[mask], ref["labels"][mask])
