"""The tensor-core basis passes (projection Z = Q_n^T P-hat_n and back-projection U-hat_n = Q_n C
of Eq. U_lin_comb on tcgen05, csrc/proj_tc.cu) against the CUDA-core kernels on the same
inputs, through the C ABI: every label padding (4, 8, 16), ragged m (1, 17, 50 and the adaptive
choice), 0 and 3 refinement steps, the FP16 and BF16 copies, gamma = 0 (the null-vector term of
the back-projection), a 200-column copy, and the unseeded registration solve; the tensor-core
results also against the oracle."""
import numpy as np
import pytest

import synth
from oracle import eig, graph, pipeline, priors, registration
from tests.gpu_common import TOL_PROB, c1_case, dev, f32, gap_mask, to_dev

pytestmark = pytest.mark.gpu

rw = pytest.importorskip("paper_1607_04174_gb300")
torch = pytest.importorskip("torch")

TOL_SAME = {rw.RW_BASIS_F16: 2e-5, rw.RW_BASIS_BF16: 2e-4}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1607_04174_gb300 import build
    build.build()
    yield
    rw.rw_set_tc_passes(4)


def _both(case, n_labels, **kw):
    g = rw.rw_build_graph(to_dev(case["J"], torch.float32), case["dims"], case["beta"])
    b = rw.rw_basis_create(g, to_dev(case["Q"], torch.float32), case["lam"])
    out = []
    try:
        for tc in (3, 0):
            rw.rw_set_tc_passes(tc)
            prob = torch.empty(case["g"].N, n_labels, device=dev())
            lab = torch.empty(case["g"].N, dtype=torch.uint8, device=dev())
            _, info = rw.rw_solve(g, b, to_dev(case["si"].astype(np.int32)),
                                  to_dev(case["sl"].astype(np.int32)), n_labels, prob, lab, **kw)
            out.append((prob.cpu().numpy().astype(np.float64), lab.cpu().numpy(), info))
    finally:
        rw.rw_set_tc_passes(4)
        rw.rw_basis_free(b)
        rw.rw_graph_free(g)
    return out


@pytest.fixture(scope="module")
def c1():
    return c1_case()


@pytest.mark.parametrize("fmt", [rw.RW_BASIS_F16, rw.RW_BASIS_BF16])
@pytest.mark.parametrize("m,steps", [(50, 0), (50, 3), (17, 0), (1, 0), (0, 3)])
def test_two_labels_match_cuda_cores(c1, fmt, m, steps):
    (Ut, lt, it), (Uc, lc, ic) = _both(c1, 2, gamma=1e-3, m=m, refine_steps=steps,
                                       basis_format=fmt)
    assert it["m_used"] == ic["m_used"]
    assert np.abs(Ut - Uc).max() <= TOL_SAME[fmt]
    mask = gap_mask(Uc)
    assert np.array_equal(lt[mask], lc[mask])
    if fmt == rw.RW_BASIS_F16:
        ref = pipeline.online_solve(c1["g"], c1["Q"], c1["lam"], c1["si"], c1["sl"], 2,
                                    gamma=1e-3, m=it["m_used"], refine_steps=steps)
        assert np.abs(Ut - ref["U"]).max() <= TOL_PROB


@pytest.mark.parametrize("n_labels", [6, 12])
def test_eight_and_sixteen_label_padding(n_labels):
    dims = (40, 36)
    J = f32(synth.smooth_random_image(dims, seed=31, smooth=2.0, sigma=0.02))
    truth = np.minimum((J * n_labels).astype(np.int32), n_labels - 1)
    si, sl = synth.sample_seeds(truth, dims, 3, 1, seed=32, n_labels=n_labels)
    go = graph.build_graph(J, dims, 90.0)
    lam, Q = eig.smallest_eigpairs(go.Lhat, 70)
    case = dict(J=J, dims=dims, g=go, lam=lam, Q=f32(Q), beta=90.0, si=si, sl=sl)
    P = priors.gaussian_priors(J, si, sl, n_labels)
    for steps in (0, 3):
        (Ut, _, _), (Uc, _, _) = _both(case, n_labels, gamma=0.05, m=70, refine_steps=steps)
        assert np.abs(Ut - Uc).max() <= 2e-5
        ref = pipeline.online_solve(go, case["Q"], lam, si, sl, n_labels, gamma=0.05, m=70,
                                    refine_steps=steps, P=P)
        assert np.abs(Ut - ref["U"]).max() <= TOL_PROB


def test_gamma0_null_term(c1):
    (Ut, _, _), (Uc, _, _) = _both(c1, 2, gamma=0.0, m=50, refine_steps=0)
    assert np.abs(Ut - Uc).max() <= 2e-5
    np.testing.assert_allclose(Ut.sum(axis=1), 1.0, atol=TOL_PROB)


def test_unseeded_registration_solve():
    F, Mv, dims, _ = synth.registration_pair(12, seed=synth.BASE_SEED + 5, field_smooth=3.0)
    F, Mv = f32(F), f32(Mv)
    disp = registration.displacement_labels()
    P = f32(registration.registration_priors(F, Mv, dims, disp, half=2))
    go = graph.build_graph(F, dims, 50.0)
    lam, Q = eig.smallest_eigpairs(go.Lhat, 80)
    g = rw.rw_build_graph(to_dev(F, torch.float32), dims, 50.0)
    b = rw.rw_basis_create(g, to_dev(f32(Q), torch.float32), lam)
    out = []
    try:
        for tc in (3, 0):
            rw.rw_set_tc_passes(tc)
            prob = torch.empty(go.N, 27, device=dev())
            m_used = rw.rw_solve_unseeded(g, b, to_dev(P, torch.float32), prob, gamma=1.0, m=0,
                                          m_step=10, eps=0.1, refine_steps=3)
            out.append((prob.cpu().numpy().astype(np.float64), m_used))
    finally:
        rw.rw_set_tc_passes(4)
        rw.rw_basis_free(b)
        rw.rw_graph_free(g)
    (Ut, mt), (Uc, mc) = out
    assert mt == mc
    assert np.abs(Ut - Uc).max() <= 2e-5
    ref = registration.registration_solve(go, f32(Q), lam, P, gamma=1.0, m=mt, refine_steps=3)
    assert np.abs(Ut - ref["U"]).max() <= TOL_PROB


@pytest.mark.parametrize("m", [64, 136, 200])
def test_wide_basis_each_pass_alone(m):
    """A 200-column copy (two 128-column halves in the projection, four 64-column blocks in
    the back-projection, fewer pipeline stages) on 160^2 voxels (several tiles per block):
    each pass on the tensor cores alone and both together against both on the CUDA cores."""
    J, dims, truth = synth.voronoi_image(160, 160, seed=synth.BASE_SEED + 3)
    J = f32(J)
    si, sl = synth.sample_seeds(truth, dims, 50, 3, seed=synth.BASE_SEED + 3)
    go = graph.build_graph(J, dims, 90.0)
    Q = f32(synth.dct_basis(dims, 200))
    from oracle import update
    lam = update.rayleigh_quotients(Q, go.Lhat)
    g = rw.rw_build_graph(to_dev(J, torch.float32), dims, 90.0)
    b = rw.rw_basis_create(g, to_dev(Q, torch.float32), lam)
    res = {}
    try:
        for mask in (0, 1, 2, 3):
            rw.rw_set_tc_passes(mask)
            prob = torch.empty(go.N, 4, device=dev())
            rw.rw_solve(g, b, to_dev(si.astype(np.int32)), to_dev(sl.astype(np.int32)), 4, prob,
                        gamma=1e-3, m=m, refine_steps=0)
            res[mask] = prob.cpu().numpy().astype(np.float64)
    finally:
        rw.rw_set_tc_passes(4)
        rw.rw_basis_free(b)
        rw.rw_graph_free(g)
    for mask in (1, 2, 3):
        assert np.abs(res[mask] - res[0]).max() <= 2e-5, mask
