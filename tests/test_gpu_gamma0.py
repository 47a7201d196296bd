"""GPU parity of the gamma = 0 fast RW (no priors; Sec. II-B, the paragraph after Eq. Fs: L-hat
has the null vector g, E is its pseudo-inverse and the column sums c = g^T U-hat enter the
seeded system) through the C ABI, against the oracle's bordered system (``fastrw.fast_rw_gamma0``
via ``pipeline.online_solve(gamma=0)``): fixed and adaptive m, 16-bit and FP32 basis, refinement,
2-D and 3-D, the unnormalized Laplacian, a constant labelling, the full 512^2 size, and the
basic RW (PCG) at gamma = 0 against the exact solve of Eq. (rw_eq)."""
import numpy as np
import pytest

import synth
from oracle import eig, exact, graph, pipeline, update
from tests.gpu_common import TOL_PROB, c1_case, dev, f32, gap_mask, to_dev

pytestmark = pytest.mark.gpu

rw = pytest.importorskip("paper_1607_04174_gb300")
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1607_04174_gb300 import build
    build.build()


def _solve(case, m, steps, fmt=rw.RW_BASIS_F16, n_labels=2, m_step=10, normalized=True,
           refine_mode=rw.RW_REFINE_JACOBI, si=None, sl=None):
    si = case["si"] if si is None else si
    sl = case["sl"] if sl is None else sl
    g = rw.rw_build_graph(to_dev(case["J"], torch.float32), case["dims"], case["beta"],
                          normalized=normalized)
    b = rw.rw_basis_create(g, to_dev(case["Q"], torch.float32), case["lam"])
    try:
        N = case["g"].N
        prob = torch.empty(N, n_labels, device=dev())
        lab = torch.empty(N, dtype=torch.uint8, device=dev())
        s, info = rw.rw_solve(g, b, to_dev(si.astype(np.int32)), to_dev(sl.astype(np.int32)),
                              n_labels, prob, lab, gamma=0.0, m=m, m_step=m_step,
                              refine_steps=steps, basis_format=fmt, refine_mode=refine_mode)
        return prob.cpu().numpy().astype(np.float64), lab.cpu().numpy(), info
    finally:
        rw.rw_basis_free(b)
        rw.rw_graph_free(g)


def _check(U, lab, ref, tol):
    err = np.abs(U - ref["U"]).max()
    assert err <= tol, err
    mask = gap_mask(ref["U"])
    assert np.array_equal(lab[mask], ref["labels"][mask])
    return err


@pytest.fixture(scope="module")
def c1():
    return c1_case()


@pytest.mark.parametrize("fmt,tol", [(rw.RW_BASIS_F16, TOL_PROB), (rw.RW_BASIS_F32, 1e-4)])
@pytest.mark.parametrize("m,steps", [(50, 0), (50, 3), (17, 0), (1, 0)])
def test_fixed_m_matches_oracle(c1, fmt, tol, m, steps):
    U, lab, info = _solve(c1, m, steps, fmt)
    ref = pipeline.online_solve(c1["g"], c1["Q"], c1["lam"], c1["si"], c1["sl"], 2, gamma=0.0,
                                m=m, refine_steps=steps)
    err = _check(U, lab, ref, tol)
    print(f"gamma = 0, m = {m}, {steps} steps: max |dU| = {err:.2e}")
    assert info["m_used"] == m
    assert info["mu"] == [0.0, 0.0]
    np.testing.assert_allclose(U.sum(axis=1), 1.0, atol=tol)


def test_adaptive_m_matches_oracle(c1):
    U, lab, info = _solve(c1, 0, 3, m_step=5)
    from oracle import adaptive, fastrw
    Qt = fastrw.gamma0_basis(c1["g"], c1["Q"])
    m_o, f_o, _, table = adaptive.choose_m_from_seeds(c1["g"], Qt, c1["si"], c1["sl"], 2,
                                                      Qt.shape[1], 5, 0.1)
    if info["m_used"] != m_o:   # only a candidate on the threshold may differ
        fmax = len(c1["si"]) * 0.01
        edge = min(info["m_used"], m_o)
        assert abs(table[edge].max() - fmax) / fmax < 1e-3, (info["m_used"], m_o)
    else:
        np.testing.assert_allclose(info["f"], f_o, rtol=1e-3, atol=1e-6)
    ref = pipeline.online_solve(c1["g"], c1["Q"], c1["lam"], c1["si"], c1["sl"], 2, gamma=0.0,
                                m=info["m_used"], refine_steps=3)
    _check(U, lab, ref, TOL_PROB)


def test_constant_labelling_is_reproduced(c1):
    sl = np.zeros_like(c1["sl"])
    for fmt, tol in ((rw.RW_BASIS_F32, 1e-4), (rw.RW_BASIS_F16, TOL_PROB)):
        U, lab, _ = _solve(c1, 30, 0, fmt, sl=sl)
        assert np.abs(U[:, 0] - 1.0).max() <= tol
        assert np.abs(U[:, 1]).max() <= tol
        assert np.all(lab == 0)


def test_three_labels_3d():
    dims = (18, 15, 13)
    J = f32(synth.smooth_random_image(dims, seed=synth.BASE_SEED + 9, smooth=2.0, sigma=0.02))
    truth = np.minimum((J * 3).astype(np.int32), 2)
    n_labels = 3
    si, sl = synth.sample_seeds(truth, dims, 12, 1, seed=synth.BASE_SEED + 9, n_labels=3)
    go = graph.build_graph(J, dims, 90.0)
    lam, Q = eig.smallest_eigpairs(go.Lhat, 60)
    case = dict(J=J, dims=dims, g=go, lam=lam, Q=f32(Q), beta=90.0, si=si, sl=sl)
    for m, steps in ((60, 0), (33, 3)):
        U, lab, _ = _solve(case, m, steps, n_labels=n_labels)
        ref = pipeline.online_solve(go, case["Q"], lam, si, sl, n_labels, gamma=0.0, m=m,
                                    refine_steps=steps)
        _check(U, lab, ref, TOL_PROB)


def test_unnormalized_laplacian():
    J = f32(synth.smooth_random_image((31, 27), seed=21, smooth=2.0, sigma=0.05))
    dims = (31, 27)
    go = graph.build_graph(J, dims, 60.0)
    lam, Q = eig.smallest_eigpairs(go.L, 40)
    rng = np.random.default_rng(22)
    si = np.sort(rng.choice(go.N, size=24, replace=False))
    sl = (np.arange(24) % 3).astype(np.int64)
    case = dict(J=J, dims=dims, g=go, lam=lam, Q=f32(Q), beta=60.0, si=si, sl=sl)
    U, lab, _ = _solve(case, 40, 2, rw.RW_BASIS_F32, n_labels=3, normalized=False)
    ref = pipeline.online_solve(go, case["Q"], lam, si, sl, 3, gamma=0.0, m=40, refine_steps=2,
                                normalized=False)
    _check(U, lab, ref, 1e-4)


def test_pcg_refinement_and_basic_rw_reach_the_exact_solve(c1):
    """Many PCG refinement steps after the gamma = 0 projection, and the basic RW by PCG
    (rw_solve_pcg, gamma = 0), both against the exact L_n U_n = -B^T U_s."""
    Ue = exact.exact_rw(c1["g"], c1["si"], c1["sl"], 2, None, 0.0)
    U, _, _ = _solve(c1, 50, 400, rw.RW_BASIS_F32, refine_mode=rw.RW_REFINE_PCG)
    assert np.abs(U - Ue).max() <= 1e-4
    g = rw.rw_build_graph(to_dev(c1["J"], torch.float32), c1["dims"], c1["beta"])
    try:
        prob = torch.empty(c1["g"].N, 2, device=dev())
        rw.rw_solve_pcg(g, to_dev(c1["si"].astype(np.int32)), to_dev(c1["sl"].astype(np.int32)),
                        2, prob, gamma=0.0, iters=5000, tol=1e-7)
        assert np.abs(prob.cpu().numpy() - Ue).max() <= 1e-4
        with pytest.raises(rw.RWError):   # no seeds and no priors: singular
            rw.rw_solve_pcg(g, None, None, 2, prob, gamma=0.0, prior_mode=1,
                            priors=torch.full((c1["g"].N, 2), 0.5, device=dev()))
    finally:
        rw.rw_graph_free(g)


def test_negative_gamma_is_rejected(c1):
    g = rw.rw_build_graph(to_dev(c1["J"], torch.float32), c1["dims"], c1["beta"])
    b = rw.rw_basis_create(g, to_dev(c1["Q"], torch.float32), c1["lam"])
    try:
        prob = torch.empty(c1["g"].N, 2, device=dev())
        with pytest.raises(rw.RWError):
            rw.rw_solve(g, b, to_dev(c1["si"].astype(np.int32)), to_dev(c1["sl"].astype(np.int32)),
                        2, prob, gamma=-1e-3)
    finally:
        rw.rw_basis_free(b)
        rw.rw_graph_free(g)


def test_full_size_512_dct_basis():
    """512^2, 4 labels, 200 seeds per label: fixed m = 200 and adaptive m with 3 refinement
    steps, against the oracle on every voxel (the basis is the DCT one of the gamma > 0 full-size
    test: its column 0 is replaced by g and the rest projected, on both sides)."""
    J, dims, truth = synth.voronoi_image(512, 512, seed=synth.BASE_SEED + 1)
    J = f32(J)
    si, sl = synth.sample_seeds(truth, dims, 200, 3, seed=synth.BASE_SEED + 1)
    go = graph.build_graph(J, dims, 90.0)
    Q = f32(synth.dct_basis(dims, 200))
    lam = update.rayleigh_quotients(Q, go.Lhat)
    case = dict(J=J, dims=dims, si=si, sl=sl, g=go, lam=lam, Q=Q, beta=90.0)
    for m, steps in ((200, 3), (0, 3)):
        U, lab, info = _solve(case, m, steps, n_labels=4)
        ref = pipeline.online_solve(go, Q, lam, si, sl, 4, gamma=0.0, m=info["m_used"],
                                    refine_steps=steps)
        err = _check(U, lab, ref, TOL_PROB)
        print(f"512^2 gamma = 0, m = {info['m_used']}: max |dU| = {err:.2e}")
