"""GPU parity: the offline eigensolver (Eq. L_eigs / z_eig) and the value updates of
Sec. III-B (Eq. z_ray) for beta changes, box-shaped local edits, edge lists and edge removal."""
import numpy as np
import pytest

import synth
from oracle import eig, graph, update
from tests.gpu_common import c1_case, dev, f32, to_dev

pytestmark = pytest.mark.gpu

rw = pytest.importorskip("paper_1607_04174_gb300")
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1607_04174_gb300 import build
    build.build()


def _eigs(J, dims, beta, m, normalized=True, **kw):
    g = rw.rw_build_graph(to_dev(J, torch.float32), dims, beta, rw.RW_WEIGHT_SQ, normalized)
    try:
        b, info = rw.rw_precompute(g, m, **kw)
        N = int(np.prod(dims))
        Q = torch.empty(N, m, device=dev())
        lam = rw.rw_basis_get(b, Q)
        rw.rw_basis_free(b)
        return lam, Q.cpu().numpy().astype(np.float64), info
    finally:
        rw.rw_graph_free(g)


def _check_eigs(lam_gpu, Q_gpu, lam_ref, Q_ref_ext, op):
    # eigenvalues: |d lambda| <= 1e-6 max(|lambda|, 1e-3)
    bound = 1e-6 * np.maximum(np.abs(lam_ref), 1e-3)
    assert np.all(np.abs(lam_gpu - lam_ref) <= bound), np.max(np.abs(lam_gpu - lam_ref) / bound)
    m = lam_gpu.size
    np.testing.assert_allclose(Q_gpu.T @ Q_gpu, np.eye(m), atol=2e-5)
    R = op @ Q_gpu - Q_gpu * lam_gpu
    assert np.linalg.norm(R, axis=0).max() <= 2e-5
    # the GPU columns lie in the span of the reference eigenvectors (plus guard)
    proj = Q_ref_ext.T @ Q_gpu
    assert np.linalg.norm(proj, axis=0).min() >= 1 - 1e-5


def test_lobpcg_config1_matches_dense_eigh():
    case = c1_case(m=70)
    lam, Q, info = _eigs(case["J"], case["dims"], 90.0, 50, tol=1e-6, seed=1)
    assert info["converged"] == 50
    _check_eigs(lam, Q, case["lam"][:50], case["Q"][:, :60], case["g"].Lhat)


def test_lobpcg_beta0_closed_form_unnormalized():
    dims = (24, 18)
    J = np.zeros(24 * 18)
    lam, Q, info = _eigs(J, dims, 0.0, 20, normalized=False, tol=1e-5, seed=2)
    vals = [4 * np.sin(np.pi * np.arange(n) / (2 * n)) ** 2 for n in dims]
    ref = np.sort((vals[0][:, None] + vals[1][None, :]).ravel())[:20]
    np.testing.assert_allclose(lam, ref, atol=1e-6 * 8)
    assert np.abs(Q.T @ Q - np.eye(20)).max() <= 2e-5


def test_lobpcg_3d():
    dims = (14, 12, 10)
    J = f32(synth.smooth_random_image(dims, seed=4, smooth=1.5, sigma=0.05))
    go = graph.build_graph(J, dims, 50.0)
    lr, Qr = eig.smallest_eigpairs(go.Lhat, 40)
    lam, Q, info = _eigs(J, dims, 50.0, 30, tol=1e-6, seed=3)
    _check_eigs(lam, Q, lr[:30], Qr, go.Lhat)


# ----------------------------------------------------------------------------- updates


def _basis_graph(case):
    g = rw.rw_build_graph(to_dev(case["J"], torch.float32), case["dims"], case["beta"])
    b = rw.rw_basis_create(g, to_dev(case["Q"], torch.float32), case["lam"])
    return g, b


def test_beta_update_matches_oracle_rayleigh():
    case = c1_case()
    g, b = _basis_graph(case)
    try:
        rw.rw_update_weights(g, b, rw.RW_UPDATE_BETA, beta=case["beta"])
        lam_same = rw.rw_basis_get(b)
        np.testing.assert_allclose(lam_same, case["lam"], rtol=2e-5, atol=2e-9)
        rw.rw_update_weights(g, b, rw.RW_UPDATE_BETA, beta=150.0)
        lam_new = rw.rw_basis_get(b)
        ref = update.updated_values(update.update_beta(case["g"], 150.0), case["Q"])
        np.testing.assert_allclose(lam_new, ref, rtol=2e-5, atol=1e-9)
    finally:
        rw.rw_basis_free(b)
        rw.rw_graph_free(g)


def test_roi_update_incremental_equals_oracle_full():
    dims = (24, 22, 20)
    J = f32(synth.smooth_random_image(dims, seed=6, smooth=1.5, sigma=0.05))
    go = graph.build_graph(J, dims, 50.0)
    Q = f32(synth.dct_basis(dims, 24))
    lam = update.rayleigh_quotients(Q, go.Lhat)
    case = dict(J=J, dims=dims, beta=50.0, Q=Q, lam=lam)
    lo, hi = (5, 0, 7), (15, 9, 20)   # touches two faces of the volume
    g, b = _basis_graph(case)
    try:
        rw.rw_update_weights(g, b, rw.RW_UPDATE_ROI, beta=100.0, roi_lo=lo, roi_hi=hi)
        got = rw.rw_basis_get(b)
        g2 = update.update_roi(go, lo, hi, 100.0)
        ref = update.updated_values(g2, Q)
        np.testing.assert_allclose(got, ref, rtol=2e-5, atol=1e-9)
        w = torch.empty(3 * go.N, device=dev())
        d = torch.empty(go.N, device=dev())
        rw.rw_graph_weights(g, w, d)
        np.testing.assert_allclose(w.cpu().numpy(), g2.weights_by_id(), rtol=2e-5, atol=1e-30)
        np.testing.assert_allclose(d.cpu().numpy(), g2.d, rtol=2e-5)
    finally:
        rw.rw_basis_free(b)
        rw.rw_graph_free(g)


def test_edge_list_update_and_removal():
    case = c1_case(size=40, per=8, m=30)
    go = case["g"]
    rng = np.random.default_rng(9)
    pos = np.sort(rng.choice(go.ids.size, 60, replace=False))
    ids = go.ids[pos]
    neww = f32(rng.uniform(0.05, 1.0, size=ids.size))
    g, b = _basis_graph(case)
    try:
        rw.rw_update_weights(g, b, rw.RW_UPDATE_EDGES, edge_ids=to_dev(ids.astype(np.int64)),
                             edge_w=to_dev(neww, torch.float32))
        ref = update.updated_values(update.update_edges(go, ids, neww), case["Q"])
        np.testing.assert_allclose(rw.rw_basis_get(b), ref, rtol=2e-5, atol=1e-9)
        rem = ids[:20]
        rw.rw_update_topology(g, b, rw.RW_TOPO_REMOVE_EDGES, edge_ids=to_dev(rem.astype(np.int64)))
        g2 = update.remove_edges(update.update_edges(go, ids, neww), rem)
        ref2 = update.updated_values(g2, case["Q"])
        np.testing.assert_allclose(rw.rw_basis_get(b), ref2, rtol=2e-5, atol=1e-9)
        bad = np.array([go.N - 1], np.int64)  # x = X-1: no forward edge along x
        with pytest.raises(rw.RWError) as e:
            rw.rw_update_topology(g, b, rw.RW_TOPO_REMOVE_EDGES, edge_ids=to_dev(bad))
        assert e.value.status == rw.RW_ERR_INVALID_ARG
    finally:
        rw.rw_basis_free(b)
        rw.rw_graph_free(g)


def test_multi_beta_bases_select_and_update():
    """Bases precomputed at beta' = 45, 90, 180 (Sec. III-B, last paragraph): for beta = 150
    the nearest in log beta (180) is chosen and updated by Eq. (z_ray); its values equal the
    oracle's Rayleigh quotients of that basis under beta = 150.  The distance of each choice's
    solve from the exact solve at beta = 150 is printed, not asserted (the paper compares such
    approximations only through segmentation quality)."""
    from oracle import exact, fastrw, priors
    case = c1_case(size=40, per=8, m=40)
    J, dims = case["J"], case["dims"]
    betas = [45.0, 90.0, 180.0]
    k = rw.rw_basis_nearest_beta(betas, 150.0)
    assert k == 2
    g150 = graph.build_graph(J, dims, 150.0)
    P = priors.gaussian_priors(J, case["si"], case["sl"], 2)
    Ue = exact.exact_rw(g150, case["si"], case["sl"], 2, P, 1e-3)
    errs = []
    for j, bp in enumerate(betas):
        go = graph.build_graph(J, dims, bp)
        lam, Q = eig.smallest_eigpairs(go.Lhat, 40)
        Q = f32(Q)
        g = rw.rw_build_graph(to_dev(J, torch.float32), dims, bp)
        b = rw.rw_basis_create(g, to_dev(Q, torch.float32), lam)
        try:
            rw.rw_update_weights(g, b, rw.RW_UPDATE_BETA, beta=150.0)
            got = rw.rw_basis_get(b)
            ref = update.updated_values(update.update_beta(go, 150.0), Q)
            np.testing.assert_allclose(got, ref, rtol=2e-5, atol=1e-9)
            prob = torch.empty(go.N, 2, device=dev())
            rw.rw_solve(g, b, to_dev(case["si"]), to_dev(case["sl"]), 2, prob, m=40,
                        refine_steps=0, basis_format=rw.RW_BASIS_F32, want_info=False)
            errs.append(float(np.abs(prob.cpu().numpy() - Ue).max()))
            if j == k:   # the chosen basis: GPU solve = oracle fast RW on the updated values
                Uf = fastrw.fast_rw(g150, Q, ref, case["si"], case["sl"], 2, P, 1e-3)
                assert np.abs(prob.cpu().numpy() - Uf).max() <= 1e-3
        finally:
            rw.rw_basis_free(b)
            rw.rw_graph_free(g)
    print("max |U - U_exact(beta=150)| from beta' = 45, 90, 180:", errs)
