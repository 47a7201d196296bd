"""GPU parity of registration (RWIR) through the C ABI against the FP64 oracle: the patch
priors of Sec. IV-B (3-D, 27 displacements; 2-D, 9), and the unseeded fast solve of
Eq. (U_lin_comb) with m chosen by Eq. (g) or fixed, refinement, the most probable label and the
expected displacement, with the 16-bit and the FP32 basis copies."""
import numpy as np
import pytest

import synth
from oracle import eig, graph, registration
from tests.gpu_common import TOL_PROB, dev, f32, gap_mask, to_dev

pytestmark = pytest.mark.gpu

rw = pytest.importorskip("paper_1607_04174_gb300")
torch = pytest.importorskip("torch")

BETA, GAMMA, M = 50.0, 1.0, 80


@pytest.fixture(scope="module")
def case3d():
    from paper_1607_04174_gb300 import build
    build.build()
    F, Mv, dims, u = synth.registration_pair(12, seed=synth.BASE_SEED + 5, field_smooth=3.0)
    F, Mv = f32(F), f32(Mv)
    disp = registration.displacement_labels()
    P = registration.registration_priors(F, Mv, dims, disp, half=2)
    go = graph.build_graph(F, dims, BETA)
    lam, Q = eig.smallest_eigpairs(go.Lhat, M)
    return dict(F=F, Mv=Mv, dims=dims, disp=disp, P=P, go=go, lam=lam, Q=f32(Q))


def test_registration_priors_3d(case3d):
    c = case3d
    N = c["go"].N
    P = torch.empty(N, 27, device=dev())
    rw.rw_registration_priors(to_dev(c["F"], torch.float32), to_dev(c["Mv"], torch.float32),
                              c["dims"], to_dev(c["disp"].astype(np.int32)), P, half=2)
    got = P.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(got, c["P"], rtol=2e-4, atol=2e-6)
    np.testing.assert_allclose(got.sum(axis=1), 1.0, atol=1e-5)


def test_registration_priors_2d():
    dims = (23, 17)
    F = f32(synth.smooth_random_image(dims, seed=8, smooth=2.0, sigma=0.02))
    Mv = f32(synth.smooth_random_image(dims, seed=9, smooth=2.0, sigma=0.02))
    disp = registration.displacement_labels(ndim=2)
    ref = registration.registration_priors(F, Mv, dims, disp, half=1)
    P = torch.empty(F.size, 9, device=dev())
    rw.rw_registration_priors(to_dev(F, torch.float32), to_dev(Mv, torch.float32), dims,
                              to_dev(disp.astype(np.int32)), P, half=1)
    np.testing.assert_allclose(P.cpu().numpy(), ref, rtol=2e-4, atol=2e-6)


@pytest.mark.parametrize("m,fmt", [(0, "f16"), (40, "f16"), (0, "f32")])
def test_unseeded_solve_matches_oracle(case3d, m, fmt):
    c = case3d
    go = c["go"]
    N = go.N
    g = rw.rw_build_graph(to_dev(c["F"], torch.float32), c["dims"], BETA)
    b = rw.rw_basis_create(g, to_dev(c["Q"], torch.float32), c["lam"])
    try:
        Pd = to_dev(c["P"], torch.float32)
        prob = torch.empty(N, 27, device=dev())
        lab = torch.empty(N, dtype=torch.uint8, device=dev())
        field = torch.empty(N, 3, device=dev())
        dd = to_dev(c["disp"].astype(np.int32))
        m_used = rw.rw_solve_unseeded(g, b, Pd, prob, lab, dd, field, gamma=GAMMA, m=m,
                                      m_step=10, eps=0.1, refine_steps=3,
                                      basis_format=rw.RW_BASIS_F16 if fmt == "f16" else rw.RW_BASIS_F32)
        P64 = f32(c["P"])
        if m == 0:
            from oracle import adaptive
            m_o, gv, _, table = adaptive.choose_m_from_priors(go, c["Q"], P64, M, 10, 0.1)
            if m_o != m_used:   # only a candidate sitting on the threshold may differ
                gmax = go.d.sum() * 0.01
                edge = min(m_o, m_used)
                assert abs(table[edge].max() - gmax) / gmax < 1e-3, (m_o, m_used)
        else:
            assert m_used == m
        ref = registration.registration_solve(go, c["Q"], c["lam"], P64, gamma=GAMMA, m=m_used,
                                              refine_steps=3)
        U = prob.cpu().numpy().astype(np.float64)
        err = np.abs(U - ref["U"]).max()
        print(f"unseeded solve m={m_used} ({fmt}): max |dU| = {err:.2e}")
        assert err <= TOL_PROB
        mask = gap_mask(ref["U"])
        assert np.array_equal(lab.cpu().numpy()[mask], np.argmax(ref["U"], 1)[mask])
        np.testing.assert_allclose(field.cpu().numpy(),
                                   registration.expected_displacement(U, c["disp"]),
                                   atol=1e-5)
    finally:
        rw.rw_basis_free(b)
        rw.rw_graph_free(g)


def test_unseeded_exact_solve_and_beta_gradient(case3d):
    """The basic RW with priors and no seeds (rw_solve_pcg, S = 0) and the exact-path gradient
    (rw_grad_exact, S = 0) against the oracle's FP64 solve and adjoint, 27 labels in two groups
    of columns (16 + 11)."""
    from oracle import adjoint, exact
    c = case3d
    go = c["go"]
    N = go.N
    P64 = f32(c["P"])
    none = np.zeros(0, np.int64)
    Ue = exact.exact_rw(go, none, none, 27, P64, GAMMA)
    G = np.random.default_rng(5).standard_normal((N, 27))
    gw_o, gb_o = adjoint.exact_grad(go, none, none, 27, P64, GAMMA, G, U=Ue)
    g = rw.rw_build_graph(to_dev(c["F"], torch.float32), c["dims"], BETA)
    try:
        U = np.zeros((N, 27))
        gw = np.zeros(3 * N)
        gb = 0.0
        for k0, k1 in ((0, 16), (16, 27)):
            Pc = to_dev(np.ascontiguousarray(P64[:, k0:k1]), torch.float32)
            Uc = torch.empty(N, k1 - k0, device=dev())
            rw.rw_solve_pcg(g, None, None, k1 - k0, Uc, priors=Pc, gamma=GAMMA, prior_mode=1,
                            iters=20000, tol=1e-7)
            U[:, k0:k1] = Uc.cpu().numpy()
            gwc = torch.empty(3 * N, device=dev())
            gb += rw.rw_grad_exact(g, None, None, k1 - k0, Pc, GAMMA, Uc,
                                   to_dev(np.ascontiguousarray(G[:, k0:k1]), torch.float32), gwc,
                                   rel_tol=1e-7, max_iter=20000)
            gw += gwc.cpu().numpy()
        assert np.abs(U - Ue).max() <= 1e-4
        by_id = np.zeros(3 * N)
        by_id[go.ids] = gw_o
        scale = np.abs(by_id).max()
        assert np.abs(gw - by_id).max() <= 1e-3 * scale
        print(f"registration d loss/d beta: GPU {gb:.6e}, oracle {gb_o:.6e}")
        assert abs(gb - gb_o) <= 1e-3 * abs(gb_o)
    finally:
        rw.rw_graph_free(g)


def test_unseeded_solve_few_labels_2d():
    """K = 3 labels (chunks of 4 padded columns) on a 2-D graph, fixed m, no refinement (the
    back-projection writes U directly)."""
    dims = (30, 26)
    F = f32(synth.smooth_random_image(dims, seed=14, smooth=2.0, sigma=0.02))
    go = graph.build_graph(F, dims, BETA)
    lam, Q = eig.smallest_eigpairs(go.Lhat, 50)
    Q = f32(Q)
    rng = np.random.default_rng(15)
    P = rng.random((go.N, 3)) + 0.2
    P = f32(P / P.sum(axis=1, keepdims=True))
    g = rw.rw_build_graph(to_dev(F, torch.float32), dims, BETA)
    b = rw.rw_basis_create(g, to_dev(Q, torch.float32), lam)
    try:
        prob = torch.empty(go.N, 3, device=dev())
        m_used = rw.rw_solve_unseeded(g, b, to_dev(P, torch.float32), prob, gamma=0.5, m=30,
                                      refine_steps=0)
        assert m_used == 30
        ref = registration.registration_solve(go, Q, lam, P, gamma=0.5, m=30, refine_steps=0)
        assert np.abs(prob.cpu().numpy() - ref["U"]).max() <= TOL_PROB
    finally:
        rw.rw_basis_free(b)
        rw.rw_graph_free(g)
