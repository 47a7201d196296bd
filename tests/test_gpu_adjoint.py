"""GPU parity: gradients of a squared segmentation loss through the exact random walker
(Eq. rw_eq, normalized form of Sec. II-C) with respect to every edge weight and beta (Eq. W),
against the oracle's FP64 adjoint on the same float32 inputs."""
import numpy as np
import pytest

import synth
from oracle import adjoint, exact, graph, priors
from tests.gpu_common import dev, f32, to_dev

pytestmark = pytest.mark.gpu

rw = pytest.importorskip("paper_1607_04174_gb300")
torch = pytest.importorskip("torch")

# The adjoint runs FP32 Jacobi-PCG to ||r|| <= 1e-6 ||b||; the per-edge products are FP32.
GRAD_RTOL = 2e-3   # max |g_gpu - g_ref| <= GRAD_RTOL * max |g_ref|


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1607_04174_gb300 import build
    build.build()


def _gpu_grad(J, dims, beta, normalized, si, sl, P, gamma, U, G):
    gg = rw.rw_build_graph(to_dev(J, torch.float32), dims, beta, rw.RW_WEIGHT_SQ, normalized)
    try:
        N = int(np.prod(dims))
        gw = torch.full((len(dims) * N,), float("nan"), device=dev())
        gb = rw.rw_grad_exact(gg, to_dev(si.astype(np.int32)), to_dev(sl.astype(np.int32)),
                              P.shape[1], to_dev(P, torch.float32), gamma,
                              to_dev(U, torch.float32), to_dev(G, torch.float32), gw,
                              rel_tol=1e-6, max_iter=50000)
        return gw.cpu().numpy().astype(np.float64), gb
    finally:
        rw.rw_graph_free(gg)


def _check_case(J, dims, truth, si, sl, beta, gamma, normalized):
    g = graph.build_graph(J, dims, beta)
    P = f32(priors.gaussian_priors(J, si, sl, 2))
    U = f32(exact.exact_rw(g, si, sl, 2, P, gamma, normalized))
    _, G = adjoint.mask_loss(U, truth.astype(np.float64), si, label=1)
    G = f32(G)
    gw_ref, gb_ref = adjoint.exact_grad(g, si, sl, 2, P, gamma, G, normalized, U=U)
    full_ref = np.zeros(len(dims) * g.N)
    full_ref[g.ids] = gw_ref
    gw, gb = _gpu_grad(J, dims, beta, normalized, si, sl, P, gamma, U, G)
    assert np.all(np.isfinite(gw))
    scale = np.abs(full_ref).max()
    assert scale > 0
    err = np.abs(gw - full_ref).max()
    assert err <= GRAD_RTOL * scale, (err, scale)
    # no-edge slots (last slice along each axis) are written as 0
    missing = np.setdiff1d(np.arange(len(dims) * g.N), g.ids)
    assert np.all(gw[missing] == 0.0)
    assert abs(gb - gb_ref) <= GRAD_RTOL * abs(gb_ref), (gb, gb_ref)


def test_exact_gradient_2d_normalized():
    J, dims, truth = synth.closed_curve_image(64, seed=synth.BASE_SEED)
    J = f32(J)
    si, sl = synth.sample_seeds(truth, dims, 20, 2, seed=synth.BASE_SEED)
    _check_case(J, dims, truth, si, sl, 90.0, 1e-3, True)


def test_exact_gradient_3d_unnormalized():
    J, dims, truth = synth.ellipsoid_volume(20, seed=synth.BASE_SEED + 2)
    J = f32(J)
    si, sl = synth.sample_seeds(truth, dims, 30, 2, seed=synth.BASE_SEED + 2)
    _check_case(J, dims, truth, si, sl, 50.0, 1e-2, False)


def test_exact_gradient_rejects_bad_arguments():
    J, dims, truth = synth.closed_curve_image(32, seed=synth.BASE_SEED)
    si, sl = synth.sample_seeds(truth, dims, 5, 2, seed=synth.BASE_SEED)
    gg = rw.rw_build_graph(to_dev(f32(J), torch.float32), dims, 90.0)
    try:
        N = int(np.prod(dims))
        z = torch.zeros(N, 2, device=dev())
        gw = torch.empty(2 * N, device=dev())
        args = (to_dev(si), to_dev(sl), 2, z, 1e-3, z, z, gw)
        with pytest.raises(rw.RWError) as e:
            rw.rw_grad_exact(gg, *args[:4], 0.0, *args[5:])
        assert e.value.status == rw.RW_ERR_UNSUPPORTED
        with pytest.raises(rw.RWError) as e:
            rw.rw_grad_exact(gg, *args, rel_tol=-1.0)
        assert e.value.status == rw.RW_ERR_INVALID_ARG
    finally:
        rw.rw_graph_free(gg)


# ----------------------------------------------------------------------------- fast path


def _fast_setup(m_basis=50, m=30):
    from tests.gpu_common import c1_case
    case = c1_case(m=m_basis)
    g = case["g"]
    P = f32(priors.gaussian_priors(case["J"], case["si"], case["sl"], 2))
    gg = rw.rw_build_graph(to_dev(case["J"], torch.float32), case["dims"], case["beta"])
    b = rw.rw_basis_create(gg, to_dev(case["Q"], torch.float32), case["lam"])
    # values = Eq. (z_ray) of the stored float32 columns under the current weights
    rw.rw_update_weights(gg, b, rw.RW_UPDATE_BETA, beta=case["beta"])
    return case, g, P, gg, b, m


def test_fast_gradient_matches_oracle():
    case, g, P, gg, b, m = _fast_setup()
    si, sl, gamma = case["si"], case["sl"], 1e-3
    Q = case["Q"][:, :m]
    try:
        from oracle import update
        lam = update.rayleigh_quotients(Q, g.Lhat)
        U_ref, _ = adjoint.fast_forward(g, Q, lam, si, sl, 2, P, gamma, 3, 0.8)
        _, G = adjoint.mask_loss(f32(U_ref), case["truth"].astype(np.float64), si, label=1)
        G = f32(G)
        gw_ref, gb_ref, _ = adjoint.fast_grad(g, Q, si, sl, 2, P, gamma, G, refine_steps=3,
                                              omega=0.8)
        full_ref = np.zeros(2 * g.N)
        full_ref[g.ids] = gw_ref
        N = g.N
        gw = torch.full((2 * N,), float("nan"), device=dev())
        U = torch.empty(N, 2, device=dev())
        gb = rw.rw_grad_fast(gg, b, to_dev(si), to_dev(sl), 2, to_dev(P, torch.float32), gamma,
                             m, to_dev(G, torch.float32), gw, refine_steps=3, omega=0.8, U_out=U)
        assert np.abs(U.cpu().numpy() - U_ref).max() <= 1e-4
        gw = gw.cpu().numpy().astype(np.float64)
        scale = np.abs(full_ref).max()
        assert np.abs(gw - full_ref).max() <= GRAD_RTOL * scale, (np.abs(gw - full_ref).max(), scale)
        assert abs(gb - gb_ref) <= GRAD_RTOL * abs(gb_ref), (gb, gb_ref)
    finally:
        rw.rw_basis_free(b)
        rw.rw_graph_free(gg)


def test_fast_gradient_rejects_unnormalized_graph():
    case, g, P, gg, b, m = _fast_setup(m_basis=20, m=10)
    try:
        gu = rw.rw_build_graph(to_dev(case["J"], torch.float32), case["dims"], 90.0,
                               rw.RW_WEIGHT_SQ, False)
        bu = rw.rw_basis_create(gu, to_dev(case["Q"], torch.float32), case["lam"])
        z = torch.zeros(g.N, 2, device=dev())
        gw = torch.empty(2 * g.N, device=dev())
        with pytest.raises(rw.RWError) as e:
            rw.rw_grad_fast(gu, bu, to_dev(case["si"]), to_dev(case["sl"]), 2, z, 1e-3, 10, z, gw)
        assert e.value.status == rw.RW_ERR_UNSUPPORTED
        rw.rw_basis_free(bu)
        rw.rw_graph_free(gu)
    finally:
        rw.rw_basis_free(b)
        rw.rw_graph_free(gg)


# ----------------------------------------------------------------------------- autograd


def _mask_loss_t(U, truth_t, free_t):
    return ((U[free_t, 1] - truth_t[free_t]) ** 2).sum()


def test_autograd_exact_beta_and_weights_match_oracle():
    from paper_1607_04174_gb300 import autograd as rwa
    J, dims, truth = synth.closed_curve_image(48, seed=synth.BASE_SEED + 5)
    J = f32(J)
    si, sl = synth.sample_seeds(truth, dims, 15, 2, seed=synth.BASE_SEED + 5)
    beta, gamma = 90.0, 1e-3
    g = graph.build_graph(J, dims, beta)
    P = f32(priors.gaussian_priors(J, si, sl, 2))
    U = exact.exact_rw(g, si, sl, 2, P, gamma, True)
    _, G = adjoint.mask_loss(U, truth.astype(np.float64), si, label=1)
    gw_ref, gb_ref = adjoint.exact_grad(g, si, sl, 2, P, gamma, G, True, U=U)
    full_ref = np.zeros(2 * g.N)
    full_ref[g.ids] = gw_ref
    gg = rw.rw_build_graph(to_dev(J, torch.float32), dims, beta)
    try:
        free = np.ones(g.N, bool)
        free[si] = False
        truth_t, free_t = to_dev(truth.astype(np.float32)), to_dev(free)
        Pd, sid, sld = to_dev(P, torch.float32), to_dev(si), to_dev(sl)
        bt = torch.tensor(beta, dtype=torch.float64, device=dev(), requires_grad=True)
        Ut = rwa.exact_probabilities(gg, sid, sld, 2, Pd, beta=bt, gamma=gamma, tol=1e-6)
        assert np.abs(Ut.detach().cpu().numpy() - U).max() <= 1e-4
        _mask_loss_t(Ut, truth_t, free_t).backward()
        assert abs(bt.grad.item() - gb_ref) <= GRAD_RTOL * abs(gb_ref)
        wt = to_dev(g.weights_by_id(), torch.float32).requires_grad_(True)
        Ut = rwa.exact_probabilities(gg, sid, sld, 2, Pd, weights=wt, gamma=gamma, tol=1e-6)
        _mask_loss_t(Ut, truth_t, free_t).backward()
        gwt = wt.grad.cpu().numpy().astype(np.float64)
        assert np.abs(gwt - full_ref).max() <= GRAD_RTOL * np.abs(full_ref).max()
    finally:
        rw.rw_graph_free(gg)


def test_autograd_fast_beta_matches_oracle_and_differences():
    from paper_1607_04174_gb300 import autograd as rwa
    from oracle import update
    case, g, P, gg, b, m = _fast_setup()
    si, sl, gamma, beta = case["si"], case["sl"], 1e-3, case["beta"]
    try:
        Q = case["Q"][:, :m]
        lam = update.rayleigh_quotients(Q, g.Lhat)
        U_ref, _ = adjoint.fast_forward(g, Q, lam, si, sl, 2, P, gamma, 3, 0.8)
        _, G = adjoint.mask_loss(U_ref, case["truth"].astype(np.float64), si, label=1)
        _, gb_ref, _ = adjoint.fast_grad(g, Q, si, sl, 2, P, gamma, G, refine_steps=3, omega=0.8)
        free = np.ones(g.N, bool)
        free[si] = False
        truth_t, free_t = to_dev(case["truth"].astype(np.float32)), to_dev(free)
        Pd, sid, sld = to_dev(P, torch.float32), to_dev(si), to_dev(sl)

        def loss_at(bv, grad=False):
            bt = torch.tensor(bv, dtype=torch.float64, device=dev(), requires_grad=grad)
            Ut = rwa.fast_probabilities(gg, b, sid, sld, 2, Pd, m, beta=bt, gamma=gamma)
            L_ = _mask_loss_t(Ut.double(), truth_t.double(), free_t)
            if grad:
                L_.backward()
                return L_.item(), bt.grad.item(), Ut
            return L_.item()
        _, gbt, Ut = loss_at(beta, grad=True)
        assert np.abs(Ut.detach().cpu().numpy() - U_ref).max() <= 1e-3
        assert abs(gbt - gb_ref) <= 5e-3 * abs(gb_ref), (gbt, gb_ref)
        h = 0.5
        fd = (loss_at(beta + h) - loss_at(beta - h)) / (2 * h)
        assert abs(gbt - fd) <= 2e-2 * abs(gb_ref), (gbt, fd)
    finally:
        rw.rw_basis_free(b)
        rw.rw_graph_free(gg)
