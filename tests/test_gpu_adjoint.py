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
