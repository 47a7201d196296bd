"""GPU parity of the basic random walker solved by Jacobi-preconditioned CG (Eq. rw_eq, the
normalized form of Sec. II-C): a fixed number of iterations of the cooperative two-pass kernel
against the oracle's FP64 recurrence on the same system, over 2-D and 3-D grids with ragged
row tiles (rows wider than one thread block, odd sizes), both Laplacian forms and label counts
padded to 4, 8 and 16 columns; and convergence to the oracle's sparse direct solve."""
import numpy as np
import pytest

import synth
from oracle import exact, graph, priors, refine
from tests.gpu_common import dev, f32, to_dev

pytestmark = pytest.mark.gpu

rw = pytest.importorskip("paper_1607_04174_gb300")
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1607_04174_gb300 import build
    build.build()


def random_seeds(N, S, L, seed):
    """S distinct voxels, labels cycling through 0..L-1 (every label seeded)."""
    rng = np.random.default_rng(seed)
    si = rng.choice(N, size=S, replace=False).astype(np.int32)
    sl = (np.arange(S) % L).astype(np.int32)
    return si, sl


CASES = [((37, 29), True, 2), ((700, 3), True, 3), ((13, 11, 9), True, 2),
         ((16, 12), False, 2), ((45, 40), True, 6), ((21, 17, 5), True, 12),
         ((1030, 2), True, 4)]


@pytest.mark.parametrize("dims,normalized,L", CASES)
@pytest.mark.parametrize("iters", [1, 7])
def test_pcg_iterations_match_oracle_recurrence(dims, normalized, L, iters):
    N = int(np.prod(dims))
    J = f32(synth.smooth_random_image(dims, seed=21, smooth=1.5, sigma=0.05))
    si, sl = random_seeds(N, max(2 * L, N // 40), L, seed=N + L)
    gamma = 1e-2
    g = rw.rw_build_graph(to_dev(J, torch.float32), dims, 40.0, rw.RW_WEIGHT_SQ, normalized)
    try:
        prob = torch.empty(N, L, device=dev())
        lab = torch.empty(N, dtype=torch.uint8, device=dev())
        rw.rw_solve_pcg(g, to_dev(si), to_dev(sl), L, prob, lab, gamma=gamma, iters=iters)
        go = graph.build_graph(J, dims, 40.0)
        P = priors.gaussian_priors(J, si, sl, L)
        A, b, n, sc = refine.hat_system(go, si, sl, L, P, gamma, normalized)
        x, _ = refine.pcg_steps(A, b, np.zeros_like(b), iters)
        U = np.zeros((N, L))
        U[si] = exact.onehot(sl, L)
        U[n] = x / sc[n, None]
        got = prob.cpu().numpy()
        err = np.abs(got - U).max()
        assert err <= 2e-4, err
        np.testing.assert_array_equal(got[si], exact.onehot(sl, L))
        # the label map is the argmax of the returned probabilities (ties to the lowest label)
        np.testing.assert_array_equal(lab.cpu().numpy(), np.argmax(got, axis=1))
    finally:
        rw.rw_graph_free(g)


@pytest.mark.parametrize("dims", [(48, 40), (12, 10, 8)])
def test_pcg_converges_to_sparse_direct_solve(dims):
    N = int(np.prod(dims))
    J = f32(synth.smooth_random_image(dims, seed=5, smooth=2.0, sigma=0.05))
    si, sl = random_seeds(N, N // 30, 3, seed=7)
    g = rw.rw_build_graph(to_dev(J, torch.float32), dims, 60.0)
    try:
        prob = torch.empty(N, 3, device=dev())
        it = rw.rw_solve_pcg(g, to_dev(si), to_dev(sl), 3, prob, gamma=1e-3, iters=20000,
                             tol=1e-7)
        assert 0 < it < 20000
        go = graph.build_graph(J, dims, 60.0)
        P = priors.gaussian_priors(J, si, sl, 3)
        Ue = exact.exact_rw(go, si, sl, 3, P, 1e-3)
        assert np.abs(prob.cpu().numpy() - Ue).max() <= 1e-4
    finally:
        rw.rw_graph_free(g)


def test_pcg_repeatable_bit_for_bit():
    """The dot products are summed in a fixed order (no atomics): two runs agree exactly."""
    dims = (96, 80)
    N = int(np.prod(dims))
    J = f32(synth.smooth_random_image(dims, seed=9, smooth=1.5, sigma=0.05))
    si, sl = random_seeds(N, 200, 2, seed=3)
    g = rw.rw_build_graph(to_dev(J, torch.float32), dims, 90.0)
    try:
        outs = []
        for _ in range(2):
            prob = torch.empty(N, 2, device=dev())
            rw.rw_solve_pcg(g, to_dev(si), to_dev(sl), 2, prob, gamma=1e-3, iters=40)
            outs.append(prob.cpu().numpy())
        np.testing.assert_array_equal(outs[0], outs[1])
    finally:
        rw.rw_graph_free(g)
