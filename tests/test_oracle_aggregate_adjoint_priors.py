"""Pins for the oracle's aggregation (Sec. III-C), gradients and priors."""
import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import adjoint, aggregate, eig, exact, fastrw, graph, priors, refine, update


def _graph(dims=(8, 8), seed=0, beta=30.0):
    J = synth.smooth_random_image(dims, seed=seed, smooth=1.5, sigma=0.05)
    return graph.build_graph(J, dims, beta)


def test_hard_blocks_give_hand_built_coarse_laplacian():
    g = _graph()
    eta = aggregate.block_eta((8, 8), 2, 2)
    gbar = aggregate.galerkin_graph(g, eta)
    blk = np.asarray(eta.argmax(axis=1)).ravel()
    nb = eta.shape[1]
    Wc = np.zeros((nb, nb))
    for a, b, w in zip(g.a, g.b, g.w):            # sum the weights crossing between blocks
        if blk[a] != blk[b]:
            Wc[blk[a], blk[b]] += w
            Wc[blk[b], blk[a]] += w
    np.testing.assert_allclose(gbar.W.toarray(), Wc, atol=1e-14)
    np.testing.assert_allclose(gbar.L @ np.ones(nb), 0, atol=1e-13)


def test_aggregated_basis_orthonormal_and_laplacian_null():
    g = _graph(seed=1)
    lam, Q = eig.smallest_eigpairs(g.Lhat, 12)
    hard = aggregate.block_eta((8, 8), 2, 2).toarray()
    right = hard[np.minimum(np.arange(64) + 1, 63)]      # block of the right-hand neighbour
    eta = hard + 0.25 * right                             # soft: up to two super-vertices
    eta = sp.csr_matrix(eta / eta.sum(axis=1, keepdims=True))
    assert (eta.getnnz(axis=1) == 2).sum() > 10
    for naive in (False, True):
        gbar, Qbar, lb, kept = aggregate.aggregate_basis(g, Q, eta, naive=naive)
        np.testing.assert_allclose(Qbar.T @ Qbar, np.eye(Qbar.shape[1]), atol=1e-12)
        np.testing.assert_allclose(gbar.L @ np.ones(gbar.N), 0, atol=1e-12)
        assert lb.min() > -1e-12 and lb.max() < 2 + 1e-12
    eb = aggregate.column_normalized(eta)
    np.testing.assert_allclose(np.asarray(eb.sum(axis=0)).ravel(), 1.0, atol=1e-14)


def test_delta_identity_and_consumed_edges():
    g = _graph(dims=(5, 4))
    # eta = I: Delta(x) = 2 |N(x)| (each neighbour differs in two entries by 1)
    dl = aggregate.delta(g, sp.identity(g.N, format="csr"))
    deg = np.zeros(g.N)
    np.add.at(deg, g.a, 1)
    np.add.at(deg, g.b, 1)
    np.testing.assert_allclose(dl, 2 * deg)
    # a voxel whose neighbours all share its hard block has every edge consumed: Delta = 0
    g8 = _graph()
    eta = aggregate.block_eta((8, 8), 4, 4)
    dl = aggregate.delta(g8, eta)
    assert dl[1 + 8 * 1] == 0.0 and dl[3 + 8 * 1] > 0


def _grad_case(normalized=True):
    dims = (9, 8)
    J = synth.smooth_random_image(dims, seed=7, smooth=2.0, sigma=0.03)
    truth = (J > 0.5).astype(np.int32)
    si, sl = synth.sample_seeds(truth, dims, 4, 1, seed=7, n_labels=2)
    g = graph.build_graph(J, dims, 20.0)
    P = priors.gaussian_priors(J, si, sl, 2)
    return g, si, sl, P, truth


@pytest.mark.parametrize("normalized", [True, False])
def test_exact_gradient_matches_central_differences(normalized):
    g, si, sl, P, truth = _grad_case()
    gamma = 0.05

    def loss_of(gg):
        U = exact.exact_rw(gg, si, sl, 2, P, gamma, normalized)
        return adjoint.mask_loss(U, truth, si)[0]
    U = exact.exact_rw(g, si, sl, 2, P, gamma, normalized)
    _, G = adjoint.mask_loss(U, truth, si)
    gw, gb = adjoint.exact_grad(g, si, sl, 2, P, gamma, G, normalized, U)
    pos = np.random.default_rng(0).choice(g.ids.size, 12, replace=False)
    fd = adjoint.fd_grad(loss_of, g, pos, h_beta=1e-4, h_rel=1e-4)
    np.testing.assert_allclose(gb, fd["beta"], rtol=1e-6)
    np.testing.assert_allclose(gw[pos], fd["edges"], rtol=1e-5, atol=1e-9)


def _fast_case(m=14):
    g, si, sl, P, truth = _grad_case()
    lam, Q = np.linalg.eigh(g.Lhat.toarray())
    return g, si, sl, P, truth, Q[:, :m]


def test_fast_forward_equals_pipeline_pieces():
    """The forward kept for the fast-path adjoint is the fast solve (Eqs. Fs, U_lin_comb) plus
    the damped-Jacobi refinement, as composed from the separate oracle pieces."""
    g, si, sl, P, truth, Q = _fast_case()
    lam = update.updated_values(g, Q)
    U1, _ = adjoint.fast_forward(g, Q, lam, si, sl, 2, P, 0.05, refine_steps=3, omega=0.8)
    U0 = fastrw.fast_rw(g, Q, lam, si, sl, 2, P, 0.05)
    U2, _ = refine.refine(g, U0, si, sl, 2, P, 0.05, 3, True, "jacobi", 0.8)
    np.testing.assert_allclose(U1, U2, atol=1e-12)


@pytest.mark.parametrize("steps", [0, 3])
def test_fast_gradient_matches_central_differences(steps):
    """Reverse-mode gradient of the fast path (Q fixed, values by Eq. z_ray under the changed
    weights) against central differences of the pipeline pieces, on every edge and beta."""
    g, si, sl, P, truth, Q = _fast_case()
    gamma = 0.05

    def loss_of(gg):
        lam = update.updated_values(gg, Q)
        U = fastrw.fast_rw(gg, Q, lam, si, sl, 2, P, gamma)
        if steps:
            U, _ = refine.refine(gg, U, si, sl, 2, P, gamma, steps, True, "jacobi", 0.8)
        return adjoint.mask_loss(U, truth, si)[0]
    lam = update.updated_values(g, Q)
    U, _ = adjoint.fast_forward(g, Q, lam, si, sl, 2, P, gamma, steps, 0.8)
    _, G = adjoint.mask_loss(U, truth, si)
    gw, gb, _ = adjoint.fast_grad(g, Q, si, sl, 2, P, gamma, G, refine_steps=steps, omega=0.8)
    fd = adjoint.fd_grad(loss_of, g, np.arange(g.ids.size), h_beta=1e-5, h_rel=1e-5)
    np.testing.assert_allclose(gb, fd["beta"], rtol=2e-6)
    scale = np.abs(fd["edges"]).max()
    assert np.abs(gw - fd["edges"]).max() <= 2e-6 * scale


def test_gaussian_priors_match_normal_pdf():
    from scipy.stats import norm
    rng = np.random.default_rng(3)
    J = rng.uniform(size=200)
    si = np.arange(30)
    sl = (J[:30] > 0.5).astype(np.int32)
    P = priors.gaussian_priors(J, si, sl, 2)
    mu = [J[si[sl == k]].mean() for k in range(2)]
    sd = [J[si[sl == k]].std() for k in range(2)]
    pdf = np.stack([norm.pdf(J, mu[k], sd[k]) for k in range(2)], axis=1)
    np.testing.assert_allclose(P, pdf / pdf.sum(axis=1, keepdims=True), rtol=1e-10)
    np.testing.assert_allclose(P.sum(axis=1), 1.0, atol=1e-15)


def test_gaussian_priors_degenerate_cases():
    """Special cases of the per-label Gaussian fit (Sec. IV-A): a label whose seeds share one
    intensity gets the floor sigma = 1e-3 (the fit's sample deviation is 0); a voxel far from
    every mean, where each density underflows in double precision, still gets a normalised
    prior, one-hot on the label with the largest log-density; a label without seeds is an
    error."""
    from scipy.stats import norm
    J = np.array([0.2, 0.2, 0.2, 0.7, 0.8, 0.9, 0.5, 50.0])
    si = np.arange(6)
    sl = np.array([0, 0, 0, 1, 1, 1], np.int32)
    mu, sig = priors.gaussian_fit(J, si, sl, 2)
    assert mu[0] == pytest.approx(0.2) and sig[0] == priors.SIGMA_FLOOR
    assert mu[1] == pytest.approx(0.8) and sig[1] == pytest.approx(np.sqrt(2 / 300))
    P = priors.gaussian_priors(J, si, sl, 2)
    assert np.all(np.isfinite(P)) and np.allclose(P.sum(axis=1), 1.0, atol=1e-15)
    # ordinary voxels: the normal densities with the floored deviation, normalised
    pdf = np.stack([norm.pdf(J[:7], mu[k], sig[k]) for k in range(2)], axis=1)
    np.testing.assert_allclose(P[:7], pdf / pdf.sum(axis=1, keepdims=True), rtol=1e-9, atol=1e-300)
    # J = 50: both densities are 0 in double precision; the log-densities decide
    assert norm.pdf(50.0, mu[0], sig[0]) == 0.0 and norm.pdf(50.0, mu[1], sig[1]) == 0.0
    logd = norm.logpdf(50.0, mu, sig)
    assert np.argmax(P[7]) == np.argmax(logd) == 1 and P[7, 1] == 1.0
    with pytest.raises(ValueError):
        priors.gaussian_fit(J, si, np.zeros(6, np.int32), 2)
