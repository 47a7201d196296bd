"""GPU parity: graph (Eq. W), the Laplacian stencil, the online fast-RW solve (Eqs. Fs,
U_lin_comb, normalized form), adaptive m (Eq. alpha_1), refinement, the PCG basic RW
(Eq. rw_eq) and argument errors — all through the C ABI, against the FP64 oracle."""
import numpy as np
import pytest

import synth
from oracle import adaptive, exact, fastrw, graph, pipeline, priors, refine, update
from tests.gpu_common import TOL_PROB, c1_case, dev, f32, gap_mask, to_dev

pytestmark = pytest.mark.gpu

rw = pytest.importorskip("paper_1607_04174_gb300")
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1607_04174_gb300 import build
    build.build()


# ----------------------------------------------------------------------------- graph / stencil

GRAPH_CASES = [((64, 64), "sq", True), ((37, 29), "abs", True), ((13, 11, 9), "sq", True),
               ((16, 12), "sq", False), ((1, 40), "sq", True), ((5, 1, 7), "abs", False)]


@pytest.mark.parametrize("dims,form,normalized", GRAPH_CASES)
def test_weights_and_degrees(dims, form, normalized):
    J = f32(synth.smooth_random_image(dims, seed=11, smooth=1.0, sigma=0.05))
    beta = 40.0
    g = rw.rw_build_graph(to_dev(J, torch.float32), dims, beta,
                          rw.RW_WEIGHT_SQ if form == "sq" else rw.RW_WEIGHT_ABS, normalized)
    try:
        N = int(np.prod(dims))
        w = torch.empty(len(dims) * N, device=dev())
        d = torch.empty(N, device=dev())
        rw.rw_graph_weights(g, w, d)
        go = graph.build_graph(J, dims, beta, form)
        np.testing.assert_allclose(w.cpu().numpy(), go.weights_by_id(), rtol=2e-5, atol=1e-30)
        np.testing.assert_allclose(d.cpu().numpy(), go.d, rtol=2e-5)
    finally:
        rw.rw_graph_free(g)


@pytest.mark.parametrize("dims,form,normalized", GRAPH_CASES)
@pytest.mark.parametrize("k", [1, 6, 64, 200, 601])
def test_stencil_matches_sparse_operator(dims, form, normalized, k):
    J = f32(synth.smooth_random_image(dims, seed=12, smooth=1.0, sigma=0.05))
    g = rw.rw_build_graph(to_dev(J, torch.float32), dims, 30.0,
                          rw.RW_WEIGHT_SQ if form == "sq" else rw.RW_WEIGHT_ABS, normalized)
    try:
        N = int(np.prod(dims))
        ld = (k + 3) // 4 * 4 + 4  # a pitch wider than the row
        rng = np.random.default_rng(k)
        X = np.zeros((N, ld), np.float32)
        X[:, :k] = rng.standard_normal((N, k))
        Xd = to_dev(X)
        Yd = torch.full((N, ld), 7.0, device=dev())
        rw.rw_apply_laplacian(g, Xd, Yd, k)
        go = graph.build_graph(J, dims, 30.0, form)
        ref = go.operator(normalized) @ X[:, :k].astype(np.float64)
        Y = Yd.cpu().numpy()
        scale = np.abs(ref).max() + 1.0
        assert np.abs(Y[:, :k] - ref).max() <= 2e-6 * scale * (1 + (0 if normalized else 3))
        assert np.all(Y[:, (k + 3) // 4 * 4:] == 7.0)  # pitch padding untouched
    finally:
        rw.rw_graph_free(g)


def test_isolated_node_is_rejected():
    J = np.zeros(16, np.float32)
    J[5] = 1.0  # beta huge: voxel 5's weights underflow to 0 -> degree 0
    with pytest.raises(rw.RWError) as e:
        rw.rw_build_graph(to_dev(J), (4, 4), 1e6)
    assert e.value.status == rw.RW_ERR_ISOLATED_NODE


# ----------------------------------------------------------------------------- online solve


def _gpu_solve(case, m, steps, fmt=rw.RW_BASIS_F16, gamma=1e-3, n_labels=2, eps=0.1, m_step=10,
               prior_mode=0, P=None, refine_mode=rw.RW_REFINE_JACOBI):
    g = rw.rw_build_graph(to_dev(case["J"], torch.float32), case["dims"], case["beta"])
    b = rw.rw_basis_create(g, to_dev(case["Q"], torch.float32), case["lam"])
    try:
        N = case["g"].N
        prob = torch.empty(N, n_labels, device=dev())
        lab = torch.empty(N, dtype=torch.uint8, device=dev())
        s, info = rw.rw_solve(g, b, to_dev(case["si"]), to_dev(case["sl"]), n_labels, prob, lab,
                              priors=None if P is None else to_dev(P, torch.float32),
                              gamma=gamma, m=m, m_step=m_step, eps=eps, refine_steps=steps,
                              basis_format=fmt, prior_mode=prior_mode, refine_mode=refine_mode)
        return prob.cpu().numpy().astype(np.float64), lab.cpu().numpy(), info, s
    finally:
        rw.rw_basis_free(b)
        rw.rw_graph_free(g)


@pytest.fixture(scope="module")
def c1():
    return c1_case()


@pytest.mark.parametrize("fmt,tol", [(rw.RW_BASIS_F16, TOL_PROB), (rw.RW_BASIS_F32, 1e-4)])
@pytest.mark.parametrize("steps", [0, 3])
def test_fixed_m_solve_matches_oracle(c1, fmt, tol, steps):
    U, lab, info, s = _gpu_solve(c1, 50, steps, fmt)
    ref = pipeline.online_solve(c1["g"], c1["Q"], c1["lam"], c1["si"], c1["sl"], 2, gamma=1e-3,
                                m=50, refine_steps=steps)
    err = np.abs(U - ref["U"]).max()
    assert err <= tol, err
    mask = gap_mask(ref["U"])
    assert np.array_equal(lab[mask], ref["labels"][mask])
    assert info["m_used"] == 50
    np.testing.assert_allclose(info["mu"], [c1["J"][c1["si"][c1["sl"] == k]].mean() for k in (0, 1)],
                               rtol=1e-6)


def test_bf16_basis_error_is_reported_not_hidden(c1):
    """BF16 storage of Q: the error is measured and bounded loosely (it does not meet 1e-3 in
    general; the 16-bit default is scaled FP16)."""
    U, _, _, _ = _gpu_solve(c1, 50, 3, rw.RW_BASIS_BF16)
    ref = pipeline.online_solve(c1["g"], c1["Q"], c1["lam"], c1["si"], c1["sl"], 2, gamma=1e-3,
                                m=50, refine_steps=3)
    assert np.abs(U - ref["U"]).max() <= 2e-2


@pytest.mark.parametrize("m", [1, 7, 24])
def test_small_and_ragged_m(c1, m):
    U, _, info, _ = _gpu_solve(c1, m, 0)
    ref = fastrw.fast_rw(c1["g"], c1["Q"][:, :m], c1["lam"][:m], c1["si"], c1["sl"], 2,
                         priors.gaussian_priors(c1["J"], c1["si"], c1["sl"], 2), 1e-3)
    assert np.abs(U - ref).max() <= TOL_PROB
    assert info["m_used"] == m


def test_adaptive_m_matches_oracle(c1):
    U, _, info, s = _gpu_solve(c1, 0, 3, eps=0.02, m_step=5)
    m_o, f_o, capped, table = adaptive.choose_m_from_seeds(c1["g"], c1["Q"], c1["si"], c1["sl"],
                                                           2, 50, 5, 0.02)
    fmax = len(c1["si"]) * 0.02 ** 2
    if info["m_used"] != m_o:  # allowed only at the threshold (relative 1e-3)
        f_gpu_at = table.get(info["m_used"])
        assert f_gpu_at is not None
        assert abs(f_gpu_at.max() - fmax) / fmax < 1e-3 or abs(f_o.max() - fmax) / fmax < 1e-3
    else:
        np.testing.assert_allclose(info["f"], f_o, rtol=2e-3, atol=1e-4 * fmax)
    assert info["capped"] == int(capped)
    ref = pipeline.online_solve(c1["g"], c1["Q"], c1["lam"], c1["si"], c1["sl"], 2, gamma=1e-3,
                                m=info["m_used"], refine_steps=3)
    assert np.abs(U - ref["U"]).max() <= TOL_PROB


def test_adaptive_m_active_constraint():
    """Few seeds and more columns than seeds: the minimum-norm fit leaves the ball
    ||alpha|| <= rho, exercising the secular-equation branch."""
    case = c1_case(size=32, per=3, m=30)
    U, _, info, _ = _gpu_solve(case, 0, 0, eps=1e-4, m_step=5)
    t, rho = adaptive.seed_targets(case["g"], case["si"], case["sl"], 2)
    f_o = adaptive.f_values(case["Q"], case["si"], t, rho, info["m_used"])
    np.testing.assert_allclose(info["f"], f_o, rtol=5e-3, atol=1e-5)


@pytest.mark.parametrize("n_labels", [1, 3, 5, 9])
def test_label_counts_and_caller_priors(n_labels):
    dims = (40, 36)
    J = f32(synth.smooth_random_image(dims, seed=5, smooth=3.0, sigma=0.02))
    truth = np.minimum((J * n_labels).astype(np.int32), n_labels - 1)
    si, sl = synth.sample_seeds(truth, dims, 4, 1, seed=3, n_labels=n_labels)
    go = graph.build_graph(J, dims, 60.0)
    from oracle import eig
    lam, Q = eig.smallest_eigpairs(go.Lhat, 40)
    case = dict(J=J, dims=dims, si=si, sl=sl, g=go, lam=lam, Q=f32(Q), beta=60.0)
    rng = np.random.default_rng(0)
    P = rng.uniform(0.1, 1.0, size=(go.N, n_labels))
    P = f32(P / P.sum(axis=1, keepdims=True))
    U, lab, _, _ = _gpu_solve(case, 40, 2, n_labels=n_labels, prior_mode=1, P=P, gamma=0.05)
    ref = pipeline.online_solve(go, case["Q"], lam, si, sl, n_labels, gamma=0.05, m=40,
                                refine_steps=2, P=P)
    assert np.abs(U - ref["U"]).max() <= TOL_PROB
    np.testing.assert_allclose(U.sum(axis=1), 1.0, atol=2e-3)
    mask = gap_mask(ref["U"])
    assert np.array_equal(lab[mask], ref["labels"][mask])


def test_full_size_512_dct_basis_parity():
    """Config-2 sizes (512^2, 4 labels, 200 seeds per label, m = 200): the online solve in the
    launch configuration the benchmark times, against the oracle on every voxel.  The basis is
    a generic orthonormal one (DCT) with its Rayleigh quotients as values."""
    J, dims, truth = synth.voronoi_image(512, 512, seed=synth.BASE_SEED + 1)
    J = f32(J)
    si, sl = synth.sample_seeds(truth, dims, 200, 3, seed=synth.BASE_SEED + 1)
    go = graph.build_graph(J, dims, 90.0)
    Q = f32(synth.dct_basis(dims, 200))
    lam = update.rayleigh_quotients(Q, go.Lhat)
    case = dict(J=J, dims=dims, si=si, sl=sl, g=go, lam=lam, Q=Q, beta=90.0)
    for m, steps in ((200, 3), (0, 3)):
        U, lab, info, _ = _gpu_solve(case, m, steps, n_labels=4)
        ref = pipeline.online_solve(go, Q, lam, si, sl, 4, gamma=1e-3, m=info["m_used"],
                                    refine_steps=steps)
        err = np.abs(U - ref["U"]).max()
        assert err <= TOL_PROB, (m, err)
        mask = gap_mask(ref["U"])
        assert np.array_equal(lab[mask], ref["labels"][mask])


def test_host_entry_point_matches_device(c1):
    U_dev, lab_dev, _, _ = _gpu_solve(c1, 50, 3)
    g = rw.rw_build_graph(to_dev(c1["J"], torch.float32), c1["dims"], c1["beta"])
    b = rw.rw_basis_create(g, to_dev(c1["Q"], torch.float32), c1["lam"])
    try:
        prob = np.zeros((c1["g"].N, 2), np.float32)
        lab = np.zeros(c1["g"].N, np.uint8)
        rw.rw_solve_host(g, b, c1["si"].astype(np.int32), c1["sl"].astype(np.int32), 2, prob,
                         lab, m=50, refine_steps=3)
        np.testing.assert_array_equal(prob.astype(np.float64), U_dev)
        np.testing.assert_array_equal(lab, lab_dev)
        # the asynchronous entry point, pinned buffers, several calls in flight on one stream
        si = torch.from_numpy(c1["si"].astype(np.int32)).pin_memory()
        sl = torch.from_numpy(c1["sl"].astype(np.int32)).pin_memory()
        outs = [(torch.zeros(c1["g"].N, 2).pin_memory(), torch.zeros(c1["g"].N, dtype=torch.uint8).pin_memory())
                for _ in range(3)]
        for hp, hl in outs:
            rw.rw_solve_host_async(g, b, si.numpy(), sl.numpy(), 2, hp.numpy(), hl.numpy(), m=50,
                                   refine_steps=3)
        torch.cuda.synchronize()
        for hp, hl in outs:
            np.testing.assert_array_equal(hp.numpy().astype(np.float64), U_dev)
            np.testing.assert_array_equal(hl.numpy(), lab_dev)
    finally:
        rw.rw_basis_free(b)
        rw.rw_graph_free(g)


def test_bad_arguments_raise(c1):
    g = rw.rw_build_graph(to_dev(c1["J"], torch.float32), c1["dims"], c1["beta"])
    b = rw.rw_basis_create(g, to_dev(c1["Q"], torch.float32), c1["lam"])
    N = c1["g"].N
    prob = torch.empty(N, 2, device=dev())
    try:
        bad = c1["si"].copy()
        bad[3] = N + 5
        with pytest.raises(rw.RWError) as e:
            rw.rw_solve(g, b, to_dev(bad), to_dev(c1["sl"]), 2, prob, m=20)
        assert e.value.status == rw.RW_ERR_INVALID_ARG
        dup = c1["si"].copy()
        dup[1] = dup[0]
        with pytest.raises(rw.RWError):
            rw.rw_solve(g, b, to_dev(dup), to_dev(c1["sl"]), 2, prob, m=20)
        badl = c1["sl"].copy()
        badl[0] = 7
        with pytest.raises(rw.RWError):
            rw.rw_solve(g, b, to_dev(c1["si"]), to_dev(badl), 2, prob, m=20)
        with pytest.raises(rw.RWError) as e:
            rw.rw_solve(g, b, to_dev(c1["si"]), to_dev(c1["sl"]), 2, prob, m=20, gamma=-1.0)
        assert e.value.status == rw.RW_ERR_INVALID_ARG
        with pytest.raises(rw.RWError):
            rw.rw_solve(g, b, to_dev(c1["si"]), to_dev(c1["sl"]), 2, prob, m=51)
        # the handle still works after the errors
        s, info = rw.rw_solve(g, b, to_dev(c1["si"]), to_dev(c1["sl"]), 2, prob, m=20)
        assert s == rw.RW_OK and info["device_status"] == 0
    finally:
        rw.rw_basis_free(b)
        rw.rw_graph_free(g)


# ----------------------------------------------------------------------------- PCG basic RW


def test_pcg_converges_to_exact(c1):
    g = rw.rw_build_graph(to_dev(c1["J"], torch.float32), c1["dims"], c1["beta"])
    try:
        N = c1["g"].N
        prob = torch.empty(N, 2, device=dev())
        lab = torch.empty(N, dtype=torch.uint8, device=dev())
        it = rw.rw_solve_pcg(g, to_dev(c1["si"]), to_dev(c1["sl"]), 2, prob, lab, gamma=1e-3,
                             iters=20000, tol=1e-7)
        assert 0 < it < 20000
        P = priors.gaussian_priors(c1["J"], c1["si"], c1["sl"], 2)
        Ue = exact.exact_rw(c1["g"], c1["si"], c1["sl"], 2, P, 1e-3)
        assert np.abs(prob.cpu().numpy() - Ue).max() <= 1e-4
        mask = gap_mask(Ue)
        assert np.array_equal(lab.cpu().numpy()[mask], np.argmax(Ue, 1)[mask])
    finally:
        rw.rw_graph_free(g)


def test_pcg_fixed_iterations_match_oracle_recurrence(c1):
    g = rw.rw_build_graph(to_dev(c1["J"], torch.float32), c1["dims"], c1["beta"])
    try:
        N = c1["g"].N
        prob = torch.empty(N, 2, device=dev())
        rw.rw_solve_pcg(g, to_dev(c1["si"]), to_dev(c1["sl"]), 2, prob, gamma=1e-3, iters=6)
        P = priors.gaussian_priors(c1["J"], c1["si"], c1["sl"], 2)
        A, bb, n, sc = refine.hat_system(c1["g"], c1["si"], c1["sl"], 2, P, 1e-3)
        x, _ = refine.pcg_steps(A, bb, np.zeros_like(bb), 6)
        U = np.zeros((N, 2))
        U[c1["si"]] = exact.onehot(c1["sl"], 2)
        U[n] = x / sc[n, None]
        assert np.abs(prob.cpu().numpy() - U).max() <= 1e-4
    finally:
        rw.rw_graph_free(g)


def test_consecutive_solves_on_one_graph(c1):
    """The seed labels of one call must not leak into the next: a sequence of solves on the same
    handles (different seed sets, refinement by Jacobi, by PCG and none, a PCG solve and a
    failing call with a duplicated seed in between) matches fresh solves of each seed set."""
    J, dims, truth = c1["J"], c1["dims"], c1["truth"]
    sets = [synth.sample_seeds(truth, dims, 20, 2, seed=synth.BASE_SEED + 300 + k) for k in range(4)]
    g = rw.rw_build_graph(to_dev(J, torch.float32), dims, c1["beta"])
    b = rw.rw_basis_create(g, to_dev(c1["Q"], torch.float32), c1["lam"])
    N = c1["g"].N
    prob = torch.empty(N, 2, device=dev())
    lab = torch.empty(N, dtype=torch.uint8, device=dev())
    plan = [(0, 3, rw.RW_REFINE_JACOBI), (1, 0, rw.RW_REFINE_JACOBI), (2, 4, rw.RW_REFINE_PCG),
            (3, 3, rw.RW_REFINE_JACOBI), (0, 3, rw.RW_REFINE_JACOBI)]
    try:
        for step, (k, steps, mode) in enumerate(plan):
            si, sl = sets[k]
            if step == 2:   # a basic-RW solve and a failing call in between
                rw.rw_solve_pcg(g, to_dev(sets[1][0]), to_dev(sets[1][1]), 2, prob, iters=5)
                dup_i = np.concatenate([sets[3][0], sets[3][0][:1]]).astype(np.int32)
                dup_l = np.concatenate([sets[3][1], sets[3][1][:1]]).astype(np.int32)
                with pytest.raises(rw.RWError):
                    rw.rw_solve(g, b, to_dev(dup_i), to_dev(dup_l), 2, prob, lab, m=30,
                                refine_steps=3)
            rw.rw_solve(g, b, to_dev(si), to_dev(sl), 2, prob, lab, m=30, refine_steps=steps,
                        refine_mode=mode)
            U = prob.cpu().numpy().astype(np.float64)
            ref = pipeline.online_solve(c1["g"], c1["Q"], c1["lam"], si, sl, 2, gamma=1e-3, m=30,
                                        refine_steps=steps,
                                        refine_method="pcg" if mode == rw.RW_REFINE_PCG else "jacobi")
            tol = 5e-3 if mode == rw.RW_REFINE_PCG else TOL_PROB  # PCG amplifies start differences
            assert np.abs(U - ref["U"]).max() <= tol, (step, np.abs(U - ref["U"]).max())
            onehot = np.eye(2)[sl]
            np.testing.assert_array_equal(U[si], onehot)
    finally:
        rw.rw_basis_free(b)
        rw.rw_graph_free(g)


def test_zero_pivot_takes_the_pivoting_path(c1):
    """Basis values chosen so that the Woodbury matrix diag(lambda + gamma) - Q_s^T X has a zero
    first diagonal entry: the unpivoted LU must detect it and the partial-pivoting path must
    still match the oracle's S x S solve of Eq. (Fs)."""
    m, gamma = 12, 1e-3
    Q = c1["Q"][:, :m]
    lam = c1["lam"][:m].copy()
    P = f32(priors.gaussian_priors(c1["J"], c1["si"], c1["sl"], 2))
    _, parts = fastrw.fast_rw(c1["g"], Q, lam, c1["si"], c1["sl"], 2, P, gamma, return_parts=True)
    K = Q[c1["si"]].T @ parts["X"]
    lam[0] = float(np.float32(K[0, 0])) - gamma   # M_00 = lambda_0 + gamma - K_00 = 0
    ref = fastrw.fast_rw(c1["g"], Q, lam, c1["si"], c1["sl"], 2, P, gamma)
    g = rw.rw_build_graph(to_dev(c1["J"], torch.float32), c1["dims"], c1["beta"])
    b = rw.rw_basis_create(g, to_dev(np.ascontiguousarray(Q), torch.float32), lam)
    try:
        prob = torch.empty(c1["g"].N, 2, device=dev())
        rw.rw_solve(g, b, to_dev(c1["si"]), to_dev(c1["sl"]), 2, prob, priors=to_dev(P, torch.float32),
                    prior_mode=1, gamma=gamma, m=m, refine_steps=0, basis_format=rw.RW_BASIS_F32)
        err = np.abs(prob.cpu().numpy() - ref).max()
        assert err <= 1e-3, err
    finally:
        rw.rw_basis_free(b)
        rw.rw_graph_free(g)
