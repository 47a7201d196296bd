"""GPU parity on the full 512 x 512 workload (4-connected Voronoi image, 4 labels, 200 seeds per
label, beta = 90, gamma = 1e-3) with the basis the benchmark uses: 200 eigenvectors from the
library's LOBPCG at a residual tolerance of 4e-6 (the FP32 columns stall near 1e-6).

* The basis against the oracle's shift-invert eigensolver (Eq. L_eigs): eigenvalues within
  1e-6 max(|lambda|, 1e-3), every GPU column inside the span of the oracle's first 240
  eigenvectors, FP64 residuals and orthonormality.
* The online solve (adaptive m, 3 damped-Jacobi steps) against the oracle pipeline run on the
  same basis; the CG refinement mode against the oracle's CG recurrence.
* The beta 90 -> 150 value update (Eq. z_ray) of that basis against the oracle's values."""
import numpy as np
import pytest

import synth
from oracle import adaptive, eig, graph, pipeline, update
from tests.gpu_common import TOL_PROB, dev, f32, gap_mask, to_dev

pytestmark = pytest.mark.gpu

rw = pytest.importorskip("paper_1607_04174_gb300")
torch = pytest.importorskip("torch")

BETA, GAMMA, M, PER = 90.0, 1e-3, 200, 200


@pytest.fixture(scope="module")
def c2():
    from paper_1607_04174_gb300 import build
    build.build()
    J, dims, truth = synth.voronoi_image(512, 512, seed=synth.BASE_SEED + 1)
    J = f32(J)
    go = graph.build_graph(J, dims, BETA)
    gg = rw.rw_build_graph(to_dev(J, torch.float32), dims, BETA)
    import time
    t0 = time.time()
    b, info = rw.rw_precompute(gg, M, tol=4e-6, seed=1)
    torch.cuda.synchronize()
    print(f"512^2 precompute m={M}: {time.time() - t0:.1f} s, {info}")
    Qd = torch.empty(go.N, M, device=dev())
    lam = rw.rw_basis_get(b, Qd)
    Q = Qd.cpu().numpy().astype(np.float64)
    yield dict(J=J, dims=dims, truth=truth, go=go, gg=gg, b=b, info=info, Q=Q, Qd=Qd, lam=lam)
    rw.rw_basis_free(b)
    rw.rw_graph_free(gg)


def test_c2_lobpcg_basis_matches_shift_invert(c2):
    Q, lam, go = c2["Q"], c2["lam"], c2["go"]
    assert c2["info"]["converged"] == M, c2["info"]
    assert c2["info"]["max_residual"] <= 4e-6
    lr, Qr = eig.smallest_eigpairs(go.Lhat, 240, tol=1e-10)
    bound = 1e-6 * np.maximum(np.abs(lr[:M]), 1e-3)
    ratio = np.abs(lam - lr[:M]) / bound
    print(f"512^2 LOBPCG vs shift-invert: max |dlambda| / bound = {ratio.max():.3f}")
    assert np.all(ratio <= 1.0)
    np.testing.assert_allclose(Q.T @ Q, np.eye(M), atol=2e-5)
    R = go.Lhat @ Q - Q * lam
    assert np.linalg.norm(R, axis=0).max() <= 2e-5
    # principal angles: each GPU column lies in the span of the oracle's first 240 vectors
    proj = np.linalg.norm(Qr.T @ Q, axis=0)
    print(f"512^2 LOBPCG: min norm of the projection on the oracle span = {proj.min():.7f}")
    assert proj.min() >= 1 - 1e-4


def _sets(c2, count, base):
    return [synth.sample_seeds(c2["truth"], c2["dims"], PER, 3, seed=base + 7919 * (k + 1))
            for k in range(count)]


def test_c2_online_solve_matches_oracle_same_basis(c2):
    N = c2["go"].N
    U = torch.empty(N, 4, device=dev())
    lab = torch.empty(N, dtype=torch.uint8, device=dev())
    for si, sl in _sets(c2, 2, synth.BASE_SEED + 17):
        _, info = rw.rw_solve(c2["gg"], c2["b"], to_dev(si), to_dev(sl), 4, U, labels=lab,
                              gamma=GAMMA, m=0, m_step=10, eps=0.1, refine_steps=3)
        m_gpu = info["m_used"]
        m_o, _, _, table = adaptive.choose_m_from_seeds(c2["go"], c2["Q"], si, sl, 4, M, 10, 0.1)
        if m_o != m_gpu:
            fmax = len(si) * 0.1 ** 2
            edge = min(m_o, m_gpu)
            assert abs(table[edge].max() - fmax) / fmax < 1e-3, (m_o, m_gpu)
        ref = pipeline.online_solve(c2["go"], c2["Q"], c2["lam"], si, sl, 4, gamma=GAMMA,
                                    m=m_gpu, refine_steps=3)
        Ug = U.cpu().numpy().astype(np.float64)
        err = np.abs(Ug - ref["U"]).max()
        print(f"512^2 solve on the LOBPCG basis: m={m_gpu} (oracle {m_o}), max |dU| = {err:.2e}")
        assert err <= TOL_PROB
        mask = gap_mask(ref["U"])
        assert np.array_equal(lab.cpu().numpy()[mask], ref["labels"][mask])


def test_c2_cg_refinement_mode(c2):
    """The CG refinement mode against the oracle's CG recurrence from the oracle's fast solve.
    With the FP32 basis copy the start differs by ~1e-6 and 3 CG steps stay within 1e-3; with
    the scaled-FP16 copy the start differs by ~5e-4, which CG's start-dependent step lengths
    can grow, so that error is measured and bounded more loosely."""
    N = c2["go"].N
    U = torch.empty(N, 4, device=dev())
    si, sl = _sets(c2, 1, synth.BASE_SEED + 23)[0]
    errs = {}
    for fmt in (rw.RW_BASIS_F32, rw.RW_BASIS_F16):
        _, info = rw.rw_solve(c2["gg"], c2["b"], to_dev(si), to_dev(sl), 4, U, gamma=GAMMA,
                              m=0, refine_steps=3, refine_mode=rw.RW_REFINE_PCG,
                              basis_format=fmt)
        ref = pipeline.online_solve(c2["go"], c2["Q"], c2["lam"], si, sl, 4, gamma=GAMMA,
                                    m=info["m_used"], refine_steps=3, refine_method="pcg")
        errs[fmt] = np.abs(U.cpu().numpy().astype(np.float64) - ref["U"]).max()
    print(f"512^2 CG refinement: max |dU| FP32 basis {errs[rw.RW_BASIS_F32]:.2e}, "
          f"FP16 basis {errs[rw.RW_BASIS_F16]:.2e}")
    assert errs[rw.RW_BASIS_F32] <= TOL_PROB
    assert errs[rw.RW_BASIS_F16] <= 5e-3


def test_c2_beta_update_values(c2):
    gg = rw.rw_build_graph(to_dev(c2["J"], torch.float32), c2["dims"], BETA)
    b = rw.rw_basis_create(gg, c2["Qd"], c2["lam"])
    try:
        rw.rw_update_weights(gg, b, rw.RW_UPDATE_BETA, beta=150.0)
        ref = update.updated_values(update.update_beta(c2["go"], 150.0), c2["Q"])
        np.testing.assert_allclose(rw.rw_basis_get(b), ref, rtol=2e-5, atol=1e-9)
    finally:
        rw.rw_basis_free(b)
        rw.rw_graph_free(gg)
