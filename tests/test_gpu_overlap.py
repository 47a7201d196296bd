"""The projection Z = Q_n^T P-hat_n (Eq. U_lin_comb) behind the fused m x m kernel: at a fixed m
the kernel publishes m as it starts and the projection runs beside the LU of the m x m system
of Eq. (Fs), waiting for it only before it exits; with m chosen adaptively (Sec. III-A-1) the
projection waits for the whole kernel.  These tests check both against the same solves with
events recorded between the kernels (each kernel then starts only after its predecessor has
ended; the arithmetic and the launch shapes are the same, so the results must agree bit for
bit): solves queued back to back on one workspace, with seed sets of different sizes and m
changing from solve to solve (a stale or unpublished m would change Z, unfinished factors
would change C), FP16 and BF16 copies, 2, 4 and 8 labels (4 and 8 padded)."""
import numpy as np
import pytest

import synth
from oracle import graph, pipeline, update
from tests.gpu_common import TOL_PROB, dev, f32, to_dev

pytestmark = pytest.mark.gpu

rw = pytest.importorskip("paper_1607_04174_gb300")
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1607_04174_gb300 import build
    build.build()


def _case(side, n_labels, m):
    J, dims, truth = synth.voronoi_image(side, side, n_regions=n_labels,
                                         seed=synth.BASE_SEED + 40 + n_labels)
    J = f32(J)
    go = graph.build_graph(J, dims, 90.0)
    Q = f32(synth.dct_basis(dims, m))
    lam = update.rayleigh_quotients(Q, go.Lhat)
    return J, dims, truth, go, Q, lam


def _sets(truth, dims, n_labels, pers):
    return [synth.sample_seeds(truth, dims, per, 2, seed=synth.BASE_SEED + 50 + 7 * k,
                               n_labels=n_labels) for k, per in enumerate(pers)]


def _run(J, dims, Q, lam, sets, n_labels, ms_fixed=None, **kw):
    g = rw.rw_build_graph(to_dev(J, torch.float32), dims, 90.0)
    b = rw.rw_basis_create(g, to_dev(Q, torch.float32), lam)
    N = int(np.prod(dims))
    per = [dict(kw, m=m) for m in ms_fixed] if ms_fixed else [kw] * len(sets)
    try:
        dsets = [(to_dev(si), to_dev(sl)) for si, sl in sets]
        # back to back, no host synchronization between the solves
        probs = [torch.empty(N, n_labels, device=dev()) for _ in sets]
        labs = [torch.empty(N, dtype=torch.uint8, device=dev()) for _ in sets]
        for (si, sl), p, lb, o in zip(dsets, probs, labs, per):
            rw.rw_solve(g, b, si, sl, n_labels, p, lb, want_info=False, **o)
        torch.cuda.synchronize()
        fast = [(p.cpu().numpy(), lb.cpu().numpy()) for p, lb in zip(probs, labs)]
        # one at a time, events between the kernels
        ref, ms = [], []
        for (si, sl), o in zip(dsets, per):
            p = torch.empty(N, n_labels, device=dev())
            lb = torch.empty(N, dtype=torch.uint8, device=dev())
            _, info = rw.rw_solve(g, b, si, sl, n_labels, p, lb, record_phases=True, **o)
            ref.append((p.cpu().numpy(), lb.cpu().numpy()))
            ms.append(info["m_used"])
        return fast, ref, ms
    finally:
        rw.rw_basis_free(b)
        rw.rw_graph_free(g)


@pytest.mark.parametrize("fmt", [rw.RW_BASIS_F16, rw.RW_BASIS_BF16])
def test_fixed_m_back_to_back_match_serialized(fmt):
    """512^2, 4 labels: m = 200, 60, 200, 60, 150, 8 from solve to solve (the projection beside
    the LU), seed sets of 200 and 8 per label alternating."""
    J, dims, truth, go, Q, lam = _case(512, 4, 200)
    sets = _sets(truth, dims, 4, [200, 8, 200, 8, 120, 8])
    ms_fixed = [200, 60, 200, 60, 150, 8]
    fast, ref, ms = _run(J, dims, Q, lam, sets, 4, ms_fixed=ms_fixed, gamma=1e-3,
                         refine_steps=3, basis_format=fmt)
    assert ms == ms_fixed
    for (pf, lf), (pr, lr) in zip(fast, ref):
        assert np.array_equal(pf, pr)
        assert np.array_equal(lf, lr)
    if fmt == rw.RW_BASIS_F16:
        for (si, sl), (pf, _), m in zip(sets[:2], fast[:2], ms[:2]):
            o = pipeline.online_solve(go, Q, lam, si, sl, 4, gamma=1e-3, m=m, refine_steps=3)
            assert np.abs(pf.astype(np.float64) - o["U"]).max() <= TOL_PROB


@pytest.mark.parametrize("fmt", [rw.RW_BASIS_F16, rw.RW_BASIS_BF16])
def test_back_to_back_solves_match_serialized(fmt):
    """512^2, 4 labels, m_max = 200: adaptive m alternating between the sets with 200 and with
    8 seeds per label."""
    J, dims, truth, go, Q, lam = _case(512, 4, 200)
    sets = _sets(truth, dims, 4, [200, 8, 200, 8, 120, 8])
    fast, ref, ms = _run(J, dims, Q, lam, sets, 4, gamma=1e-3, m=0, refine_steps=3,
                         basis_format=fmt)
    assert len(set(ms)) > 1, ms   # the sets really change m
    for (pf, lf), (pr, lr) in zip(fast, ref):
        assert np.array_equal(pf, pr)
        assert np.array_equal(lf, lr)
    if fmt == rw.RW_BASIS_F16:   # and the results are the method's
        for (si, sl), (pf, _), m in zip(sets[:2], fast[:2], ms[:2]):
            o = pipeline.online_solve(go, Q, lam, si, sl, 4, gamma=1e-3, m=m, refine_steps=3)
            assert np.abs(pf.astype(np.float64) - o["U"]).max() <= TOL_PROB


def test_eight_labels_and_fixed_m():
    """8 labels (padded to 8, still the bulk-copy projection) with adaptive m, and 2 labels at
    fixed m = 90, 20, 120."""
    J, dims, truth, _, Q, lam = _case(160, 8, 120)
    sets = _sets(truth, dims, 8, [30, 4, 30, 4])
    fast, ref, ms = _run(J, dims, Q, lam, sets, 8, gamma=1e-3, m=0, refine_steps=2)
    assert len(set(ms)) > 1, ms
    for (pf, lf), (pr, lr) in zip(fast, ref):
        assert np.array_equal(pf, pr) and np.array_equal(lf, lr)
    J, dims, truth, _, Q, lam = _case(160, 2, 120)
    sets = _sets(truth, dims, 2, [40, 5, 40])
    fast, ref, ms = _run(J, dims, Q, lam, sets, 2, ms_fixed=[90, 20, 120], gamma=1e-3,
                         refine_steps=0)
    assert ms == [90, 20, 120]
    for (pf, lf), (pr, lr) in zip(fast, ref):
        assert np.array_equal(pf, pr) and np.array_equal(lf, lr)
