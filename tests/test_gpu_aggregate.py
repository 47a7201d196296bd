"""GPU parity: aggregation onto super-vertices (Sec. III-C, Eqs. q_agg_1 / q_agg_2), with hard
block and soft (bilinear) projection functions, against the oracle's aggregated basis,
Galerkin graph and values."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import aggregate
from tests.gpu_common import c1_case, dev, f32, to_dev

pytestmark = pytest.mark.gpu

rw = pytest.importorskip("paper_1607_04174_gb300")
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1607_04174_gb300 import build
    build.build()


def soft_eta(dims, bx, by):
    """Bilinear interpolation weights of every voxel onto a coarse grid with nodes at
    (i bx, j by): rows sum to 1, up to four super-vertices per voxel."""
    X, Y = dims
    nx, ny = -(-(X - 1) // bx) + 1, -(-(Y - 1) // by) + 1   # nodes up to the last voxel
    rows, cols, vals = [], [], []
    for y in range(Y):
        for x in range(X):
            fx, fy = x / bx, y / by
            i0, j0 = int(fx), int(fy)
            tx, ty = fx - i0, fy - j0
            for di, wx in ((0, 1 - tx), (1, tx)):
                for dj, wy in ((0, 1 - ty), (1, ty)):
                    if wx * wy > 0:
                        rows.append(x + X * y)
                        cols.append((i0 + di) + nx * (j0 + dj))
                        vals.append(wx * wy)
    eta = sp.csr_matrix((vals, (rows, cols)), shape=(X * Y, nx * ny))
    return eta


def _as_f32_csr(eta):
    eta = sp.csr_matrix(eta, dtype=np.float64)
    eta.sort_indices()
    eta.data = f32(eta.data)
    return eta


def _dev_csr(eta, data=None):
    return (to_dev(eta.indptr.astype(np.int32)), to_dev(eta.indices.astype(np.int32)),
            to_dev((eta.data if data is None else data).astype(np.float32)))


def _run(case, eta, naive, with_bar=False):
    eta = _as_f32_csr(eta)
    eta_bar = None
    if with_bar:
        eta_bar = aggregate.column_normalized(eta)
        eta_bar.sort_indices()
        eta_bar.data = f32(eta_bar.data)
    gbar, Qbar, lbar, kept = aggregate.aggregate_basis(case["g"], case["Q"], eta, eta_bar,
                                                       naive=naive)
    gg = rw.rw_build_graph(to_dev(case["J"], torch.float32), case["dims"], case["beta"])
    b = rw.rw_basis_create(gg, to_dev(case["Q"], torch.float32), case["lam"])
    rp, cl, vl = _dev_csr(eta)
    vb = to_dev(eta_bar.data.astype(np.float32)) if with_bar else None
    try:
        _, ga, ba = rw.rw_update_topology(gg, b, rw.RW_TOPO_AGGREGATE, n_bar=eta.shape[1],
                                          eta_rowptr=rp, eta_col=cl, eta_val=vl, etabar_val=vb,
                                          naive=naive)
        try:
            k = rw.rw_basis_m(ba)
            assert k == kept.size
            nb = eta.shape[1]
            Qd = torch.empty(nb, k, device=dev())
            lam = rw.rw_basis_get(ba, Qd)
            np.testing.assert_allclose(Qd.cpu().numpy(), Qbar, atol=2e-5)
            np.testing.assert_allclose(lam, lbar, rtol=2e-5, atol=1e-7)
            dd = torch.empty(nb, device=dev())
            rw.rw_graph_weights(ga, None, dd)
            np.testing.assert_allclose(dd.cpu().numpy(), gbar.d, rtol=2e-5)
            Xr = f32(np.random.default_rng(3).standard_normal((nb, 8)))
            Y = torch.empty(nb, 8, device=dev())
            rw.rw_apply_laplacian(ga, to_dev(Xr, torch.float32), Y)
            np.testing.assert_allclose(Y.cpu().numpy(), gbar.Lhat @ Xr, atol=2e-5)
        finally:
            rw.rw_basis_free(ba)
            rw.rw_graph_free(ga)
    finally:
        rw.rw_basis_free(b)
        rw.rw_graph_free(gg)


@pytest.mark.parametrize("naive", [False, True])
def test_hard_block_aggregation(naive):
    case = c1_case(m=40)
    _run(case, aggregate.block_eta(case["dims"], 4, 4), naive)


@pytest.mark.parametrize("naive", [False, True])
def test_soft_bilinear_aggregation(naive):
    case = c1_case(m=40)
    _run(case, soft_eta(case["dims"], 5, 3), naive)


def test_given_etabar_and_rank_loss():
    # 64 super-vertices carry at most 64 independent columns of the 80: columns are dropped
    case = c1_case(m=80)
    _run(case, aggregate.block_eta(case["dims"], 8, 8), False, with_bar=True)


def test_bad_eta_is_rejected():
    case = c1_case(m=10)
    eta = _as_f32_csr(aggregate.block_eta(case["dims"], 4, 4))
    gg = rw.rw_build_graph(to_dev(case["J"], torch.float32), case["dims"], case["beta"])
    b = rw.rw_basis_create(gg, to_dev(case["Q"], torch.float32), case["lam"])
    try:
        rp, cl, _ = _dev_csr(eta)
        bad = to_dev((0.5 * eta.data).astype(np.float32))   # rows sum to 1/2
        with pytest.raises(rw.RWError) as e:
            rw.rw_update_topology(gg, b, rw.RW_TOPO_AGGREGATE, n_bar=eta.shape[1], eta_rowptr=rp,
                                  eta_col=cl, eta_val=bad)
        assert e.value.status == rw.RW_ERR_INVALID_ARG
    finally:
        rw.rw_basis_free(b)
        rw.rw_graph_free(gg)
