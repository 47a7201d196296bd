"""Saving and loading a basis (Sec. V: eigenvectors stored offline, loaded as needed, possibly
only the leading ones) through the C ABI: a round trip returns the same columns and values bit
for bit and the same online solve; loading the first m columns equals a basis made from those
columns; a basis updated to a new beta saves its updated values; foreign, truncated and
mismatched files are refused."""
import numpy as np
import pytest

import synth
from tests.gpu_common import c1_case, dev, to_dev

pytestmark = pytest.mark.gpu

rw = pytest.importorskip("paper_1607_04174_gb300")
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1607_04174_gb300 import build
    build.build()


def _columns(b, N):
    m = rw.rw_basis_m(b)
    Q = torch.empty(N, m, device=dev())
    lam = rw.rw_basis_get(b, Q)
    return Q.cpu().numpy(), lam


def test_basis_round_trip_and_leading_columns(tmp_path):
    case = c1_case(size=48, per=10, m=40)
    N = case["g"].N
    g = rw.rw_build_graph(to_dev(case["J"], torch.float32), case["dims"], case["beta"])
    b = rw.rw_basis_create(g, to_dev(case["Q"], torch.float32), case["lam"])
    path = tmp_path / "basis.rwb"
    loaded = []
    try:
        rw.rw_update_weights(g, b, rw.RW_UPDATE_BETA, beta=120.0)   # values now updated
        Q0, lam0 = _columns(b, N)
        rw.rw_basis_save(b, path)
        b1 = rw.rw_basis_load(g, path)
        loaded.append(b1)
        Q1, lam1 = _columns(b1, N)
        np.testing.assert_array_equal(Q1, Q0)
        np.testing.assert_array_equal(lam1, lam0)
        # the same solve on the saved and the loaded basis
        outs = []
        for bb in (b, b1):
            prob = torch.empty(N, 2, device=dev())
            rw.rw_solve(g, bb, to_dev(case["si"]), to_dev(case["sl"]), 2, prob, m=30,
                        refine_steps=3)
            outs.append(prob.cpu().numpy())
        np.testing.assert_array_equal(outs[0], outs[1])
        # leading 25 columns
        b2 = rw.rw_basis_load(g, path, m_load=25)
        loaded.append(b2)
        Q2, lam2 = _columns(b2, N)
        assert Q2.shape[1] == 25
        np.testing.assert_array_equal(Q2, Q0[:, :25])
        np.testing.assert_array_equal(lam2, lam0[:25])
    finally:
        for bb in loaded:
            rw.rw_basis_free(bb)
        rw.rw_basis_free(b)
        rw.rw_graph_free(g)


def test_basis_load_refusals(tmp_path):
    case = c1_case(size=32, per=6, m=20)
    g = rw.rw_build_graph(to_dev(case["J"], torch.float32), case["dims"], case["beta"])
    J2 = synth.smooth_random_image((32, 30), seed=2)
    g2 = rw.rw_build_graph(to_dev(J2, torch.float32), (32, 30), 90.0)
    b = rw.rw_basis_create(g, to_dev(case["Q"], torch.float32), case["lam"])
    path = tmp_path / "basis.rwb"
    try:
        rw.rw_basis_save(b, path)
        raw = path.read_bytes()
        cases = {"missing": tmp_path / "none.rwb"}
        bad = tmp_path / "bad.rwb"
        bad.write_bytes(b"NOTBASIS" + raw[8:])
        cases["foreign"] = bad
        short = tmp_path / "short.rwb"
        short.write_bytes(raw[:len(raw) - 100])
        cases["truncated"] = short
        for name, p in cases.items():
            with pytest.raises(rw.RWError) as e:
                rw.rw_basis_load(g, p)
            assert e.value.status == rw.RW_ERR_INVALID_ARG, name
        with pytest.raises(rw.RWError) as e:   # another graph shape
            rw.rw_basis_load(g2, path)
        assert e.value.status == rw.RW_ERR_INVALID_ARG
        with pytest.raises(rw.RWError) as e:   # more columns than saved
            rw.rw_basis_load(g, path, m_load=21)
        assert e.value.status == rw.RW_ERR_INVALID_ARG
    finally:
        rw.rw_basis_free(b)
        rw.rw_graph_free(g)
        rw.rw_graph_free(g2)
