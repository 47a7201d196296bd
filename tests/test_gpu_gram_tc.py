"""GPU parity of the tensor-core Gram product G = A^T B (rw_block_gram), the dense contraction
of the eigensolver's projected matrices (Sec. II-B, Eq. L_eigs), against the FP64 product of
the same FP32 inputs: ragged tile edges in every dimension (p, q not multiples of the 128 x 256
output tile, N not a multiple of the 32-row stage or the 1024-row slice), pitches wider than
the rows, a single row, and two calls in a row on one scratch buffer."""
import numpy as np
import pytest

from tests.gpu_common import dev

pytestmark = pytest.mark.gpu

rw = pytest.importorskip("paper_1607_04174_gb300")
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1607_04174_gb300 import build
    build.build()


CASES = [(5000, 200, 300), (1030, 7, 513), (1, 130, 3), (40000, 360, 260), (2048, 256, 256)]


def _gram(A, B, pad=0):
    N, p = A.shape
    q = B.shape[1]
    Ad = torch.zeros(N, p + pad, device=dev())
    Bd = torch.zeros(N, q + pad, device=dev())
    Ad[:, :p] = torch.from_numpy(A).to(dev())
    Bd[:, :q] = torch.from_numpy(B).to(dev())
    G = torch.full((p, q + pad), float("nan"), dtype=torch.float64, device=dev())
    nbytes = rw.rw_block_gram_scratch_bytes(N, p, q)
    scratch = torch.empty(nbytes, dtype=torch.uint8, device=dev())
    rw.rw_block_gram(Ad[:, :p], Bd[:, :q], G, scratch)
    torch.cuda.synchronize()
    status = int(scratch[:4].view(torch.int32).item())
    return G[:, :q].cpu().numpy(), status, (Ad, Bd, G, scratch)


@pytest.mark.parametrize("N,p,q", CASES)
def test_block_gram_matches_fp64_product(N, p, q):
    rng = np.random.default_rng(N + p + q)
    A = rng.standard_normal((N, p)).astype(np.float32)
    B = (rng.standard_normal((N, q)) * np.logspace(-3, 2, q)).astype(np.float32)
    G, status, _ = _gram(A, B, pad=4)
    assert status == 0
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    ref = A64.T @ B64
    scale = np.abs(A64).T @ np.abs(B64)
    ratio = np.abs(G - ref) / (scale + 1e-300)
    print(f"gram N={N} p={p} q={q}: max |err| / (|A|^T |B|) = {ratio.max():.2e}")
    assert ratio.max() <= 1e-5


def test_block_gram_orthonormal_block_and_repeat():
    """Columns of an orthonormal block give the identity to well below FP32 Cholesky-QR's
    needs; a second call on the same scratch returns the same bits."""
    rng = np.random.default_rng(3)
    N, k = 70000, 240
    Q, _ = np.linalg.qr(rng.standard_normal((N, k)))
    Q = Q.astype(np.float32)
    G1, s1, bufs = _gram(Q, Q)
    Ad, Bd, G, scratch = bufs
    rw.rw_block_gram(Ad, Bd, G, scratch)
    torch.cuda.synchronize()
    G2 = G.cpu().numpy()
    assert s1 == 0
    np.testing.assert_array_equal(G1, G2)
    Q64 = Q.astype(np.float64)
    ref = Q64.T @ Q64
    err = np.abs(G1 - ref).max()
    print(f"gram of an orthonormal 70000 x 240 block: max |err| = {err:.2e}")
    assert err <= 2e-6


def test_block_gram_rejects_small_scratch():
    A = torch.zeros(100, 8, device=dev())
    G = torch.zeros(8, 8, dtype=torch.float64, device=dev())
    small = torch.empty(256, dtype=torch.uint8, device=dev())
    with pytest.raises(rw.RWError) as e:
        rw.rw_block_gram(A, A, G, small)
    assert e.value.status == rw.RW_ERR_INVALID_ARG
