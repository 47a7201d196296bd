"""GPU test of the entry point that allocates nothing (rw_rayleigh_quotients_noalloc).

It must return what the allocating path returns: the Rayleigh quotients that the value update
computes when the weights are unchanged.  Two calls in a row check that the shared scratch
array is cleared between calls.  This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_noalloc_rayleigh_matches_allocating_update_path():
    import paper_1607_04174_gb300 as rw
    from paper_1607_04174_gb300 import abi, build
    from tests.gpu_common import c1_case, dev, to_dev
    build.build()
    case = c1_case(size=48, per=8, m=40)
    lib = abi.lib()
    g = rw.rw_build_graph(to_dev(case["J"], torch.float32), case["dims"], case["beta"])
    Qd = to_dev(case["Q"], torch.float32)
    b = rw.rw_basis_create(g, Qd, case["lam"])
    try:
        rw.rw_update_weights(g, b, rw.RW_UPDATE_BETA, beta=case["beta"])
        ref = rw.rw_basis_get(b)
        stream = torch.cuda.current_stream().cuda_stream
        m = Qd.shape[1]
        for call in range(2):
            out = torch.full((m,), float("nan"), dtype=torch.float64, device=dev())
            s = lib.rw_rayleigh_quotients_noalloc(g, Qd.data_ptr(), Qd.stride(0), m,
                                                  out.data_ptr(), stream)
            assert s == rw.RW_OK, (call, lib.rw_status_str(s))
            torch.cuda.synchronize()
            np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=2e-5, atol=1e-9)
        # a size beyond the stated maximum is rejected
        s = lib.rw_rayleigh_quotients_noalloc(g, Qd.data_ptr(), 1028, abi.RW_NOALLOC_MAX_M + 4,
                                              out.data_ptr(), stream)
        assert s == rw.RW_ERR_INVALID_ARG
        assert b"1024" in lib.rw_last_error_message()
    finally:
        rw.rw_basis_free(b)
        rw.rw_graph_free(g)
