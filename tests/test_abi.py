"""CPU checks of the C ABI: the library builds, loads, exports every entry point that
include/rw.h declares, and the ctypes structs match the C layouts (sizes and offsets from a
gcc-compiled probe).  No compute calls: there is no GPU here."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rw.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rw_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1607_04174_gb300 import abi, build
    build.build()
    return abi.lib()


def test_every_declared_entry_point_is_exported(lib):
    names = _declared()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_entry_point():
    from paper_1607_04174_gb300 import abi
    import paper_1607_04174_gb300 as rw
    for n in _declared():
        assert n in abi.PROTOTYPES, n
        assert hasattr(rw, n), n


def test_status_strings(lib):
    lib.rw_status_str.restype = C.c_char_p
    assert lib.rw_status_str(0) == b"RW_OK"
    assert lib.rw_status_str(-1) == b"RW_ERR_INVALID_ARG"
    assert lib.rw_status_str(-9) == b"RW_ERR_UNSUPPORTED"
    assert lib.rw_status_str(12345) == b"RW_UNKNOWN_STATUS"


def test_struct_layouts_match_c(tmp_path):
    from paper_1607_04174_gb300 import abi
    structs = {
        "rw_graph_desc": ["ndim", "dims", "beta", "weight_form", "normalized"],
        "rw_eig_opts": ["m", "guard", "max_iter", "tol", "cheb_degree", "seed"],
        "rw_eig_info": ["iterations", "converged", "max_residual", "stencil_applies"],
        "rw_solve_opts": ["gamma", "m", "m_step", "eps", "refine_steps", "refine_mode", "omega",
                          "basis_format", "prior_mode", "record_phases"],
        "rw_solve_info": ["m_used", "capped", "device_status", "f_max", "f", "mu", "sigma",
                          "phase_ms"],
        "rw_weight_update": ["kind", "beta", "roi_lo", "roi_hi", "edge_ids_dev", "edge_w_dev",
                             "n_edges"],
        "rw_topology_update": ["kind", "naive", "edge_ids_dev", "n_edges", "n_bar",
                               "eta_rowptr_dev", "eta_col_dev", "eta_val_dev", "etabar_val_dev"],
        "rw_batch_item": ["g", "b", "seed_idx_dev", "seed_lab_dev", "S", "n_labels",
                          "priors_dev", "prob_dev", "labels_dev"],
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', "int main(){"]
    for s, fields in structs.items():
        lines.append(f'printf("{s} %zu\\n", sizeof({s}));')
        for f in fields:
            lines.append(f'printf("{s}.{f} %zu\\n", offsetof({s}, {f}));')
    lines.append("return 0;}")
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-std=c11", str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    got = dict(line.split() for line in out.strip().splitlines())
    for s, fields in structs.items():
        cls = getattr(abi, s)
        assert int(got[s]) == C.sizeof(cls), s
        for f in fields:
            assert int(got[f"{s}.{f}"]) == getattr(cls, f).offset, f"{s}.{f}"


def _null_args(argtypes):
    """Integers 1, doubles 1.0, every pointer NULL."""
    args = []
    for t in argtypes:
        if t in (C.c_int32, C.c_int64, C.c_size_t):
            args.append(1)
        elif t is C.c_double:
            args.append(1.0)
        else:
            args.append(None)
    return args


def test_null_handles_are_refused_on_the_host(lib):
    """Every entry point that returns a status checks its arguments before any device work:
    with NULL handles and buffers it returns RW_ERR_INVALID_ARG and launches nothing (the
    library's launch counter stays put).  The accessors and destructors accept NULL."""
    from paper_1607_04174_gb300 import abi
    before = lib.rw_kernel_launches()
    status_calls = [n for n, (res, _) in abi.PROTOTYPES.items()
                    if res is C.c_int32 and n not in ("rw_basis_m", "rw_set_launch_shape",
                                                      "rw_basis_nearest_beta",
                                                      "rw_set_tc_passes")]
    assert len(status_calls) >= 17
    for name in status_calls:
        st = getattr(lib, name)(*_null_args(abi.PROTOTYPES[name][1]))
        assert st == -1, (name, st)
    assert lib.rw_basis_m(None) == 0
    assert lib.rw_graph_num_nodes(None) == 0
    assert lib.rw_block_gram_scratch_bytes(1, 0, 1) == 0
    assert lib.rw_set_launch_shape(4096, 0, 3) == -1      # a shape out of range
    assert lib.rw_set_launch_shape(4096, 1, 9) == -1
    assert lib.rw_set_launch_shape(0, 1, 1) == 0          # clears the (host-side) table
    assert lib.rw_set_tc_passes(0) == 0 and lib.rw_set_tc_passes(3) == 0   # host-side switch
    assert lib.rw_set_tc_passes(5) == -1 and lib.rw_set_tc_passes(4) == 0
    assert lib.rw_basis_nearest_beta(None, 1, 1.0) == -1
    lib.rw_batch_free(None)
    assert lib.rw_block_gram_scratch_bytes(2048, 128, 256) == 256 + 4 * 128 * 256 * 2
    lib.rw_graph_free(None)
    lib.rw_basis_free(None)
    assert lib.rw_kernel_launches() == before
    # every declared entry point is one of the calls above or an accessor checked elsewhere
    covered = set(status_calls) | {"rw_basis_m", "rw_graph_num_nodes", "rw_graph_free",
                                   "rw_block_gram_scratch_bytes", "rw_set_launch_shape",
                                   "rw_basis_nearest_beta", "rw_set_tc_passes",
                                   "rw_batch_free",
                                   "rw_basis_free", "rw_status_str", "rw_last_error_message",
                                   "rw_kernel_launches"}
    assert set(_declared()) <= covered, sorted(set(_declared()) - covered)


@pytest.mark.parametrize("field,value", [("ndim", 1), ("ndim", 4), ("beta", -1.0),
                                         ("beta", float("nan")), ("weight_form", 7),
                                         ("dims0", 0), ("dims2", 0), ("huge", None)])
def test_invalid_graph_descriptors_are_refused(lib, field, value):
    """rw_build_graph rejects a bad descriptor before it touches the image or the device
    (the image pointer below is a host address that is never read) and clears *out."""
    from paper_1607_04174_gb300 import abi
    import numpy as np
    desc = abi.rw_graph_desc()
    desc.ndim, desc.beta, desc.weight_form, desc.normalized = 3, 90.0, 0, 1
    desc.dims[0], desc.dims[1], desc.dims[2] = 8, 8, 8
    if field == "dims0":
        desc.dims[0] = value
    elif field == "dims2":
        desc.dims[2] = value
    elif field == "huge":  # N = 2^33 nodes does not fit the 32-bit node index
        desc.dims[0], desc.dims[1], desc.dims[2] = 2048, 2048, 2048
    else:
        setattr(desc, field, value)
    image = np.zeros(4, np.float32)
    out = C.c_void_p(12345)
    before = lib.rw_kernel_launches()
    st = lib.rw_build_graph(C.byref(desc), image.ctypes.data, None, C.byref(out))
    assert st == -1
    assert out.value is None
    assert lib.rw_kernel_launches() == before


class _FakeCudaTensor:
    """Stands in for a CUDA tensor (no GPU here): only the two attributes the binding reads."""
    is_cuda = True

    def data_ptr(self):
        return 0x1000


def test_binding_refuses_the_wrong_kind_of_memory(lib):
    """Device entry points refuse host memory (NumPy arrays, CPU tensors) and the host entry
    points refuse CUDA tensors, in the binding, before the library is called."""
    import numpy as np
    import torch

    import paper_1607_04174_gb300 as rw
    before = lib.rw_kernel_launches()
    si, sl = np.zeros(4, np.int32), np.zeros(4, np.int32)
    prob = np.zeros((8, 2), np.float32)
    with pytest.raises(ValueError, match="device buffer"):
        rw.rw_solve(1, 1, si, sl, 2, prob)
    with pytest.raises(ValueError, match="device buffer"):
        rw.rw_solve(1, 1, torch.from_numpy(si), torch.from_numpy(sl), 2, torch.from_numpy(prob))
    with pytest.raises(ValueError, match="device buffer"):
        rw.rw_build_graph(np.zeros(16, np.float32), (4, 4), 1.0)
    with pytest.raises(ValueError, match="device buffer"):
        rw.rw_solve_pcg(1, torch.from_numpy(si), torch.from_numpy(sl), 2, prob)
    with pytest.raises(ValueError, match="host buffer"):
        rw.rw_solve_host(1, 1, si, sl, 2, _FakeCudaTensor())
    with pytest.raises(ValueError, match="host buffer"):
        rw.rw_solve_host_async(1, 1, _FakeCudaTensor(), sl, 2, prob)
    with pytest.raises(ValueError, match="C-contiguous"):
        rw.rw_solve_host(1, 1, si, sl, 2, np.zeros((2, 8), np.float32).T)
    assert lib.rw_kernel_launches() == before


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without the built library every call raises ImportError: there is no CPU fallback."""
    from paper_1607_04174_gb300 import abi
    import paper_1607_04174_gb300 as rw
    monkeypatch.setattr(abi, "LIB_PATH", str(tmp_path / "librwgb.so"))
    monkeypatch.setattr(abi, "_lib", None)
    with pytest.raises(ImportError, match="missing"):
        rw.rw_kernel_launches()
    with pytest.raises(ImportError, match="missing"):
        rw.rw_status_str(0)


def test_nearest_beta_in_log_space(lib):
    """Host-only selection among bases precomputed at several beta' (Sec. III-B): nearest in
    log beta, ties to the lower index, invalid input refused."""
    import numpy as np
    import paper_1607_04174_gb300 as rw
    betas = [45.0, 90.0, 180.0]
    assert rw.rw_basis_nearest_beta(betas, 150.0) == 2      # |log 150/180| < |log 150/90|
    assert rw.rw_basis_nearest_beta(betas, 120.0) == 1      # |log 120/90| < |log 120/180|
    assert rw.rw_basis_nearest_beta(betas, 10.0) == 0
    assert rw.rw_basis_nearest_beta([40.0, 160.0], 80.0) == 0   # equal ratios: lower index
    assert rw.rw_basis_nearest_beta(betas, 0.0) == -1
    assert rw.rw_basis_nearest_beta([1.0, -2.0], 1.0) == -1
    for beta in np.geomspace(5.0, 500.0, 23):
        want = int(np.argmin(np.abs(np.log(betas) - np.log(beta))))
        assert rw.rw_basis_nearest_beta(betas, beta) == want
