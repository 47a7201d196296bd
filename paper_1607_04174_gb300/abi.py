"""ctypes mirror of include/rw.h: the structs and the function prototypes of the C ABI.

Argument marshalling only.  Every computation happens inside librwgb.so; if the library is
missing this module raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librwgb.so")

RW_OK = 0
RW_WARN_M_CAPPED = 1
RW_WARN_NOT_CONVERGED = 2
RW_ERR_INVALID_ARG = -1
RW_ERR_CUDA = -2
RW_ERR_OOM = -3
RW_ERR_NOT_CONVERGED = -4
RW_ERR_ISOLATED_NODE = -5
RW_ERR_SINGULAR = -6
RW_ERR_TIMEOUT = -7
RW_ERR_UNSUPPORTED = -9

RW_WEIGHT_SQ, RW_WEIGHT_ABS = 0, 1
RW_REFINE_JACOBI, RW_REFINE_PCG = 0, 1
RW_BASIS_F16, RW_BASIS_BF16, RW_BASIS_F32 = 0, 1, 2
RW_MAX_LABELS = 16
RW_NOALLOC_MAX_M = 1024
RW_UPDATE_BETA, RW_UPDATE_EDGES, RW_UPDATE_ROI, RW_UPDATE_ALL = 0, 1, 2, 3
RW_TOPO_REMOVE_EDGES, RW_TOPO_AGGREGATE = 0, 1
RW_PHASES = ("seeds", "gather", "adapt", "project", "small", "back", "refine")


class rw_graph_desc(C.Structure):
    _fields_ = [("ndim", C.c_int32), ("dims", C.c_int32 * 3), ("beta", C.c_double),
                ("weight_form", C.c_int32), ("normalized", C.c_int32)]


class rw_eig_opts(C.Structure):
    _fields_ = [("m", C.c_int32), ("guard", C.c_int32), ("max_iter", C.c_int32),
                ("tol", C.c_double), ("cheb_degree", C.c_int32), ("seed", C.c_uint64)]


class rw_eig_info(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("converged", C.c_int32),
                ("max_residual", C.c_double), ("stencil_applies", C.c_int32)]


class rw_solve_opts(C.Structure):
    _fields_ = [("gamma", C.c_double), ("m", C.c_int32), ("m_step", C.c_int32),
                ("eps", C.c_double), ("refine_steps", C.c_int32), ("refine_mode", C.c_int32),
                ("omega", C.c_double), ("basis_format", C.c_int32), ("prior_mode", C.c_int32),
                ("record_phases", C.c_int32)]


class rw_solve_info(C.Structure):
    _fields_ = [("m_used", C.c_int32), ("capped", C.c_int32), ("device_status", C.c_int32),
                ("pad_", C.c_int32), ("f_max", C.c_double), ("f", C.c_double * RW_MAX_LABELS),
                ("mu", C.c_double * RW_MAX_LABELS), ("sigma", C.c_double * RW_MAX_LABELS),
                ("phase_ms", C.c_float * 8)]


class rw_weight_update(C.Structure):
    _fields_ = [("kind", C.c_int32), ("pad_", C.c_int32), ("beta", C.c_double),
                ("roi_lo", C.c_int32 * 3), ("roi_hi", C.c_int32 * 3),
                ("edge_ids_dev", C.c_void_p), ("edge_w_dev", C.c_void_p), ("n_edges", C.c_int64)]


class rw_topology_update(C.Structure):
    _fields_ = [("kind", C.c_int32), ("naive", C.c_int32), ("edge_ids_dev", C.c_void_p),
                ("n_edges", C.c_int64), ("n_bar", C.c_int64), ("eta_rowptr_dev", C.c_void_p),
                ("eta_col_dev", C.c_void_p), ("eta_val_dev", C.c_void_p),
                ("etabar_val_dev", C.c_void_p)]


class rw_batch_item(C.Structure):
    _fields_ = [("g", C.c_void_p), ("b", C.c_void_p), ("seed_idx_dev", C.c_void_p),
                ("seed_lab_dev", C.c_void_p), ("S", C.c_int32), ("n_labels", C.c_int32),
                ("priors_dev", C.c_void_p), ("prob_dev", C.c_void_p), ("labels_dev", C.c_void_p)]


P = C.c_void_p
I32, I64, D = C.c_int32, C.c_int64, C.c_double
HP = C.POINTER(C.c_void_p)

PROTOTYPES = {
    "rw_status_str": (C.c_char_p, [I32]),
    "rw_last_error_message": (C.c_char_p, []),
    "rw_kernel_launches": (I64, []),
    "rw_build_graph": (I32, [C.POINTER(rw_graph_desc), P, P, HP]),
    "rw_graph_free": (None, [P]),
    "rw_graph_num_nodes": (I64, [P]),
    "rw_graph_weights": (I32, [P, P, P, P]),
    "rw_apply_laplacian": (I32, [P, P, I64, P, I64, I32, P]),
    "rw_precompute": (I32, [P, C.POINTER(rw_eig_opts), P, HP, C.POINTER(rw_eig_info)]),
    "rw_basis_create": (I32, [P, I32, P, C.POINTER(D), P, HP]),
    "rw_basis_get": (I32, [P, P, C.POINTER(D), P]),
    "rw_basis_m": (I32, [P]),
    "rw_basis_free": (None, [P]),
    "rw_solve": (I32, [P, P, P, P, I32, I32, P, C.POINTER(rw_solve_opts), P, P,
                       C.POINTER(rw_solve_info), P]),
    "rw_solve_host": (I32, [P, P, P, P, I32, I32, P, C.POINTER(rw_solve_opts), P, P,
                            C.POINTER(rw_solve_info), P]),
    "rw_solve_host_async": (I32, [P, P, P, P, I32, I32, P, C.POINTER(rw_solve_opts), P, P,
                                  C.POINTER(rw_solve_info), P]),
    "rw_last_device_status": (I32, [P, P]),
    "rw_solve_pcg": (I32, [P, P, P, I32, I32, P, D, I32, I32, D, P, P, C.POINTER(I32), P]),
    "rw_update_weights": (I32, [P, P, C.POINTER(rw_weight_update), P]),
    "rw_update_topology": (I32, [P, P, C.POINTER(rw_topology_update), P, HP, HP]),
    "rw_grad_exact": (I32, [P, P, P, I32, I32, P, D, P, P, D, I32, P, C.POINTER(D), P]),
    "rw_grad_fast": (I32, [P, P, P, P, I32, I32, P, D, I32, I32, D, P, P, P, C.POINTER(D), P]),
    "rw_solve_priors": (I32, [P, P, P, I32, I32, P, P]),
    "rw_rayleigh_quotients_noalloc": (I32, [P, P, I64, I32, P, P]),
    "rw_block_gram_scratch_bytes": (C.c_size_t, [I64, I32, I32]),
    "rw_basis_save": (I32, [P, C.c_char_p, P]),
    "rw_batch_create": (I32, [I32, HP]),
    "rw_batch_free": (None, [P]),
    "rw_batch_solve": (I32, [P, C.POINTER(rw_batch_item), I32, C.POINTER(rw_solve_opts), P]),
    "rw_batch_capture": (I32, [P, C.POINTER(rw_batch_item), I32, C.POINTER(rw_solve_opts), P,
                               C.POINTER(I32)]),
    "rw_batch_launch": (I32, [P, P]),
    "rw_set_launch_shape": (I32, [I64, I32, I32]),
    "rw_set_tc_passes": (I32, [I32]),
    "rw_basis_nearest_beta": (I32, [C.POINTER(D), I32, D]),
    "rw_registration_priors": (I32, [P, P, I32, C.POINTER(I32), P, I32, I32, P, P]),
    "rw_solve_unseeded": (I32, [P, P, P, I32, C.POINTER(rw_solve_opts), P, P, P, I32, P,
                                C.POINTER(I32), P]),
    "rw_basis_load": (I32, [P, C.c_char_p, I32, P, HP]),
    "rw_block_gram": (I32, [P, I64, P, I64, I64, I32, I32, P, I32, P, C.c_size_t, P]),
}

_lib = None


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "paper_1607_04174_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in PROTOTYPES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib
