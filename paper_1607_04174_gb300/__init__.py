"""GB300 (sm_103a) precomputed random walker: thin Python binding of the C ABI in include/rw.h.

Each function here has the name of the C entry point it calls and only marshals arguments:
device buffers are PyTorch CUDA tensors (passed by pointer), host buffers NumPy arrays, the
stream is the current PyTorch stream unless given.  Handles are opaque integers.  A negative
status raises RWError; there is no fallback path.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import abi
from .abi import *  # noqa: F401,F403  (status codes and enums)


class RWError(RuntimeError):
    def __init__(self, status, what):
        msg = abi.lib().rw_status_str(status).decode()
        detail = abi.lib().rw_last_error_message().decode()
        super().__init__(f"{what}: {msg}" + (f" ({detail})" if detail else ""))
        self.status = status


def _check(s, what):
    if s < 0:
        raise RWError(s, what)
    return s


def _dp(x):
    """Address of a device buffer: a CUDA tensor, an integer address or None.  Host memory
    (a NumPy array or a CPU tensor) is refused here rather than handed to a kernel."""
    if x is None or isinstance(x, int):
        return x
    if isinstance(x, np.ndarray) or not getattr(x, "is_cuda", False):
        raise ValueError("a device buffer (CUDA tensor) is expected here, not host memory")
    return x.data_ptr()


def _hp(x):
    """Address of a host buffer: a C-contiguous NumPy array, a CPU tensor, an integer address
    or None.  A CUDA tensor is refused (the host entry points copy from and to host memory)."""
    if x is None or isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("host arrays must be C-contiguous")
        return x.ctypes.data
    if getattr(x, "is_cuda", False):
        raise ValueError("a host buffer is expected here, not a CUDA tensor")
    return x.data_ptr()


def _stream(stream):
    if stream is not None:
        return stream if isinstance(stream, int) else stream.cuda_stream
    import torch
    return torch.cuda.current_stream().cuda_stream


def _ld(t):
    return t.stride(0) if t.dim() == 2 else t.shape[-1]


def rw_status_str(s):
    return abi.lib().rw_status_str(s).decode()


def rw_last_error_message():
    return abi.lib().rw_last_error_message().decode()


def rw_kernel_launches():
    return abi.lib().rw_kernel_launches()


def rw_build_graph(J, dims, beta, weight_form=abi.RW_WEIGHT_SQ, normalized=True, stream=None):
    d = abi.rw_graph_desc()
    d.ndim = len(dims)
    for i in range(3):
        d.dims[i] = int(dims[i]) if i < len(dims) else 1
    d.beta = float(beta)
    d.weight_form = int(weight_form)
    d.normalized = 1 if normalized else 0
    h = C.c_void_p()
    _check(abi.lib().rw_build_graph(C.byref(d), _dp(J), _stream(stream), C.byref(h)),
           "rw_build_graph")
    return h.value


def rw_graph_free(g):
    abi.lib().rw_graph_free(g)


def rw_graph_num_nodes(g):
    return abi.lib().rw_graph_num_nodes(g)


def rw_graph_weights(g, w=None, d=None, stream=None):
    return _check(abi.lib().rw_graph_weights(g, _dp(w), _dp(d), _stream(stream)), "rw_graph_weights")


def rw_apply_laplacian(g, X, Y, k=None, stream=None):
    k = X.shape[1] if k is None else k
    return _check(abi.lib().rw_apply_laplacian(g, _dp(X), _ld(X), _dp(Y), _ld(Y), k,
                                               _stream(stream)), "rw_apply_laplacian")


def rw_precompute(g, m, guard=-1, max_iter=0, tol=0.0, cheb_degree=-1, seed=0, stream=None):
    o = abi.rw_eig_opts(m=m, guard=guard, max_iter=max_iter, tol=tol, cheb_degree=cheb_degree,
                        seed=seed)
    info = abi.rw_eig_info()
    h = C.c_void_p()
    s = _check(abi.lib().rw_precompute(g, C.byref(o), _stream(stream), C.byref(h), C.byref(info)),
               "rw_precompute")
    return h.value, dict(status=s, iterations=info.iterations, converged=info.converged,
                         max_residual=info.max_residual, stencil_applies=info.stencil_applies)


def rw_basis_create(g, Q, lam, stream=None):
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    h = C.c_void_p()
    _check(abi.lib().rw_basis_create(g, Q.shape[1], _dp(Q),
                                     lam.ctypes.data_as(C.POINTER(C.c_double)), _stream(stream),
                                     C.byref(h)), "rw_basis_create")
    return h.value


def rw_basis_m(b):
    return abi.lib().rw_basis_m(b)


def rw_basis_get(b, Q=None, stream=None):
    lam = np.zeros(rw_basis_m(b))
    _check(abi.lib().rw_basis_get(b, _dp(Q), lam.ctypes.data_as(C.POINTER(C.c_double)),
                                  _stream(stream)), "rw_basis_get")
    return lam


def rw_basis_free(b):
    abi.lib().rw_basis_free(b)


def _solve_opts(gamma, m, m_step, eps, refine_steps, refine_mode, omega, basis_format,
                prior_mode, record_phases=0):
    return abi.rw_solve_opts(gamma=gamma, m=m, m_step=m_step, eps=eps, refine_steps=refine_steps,
                             refine_mode=refine_mode, omega=omega, basis_format=basis_format,
                             prior_mode=prior_mode, record_phases=record_phases)


def _info_dict(info, n_labels):
    return dict(m_used=info.m_used, capped=info.capped, device_status=info.device_status,
                f_max=info.f_max, f=list(info.f)[:n_labels], mu=list(info.mu)[:n_labels],
                sigma=list(info.sigma)[:n_labels],
                phase_ms=dict(zip(abi.RW_PHASES, list(info.phase_ms)[:len(abi.RW_PHASES)])))


def rw_solve(g, b, seed_idx, seed_lab, n_labels, prob, labels=None, priors=None, gamma=1e-3,
             m=0, m_step=10, eps=0.1, refine_steps=3, refine_mode=abi.RW_REFINE_JACOBI,
             omega=0.8, basis_format=abi.RW_BASIS_F16, prior_mode=0, want_info=True,
             record_phases=False, stream=None):
    o = _solve_opts(gamma, m, m_step, eps, refine_steps, refine_mode, omega, basis_format,
                    prior_mode, 1 if record_phases else 0)
    info = abi.rw_solve_info()
    s = _check(abi.lib().rw_solve(g, b, _dp(seed_idx), _dp(seed_lab), len(seed_idx), n_labels,
                                  _dp(priors), C.byref(o), _dp(prob), _dp(labels),
                                  C.byref(info) if want_info else None, _stream(stream)),
               "rw_solve")
    return s, (_info_dict(info, n_labels) if want_info else None)


def rw_solve_host(g, b, seed_idx, seed_lab, n_labels, prob, labels=None, priors=None, gamma=1e-3,
                  m=0, m_step=10, eps=0.1, refine_steps=3, refine_mode=abi.RW_REFINE_JACOBI,
                  omega=0.8, basis_format=abi.RW_BASIS_F16, prior_mode=0, want_info=False,
                  stream=None):
    o = _solve_opts(gamma, m, m_step, eps, refine_steps, refine_mode, omega, basis_format,
                    prior_mode)
    info = abi.rw_solve_info()
    s = _check(abi.lib().rw_solve_host(g, b, _hp(seed_idx), _hp(seed_lab), len(seed_idx),
                                       n_labels, _hp(priors), C.byref(o), _hp(prob), _hp(labels),
                                       C.byref(info) if want_info else None, _stream(stream)),
               "rw_solve_host")
    return s, (_info_dict(info, n_labels) if want_info else None)


def rw_solve_host_async(g, b, seed_idx, seed_lab, n_labels, prob, labels=None, priors=None,
                        gamma=1e-3, m=0, m_step=10, eps=0.1, refine_steps=3,
                        refine_mode=abi.RW_REFINE_JACOBI, omega=0.8,
                        basis_format=abi.RW_BASIS_F16, prior_mode=0, stream=None):
    """rw_solve_host without the final synchronization: the host buffers (pinned) must stay
    valid and prob / labels unread until the stream has passed the call."""
    o = _solve_opts(gamma, m, m_step, eps, refine_steps, refine_mode, omega, basis_format,
                    prior_mode)
    return _check(abi.lib().rw_solve_host_async(g, b, _hp(seed_idx), _hp(seed_lab), len(seed_idx),
                                                n_labels, _hp(priors), C.byref(o), _hp(prob),
                                                _hp(labels), None, _stream(stream)),
                  "rw_solve_host_async")


def rw_last_device_status(g, stream=None):
    return abi.lib().rw_last_device_status(g, _stream(stream))


def rw_solve_pcg(g, seed_idx, seed_lab, n_labels, prob, labels=None, priors=None, gamma=1e-3,
                 prior_mode=0, iters=1000, tol=0.0, want_iters=True, stream=None):
    it = C.c_int32(0)
    S = 0 if seed_idx is None else len(seed_idx)   # no seeds (registration): priors given
    _check(abi.lib().rw_solve_pcg(g, _dp(seed_idx), _dp(seed_lab), S, n_labels,
                                  _dp(priors), gamma, prior_mode, iters, tol, _dp(prob), _dp(labels),
                                  C.byref(it) if want_iters else None, _stream(stream)),
           "rw_solve_pcg")
    return it.value if want_iters else None


def rw_update_weights(g, b, kind, beta=0.0, roi_lo=(0, 0, 0), roi_hi=(1, 1, 1), edge_ids=None,
                      edge_w=None, stream=None):
    u = abi.rw_weight_update()
    u.kind = kind
    u.beta = beta
    for i in range(3):
        u.roi_lo[i] = roi_lo[i] if i < len(roi_lo) else 0
        u.roi_hi[i] = roi_hi[i] if i < len(roi_hi) else 1
    u.edge_ids_dev = _dp(edge_ids)
    u.edge_w_dev = _dp(edge_w)
    u.n_edges = 0 if edge_ids is None else len(edge_ids)
    return _check(abi.lib().rw_update_weights(g, b, C.byref(u), _stream(stream)),
                  "rw_update_weights")


def rw_update_topology(g, b, kind, edge_ids=None, n_bar=0, eta_rowptr=None, eta_col=None,
                       eta_val=None, etabar_val=None, naive=False, stream=None):
    u = abi.rw_topology_update()
    u.kind = kind
    u.naive = 1 if naive else 0
    u.edge_ids_dev = _dp(edge_ids)
    u.n_edges = 0 if edge_ids is None else len(edge_ids)
    u.n_bar = n_bar
    u.eta_rowptr_dev = _dp(eta_rowptr)
    u.eta_col_dev = _dp(eta_col)
    u.eta_val_dev = _dp(eta_val)
    u.etabar_val_dev = _dp(etabar_val)
    ga, ba = C.c_void_p(), C.c_void_p()
    s = _check(abi.lib().rw_update_topology(g, b, C.byref(u), _stream(stream), C.byref(ga),
                                            C.byref(ba)), "rw_update_topology")
    return s, ga.value, ba.value


def rw_grad_exact(g, seed_idx, seed_lab, n_labels, priors, gamma, U, dloss_dU, grad_w,
                  rel_tol=1e-7, max_iter=20000, stream=None):
    gb = C.c_double(0.0)
    S = 0 if seed_idx is None else len(seed_idx)
    _check(abi.lib().rw_grad_exact(g, _dp(seed_idx), _dp(seed_lab), S, n_labels,
                                   _dp(priors), gamma, _dp(U), _dp(dloss_dU), rel_tol, max_iter,
                                   _dp(grad_w), C.byref(gb), _stream(stream)), "rw_grad_exact")
    return gb.value


def rw_grad_fast(g, b, seed_idx, seed_lab, n_labels, priors, gamma, m, dloss_dU, grad_w,
                 refine_steps=3, omega=0.8, U_out=None, stream=None):
    gb = C.c_double(0.0)
    _check(abi.lib().rw_grad_fast(g, b, _dp(seed_idx), _dp(seed_lab), len(seed_idx), n_labels,
                                  _dp(priors), gamma, m, refine_steps, omega, _dp(dloss_dU),
                                  _dp(U_out), _dp(grad_w), C.byref(gb), _stream(stream)),
           "rw_grad_fast")
    return gb.value


def rw_solve_priors(g, seed_idx, seed_lab, n_labels, priors, stream=None):
    return _check(abi.lib().rw_solve_priors(g, _dp(seed_idx), _dp(seed_lab), len(seed_idx),
                                            n_labels, _dp(priors), _stream(stream)),
                  "rw_solve_priors")


def rw_rayleigh_quotients_noalloc(g, Q, lam_out, m=None, stream=None):
    import torch
    m = Q.shape[1] if m is None else m
    if Q.dtype != torch.float32 or Q.dim() != 2 or Q.stride(1) != 1:
        raise ValueError("Q must be a 2-D float32 tensor with unit column stride")
    if Q.shape[0] != abi.lib().rw_graph_num_nodes(g):
        raise ValueError("Q must have one row per graph node")
    if not 1 <= m <= Q.shape[1]:
        raise ValueError("m must be in [1, Q.shape[1]]")
    if lam_out.dtype != torch.float64 or not lam_out.is_contiguous() or lam_out.numel() < m:
        raise ValueError("lam_out must be a contiguous float64 tensor of at least m entries")
    return _check(abi.lib().rw_rayleigh_quotients_noalloc(g, _dp(Q), _ld(Q), m, _dp(lam_out),
                                                          _stream(stream)),
                  "rw_rayleigh_quotients_noalloc")


def rw_block_gram_scratch_bytes(N, p, q):
    return abi.lib().rw_block_gram_scratch_bytes(N, p, q)


def rw_block_gram(A, B, G, scratch, stream=None):
    """G (p x q float64, CUDA) = A^T B for CUDA float32 blocks A (N x p), B (N x q) on the
    tensor cores; scratch: a CUDA byte tensor of rw_block_gram_scratch_bytes(N, p, q)."""
    N, p = A.shape
    q = B.shape[1]
    if B.shape[0] != N or G.shape[0] < p or G.shape[1] < q:
        raise ValueError("shapes: A N x p, B N x q, G at least p x q")
    return _check(abi.lib().rw_block_gram(_dp(A), _ld(A), _dp(B), _ld(B), N, p, q, _dp(G),
                                          _ld(G), _dp(scratch), scratch.numel() * scratch.element_size(),
                                          _stream(stream)), "rw_block_gram")


def rw_basis_save(b, path, stream=None):
    return _check(abi.lib().rw_basis_save(b, str(path).encode(), _stream(stream)),
                  "rw_basis_save")


def rw_basis_load(g, path, m_load=0, stream=None):
    h = C.c_void_p()
    _check(abi.lib().rw_basis_load(g, str(path).encode(), m_load, _stream(stream), C.byref(h)),
           "rw_basis_load")
    return h.value


# ----------------------------------------------------------------------------- batched serving


def rw_batch_create(n_streams=8):
    h = C.c_void_p()
    _check(abi.lib().rw_batch_create(n_streams, C.byref(h)), "rw_batch_create")
    return h.value


def rw_batch_free(bt):
    abi.lib().rw_batch_free(bt)


def _batch_items(items):
    """items: sequence of dicts with g, b, seed_idx, seed_lab, n_labels, prob, and optionally
    labels and priors (CUDA tensors)."""
    arr = (abi.rw_batch_item * len(items))()
    for k, it in enumerate(items):
        a = arr[k]
        a.g, a.b = it["g"], it["b"]
        a.seed_idx_dev, a.seed_lab_dev = _dp(it["seed_idx"]), _dp(it["seed_lab"])
        a.S = len(it["seed_idx"])
        a.n_labels = it["n_labels"]
        a.priors_dev = _dp(it.get("priors"))
        a.prob_dev = _dp(it["prob"])
        a.labels_dev = _dp(it.get("labels"))
    return arr


def rw_batch_solve(bt, items, gamma=1e-3, m=0, m_step=10, eps=0.1, refine_steps=3,
                   refine_mode=abi.RW_REFINE_JACOBI, omega=0.8, basis_format=abi.RW_BASIS_F16,
                   prior_mode=0, stream=None):
    o = _solve_opts(gamma, m, m_step, eps, refine_steps, refine_mode, omega, basis_format,
                    prior_mode)
    arr = _batch_items(items)
    return _check(abi.lib().rw_batch_solve(bt, arr, len(items), C.byref(o), _stream(stream)),
                  "rw_batch_solve")


def rw_batch_capture(bt, items, gamma=1e-3, m=0, m_step=10, eps=0.1, refine_steps=3,
                     refine_mode=abi.RW_REFINE_JACOBI, omega=0.8, basis_format=abi.RW_BASIS_F16,
                     prior_mode=0, stream=None):
    """Returns 1 when the held graph was updated in place, 0 when it was instantiated."""
    o = _solve_opts(gamma, m, m_step, eps, refine_steps, refine_mode, omega, basis_format,
                    prior_mode)
    arr = _batch_items(items)
    upd = C.c_int32(0)
    _check(abi.lib().rw_batch_capture(bt, arr, len(items), C.byref(o), _stream(stream),
                                      C.byref(upd)), "rw_batch_capture")
    return upd.value


def rw_batch_launch(bt, stream=None):
    return _check(abi.lib().rw_batch_launch(bt, _stream(stream)), "rw_batch_launch")


def rw_set_launch_shape(n_max, proj_per_sm, back_per_sm):
    return _check(abi.lib().rw_set_launch_shape(n_max, proj_per_sm, back_per_sm),
                  "rw_set_launch_shape")


def rw_set_tc_passes(mask):
    """bit 0: projection on the tensor cores, bit 1: back-projection; 4 (the default): both on
    the tensor cores for passes of more than 8 labels; 0: CUDA cores; 3: tensor cores."""
    return _check(abi.lib().rw_set_tc_passes(int(mask)), "rw_set_tc_passes")


def load_launch_shapes(path=None):
    """Installs the launch-shape table measured by the project's autotuner
    (paper_1607_04174_gb300/autotune.py); returns the entries installed."""
    import json
    import os
    path = path or os.path.join(os.path.dirname(os.path.abspath(__file__)), "launch_shapes.json")
    if not os.path.exists(path):
        return []
    with open(path) as f:
        table = json.load(f)
    rw_set_launch_shape(0, 1, 1)
    for e in table["entries"]:
        rw_set_launch_shape(int(e["n_max"]), int(e["proj_per_sm"]), int(e["back_per_sm"]))
    return table["entries"]


# ----------------------------------------------------------------------------- registration


def rw_registration_priors(fixed, moving, dims, disp, priors, half=2, stream=None):
    """priors (N x K float32, CUDA) from the fixed and moving images (N float32, CUDA) and the
    K x ndim int32 displacements disp (CUDA)."""
    d = (C.c_int32 * 3)(*(list(int(v) for v in dims) + [1] * (3 - len(dims))))
    return _check(abi.lib().rw_registration_priors(_dp(fixed), _dp(moving), len(dims), d,
                                                   _dp(disp), disp.shape[0], half, _dp(priors),
                                                   _stream(stream)), "rw_registration_priors")


def rw_solve_unseeded(g, b, priors, prob, labels=None, disp=None, field=None, gamma=1.0, m=0,
                      m_step=10, eps=0.1, refine_steps=3, omega=0.8,
                      basis_format=abi.RW_BASIS_F16, want_m=True, stream=None):
    """Returns the m used (want_m) or None."""
    o = _solve_opts(gamma, m, m_step, eps, refine_steps, abi.RW_REFINE_JACOBI, omega,
                    basis_format, 1)
    mu = C.c_int32(0)
    _check(abi.lib().rw_solve_unseeded(g, b, _dp(priors), priors.shape[1], C.byref(o), _dp(prob),
                                       _dp(labels), _dp(disp),
                                       0 if disp is None else disp.shape[1], _dp(field),
                                       C.byref(mu) if want_m else None, _stream(stream)),
           "rw_solve_unseeded")
    return mu.value if want_m else None


def rw_basis_nearest_beta(betas, beta):
    """Index of the precomputed beta' nearest to beta in log beta (-1 if invalid)."""
    arr = np.ascontiguousarray(betas, dtype=np.float64)
    return abi.lib().rw_basis_nearest_beta(arr.ctypes.data_as(C.POINTER(C.c_double)), len(arr),
                                           float(beta))
