"""Label probabilities of the random walker as differentiable PyTorch functions.

``exact_probabilities`` solves Eq. (rw_eq) in the normalized form of Sec. II-C with the
library's PCG kernel; ``fast_probabilities`` runs the eigenvector solve of Sec. II-B at a fixed
m with the basis held fixed and its values recomputed by Eq. (z_ray) under the current weights,
followed by damped-Jacobi refinement.  Each is a function of beta (Eq. W) or of the edge weights
(ndim x N, edge-id layout: entry axis * N + i is the edge from voxel i to its successor along
that axis).  The forward pass installs the weights in the graph handle (it mutates the graph,
and for the fast path the basis values) and solves; the backward pass calls the library's
adjoint entry points (``rw_grad_exact`` / ``rw_grad_fast``).  This module only passes
arguments: every step of both passes runs in the library's kernels.
"""
from __future__ import annotations

import torch

from . import abi
from . import (rw_grad_exact, rw_grad_fast, rw_graph_num_nodes, rw_solve, rw_solve_pcg,
               rw_update_weights)


def _install(graph, basis, kind, param):
    if kind == "beta":
        rw_update_weights(graph, basis, abi.RW_UPDATE_BETA, beta=float(param))
    else:
        rw_update_weights(graph, basis, abi.RW_UPDATE_ALL,
                          edge_w=param.detach().to(torch.float32).contiguous())


def _grad_out(kind, param, gw, gb):
    if kind == "beta":
        return torch.as_tensor(gb, dtype=param.dtype, device=param.device).reshape(param.shape)
    return gw[: param.numel()].to(param.dtype).reshape(param.shape)


class _Exact(torch.autograd.Function):
    @staticmethod
    def forward(ctx, param, kind, graph, seed_idx, seed_lab, n_labels, priors, gamma, tol,
                max_iter):
        _install(graph, None, kind, param)
        N = rw_graph_num_nodes(graph)
        U = torch.empty(N, n_labels, device=priors.device, dtype=torch.float32)
        rw_solve_pcg(graph, seed_idx, seed_lab, n_labels, U, priors=priors, gamma=gamma,
                     prior_mode=1, iters=max_iter, tol=tol, want_iters=False)
        ctx.save_for_backward(U)
        ctx.args = (param, kind, graph, seed_idx, seed_lab, n_labels, priors, gamma, tol, max_iter)
        return U

    @staticmethod
    def backward(ctx, dU):
        (U,) = ctx.saved_tensors
        param, kind, graph, si, sl, L, priors, gamma, tol, max_iter = ctx.args
        gw = torch.empty(3 * U.shape[0], device=U.device, dtype=torch.float32)
        gb = rw_grad_exact(graph, si, sl, L, priors, gamma, U, dU.to(torch.float32).contiguous(),
                           gw, rel_tol=tol, max_iter=max_iter)
        return (_grad_out(kind, param, gw, gb),) + (None,) * 9


class _Fast(torch.autograd.Function):
    @staticmethod
    def forward(ctx, param, kind, graph, basis, seed_idx, seed_lab, n_labels, priors, gamma, m,
                refine_steps, omega):
        _install(graph, basis, kind, param)
        N = rw_graph_num_nodes(graph)
        U = torch.empty(N, n_labels, device=priors.device, dtype=torch.float32)
        rw_solve(graph, basis, seed_idx, seed_lab, n_labels, U, priors=priors, gamma=gamma, m=m,
                 refine_steps=refine_steps, omega=omega, basis_format=abi.RW_BASIS_F32,
                 prior_mode=1, want_info=False)
        ctx.args = (param, kind, graph, basis, seed_idx, seed_lab, n_labels, priors, gamma, m,
                    refine_steps, omega, N)
        return U

    @staticmethod
    def backward(ctx, dU):
        param, kind, graph, basis, si, sl, L, priors, gamma, m, steps, omega, N = ctx.args
        gw = torch.empty(3 * N, device=dU.device, dtype=torch.float32)
        gb = rw_grad_fast(graph, basis, si, sl, L, priors, gamma, m,
                          dU.to(torch.float32).contiguous(), gw, refine_steps=steps, omega=omega)
        return (_grad_out(kind, param, gw, gb),) + (None,) * 11


def _param(beta, weights):
    if (beta is None) == (weights is None):
        raise ValueError("give exactly one of beta and weights")
    return ("beta", beta) if beta is not None else ("weights", weights)


def exact_probabilities(graph, seed_idx, seed_lab, n_labels, priors, *, beta=None, weights=None,
                        gamma=1e-3, tol=1e-6, max_iter=20000):
    """U (N x n_labels) of Eq. (rw_eq), differentiable w.r.t. ``beta`` (a scalar tensor) or
    ``weights`` (ndim * N tensor).  ``priors``: N x n_labels device tensor."""
    kind, p = _param(beta, weights)
    return _Exact.apply(p, kind, graph, seed_idx, seed_lab, n_labels, priors, gamma, tol,
                        max_iter)


def fast_probabilities(graph, basis, seed_idx, seed_lab, n_labels, priors, m, *, beta=None,
                       weights=None, gamma=1e-3, refine_steps=3, omega=0.8):
    """U (N x n_labels) of the eigenvector solve with the first ``m`` basis columns,
    differentiable w.r.t. ``beta`` or ``weights``."""
    kind, p = _param(beta, weights)
    return _Fast.apply(p, kind, graph, basis, seed_idx, seed_lab, n_labels, priors, gamma, m,
                       refine_steps, omega)
