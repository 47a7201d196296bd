"""Gradients of a loss on the label probabilities w.r.t. the edge weights and beta (oracle, FP64).

The paper has no gradients; they differentiate its equations.  Exact path: U_n solves
r(U_n, w) = [(L + gamma D~) U - gamma D~ P]_n = 0 (Eq. rw_eq, normalized form of Sec. II-C with
D~ = D; D~ = I unnormalized), U_s fixed.  With G = d loss / d U_n and the adjoint A lambda = G
(A = L_n + gamma D~_n is symmetric), d loss / d w_e = -lambda-bar^T (d r / d w_e), lambda-bar the
adjoint padded with zeros on the seeds.  For the edge e = (a, b), d L / d w_e = (e_a - e_b)
(e_a - e_b)^T and d D / d w_e = e_a e_a^T + e_b e_b^T, so

  d loss / d w_e = - sum_k [ (lam_a - lam_b)(u_a - u_b)
                             + c gamma (lam_a (u_a - p_a) + lam_b (u_b - p_b)) ],

c = 1 with the normalized Laplacian, 0 otherwise.  d loss / d beta = sum_e (d loss / d w_e)
(d w_e / d beta) with d w_e / d beta from Eq. (W).  The priors depend on the intensities only.

The fast path (Q fixed, values from Eq. z_ray under the changed weights) is differentiated here
only by central finite differences (``fd_grad``): its analytic adjoint is a GPU-side product,
checked against these differences.
Test infrastructure only.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from .exact import exact_rw, onehot, split, system
from .graph import edge_dweight_dbeta


def mask_loss(U, truth, seed_idx, label=1):
    """loss = sum over unseeded voxels of (U[x, label] - truth[x])^2 and its gradient."""
    n = split(U.shape[0], seed_idx)
    diff = U[n, label] - truth[n]
    G = np.zeros_like(U)
    G[n, label] = 2.0 * diff
    return float(diff @ diff), G


def exact_grad(g, seed_idx, seed_lab, n_labels, P, gamma, dloss_dU, normalized=True, U=None):
    """Returns (dloss/dw over g.ids order, dloss/dbeta)."""
    if U is None:
        U = exact_rw(g, seed_idx, seed_lab, n_labels, P, gamma, normalized)
    A, _, n = system(g, seed_idx, seed_lab, n_labels, P, gamma, normalized)
    lam_n = spla.splu(A.tocsc()).solve(np.asarray(dloss_dU[n]))
    lam = np.zeros_like(U)
    lam[n] = lam_n
    a, b = g.a, g.b
    gw = -np.sum((lam[a] - lam[b]) * (U[a] - U[b]), axis=1)
    if normalized and gamma > 0:
        gw -= gamma * np.sum(lam[a] * (U[a] - P[a]) + lam[b] * (U[b] - P[b]), axis=1)
    dwdb = edge_dweight_dbeta(g.J, a, b, g.w, g.form)
    return gw, float(gw @ dwdb)


def fd_grad(loss_of_graph, g, edge_pos=None, h_beta=1e-4, h_rel=1e-4, beta=True):
    """Central differences: d loss / d beta (absolute step h_beta) and d loss / d w_e for the
    edges at positions ``edge_pos`` of g.ids (relative step h_rel * w_e)."""
    from .graph import build_graph
    out = {}
    if beta:
        lp = loss_of_graph(build_graph(g.J, g.dims, g.beta + h_beta, g.form))
        lm = loss_of_graph(build_graph(g.J, g.dims, g.beta - h_beta, g.form))
        out["beta"] = (lp - lm) / (2 * h_beta)
    if edge_pos is not None:
        ge = []
        for p in edge_pos:
            h = h_rel * g.w[p]
            wp = g.w.copy(); wp[p] += h
            wm = g.w.copy(); wm[p] -= h
            ge.append((loss_of_graph(g.with_weights(wp)) - loss_of_graph(g.with_weights(wm)))
                      / (2 * h))
        out["edges"] = np.array(ge)
    return out


__all__ = ["mask_loss", "exact_grad", "fd_grad", "onehot"]
