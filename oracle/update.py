"""Updating the precomputed values when edge weights change, Sec. III-B (oracle, FP64).

Ncut(v) = v^T L-hat v / v^T v (Eq. z_ray).  After the weights change, each stored column q^i of
Q keeps its direction and its value becomes lambda-hat_i = Ncut_new(q^i), evaluated with the new
normalized Laplacian; E is then approximated by Q (Lambda-hat + gamma I)^{-1} Q^T.  Edge
removal (topology change with the same vertex set) is the same update with w_e = 0.

The weight changes supported here:
* a new beta for every edge (Eq. W recomputed);
* new weights for a listed set of edges;
* a box-shaped region of interest whose internal edges (both end voxels inside the box) are
  recomputed from Eq. (W) with a local beta;
* removal of listed edges (w_e = 0).
Test infrastructure only.
"""
from __future__ import annotations

import numpy as np

from .graph import build_graph, edge_weights, set_edge_weights


def rayleigh_quotients(Q, op):
    """Eq. (z_ray) for every column of Q."""
    Q = np.asarray(Q, dtype=np.float64)
    return np.einsum("ij,ij->j", Q, op @ Q) / np.einsum("ij,ij->j", Q, Q)


def update_beta(g, beta_new):
    return build_graph(g.J, g.dims, beta_new, g.form)


def update_edges(g, edge_ids, w_new):
    return set_edge_weights(g, np.asarray(edge_ids), np.asarray(w_new, dtype=np.float64))


def roi_mask(g, lo, hi):
    from .graph import _coords
    c = _coords(g.dims)
    inside = np.ones(g.N, dtype=bool)
    for ax in range(len(g.dims)):
        inside &= (c[ax] >= lo[ax]) & (c[ax] < hi[ax])
    return inside


def update_roi(g, lo, hi, beta_local):
    inside = roi_mask(g, lo, hi)
    sel = inside[g.a] & inside[g.b]
    w = g.w.copy()
    w[sel] = edge_weights(g.J, g.a[sel], g.b[sel], beta_local, g.form)
    return g.with_weights(w)


def remove_edges(g, edge_ids):
    return set_edge_weights(g, np.asarray(edge_ids), 0.0)


def updated_values(g_new, Q, normalized=True):
    """lambda-hat for the stored columns under the new graph (Sec. III-B)."""
    return rayleigh_quotients(Q, g_new.operator(normalized))
