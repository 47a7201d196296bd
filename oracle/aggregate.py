"""Aggregated image graphs, Sec. III-C (oracle, FP64).

A projection function eta (N x N-bar, rows sum to 1) and an aggregation function eta-bar
(N x N-bar, columns sum to 1) relate the vertices to super-vertices.  A column q of Q is carried
to the super-vertices either naively, Eq. (q_agg_1):
    q-bar_y = sum_x eta-bar(x, y) q_x,
or with the paper's weighting by the local change of eta, Eq. (q_agg_2):
    Delta(x) = sum_{x' in N(x)} sum_y |eta(x, y) - eta(x', y)|,
    q-bar_y  = sum_x Delta(x) eta-bar(x, y) q_x.
The aggregated columns are made orthonormal by Gram-Schmidt (classical, with one
re-orthogonalization pass, in column order; a column whose norm after projection falls below
1e-10 of its norm before is dropped) and their Ncut values (Eq. z_ray) on the aggregate graph
become the new values.

The paper does not define the aggregate graph's Laplacian.  The reading taken here is the
Galerkin product L-bar = eta^T L eta (rows of eta sum to 1, so L-bar 1 = 0); its degree matrix is
D-bar = diag(L-bar) and its weights W-bar = D-bar - L-bar.  For a hard 0/1 eta this is the usual
coarse graph whose edge weights are the summed weights crossing between the blocks.  If eta-bar
is not given it is eta with its columns normalized to sum to 1.  The columns of Q are aggregated
as stored (in the normalized, "hat" variables) and treated as hat-space vectors of the aggregate
graph.  Test infrastructure only.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


class CSRGraph:
    """A general weighted graph given by its symmetric weight matrix (same interface as the
    grid graph where the solvers need it: N, W, d, L, Lhat, operator)."""

    def __init__(self, W):
        self.W = sp.csr_matrix(W)
        self.N = self.W.shape[0]
        self.d = np.asarray(self.W.sum(axis=1)).ravel()

    @property
    def L(self):
        return (sp.diags(self.d) - self.W).tocsr()

    @property
    def Lhat(self):
        if np.any(self.d <= 0):
            raise ValueError("isolated node")
        s = 1.0 / np.sqrt(self.d)
        return (sp.identity(self.N) - sp.diags(s) @ self.W @ sp.diags(s)).tocsr()

    def operator(self, normalized=True):
        return self.Lhat if normalized else self.L


def column_normalized(eta):
    eta = sp.csc_matrix(eta, dtype=np.float64)
    cs = np.asarray(eta.sum(axis=0)).ravel()
    return (eta @ sp.diags(1.0 / cs)).tocsr()


def delta(g, eta):
    """Delta(x) of Eq. (q_agg_2): sum over graph neighbours x' (edges with w > 0) of the L1
    distance between rows x and x' of eta."""
    eta = sp.csr_matrix(eta, dtype=np.float64)
    live = g.w > 0
    a, b = g.a[live], g.b[live]
    diff = eta[a] - eta[b]
    t = np.asarray(abs(diff).sum(axis=1)).ravel()
    out = np.zeros(g.N)
    np.add.at(out, a, t)
    np.add.at(out, b, t)
    return out


def aggregate_columns(g, Q, eta, eta_bar=None, naive=False):
    eta_bar = column_normalized(eta) if eta_bar is None else sp.csr_matrix(eta_bar)
    Q = np.asarray(Q, dtype=np.float64)
    if naive:
        return np.asarray(eta_bar.T @ Q)                               # Eq. (q_agg_1)
    return np.asarray(eta_bar.T @ (delta(g, eta)[:, None] * Q))        # Eq. (q_agg_2)


def gram_schmidt(A, drop_tol=1e-10):
    """Classical Gram-Schmidt with one re-orthogonalization, column order.  Returns (Qbar,
    kept) where kept lists the surviving column indices."""
    A = np.asarray(A, dtype=np.float64)
    cols, kept = [], []
    for j in range(A.shape[1]):
        v = A[:, j].copy()
        n0 = np.linalg.norm(v)
        if n0 == 0:
            continue
        for _ in range(2):
            if cols:
                Qc = np.stack(cols, axis=1)
                v -= Qc @ (Qc.T @ v)
        nv = np.linalg.norm(v)
        if nv < drop_tol * n0:
            continue
        cols.append(v / nv)
        kept.append(j)
    return np.stack(cols, axis=1), np.array(kept, dtype=np.int64)


def galerkin_graph(g, eta):
    eta = sp.csr_matrix(eta, dtype=np.float64)
    Lbar = (eta.T @ g.L @ eta).tocsr()
    Dbar = Lbar.diagonal()
    Wbar = (sp.diags(Dbar) - Lbar).tocsr()
    Wbar.eliminate_zeros()
    return CSRGraph(Wbar)


def aggregate_basis(g, Q, eta, eta_bar=None, naive=False, normalized=True):
    """Returns (aggregate graph, Q-bar, lambda-bar, kept columns)."""
    from .update import rayleigh_quotients
    gbar = galerkin_graph(g, eta)
    Qbar, kept = gram_schmidt(aggregate_columns(g, Q, eta, eta_bar, naive))
    lam = rayleigh_quotients(Qbar, gbar.operator(normalized))
    return gbar, Qbar, lam, kept


def block_eta(dims, bx, by):
    """Hard 0/1 aggregation of a 2-D grid into bx x by blocks (a test input)."""
    X, Y = dims
    x = np.arange(X * Y) % X
    y = np.arange(X * Y) // X
    nbx = (X + bx - 1) // bx
    col = (x // bx) + nbx * (y // by)
    nbar = int(col.max()) + 1
    return sp.csr_matrix((np.ones(X * Y), (np.arange(X * Y), col)), shape=(X * Y, nbar))
