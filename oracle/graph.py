"""Image graph of Sec. II-A and the normalized Laplacian of Sec. II-C (oracle, FP64).

Edges join 4-neighbours (2-D) or 6-neighbours (3-D).  Weight of edge (x, y), Eq. (W):
    w_xy = exp(-beta * |J(x) - J(y)|)        (the paper's form, ``form="abs"``)
    w_xy = exp(-beta * (J(x) - J(y))^2)      (the squared form, ``form="sq"``, the default)
D = diag(row sums of W), L = D - W (Sec. II-A).  L-hat = D^{-1/2} L D^{-1/2} (Eq. z_eig).
Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp


def _strides(dims):
    s = [1]
    for k in dims[:-1]:
        s.append(s[-1] * int(k))
    return s


def _coords(dims):
    N = int(np.prod(dims))
    i = np.arange(N, dtype=np.int64)
    out = []
    for k in dims:
        out.append(i % k)
        i = i // k
    return out


def forward_edges(dims):
    """All edges (a, b = a + stride[axis]) with ids axis*N + a, as three int64 arrays."""
    dims = tuple(int(k) for k in dims)
    N = int(np.prod(dims))
    c = _coords(dims)
    ids, A, B = [], [], []
    for ax, (n, st) in enumerate(zip(dims, _strides(dims))):
        a = np.nonzero(c[ax] < n - 1)[0]
        ids.append(ax * N + a)
        A.append(a)
        B.append(a + st)
    return np.concatenate(ids), np.concatenate(A), np.concatenate(B)


def edge_weights(J, a, b, beta, form="sq"):
    """Eq. (W) for the listed edges."""
    diff = np.asarray(J, dtype=np.float64)[a] - np.asarray(J, dtype=np.float64)[b]
    if form == "sq":
        return np.exp(-beta * diff * diff)
    if form == "abs":
        return np.exp(-beta * np.abs(diff))
    raise ValueError(form)


def edge_dweight_dbeta(J, a, b, w, form="sq"):
    """d w_e / d beta for Eq. (W): -(dJ)^2 w (squared form) or -|dJ| w (paper's form)."""
    diff = np.asarray(J, dtype=np.float64)[a] - np.asarray(J, dtype=np.float64)[b]
    return -(diff * diff) * w if form == "sq" else -np.abs(diff) * w


@dataclass
class Graph:
    """Weighted image graph.  ``w`` is indexed like ``ids`` (edge id = axis*N + a)."""
    dims: tuple
    J: np.ndarray
    beta: float
    form: str
    ids: np.ndarray
    a: np.ndarray
    b: np.ndarray
    w: np.ndarray
    N: int = 0
    W: sp.csr_matrix = field(default=None, repr=False)
    d: np.ndarray = field(default=None, repr=False)

    def __post_init__(self):
        self.N = int(np.prod(self.dims))
        self.rebuild()

    def rebuild(self):
        N = self.N
        W = sp.coo_matrix((self.w, (self.a, self.b)), shape=(N, N))
        self.W = (W + W.T).tocsr()
        self.d = np.asarray(self.W.sum(axis=1)).ravel()

    # Sec. II-A: L = D - W
    @property
    def L(self):
        return (sp.diags(self.d) - self.W).tocsr()

    # Sec. II-C: L-hat = D^{-1/2} L D^{-1/2} = I - D^{-1/2} W D^{-1/2}
    @property
    def Lhat(self):
        if np.any(self.d <= 0):
            raise ValueError("isolated node: the normalized Laplacian needs every degree > 0")
        s = 1.0 / np.sqrt(self.d)
        return (sp.identity(self.N) - sp.diags(s) @ self.W @ sp.diags(s)).tocsr()

    def operator(self, normalized=True):
        return self.Lhat if normalized else self.L

    def weights_by_id(self):
        """Dense per-axis weight array [ndim * N] (0 where the edge does not exist)."""
        out = np.zeros(len(self.dims) * self.N)
        out[self.ids] = self.w
        return out

    def with_weights(self, w):
        return Graph(self.dims, self.J, self.beta, self.form, self.ids, self.a, self.b,
                     np.asarray(w, dtype=np.float64).copy())


def build_graph(J, dims, beta, form="sq"):
    """Eq. (W) on the 4-/6-neighbour grid graph of ``dims``."""
    dims = tuple(int(k) for k in dims)
    ids, a, b = forward_edges(dims)
    w = edge_weights(J, a, b, beta, form)
    return Graph(dims, np.asarray(J, dtype=np.float64), float(beta), form, ids, a, b, w)


def set_edge_weights(g, edge_ids, new_w):
    """Return a copy of ``g`` with the listed edges (by id) given new weights (Sec. III-B)."""
    pos = np.searchsorted(g.ids, edge_ids)
    if np.any(pos >= g.ids.size) or np.any(g.ids[np.minimum(pos, g.ids.size - 1)] != edge_ids):
        raise ValueError("edge id does not exist")
    w = g.w.copy()
    w[pos] = new_w
    return g.with_weights(w)
