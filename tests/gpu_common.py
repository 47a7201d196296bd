"""Shared set-up for the GPU parity tests: seeded inputs, the oracle's reference values and the
library handles.  Inputs go to both sides as the same float32 arrays; the oracle sees them
widened to float64."""
from __future__ import annotations

import numpy as np

import synth
from oracle import eig, graph

TOL_PROB = 1e-3  # max-abs probability error against the oracle


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def dev():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch.device("cuda:0")


def to_dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(dev())


def c1_case(size=64, per=20, beta=90.0, m=50, seed=synth.BASE_SEED):
    """Config-1-like: closed-curve image, 2 labels, seeds at Chebyshev distance >= 2."""
    J, dims, truth = synth.closed_curve_image(size, seed=seed)
    J = f32(J)
    si, sl = synth.sample_seeds(truth, dims, per, 2, seed=seed)
    g = graph.build_graph(J, dims, beta)
    lam, Q = eig.smallest_eigpairs(g.Lhat, m)
    return dict(J=J, dims=dims, truth=truth, si=si, sl=sl, g=g, lam=lam, Q=f32(Q), beta=beta)


def gap_mask(U, thresh=1e-2):
    s = np.sort(U, axis=1)
    return (s[:, -1] - s[:, -2]) > thresh if U.shape[1] > 1 else np.ones(U.shape[0], bool)
