"""Writes tests/golden/c3_adjoint_grad.json: the FP64 oracle's exact-path gradient on the 128^3
volume (the 6-connected ellipsoid workload: beta = 90, gamma = 1e-3, 2 labels, 500 seeds per
label), for the GPU adjoint test.  Calls only oracle/ and synth/.

The loss is the squared error of the label-1 probabilities against the true mask over the
unseeded voxels; the gradient is taken through the normalized-form system of Eq. (rw_eq)
(Sec. II-C) with respect to every edge weight of Eq. (W) and to beta.  At this size the sparse
LU is out of reach, so the forward and adjoint systems are solved by FP64 conjugate gradients
to a relative residual of 1e-10.  Stored: the loss, d loss / d beta, the gradient on the 952
edges drawn from the 32^3 region of interest (1% of its internal edges), and two summaries
over all ROI-internal edges.  Takes several minutes:

    python tests/golden/make_c3_adjoint.py
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle import adjoint, exact, graph, priors  # noqa: E402

BETA, GAMMA, SEEDS = 90.0, 1e-3, 500
SEED = synth.BASE_SEED + 2
OUT = os.path.join(HERE, "c3_adjoint_grad.json")


def main():
    J, dims, truth = synth.ellipsoid_volume(128, seed=SEED)
    J = np.asarray(J, dtype=np.float32).astype(np.float64)
    si, sl = synth.sample_seeds(truth, dims, SEEDS, 2, seed=SEED)
    g = graph.build_graph(J, dims, BETA)
    P = priors.gaussian_priors(J, si, sl, 2)
    U = exact.exact_rw(g, si, sl, 2, P, GAMMA, method="cg", tol=1e-10)
    loss, G = adjoint.mask_loss(U, truth.astype(np.float64), si)
    gw, gb = adjoint.exact_grad(g, si, sl, 2, P, GAMMA, G, U=U, method="cg", tol=1e-10)
    center = synth.boundary_voxel(truth, dims, seed=SEED)
    lo, hi = synth.roi_box(center, 32, dims)
    roi = synth.roi_edge_ids(dims, lo, hi)
    ids = synth.pick_edges(roi, 0.01, seed=SEED)
    by_id = np.zeros(3 * g.N)
    by_id[g.ids] = gw
    w_by_id = g.weights_by_id()
    out = {
        "what": "FP64 oracle exact-path gradient, 128^3 ellipsoid, beta 90, gamma 1e-3, "
                "2 labels x 500 seeds, loss = sum over unseeded voxels (U[:,1] - mask)^2",
        "solver": "FP64 CG, relative residual 1e-10 (forward and adjoint)",
        "loss": loss,
        "dloss_dbeta": gb,
        "edge_ids": [int(e) for e in ids],
        "dloss_dw": [float(by_id[e]) for e in ids],
        "roi_lo": [int(v) for v in lo], "roi_hi": [int(v) for v in hi],
        "roi_sum_w_dloss_dw": float(np.sum(by_id[roi] * w_by_id[roi])),
        "roi_max_abs_dloss_dw": float(np.abs(by_id[roi]).max()),
    }
    with open(OUT, "w") as f:
        json.dump(out, f, indent=0)
    print(f"wrote {OUT}: loss {loss:.6e}, d/dbeta {gb:.6e}, {len(ids)} edges")


if __name__ == "__main__":
    main()
