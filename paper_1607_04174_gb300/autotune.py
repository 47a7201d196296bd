"""Launch-shape autotuner for the online solve's two 16-bit basis passes (the projection
Z = Q_n^T P-hat_n and the back-projection U-hat_n = Q_n C of Eq. U_lin_comb).

Their grids are the one free launch parameter of the solve that depends on the image size: a
128 x 128 image has 16k rows to split, a 512 x 512 one 262k.  For each size class this sweeps
the blocks per SM of both passes, times complete solves with CUDA events (L2 flushed before
each), and writes the fastest pair per class to a JSON table that `load_launch_shapes()`
installs through `rw_set_launch_shape`.  The inputs are synthetic (a smooth random image, a
random orthonormal basis of m columns, random seeds); the timing depends only on the sizes.

    python -m paper_1607_04174_gb300.autotune [--out FILE] [--m 100] [--labels 4]
"""
from __future__ import annotations

import argparse
import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_OUT = os.path.join(HERE, "launch_shapes.json")
SIDES = (128, 256, 384, 512)
PROJ = (1, 2, 3, 4)
BACK = (1, 2, 3, 4, 6)


def _problem(side, m, labels, seeds_per_label, rng, dev):
    import torch
    import paper_1607_04174_gb300 as rw
    N = side * side
    J = rng.random((side, side)).astype(np.float32)
    for _ in range(3):   # smooth it a little: neighbouring weights then vary like an image's
        J = 0.25 * (np.roll(J, 1, 0) + np.roll(J, -1, 0) + np.roll(J, 1, 1) + np.roll(J, -1, 1))
    g = rw.rw_build_graph(torch.from_numpy(J.ravel().copy()).to(dev), (side, side), 90.0)
    Q, _ = torch.linalg.qr(torch.randn(N, m, device=dev, dtype=torch.float32))
    lam = np.linspace(0.0, 1e-2, m)
    b = rw.rw_basis_create(g, Q.contiguous(), lam)
    idx = rng.choice(N, size=labels * seeds_per_label, replace=False).astype(np.int32)
    lab = np.repeat(np.arange(labels, dtype=np.int32), seeds_per_label)
    return g, b, torch.from_numpy(idx).to(dev), torch.from_numpy(lab).to(dev), N


def _time_solves(g, b, si, sl, labels, N, m, reps, dev):
    import torch
    import paper_1607_04174_gb300 as rw
    prob = torch.empty(N, labels, device=dev)
    flush = torch.empty(64 << 20, device=dev)
    for _ in range(3):
        rw.rw_solve(g, b, si, sl, labels, prob, m=m, want_info=False)
    st = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(reps)]
    for k, (a, z) in enumerate(ev):
        flush.fill_(float(k))
        a.record(st)
        rw.rw_solve(g, b, si, sl, labels, prob, m=m, want_info=False)
        z.record(st)
    torch.cuda.synchronize()
    return float(np.median([a.elapsed_time(z) for a, z in ev]))


def tune(out=DEFAULT_OUT, m=100, labels=4, seeds_per_label=100, reps=30, seed=7):
    import torch
    import paper_1607_04174_gb300 as rw
    from paper_1607_04174_gb300 import build
    build.build()
    dev = torch.device("cuda", torch.cuda.current_device())
    rng = np.random.default_rng(seed)
    entries, sweep = [], []
    for k, side in enumerate(SIDES):
        g, b, si, sl, N = _problem(side, m, labels, seeds_per_label, rng, dev)
        best = None
        try:
            for p in PROJ:
                for q in BACK:
                    rw.rw_set_launch_shape(0, 1, 1)
                    rw.rw_set_launch_shape(1 << 40, p, q)
                    ms = _time_solves(g, b, si, sl, labels, N, m, reps, dev)
                    sweep.append({"side": side, "proj_per_sm": p, "back_per_sm": q, "ms": ms})
                    if best is None or ms < best[2]:
                        best = (p, q, ms)
        finally:
            rw.rw_set_launch_shape(0, 1, 1)
            rw.rw_basis_free(b)
            rw.rw_graph_free(g)
        # the class covers sizes up to halfway (in N) to the next class
        n_max = (side * side + SIDES[k + 1] ** 2) // 2 if k + 1 < len(SIDES) else 1 << 40
        entries.append({"n_max": int(n_max), "side": side, "proj_per_sm": best[0],
                        "back_per_sm": best[1], "ms": best[2]})
    table = {"device": torch.cuda.get_device_name(dev), "m": m, "labels": labels,
             "seeds_per_label": seeds_per_label, "reps": reps, "entries": entries,
             "sweep": sweep}
    with open(out, "w") as f:
        json.dump(table, f, indent=1)
    return table


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=DEFAULT_OUT)
    ap.add_argument("--m", type=int, default=100)
    ap.add_argument("--labels", type=int, default=4)
    ap.add_argument("--reps", type=int, default=30)
    a = ap.parse_args()
    t = tune(a.out, a.m, a.labels, reps=a.reps)
    for e in t["entries"]:
        print(e)


if __name__ == "__main__":
    main()
