"""Benchmark: online random-walker label maps per second on one GB300.

Workload (the paper's RWIS online step, Sec. II-B / III-A, on a synthetic stand-in for its 2-D
data): a 512 x 512 image of 4 Voronoi regions (means U(0,1), noise 0.05, 4-connected graph,
beta = 90, normalized Laplacian), a basis of 200 eigenvectors precomputed offline by the
library's LOBPCG, and per step one complete `rw_solve`: 4 labels, 200 fresh seeds per label,
Gaussian-fit priors, gamma = 1e-3, m chosen adaptively (<= 200, eps = 0.1), 3 damped-Jacobi
refinement steps, probabilities plus the hard label map.  A step is one label map.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs N independent replicas (one per GPU, launched by torch.distributed.run); the value
is the label maps of all ranks divided by the slowest rank's time ("scaling": "weak").
`--impl reference` times the FP64 oracle (the paper's method restated on the CPU) on the same
workload, on rank 0 only.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

SIZE = 512
LABELS = 4
SEEDS_PER_LABEL = 200
BETA = 90.0
GAMMA = 1e-3
M = 200
EPS = 0.1
M_STEP = 10
REFINE = 3
METRIC = "online RW label maps/s at 512² & 128³ vs plain PCG on GPU, ≤1e-3 prob err"
WORKLOAD = "rwis-512x512-4label-voronoi"
L2_FLUSH_BYTES = 256 << 20


def seed_sets(truth, dims, count, base):
    return [synth.sample_seeds(truth, dims, SEEDS_PER_LABEL, 3, seed=base + 7919 * (k + 1))
            for k in range(count)]


# ----------------------------------------------------------------------------- clocks


class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- oracle arms


def oracle_problem():
    from oracle import graph, update
    J, dims, truth = synth.voronoi_image(SIZE, SIZE, seed=synth.BASE_SEED + 1)
    J = J.astype(np.float32).astype(np.float64)
    g = graph.build_graph(J, dims, BETA)
    # the oracle's eigensolver is offline-only at this size; its online solve is timed on a
    # generic orthonormal basis of the same shape (DCT columns, Rayleigh-quotient values)
    Q = synth.dct_basis(dims, M)
    lam = update.rayleigh_quotients(Q, g.Lhat)
    return J, dims, truth, g, Q, lam


def time_oracle(n_solves, budget_s=25.0):
    from oracle import pipeline
    J, dims, truth, g, Q, lam = oracle_problem()
    sets = seed_sets(truth, dims, n_solves, synth.BASE_SEED + 101)
    times = []
    t_start = time.perf_counter()
    for si, sl in sets:
        t0 = time.perf_counter()
        pipeline.online_solve(g, Q, lam, si, sl, LABELS, gamma=GAMMA, m=0, m_step=M_STEP,
                              eps=EPS, refine_steps=REFINE)
        times.append(time.perf_counter() - t0)
        if time.perf_counter() - t_start > budget_s:
            break
    return times


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def reference_arm(args):
    """--impl reference: the FP64 oracle (NumPy/SciPy on the host cores) as the reference."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    for _ in range(max(0, min(args.warmup, 1))):
        time_oracle(1)
    times = time_oracle(args.steps, budget_s=240.0)
    ms = 1000.0 * float(np.mean(times))
    value = 1000.0 / ms
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "label_maps/s",
        "n_gpus": args.gpus, "steps": len(times), "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "size": [SIZE, SIZE], "labels": LABELS,
                   "seeds_per_label": SEEDS_PER_LABEL, "m_max": M, "refine_steps": REFINE,
                   "basis": "DCT columns with Rayleigh-quotient values (oracle eigensolver is "
                            "offline-only at this size)"},
        "cpu_baseline": {"value": value, "unit": "label_maps/s", "cores": cpu_cores(),
                         "kind": "oracle",
                         "sample": f"{len(times)} full 512x512 online solves"},
        "e2e": {"value": value, "unit": "label_maps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------------------- GPU arm


def algorithmic_bytes(phase, N, m, lp, steps):
    """Bytes each phase must move at minimum (per launch), for the roofline."""
    if phase == "project":   # 16-bit basis rows (m cols) + hat priors + seed labels
        return N * (2 * m + 4 * lp + 4)
    if phase == "back":      # basis rows again + write U-hat (lp) + seed labels + d^{1/2}
        return N * (2 * m + 4 * lp + 4 + 4)
    if phase == "refine":    # per step: read x, p-hat, labels, coefficients; write x
        return steps * N * (4 * lp * 2 + 4 * lp + 4 + 4 * 2 + 4 * 2) + N * (4 * LABELS + 1)
    return None


def gpu_arm(args):
    import torch
    import torch.distributed as dist

    import paper_1607_04174_gb300 as rw
    from paper_1607_04174_gb300 import build

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    peaks = {}
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        with open(pk) as f:
            peaks = json.load(f)

    J, dims, truth = synth.voronoi_image(SIZE, SIZE, seed=synth.BASE_SEED + 1)
    N = SIZE * SIZE
    J32 = torch.from_numpy(J.astype(np.float32)).to(dev)
    g = rw.rw_build_graph(J32, dims, BETA)
    t0 = time.perf_counter()
    b, eig_info = rw.rw_precompute(g, M, tol=1e-5, seed=1)
    torch.cuda.synchronize()
    precompute_s = time.perf_counter() - t0

    sets = seed_sets(truth, dims, args.warmup + args.steps, synth.BASE_SEED + 17 + 1000 * rank)
    dsets = [(torch.from_numpy(si).to(dev), torch.from_numpy(sl).to(dev)) for si, sl in sets]
    prob = torch.empty(N, LABELS, device=dev)
    labels = torch.empty(N, dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, device=dev)
    stream = torch.cuda.current_stream()
    kw = dict(gamma=GAMMA, m=0, m_step=M_STEP, eps=EPS, refine_steps=REFINE)

    for si, sl in dsets[:args.warmup]:
        rw.rw_solve(g, b, si, sl, LABELS, prob, labels, **kw)
    torch.cuda.synchronize()

    # timed region: K steps, L2 flushed (a 256 MB write) before each, CUDA events per step
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    infos = []
    sampler = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    launches0 = rw.rw_kernel_launches()
    wall0 = time.perf_counter()
    for k, (si, sl) in enumerate(dsets[args.warmup:]):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        torch.cuda.nvtx.range_push("rw_solve")
        _, info = rw.rw_solve(g, b, si, sl, LABELS, prob, labels, record_phases=True, **kw)
        torch.cuda.nvtx.range_pop()
        ev[k][1].record(stream)
        infos.append(info)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    launches = rw.rw_kernel_launches() - launches0
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    step_ms = np.array([a.elapsed_time(z) for a, z in ev])
    ms = float(step_ms.mean())
    if world > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * 1000.0 / ms

    # per-phase device times (events recorded by the library on this stream, same steps)
    phases = {p: float(np.mean([i["phase_ms"][p] for i in infos])) for p in rw.RW_PHASES}
    m_used = [i["m_used"] for i in infos]
    m_mean = float(np.mean(m_used))
    lp = 4
    hbm = peaks.get("hbm_gbs")
    dom = max(("project", "back", "refine"), key=lambda p: phases[p])
    top = max(phases, key=lambda p: phases[p])
    abytes = algorithmic_bytes(dom, N, m_mean, lp, REFINE)
    achieved = abytes / (phases[dom] * 1e-3) / 1e9
    roofline = {"kernel": {"project": "k_project", "back": "k_backproject",
                           "refine": "k_jacobi_step"}[dom],
                "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm if hbm else None, "traffic": None,
                "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if hbm else "fallback 6800",
                "phase_ms": phases, "largest_phase": top}
    if not hbm:
        roofline["peak"] = 6800.0
        roofline["frac"] = achieved / 6800.0

    if args.no_competitor:
        print(json.dumps({"metric": METRIC, "value": value, "unit": "label_maps/s",
                          "ms_per_step": ms, "phase_ms": phases, "m_used_mean": m_mean,
                          "partial": "profiling run (--no-competitor)"}))
        return 0
    # end to end: host seeds in (pinned), probabilities + labels out, through rw_solve_host
    hs = [(torch.from_numpy(si).pin_memory(), torch.from_numpy(sl).pin_memory())
          for si, sl in sets[args.warmup:]]
    hprob = torch.empty(N, LABELS).pin_memory()
    hlab = torch.empty(N, dtype=torch.uint8).pin_memory()
    e2e_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in hs]
    rw.rw_solve_host(g, b, hs[0][0].numpy(), hs[0][1].numpy(), LABELS, hprob.numpy(),
                     hlab.numpy(), **kw)
    for k, (si, sl) in enumerate(hs):
        flush.fill_(float(k))
        e2e_ev[k][0].record(stream)
        rw.rw_solve_host(g, b, si.numpy(), sl.numpy(), LABELS, hprob.numpy(), hlab.numpy(), **kw)
        e2e_ev[k][1].record(stream)
    torch.cuda.synchronize()
    e2e_ms = float(np.mean([a.elapsed_time(z) for a, z in e2e_ev]))

    # GPU comparison solver: Jacobi-PCG from zero (basic RW, Eq. rw_eq) at the iteration count
    # that reaches 1e-3 max-abs against its own converged solution (calibrated untimed)
    si0, sl0 = dsets[args.warmup]
    conv = torch.empty(N, LABELS, device=dev)
    it_conv = rw.rw_solve_pcg(g, si0, sl0, LABELS, conv, gamma=GAMMA, iters=50000, tol=1e-7)
    lo, hi = 1, it_conv
    tmp = torch.empty(N, LABELS, device=dev)
    while lo < hi:
        mid = (lo + hi) // 2
        rw.rw_solve_pcg(g, si0, sl0, LABELS, tmp, gamma=GAMMA, iters=mid)
        if float((tmp - conv).abs().max()) <= 1e-3:
            hi = mid
        else:
            lo = mid + 1
    pcg_iters = lo
    pev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(min(args.steps, 10))]
    for k, (a, z) in enumerate(pev):
        si, sl = dsets[args.warmup + k]
        flush.fill_(float(k))
        a.record(stream)
        rw.rw_solve_pcg(g, si, sl, LABELS, tmp, labels, gamma=GAMMA, iters=pcg_iters,
                        want_iters=False)
        z.record(stream)
    torch.cuda.synchronize()
    pcg_ms = float(np.mean([a.elapsed_time(z) for a, z in pev]))
    # accuracy of the fast path against the converged basic RW on the same seeds
    rw.rw_solve(g, b, si0, sl0, LABELS, prob, labels, **kw)
    fast_vs_exact = float((prob - conv).abs().max())

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        times = time_oracle(20, budget_s=25.0)
        cpu = {"value": 1000.0 / (1000.0 * float(np.mean(times))), "unit": "label_maps/s",
               "cores": cpu_cores(), "kind": "oracle",
               "sample": f"{len(times)} full 512x512 online solves of the FP64 oracle (DCT basis "
                         f"of the same shape; adaptive m, 3 refinement steps)"}

    line = {
        "metric": METRIC, "value": value, "unit": "label_maps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "size": [SIZE, SIZE], "labels": LABELS,
                   "seeds_per_label": SEEDS_PER_LABEL, "m_max": M, "eps": EPS,
                   "refine_steps": REFINE, "basis_format": "f16-scaled",
                   "l2": "flushed (256 MB write) before every timed step",
                   "parallelism": f"replicas x{world}"},
        "p50_ms": float(np.percentile(step_ms, 50)), "p99_ms": float(np.percentile(step_ms, 99)),
        "wall_s": wall, "m_used_mean": m_mean,
        "roofline": roofline, "cpu_baseline": cpu,
        "e2e": {"value": world * 1000.0 / e2e_ms, "unit": "label_maps/s",
                "h2d_bytes_per_step": int(sets[0][0].nbytes + sets[0][1].nbytes),
                "d2h_bytes_per_step": int(N * LABELS * 4 + N)},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "pcg_competitor": {"iters_to_1e-3": pcg_iters, "iters_converged_1e-7": it_conv,
                           "ms_per_step": pcg_ms, "label_maps_per_s": 1000.0 / pcg_ms},
        "fast_vs_exact_maxabs": fast_vs_exact,
        "precompute": {"seconds": precompute_s, **eig_info},
    }
    rw.rw_basis_free(b)
    rw.rw_graph_free(g)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-competitor", action="store_true",
                    help="skip the e2e, PCG and CPU legs (profiling runs)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return reference_arm(args)
    return gpu_arm(args)


if __name__ == "__main__":
    sys.exit(main())
