#!/usr/bin/env python
"""Benchmark of the GPU Greedy Frank-Wolfe path: FW iterations per second.

One step = one full solve (reset to U_0, then `iters` GFW iterations) of the
200,000-node stochastic-block-model workload (K = 10, FP32 weights and iterate,
eps = 50, omega_0 = 1000), with the graph resident in HBM.  Under torchrun each
rank solves its own replica (weak scaling, no data-path collective).

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle on
the host cores on the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2508_09738_gb300 import workloads as W  # noqa: E402

METRIC = "FW iters/s"
L2_FLUSH_BYTES = 256 << 20


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="sbm200k")
    p.add_argument("--iters", type=int, default=0, help="iterations per solve (default: config)")
    p.add_argument("--iters-per-launch", type=int, default=0)
    p.add_argument("--lanes", type=int, default=0)
    p.add_argument("--weights", default="")
    p.add_argument("--profile-iters", type=int, default=100)
    p.add_argument("--cpu-iters", type=int, default=0, help="oracle iterations in the CPU sample")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    return p.parse_args()


# ------------------------------------------------------------------ clocks --
class ClockSampler:
    """nvidia-smi samples (200 ms) during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------- byte counting --
def bytes_per_unit(n, nnz, K, wbytes, tbytes=4):
    """Algorithmic bytes of one FW iteration and of each pass."""
    row_pass = 5 * tbytes * n * K + 3 * n                 # U, LU, LS in; U, LU out; choice, fid
    csr_pass = (2 * tbytes * n * K + (4 + wbytes) * nnz   # U in, LS out; col + weights
                + 4 * (n + 1) + 2 * n)                    # row_ptr; choice of the row + gathers
    iteration = 4 * tbytes * n * K + (4 + wbytes) * nnz + 4 * n + 3 * n
    return dict(row_pass=row_pass, csr_pass=csr_pass, iteration=iteration)


def source_hash() -> str:
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2508_09738_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        if f.endswith((".cu", ".cuh", ".h")):
            h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def load_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": d.get("hbm_gbs"), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


def ncu_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if still current."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p))
        e = d.get(workload, {}).get(kernel)
        if e and e.get("source_hash") == source_hash():
            return e.get("dram_bytes_per_launch")
    except Exception:
        return None
    return None


# ---------------------------------------------------------------- oracle --
def cpu_oracle_rate(g, c, iters):
    """Oracle iterations/s on a bounded sample: `iters` GFW iterations from U_0."""
    import oracle as O
    P = O.make_problem(g, c["eps"], c["omega0"], c["weights"])
    t = time.perf_counter()
    U, info = O.gfw_solve(P, max_iters=iters)
    dt = time.perf_counter() - t
    return info["iters"] / dt, dt, info["iters"]


def run_reference(args, c, rank):
    if rank != 0:
        return
    g = W.make_config_graph(args.workload)
    iters = args.cpu_iters or max(2, int(20 * 200_000 / g.n))
    for _ in range(args.warmup):
        cpu_oracle_rate(g, c, iters)
    total, done = 0.0, 0
    for _ in range(args.steps):
        _, dt, it = cpu_oracle_rate(g, c, iters)
        total += dt
        done += it
    v = done / total
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "iter/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_dict(args, c, g, iters),
        "cpu_baseline": {"value": v, "unit": "iter/s", "cores": 1, "kind": "oracle",
                         "sample": f"{iters} GFW iterations from U_0 per step (numpy/scipy FP64, "
                                   f"one thread)"},
        "e2e": {"value": v, "unit": "iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def config_dict(args, c, g, iters):
    return {"workload": args.workload, "n": g.n, "nnz": g.nnz, "K": g.K,
            "iters_per_solve": iters, "weights": args.weights or c["weights"],
            "eps": c["eps"], "omega0": c["omega0"],
            "l2": "256 MiB buffer written between timed steps",
            "parallelism": f"replicas x{args.gpus}"}


# ----------------------------------------------------------- multi-rank --
def max_over_ranks(x: float, device: str) -> float:
    """Max of a per-rank scalar over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, seconds_local: float, world: int, device: str) -> tuple:
    """(rate, seconds): units of all ranks / the slowest rank's time (weak scaling)."""
    sec = max_over_ranks(seconds_local, device)
    return world * units_per_rank / sec, sec


# ------------------------------------------------------------------ ours --
def main():
    args = parse()
    c = W.CONFIGS[args.workload]
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, c, rank)
        return

    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    from paper_2508_09738_gb300 import build as Bld
    if rank == 0:
        Bld.build()
    if world > 1:
        dist.barrier()
    from paper_2508_09738_gb300 import binding as B

    weights = args.weights or c["weights"]
    iters = args.iters or c["iters"]
    g = W.make_config_graph(args.workload)
    stream = torch.cuda.Stream()          # one stream for flush, events and solver
    torch.cuda.set_stream(stream)
    ipl = args.iters_per_launch or iters
    opts = dict(eps=c["eps"], omega0=c["omega0"], weight_dtype=weights, max_iters=iters,
                iters_per_launch=ipl, lanes_per_row=args.lanes, cuda_stream=stream.cuda_stream)
    seg = B.Segmenter(g, **opts)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    for _ in range(args.warmup):
        flush.zero_()
        seg.reset()
        seg.solve()
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches = 0
    stats = None
    for s in range(args.steps):
        flush.zero_()
        ev[s][0].record(stream)
        seg.reset()
        stats = seg.solve()
        ev[s][1].record(stream)
        launches += stats.launches + 4     # reset: reinit, spmm, spmm, objective
    torch.cuda.synchronize()
    clk = clocks.stop()
    t_ms = sum(a.elapsed_time(b) for a, b in ev)
    value, t_s = whole_job_rate(args.steps * stats.iters, t_ms / 1000.0, world, "cuda")
    t_ms = 1000.0 * t_s
    if world > 1:
        dist.barrier()
    labels = seg.labels()
    solves = world * args.steps / t_s

    # per-pass device times (CUDA events on the solver's stream) -> roofline
    seg.reset()
    ms_a, ms_b = seg.profile(min(args.profile_iters, iters))
    wb = {"f32": 4, "bf16": 2, "f64": 8}[weights]
    tb = 8 if weights == "f64" else 4
    by = bytes_per_unit(g.n, g.nnz, g.K, wb, tb)
    dom = "csr_pass" if ms_b >= ms_a else "row_pass"
    dom_ms = max(ms_a, ms_b)
    peaks = load_peaks()
    achieved = by[dom] / (dom_ms / 1000.0) / 1e9
    kernel_name = {"csr_pass": "k_passB", "row_pass": "k_passA"}[dom]
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"],
                "traffic": ncu_traffic(kernel_name, args.workload),
                "kernel": kernel_name, "peak_source": peaks["source"],
                "algorithmic_bytes_per_launch": by[dom],
                "kernel_ms": {"k_passA": ms_a, "k_passB": ms_b}}
    seg.close()

    # end to end through the C ABI from pinned host buffers
    e2e = None
    if not args.no_e2e:
        def pinned(a):
            t = torch.empty(a.shape, dtype=getattr(torch, str(a.dtype)), pin_memory=True)
            t.numpy()[...] = a
            return t
        rp, col, w, lab = (pinned(g.row_ptr), pinned(g.col), pinned(g.w), pinned(g.labels))
        out = torch.empty(g.n, dtype=torch.int32, pin_memory=True)
        o = B.fw_seg_default_opts(**opts)
        steps_e2e = max(1, min(args.steps, 3))
        h = B.fw_seg_create(g.n, rp.numpy(), col.numpy(), w.numpy(), g.K, lab.numpy(), o)
        B.fw_seg_solve(h)
        B.fw_seg_destroy(h)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        it_e2e = 0
        for _ in range(steps_e2e):
            h = B.fw_seg_create(g.n, rp.numpy(), col.numpy(), w.numpy(), g.K, lab.numpy(), o)
            st = B.fw_seg_solve(h)
            B.fw_seg_labels(h, out.numpy())
            B.fw_seg_destroy(h)
            it_e2e += st.iters
        dt = time.perf_counter() - t0
        e2e_rate, dt = whole_job_rate(it_e2e, dt, world, "cuda")
        e2e = {"value": e2e_rate, "unit": "iter/s",
               "h2d_bytes_per_step": int(4 * (g.n + 1) + 12 * g.nnz + 4 * g.n),
               "d2h_bytes_per_step": int(4 * g.n),
               "steps": steps_e2e, "includes": "create (H2D, validation, Laplacian assembly, "
                                                "L U_0), solve, labels D2H, destroy"}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    line = {
        "metric": METRIC, "value": value, "unit": "iter/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if weights == "f64" else "f32", "data": "synthetic",
        "config": config_dict(args, c, g, iters),
        "solves_per_s": solves,
        "effective_gbs": by["iteration"] * value / world / 1e9,
        "clocks": clk, "e2e": e2e, "gpu_launches": launches, "roofline": roofline,
    }
    gold = os.path.join(ROOT, "tests", "golden", f"{args.workload}_oracle{iters}.npz")
    if os.path.exists(gold) and weights == c["weights"]:
        ref = np.load(gold)
        line["label_agreement"] = float(np.mean(labels == ref["labels"]))
    if not args.no_cpu_baseline and world == 1:
        ci = args.cpu_iters or max(2, int(40 * 200_000 / g.n))
        v, dt, it = cpu_oracle_rate(g, c, ci)
        line["cpu_baseline"] = {"value": v, "unit": "iter/s", "cores": 1, "kind": "oracle",
                                "sample": f"{it} GFW iterations from U_0 on the same graph "
                                          f"(numpy/scipy FP64, one thread), {dt:.1f} s"}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
