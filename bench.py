#!/usr/bin/env python
"""Benchmark of the GPU Greedy Frank-Wolfe path: FW iterations per second.

Default workload: the 2048 x 2048 noisy Voronoi image (n = 4,194,304 pixels,
8-neighbour graph, 33,529,860 stored entries, K = 4, eps = 50, omega_0 = 1e5,
200 GFW iterations per solve), the largest single-GPU configuration.  One step
= one full solve (reset to U_0, then the iterations) with the graph resident
in HBM.  The line's headline numbers are for FP32 weights; the same run times
BF16 weights as a second record.  Under torchrun each rank solves its own
replica (weak scaling, no data-path collective).

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle on
the host cores on the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
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
GOLDEN = os.path.join(ROOT, "tests", "golden")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="voronoi2048")
    p.add_argument("--iters", type=int, default=0, help="iterations per solve (default: config)")
    p.add_argument("--iters-per-launch", type=int, default=0)
    p.add_argument("--lanes", type=int, default=0)
    p.add_argument("--class-table", default="auto", choices=["auto", "off", "on"],
                   help="pass-B form: class table in shared memory (auto: where it pays)")
    p.add_argument("--weights", default="", help="one weight dtype instead of the config's arms")
    p.add_argument("--profile-iters", type=int, default=100)
    p.add_argument("--cpu-seconds", type=float, default=15.0,
                   help="target length of each CPU-oracle sample")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-trajectory", action="store_true")
    p.add_argument("--problems", type=int, default=256, help="batched: number of problems")
    p.add_argument("--no-extras", action="store_true",
                   help="single-problem workloads: skip the batched and serving sub-records")
    return p.parse_args()


# ------------------------------------------------------------------ clocks --
class ClockSampler:
    """nvidia-smi samples (200 ms) during the timed regions: start() / stop()
    around each timed region, summary() over all of them."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None
        self.rows = []
        self.failed = False

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
            self.failed = True

    def stop(self):
        if self.proc is None:
            return
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                self.rows.append(f)
        os.unlink(self.path)
        self.proc = None

    def summary(self) -> dict:
        if self.failed and not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = self.rows
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------- byte counting --
def column_bytes(g) -> int:
    """Bytes per stored column index: the library keeps 16-bit offsets j - i
    when every |j - i| < 2^15 (banded graphs such as pixel grids)."""
    rows = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.row_ptr))
    far = g.nnz and int(np.max(np.abs(g.col.astype(np.int64) - rows))) >= 32768
    return 4 if far else 2


def bytes_per_unit(n, nnz, K, wbytes, tbytes=4, cbytes=4):
    """Algorithmic bytes of one FW iteration (the method's minimum: U and L U
    read and written, the CSR once, row_ptr, choice and fidelity bytes) and of
    each pass of the two-pass design (pass A: U, L U, L S in, U, L U out;
    pass B: U in for the moved rows, L S out, the CSR, row_ptr, the row's own
    choice and the gathered neighbour classes)."""
    row_pass = 5 * tbytes * n * K + 3 * n                 # U, LU, LS in; U, LU out; choice, fid
    csr_pass = (2 * tbytes * n * K + (cbytes + wbytes) * nnz   # U in, LS out; col + weights
                + 4 * (n + 1) + 2 * n)                    # row_ptr; choice of the row + gathers
    iteration = 4 * tbytes * n * K + (4 + wbytes) * nnz + 4 * n + 3 * n
    return dict(row_pass=row_pass, csr_pass=csr_pass, iteration=iteration)


# the sources that define and instantiate the profiled kernels (pass A,
# pass B, finish, one-shot); host-only set-up and driver code is not included
KERNEL_SOURCES = ("fw_types.h", "fw_device.cuh", "fw_kernels.cuh", "fw_ops.cuh",
                  "fw_ops_f32.cu", "fw_ops_bf16.cu", "fw_ops_f64.cu")


def source_hash() -> str:
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2508_09738_gb300", "csrc")
    for f in KERNEL_SOURCES:
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
def cpu_model() -> str:
    """The host CPU's model name (/proc/cpuinfo, else lscpu)."""
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.processor() or platform.machine()


def _oracle_problem(g, c, weights):
    import oracle as O
    return O.make_problem(g, c["eps"], c["omega0"], weights)


def oracle_sample_iters(g, c, weights, seconds):
    """Iterations of an oracle sample that take about `seconds` on one core
    (from the time of one GFW iteration at U_0)."""
    import oracle as O
    P = _oracle_problem(g, c, weights)
    t = time.perf_counter()
    O.gfw_iteration(P.Uhat, P)
    dt = time.perf_counter() - t
    return int(min(500, max(2, round(seconds / max(dt, 1e-6))))), dt


def cpu_oracle_rate(g, c, weights, iters):
    """Oracle iterations/s on one thread: `iters` GFW iterations from U_0."""
    import oracle as O
    P = _oracle_problem(g, c, weights)
    t = time.perf_counter()
    U, info = O.gfw_solve(P, max_iters=iters)
    dt = time.perf_counter() - t
    return info["iters"] / dt, dt, info["iters"]


def _oracle_replica(path, c, weights, iters, steps, barrier, q):
    """One replica process of the oracle: load the graph, build the problem
    (not timed), then per step wait for the other replicas and time `iters`
    GFW iterations from U_0."""
    import oracle as O
    d = np.load(path)
    g = W.Graph(int(d["n"]), d["row_ptr"], d["col"], d["w"], int(d["K"]), d["labels"],
                d["labels"])
    P = O.make_problem(g, c["eps"], c["omega0"], weights)
    for _ in range(steps):
        barrier.wait()
        t = time.perf_counter()
        _, info = O.gfw_solve(P, max_iters=iters)
        q.put((info["iters"], time.perf_counter() - t))


def cpu_oracle_replicas(g, c, weights, iters, procs, steps=1):
    """The oracle as it stands on `procs` host cores: `procs` spawned
    processes, each solving its own copy of the problem (the oracle itself
    is single-threaded).  Returns per step (iterations of all replicas, the
    slowest replica's seconds)."""
    import multiprocessing as mp
    env = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS",
                                          "MKL_NUM_THREADS")}
    for k in env:
        os.environ[k] = "1"
    fd, path = tempfile.mkstemp(suffix=".npz")
    os.close(fd)
    try:
        np.savez(path, n=g.n, K=g.K, row_ptr=g.row_ptr, col=g.col, w=g.w, labels=g.labels)
        ctx = mp.get_context("spawn")
        barrier = ctx.Barrier(procs)
        q = ctx.Queue()
        ps = [ctx.Process(target=_oracle_replica, args=(path, c, weights, iters, steps, barrier, q))
              for _ in range(procs)]
        for p_ in ps:
            p_.start()
        out = []
        for _ in range(steps):
            res = [q.get(timeout=3600) for _ in range(procs)]
            out.append((sum(r[0] for r in res), max(r[1] for r in res)))
        for p_ in ps:
            p_.join(timeout=600)
        return out
    finally:
        os.unlink(path)
        for k, v in env.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def cpu_baseline(g, c, weights, seconds):
    """The oracle timed on one thread and on every host core (replicas)."""
    iters, t1 = oracle_sample_iters(g, c, weights, seconds)
    v1, dt1, it1 = cpu_oracle_rate(g, c, weights, iters)
    T = os.cpu_count() or 1
    (tot, dtT), = cpu_oracle_replicas(g, c, weights, iters, T)
    vT = tot / dtT
    return {"value": vT, "unit": "iter/s", "cores": T, "kind": "oracle",
            "cpu_model": cpu_model(),
            "sample": f"{T} processes, each running the first {iters} GFW iterations from U_0 "
                      f"of its own copy of this workload (numpy/scipy FP64, "
                      f"{weights}-rounded weights), {dtT:.1f} s; one process alone: "
                      f"{it1} iterations in {dt1:.1f} s",
            "single_thread": {"value": v1, "unit": "iter/s", "cores": 1, "seconds": dt1,
                              "iterations": it1}}


def run_reference(args, c, rank):
    """The reference arm: the FP64 oracle as it stands on every host core (one
    replica process per core), each step a bounded sample of the workload."""
    if rank != 0:
        return
    g = W.make_config_graph(args.workload)
    weights = args.weights or c["weights"]
    per_step = max(1.0, 120.0 / max(1, args.steps + args.warmup))
    iters, _ = oracle_sample_iters(g, c, weights, per_step)
    T = os.cpu_count() or 1
    res = cpu_oracle_replicas(g, c, weights, iters, T, steps=args.warmup + args.steps)
    timed = res[args.warmup:]
    total = sum(dt for _, dt in timed)
    done = sum(it for it, _ in timed)
    v = done / total
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "iter/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_dict(args, c, g, args.iters or c["iters"], weights),
        "cpu_baseline": {"value": v, "unit": "iter/s", "cores": T, "kind": "oracle",
                         "cpu_model": cpu_model(),
                         "sample": f"each step: {T} processes, each running the first {iters} GFW "
                                   f"iterations from U_0 of its own copy of the workload "
                                   f"(numpy/scipy FP64, {weights}-rounded weights)"},
        "e2e": {"value": v, "unit": "iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def config_dict(args, c, g, iters, weights):
    wb = {"f32": 4, "bf16": 2, "f64": 8}[weights]
    return {"workload": args.workload, "n": g.n, "nnz": g.nnz, "K": g.K,
            "iters_per_solve": iters, "weights": weights,
            "eps": c["eps"], "omega0": c["omega0"],
            "l2": "256 MiB buffer written between timed steps; CSR %.0f MB" %
                  ((4 + wb) * g.nnz / 1e6),
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


# --------------------------------------------------------------- batched --
def run_batched(args, rank, world, local, emit=True):
    """256 uneven blob problems in one persistent launch vs 256 sequential
    solves; prints the JSON line (emit) and returns it."""
    import torch
    from paper_2508_09738_gb300 import binding as B
    from paper_2508_09738_gb300 import build as Bld
    torch.cuda.set_device(local)
    Bld.build()
    P = args.problems
    t0 = time.time()
    gs = W.batched_blobs(P=P, n_min=1000, n_max=200_000, K_min=3, K_max=10, label_frac=0.02,
                         seed=W.SEED0 + 3, device="cuda")
    gen_s = time.time() - t0
    iters = args.iters or 200
    weights = args.weights or "bf16"
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    opts = B.fw_seg_default_opts(max_iters=iters, weight_dtype=weights, lanes_per_row=args.lanes)
    cache = os.environ.get("FW_TUNE_CACHE") or os.path.join(tempfile.gettempdir(), "fwseg_tune.txt")
    t0 = time.time()
    bt = B.Batch(gs, opts, weight_dtype=weights, cuda_stream=stream.cuda_stream, tune_cache=cache)
    create_s = time.time() - t0
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def timed(fn, steps):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        out = None
        for s_ in range(steps):
            flush.zero_()
            ev[s_][0].record(stream)
            out = fn()
            ev[s_][1].record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in ev) / 1000.0, out

    def batched_step():
        bt.reset()
        return bt.solve()

    for _ in range(args.warmup):
        batched_step()
    torch.cuda.synchronize()
    info = bt.info().as_dict()         # after solves: the launch as it ran
    clocks = ClockSampler(local)
    clocks.start()
    t_b, stats = timed(batched_step, args.steps)
    clocks.stop()
    clk = clocks.summary()
    total_iters = sum(s_.iters for s_ in stats)
    # the plain one-problem-at-a-time path on the same problems, resident on the device
    segs = [B.Segmenter(g, max_iters=iters, weight_dtype=weights, iters_per_launch=iters,
                        lanes_per_row=info["lanes_per_row"], cuda_stream=stream.cuda_stream)
            for g in gs]

    def sequential_step():
        it = 0
        for sg in segs:
            sg.reset()
            it += sg.solve().iters
        return it

    sequential_step()
    steps_seq = max(1, min(args.steps, 2))
    t_s, it_seq = timed(sequential_step, steps_seq)
    same = all(np.array_equal(bt.labels(p), segs[p].labels()) for p in range(P))
    for sg in segs:
        sg.close()
    # the FP64 oracle on the same rounded weights, for the smallest problems
    sample = []
    if not args.no_cpu_baseline:
        import oracle as O
        for p in sorted(range(P), key=lambda q: gs[q].n)[:4]:
            Pp = O.make_problem(gs[p], 50.0, 1000.0, weights)
            Uo, _ = O.gfw_solve(Pp, max_iters=iters)
            Eo = O.energy(Uo, Pp)
            sample.append({"problem": p, "n": gs[p].n, "K": gs[p].K,
                           "label_agreement": float(np.mean(bt.labels(p) ==
                                                            O.labels_from_U(Uo))),
                           "objective_rel_err": rel(O.energy(bt.U(p), Pp), Eo)})
    wb = {"f32": 4, "bf16": 2, "f64": 8}[weights]
    byt = sum(bytes_per_unit(g.n, g.nnz, g.K, wb)["iteration"] * st.iters
              for g, st in zip(gs, stats))
    peaks = load_peaks()
    achieved = byt * args.steps / t_b / 1e9
    line = {
        "metric": "FW iters/s", "value": total_iters * args.steps / t_b, "unit": "iter/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * t_b / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "batched256" if P == 256 else f"batched{P}", "problems": P, "rows": sum(g.n for g in gs),
                   "nnz": sum(g.nnz for g in gs), "K": "3..10", "iters_per_solve": iters,
                   "weights": weights, "eps": 50.0, "omega0": 1000.0,
                   "l2": "256 MiB buffer written between timed steps"},
        "solves_per_s": P * args.steps / t_b,
        "sequential_plain": {"iters_per_s": it_seq * steps_seq / t_s,
                             "solves_per_s": P * steps_seq / t_s,
                             "ms_per_step": 1000 * t_s / steps_seq},
        "speedup_vs_sequential": (P * args.steps / t_b) / (P * steps_seq / t_s),
        "labels_equal_to_single": same, "batch_info": info, "clocks": clk,
        "oracle_sample": sample,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
                     "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "traffic": None,
                     "kernel": ("k_itemA + k_itemB" if info.get("schedule") == 3 else "k_persistent"),
                     "peak_source": peaks["source"],
                     "algorithmic_bytes": "sum over problems of iteration bytes x iterations; "
                                          "whole solves timed (all of the batch's kernels)"},
        "setup_s": {"generate": gen_s, "create_and_tune": create_s},
    }
    bt.close()
    if rank == 0 and emit:
        print(json.dumps(line), flush=True)
    return line


# --------------------------------------------------------------- serving --
def run_serving(args, rank, world, local, emit=True):
    """Poisson requests at swept rates: continuous batching vs sequential
    solves; prints the JSON line (emit) and returns it."""
    import torch
    from paper_2508_09738_gb300 import binding as B
    from paper_2508_09738_gb300 import build as Bld
    torch.cuda.set_device(local)
    Bld.build()
    rng = np.random.default_rng(W.SEED0 + 4)
    pool = []
    t0 = time.time()
    for i in range(12):
        n = int(round(np.exp(rng.uniform(np.log(1e3), np.log(2e5)))))
        K = int(rng.integers(3, 9))
        g = W.blobs_knn(n=max(n, 4 * K), K=K, label_frac=0.02, seed=W.SEED0 + 400 + i,
                        device="cuda")
        pool.append((g, dict(eps=50.0, omega0=1000.0)))
    for i in range(12):
        side = int(rng.choice([256, 512, 768, 1024]))
        K = int(rng.integers(3, 9))
        g = W.voronoi_image(side=side, K=K, label_frac=0.005, seed=W.SEED0 + 500 + i)
        pool.append((g, dict(eps=50.0, omega0=1e5)))
    gen_s = time.time() - t0
    common = dict(gap_tol=1e-4, tol_mode="rel", max_iters=2000, weight_dtype="f32")

    def plain(g, o):
        with B.Segmenter(g, iters_per_launch=64, **o, **common) as sg:
            st = sg.solve()
            return sg.labels(), st

    for g, o in pool[:3]:
        plain(g, o)
    service = []
    alone = []
    for g, o in pool:
        t = time.perf_counter()
        lab, st = plain(g, o)
        service.append(time.perf_counter() - t)
        alone.append((lab, st.iters))
    cap = 1.0 / float(np.mean(service))
    budget = 16 << 30
    R = args.steps * 20
    rates = []
    with B.Server(hbm_budget_bytes=budget, max_slots=32, max_K=8, iters_per_epoch=16,
                  weight_dtype="f32") as srv:
        for mult in (0.5, 1.0, 2.0):
            lam = mult * cap
            arr = np.cumsum(rng.exponential(1.0 / lam, size=R))
            pick = rng.integers(0, len(pool), size=R)
            # served: submit on schedule; between arrivals, sleep in the server
            # until a request finishes (or the next arrival is due)
            lat, t_start = [], time.perf_counter()
            pending = {}
            i = 0
            equal = True
            while i < R or pending:
                now = time.perf_counter() - t_start
                while i < R and arr[i] <= now:
                    g, o = pool[pick[i]]
                    pending[srv.submit(g, **o, **common)] = (i, arr[i])
                    i += 1
                wait_ms = int((arr[i] - now) * 1000.0) if i < R else 1000
                rc, tk = srv.wait_any(max(0, wait_ms))
                if rc == B.FW_OK and tk in pending:
                    done_t = time.perf_counter() - t_start
                    idx, ta = pending.pop(tk)
                    g, _ = pool[pick[idx]]
                    rc2, lab, st = srv.poll(tk, g.n)
                    lat.append(done_t - ta)
                    equal &= bool(np.array_equal(lab, alone[pick[idx]][0]))
            span_srv = time.perf_counter() - t_start
            # sequential plain solves of the same arrival process
            lat_seq, t_start = [], time.perf_counter()
            for j in range(R):
                now = time.perf_counter() - t_start
                if now < arr[j]:
                    time.sleep(arr[j] - now)
                g, o = pool[pick[j]]
                plain(g, o)
                lat_seq.append(time.perf_counter() - t_start - arr[j])
            span_seq = time.perf_counter() - t_start
            rates.append({
                "rate_per_s": lam, "x_capacity": mult, "requests": R,
                "served": {"solves_per_s": R / span_srv, "p50_ms": 1e3 * np.percentile(lat, 50),
                           "p99_ms": 1e3 * np.percentile(lat, 99)},
                "sequential": {"solves_per_s": R / span_seq,
                               "p50_ms": 1e3 * np.percentile(lat_seq, 50),
                               "p99_ms": 1e3 * np.percentile(lat_seq, 99)},
                "labels_equal_to_alone": equal})
        info = srv.info().as_dict()
    best = max(rates, key=lambda r: r["served"]["solves_per_s"])
    line = {
        "metric": "solves/s", "value": best["served"]["solves_per_s"], "unit": "solves/s",
        "n_gpus": 1, "steps": args.steps, "warmup": 3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "serving", "pool": "12 blob graphs (n 1e3..2e5) + 12 Voronoi "
                   "images (256^2..1024^2), K 3..8", "stop": "gap <= 1e-4 g_0, cap 2000",
                   "hbm_budget_bytes": budget, "max_slots": 32, "iters_per_epoch": 16},
        "sequential_capacity_per_s": cap, "rates": rates, "server": info,
        "setup_s": {"generate": gen_s},
    }
    if rank == 0 and emit:
        print(json.dumps(line), flush=True)
    return line


# ------------------------------------------------------------------ ours --
# -------------------------------------------------------------- one shot --
def run_oneshot(args, rank, world, local):
    """One-Shot Frank-Wolfe (Alg. 4) on the 2048x2048 image at eps = 0.1: the
    fused single-pass kernel, against the GFW iteration path that reaches the
    same labels in one step (Cor. nonconvb2).  Replicas only for N > 1."""
    name = "voronoi2048_oneshot"
    c = W.CONFIGS[name]
    if args.impl == "reference":
        if rank == 0:
            g = W.make_config_graph(name)
            v, dt, _ = cpu_oracle_oneshot(g, c)
            print(json.dumps({"impl": "reference", "metric": "one-shot segmentations/s",
                              "value": v, "unit": "solves/s", "n_gpus": world,
                              "higher_is_better": True, "config": {"workload": name},
                              "cpu_baseline": {"value": v, "unit": "solves/s", "cores": 1,
                                               "kind": "oracle",
                                               "sample": f"one OSFW on the full image, {dt:.1f} s"},
                              "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0,
                                      "d2h_bytes_per_step": 0}}), flush=True)
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
    g = W.make_config_graph(name)
    weights = args.weights or c["weights"]
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    opts = dict(eps=c["eps"], omega0=c["omega0"], weight_dtype=weights, max_iters=c["iters"],
                cuda_stream=stream.cuda_stream)
    seg = B.Segmenter(g, **opts)
    for _ in range(args.warmup):
        seg.oneshot(with_labels=False)
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    kms = [seg.oneshot(with_labels=False)[1] for _ in range(args.steps)]
    clocks.stop()
    clk = clocks.summary()
    value, t_s = whole_job_rate(args.steps, sum(kms) / 1000.0, world, "cuda")
    lab, _ = seg.oneshot()
    # the GFW path: reset + solve stops after its single step (alpha = 1)
    gfw_ms = []
    for _ in range(3):
        seg.reset()
        st = seg.solve()
        gfw_ms.append(st.ms)
    lab_gfw = seg.labels()
    seg.close()
    wb = {"f32": 4, "bf16": 2, "f64": 8}[weights]
    nbytes = 4 * (g.n + 1) + (column_bytes(g) + wb) * g.nnz + g.n + 4 * g.n
    mean_ms = float(np.mean(kms))
    peaks = load_peaks()
    achieved = nbytes / (mean_ms / 1000.0) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": ncu_traffic("k_osfw", name),
                "kernel": "k_osfw", "peak_source": peaks["source"],
                "algorithmic_bytes_per_launch": nbytes, "kernel_ms": {"k_osfw": mean_ms}}
    e2e = None
    if not args.no_e2e:
        def pinned(a):
            t = torch.empty(a.shape, dtype=getattr(torch, str(a.dtype)), pin_memory=True)
            t.numpy()[...] = a
            return t
        rp, col, w, lb = (pinned(g.row_ptr), pinned(g.col), pinned(g.w), pinned(g.labels))
        out = torch.empty(g.n, dtype=torch.int32, pin_memory=True)
        o = B.fw_seg_default_opts(**opts)
        steps_e2e = max(1, min(args.steps, 3))
        t0 = time.perf_counter()
        for _ in range(steps_e2e):
            h = B.fw_seg_create(g.n, rp.numpy(), col.numpy(), w.numpy(), g.K, lb.numpy(), o)
            _check = B.lib().fw_seg_oneshot(h.ptr, B.c_void_p(out.data_ptr()), None)
            B.fw_seg_destroy(h)
            if _check < 0:
                raise B.FwError(_check, B.fw_seg_last_error())
        dt = time.perf_counter() - t0
        e2e_rate, _ = whole_job_rate(steps_e2e, dt, world, "cuda")
        e2e = {"value": e2e_rate, "unit": "solves/s",
               "h2d_bytes_per_step": int(4 * (g.n + 1) + 12 * g.nnz + 4 * g.n),
               "d2h_bytes_per_step": int(4 * g.n), "steps": steps_e2e,
               "includes": "create (H2D, validation, Laplacian assembly, L U_0), one-shot "
                           "kernel, labels D2H, destroy"}
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    line = {
        "metric": "one-shot segmentations/s", "value": value, "unit": "solves/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": mean_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if weights == "f64" else "f32",
        "data": "synthetic",
        "config": {"workload": name, "n": g.n, "nnz": g.nnz, "K": g.K, "eps": c["eps"],
                   "omega0": c["omega0"], "weights": weights,
                   "l2": "inputs (CSR %.0f MB) larger than L2" % ((4 + wb) * g.nnz / 1e6),
                   "parallelism": f"replicas x{world}"},
        "gfw_one_step_ms": float(np.median(gfw_ms)),
        "labels_equal_gfw": bool(np.array_equal(lab, lab_gfw)),
        "clocks": clk, "e2e": e2e, "gpu_launches": args.steps, "roofline": roofline,
    }
    if not args.no_cpu_baseline and world == 1:
        v, dt, s_o = cpu_oracle_oneshot(g, c)
        line["label_agreement"] = float(np.mean(lab == s_o))
        line["cpu_baseline"] = {"value": v, "unit": "solves/s", "cores": 1, "kind": "oracle",
                                "sample": f"one OSFW (Alg. 4) of the oracle on the full image "
                                          f"(numpy/scipy FP64, one thread), {dt:.1f} s"}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def cpu_oracle_oneshot(g, c):
    """Oracle OSFW on the whole graph (problem set-up not timed)."""
    import oracle as O
    P = O.make_problem(g, c["eps"], c["omega0"], c["weights"])
    t0 = time.perf_counter()
    _, s = O.osfw(P)
    dt = time.perf_counter() - t0
    return 1.0 / dt, dt, s


# ---------------------------------------------------------- stored oracle --
def golden(workload, iters, weights):
    """The stored FP64 oracle run of this workload, if there is one
    (tests/golden/make_oracle_golden.py)."""
    p = os.path.join(GOLDEN, f"{workload}_oracle{iters}_{weights}.npz")
    return np.load(p) if os.path.exists(p) else None


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def trajectory(seg, iters):
    """(g_k, q_k, alpha_k, E_{k+1}) of iterations k = 0.. of a stepwise run from
    U_0; stepwise runs are bitwise the solve's trajectory."""
    seg.reset()
    out = []
    for _ in range(iters):
        st = seg.step(1)
        out.append((st.gap, st.q, st.alpha, st.objective))
        if st.status != 2:   # FW_PENDING: not stopped
            break
    return np.array(out)


def compare_golden(gold, labels, E_gpu, traj, truth):
    """Agreement of a GPU solve with the stored oracle run: labels, the final
    objective, accuracy against the generator's truth, and the per-iteration
    gap, curvature, step and objective."""
    ref = gold["labels"].astype(np.int32)
    off = ref != 0
    d = {"label_agreement": float(np.mean(labels == ref)),
         "label_agreement_off_class0": {
             "value": float(np.mean(labels[off] == ref[off])) if off.any() else None,
             "rows": int(off.sum())},
         "objective_rel_err": rel(E_gpu, float(gold["energy"])),
         "accuracy_vs_truth": {"gpu": float(np.mean(labels == truth)),
                               "oracle": float(gold["accuracy"])}}
    if traj is not None and "q" in gold:
        m = min(len(traj), len(gold["gap"]) - 1)
        t = {}
        for name, col, ref_arr in (("gap", 0, gold["gap"][:m]), ("q", 1, gold["q"][:m]),
                                   ("alpha", 2, gold["alpha"][:m]),
                                   ("objective", 3, gold["E"][1:m + 1])):
            e = np.abs(traj[:m, col] - ref_arr) / np.maximum(np.abs(ref_arr), 1e-300)
            t[name] = {"max_rel": float(e.max()), "median_rel": float(np.median(e)),
                       "at_iter": int(e.argmax())}
        t["iterations"] = m
        d["trajectory_vs_oracle"] = t
    return d


def roofline_of(prof, g, weights, workload, peaks, forms=None):
    wb = {"f32": 4, "bf16": 2, "f64": 8}[weights]
    tb = 8 if weights == "f64" else 4
    by = bytes_per_unit(g.n, g.nnz, g.K, wb, tb, column_bytes(g))
    dom = "csr_pass" if prof["pass_b"] >= prof["pass_a"] else "row_pass"
    dom_ms = prof["pass_b"] if dom == "csr_pass" else prof["pass_a"]
    kernel = {"csr_pass": "k_passB", "row_pass": "k_passA"}[dom]
    achieved = by[dom] / (dom_ms / 1000.0) / 1e9
    key = workload if weights == "f32" else f"{workload}_{weights}"
    return {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "traffic": ncu_traffic(kernel, key),
            "kernel": kernel, "peak_source": peaks["source"],
            "kernel_form": (("k_passB_tab (class table in shared memory)"
                             if forms and forms.get("class_table") else "k_passB_lc / k_passB")
                            if kernel == "k_passB" else "k_passA"),
            "algorithmic_bytes_per_launch": by[dom],
            "timing": "CUDA events on the solver's stream around a captured graph of "
                      "back-to-back launches of the kernel" if prof["in_graph"] else
                      "CUDA events around back-to-back direct launches of the kernel",
            "kernel_ms": {"k_passA": prof["pass_a"], "k_passB": prof["pass_b"],
                          "k_finish": prof["finish"]}}, by


def time_arm(args, B, torch, g, c, weights, iters, stream, flush, clocks, world, rank):
    """Warm-up and timed solves of one weight dtype, then its in-graph kernel
    times and (rank 0) its stepwise trajectory."""
    import torch.distributed as dist
    ipl = args.iters_per_launch or 32     # the library default
    opts = dict(eps=c["eps"], omega0=c["omega0"], weight_dtype=weights, max_iters=iters,
                iters_per_launch=ipl, lanes_per_row=args.lanes, class_table=args.class_table,
                cuda_stream=stream.cuda_stream)
    seg = B.Segmenter(g, **opts)
    forms = seg.forms().as_dict()
    for _ in range(args.warmup):
        flush.zero_()
        seg.reset()
        seg.solve()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches = 0
    st = None
    for s in range(args.steps):
        flush.zero_()
        ev[s][0].record(stream)
        seg.reset()
        st = seg.solve()
        ev[s][1].record(stream)
        launches += st.launches + 4     # reset: reinit, L U_hat, objective, state
    torch.cuda.synchronize()
    clocks.stop()
    t_ms = sum(a.elapsed_time(b) for a, b in ev)
    value, t_s = whole_job_rate(args.steps * st.iters, t_ms / 1000.0, world, "cuda")
    labels = seg.labels()
    E = seg.objective()
    seg.reset()
    prof = seg.profile(min(args.profile_iters, iters))
    traj = None if (args.no_trajectory or rank != 0) else trajectory(seg, iters)
    seg.close()
    return dict(value=value, t_s=t_s, iters=st.iters, launches=launches, labels=labels, E=E,
                prof=prof, traj=traj, opts=opts, forms=forms)


def arm_record(args, arm, g, c, weights, iters, world, peaks):
    """The JSON fields of one timed weight dtype."""
    roof, by = roofline_of(arm["prof"], g, weights, args.workload, peaks, arm.get("forms"))
    ms_step = 1000.0 * arm["t_s"] / args.steps
    rec = {"value": arm["value"], "unit": "iter/s", "weights": weights,
           "ms_per_step": ms_step, "solves_per_s": world * args.steps / arm["t_s"],
           "effective_gbs": by["iteration"] * arm["value"] / world / 1e9,
           "gpu_launches": arm["launches"], "roofline": roof, "kernel_forms": arm["forms"],
           "per_iteration_ms": {
               "timed_step": ms_step / max(1, arm["iters"]),
               "fused_graph": arm["prof"]["per_iter"],
               "passes": arm["prof"]["pass_a"] + arm["prof"]["pass_b"]
               + arm["prof"]["finish"] / arm["opts"]["iters_per_launch"],
               "note": "timed_step: the timed solves per iteration, reset (U_0, L U_0, E_0) "
                       "included; fused_graph: a graph of the solve's fused iterations; "
                       "passes: graphs of back-to-back pass A and pass B launches plus one "
                       "finish per graph launch of the solve"}}
    gold = golden(args.workload, iters, weights)
    if gold is not None and int(gold["nnz"]) == g.nnz:
        rec.update(compare_golden(gold, arm["labels"], arm["E"], arm["traj"], g.truth))
    else:
        rec["accuracy_vs_truth"] = {"gpu": float(np.mean(arm["labels"] == g.truth))}
    g32, g64 = golden(args.workload, iters, "f32"), golden(args.workload, iters, "f64")
    if g64 is not None and int(g64["nnz"]) == g.nnz:
        rec["label_agreement_vs_unrounded_weights_oracle"] = float(
            np.mean(arm["labels"] == g64["labels"].astype(np.int32)))
        if g32 is not None:
            # the oracle against itself: its run on FP32-rounded weights vs its
            # run on the unrounded weights (a rounding-level input change)
            ctl = {"label_agreement": float(np.mean(g32["labels"] == g64["labels"]))}
            for k in ("gap", "q", "alpha", "E"):
                m = min(len(g32[k]), len(g64[k]))
                ctl[k + "_max_rel"] = float(np.max(np.abs(g32[k][:m] - g64[k][:m]) /
                                                   np.abs(g64[k][:m])))
            rec["oracle_rounding_control"] = ctl
    return rec


def e2e_rate(args, B, torch, g, opts, world):
    """The same metric through the C ABI from pinned host buffers: create
    (upload, validation, assembly, L U_0), solve, labels to the host, destroy."""
    import torch.distributed as dist

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
    rate, _ = whole_job_rate(it_e2e, dt, world, "cuda")
    return {"value": rate, "unit": "iter/s",
            "h2d_bytes_per_step": int(4 * (g.n + 1) + 12 * g.nnz + 4 * g.n),
            "d2h_bytes_per_step": int(4 * g.n), "steps": steps_e2e,
            "includes": "create (H2D, validation, Laplacian assembly, L U_0), solve, labels "
                        "D2H, destroy"}


def run_single(args, rank, world, local):
    """One problem per GPU (replicas under torchrun): every weight dtype of
    the workload's arms, the first one the line's headline."""
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

    c = W.CONFIGS[args.workload]
    arms = [args.weights] if args.weights else list(c.get("arms", (c["weights"],)))
    iters = args.iters or c["iters"]
    g = W.make_config_graph(args.workload)
    stream = torch.cuda.Stream()          # one stream for flush, events and solver
    torch.cuda.set_stream(stream)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    clocks = ClockSampler(local)
    peaks = load_peaks()
    res = {w: time_arm(args, B, torch, g, c, w, iters, stream, flush, clocks, world, rank)
           for w in arms}
    clk = clocks.summary()
    e2e = None if args.no_e2e else e2e_rate(args, B, torch, g, res[arms[0]]["opts"], world)
    if world > 1:
        dist.barrier()
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    recs = {w: arm_record(args, res[w], g, c, w, iters, world, peaks) for w in arms}
    head = recs[arms[0]]
    line = {
        "metric": METRIC, "value": head.pop("value"), "unit": head.pop("unit"),
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": head.pop("ms_per_step"), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if arms[0] == "f64" else "f32",
        "data": "synthetic", "config": config_dict(args, c, g, iters, arms[0]),
        "clocks": clk, "e2e": e2e, "gpu_launches": head.pop("gpu_launches"),
        "roofline": head.pop("roofline"),
    }
    head.pop("weights")
    line.update(head)
    for w in arms[1:]:
        line[w] = recs[w]
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(g, c, arms[0], args.cpu_seconds)
    if not args.no_extras and world == 1:
        line.update(extras(args, rank, world, local))
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def extras(args, rank, world, local):
    """Compact runs of the batched (256 problems, 2 timed steps) and serving
    (100 Poisson requests per rate) workloads, as sub-records of the line."""
    import copy
    a = copy.copy(args)
    a.steps, a.warmup, a.iters, a.weights, a.lanes, a.problems = 2, 1, 0, "", 0, 256
    out = {"batched256": run_batched(a, rank, world, local, emit=False)}
    s = copy.copy(args)
    s.steps = 5
    out["serving"] = run_serving(s, rank, world, local, emit=False)
    return out


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.workload == "batched256":
        return run_batched(args, rank, world, local)
    if args.workload == "serving":
        return run_serving(args, rank, world, local)
    if args.workload == "oneshot":
        return run_oneshot(args, rank, world, local)
    if args.impl == "reference":
        return run_reference(args, W.CONFIGS[args.workload], rank)
    return run_single(args, rank, world, local)


if __name__ == "__main__":
    main()
