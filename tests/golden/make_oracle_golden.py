"""Writes the stored FP64 oracle runs used by the free-running parity tests
and by bench.py's agreement figures:

    tests/golden/<workload>_oracle<iters>_<dtype>.npz

Each file holds the oracle's whole GFW trajectory from U_0 (Alg. 3 with the
exact line search): per iteration k the FW gap g_k, the curvature q_k, the
step alpha_k, the energy E(U_k) evaluated directly (eq. gradgl_vv2) and the
number of active rows; then the final labels (row argmax), the final energy,
the iteration count and stop status, and the accuracy against the
generator's ground truth.  The weights are rounded to the storage precision
of the GPU path being checked (`dtype`), so both sides work on the same
matrix.  Calls only the oracle and the input generators.

    python tests/golden/make_oracle_golden.py sbm200k f32
    python tests/golden/make_oracle_golden.py voronoi2048 f32
    python tests/golden/make_oracle_golden.py voronoi2048 bf16
    python tests/golden/make_oracle_golden.py voronoi2048 f64   (unrounded weights)
    python tests/golden/make_oracle_golden.py sbm200k f64
"""
import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_2508_09738_gb300 import workloads as W  # noqa: E402


def golden_path(workload: str, iters: int, dtype: str) -> str:
    return os.path.join(HERE, f"{workload}_oracle{iters}_{dtype}.npz")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("workload", choices=["sbm200k", "voronoi2048"])
    ap.add_argument("dtype", choices=["f32", "bf16", "f64"])
    a = ap.parse_args()
    c = W.CONFIGS[a.workload]
    g = W.make_config_graph(a.workload)
    P = O.make_problem(g, c["eps"], c["omega0"], a.dtype)
    t = time.time()
    U, info = O.gfw_solve(P, max_iters=c["iters"], record=True, with_energy=True)
    dt = time.time() - t
    h = info["hist"]
    lab = O.labels_from_U(U)
    out = golden_path(a.workload, c["iters"], a.dtype)
    np.savez_compressed(
        out, labels=lab.astype(np.uint8), gap=np.array(h["g"]), q=np.array(h["q"]),
        alpha=np.array(h["alpha"]), E=np.array(h["E"]), active=np.array(h["active"]),
        iters=info["iters"], status=info["status"], energy=O.energy(U, P),
        accuracy=float(np.mean(lab == g.truth)), seconds=dt, n=g.n, nnz=g.nnz,
        seed=c["seed"], eps=c["eps"], omega0=c["omega0"], weights=a.dtype)
    print(out, info["iters"], info["status"], f"{dt:.1f}s",
          f"accuracy {np.mean(lab == g.truth):.4f}")


if __name__ == "__main__":
    main()
