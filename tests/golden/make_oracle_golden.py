"""Writes tests/golden/sbm200k_oracle500.npz: the FP64 oracle's result of 500
GFW iterations on the 200k-node SBM workload (weights rounded to FP32, the
storage of the FP32 path).  Calls only the oracle and the input generators.

    python tests/golden/make_oracle_golden.py
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_2508_09738_gb300 import workloads as W  # noqa: E402


def main():
    c = W.CONFIGS["sbm200k"]
    g = W.make_config_graph("sbm200k")
    P = O.make_problem(g, c["eps"], c["omega0"], c["weights"])
    t = time.time()
    U, info = O.gfw_solve(P, max_iters=c["iters"], record=True)
    dt = time.time() - t
    out = os.path.join(HERE, "sbm200k_oracle500.npz")
    np.savez_compressed(out, labels=O.labels_from_U(U).astype(np.uint8),
                        gap=np.array(info["hist"]["g"]), alpha=np.array(info["hist"]["alpha"]),
                        iters=info["iters"], energy=O.energy(U, P), seconds=dt,
                        n=g.n, nnz=g.nnz, seed=c["seed"])
    print(out, info["iters"], info["status"], f"{dt:.1f}s")


if __name__ == "__main__":
    main()
