"""Writes oracle_solves.json: full FP64 oracle solves (Alg. 5, default
parameters, relaxed random start) of benchmark workloads, with the right-hand
side the benchmark uses (N(0,1) minus its mean, seed 11).

Per workload it stores the oracle's own counts (iterations, re-setups, cycles,
W-cycles), its wall time on the host that ran this script, and the solution
at 4,096 seeded sample indices plus its 2-norm, so that a GPU solution's error
to the oracle's can be stated without storing the whole vector. Calls only
the oracle. Usage: python tests/golden/make_oracle_solves.py C1 C2 C5-mid
"""
import json
import os
import platform
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_1806_07028_gb300 import inputs as I  # noqa: E402

OUT = os.path.join(HERE, "oracle_solves.json")
NSAMPLE = 4096


def sample_indices(n):
    return np.sort(np.random.default_rng(20240607).choice(n, size=min(NSAMPLE, n), replace=False))


def one(name):
    g = I.workload(name)
    b = I.rhs_normal(g.n, 11)
    t0 = time.perf_counter()
    x, st, hist = O.solve(g, b, params=O.default_params(keep_setup=0), hist_cap=100000)
    sec = time.perf_counter() - t0
    idx = sample_indices(g.n)
    return {"workload": name, "n": g.n, "nnz": g.nnz, "rhs": "rhs_normal(n, 11)",
            "iters": st["iters"], "resetups": st["resetups"], "cycles": st["cycles"],
            "wcycles": st["wcycles"], "rel_res": st["rel_res"], "oc_mean": st["oc_mean"],
            "status": st["status"], "seconds": sec, "threads": 1,
            "host": f"{platform.machine()} {os.cpu_count()} logical cores",
            "x_norm": float(np.linalg.norm(x)), "sample_seed": 20240607,
            "sample_idx": idx.tolist(), "sample_x": x[idx].tolist()}


def main(names):
    d = {}
    if os.path.exists(OUT):
        d = json.load(open(OUT))
    for name in names:
        rec = one(name)
        print(name, {k: rec[k] for k in ("iters", "resetups", "cycles", "wcycles", "seconds", "status")},
              flush=True)
        d[name] = rec
        with open(OUT, "w") as f:
            json.dump(d, f)


if __name__ == "__main__":
    main(sys.argv[1:] or ["C1"])
