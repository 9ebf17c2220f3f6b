"""Train and evaluate the learned start-vector network.

Training set: seeded random geometric graphs in the unit square (mean degree
12, weights 1/distance, largest component), n uniform in [nmin, nmax]. The
target of every graph is the first Alg. 2 smooth error of a plain run on it
(relaxed random start, right-hand side N(0,1) minus its mean, stopped right
after the first re-setup). One Adam step per graph per epoch, graphs in a
seeded random order, learning rate on a cosine schedule from lr to lr/10.
Every step (the plain runs, forward, loss, backward, Adam) runs in the
library's kernels on the GPU.

    python -m paper_1806_07028_gb300.train_mpnn --graphs 200 --epochs 30 --out net.mpnn
    python -m paper_1806_07028_gb300.train_mpnn --evaluate net.mpnn

Evaluation compares, on held-out graphs, the relaxed random start, the
network's start and the target itself used as the start vector (what a
perfect prediction would give): the mean convergence factor of the first
five V-cycles on the first hierarchy, the number of re-setups, and the time
of the full solve to 1e-8 (setup excluded).
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import inputs as I


def rgg_set(count, nmin, nmax, seed):
    rng = np.random.default_rng(seed)
    ns = rng.integers(nmin, nmax + 1, size=count)
    return [I.rgg(int(n), 12.0, seed=seed * 1_000_003 + k) for k, n in enumerate(ns)]


def examples(graphs, log=print):
    from .solver import training_example
    out = []
    t0 = time.time()
    for k, g in enumerate(graphs):
        ex = training_example(g, seed=k)
        if ex is not None:
            out.append(ex)
    log(f"{len(out)} training examples from {len(graphs)} graphs in {time.time() - t0:.1f} s")
    return out


def train(net, ex, epochs, lr, seed=0, log=print):
    rng = np.random.default_rng(seed)
    hist = []
    for ep in range(epochs):
        rate = lr * (0.1 + 0.9 * 0.5 * (1.0 + math.cos(math.pi * ep / max(1, epochs))))
        order = rng.permutation(len(ex))
        tot = 0.0
        for k in order:
            s, u, t = ex[k]
            tot += net.loss_grad(s, u, t)
            net.adam_step(rate)
        hist.append(tot / len(ex))
        log(f"epoch {ep:3d}  lr {rate:.2e}  mean loss {hist[-1]:.4f}")
    return hist


def _time_solve(g, b, **kw):
    import torch
    from .solver import Solver
    s = Solver(g, **kw)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, st = s.solve(b)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    s.close()
    return st, dt


def evaluate(net, graphs, cycles=5):
    """Per graph and start: mean convergence factor of the first `cycles`
    V-cycles on the first hierarchy, re-setups and time of the full solve."""
    from .solver import first_cycles, training_example
    rows = []
    for k, g in enumerate(graphs):
        b = I.rhs_normal(g.n, 7 + k)
        ex = training_example(g, seed=k)
        row = {"n": g.n, "name": g.name}
        starts = [("random", {}), ("learned", {"mpnn": net})]
        if ex is not None:
            starts.append(("target", {"e0": ex[2]}))
        for tag, kw in starts:
            cr = first_cycles(g, cycles=cycles, seed=7 + k, **kw)
            st, dt = _time_solve(g, b, **kw)
            row[tag] = {"conv": float(np.mean(cr)), "resetups": st["resetups"], "iters": st["iters"],
                        "ms": 1e3 * dt, "status": st["status"]}
        if ex is not None:
            ex[0].close()
        rows.append(row)
    return rows


def summarise(rows):
    out = {}
    for tag in ("random", "learned", "target"):
        r = [x[tag] for x in rows if tag in x]
        if r:
            out[tag] = {"conv": float(np.mean([x["conv"] for x in r])),
                        "resetups": float(np.mean([x["resetups"] for x in r])),
                        "ms": float(np.mean([x["ms"] for x in r]))}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--graphs", type=int, default=200)
    ap.add_argument("--nmin", type=int, default=10_000)
    ap.add_argument("--nmax", type=int, default=100_000)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default=None)
    ap.add_argument("--evaluate", default=None, metavar="WEIGHTS")
    ap.add_argument("--eval-graphs", type=int, default=6)
    a = ap.parse_args()
    from .solver import Mpnn
    held_out = rgg_set(a.eval_graphs, a.nmin, a.nmax, seed=a.seed + 7777)
    if a.evaluate:
        net = Mpnn.load(a.evaluate)
    else:
        ex = examples(rgg_set(a.graphs, a.nmin, a.nmax, a.seed))
        net = Mpnn(seed=a.seed)
        t0 = time.time()
        train(net, ex, a.epochs, a.lr, seed=a.seed)
        print(f"trained {a.epochs} epochs x {len(ex)} graphs in {time.time() - t0:.1f} s")
        for s, _, _ in ex:
            s.close()
        if a.out:
            net.save(a.out)
    rows = evaluate(net, held_out)
    print(json.dumps({"held_out": rows, "mean": summarise(rows)}, indent=1))


if __name__ == "__main__":
    main()
