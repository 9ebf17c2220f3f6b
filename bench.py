#!/usr/bin/env python
"""Benchmark: unknowns/s to a 1e-8 relative residual with PC-alphaAMG on GB300.

One step = one complete adaptive solve of the 3D 7-point grid-graph Laplacian
128^3 (n = 2,097,152) with high-contrast weights (8^3 checkerboard blocks of
weight 1 or 1e-4, x-edges x100), right-hand side N(0,1) minus its mean:
pcamg_setup (validation, colouring, start vector, first hierarchy) plus
pcamg_solve (Alg. 5 with Alg. 2 re-setups) to ||b-Ax||/||b|| <= 1e-8, starting
from the CSR already resident in HBM. value = n * ranks / step time.
The matrix (175 MB) is larger than L2 (129 MB), so no flush is needed.

Forms: "fp32ir" (FP32 hierarchy and cycles inside FP64 iterative refinement,
the headline) and "fp64" (plain FP64). --impl reference times the CPU oracle
on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "unknowns/s to 1e-8 relative residual (setup + adaptive solve)"
UNIT = "unknowns/s"
WORKLOAD = "C2: 3D 7-point grid Laplacian 128^3, 8^3 checkerboard weights 1/1e-4, x-edges x100"


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="C2")
    ap.add_argument("--form", default="fp32ir", choices=["fp32ir", "fp64", "fp32ir+learned"])
    ap.add_argument("--no-extras", action="store_true", help="skip fp64 form, e2e and oracle legs")
    ap.add_argument("--only-kernel", default=None, choices=["residual64", "vcycle", "wcycle", "adapt", "mpnn"],
                    help="time one kernel alone on the workload (used for ncu captures)")
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--no-graphs", action="store_true",
                    help="run cycles as plain launches instead of CUDA graph replays (for profilers)")
    ap.add_argument("--summarize-launches", default=None, metavar="CSV",
                    help="reduce an ncu --csv launch list to per-kernel launches, time and share")
    return ap.parse_args()


def _graphs(a):
    return 0 if a.no_graphs else 1


def barrier():
    """Barrier across the ranks of a torchrun launch (no-op for one process)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def max_over_ranks(ms, device=None):
    """The slowest rank's time: the job's time for weak-scaling replicas."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(n, world, ms):
    """Whole-job throughput: every rank solves its own n-unknown system."""
    return n * world / (ms / 1e3)


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """Samples nvidia-smi during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.f = tempfile.NamedTemporaryFile(prefix="clocks", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _traffic_per_launch():
    """DRAM bytes per launch of the fine residual kernel from the committed ncu
    summary (profiles/residual64_C2.md, line 'traffic_bytes_per_launch: N')."""
    path = os.path.join(ROOT, "profiles", "residual64_C2.md")
    try:
        for line in open(path):
            if line.startswith("traffic_bytes_per_launch:"):
                v = line.split(":", 1)[1].strip()
                return None if v in ("", "null") else float(v)
    except Exception:
        pass
    return None


def _device_graph(g, device):
    import torch

    class DG:
        pass
    d = DG()
    d.n, d.nnz = g.n, g.nnz
    d.rowptr = torch.as_tensor(g.rowptr, device=device)
    d.col = torch.as_tensor(g.col, device=device)
    d.val = torch.as_tensor(g.val, device=device)
    return d


def run_ours(a):
    import numpy as np
    import torch

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    from paper_1806_07028_gb300 import Solver, default_params, inputs as I, native as N
    from paper_1806_07028_gb300 import solve_host

    g = I.workload(a.workload)
    b_host = I.rhs_normal(g.n, 11 + rank)
    dg = _device_graph(g, dev)
    b = torch.as_tensor(b_host, device=dev)
    prec = 0 if a.form == "fp64" else 1
    nets = {}

    def step(form, profile=0):
        """One solve in a form: fp64, fp32ir, or fp32ir+learned (the shipped
        start-vector network, its forward inside the setup)."""
        p = default_params(precision=0 if form == "fp64" else 1, profile=profile, use_graphs=_graphs(a))
        net = None
        if form.endswith("+learned"):
            if "net" not in nets:
                from paper_1806_07028_gb300 import Mpnn
                nets["net"] = Mpnn.pretrained()
            net = nets["net"]
        s = Solver(dg, params=p, device=dev, mpnn=net)
        x, st = s.solve(b)
        s.close()
        return x, st

    for _ in range(a.warmup):
        step(a.form, profile=1)
    torch.cuda.synchronize()
    barrier()
    clocks = Clocks(local)
    clocks.start()
    launches0 = N.lib().pcamg_kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    barrier()
    ev0.record()
    torch.cuda.nvtx.range_push("timed")   # lets a profiler select the timed steps
    stats = []
    for _ in range(a.steps):
        x, st = step(a.form, profile=1)
        stats.append(st)
    torch.cuda.nvtx.range_pop()
    ev1.record()
    torch.cuda.synchronize()
    launches = N.lib().pcamg_kernel_launches() - launches0
    ms = ev0.elapsed_time(ev1) / a.steps
    clk = clocks.stop()
    ms = max_over_ranks(ms, device=dev)
    x_host = x.cpu().numpy()
    rel = float(np.linalg.norm(b_host - g.to_scipy() @ x_host) / np.linalg.norm(b_host))
    value = job_value(g.n, world, ms)

    # roofline of the fine-level FP64 residual kernel (events on its own stream)
    peak, peak_kind = _peaks()
    pl = sum(s["prof_launches"] for s in stats)
    pms = sum(s["prof_ms"] for s in stats)
    bytes_per_launch = 12.0 * g.nnz + 28.0 * g.n
    achieved = (bytes_per_launch / (pms / pl / 1e3) / 1e9) if pl else None
    roofline = {"bound": "hbm", "kernel": "k_res_stream<double,1> (fine-level r = b - A x with ||r||^2)",
                "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None,
                "traffic": _traffic_per_launch(),
                "algorithmic_bytes_per_launch": bytes_per_launch,
                "peak_kind": f"{peak_kind} (hbm_gbs)", "launches_timed": pl}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
           "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": ("f64" if not prec else "f32 cycles in f64 refinement" +
                     (", bf16 tensor-core start network" if a.form.endswith("+learned") else "")),
           "data": "synthetic (seeded generator, same recipe as the configuration)",
           "config": {"workload": WORKLOAD, "n": g.n, "nnz": g.nnz, "form": a.form,
                      "tol": 1e-8, "parallelism": "replicas" if world > 1 else "single GPU",
                      "l2": "inputs larger than L2 (matrix 175 MB > 129 MB)"},
           "solve": {"iters": stats[-1]["iters"], "resetups": stats[-1]["resetups"],
                     "levels": stats[-1]["levels"], "oc_mean": stats[-1]["oc_mean"],
                     "rel_res_device": stats[-1]["rel_res"], "rel_res_host_check": rel,
                     "t_alg2_ms": stats[-1]["t_alg2_ms"], "t_alg4_ms": stats[-1]["t_alg4_ms"],
                     "cycles": stats[-1]["cycles"]},
           "roofline": roofline, "clocks": clk, "gpu_launches": int(launches)}

    if not a.no_extras and rank == 0:
        # the other forms, same graph and b (one warm-up solve, one timed)
        out["forms"] = {a.form: {"ms": ms, "unknowns_per_s": g.n / (ms / 1e3), "iters": stats[-1]["iters"],
                                 "resetups": stats[-1]["resetups"]}}
        for other in ("fp64", "fp32ir", "fp32ir+learned"):
            if other == a.form:
                continue
            step(other)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            _, st2 = step(other)
            e1.record()
            torch.cuda.synchronize()
            ms2 = e0.elapsed_time(e1)
            out["forms"][other] = {"ms": ms2, "unknowns_per_s": g.n / (ms2 / 1e3), "iters": st2["iters"],
                                   "resetups": st2["resetups"]}
        # end to end through the public host-buffer call: pinned host inputs,
        # H2D of A, b, x and D2H of x inside the timed region
        rp = torch.as_tensor(g.rowptr).pin_memory().numpy()
        ci = torch.as_tensor(g.col).pin_memory().numpy()
        va = torch.as_tensor(g.val).pin_memory().numpy()
        bh = torch.as_tensor(b_host).pin_memory().numpy()

        class HG:
            pass
        hg = HG()
        hg.n, hg.nnz, hg.rowptr, hg.col, hg.val = g.n, g.nnz, rp, ci, va
        def host_params():
            hp = default_params(precision=prec)
            if a.form.endswith("+learned"):
                hp.start, hp.mpnn = N.START_LEARNED, nets["net"]._h
            return hp
        solve_host(hg, bh, params=host_params())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        xe, ste = solve_host(hg, bh, params=host_params())
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        h2d = rp.nbytes + ci.nbytes + va.nbytes + bh.nbytes + 8 * g.n
        out["e2e"] = {"value": g.n / te, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                      "d2h_bytes_per_step": int(8 * g.n), "ms": te * 1e3,
                      "status": ste["status"]}
        if world == 1:
            out["cpu_baseline"] = oracle_sample(g, b_host, stats[-1])
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _host_cpu():
    """The host the CPU oracle ran on: its logical core count and CPU model."""
    import platform
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k = line.split(":", 1)[0].strip().lower()
                if k in ("model name", "cpu model", "hardware"):
                    model = line.split(":", 1)[1].strip()
                    break
            if model is None:   # Arm: implementer and part numbers instead of a model name
                f.seek(0)
                ids = {}
                for line in f:
                    k = line.split(":", 1)[0].strip()
                    if k in ("CPU implementer", "CPU part") and k not in ids:
                        ids[k] = line.split(":", 1)[1].strip()
                if ids:
                    model = " ".join(f"{k} {v}" for k, v in ids.items())
    except OSError:
        pass
    return {"logical_cores": os.cpu_count(), "machine": platform.machine(), "model": model}


def oracle_sample(g, b, gpu_stats, max_seconds=40.0):
    """The CPU oracle (single thread) on a bounded sample of the same workload:
    its start vector, one hierarchy build (Alg. 4) and one V- and one W-cycle on
    the full graph, scaled to a whole solve with the GPU run's own counts of
    hierarchies and cycles (the oracle reproduces those counts on this graph)."""
    import numpy as np

    import oracle as O
    t0 = time.perf_counter()
    e = O.start_vector(g)
    t1 = time.perf_counter()
    h = O.Hierarchy(g, e)
    t2 = time.perf_counter()
    r = b.copy()
    h.vcycle(r)
    t3 = time.perf_counter()
    wc = None
    if t3 - t0 < max_seconds:
        h.wcycle(r)
        wc = time.perf_counter() - t3
    t_start, t_build, t_v = t1 - t0, t2 - t1, t3 - t2
    H = gpu_stats["resetups"] + 1
    cyc = gpu_stats["cycles"]
    # W-cycles are applied in the first two re-setups' PCG (7 each); counted as W
    nw = min(gpu_stats["resetups"], 2) * 7
    est = t_start + H * t_build + (cyc - nw) * t_v + nw * (wc if wc is not None else 2 * t_v)
    h.close()
    return {"value": g.n / est, "unit": UNIT, "cores": 1, "kind": "oracle", "host": _host_cpu(),
            "sample": (f"oracle start vector ({t_start:.2f}s) + 1 hierarchy build ({t_build:.2f}s) + "
                       f"1 V-cycle ({t_v:.3f}s) + 1 W-cycle ({wc if wc is not None else float('nan'):.3f}s) "
                       f"on the full graph, scaled by the GPU solve's {H} builds and {cyc} cycles "
                       f"({nw} W) to {est:.1f}s per solve"),
            "measured_seconds": time.perf_counter() - t0}


# Iteration structure of one solve of the C2 workload (hierarchies built and
# cycles applied), as reported by the solver's own statistics; the oracle's
# solve follows the same trajectory on this graph (same counts).
SOLVE_COUNTS = {"C2": {"builds": 21, "cycles": 1690, "wcycles": 14}}


def run_reference(a):
    """The CPU oracle as the reference arm: each step is a bounded sample of the
    workload (start vector, one hierarchy build, one V- and one W-cycle on the
    full graph), scaled to a whole solve with the workload's iteration counts."""
    rank, world, _ = _dist()
    if rank != 0:
        return
    import oracle as O
    from paper_1806_07028_gb300 import inputs as I
    g = I.workload(a.workload)
    b = I.rhs_normal(g.n, 11)
    cnt = SOLVE_COUNTS.get(a.workload, SOLVE_COUNTS["C2"])
    est, steps_ms = [], []
    for k in range(a.warmup + a.steps):
        t0 = time.perf_counter()
        e = O.start_vector(g)
        t1 = time.perf_counter()
        h = O.Hierarchy(g, e)
        t2 = time.perf_counter()
        h.vcycle(b)
        t3 = time.perf_counter()
        h.wcycle(b)
        t4 = time.perf_counter()
        h.close()
        if k >= a.warmup:
            steps_ms.append(1e3 * (t4 - t0))
            est.append((t1 - t0) + cnt["builds"] * (t2 - t1) +
                       (cnt["cycles"] - cnt["wcycles"]) * (t3 - t2) + cnt["wcycles"] * (t4 - t3))
    t_solve = sum(est) / len(est)
    value = g.n / t_solve
    sample = (f"per step: oracle start vector + 1 hierarchy build + 1 V-cycle + 1 W-cycle on the "
              f"full graph ({statistics.mean(steps_ms)/1e3:.1f}s), scaled by {cnt['builds']} builds "
              f"and {cnt['cycles']} cycles ({cnt['wcycles']} W) to {t_solve:.0f}s per solve")
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
           "warmup": a.warmup, "ms_per_step": 1e3 * t_solve, "higher_is_better": True,
           "impl": "reference", "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "n": g.n, "nnz": g.nnz, "form": "oracle fp64"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "host": _host_cpu(),
                            "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_kernel(a):
    """One kernel (or one multigrid cycle) alone on the workload, timed with
    CUDA events on the launching stream."""
    import numpy as np
    import torch

    if a.only_kernel == "adapt":
        from paper_1806_07028_gb300 import Solver, default_params, inputs as I
        g = I.workload(a.workload)
        prec = 0 if a.form == "fp64" else 1
        dev = torch.device("cuda", 0)
        s = Solver(_device_graph(g, dev), params=default_params(precision=prec, use_graphs=_graphs(a)), device=dev)
        e = s.start_vector()
        s.adapt(e)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("adapt")
        t0 = time.perf_counter()
        for _ in range(a.reps):
            s.adapt(e)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1e3 / a.reps
        torch.cuda.nvtx.range_pop()
        print(json.dumps({"adapt": a.workload, "form": a.form, "ms": ms, "levels": s.num_levels(-1)}),
              flush=True)
        s.close()
        return
    if a.only_kernel == "mpnn":
        # the learned start's forward pass (shipped weights) on the workload's graph
        from paper_1806_07028_gb300 import Mpnn, Solver, default_params, inputs as I
        g = I.workload(a.workload)
        dev = torch.device("cuda", 0)
        s = Solver(_device_graph(g, dev), params=default_params(precision=1), device=dev)
        u = s.start_vector()
        net = Mpnn.pretrained()
        for _ in range(2):
            net.forward(s, u)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("mpnn")
        t0 = time.perf_counter()
        for _ in range(a.reps):
            net.forward(s, u)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1e3 / a.reps
        torch.cuda.nvtx.range_pop()
        print(json.dumps({"mpnn_forward": a.workload, "n": g.n, "nnz": g.nnz, "ms": ms}), flush=True)
        net.close()
        s.close()
        return
    if a.only_kernel in ("vcycle", "wcycle"):
        from paper_1806_07028_gb300 import Solver, default_params, inputs as I
        g = I.workload(a.workload)
        prec = 0 if a.form == "fp64" else 1
        dev = torch.device("cuda", 0)
        s = Solver(_device_graph(g, dev), params=default_params(precision=prec, use_graphs=_graphs(a)), device=dev)
        r = torch.as_tensor(I.rhs_normal(g.n, 3), device=dev)
        gamma = 1 if a.only_kernel == "vcycle" else 2
        for _ in range(2):
            s.cycle(r, 0, gamma)
        torch.cuda.synchronize()
        # NVTX range "cycles" lets a profiler select the timed cycles only
        torch.cuda.nvtx.range_push("cycles")
        t0 = time.perf_counter()
        for _ in range(a.reps):
            s.cycle(r, 0, gamma)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1e3 / a.reps
        torch.cuda.nvtx.range_pop()
        print(json.dumps({"cycle": a.only_kernel, "workload": a.workload, "form": a.form, "ms": ms,
                          "levels": s.num_levels(0)}), flush=True)
        s.close()
        return

    from paper_1806_07028_gb300 import inputs as I, residual
    g = I.workload(a.workload)
    dg = _device_graph(g, torch.device("cuda", 0))
    rng = np.random.default_rng(0)
    x = torch.as_tensor(rng.standard_normal(g.n), device="cuda:0")
    b = torch.as_tensor(rng.standard_normal(g.n), device="cuda:0")
    for _ in range(3):
        residual(dg.rowptr, dg.col, dg.val, x, b)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.reps):
        residual(dg.rowptr, dg.col, dg.val, x, b)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.reps
    byt = 12.0 * g.nnz + 28.0 * g.n
    peak, kind = _peaks()
    print(json.dumps({"kernel": "residual64", "workload": a.workload, "ms": ms,
                      "algorithmic_bytes": byt, "GBs": byt / ms / 1e6, "peak": peak,
                      "frac": byt / ms / 1e6 / peak, "peak_kind": kind}), flush=True)


def _kernel_short_name(full):
    """Kernel name without its call arguments, return type and namespaces:
    'void pc::<unnamed>::k_rowprod_warp<pc::<unnamed>::GalSrc, 2>(int, ...)'
    becomes 'k_rowprod_warp<GalSrc, 2>'."""
    import re
    full = re.sub(r"(\(anonymous namespace\)|<unnamed>)::", "", full)
    name = full
    depth = 0
    for i, ch in enumerate(full):   # cut at the '(' of the parameter list (outside <...>)
        if ch == "<":
            depth += 1
        elif ch == ">":
            depth -= 1
        elif ch == "(" and depth == 0:
            name = full[:i]
            break
    name = re.sub(r"^void ", "", name)
    return re.sub(r"\bpc::", "", name).strip()


def summarize_launches(path):
    """Per-kernel launches, total device time and share from an ncu launch list
    (--metrics gpu__time_duration.sum --csv); template arguments are kept, call
    arguments dropped."""
    import collections
    import csv
    import re
    by = collections.defaultdict(lambda: [0, 0.0])
    with open(path) as f:
        rows = csv.reader(line for line in f if line.startswith('"'))
        hdr = next(rows)
        ki, vi = hdr.index("Kernel Name"), hdr.index("Metric Value")
        ui = hdr.index("Metric Unit")
        for r in rows:
            name = _kernel_short_name(r[ki])
            scale = {"ns": 1e-3, "usecond": 1.0, "us": 1.0, "msecond": 1e3, "ms": 1e3, "nsecond": 1e-3}.get(r[ui], 1e-3)
            by[name][0] += 1
            by[name][1] += float(r[vi].replace(",", "")) * scale
    tot = sum(t for _, t in by.values())
    n = sum(c for c, _ in by.values())
    lines = [f"launches: {n}   total device time: {tot / 1e3:.3f} ms (one launch at a time)",
             f"{'kernel':60s} {'launches':>9s} {'total ms':>10s} {'share':>7s}"]
    for k, (c, t) in sorted(by.items(), key=lambda x: -x[1][1]):
        lines.append(f"{k[:60]:60s} {c:9d} {t / 1e3:10.3f} {100 * t / tot:6.2f}%")
    print("\n".join(lines))


def main():
    a = _args()
    if a.summarize_launches:
        summarize_launches(a.summarize_launches)
    elif a.only_kernel:
        run_kernel(a)
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
