#!/usr/bin/env python
"""Benchmark: time to a 1e-8 relative residual and unknowns/s with PC-alphaAMG on
GB300, FP32 hierarchy with the learned start inside FP64 refinement against
plain FP64, on the same graph and right-hand side.

One step = one complete adaptive solve of the workload (default C5: the 3D
7-point grid Laplacian 256^3, n = 16,777,216, jump coefficients 10^U(-6,0) on
16^3 blocks), right-hand side N(0,1) minus its mean: pcamg_setup (validation,
colouring, start vector -- the learned network's forward pass in the headline
form -- and the first hierarchy) plus pcamg_solve (Alg. 5 with Alg. 2
re-setups) to ||b-Ax||/||b|| <= 1e-8, from the CSR already resident in HBM.
value = n * ranks / step time. The matrix (1.4 GB) is larger than L2
(129 MB), so no flush is needed.

Forms: "fp32ir+learned" (the headline: FP32 hierarchy and cycles inside FP64
iterative refinement, learned start vector), "fp32ir" (same, relaxed random
start) and "fp64" (plain FP64, relaxed random start); the two others are
timed once each on the same graph and b. --impl reference times the CPU
oracle on a bounded sample of the same workload instead.
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

METRIC = "time to 1e-8 residual & unknowns/s: plain FP64 vs FP32+learned form, same GB300"
UNIT = "unknowns/s"
GOLDEN_SOLVES = os.path.join(ROOT, "tests", "golden", "oracle_solves.json")
# the oracle's recorded full solve whose counts stand in for a workload whose
# own full oracle solve was not recorded (same recipe, smaller grid)
COUNTS_FROM = {"C5": "C5-mid"}


def workload_label(name):
    from paper_1806_07028_gb300 import inputs as I
    return f"{name}: {I.DESCRIPTIONS.get(name, name)}"


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="C5")
    ap.add_argument("--form", default="fp32ir+learned", choices=["fp32ir", "fp64", "fp32ir+learned"])
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


def _golden_solves():
    """Full oracle solves recorded by tests/golden/make_oracle_solves.py."""
    try:
        return json.load(open(GOLDEN_SOLVES))
    except Exception:
        return {}


def oracle_counts(workload):
    """The oracle's own counts of one full solve (hierarchies built, cycles, W-cycles)
    of this workload, or of the recorded same-recipe workload standing in for it."""
    rec = _golden_solves()
    src = workload if workload in rec else COUNTS_FROM.get(workload)
    if src not in rec:
        return None
    r = rec[src]
    return {"from": src, "builds": r["resetups"] + 1, "cycles": r["cycles"], "wcycles": r["wcycles"],
            "iters": r["iters"], "n": r["n"], "seconds_full_solve": r["seconds"], "host": r["host"]}


def error_vs_recorded_oracle(workload, x):
    """||x - x_oracle|| / ||x_oracle|| on the recorded sample indices."""
    import numpy as np
    rec = _golden_solves().get(workload)
    if rec is None:
        return None
    idx = np.asarray(rec["sample_idx"], dtype=np.int64)
    xo = np.asarray(rec["sample_x"])
    return {"value": float(np.linalg.norm(x[idx] - xo) / np.linalg.norm(xo)),
            "over": f"{len(idx)} seeded sample entries of the oracle's recorded FP64 solution"}


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


def _oracle_sample_proc(workload, rank_seed, q):
    """Child process (spawned before any GPU work) timing the oracle sample."""
    try:
        from paper_1806_07028_gb300 import inputs as I
        g = I.workload(workload)
        q.put(oracle_sample(g, I.rhs_normal(g.n, rank_seed), workload))
    except Exception as ex:   # reported, never fatal to the GPU measurement
        q.put({"error": repr(ex)})


def _small_oracle_check(P, form_params):
    """The oracle's full FP64 solve of C1 next to the GPU's forms on the same b:
    the relative error of each GPU solution to the oracle's."""
    import numpy as np
    import oracle as O
    from paper_1806_07028_gb300 import inputs as I
    g = I.workload("C1")
    b = I.rhs_normal(g.n, 11)
    xo, so, _ = O.solve(g, b)
    out = {"workload": "C1", "oracle_iters": so["iters"], "oracle_resetups": so["resetups"]}
    for form, (prm, net) in form_params.items():
        s = P.Solver(g, params=prm, mpnn=net)
        x, st = s.solve(b)
        s.close()
        x = x.cpu().numpy()
        out[form] = {"error": float(np.linalg.norm(x - xo) / np.linalg.norm(xo)),
                     "rel_res": float(np.linalg.norm(b - g.to_scipy() @ x) / np.linalg.norm(b)),
                     "iters": st["iters"], "resetups": st["resetups"]}
    return out


def run_ours(a):
    import multiprocessing as mp

    import numpy as np

    rank, world, local = _dist()
    want_cpu = (not a.no_extras) and rank == 0 and world == 1
    oq = None
    if want_cpu:   # the oracle sample runs on one host core while the GPU is timed
        ctx = mp.get_context("spawn")
        oq = ctx.Queue()
        op = ctx.Process(target=_oracle_sample_proc, args=(a.workload, 11 + rank, oq), daemon=True)
        op.start()

    import torch
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    import paper_1806_07028_gb300 as P
    from paper_1806_07028_gb300 import Solver, default_params, inputs as I, native as N
    from paper_1806_07028_gb300 import solve_host

    g = I.workload(a.workload)
    b_host = I.rhs_normal(g.n, 11 + rank)
    dg = _device_graph(g, dev)
    b = torch.as_tensor(b_host, device=dev)
    nets = {}

    def net_for(form):
        if "+learned" not in form:
            return None
        if "net" not in nets:
            from paper_1806_07028_gb300 import Mpnn
            nets["net"] = Mpnn.pretrained()
        return nets["net"]

    def params_for(form, profile=0):
        return default_params(precision=0 if form == "fp64" else 1, profile=profile, use_graphs=_graphs(a),
                              outer=1 if form.endswith("+fcg") else 0)

    def step(form, profile=0):
        """One solve in a form: fp64, fp32ir, or fp32ir+learned (the shipped
        start-vector network, its forward pass inside the setup)."""
        s = Solver(dg, params=params_for(form, profile), device=dev, mpnn=net_for(form))
        x, st = s.solve(b)
        s.close()
        return x, st

    for _ in range(a.warmup):
        step(a.form, profile=2)
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
        x, st = step(a.form, profile=2)
        stats.append(st)
    torch.cuda.nvtx.range_pop()
    ev1.record()
    torch.cuda.synchronize()
    launches = N.lib().pcamg_kernel_launches() - launches0
    ms = ev0.elapsed_time(ev1) / a.steps
    clk = clocks.stop()
    ms = max_over_ranks(ms, device=dev)
    x_host = x.cpu().numpy()
    A = g.to_scipy()
    rel = float(np.linalg.norm(b_host - A @ x_host) / np.linalg.norm(b_host))
    value = job_value(g.n, world, ms)

    # rooflines of the finest level's two kernels inside the V-cycle, timed live
    # with CUDA events (event-record nodes in the captured cycle graph, on the
    # library's stream) over every V-cycle of the timed solves: the residual and
    # the pre-smoothing Gauss-Seidel sweep (all colours); the line's "roofline"
    # is the one with the larger total time
    peak, peak_kind = _peaks()
    w = 8.0 if a.form == "fp64" else 4.0
    bytes_per_launch = (4.0 + w) * g.nnz + (4.0 + 3.0 * w) * g.n
    tname = "double" if a.form == "fp64" else "float"

    def _roof(count_key, ms_key, kernel, what):
        cl = sum(s[count_key] for s in stats)
        cms = sum(s[ms_key] for s in stats)
        achieved = (bytes_per_launch / (cms / cl / 1e3) / 1e9) if cl else None
        return {"bound": "hbm", "kernel": kernel, "what": what,
                "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None, "traffic": None,
                "algorithmic_bytes_per_launch": bytes_per_launch,
                "mean_launch_us": (1e3 * cms / cl) if cl else None, "total_ms": cms,
                "peak_kind": f"{peak_kind} (hbm_gbs)", "launches_timed": cl,
                "timing": "CUDA events on the library stream around every instance in the timed solves"}

    roof_res = _roof("cyc_launches", "cyc_ms", f"k_res_stream<{tname},0,1>, finest level",
                     "r = b - A x inside every V-cycle (one launch)")
    roof_gs = _roof("gs_sweeps", "gs_ms", f"k_gs_stream<{tname},1>, finest level",
                    "pre-smoothing Gauss-Seidel sweep of every V-cycle (one launch per colour; "
                    "bytes: A, b, x written, every x gathered once)")
    if (roof_gs["total_ms"] or 0) > (roof_res["total_ms"] or 0):
        roofline, roofline_other = roof_gs, roof_res
    else:
        roofline, roofline_other = roof_res, roof_gs

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
           "warmup": a.warmup, "ms_per_step": ms, "time_to_tol_s": ms / 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": ("f64" if a.form == "fp64" else "f32 cycles in f64 refinement" +
                     (", bf16 tensor-core start network" if a.form.endswith("+learned") else "")),
           "data": "synthetic (seeded generator, same recipe as the configuration)",
           "config": {"workload": workload_label(a.workload), "n": g.n, "nnz": g.nnz, "form": a.form,
                      "tol": 1e-8, "parallelism": "replicas" if world > 1 else "single GPU",
                      "l2": f"inputs larger than L2 (matrix {12 * g.nnz / 1e6:.0f} MB > 129 MB)"},
           "solve": {"iters": stats[-1]["iters"], "resetups": stats[-1]["resetups"],
                     "levels": stats[-1]["levels"], "oc_mean": stats[-1]["oc_mean"],
                     "rel_res_device": stats[-1]["rel_res"], "rel_res_host_check": rel,
                     "t_alg2_ms": stats[-1]["t_alg2_ms"], "t_alg4_ms": stats[-1]["t_alg4_ms"],
                     "cycles": stats[-1]["cycles"], "wcycles": stats[-1]["wcycles"]},
           "roofline": roofline, "roofline_other": roofline_other, "clocks": clk,
           "gpu_launches": int(launches)}

    if not a.no_extras and rank == 0:
        # the other forms, same graph and b (one warm-up solve, one timed)
        out["forms"] = {a.form: {"ms": ms, "unknowns_per_s": g.n / (ms / 1e3), "iters": stats[-1]["iters"],
                                 "resetups": stats[-1]["resetups"], "cycles": stats[-1]["cycles"]}}
        xs = {a.form: x_host}
        # "+fcg": flexible CG outer iteration instead of the paper's stationary one
        for other in ("fp64", "fp32ir", "fp32ir+learned", "fp32ir+learned+fcg"):
            if other == a.form:
                continue
            step(other)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            x2, st2 = step(other)
            e1.record()
            torch.cuda.synchronize()
            ms2 = e0.elapsed_time(e1)
            xs[other] = x2.cpu().numpy()
            out["forms"][other] = {"ms": ms2, "unknowns_per_s": g.n / (ms2 / 1e3), "iters": st2["iters"],
                                   "resetups": st2["resetups"], "cycles": st2["cycles"],
                                   "rel_res_host_check": float(np.linalg.norm(b_host - A @ xs[other]) /
                                                               np.linalg.norm(b_host))}
        if "fp64" in out["forms"] and a.form != "fp64":
            out["speedup_vs_fp64"] = out["forms"]["fp64"]["ms"] / ms
        out["multi_rhs"] = multi_rhs_leg(dg, g, b_host, params_for(a.form), net_for(a.form), dev)
        # errors: to the oracle's recorded solution of this workload where one
        # exists, between the forms here, and to the oracle's full solve of C1
        err = {}
        rec = error_vs_recorded_oracle(a.workload, x_host) if world == 1 else None
        err["headline_vs_oracle"] = rec if rec else (
            "not recorded: the oracle's full solve of this workload keeps every hierarchy in host "
            "memory (Alg. 2 recycles them) and does not fit the recording host")
        if "fp64" in xs and a.form != "fp64":
            xf = xs["fp64"]
            err["headline_vs_fp64_gpu"] = float(np.linalg.norm(x_host - xf) / np.linalg.norm(xf))
        err["C1_full_oracle"] = _small_oracle_check(
            P, {f: (params_for(f), net_for(f)) for f in ("fp64", "fp32ir", "fp32ir+learned")})
        out["error_vs_oracle"] = err
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
            hp = params_for(a.form)
            if a.form.endswith("+learned"):
                hp.start, hp.mpnn = N.START_LEARNED, net_for(a.form)._h
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
    if oq is not None:
        try:
            cb = oq.get(timeout=900)
        except Exception as ex:
            cb = {"error": f"oracle sample did not finish: {ex!r}"}
        out["cpu_baseline"] = cb
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


class OracleSample:
    """The CPU oracle (one thread) on the workload's full graph: its start vector,
    one hierarchy build (Alg. 4), one W-cycle and V-cycles, timed; a whole
    solve is extrapolated with the oracle's own counts of builds and cycles from
    its recorded full solve of the workload (or of the same recipe on a smaller
    grid, named in the result)."""

    def __init__(self, g, workload):
        import oracle as O
        self.O, self.g, self.workload = O, g, workload
        t0 = time.perf_counter()
        self.e = O.start_vector(g)
        t1 = time.perf_counter()
        self.h = O.Hierarchy(g, self.e, O.default_params(keep_setup=0))
        t2 = time.perf_counter()
        self.t_start, self.t_build = t1 - t0, t2 - t1
        self.t_w = None
        self.t_v = []
        self.counts = oracle_counts(workload)

    def wcycle(self, r):
        t0 = time.perf_counter()
        self.h.wcycle(r)
        self.t_w = time.perf_counter() - t0

    def vcycle(self, r):
        t0 = time.perf_counter()
        self.h.vcycle(r)
        self.t_v.append(time.perf_counter() - t0)
        return self.t_v[-1]

    def estimate(self):
        c = self.counts
        tv = statistics.mean(self.t_v)
        tw = self.t_w if self.t_w is not None else 6.0 * tv
        est = self.t_start + c["builds"] * self.t_build + (c["cycles"] - c["wcycles"]) * tv + c["wcycles"] * tw
        return est, tv, tw

    def close(self):
        self.h.close()


def oracle_sample(g, b, workload):
    t0 = time.perf_counter()
    smp = OracleSample(g, workload)
    if smp.counts is None:
        smp.close()
        return {"error": f"no recorded oracle solve for {workload}"}
    smp.wcycle(b)
    smp.vcycle(b)
    est, tv, tw = smp.estimate()
    smp.close()
    c = smp.counts
    return {"value": g.n / est, "unit": UNIT, "cores": 1, "kind": "oracle", "extrapolated": True,
            "host": _host_cpu(), "measured_seconds": time.perf_counter() - t0,
            "sample": (f"oracle start vector ({smp.t_start:.2f}s) + 1 hierarchy build ({smp.t_build:.2f}s) + "
                       f"1 W-cycle ({tw:.2f}s) + 1 V-cycle ({tv:.3f}s) on the full {workload} graph, "
                       f"extrapolated to {est:.0f}s per solve with the oracle's own counts of its "
                       f"recorded full solve of {c['from']} (n = {c['n']:,}): {c['builds']} builds, "
                       f"{c['cycles']} cycles ({c['wcycles']} W)")}


def run_reference(a):
    """The CPU oracle as the reference arm. Set-up (untimed per step): the
    oracle's start vector, one hierarchy build and one W-cycle on the full graph.
    Each step: one oracle V-cycle on the full graph. The step's value is the
    whole solve extrapolated from these measurements with the oracle's own counts
    of builds and cycles from its recorded full solve (extrapolated: true)."""
    rank, world, _ = _dist()
    if rank != 0:
        return
    from paper_1806_07028_gb300 import inputs as I
    g = I.workload(a.workload)
    b = I.rhs_normal(g.n, 11)
    t_setup0 = time.perf_counter()
    smp = OracleSample(g, a.workload)
    if smp.counts is None:
        print(json.dumps({"impl": "reference", "unavailable": f"no recorded oracle solve for {a.workload}"}))
        return
    smp.wcycle(b)
    t_setup = time.perf_counter() - t_setup0
    for _ in range(a.warmup):
        smp.vcycle(b)
    smp.t_v = []
    step_s = [smp.vcycle(b) for _ in range(a.steps)]
    est, tv, tw = smp.estimate()
    smp.close()
    c = smp.counts
    value = g.n / est
    sample = (f"set-up: oracle start vector ({smp.t_start:.1f}s) + 1 hierarchy build ({smp.t_build:.1f}s) + "
              f"1 W-cycle ({tw:.1f}s); per step: 1 V-cycle on the full graph (mean {tv:.2f}s); "
              f"extrapolated to {est:.0f}s per solve with the oracle's counts of its recorded full solve "
              f"of {c['from']}: {c['builds']} builds, {c['cycles']} cycles ({c['wcycles']} W)")
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
           "warmup": a.warmup, "ms_per_step": 1e3 * est, "higher_is_better": True,
           "impl": "reference", "dtype": "f64", "data": "synthetic", "extrapolated": True,
           "measured_seconds": {"setup": t_setup, "steps": sum(step_s)},
           "config": {"workload": workload_label(a.workload), "n": g.n, "nnz": g.nnz, "form": "oracle fp64"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "host": _host_cpu(),
                            "extrapolated": True, "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def multi_rhs_leg(dg, g, b_host, params, net, dev, k=8):
    """Several right-hand sides of the workload's operator (pcamg_solve_multi):
    an adaptive solve builds the hierarchies, then k new columns are solved in
    one batch (flexible CG per column, Alg. 2's composite over every hierarchy)
    and the same columns one at a time (batches of one), timed with CUDA events."""
    import numpy as np
    import torch
    from paper_1806_07028_gb300 import Solver, inputs as I
    params.outer = 1
    s = Solver(dg, params=params, device=dev, mpnn=net)
    s.solve(torch.as_tensor(b_host, device=dev))
    B = torch.stack([torch.as_tensor(I.rhs_normal(g.n, 500 + c), device=dev) for c in range(k)], 1)
    s.solve_multi(B[:, :1])   # warm-up: batched buffers and kernels
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize()
    ev[0].record()
    X, sm = s.solve_multi(B)
    ev[1].record()
    torch.cuda.synchronize()
    batched = ev[0].elapsed_time(ev[1])
    one, iters_one = 0.0, []
    for c in range(k):
        ev[0].record()
        x1, s1 = s.solve_multi(B[:, c:c + 1])
        ev[1].record()
        torch.cuda.synchronize()
        one += ev[0].elapsed_time(ev[1])
        iters_one.append(int(s1["iters"][0]))
    A = g.to_scipy()
    Xh = X.cpu().numpy()
    rel = [float(np.linalg.norm(B[:, c].cpu().numpy() - A @ Xh[:, c]) / np.linalg.norm(B[:, c].cpu().numpy()))
           for c in range(k)]
    out = {"k": k, "hierarchies": s.num_hierarchies, "status": sm["status"],
           "iters": [int(v) for v in sm["iters"]], "rel_res_host_check": rel,
           "batched_ms": batched, "one_at_a_time_ms": one, "iters_one_at_a_time": iters_one,
           "speedup_batched": one / batched, "unknowns_per_s_batched": k * g.n / (batched / 1e3)}
    s.close()
    return out


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
