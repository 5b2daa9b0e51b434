#!/usr/bin/env python
"""Benchmark of the compact fourth-order Maxwell scheme on GB300.

One benchmark step = one full time step of the scheme (Step 1 + Step 2, every kernel of the
hot path) on the 2048 x 2048 2D TM_z cavity with 8 seeded modes (the configuration the
cell-updates/s metric is quoted on).  The default run is the whole 4000-step workload.

Output: one JSON line (rank 0).  `value` = cell-updates/s over all ranks, where one
cell-update is one Yee cell advanced one full step.  L2 is flushed (256 MB write) between
timed steps; each step is timed with CUDA events on the grid's stream.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32_refined|fp64]
  python bench.py --impl reference ...   # the FP64 CPU oracle on the host cores
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

WORKLOAD = "2D TM_z PEC cavity 2048x2048 cells, 8 seeded modes (m,n in [1,40], N(0,1) amplitudes, seed 0), r=0.5"
FALLBACK_HBM_GBS = 6800.0
# FP64 ALU peak of GB300: 152 SMs x 2 FP64 FMA/clk/SM x 2 flop x 2070 MHz (measured 1.19 TF/s)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=None)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--precision", default="fp32_refined", choices=["fp32_refined", "fp64"])
    p.add_argument("--closure", default="paper", choices=["paper", "reflect"])
    p.add_argument("--no-extras", action="store_true", help="skip the e2e, FP64 and CPU legs")
    p.add_argument("--only-3d", type=int, default=None, metavar="STEPS",
                   help="run only the 3D leg (FP32_REFINED, STEPS steps) and print its JSON (profiling)")
    p.add_argument("--only-reverse", type=int, default=None, metavar="STEPS",
                   help="run only the gradient workload (1024^2, STEPS forward and reverse steps) and print its "
                        "JSON (profiling)")
    p.add_argument("--only-sources", type=int, default=None, metavar="STEPS",
                   help="run only the FP32_REFINED 2048^2 step with two current sources (STEPS profiled "
                        "steps and STEPS graph-replayed ones) and print its JSON (profiling)")
    p.add_argument("--only-batched", type=int, default=None, metavar="STEPS",
                   help="run only the batch leg (512 uneven cavities, autotuned plan, STEPS timed steps) and print "
                        "its JSON (profiling)")
    p.add_argument("--only-variants", action="store_true",
                   help="run only the step-variants leg (sources, wall sources, tracked Delta E; FP64 and "
                        "FP32_REFINED) and print its JSON (profiling)")
    return p.parse_args()


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def job_step_ms(ms_local: float, dist, device) -> float:
    """The job's time per step: the slowest rank's (max over ranks); replicas run in lock step
    between the barriers that bracket the timed region."""
    if dist is None:
        return ms_local
    import torch

    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(ws: int, cells_per_rank: int, ms_step: float) -> float:
    """Whole-job cell-updates/s: every rank advances its own replica of cells_per_rank cells."""
    return ws * cells_per_rank / (ms_step * 1e-3)


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def bf16_peak():
    """Dense bf16 tensor peak of the pod (burst), TFLOP/s; the recipe's fallback if unmeasured."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"])
    except (OSError, KeyError, ValueError):
        return 1900.0


# source files that define each kernel kind reported by ms_step_profiled
KIND_SOURCES = {
    "curl32": ["k_tiled.cu", "k_tiled.cuh"], "solve32": ["k_tiled.cu", "k_tiled.cuh"],
    "filter64": ["k_fp64.cu", "k_fp64.cuh"], "pade64": ["k_fp64.cu", "k_fp64.cuh"],
    "filt3d32": ["grid3d.cu", "grid3d.cuh"], "band3d32": ["grid3d.cu", "grid3d.cuh"],
    "term3d32": ["grid3d.cu", "grid3d.cuh"], "tsgemm": ["k_transform.cu", "k_transform.cuh"],
    "sweep3d32": ["grid3d.cu", "grid3d.cuh"],
    "p1sweep64": ["k_fp64.cu", "k_fp64.cuh"], "yee64": ["k_fp64.cu", "k_fp64.cuh"],
}


def _code_only(text: str) -> str:
    """C/CUDA source without comments and blank lines (so that a comment edit keeps the hash)."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    lines = [re.sub(r"//.*$", "", l).rstrip() for l in text.splitlines()]
    return "\n".join(l for l in lines if l.strip())


def kernel_sources_hash(kind: str):
    """Hash of the code (not the comments) of the files that define a kernel kind."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2306_17263_gb300", "csrc")
    for f in KIND_SOURCES.get(kind, []):
        with open(os.path.join(csrc, f), encoding="utf-8") as fh:
            h.update(f.encode() + _code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def ncu_traffic(kind: str):
    """DRAM bytes per launch of `kind` from the committed ncu summary, if it was taken on the
    current sources of that kernel (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    e = d.get(kind)
    if not e or e.get("sources_sha") != kernel_sources_hash(kind):
        return None
    return float(e["dram_bytes_per_launch"])


# ---------------------------------------------------------------------------------------
def oracle_rate(n: int, steps: int, modes, time_budget: float = None):
    """Cell-updates/s of the FP64 CPU oracle (1 thread) on an n x n grid."""
    import oracle
    o = oracle.Oracle2D(n, 0.5)
    ez, hx, hy = o.init_modes([m for m in modes if m[0] < n and m[1] < n] or [(1, 1, 1.0)])
    done, t0 = 0, time.perf_counter()
    while done < steps:
        o.step(ez, hx, hy)
        done += 1
        if time_budget is not None and time.perf_counter() - t0 > time_budget:
            break
    dt = time.perf_counter() - t0
    return n * n * done / dt, done, dt


def _oracle_worker(job):
    """One host process: the oracle on its own n x n copy of the workload for `steps` steps (or
    until `budget` seconds have passed).  Returns (cell-updates, seconds)."""
    n, steps, modes, budget = job
    sys.path.insert(0, ROOT)
    v, done, dt = oracle_rate(n, steps, modes, time_budget=budget)
    return n * n * done, dt


def host_info():
    """Host core count and CPU model (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.split(":")[0].strip() in ("Model name", "Model"):
                model = ln.split(":", 1)[1].strip()
                if ln.startswith("Model name"):
                    break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            for ln in open("/proc/cpuinfo"):
                if ln.lower().startswith("model name"):
                    model = ln.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return os.cpu_count() or 1, model or "unknown"


def oracle_all_cores(n: int, steps: int, modes, budget: float, procs: int):
    """The oracle as it stands on every host core: `procs` independent processes (spawned, so none
    inherits a CUDA context), each stepping its own copy of an n x n sample.  Returns
    (cell-updates/s over all processes, cell-updates, wall seconds)."""
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        pool.map(_oracle_worker, [(64, 1, modes, None)] * procs)  # start-up outside the timing
        t0 = time.perf_counter()
        res = pool.map(_oracle_worker, [(n, steps, modes, budget)] * procs)
        wall = time.perf_counter() - t0
    cells = sum(c for c, _ in res)
    return cells / wall, cells, wall


def run_reference(args, ws, rank):
    """The reference arm: the FP64 CPU oracle as it stands, on the host cores."""
    if rank != 0:
        return 0
    cfg = workloads.config2()
    K = args.steps if args.steps is not None else 20
    W = args.warmup
    # each step is one oracle step on an n_s x n_s sample of the workload; n_s keeps the run
    # within about two minutes (an oracle step costs ~0.45 us per cell on one core)
    # one oracle process per host core, each on its own n_s x n_s copy (the oracle is one thread);
    # an oracle step costs ~0.45 us per cell on one core, more when every core shares the memory
    ncores, model = host_info()
    n_s = int(min(2048, max(64, math.sqrt(100.0 / (max(K + W, 1) * 0.9e-6)))))
    n_s -= n_s % 32
    if W:
        oracle_all_cores(n_s, W, cfg["modes"], None, ncores)
    value, cells, wall = oracle_all_cores(n_s, K, cfg["modes"], None, ncores)
    line = {
        "impl": "reference", "metric": "cell-updates/s", "value": value, "unit": "cell-updates/s",
        "n_gpus": args.gpus, "steps": K, "warmup": W, "ms_per_step": 1e3 * wall / max(K, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample_n": n_s, "precision": "fp64 (CPU oracle)"},
        "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": ncores, "cpu_model": model,
                         "kind": "oracle",
                         "sample": f"{ncores} oracle processes, one per host core, each {K} steps on its own "
                                   f"{n_s}x{n_s} grid of the same workload"},
        "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------------------
def batched_leg(pkg, torch, steps: int = 64):
    """512 cavities of sides 64..768 (4 seeded modes each) advanced by one launch per kernel, with
    the launch plan chosen by the batch autotuner (and the default plan's rate beside it); the state
    (2.7 GB) is far larger than L2, so no flush is needed between steps."""
    c = workloads.config4()

    def timed(b):
        b.run(16)  # warm-up (also captures the graph)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        b.run(steps)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    with pkg.Batch(c["sizes"], c["r"], stream="torch") as b:
        count, cells, launches = b.info()
        t0 = time.perf_counter()
        plan, cached = b.autotune(16)  # on the zero state, before the fields are set
        tune_s = time.perf_counter() - t0
        for k in range(count):
            b.init_modes(k, c["modes"][k])
        ms = timed(b)
        err = b.error_vs_exact(count - 1, c["modes"][count - 1])
        b.set_plan(0, 16, 0)
        ms_default = timed(b)
    return {"workload": "512 cavities, sides uniform in {64,96,...,768} (seed 0), 4 modes each, r=0.5, FP32_REFINED",
            "cells_per_step": cells, "launches_per_step": launches, "steps": steps, "ms_per_step": ms,
            "value": cells / (ms * 1e-3), "unit": "cell-updates/s",
            "plan": {"order": plan[0], "steps_per_graph": plan[1], "persistent": plan[2], "from_cache": cached,
                     "autotune_s": tune_s},
            "default_plan_value": cells / (ms_default * 1e-3),
            "l2_rel_last_cavity": err[1]}


def reverse_leg(pkg, torch, steps=None):
    """Gradient workload: 1024^2 cells, 2000 steps, Taylor-initialised random field; the FP32_REFINED
    forward run, the FP32 reverse pass (float-float adjoint state, the grid's default) and the FP64
    reverse pass on the same grid, each timed with CUDA events, and the two gradients compared."""
    c = workloads.config5()
    n, K = c["n"], steps or c["steps"]
    g = pkg.Grid(n, c["r"], precision=pkg.FP32_REFINED, stream="torch")
    ez0 = torch.tensor(workloads.sine_series_field(n, c["ell"], c["ez0_seed"]), device="cuda")
    lam = torch.zeros_like(ez0)
    out32, out64 = torch.empty_like(ez0), torch.empty_like(ez0)
    lam[1:-1, 1:-1] = torch.tensor(workloads.sine_series_field(n, c["ell"], c["direction_seeds"][0]),
                                   device="cuda")[1:-1, 1:-1]
    g.taylor_init_device(ez0)
    g.run(16)
    g.adjoint_run_device(16, lam, out32)  # builds the graphs of the FP32 reverse pass
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    ev[0].record()
    g.taylor_init_device(ez0)
    g.run(K)
    ev[1].record()
    ev[2].record()
    g.adjoint_run_device(K, lam, out32)
    ev[3].record()
    g.set_adjoint_precision(pkg.FP64)
    g.adjoint_run_device(16, lam, out64)  # builds the FP64 graphs and tables
    torch.cuda.synchronize()
    ev[4].record()
    g.adjoint_run_device(K, lam, out64)
    ev[5].record()
    torch.cuda.synchronize()
    fwd_ms, rev_ms, rev64_ms = ev[0].elapsed_time(ev[1]), ev[2].elapsed_time(ev[3]), ev[4].elapsed_time(ev[5])
    g.close()
    ok = bool(torch.isfinite(out32).all().item())
    rel = float(torch.linalg.norm(out32 - out64) / torch.linalg.norm(out64))
    return {"workload": "1024x1024 cells, 2000 steps, Gaussian random field E_z^0 (correlation length 0.05), "
                        "H^(1/2) by Taylor series", "forward_precision": "fp32_refined",
            "reverse_precision": "fp32 (float-float adjoint state)",
            "forward_ms": fwd_ms, "reverse_ms": rev_ms, "reverse_fp64_ms": rev64_ms,
            "forward_value": n * n * K / (fwd_ms * 1e-3), "reverse_value": n * n * K / (rev_ms * 1e-3),
            "reverse_fp64_value": n * n * K / (rev64_ms * 1e-3), "unit": "cell-updates/s", "finite": ok,
            "gradient_rel_diff_fp32_vs_fp64_reverse": rel,
            "memory": "no trajectory stored: the step is linear, the reverse pass needs only the final adjoint"}


def _profiled_rate(pkg, torch, g, n, K, flush):
    """Mean step time of K profiled steps (each kernel timed with CUDA events on the grid's stream,
    launched one by one, L2 flushed between steps) and the share of the source kernels; then K steps
    replayed from the captured graph (ms_run, as a user runs them), timed with CUDA events around the
    replay (no flush inside it)."""
    for _ in range(3):
        g.step_profiled()
    tot, src = 0.0, 0.0
    for _ in range(K):
        for kind, ms, _ in g.step_profiled():
            tot += ms
            if kind == "source":
                src += ms
        flush.zero_()
    g.run(K)  # captures the graph
    flush.zero_()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    g.run(K)
    ev[1].record()
    torch.cuda.synchronize()
    graph_ms = ev[0].elapsed_time(ev[1]) / K
    return {"steps": K, "ms_per_step": tot / K, "value": n * n / (tot / K * 1e-3), "unit": "cell-updates/s",
            "source_kernel_share": src / tot, "graph_ms_per_step": graph_ms,
            "graph_value": n * n / (graph_ms * 1e-3)}


SOURCES = [(2, 3, 1.0, 5.0), (1, 1, -0.5, 11.0)]  # (m, n, amplitude, omega) of J_z = a sin sin sin(w t)


def sources_leg(pkg, torch, r, steps, flush):
    """FP32_REFINED 2048^2 step with two sine-mode current sources, from their driven solution."""
    with pkg.Grid(2048, r, z=1.3, precision=pkg.FP32_REFINED, stream="torch") as g:
        g.set_sources(SOURCES)
        g.init_driven(SOURCES)
        res = _profiled_rate(pkg, torch, g, 2048, steps, flush)
        res["l2_rel_vs_driven"] = g.error_vs_driven(SOURCES)[1]
    return res


def variants_leg(pkg, torch, modes, r):
    """The step variants: current sources (sine modes, both precisions, 2048^2), currents that do not
    vanish on the walls (FP64, 1024^2, against the same FP64 step without sources) and the tracked-DE
    step as printed in Sec. 3.4 (FP64, 1024^2)."""
    import numpy as np

    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    out = {}
    with pkg.Grid(2048, r, z=1.3, precision=pkg.FP32_REFINED, stream="torch") as g:
        g.init_modes(modes)
        out["plain_fp32_refined_2048"] = _profiled_rate(pkg, torch, g, 2048, 200, flush)
    out["sources_fp32_refined_2048"] = sources_leg(pkg, torch, r, 200, flush)
    # a current that does not vanish on y = 0, 1 and is compatible at the corners:
    # J_z = (1/(4w)) sin(w t) (w^2 + (4 pi^2 - w^2) cos 2 pi x + (4 pi^2 - w^2) cos 2 pi y
    #                          + (w^2 - 8 pi^2) cos 2 pi x cos 2 pi y)
    w, p2 = 3.0, math.pi ** 2
    wall = [(0, 0, w / 4, w, 1, 1), (2, 0, (4 * p2 - w * w) / (4 * w), w, 1, 1),
            (0, 2, (4 * p2 - w * w) / (4 * w), w, 1, 1), (2, 2, (w * w - 8 * p2) / (4 * w), w, 1, 1)]
    for key, rows in (("plain_fp64_1024", None), ("wall_sources_fp64_1024", wall)):
        with pkg.Grid(1024, r, precision=pkg.FP64, stream="torch") as g:
            g.init_modes(modes)
            if rows:
                g.set_sources_xy(rows)
            out[key] = _profiled_rate(pkg, torch, g, 1024, 50, flush)
            out[key]["finite"] = bool(all(np.isfinite(a).all() for a in g.get_fields()))
    with pkg.Grid(1024, r, precision=pkg.FP64, scheme=pkg.SCHEME_C4_DE, stream="torch") as g:
        g.init_modes(modes)
        out["tracked_de_fp64_1024"] = _profiled_rate(pkg, torch, g, 1024, 50, flush)
        out["tracked_de_fp64_1024"]["l2_rel"] = g.error_vs_exact(modes)[1]
    with pkg.Grid(2048, r, z=1.3, precision=pkg.FP32_REFINED, scheme=pkg.SCHEME_C4_DE, stream="torch") as g:
        g.init_modes(modes)
        out["tracked_de_fp32_refined_2048"] = _profiled_rate(pkg, torch, g, 2048, 200, flush)
        out["tracked_de_fp32_refined_2048"]["l2_rel"] = g.error_vs_exact(modes)[1]
    del flush
    return out


def leg_3d(pkg, torch, steps32=None, with_fp64=True):
    """3D six-component workload: 256^3 cells, r = 0.4, 500 steps, 2 seeded modes, FP32_REFINED
    (every step timed with CUDA events; the 6-component state, 0.8 GB, exceeds L2), plus 20 FP64
    steps for the FP64-vs-refined comparison."""
    c = workloads.config3()
    n, r, modes, K = c["n"], c["r"], c["modes"], c["steps"]
    out = {"workload": "3D PEC cube 256^3 cells, modes (2,3,1) + one seeded mode (indices in [1,16]), r=0.4",
           "unit": "cell-updates/s", "l2": "state 0.8 GB > L2; no flush"}
    legs = [(pkg.FP32_REFINED, steps32 or K, "fp32_refined", pkg.SOLVER_RICHARDSON),
            (pkg.FP32_REFINED, min(steps32 or K, 50), "fp32_refined_transform_tc", pkg.SOLVER_TRANSFORM_TC)]
    legs += [(pkg.FP64, 20, "fp64", pkg.SOLVER_RICHARDSON)] if with_fp64 else []
    for prec, steps, key, solver in legs:
        g = pkg.Grid(n, r, precision=prec, dim=3, stream="torch")
        if solver != pkg.SOLVER_RICHARDSON:
            g.set_solver(solver)
        g.init_modes(modes)
        for _ in range(3):
            g.step_profiled()
        g.init_modes(modes)
        total, per = 0.0, {}
        for _ in range(steps):
            for kind, ms, nbytes in g.step_profiled():
                total += ms
                a = per.setdefault(kind, [0, 0.0, 0.0])
                a[0] += 1
                a[1] += ms
                a[2] += nbytes
        l2_abs, l2_rel, _, _ = g.error_vs_exact(modes)
        kinds = {k: {"launches": v[0], "ms_total": v[1], "share": v[1] / total, "GBps": v[2] / (v[1] * 1e-3) / 1e9}
                 for k, v in sorted(per.items(), key=lambda kv: -kv[1][1])}
        out[key] = {"steps": steps, "ms_per_step": total / steps, "value": n ** 3 * steps / (total * 1e-3),
                    "l2_abs": l2_abs, "l2_rel": l2_rel, "launches_per_step": g.launches_per_step, "kernels": kinds,
                    "step_roofline": {"bytes_per_step": 96.0 * n ** 3,
                                      "achieved_GBps": 96.0 * n ** 3 / (total / steps * 1e-3) / 1e9,
                                      "bytes": "96 B per cell-update (6 components, hi+lo, read + write)"}}
        if "tsgemm" in per:
            P = -(-n // 128) * 128
            cnt, ms_tot = per["tsgemm"][0], per["tsgemm"][1]
            flops = 6.0 * P ** 4  # three bf16 products of a P x P transform over P^3 points
            tflops = flops / (ms_tot / cnt * 1e-3) / 1e12
            out[key]["tensor"] = {"kernel": "tsgemm", "flop_per_launch": flops, "avg_launch_ms": ms_tot / cnt,
                                  "achieved_tflops": tflops, "peak_tflops": bf16_peak(), "frac": tflops / bf16_peak(),
                                  "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst)"}
        g.close()
    return out


def wavenumber_mae(pkg, k: int, scheme, N: int = 64, r: float = 0.5, T: float = 4.0 / math.sqrt(2.0)):
    """Mean absolute error of Sec. 5.1 for the single mode k_x = k_y = k at h = 1/N after
    round(T / h_tau) steps: the sum of |u - u_exact| over all stored points and steps, divided by
    3 n_steps N^2; per-step sums from ms_error_vs_exact."""
    modes = [(k, k, 1.0)]
    with pkg.Grid(N, r, precision=pkg.FP64, scheme=scheme) as g:
        g.init_modes(modes)
        K = int(round(T / g.ht))
        acc = 0.0
        for _ in range(K):
            g.step()
            acc += g.error_vs_exact(modes)[3]
    return acc / (3.0 * K * N * N), K


def wavenumber_leg(pkg):
    """Error against wavenumber at h = 1/64 (the setting of Fig. "fig:error(k)": k_x = k_y = k,
    T = 4/sqrt(2), Z = 1), points per wavelength 2N/k from 64 (k = 2) to 2.56 (k = 50); compact
    scheme, the non-compact fourth-order comparator NC and plain Yee, FP64."""
    ks = list(range(2, 51, 2))
    c4 = [wavenumber_mae(pkg, k, pkg.SCHEME_C4)[0] for k in ks]
    yee = [wavenumber_mae(pkg, k, pkg.SCHEME_YEE2)[0] for k in ks]
    nc = [wavenumber_mae(pkg, k, pkg.SCHEME_NC4)[0] for k in ks]
    return {"N": 64, "r": 0.5, "T": 4.0 / math.sqrt(2.0), "k": ks, "ppw": [128.0 / k for k in ks],
            "mae_c4": c4, "mae_nc": nc, "mae_yee": yee}


def accuracy_leg(pkg, torch, cfg, closure):
    """The whole 4000-step workload (T = 0.9765625) in FP32_REFINED and in FP64, each replayed from
    its captured graph and timed with CUDA events: the L2 errors against the exact modes at T and
    the distance between the two states (the mixed-path criterion: e32 <= 2 e64 and
    |u32 - u64| <= e64; the FP64 path is the oracle's parity-pinned stand-in at this size)."""
    import numpy as np

    N, r, modes, K = cfg["n"], cfg["r"], cfg["modes"], cfg["steps"]
    out, fields = {}, {}
    for prec, key in ((pkg.FP32_REFINED, "fp32_refined"), (pkg.FP64, "fp64")):
        with pkg.Grid(N, r, precision=prec, closure=closure, stream="torch") as g:
            g.init_modes(modes)
            g.run(17)  # captures the 16-step and 1-step graphs
            g.init_modes(modes)
            torch.cuda.synchronize()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record()
            g.run(K)
            ev[1].record()
            torch.cuda.synchronize()
            ms = ev[0].elapsed_time(ev[1])
            l2_abs, l2_rel, max_abs, _ = g.error_vs_exact(modes)
            fields[key] = g.get_fields()
            out[key] = {"l2_abs": l2_abs, "l2_rel": l2_rel, "max_abs": max_abs, "ms_per_step": ms / K,
                        "value": N * N * K / (ms * 1e-3), "unit": "cell-updates/s"}
    diff = math.sqrt(sum(float(np.sum((a - b) ** 2)) for a, b in zip(fields["fp32_refined"], fields["fp64"])) / N ** 2)
    e32, e64 = out["fp32_refined"]["l2_abs"], out["fp64"]["l2_abs"]
    out.update({"t": K * r / N, "steps": K, "l2_fp32_vs_fp64": diff, "mixed_criterion_holds": bool(e32 <= 2 * e64 and diff <= e64),
                "timing": "graph replay of all 4000 steps, CUDA events, no L2 flush (state 100 MB in FP32_REFINED)"})
    return out


def yee_leg(pkg, torch, modes, r, c4_l2_abs, c4_value, T=4000 * 0.5 / 2048):
    """Plain second-order Yee (FP64) on the same modes and end time: its L2 error at three
    resolutions, the fitted order, and the resolution and time-to-solution it would need to
    reach the compact scheme's error (extrapolated from the measured error and rate)."""
    errs, rates = [], []
    for n in (512, 1024, 2048):
        steps = int(round(T * n / r))
        with pkg.Grid(n, r, scheme=pkg.SCHEME_YEE2, stream="torch") as g:
            g.init_modes(modes)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            g.run(steps)
            e1.record()
            torch.cuda.synchronize()
            rates.append(n * n * steps / (e0.elapsed_time(e1) * 1e-3))
            errs.append(g.error_vs_exact(modes)[0])
    order = math.log2(errs[1] / errs[2])
    n_eq = 2048 * (errs[2] / c4_l2_abs) ** (1.0 / max(order, 1e-3))
    # cost of a run to time T: n^2 cells x (T n / r) steps at the measured 2048^2 rate
    t_yee = n_eq ** 3 * T / r / rates[2]
    t_c4 = 2048 ** 3 * T / r / c4_value
    return {"t": T, "l2_abs": dict(zip(("512", "1024", "2048"), errs)), "order": order,
            "value_2048": rates[2], "unit": "cell-updates/s", "c4_l2_abs_2048": c4_l2_abs,
            "n_for_equal_error": n_eq, "time_to_solution_s": {"yee_extrapolated": t_yee, "c4_measured": t_c4}}


def run_ours(args, ws, rank, local):
    import numpy as np
    import torch

    import paper_2306_17263_gb300 as pkg

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    # one non-default stream for the grid and every torch op (the L2 flush), so they are ordered
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist:
            dist.barrier()

    cfg = workloads.config2()
    N, r, modes = cfg["n"], cfg["r"], cfg["modes"]
    K = args.steps if args.steps is not None else cfg["steps"]
    W = max(3, args.warmup)
    prec = pkg.FP32_REFINED if args.precision == "fp32_refined" else pkg.FP64
    closure = pkg.CLOSURE_PAPER if args.closure == "paper" else pkg.CLOSURE_REFLECT
    g = pkg.Grid(N, r, precision=prec, closure=closure, stream="torch")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > 129 MB L2

    g.init_modes(modes)
    for _ in range(W):
        g.step_profiled()
        flush.zero_()
    g.init_modes(modes)  # the timed steps are the workload from t = 0
    torch.cuda.synchronize()
    barrier()

    clocks = ClockSampler(local)
    clocks.start()
    total_ms = 0.0
    per_kind = {}
    launches = 0
    t_wall = time.perf_counter()
    for _ in range(K):
        prof = g.step_profiled()
        launches += len(prof)
        for kind, ms, nbytes in prof:
            total_ms += ms
            a = per_kind.setdefault(kind, [0, 0.0, 0.0])
            a[0] += 1
            a[1] += ms
            a[2] += nbytes
        flush.zero_()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    barrier()
    ms_step = job_step_ms(total_ms / K, dist, "cuda")
    value = job_value(ws, N * N, ms_step)

    l2_abs, l2_rel, max_abs, _ = g.error_vs_exact(modes)

    # dominant kernel and its roofline
    dom = max(per_kind.items(), key=lambda kv: kv[1][1])
    kind, (cnt, kms, kbytes) = dom
    avg_ms = kms / cnt
    bytes_per_launch = kbytes / cnt
    hbm, hbm_src = measured_peaks()
    achieved_gbs = bytes_per_launch / (avg_ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm, "unit": "GB/s",
                "frac": achieved_gbs / hbm, "traffic": ncu_traffic(kind), "kernel": kind,
                "peak_source": f"{hbm_src} (MEASURED_PEAKS.json hbm_gbs)" if hbm_src == "measured" else "fallback",
                "bytes_per_launch": bytes_per_launch, "avg_launch_ms": avg_ms,
                "bytes": "state bytes the launch must move: 8 B per float-float (or FP64) point read or written"}
    # whole step on the algorithmic bytes: every state component read and written once, 48 B per cell
    step_bytes = 48.0 * N * N
    step_gbs = step_bytes / (ms_step * 1e-3) / 1e9
    step_roofline = {"achieved": step_gbs, "peak": hbm, "unit": "GB/s", "frac": step_gbs / hbm,
                     "bytes_per_step": step_bytes, "bytes": "48 B per cell-update (3 components, hi+lo, read + write)"}
    # bytes the four-launch FP32_REFINED step moves by design, right-hand-side planes b included
    ne, nh = (N + 1.0) ** 2, N * (N + 1.0)
    traffic_model = {"curl_step1": 16 * nh + 4 * ne, "solve_E": 4 * ne + 16 * ne, "curl_step2": 8 * ne + 8 * nh,
                     "solve_H": 8 * nh + 32 * nh}
    traffic_model["per_step"] = sum(traffic_model.values())
    traffic_model["what"] = "bytes per launch if every array a launch reads or writes (state hi/lo and b) moves once"
    kernels = {k: {"launches": v[0], "ms_total": v[1], "share": v[1] / total_ms, "GBps": v[2] / (v[1] * 1e-3) / 1e9}
               for k, v in sorted(per_kind.items(), key=lambda kv: -kv[1][1])}

    line = {
        "metric": "cell-updates/s", "value": value, "unit": "cell-updates/s", "n_gpus": ws, "steps": K,
        "warmup": W, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if prec == pkg.FP32_REFINED else "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": N, "r": r, "precision": args.precision, "closure": args.closure,
                   "l2": "flushed between timed steps (256 MB write); each step timed with CUDA events",
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "gpu_launches": launches,
        "roofline": roofline,
        "step_roofline": step_roofline,
        "traffic_model": traffic_model if prec == pkg.FP32_REFINED else None,
        "kernels": kernels,
        "accuracy": {"t": K * r / N, "l2_abs": l2_abs, "l2_rel": l2_rel, "max_abs": max_abs},
        "clocks": clk,
        "wall_s_timed_loop": wall,
    }

    if not args.no_extras and rank == 0:
        # end to end through the C ABI with pinned host buffers: upload E^0, H^{1/2}, run K steps,
        # download the final fields
        shapes = g.shapes()
        host_in = [torch.empty(s, dtype=torch.float64, pin_memory=True) for s in shapes]
        host_out = [torch.empty(s, dtype=torch.float64, pin_memory=True) for s in shapes]
        g.init_modes(modes)
        L = pkg.load()
        ptr_in = pkg._ptrs([t.data_ptr() for t in host_in])
        ptr_out = pkg._ptrs([t.data_ptr() for t in host_out])
        pkg._check(L.ms_get_fields(g._h, ptr_in))
        pkg._check(L.ms_run(g._h, 17))  # captures the step graphs outside the timed region
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pkg._check(L.ms_set_fields(g._h, ptr_in, 0))
        pkg._check(L.ms_run(g._h, K))
        pkg._check(L.ms_get_fields(g._h, ptr_out))
        e2e_s = time.perf_counter() - t0
        nbytes = sum(t.numel() * 8 for t in host_in)
        line["e2e"] = {"value": N * N * K / e2e_s, "unit": "cell-updates/s", "h2d_bytes_per_step": nbytes / K,
                       "d2h_bytes_per_step": nbytes / K, "seconds": e2e_s,
                       "what": "ms_set_fields (host) + ms_run(K) (graph replay, graphs captured beforehand, "
                               "no L2 flush) + ms_get_fields (host)"}
        # the whole workload in both precisions: errors at T, the mixed-path criterion, and the FP64
        # GPU form's rate on the same workload
        acc = accuracy_leg(pkg, torch, cfg, closure)
        line["accuracy_at_T"] = acc
        line["fp64_gpu"] = {"value": acc["fp64"]["value"], "unit": "cell-updates/s", "steps": cfg["steps"],
                            "ms_per_step": acc["fp64"]["ms_per_step"], "timing": acc["timing"]}
        line["batched"] = batched_leg(pkg, torch)
        line["reverse_pass"] = reverse_leg(pkg, torch)
        line["three_d"] = leg_3d(pkg, torch)
        line["error_vs_wavenumber"] = wavenumber_leg(pkg)
        line["yee_equal_error"] = yee_leg(pkg, torch, modes, r, acc["fp32_refined"]["l2_abs"], value)
        line["variants"] = variants_leg(pkg, torch, modes, r)
        # CPU oracle on a bounded sample of the workload (rank 0): every host core, one oracle process
        # per core on its own copy of the full 2048^2 grid, and one core alone
        ncores, model = host_info()
        v_all, cells_all, wall_all = oracle_all_cores(N, 1000, modes, 10.0, ncores)
        v1, done, dt = oracle_rate(N, 1000, modes, time_budget=8.0)
        line["cpu_baseline"] = {"value": v_all, "unit": "cell-updates/s", "cores": ncores, "cpu_model": model,
                                "kind": "oracle",
                                "sample": f"{ncores} oracle processes (one per core), each stepping its own full "
                                          f"2048x2048 grid for ~10 s: {cells_all / N ** 2:.0f} steps in {wall_all:.1f} s",
                                "one_core": {"value": v1, "sample": f"{done} oracle steps ({dt:.1f} s) on one core"}}
    g.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    ws, rank, local = dist_info()
    if args.only_3d is not None:
        import torch

        import paper_2306_17263_gb300 as pkg
        torch.cuda.set_device(local)
        torch.cuda.set_stream(torch.cuda.Stream())
        print(json.dumps(leg_3d(pkg, torch, steps32=args.only_3d, with_fp64=False)), flush=True)
        return 0
    if args.only_reverse is not None:
        import torch

        import paper_2306_17263_gb300 as pkg
        torch.cuda.set_device(local)
        torch.cuda.set_stream(torch.cuda.Stream())
        print(json.dumps(reverse_leg(pkg, torch, steps=args.only_reverse)), flush=True)
        return 0
    if args.only_sources is not None:
        import torch

        import paper_2306_17263_gb300 as pkg
        torch.cuda.set_device(local)
        torch.cuda.set_stream(torch.cuda.Stream())
        flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
        print(json.dumps(sources_leg(pkg, torch, workloads.config2()["r"], args.only_sources, flush)), flush=True)
        return 0
    if args.only_batched is not None or args.only_variants:
        import torch

        import paper_2306_17263_gb300 as pkg
        torch.cuda.set_device(local)
        torch.cuda.set_stream(torch.cuda.Stream())
        if args.only_batched is not None:
            print(json.dumps(batched_leg(pkg, torch, steps=args.only_batched)), flush=True)
        else:
            c = workloads.config2()
            print(json.dumps(variants_leg(pkg, torch, c["modes"], c["r"])), flush=True)
        return 0
    if args.impl == "reference":
        return run_reference(args, ws, rank)
    return run_ours(args, ws, rank, local)


if __name__ == "__main__":
    sys.exit(main())
