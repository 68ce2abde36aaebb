#!/usr/bin/env python
"""Throughput benchmark of the fused D2Q9 TRT-RLB step on GB300.

Default workload: the double shear layer (Sec. III A) of the three Reynolds
numbers Re = 1e4, 1e5, 1e7 (kappa = 80, delta = 0.05, u_c = 0.04,
tau_{s,2} = 0.625), each on a 4096 x 4096 periodic lattice, FP32 storage, lagged
G.  One benchmark step is one time step of all three lattices (one batched
launch, 50.3M node updates, 4.4 GB of algorithmic traffic).  The working set
(2.6 GB of populations and Phi) is twenty times the L2, so the timed steps run
back to back with no flush: CUDA events on the launching stream bracket the K
timed steps, and the write-back of each step's dirty lines falls inside the
next one.  Beside it the line reports a 1000-step steady-state sample and the
older per-step figure with the L2 flushed before every step (outside its
events).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank advances its own replica of the workload
(weak scaling, no collective on the data path); rank 0 prints one JSON line.
The CPU baseline and the served stream are one-GPU measurements (N = 1 only).
--impl reference times the FP64 CPU oracle on the same workload on the host
cores (rank 0 only).
"""
from __future__ import annotations

import argparse
import glob
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "D2Q9 TRT-RLB MLUPS & % HBM roofline; served solves/s, p50/p99 latency"
UNIT = "MLUPS"
STORAGE_BYTES = {"f64": 8, "f32": 4, "f16": 2, "bf16": 2, "f64dw": 8}
PHI_BYTES = {"f64": 8, "f32": 4, "f16": 4, "bf16": 4, "f64dw": 8}


def workload(name: str, size=None, storage=None, g_mode: str = "lagged"):
    """(problems, storage, description) of a named workload; size "NXxNY",
    storage and the G mode override the defaults (for profiling runs)."""
    from paper_2312_10318_gb300 import workloads as W
    if name == "dsl1024":
        res = (1e4, 1e5, 1e7)
        n = 1024
        nx, ny = (n, n) if size is None else size
        probs = [W.double_shear_layer(nx, re=r) for r in res]
        if size is not None:
            probs = [_rect(p, nx, ny) for p in probs]
        st = storage or "f32"
        desc = (f"double shear layer, 3 lattices {nx}x{ny} periodic (Re 1e4, 1e5, 1e7), kappa=80, "
                f"delta=0.05, u_c=0.04, tau_s2=0.625, {st.upper()} storage, G {g_mode}")
        return probs, st, desc
    if name == "dsl4096x3":
        res = (1e4, 1e5, 1e7)
        nx, ny = (4096, 4096) if size is None else size
        probs = [W.double_shear_layer(nx, re=r) for r in res]
        if size is not None:
            probs = [_rect(p, nx, ny) for p in probs]
        st = storage or "f32"
        desc = (f"double shear layer, 3 lattices {nx}x{ny} periodic (Re 1e4, 1e5, 1e7), kappa=80, "
                f"delta=0.05, u_c=0.04, tau_s2=0.625, {st.upper()} storage, G {g_mode}")
        return probs, st, desc
    if name == "dsl4096":
        nx, ny = (4096, 4096) if size is None else size
        p = W.double_shear_layer(nx, re=1e5)
        if size is not None:
            p = _rect(p, nx, ny)
        st = storage or "f32"
        return [p], st, f"double shear layer, 1 lattice {nx}x{ny} periodic, Re 1e5, {st.upper()} storage, G {g_mode}"
    if name == "creeping4096x2048":
        # the creeping-flow configuration: a 64^2 solid square at x = 1024, moving-wall
        # inlet column, zero-gradient outlet ghosts, y periodic (mask: 1 B per node)
        nx, ny = (4096, 2048) if size is None else size
        p = W.creeping_flow(nx, ny, 64, center_x=nx // 4, re=1.0, ma=0.1)
        st = storage or "f32"
        return [p], st, (f"creeping flow past a 64x64 square, {nx}x{ny}, inlet / zero-gradient outlet, "
                         f"y periodic, Re 1 (Ma 0.1), {st.upper()} storage, G {g_mode}")
    if name == "channel4096":
        # force-driven channel with half-way walls in y (the walled kernel, no mask)
        nx, ny = (4096, 4096) if size is None else size
        p = W.poiseuille(ny, 0.8, 3.0 / 16.0, nx=nx, u_c=0.01)
        st = storage or "f32"
        return [p], st, (f"force-driven channel {nx}x{ny}, half-way walls in y, tau_s 0.8, magic 3/16, "
                         f"{st.upper()} storage, G {g_mode}")
    if name == "tg64":
        probs = [W.taylor_green(64, 0.04, 100.0, magic=0.25)]
        st = storage or "f64"
        return probs, st, f"Taylor-Green 64x64 periodic, u0=0.04, Re=100, magic 1/4, {st.upper()}, G {g_mode}"
    raise SystemExit(f"unknown workload {name}")


def _rect(p, nx, ny):
    """The problem's parameters on an nx x ny lattice (fields cut or tiled)."""
    reps = (-(-ny // p.ny), -(-nx // p.nx))
    p.ux = np.tile(p.ux, reps)[:ny, :nx].copy()
    p.uy = np.tile(p.uy, reps)[:ny, :nx].copy()
    p.nx, p.ny = nx, ny
    return p


def bytes_per_node(storage: str, g_mode: str = "lagged", mask: bool = False) -> int:
    """Algorithmic bytes of one node update: 9 populations read and written, plus
    (lagged G) two Phi values read and two written; the current-Phi kernel
    computes Phi on chip and moves populations only; a mask adds its byte."""
    b = 2 * 9 * STORAGE_BYTES[storage]
    if g_mode == "lagged":
        b += 4 * PHI_BYTES[storage]
    return b + (1 if mask else 0)


# FP64 storage runs its collision on GB300's FP64 pipe, which bounds it long
# before HBM does: its roofline is arithmetic, against the FP64 FMA throughput
# measured on the same GPU in the same run (trtrlb_fp64_fma_rate).  FP64
# operations per node update (an FMA counts two): FP64_OPS_PER_NODE, from the
# FP64 instruction counters of the step kernel (profiles/ names the capture).
FP64_OPS_PER_NODE = 135
FP64_NOMINAL_TFLOPS = 1.25


def fp64_fma_rate(stream) -> float:
    """Measured FP64 FMA throughput of the current GPU, TFLOP/s."""
    import ctypes as C
    from paper_2312_10318_gb300 import _lib
    out = C.c_double()
    _lib.check(_lib.load().trtrlb_fp64_fma_rate(C.c_void_p(stream.cuda_stream), 0.05, C.byref(out)))
    return out.value


def alu_roofline(storage: str, nodes_per_launch: float, launch_s: float, peak_tflops=None):
    """The arithmetic roofline of an FP64-storage step, or None for the formats
    whose step is bound by memory traffic."""
    if storage != "f64":
        return None
    achieved = FP64_OPS_PER_NODE * nodes_per_launch / launch_s / 1e12
    peak = peak_tflops if peak_tflops else FP64_NOMINAL_TFLOPS
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak,
            "peak_kind": "measured FP64 FMA throughput" if peak_tflops else "nominal FP64 (not measured)",
            "traffic": None, "ops_per_node": FP64_OPS_PER_NODE}


# GB300's nominal HBM3e bandwidth; the line reports its fraction beside the
# measured copy bandwidth's (the roofline's denominator).
HBM_NOMINAL_GBS = 7900.0
# GB300's L2 cache
L2_BYTES = 129 * 2 ** 20


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash(csrc: str | None = None) -> str:
    """Hash of the device-code sources (headers with the kernels and their
    launch code, and the per-format instantiation units) with comments and
    blank lines removed, so that only a change of code invalidates a capture."""
    h = hashlib.sha256()
    csrc = csrc or os.path.join(ROOT, "paper_2312_10318_gb300", "csrc")
    for p in sorted(glob.glob(os.path.join(csrc, "*.cuh")) + glob.glob(os.path.join(csrc, "lb_ops_*.cu"))):
        with open(p, encoding="utf-8") as fh:
            text = re.sub(r"/\*.*?\*/", "", fh.read(), flags=re.S)
        for line in text.splitlines():
            code = re.sub(r"//.*", "", line).rstrip()
            if code:
                h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


# step kernels by the kind the library reports for a lattice (Lattice.step_kernel)
KERNEL_NAMES = {
    "aa": "trt::k_step (fused AA stream-collide)",
    "aa_vector": "trt::k_step_vec (fused AA stream-collide)",
    "ab": "trt::k_step_ab (two-buffer step, Phi at the current level, one launch per lattice)",
    "ab_tma": "trt::k_step_ab_tma (two-buffer step fed by TMA, Phi at the current level, one launch per lattice)",
    "ab_tma_shared": "trt::k_step_ab_tma (two-buffer step fed by TMA, Phi at the current level, one launch per lattice)",
    "ab_column": "trt::k_step_ab_col (two-buffer step walking columns, Phi at the current level, one launch per lattice)",
}
BATCH_KERNEL_NAMES = {
    "aa": "trt::k_step_group (fused AA stream-collide, all lattices in one launch)",
    "aa_vector": "trt::k_step_group_vec (fused AA stream-collide, all lattices in one launch)",
    "ab_tma_shared": "trt::k_step_ab_tma (two-buffer step fed by TMA, Phi at the current level, "
                     "up to 16 lattices in one launch)",
}
TMA_GROUP_MAX = 16      # lattices per shared TMA-fed launch


def kernel_label(mode: str, kinds) -> str:
    """Name of the step kernel(s) the timed region launches, from the kinds the
    library reports for the lattices (in a batch the AA and small TMA-fed
    lattices share launches)."""
    names = []
    for k in dict.fromkeys(kinds):
        names.append(BATCH_KERNEL_NAMES.get(k, KERNEL_NAMES[k]) if mode == "batch" else KERNEL_NAMES[k])
    return " + ".join(names)


def step_launches(mode: str, kinds) -> int:
    """Step-kernel launches per time step: one per lattice outside a batch; in a
    batch one per AA kernel kind (the benchmark's lattices share format, boundary
    flavour and parity), one per TMA_GROUP_MAX lattices that share TMA-fed
    launches, and one per other two-buffer lattice."""
    kinds = list(kinds)
    if mode != "batch":
        return len(kinds)
    aa = {k for k in kinds if k in ("aa", "aa_vector")}
    shared = sum(k == "ab_tma_shared" for k in kinds)
    alone = sum(k in ("ab", "ab_tma", "ab_column") for k in kinds)
    return len(aa) + -(-shared // TMA_GROUP_MAX) + alone


def recorded_traffic(workload_name: str):
    """DRAM bytes per launch of the step kernel from a committed ncu summary, or None
    when the kernel sources changed since that capture.  workload_name is
    '<workload>/<storage>/<g mode>'."""
    pat = re.compile(r"^traffic_per_launch_bytes\[([\w/]+)\]:\s*([0-9.eE+]+)\s+source_hash:\s*(\w+)")
    for p in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        for line in open(p):
            m = pat.match(line.strip())
            if m and m.group(1) == workload_name and m.group(3) == kernel_source_hash():
                return float(m.group(2))
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        threading.Thread(target=self._read, daemon=True).start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) != 7:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[3:]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, r in rows for k in range(4) if r[k].lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x: float, dist=None, device="cuda") -> float:
    """The largest x over all ranks (the slowest replica's time); x itself
    without a process group."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput of `world` replicas that each processed
    units_per_rank units, timed by the slowest (weak scaling)."""
    return units_per_rank * world / seconds


def oracle_g_mode(g_mode: str) -> int:
    """The oracle's code of a G mode name (lagged, current, off)."""
    import oracle as O
    return {"lagged": O.G_LAGGED, "current": O.G_CURRENT, "off": O.G_OFF}[g_mode]


def cpu_baseline(problems, seconds: float = 12.0, g_mode: str = "lagged"):
    """The FP64 CPU oracle on a bounded sample of the workload: as many time steps
    of the first lattice as fit in about `seconds`."""
    import oracle as O
    pr = problems[0]
    lat = O.Lattice(O.Params(nx=pr.nx, ny=pr.ny, tau1=pr.tau_s, tau2=pr.tau_s2,
                             periodic_x=pr.periodic[0], periodic_y=pr.periodic[1],
                             gx=pr.g[0], gy=pr.g[1], wall_ux=pr.wall_u[0], wall_uy=pr.wall_u[1],
                             wall_rho=pr.wall_rho, g_mode=oracle_g_mode(g_mode)), mask=pr.mask)
    lat.init(pr.ux, pr.uy, pr.rho)
    lat.step(1)

    def rate(budget):
        n, t0 = 0, time.perf_counter()
        while time.perf_counter() - t0 < budget:
            lat.step(1)
            n += 1
        return n, time.perf_counter() - t0

    n, dt = rate(seconds)
    cores = O.num_threads()
    # the same sample on one core, then the thread count restored
    O.set_num_threads(1)
    try:
        n1, dt1 = rate(seconds / 3)
    finally:
        O.set_num_threads(cores)
    return {"value": pr.nodes * n / dt / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} time steps of one {pr.nx}x{pr.ny} lattice ({pr.name}) of the workload, "
                      f"{dt:.1f} s",
            "one_core": {"value": pr.nodes * n1 / dt1 / 1e6, "unit": UNIT,
                         "sample": f"{n1} time steps of the same lattice, {dt1:.1f} s"},
            "cpu_model": cpu_model()}


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip() + f" ({os.cpu_count()} logical CPUs)"
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip() + f" ({os.cpu_count()} logical CPUs)"
    except OSError:
        pass
    import platform
    return f"{platform.machine()} ({os.cpu_count()} logical CPUs)"


def run_serving(args) -> dict:
    """The served-stream measurement: a seeded Poisson stream of Taylor-Green,
    double-shear-layer and channel solves (sides log-uniform 64..4096, Re
    log-uniform 1..1e6, FP64/FP32/FP16 uniform), served by the continuous-batching
    server with the precision guard, and by the FP64 one-lattice-at-a-time
    reference on the same stream."""
    from paper_2312_10318_gb300 import serve as S
    lo, hi = (max(1, int(1000 * args.serve_scale)), max(2, int(20000 * args.serve_scale)))
    reqs = S.make_stream(args.serve_requests, seed=0, rate=1.0, steps_range=(lo, hi))
    work = sum(r.work for r in reqs)
    guard = S.PrecisionGuard()
    from paper_2312_10318_gb300.tune import Tuner
    tuner = Tuner(persist=False, steps=32, reps=2)
    # kernel shapes of every format a request may run in (FP64 needs none),
    # tuned before the stream starts: a deployment-time cost, like capturing graphs
    t0 = time.perf_counter()
    tuner.warm(S.shapes_of(reqs, storages=("f32", "f16") + (("f64dw",) if args.serve_fp64_as == "f64dw" else ())))
    tune_s = time.perf_counter() - t0
    # capacity: the whole stream available at once; then arrivals at the rate
    # that offers `serve_load` x that capacity (Poisson inter-arrival times of
    # the seeded stream, rescaled)
    capacity = warm_pass_s = None
    if args.serve_rate <= 0:      # a given rate needs no capacity pass
        def whole_stream_makespan():
            cal = S.Server(hbm_budget=args.serve_budget_gb * 1e9, chunk=512, guard=S.PrecisionGuard(),
                           tuner=tuner, fp64_as=args.serve_fp64_as)
            cal.run(reqs, realtime=False)
            return cal.makespan
        # an untimed pass first, like warm-up steps, so that one-time costs
        # (the first launch of each kernel variant, the first use of tens of
        # GB of device memory on the GPU) do not count as serving throughput;
        # its makespan is reported beside the capacity
        warm_pass_s = whole_stream_makespan()
        capacity = len(reqs) / whole_stream_makespan()
    rate = args.serve_rate if args.serve_rate > 0 else args.serve_load * capacity
    for r in reqs:
        r.arrival = r.arrival / rate
    srv = S.Server(hbm_budget=args.serve_budget_gb * 1e9, chunk=512, guard=guard, tuner=tuner,
                   fp64_as=args.serve_fp64_as)
    res = srv.run(reqs, realtime=True)
    by_rid = {r.rid: r for r in reqs}
    gsum = {}
    for rid, storage, e_end, pred, tol in guard.checked:
        g = gsum.setdefault(storage, {"checked": 0, "widened": 0, "predicted": []})
        g["checked"] += 1
        g["widened"] += int(not (pred <= tol))
        g["predicted"].append(pred)
    for g in gsum.values():
        g["predicted_median"] = float(np.median(g.pop("predicted")))
    finished = {}
    for r in res:
        finished[r.storage] = finished.get(r.storage, 0) + 1
    out = {"stream": {"requests": len(reqs), "seed": 0, "rate_per_s": rate,
                      "batched_capacity_solves_per_s": capacity, "warm_up_pass_makespan_s": warm_pass_s,
                      "offered_load": None if capacity is None else rate / capacity,
                      "steps": [lo, hi], "sides": [64, 4096], "re": [1, 1e6],
                      "storages": ["f64", "f32", "f16"], "node_updates": work,
                      "hbm_budget_gb": args.serve_budget_gb, "tuning_s_before_stream": tune_s,
                      "fp64_requests_run_as": args.serve_fp64_as},
           "batched": S.summarize(res, srv.makespan, srv.node_updates),
           "precision_guard": {"stated_bounds": {"rule": "min(e0 + r * steps, cap), RMS |u - u_FP64| / U",
                                                 "e0_r": S.STATED, "cap": S.ACCURACY_CAP},
                               "by_storage": gsum,
                               "finished_in": finished}}
    if not args.no_serve_reference:
        ref = S.run_fifo(reqs, storage="f64", realtime=True)
        out["fp64_fifo"] = S.summarize(ref, S.run_fifo.makespan, work)
    return out


def run_reference(args, problems, desc, budget_s: float = 60.0):
    """The FP64 CPU oracle on the workload, on the host cores (rank 0 only).  Each
    step advances every lattice of the workload by one time step on a strip of
    its rows (periodic in y with the strip's height), sized so the whole run takes
    about `budget_s`; MLUPS counts the nodes actually updated."""
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    import oracle as O

    def make(pr, rows):
        lat = O.Lattice(O.Params(nx=pr.nx, ny=rows, tau1=pr.tau_s, tau2=pr.tau_s2,
                                 periodic_x=pr.periodic[0], periodic_y=pr.periodic[1] or rows < pr.ny,
                                 gx=pr.g[0], gy=pr.g[1], wall_ux=pr.wall_u[0], wall_uy=pr.wall_u[1],
                                 wall_rho=pr.wall_rho, g_mode=oracle_g_mode(args.g_mode)),
                        mask=None if pr.mask is None else pr.mask[:rows])
        rho = None if pr.rho is None else pr.rho[:rows]
        return lat.init(pr.ux[:rows], pr.uy[:rows], rho)

    # cost of one full step, extrapolated from a strip of at most 64 rows
    probe_rows = min(problems[0].ny, 64)
    probe = make(problems[0], probe_rows)
    probe.step(1)
    t0 = time.perf_counter()
    probe.step(1)
    full = (time.perf_counter() - t0) * problems[0].ny / probe_rows * len(problems)
    frac = min(1.0, budget_s / max(1e-9, (args.steps + args.warmup) * full))
    lats = []
    for pr in problems:
        rows = max(8, min(pr.ny, int(pr.ny * frac) // 8 * 8))
        lats.append(make(pr, rows))
    for _ in range(args.warmup):
        for lat in lats:
            lat.step(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for lat in lats:
            lat.step(1)
    dt = time.perf_counter() - t0
    nodes = sum(l.p.nx * l.p.ny for l in lats)
    value = nodes * args.steps / dt / 1e6
    sample = (f"each step: one time step of {len(lats)} lattice(s) on {lats[0].p.nx}x{lats[0].p.ny} "
              f"row strips of the workload")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": desc, "nodes_per_step": nodes, "implementation": "FP64 CPU oracle"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                             "sample": sample, "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="dsl4096x3")
    ap.add_argument("--flush-mib", type=int, default=512)
    ap.add_argument("--reference-seconds", type=float, default=60.0,
                    help="--impl reference: about how long the timed oracle steps take in total")
    ap.add_argument("--e2e-steps", type=int, default=100, help="time steps per end-to-end solve")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--size", default=None, help="override the lattice size, NXxNY")
    ap.add_argument("--storage", default=None, choices=["f64", "f32", "f16", "bf16", "f64dw"])
    ap.add_argument("--kernel", default="tuned", choices=["tuned", "auto", "scalar", "vector", "column"],
                    help="tuned: the autotuner picks the kernel shape per lattice (default)")
    ap.add_argument("--tile-w", type=int, default=0, help="scalar kernel tile width (with --kernel scalar)")
    ap.add_argument("--g-mode", default="lagged", choices=["lagged", "current", "off"],
                    help="time level of Phi in G_i: lagged (in-place kernels) or current (two-buffer kernel)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serve", action="store_true", help="skip the served-stream measurement")
    ap.add_argument("--no-serve-reference", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=512,
                    help="requests in the served stream (512: the configuration's stream)")
    ap.add_argument("--serve-rate", type=float, default=0.0,
                    help="Poisson arrivals per second (0: serve-load x the measured batched capacity)")
    ap.add_argument("--serve-load", type=float, default=1.2)
    ap.add_argument("--serve-scale", type=float, default=0.05,
                    help="step counts of the stream: [1000, 20000] x scale")
    ap.add_argument("--serve-budget-gb", type=float, default=150.0)
    ap.add_argument("--serve-fp64-as", default="f64dw", choices=["f64dw", "f64"],
                    help="format the server runs FP64 requests in (the reference is always f64)")
    ap.add_argument("--mode", default="batch", choices=["batch", "single"],
                    help="batch: one launch per time step for all lattices; single: one per lattice")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    size = None
    if args.size:
        nx_s, ny_s = args.size.lower().split("x")
        size = (int(nx_s), int(ny_s))
    problems, storage, desc = workload(args.workload, size, args.storage, args.g_mode)
    if args.impl == "reference":
        return run_reference(args, problems, desc, budget_s=args.reference_seconds)

    import torch
    from paper_2312_10318_gb300 import Lattice
    from paper_2312_10318_gb300.lattice import Batch

    world, rank, local = dist_setup()
    if args.gpus != world:
        raise SystemExit(f"--gpus {args.gpus} needs torchrun with {args.gpus} processes (WORLD_SIZE={world})")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    from paper_2312_10318_gb300.tune import Tuner
    tuner = Tuner(persist=False)      # measured afresh on this GPU, not cached on disk
    lats = []
    for pr in problems:
        lat = Lattice(pr.nx, pr.ny, pr.tau_s, storage=storage, g_mode=args.g_mode, stream=stream,
                      **pr.lattice_kwargs())
        if args.kernel == "tuned":
            tuner.apply(lat, pr.periodic, pr.mask is not None)
        else:
            lat.set_kernel(args.kernel, args.tile_w)
        lat.init(*(torch.from_numpy(np.ascontiguousarray(a)).cuda() if a is not None else None
                   for a in (pr.ux, pr.uy, pr.rho)))
        lats.append(lat)
    nodes = sum(p.nodes for p in problems)
    # device bytes the step touches: populations and Phi of every lattice
    working_set = sum(lat.device_bytes() for lat in lats)
    flush = torch.empty(args.flush_mib << 20, dtype=torch.uint8, device="cuda")
    # all lattices of the workload advance in one launch per time step
    batch = Batch(stream).set(lats)

    def advance(n):
        if args.mode == "batch":
            batch.step(n)
        else:
            for lat in lats:
                lat.step(n)

    def flush_l2():
        # write a buffer 4x the L2, then read it back, so L2 holds only clean
        # lines of the flush buffer (no dirty write-backs charged to the step)
        flush.zero_()
        flush_sink.copy_(flush.view(torch.int64).sum())

    flush_sink = torch.empty((), dtype=torch.int64, device="cuda")
    for _ in range(args.warmup):
        advance(1)
    barrier()

    def timed(n, flush_each=False):
        """CUDA-event milliseconds of n steps on the launching stream: one event
        pair around all of them (back to back), or with flush_each one pair
        per step and the L2 flushed before it, outside the pair."""
        if not flush_each:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            advance(n)
            e1.record(stream)
            e1.synchronize()
            return e0.elapsed_time(e1)
        evs = []
        for _ in range(n):
            flush_l2()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            advance(1)
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in evs)

    clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if clocks:
        clocks.start()
        time.sleep(0.5)
    barrier()
    # the timed region: exactly K steps, back to back (the working set is far
    # larger than L2, so each step's reads come from HBM and the write-back of
    # the previous step's dirty lines is paid inside the region)
    local_ms = timed(args.steps)
    barrier()
    # beside it, not part of the value: a steady-state sample of at least 1000
    # back-to-back steps (long enough for the clock samples to see the load)
    # and the per-step figure with the L2 flushed before every step
    steady_n = max(1000, args.steps)
    steady_ms = timed(steady_n)
    flushed_n = min(args.steps, 50)
    flushed_ms = timed(flushed_n, flush_each=True)
    clk = clocks.stop() if clocks else None
    total_ms = max_over_ranks(local_ms, dist)
    value = whole_job_rate(nodes * args.steps, world, total_ms / 1e3) / 1e6
    fp64_tflops = fp64_fma_rate(stream)

    # roofline of the step kernel: algorithmic bytes per launch / mean launch time
    kinds = [lat.step_kernel() for lat in lats]
    per_step_launches = step_launches(args.mode, kinds)
    launches = args.steps * per_step_launches
    launch_s = local_ms / 1e3 / launches
    masked = any(p.mask is not None for p in problems)
    per_launch_bytes = bytes_per_node(storage, args.g_mode, masked) * nodes / per_step_launches
    achieved = per_launch_bytes / launch_s / 1e9
    peak, peak_kind = hbm_peak()
    steady_gbs = per_launch_bytes * per_step_launches * steady_n / (steady_ms / 1e3) / 1e9
    flushed_gbs = per_launch_bytes * per_step_launches * flushed_n / (flushed_ms / 1e3) / 1e9
    traffic = recorded_traffic(f"{args.workload}/{storage}/{args.g_mode}") if args.mode == "batch" else None

    # end to end through the C ABI with pinned host buffers: initial fields from
    # the host (the density only where the workload has one; else rho0), e2e_steps
    # time steps, macroscopic fields back to the host.  Batched, one
    # trtrlb_batch_solve call: the lattices step one after another while the
    # next one's fields go up and the previous one's come down on copy streams
    host_in = [tuple(None if a is None else torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
                     for a in (p.ux, p.uy, p.rho)) for p in problems]
    host_out = [tuple(torch.empty((p.ny, p.nx), dtype=torch.float64).pin_memory() for _ in range(3))
                for p in problems]
    h2d_bytes = sum(a.numel() * a.element_size() for f in host_in for a in f if a is not None)
    d2h_bytes = sum(a.numel() * a.element_size() for f in host_out for a in f)
    e2e_times = []
    for rep in range(0 if args.no_e2e else 9):
        barrier()
        t0 = time.perf_counter()
        if args.mode == "batch":
            batch.solve(host_in, args.e2e_steps, host_out)
        else:
            for lat, (ux, uy, rho) in zip(lats, host_in):
                lat.init(ux, uy, rho)
            advance(args.e2e_steps)
            for lat, out in zip(lats, host_out):
                lat.moments(*out)
        torch.cuda.synchronize()
        e2e_times.append(time.perf_counter() - t0)
    e2e_t = max_over_ranks(statistics.median(e2e_times) if e2e_times else float("nan"), dist)
    e2e_value = whole_job_rate(nodes * args.e2e_steps, world, e2e_t) / 1e6
    if not math.isfinite(e2e_value):
        e2e_value = None          # --no-e2e: no end-to-end number (null, not NaN, in the JSON)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": storage, "data": "synthetic",
            "config": {"workload": desc, "lattices": len(problems), "nx": problems[0].nx,
                       "ny": problems[0].ny, "nodes_per_step": nodes, "storage": storage,
                       "g_mode": args.g_mode,
                       "kernel": ", ".join(dict.fromkeys(
                           k + (f", tile {lat.kernel()[1]}" if k == "aa" else "") for k, lat in zip(kinds, lats)))
                                 + (" (autotuned)" if args.kernel == "tuned" else ""),
                       "tuning": tuner.measured if args.kernel == "tuned" else None,
                       "parallelism": f"replicas x{world}",
                       "launch": (f"{per_step_launches} step-kernel launch(es) per time step, "
                                  + ("batched" if args.mode == "batch" else "one lattice each")),
                       "working_set_bytes": working_set,
                       "l2": ("inputs larger than L2: the timed steps run back to back, no flush "
                              f"(working set {working_set / 1e9:.2f} GB against a 129 MB L2)"
                              if working_set > 4 * L2_BYTES else
                              "inputs not much larger than L2: see roofline.flushed (L2 flushed "
                              "before every step); the value is back to back")},
            "roofline": alu_roofline(storage, nodes / per_step_launches, launch_s, fp64_tflops) or
                        {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind,
                         "traffic": None if traffic is None else traffic,
                         "algorithmic_bytes_per_node": bytes_per_node(storage, args.g_mode, masked)},
            "e2e": {"value": e2e_value, "unit": UNIT,
                    "solves_ms": [round(t * 1e3, 2) for t in e2e_times],
                    "h2d_bytes_per_step": h2d_bytes / args.e2e_steps,
                    "d2h_bytes_per_step": d2h_bytes / args.e2e_steps,
                    "solve": (f"init from pinned host fields (u; rho where the workload has one) + "
                              f"{args.e2e_steps} steps + rho, u to the host"
                              + (", one trtrlb_batch_solve: copies beside the steps" if args.mode == "batch"
                                 else ""))},
            "gpu_launches": launches,
            "clocks": clk,
            "fp64_fma_tflops": fp64_tflops,
        }
        line["roofline"]["kernel"] = kernel_label(args.mode, kinds)
        line["roofline"]["launch_ms"] = launch_s * 1e3
        line["roofline"]["hbm_gbs"] = achieved        # algorithmic bytes / time, every format
        line["roofline"]["frac_of_nominal_hbm"] = achieved / HBM_NOMINAL_GBS
        line["roofline"]["steady"] = {"steps": steady_n, "ms_per_step": steady_ms / steady_n,
                                      "mlups": nodes * steady_n / (steady_ms / 1e3) / 1e6,
                                      "gbs": steady_gbs, "frac": steady_gbs / peak,
                                      "timing": "one event pair around back-to-back steps"}
        line["roofline"]["flushed"] = {"steps": flushed_n, "ms_per_step": flushed_ms / flushed_n,
                                       "mlups": nodes * flushed_n / (flushed_ms / 1e3) / 1e6,
                                       "gbs": flushed_gbs, "frac": flushed_gbs / peak,
                                       "timing": f"{args.flush_mib} MiB written then read before "
                                                 "every step, outside its event pair"}
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(problems, g_mode=args.g_mode)
        if world == 1 and not args.no_serve:
            # the served stream is a one-GPU measurement: under torchrun the
            # other GPUs would only wait for it
            line["serving"] = run_serving(args)
        print(json.dumps(line), flush=True)
    batch.close()
    for lat in lats:
        lat.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
