"""Benchmark: cell-updates/s of the WENO5-LF / SSP-RK3 shallow-water step on
one GB300, on the synthetic coastal DEM (4096 x 4096, dx = 5 m, N-wave
inflow, FP32 state with FP64 reductions).

One "step" is one full RK3 time step (three fused stage kernels) over the
whole grid: 16.8 M cell-updates.  Inputs are resident in HBM and larger than
L2 (ten 64 MB planes), so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

For N > 1 (torchrun), each rank runs an independent replica of the same
workload (the single-scenario path does not shard: replicas only) and the
value is the sum over ranks of cell-updates divided by the slowest rank's
time.  ``--impl reference`` times the FP64 CPU oracle on the host cores on a
bounded window of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s/GPU FP32 vs FP64 (oracle-matched), %HBM roofline; p50/p99 solve ms"
WORKLOAD = "synthetic coastal DEM 4096x4096, dx=5 m, shelf ramp -200 m to 0 + fractal noise (slope -2, 3 m rms), " \
           "land to +20 m, N-wave inflow 4 m / 600 s, Manning n=0.025, FP32 state, FP64 dt/mass reductions"

# Algorithmic HBM bytes per cell and RK stage (the roofline the metric names):
# stage 1 reads U^n (12 B) and b (4 B) and writes U1 (12 B); stages 2 and 3
# also read U^n for the RK combination.  108 B per cell-update over a step.
BYTES_PER_CELL_STAGE = {1: 28.0, 2: 40.0, 3: 40.0}

# ncu counters of one launch of each RK stage of the FP32 stage kernel (tile
# shape 7): dram__bytes_read.sum + dram__bytes_write.sum per launch on the
# bench's own workload (4096 x 4096 coastal DEM, `cells`), and, from the
# 2048 x 2048 case of the same workload, executed thread instructions per cell
# (smsp__thread_inst_executed.sum / cells) and the issue-active percent
# (sm__inst_issued.avg.pct_of_peak_sustained_active).  Reported only while the
# kernel's sources hash to the captured version (its device code, its
# translation unit and the tile-shape table).
NCU_CAPTURE = {"tile": 7, "cells": 4096 * 4096,
               "profile": "profiles/stage_kernel_f32_coastal_dem_4096_dram.md, "
                          "profiles/stage_kernel_f32_coastal_dem_2048_pipes.md",
               "dram_bytes": {1: 269617408 + 166553600, 2: 470975488 + 176506880, 3: 470625792 + 165633792},
               "thread_inst_per_cell": {1: 566.3, 2: 594.7, 3: 601.2},
               "issue_active_pct": {1: 61.25, 2: 62.32, 3: 63.33},
               "sources": ("swe_core.cuh", "swe_kernels.cu", "swe_launch.h:SWE_SHAPES"),
               "sha256": "39123cb4c1e5065daf179c056e8e27fca5393600b7d9d4845a3b376f9908cafd"}


def kernel_sources_sha256() -> str:
    """sha256 over the stage kernel's sources; "file:NAME" takes only the
    #define NAME block of that file."""
    import hashlib
    h = hashlib.sha256()
    for name in NCU_CAPTURE["sources"]:
        fname, _, block = name.partition(":")
        with open(os.path.join(ROOT, "paper_2301_12010_gb300", "csrc", fname), "rb") as f:
            data = f.read()
        if block:
            a = data.index(b"#define " + block.encode())
            data = data[a:data.index(b"\n\n", a)]
        h.update(data)
    return h.hexdigest()


def issue_ceiling(value: float, clk):
    """The cell-update rate at which the stage kernels would issue one warp
    instruction per scheduler and cycle (152 SMs x 4 schedulers x 32 lanes at
    the sampled SM clock over the captured thread instructions of the three
    stages), and the fraction of it reached; None without valid counters."""
    c = NCU_CAPTURE
    try:
        if c["sha256"] is None or kernel_sources_sha256() != c["sha256"] or not c["thread_inst_per_cell"]:
            return None
    except OSError:
        return None
    mhz = (clk or {}).get("sm_mhz") or 2070.0
    per_update = sum(c["thread_inst_per_cell"].values())
    ceil = 152 * 4 * 32 * mhz * 1e6 / per_update
    return {"value": ceil, "unit": "cell-updates/s", "frac": value / ceil, "sm_mhz": mhz,
            "thread_inst_per_cell_update": per_update}


def ncu_counters(tile: int, stage: int, cells: int):
    """The captured counters of one launch of this RK stage, DRAM bytes scaled
    to `cells` if the capture was of another size, or None if nothing was
    captured for this tile, or the kernel changed since the capture."""
    c = NCU_CAPTURE
    try:
        if c["sha256"] is None or tile != c["tile"] or kernel_sources_sha256() != c["sha256"]:
            return None
    except OSError:
        return None
    out = {"profile": c["profile"]}
    if c["dram_bytes"]:
        out["dram_bytes"] = c["dram_bytes"][stage] / c["cells"] * cells
    if c["thread_inst_per_cell"]:
        out["thread_inst_per_cell"] = c["thread_inst_per_cell"][stage]
    if c["issue_active_pct"]:
        out["issue_active_pct"] = c["issue_active_pct"][stage]
    return out


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        try:
            self.proc.terminate()
            self.proc.wait(timeout=5)
        except Exception:
            pass
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(sc, budget_s: float = 12.0):
    """The FP64 oracle on the host cores, on a bounded window of the same
    workload: whole RK3 steps of the full grid until the budget is spent."""
    import oracle
    sim = oracle.Simulation(sc)
    t0 = time.perf_counter()
    steps = 0
    while steps < 3:
        sim.step(1)
        steps += 1
        if time.perf_counter() - t0 > budget_s:
            break
    el = time.perf_counter() - t0
    return {"value": sc.cells * steps / el, "unit": "cell-updates/s", "cores": oracle.num_threads(),
            "kind": "oracle", "sample": "%d RK3 step(s) of the full %dx%d grid (FP64, %d threads)"
            % (steps, sc.nx, sc.ny, oracle.num_threads())}


def ensemble_bench(swe, W, torch, steps: int = 20):
    """C4: the 64-scenario mitigation ensemble advanced by one persistent
    batched launch per run, against the same 64 scenarios stepped one after
    another by the single-scenario path, on the same GPU."""
    ens = W.mitigation_ensemble()
    cells = sum(sc.cells for sc in ens)
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    best, ms_shapes = swe.autotune([(sc.nx, sc.ny) for sc in ens], precision=swe.F32, batch=True, steps=3)
    with swe.Batch(len(ens), 150 << 30, ens[0], stream=stream.cuda_stream, tile=0) as b:
        for sc in ens:
            b.admit(sc)
        b.run(2)
        b.poll()
        ev[0].record(stream)
        b.run(steps)
        ev[1].record(stream)
        torch.cuda.synchronize()
        assert b.status() == swe.OK
    solvers = [swe.Solver(sc, precision=swe.F32, stream=stream.cuda_stream) for sc in ens]
    for s in solvers:
        s.step(2)
    torch.cuda.synchronize()
    ev[2].record(stream)
    for s in solvers:
        s.step(steps)
    ev[3].record(stream)
    torch.cuda.synchronize()
    for s in solvers:
        s.close()
    tb = ev[0].elapsed_time(ev[1]) / 1e3
    ts = ev[2].elapsed_time(ev[3]) / 1e3
    return {"scenarios": len(ens), "cells": cells, "steps": steps, "batch_tile": best, "autotune_ms": ms_shapes,
            "batched_cell_updates_per_s": cells * steps / tb, "sequential_cell_updates_per_s": cells * steps / ts,
            "speedup_batched_vs_sequential": ts / tb, "launches_batched": 1, "launches_sequential": 3 * steps * len(ens)}


def ensemble_fp64_rate(swe, W, torch, steps: int = 3) -> float:
    """The 64-scenario ensemble in one FP64 batch (the batch path's parity
    mode, 32x32 tiles): cell-updates/s of one persistent launch of `steps`."""
    ens = W.mitigation_ensemble()
    cells = sum(sc.cells for sc in ens)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with swe.Batch(len(ens), 150 << 30, ens[0], stream=stream.cuda_stream, precision=swe.F64) as b:
        for sc in ens:
            b.admit(sc)
        b.run(1)
        b.poll()
        e0.record(stream)
        b.run(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        assert b.status() == swe.OK
    return cells * steps / (e0.elapsed_time(e1) / 1e3)


def fp64_bench(swe, W, torch, sc, steps: int = 10):
    """The same coastal-DEM workload with FP64 state and arithmetic (the
    parity path; GB300's FP64 rate is a small fraction of FP32)."""
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best, ms_shapes = swe.autotune([(sc.nx, sc.ny)], precision=swe.F64, steps=2)
    with swe.Solver(sc, precision=swe.F64, stream=stream.cuda_stream, tile=best) as s:
        s.step(2)
        s.sync()
        e0.record(stream)
        s.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        s.sync()
    ms = e0.elapsed_time(e1)
    return {"value": sc.cells * steps / (ms / 1e3), "unit": "cell-updates/s", "steps": steps,
            "ms_per_step": ms / steps, "dtype": "f64", "tile": best,
            "autotune_ms": [round(x, 3) for x in ms_shapes]}


FUSED_BYTES_PER_CELL = 28.0  # FP32: U^n (12 B) and the bed (4 B) read, U^{n+1} (12 B) written, once per step


def fused_bench(swe, W, torch, sc, steps: int = 20, margin: float = 1.1, warmup: int = 4,
                per_stage_ms: float = 0.0, hbm_peak: float = 6800.0):
    """The fused-step variant on the same workload: one kernel per RK3 step
    (9-cell halo frames in shared memory), all three stages split with
    margin x alpha(U^n) instead of the paper's per-stage alpha."""
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with swe.Solver(sc.copy(alpha_margin=margin), precision=swe.F32, stream=stream.cuda_stream) as s:
        s.step(warmup)
        s.sync()
        e0.record(stream)
        s.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        s.sync()
        ms = e0.elapsed_time(e1) / steps
        nk = 10
        _, kst = s.time_stages(nk)
    k_ms = kst[0] / nk
    achieved = FUSED_BYTES_PER_CELL * sc.cells / (k_ms / 1e3) / 1e9
    out = {"value": sc.cells / (ms / 1e3), "unit": "cell-updates/s", "steps": steps, "ms_per_step": ms,
           "kernel_ms": k_ms, "bookkeeping_ms": kst[1] / nk, "alpha_margin": margin, "dtype": "f32",
           "scheme": "fused-step variant: one splitting speed per step (margin x alpha of U^n), not the "
                     "paper's per-stage alpha",
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                        "frac": achieved / hbm_peak, "bytes_per_cell_update": FUSED_BYTES_PER_CELL},
           "gpu_launches": 3 * steps}
    if per_stage_ms > 0:
        out["speed_vs_stage_kernels"] = per_stage_ms / ms
    return out


def shore_bench(swe, W, torch, sc, steps: int = 20, warmup: int = 4, per_stage_ms: float = 0.0):
    """The shoreline variant on the same workload (hydrostatic-reconstruction
    faces wherever a stencil meets a dry cell: the DEM's land and its wet/dry
    front); its one compiled tile shape (96 x 32 in FP32)."""
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with swe.Solver(sc.copy(shore=1), precision=swe.F32, stream=stream.cuda_stream) as s:
        s.step(warmup)
        s.sync()
        e0.record(stream)
        s.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        s.sync()
        ms = e0.elapsed_time(e1) / steps
    dry = float((sc.h < sc.h_dry).mean())
    out = {"value": sc.cells / (ms / 1e3), "unit": "cell-updates/s", "steps": steps, "ms_per_step": ms,
           "dtype": "f32", "dry_cell_fraction": dry,
           "scheme": "shoreline variant: hydrostatic-reconstruction faces next to dry cells, WENO elsewhere"}
    if per_stage_ms > 0:
        out["speed_vs_stage_kernels"] = per_stage_ms / ms
    return out


def profile_fp64_case(n: int = 2048, tile: int = 2) -> int:
    """A few FP64 steps on the n x n coastal DEM with the FP64 path's tile
    shape (64 x 32), for ncu; no timing."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2301_12010_gb300 as swe
    import workloads as W
    torch.cuda.set_device(0)
    st = torch.cuda.current_stream().cuda_stream
    with swe.Solver(W.coastal_dem(n=n), precision=swe.F64, stream=st, tile=tile) as s:
        s.step(3)
        s.sync()
    print("profile-fp64: ok")
    return 0


def profile_shore_case(n: int = 2048) -> int:
    """A few steps of the shoreline variant on the n x n coastal DEM, for ncu; no timing."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2301_12010_gb300 as swe
    import workloads as W
    torch.cuda.set_device(0)
    st = torch.cuda.current_stream().cuda_stream
    with swe.Solver(W.coastal_dem(n=n).copy(shore=1), precision=swe.F32, stream=st) as s:
        s.step(3)
        s.sync()
    print("profile-shore: ok")
    return 0


def profile_fused_case(n: int = 2048) -> int:
    """A few fused steps on the n x n coastal DEM, for ncu; no timing."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2301_12010_gb300 as swe
    import workloads as W
    torch.cuda.set_device(0)
    st = torch.cuda.current_stream().cuda_stream
    with swe.Solver(W.coastal_dem(n=n).copy(alpha_margin=1.1), precision=swe.F32, stream=st) as s:
        s.step(4)
        s.sync()
    print("profile-fused: ok")
    return 0


def serving_bench(swe, W, torch, rates=(5.0, 20.0), count: int = 12, horizon: float = 20.0,
                  policies=("srpt", "all"), fill_waves: int = 4):
    """C5: Poisson requests, N log-uniform in [256, 2048], coast and hills as
    the ensemble, 150 GB budget, continuous batching.  The default bench line
    runs a bounded sample (count requests per rate, `horizon` simulated
    seconds each); --serving-sweep runs the configuration's rates and 600 s
    horizon."""
    from paper_2301_12010_gb300.serve import Server
    stream = torch.cuda.current_stream().cuda_stream
    # the batch tile shape, tuned on grids of the request mix
    mix = W.serving_requests(rate=rates[0], count=count, horizon=horizon)
    tile, _ = swe.autotune([(r.scenario.nx, r.scenario.ny) for r in mix[:8]], precision=swe.F32, batch=True, steps=3)
    out = {}
    for policy in policies:
        res = {}
        for rate in rates:
            reqs = W.serving_requests(rate=rate, count=count, horizon=horizon)
            with Server(reqs[0].scenario, nslots=64, budget_bytes=150 << 30, k_steps=50, stream=stream,
                        policy=policy, tile=tile, fill_cells=152 * fill_waves * 3072) as srv:
                rep = srv.serve(reqs)
            res["%g_req_per_s" % rate] = rep.summary()
        out[policy] = res
    full = horizon >= 600.0 and count >= 50
    return {"sample": "%d requests per rate at %s req/s, %g s simulated horizon per request%s"
                      % (count, ", ".join("%g" % r for r in rates), horizon,
                         "" if full else " (a bounded sample: configuration 5 asks for 1-50 req/s, at least 200 "
                                         "requests per rate and a 600 s horizon; python bench.py --serving-sweep "
                                         "runs 1, 5, 20 and 50 req/s at the 600 s horizon)"),
            "policies": {"srpt": "shortest remaining work first, enough requests per launch to fill %d waves of "
                                 "tiles" % fill_waves,
                         "all": "every live request advances each launch"},
            "batch_tile": tile, "rates": out.get("srpt"), "rates_all": out.get("all")}


def profile_batch_case() -> int:
    """One step of each batch work order and of the single-scenario path
    (96x32 tiles), for ncu; no timing."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2301_12010_gb300 as swe
    import workloads as W
    torch.cuda.set_device(0)
    st = torch.cuda.current_stream().cuda_stream
    ens = W.mitigation_ensemble()
    with swe.Batch(len(ens), 150 << 30, ens[0], stream=st, tile=7) as b:
        for sc in ens:
            b.admit(sc.copy(t_end=1e9))
        b.run(1)
        torch.cuda.synchronize()
    dem = W.coastal_dem(n=2048).copy(bc=(W.WALL,) * 4, inflow_amp=0.0)
    with swe.Batch(2, 64 << 30, dem, stream=st, tile=7) as b:
        b.admit(dem.copy(t_end=1e9))
        b.run(1)
        torch.cuda.synchronize()
    with swe.Solver(dem, precision=swe.F32, stream=st, tile=7) as s:
        s.step(1)
        s.sync()
    print("profile-batch: ok")
    return 0


def config_table() -> int:
    """Per configuration: GPU FP32 and FP64 cell-updates/s beside the FP64
    oracle's at one thread and at all host cores (bounded samples where a
    full run would take minutes, marked as such).  Prints one JSON object."""
    import platform

    import torch

    import __graft_entry__
    __graft_entry__.build()
    import oracle
    import paper_2301_12010_gb300 as swe
    import workloads as W
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    all_threads = oracle.num_threads()

    def gpu_rate(sc, steps, precision, tile=0):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with swe.Solver(sc, precision=precision, stream=stream.cuda_stream, tile=tile) as s:
            s.step(3)
            s.sync()
            e0.record(stream)
            s.step(steps)
            e1.record(stream)
            torch.cuda.synchronize()
            s.sync()
        return sc.cells * steps / (e0.elapsed_time(e1) / 1e3)

    def oracle_rate(scs, steps, threads):
        oracle.set_threads(threads)
        sims = [oracle.Simulation(sc) for sc in scs]
        t0 = time.perf_counter()
        for sim in sims:
            sim.step(steps)
        dt = time.perf_counter() - t0
        oracle.set_threads(all_threads)
        return sum(sc.cells for sc in scs) * steps / dt

    rows = {}
    sc = W.gaussian_hump()
    rows["C1 hump 128x128, 200 steps"] = {
        "gpu_f32": gpu_rate(sc, 200, swe.F32), "gpu_f64": gpu_rate(sc, 200, swe.F64),
        "oracle_1_thread": oracle_rate([sc], 200, 1), "oracle_all_threads": oracle_rate([sc], 200, all_threads),
        "oracle_sample": "full run"}
    sc = W.planar_beach()
    rows["C2 planar beach 2048x64, 5000 steps"] = {
        "gpu_f32": gpu_rate(sc, 5000, swe.F32), "gpu_f64": gpu_rate(sc, 5000, swe.F64),
        "oracle_1_thread": oracle_rate([sc], 200, 1), "oracle_all_threads": oracle_rate([sc], 1000, all_threads),
        "oracle_sample": "200 steps at 1 thread, 1000 at all threads (rate extrapolated to the 5000-step run)"}
    sc = W.coastal_dem()
    rows["C3 coastal DEM 4096x4096"] = {
        "gpu_f32": gpu_rate(sc, 100, swe.F32, tile=7), "gpu_f64": gpu_rate(sc, 10, swe.F64, tile=2),
        "oracle_1_thread": oracle_rate([sc], 1, 1), "oracle_all_threads": oracle_rate([sc], 2, all_threads),
        "oracle_sample": "1 step at 1 thread, 2 at all threads of the 1.6e5-step hour (rate extrapolated)"}
    ens = W.mitigation_ensemble()
    e = ensemble_bench(swe, W, torch)
    rows["C4 ensemble of 64 coasts (29.7 M cells)"] = {
        "gpu_f32": e["batched_cell_updates_per_s"], "gpu_f64": ensemble_fp64_rate(swe, W, torch),
        "gpu_note": "one batched persistent launch (FP64: the batch path's parity mode, 32x32 tiles)",
        "oracle_1_thread": oracle_rate(ens[:4], 1, 1), "oracle_all_threads": oracle_rate(ens[:4], 2, all_threads),
        "oracle_sample": "4 of the 64 scenarios, 1 step at 1 thread and 2 at all threads (rate extrapolated)"}
    cpu = platform.processor() or platform.machine()
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    cpu = "%s (%s)" % (platform.machine(), line.split(":", 1)[1].strip())
                    break
    except OSError:
        pass
    print(json.dumps({"config_table": rows, "unit": "cell-updates/s", "host": cpu, "nproc": os.cpu_count(),
                      "oracle_threads": all_threads, "gpu": torch.cuda.get_device_name(0)}))
    return 0


def run_reference(args):
    """--impl reference: the FP64 CPU oracle on the host cores, each step one
    RK3 step of a 512 x 512 window (the inflow edge) of the coastal DEM."""
    ws, rank, local = dist_env()
    if rank != 0:
        return 0
    import oracle
    import workloads as W
    oracle.build()
    full = W.coastal_dem()
    win = 512
    sc = full.copy(b=full.b[:win, :win].copy(), h=full.h[:win, :win].copy(), hu=full.hu[:win, :win].copy(),
                   hv=full.hv[:win, :win].copy())
    sim = oracle.Simulation(sc)
    sim.step(args.warmup)
    t0 = time.perf_counter()
    sim.step(args.steps)
    el = time.perf_counter() - t0
    v = sc.cells * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "cell-updates/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": "512x512 window at the inflow edge per step"},
            "cpu_baseline": {"kind": "oracle", "cores": oracle.num_threads(), "value": v,
                             "unit": "cell-updates/s",
                             "sample": "one RK3 step of a 512x512 window of the 4096x4096 coastal DEM per step"},
            "e2e": {"value": v, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def replica_throughput(ms_local: float, cells: int, steps: int, dist=None):
    """Whole-job throughput of independent replicas, one per rank: the job
    takes as long as its slowest rank (all-reduce MAX of the timed region over
    the process group), and value = the cell-updates of all ranks / that time.
    Returns (value, ms_max)."""
    ws, ms_max = 1, float(ms_local)
    if dist is not None and dist.is_initialized():
        import torch
        ws = dist.get_world_size()
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([ms_max], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_max = float(t.item())
    return cells * steps * ws / (ms_max / 1e3), ms_max


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=4096, help="grid size of the coastal DEM")
    ap.add_argument("--tile", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--serving-sweep", default=None, metavar="RATES", nargs="?", const="1,5,20,50",
                    help="only the serving measurement, at these comma-separated request rates (req/s; "
                         "default 1,5,20,50); prints one JSON object, not a bench line")
    ap.add_argument("--serving-count", type=int, default=50, help="requests per rate of --serving-sweep")
    ap.add_argument("--serving-horizon", type=float, default=600.0,
                    help="simulated seconds per request of --serving-sweep (configuration 5: 600)")
    ap.add_argument("--serving-policies", default="srpt", help="comma-separated: srpt, all")
    ap.add_argument("--serving-fill-waves", type=int, default=4,
                    help="srpt: waves of tiles (152 x this x 3072 cells) each launch advances at least")
    ap.add_argument("--profile-batch", action="store_true",
                    help="only one RK3 step of the batch kernel on the 64-scenario ensemble (contiguous order) "
                         "and on one walled 2048x2048 DEM (strided order), then the same DEM by the "
                         "single-scenario kernels: a short case for a profiler")
    ap.add_argument("--no-fused", action="store_true", help="skip the fused-step variant's measurement")
    ap.add_argument("--no-shore", action="store_true", help="skip the shoreline variant's measurement")
    ap.add_argument("--profile-fp64", action="store_true",
                    help="only three FP64 steps on the --n coastal DEM (64x32 tiles): a short case for a profiler")
    ap.add_argument("--profile-shore", action="store_true",
                    help="only three steps of the shoreline variant on the --n coastal DEM: a short case for a profiler")
    ap.add_argument("--profile-fused", action="store_true",
                    help="only four fused steps on the --n coastal DEM: a short case for a profiler")
    ap.add_argument("--config-table", action="store_true",
                    help="only the per-configuration table: GPU FP32/FP64 beside the oracle at 1 thread and all "
                         "cores; prints one JSON object")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_batch:
        return profile_batch_case()
    if args.profile_fused:
        return profile_fused_case(args.n)
    if args.profile_shore:
        return profile_shore_case(args.n)
    if args.profile_fp64:
        return profile_fp64_case(args.n)
    if args.config_table:
        return config_table()
    if args.serving_sweep:
        import torch

        import __graft_entry__
        __graft_entry__.build()
        import paper_2301_12010_gb300 as swe
        import workloads as W
        torch.cuda.set_device(0)
        rates = tuple(float(r) for r in args.serving_sweep.split(","))
        res = serving_bench(swe, W, torch, rates=rates, count=args.serving_count, horizon=args.serving_horizon,
                            policies=tuple(args.serving_policies.split(",")), fill_waves=args.serving_fill_waves)
        print(json.dumps({"serving_sweep": res}))
        return 0

    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2301_12010_gb300 as swe
    import workloads as W

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    sc = W.coastal_dem(n=args.n)
    stream = torch.cuda.current_stream()
    tune = None
    if args.tile == 0:
        best, ms_shapes = swe.autotune([(sc.nx, sc.ny)], precision=swe.F32, steps=5)
        tune = {"best": best, "ms_per_step": ms_shapes, "shapes": swe.tile_shapes()}
    solver = swe.Solver(sc, precision=swe.F32, stream=stream.cuda_stream, tile=args.tile)
    solver.step(args.warmup)
    solver.sync()

    clocks = ClockSampler(local)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    e0.record(stream)
    solver.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    solver.sync()
    cells = sc.cells
    value, ms_max = replica_throughput(ms, cells, args.steps, dist)

    # per-stage kernel durations (CUDA events on the launching stream)
    nst = 30
    tot, st3 = solver.time_stages(nst)
    stage_ms = [x / nst for x in st3]
    dom = int(np.argmax(stage_ms)) + 1
    pk, pk_kind = peaks()
    dom_s = stage_ms[dom - 1] / 1e3
    achieved_gbs = BYTES_PER_CELL_STAGE[dom] * cells / dom_s / 1e9
    hbm_peak = float(pk.get("hbm_gbs", 6800.0))
    diag = solver.diagnostics()
    counters = ncu_counters(diag["tile"], dom, cells)

    # end to end through the public API: every step uploads its input state
    # from pinned host FP64 arrays, advances one step and reads its result back
    # into pinned host FP64 arrays (bytes counted from the arrays copied).
    # Pipelined: swe_set_state_async and swe_get_state_async let copy engines
    # carry the next step's input and this step's result while the step runs;
    # the last read-back is waited for inside the timed region.  The fully
    # synchronous loop is reported beside it.
    pin = [torch.empty((sc.ny, sc.nx), dtype=torch.float64, pin_memory=True) for _ in range(6)]
    for a, src in zip(pin[:3], (sc.h, sc.hu, sc.hv)):
        a.numpy()[...] = src
    hin = [a.numpy() for a in pin[:3]]
    hout = tuple(a.numpy() for a in pin[3:])
    for _ in range(3):  # warm the pipeline: both staging slots of each direction in use
        solver.set_state_async(*hin)
        solver.step(1)
        solver.get_state_async(hout)
    solver.wait_state()
    torch.cuda.synchronize()
    e2e_runs = []  # three timed loops; the median is reported, all three beside it
    for _ in range(3):
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            solver.set_state_async(*hin)
            solver.step(1)
            solver.get_state_async(hout)
        solver.wait_state()
        e2e_runs.append(cells * ws / ((time.perf_counter() - t0) / args.e2e_steps))
    e2e_v = sorted(e2e_runs)[1]
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        solver.set_state(*hin)
        solver.step(1)
        solver.get_state(hout)
    e2e_seq = cells * ws / ((time.perf_counter() - t0) / args.e2e_steps)
    solver.close()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "nx": sc.nx, "ny": sc.ny, "cells": cells,
                       "l2": "inputs larger than L2 (10 planes x %.0f MB)" % (cells * 4 / 1e6),
                       "parallelism": "replicas" if ws > 1 else "single", "tile": diag["tile"]},
            "roofline": {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved_gbs / hbm_peak,
                         "traffic": counters.get("dram_bytes") if counters else None,
                         "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
                         "kernel": "stage_kernel<float> RK stage %d" % dom,
                         "peak_source": "%s (MEASURED_PEAKS.json hbm_gbs)" % pk_kind,
                         "bytes_per_cell_stage": BYTES_PER_CELL_STAGE[dom],
                         "step_frac": (108.0 * cells * args.steps * ws / (ms_max / 1e3) / 1e9) / hbm_peak,
                         "alu": {"thread_inst_per_cell_stage": counters.get("thread_inst_per_cell")
                                 if counters else None,
                                 "issue_active_pct": counters.get("issue_active_pct") if counters else None,
                                 "source": counters.get("profile") if counters else None,
                                 "issue_ceiling": issue_ceiling(value, clk),
                                 "note": "the kernel is bound by FP32 instruction issue, not HBM: executed thread "
                                         "instructions per cell and RK stage and the issue-active share, from ncu"}},
            "stage_ms": stage_ms,
            "autotune": tune,
            "gpu_launches": 3 * args.steps,
            "clocks": clk,
            "e2e": {"value": e2e_v, "unit": "cell-updates/s", "h2d_bytes_per_step": 3 * 8 * cells,
                    "d2h_bytes_per_step": 3 * 8 * cells,
                    "how": "per step swe_set_state_async(pinned FP64 host) + swe_step(1) + swe_get_state_async("
                           "pinned FP64 host): copy engines carry the next input and the last result while the "
                           "step runs; swe_wait_state at the end; the median of three timed loops",
                    "repeats": e2e_runs,
                    "sequential_value": e2e_seq,
                    "sequential_how": "per step swe_set_state + swe_step(1) + swe_get_state, all synchronous"},
            "sim": {"t": diag["t"], "steps": diag["steps"], "last_dt": diag["last_dt"]},
        }
        if ws == 1 and not args.no_fused:
            line["fused_step"] = fused_bench(swe, W, torch, sc, per_stage_ms=ms_max / args.steps,
                                             hbm_peak=hbm_peak)
        if ws == 1 and not args.no_shore:
            line["shore_step"] = shore_bench(swe, W, torch, sc, per_stage_ms=ms_max / args.steps)
        if ws == 1 and not args.no_fp64:
            line["fp64"] = fp64_bench(swe, W, torch, sc)
        if ws == 1 and not args.no_ensemble:
            line["ensemble"] = ensemble_bench(swe, W, torch)
        if ws == 1 and not args.no_serving:
            line["serving"] = serving_bench(swe, W, torch)
        if ws == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(sc)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
