#!/usr/bin/env python
"""Benchmark: batched P1 quadrature element integration on GB300.

Headline workload: the 3D P1 Laplacian with variable coefficient on the unit cube as
64^3 hexes x 6 = 1,572,864 jittered tets (interior jitter +-0.15h), 4-point degree-2
rule, K ~ lognormal(0,1) per quadrature point, nodal u ~ U[-1,1]. One step = one
element-residual evaluation of the whole mesh (gather, geometry, quadrature phase,
basis phase) in the FP32-mixed form; the float64 form is timed beside it.

Timing: W warm-up steps, then K steps back to back between one pair of CUDA events on
the launching stream, with inputs larger than the L2: the steps cycle through n
resident copies of the workload, n chosen so that the other copies' bytes between two
uses of one copy are at least 3x the L2 (the headline: 6 copies, 499 MB). Workloads too
small for that (at most 128 copies) are timed one launch at a time after an L2 flush (a
read of a 512 MiB buffer), as are the rows that do not take copies; the headline also
reports that per-launch figure. Barrier + synchronize around the timed loop; max over
ranks.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--rows all|none|PREFIX,...] [--no-cpu-baseline]

Rank 0 prints one JSON line. With N > 1 (torchrun), every rank integrates its own
copy of the workload (independent problems, no data-path collective): weak scaling.
"""

from __future__ import annotations

import argparse
import datetime as _dt
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads  # noqa: E402
from paper_1607_04245_gb300 import perfmodel  # noqa: E402

METRIC = "cells/s and HBM GB/s (% of GB300 peak), FP32 vs FP64 at stated error; served p99"
WORKLOAD = "3D P1 Laplacian, variable coefficient: 64^3 hexes x 6 = 1,572,864 jittered tets, 4-pt degree-2 rule"
HEADLINE_CELLS = 1572864
HEADLINE_KERNEL = ("lap_pair_kernel<3, FP32_MIXED, NQ=4> (two consecutive cells per thread as f32x2 pairs, "
                   "8-byte row loads and streaming stores, one wave of 3 x 256-thread CTAs per SM)")
FLUSH_BYTES = 512 << 20
# float64 instructions per cell of the float64 3D Laplacian kernel, counted by ncu
# (smsp__sass_thread_inst_executed_op_dfma/dadd/dmul_pred_on.sum over one launch on the
# 1,572,864-tet workload, divided by the cells): DFMA 30, DADD 16, DMUL 21
FP64_INST_PER_CELL_LAP3D = {"dfma": 30, "dadd": 16, "dmul": 21}
# FP64 peak: 1.25 TFLOP/s nominal for GB300 = 0.625 T FMA instructions/s, i.e. 2 float64
# instructions per clock per SM at 2070 MHz on 152 SMs
FP64_NOMINAL_TFLOPS = 1.25
TOL = {"fp64": 1e-12, "mixed": 2e-5, "fp32": 1e-3, "fp64_df": 1e-12}


# ----------------------------------------------------------------------------- helpers


def algorithmic_bytes(physics, dim, prec, C, V, nq):
    """Compulsory HBM bytes of one residual launch: every cell-indexed array once,
    every vertex once."""
    s = 8 if prec in ("fp64", "fp64_df") else 4
    ncomp = 1 if physics == "laplacian" else dim
    ncoef = 1 if physics == "laplacian" else 2
    return ((dim + 1) * 4 * C + ncoef * nq * s * C + (dim + 1) * ncomp * s * C + dim * 8 * V + ncomp * s * V)


def adjoint_bytes(dim, prec, C, V, nq):
    """Element kernel (conn, K, lambda, coords, u in; dK, per-element dJ/du out) plus the
    vertex gather (lists and per-element values in, dJ/du out)."""
    s = 8 if prec in ("fp64", "fp64_df") else 4
    nb = dim + 1
    elem = nb * 4 * C + nq * s * C + nb * s * C + dim * 8 * V + s * V + nq * s * C + nb * s * C
    gather = (V + 1) * 4 + nb * C * 4 + nb * s * C + s * V
    return elem + gather


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


KERNEL_SOURCES = {
    # fem_core.cu sizes the launches (grid, occupancy), so it belongs to the kernel's definition
    "lap": ("fem_internal.cuh", "fem_cell.cuh", "fem_f2.cuh", "fem_pipe.cuh", "fem_laplacian.cu", "fem_core.cu"),
    "el": ("fem_internal.cuh", "fem_cell.cuh", "fem_f2.cuh", "fem_elasticity.cu"),
}


def src_hash(files):
    """Hash of the sources that define a kernel (a recorded ncu figure is only reused
    while they are unchanged)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1607_04245_gb300", "csrc")
    for f in files:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel_key, family="lap"):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on the current
    kernel sources (profiles/dram_traffic.txt: '<key> src=<hash> bytes=<n> ...' lines)."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(p):
        return None
    cur = src_hash(KERNEL_SOURCES[family])
    for line in open(p):
        parts = line.split()
        if len(parts) >= 3 and parts[0] == kernel_key:
            kv = dict(x.split("=", 1) for x in parts[1:] if "=" in x)
            if kv.get("src") == cur:
                return float(kv["bytes"])
    return None


class ClockSampler:
    """nvidia-smi samples (100 ms) of SM clock, power and throttle reasons."""

    FIELDS = ("timestamp,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.uuid = uuid
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100"], stdout=self.file, stderr=subprocess.DEVNULL)
            time.sleep(0.6)  # nvidia-smi start-up
        except Exception:
            self.proc = None
        return self

    def stop(self, t_begin, t_end):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        rows = []
        with open(self.file.name) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    ts = _dt.datetime.strptime(p[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                except ValueError:
                    continue
                if self.uuid and p[1] != self.uuid:
                    continue
                rows.append((ts, p))
        os.unlink(self.file.name)
        inside = [p for ts, p in rows if t_begin - 0.05 <= ts <= t_end + 0.05] or [p for _, p in rows[-3:]]
        if not inside:
            return None

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(p[2]) for p in inside if num(p[2]) is not None]
        reasons = set()
        for p in inside:
            for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"), p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": num(inside[0][3]),
                "power_w_max": max((num(p[4]) or 0.0) for p in inside), "samples": len(inside),
                "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------- distributed


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    return int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")), ws


def dist_init(ws, backend):
    import torch.distributed as dist

    if ws > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return dist


def barrier(dist, ws):
    if ws > 1:
        dist.barrier()


def max_over_ranks(dist, ws, x, device):
    if ws == 1:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(ws, cells_per_rank, steps, t_max):
    """Whole-job throughput: every rank integrates its own copy of the workload (independent
    problems, no data-path collective); the job's time is the slowest rank's."""
    return ws * cells_per_rank * steps / t_max


# ----------------------------------------------------------------------------- timing


WARM_S = 0.25  # minimum wall time of the warm-up: the GPU leaves its idle clocks first


def timed_steps(step_fn, steps, warmup, stream, flush, dist=None, ws=1, sampler=None):
    """Per-step device time (ms) of step_fn with an L2 flush before every step.

    The clock sampler starts first (its start-up leaves the GPU idle for a moment); then
    come the warm-up steps -- at least `warmup` of them and at least WARM_S seconds of
    them, so that the timed steps do not run while the clocks ramp up from idle."""
    import torch

    if sampler:
        sampler.start()
    t_w, n = time.time(), 0
    while n < warmup or time.time() - t_w < WARM_S:
        flush()
        step_fn()
        n += 1
        if n % 16 == 0:
            torch.cuda.synchronize()  # keep the queue of enqueued steps short
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    barrier(dist, ws)
    torch.cuda.synchronize()
    t0 = time.time()
    for a, b in evs:
        flush()
        a.record(stream)
        step_fn()
        b.record(stream)
    torch.cuda.synchronize()
    barrier(dist, ws)
    t1 = time.time()
    clocks = sampler.stop(t0, t1) if sampler else None
    ms = [a.elapsed_time(b) for a, b in evs]
    return ms, t1 - t0, clocks


ROTATE_L2_MULT = 3  # bytes of the other copies between two uses of one copy, in L2 sizes
ROTATE_MAX_SETS = 128


def l2_bytes(device):
    import torch

    return getattr(torch.cuda.get_device_properties(device), "L2_cache_size", 0) or (129 << 20)


def rotating_sets(set_bytes, l2):
    """Copies of a workload to cycle through so that a step never finds its inputs in the
    L2 (of l2 bytes): enough that the other copies' bytes between two uses of one copy are
    at least ROTATE_L2_MULT x the L2. None when that takes more than ROTATE_MAX_SETS."""
    n = max(2, 1 + -(-ROTATE_L2_MULT * l2 // max(1, set_bytes)))
    return n if n <= ROTATE_MAX_SETS else None


def timed_rotating(step_fns, steps, warmup, stream, dist=None, ws=1, sampler=None):
    """Device time (ms) of `steps` steps run back to back between one pair of CUDA events,
    step i on input copy i mod len(step_fns); warm-up as in timed_steps. Returns the mean
    per step of each of up to 5 contiguous chunks of the steps, one entry per step (so that
    sum() is the timed region and the median is over chunks), the wall time, the clock record and
    the host's enqueue time per step (well below the device time per step: the device never
    waits for the host)."""
    import torch

    n = len(step_fns)
    if sampler:
        sampler.start()
    t_w, i = time.time(), 0
    while i < warmup or time.time() - t_w < WARM_S:
        step_fns[i % n]()
        i += 1
        if i % 16 == 0:
            torch.cuda.synchronize()
    torch.cuda.synchronize()
    # events at the bounds of up to 5 contiguous chunks of at least 50 steps: their sum is
    # the timed region, their per-step means give a median. (An event between two steps
    # costs the second one its overlapped start, so chunks are few and long.)
    chunk = max(50, -(-steps // 5))
    bounds = list(range(0, steps, chunk)) + [steps]
    evs = [torch.cuda.Event(enable_timing=True) for _ in bounds]
    barrier(dist, ws)
    torch.cuda.synchronize()
    t0 = time.time()
    evs[0].record(stream)
    for j in range(1, len(bounds)):
        for k in range(bounds[j - 1], bounds[j]):
            step_fns[(i + k) % n]()
        evs[j].record(stream)
    t_enq = time.time() - t0
    torch.cuda.synchronize()
    barrier(dist, ws)
    t1 = time.time()
    clocks = sampler.stop(t0, t1) if sampler else None
    ms = []
    for j in range(1, len(bounds)):
        cnt = bounds[j] - bounds[j - 1]
        ms += [evs[j - 1].elapsed_time(evs[j]) / cnt] * cnt
    return ms, t1 - t0, clocks, t_enq * 1e3 / steps


def _nbytes(ts):
    return sum(t.numel() * t.element_size() for t in ts if t is not None)


def timed_copies(make_step, set_bytes, device, stream, flush, steps, warmup):
    """Time one row. make_step(i) makes copy i of the row's device inputs and outputs
    (i = 0: the originals) and returns (step, outputs): back to back over rotating copies
    when rotating_sets allows (every copy's outputs must then equal copy 0's), else one
    launch at a time after an L2 flush. Returns (per-step ms, timing note, extra fields)."""
    import torch

    n = rotating_sets(set_bytes, l2_bytes(device))
    with torch.cuda.stream(stream):
        if not n:
            ms, _, _ = timed_steps(make_step(0)[0], steps, warmup, stream, flush)
            return ms, "one launch at a time after an L2 flush, CUDA events around each launch", {}
        made = [make_step(i) for i in range(n)]
        ms, _, _, host = timed_rotating([m[0] for m in made], steps, warmup, stream)
    torch.cuda.synchronize()
    for _, outs in made[1:]:
        if not all(torch.equal(a, b) for a, b in zip(outs, made[0][1])):
            raise RuntimeError("an input copy gave different results")
    note = (f"back to back over {n} resident input copies ({n * set_bytes / 1e6:.0f} MB, inputs larger than L2), "
            "one event pair around the timed steps")
    return ms, note, {"host_enqueue_ms_per_step": round(host, 6)}


def measure_fp64_fma_rate(device):
    """float64 FMA instructions per second on this GPU: the library's probe kernel (every
    thread runs 8 independent chains of dependent float64 FMAs), timed with CUDA events;
    the measured peak of the float64 forms' ALU roofline."""
    import torch

    import paper_1607_04245_gb300 as fem

    sms = torch.cuda.get_device_properties(device).multi_processor_count
    n, iters = 256 * 8 * sms, 2048
    out = torch.empty(n, dtype=torch.float64, device=device)
    fem.fem_probe(0, n, iters, out=out)
    best = None
    for _ in range(3):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fem.fem_probe(0, n, iters, out=out)
        b.record()
        torch.cuda.synchronize()
        t = a.elapsed_time(b) * 1e-3
        best = t if best is None else min(best, t)
    return {"fma_per_s": n * iters * 8 / best, "threads": n}


def make_flush(device):
    import torch

    buf = torch.ones(FLUSH_BYTES // 4, dtype=torch.float32, device=device)
    sink = torch.empty((), dtype=torch.float32, device=device)

    def flush():
        torch.sum(buf, dim=(0,), out=sink)  # a full read of the buffer evicts the working set from L2

    return flush


# ----------------------------------------------------------------------------- rows


def device_case(case, prec, device):
    import torch

    import paper_1607_04245_gb300 as fem

    c = case if prec in ("fp64", "fp64_df") else case.rounded_to_f32()
    dt = fem.value_dtype(prec)
    f = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device=device, dtype=dt)
    d = {"coords": torch.from_numpy(c.mesh.coords).to(device), "conn": torch.from_numpy(c.mesh.conn).to(device),
         "u": f(c.u)}
    for k in ("K", "lam", "mu", "adj"):
        if getattr(c, k) is not None:
            d[k] = f(getattr(c, k))
    return c, d


def residual_fn(c, d, prec, stream):
    import paper_1607_04245_gb300 as fem

    q = c.rule
    C = c.n_cells
    dt = fem.value_dtype(prec)
    import torch

    out = torch.empty(((c.dim + 1) * c.n_comp, C), dtype=dt, device=d["coords"].device)
    # the C-ABI call with its arguments marshalled once (PreparedCall): the host enqueues a
    # launch in a few microseconds, well inside the kernel's own time
    if c.physics == "laplacian":
        return out, fem.prepared_integrate_laplacian(d["coords"], d["conn"], d["u"], d["K"], q.points, q.weights,
                                                     out, prec=prec, stream=stream)
    return out, fem.prepared_integrate_elasticity(d["coords"], d["conn"], d["u"], d["lam"], d["mu"], q.points,
                                                  q.weights, out, prec=prec, stream=stream)


def rel_err(gpu, ref):
    g = gpu.double().cpu().numpy()
    return float(np.abs(g - ref).max() / np.abs(ref).max())


def oracle_timed(row, n_cells, fn):
    """Run an oracle call, record its rate beside the GPU row (the CPU oracle on all host
    threads, float64, the same workload) and return its result."""
    import oracle

    t0 = time.perf_counter()
    ref = fn()
    dt = time.perf_counter() - t0
    row["oracle_cells_per_s"] = n_cells / dt
    row["oracle_threads"] = oracle.num_threads()
    return ref


def measure_residual(case, prec, device, stream, flush, steps, warmup, peak, oracle_mod=None, dist=None, ws=1,
                     sampler=None, also_flushed=False):
    """One residual row. Timed back to back over rotating input copies (rotating_sets)
    when the workload allows, else one launch at a time after an L2 flush; with
    also_flushed, the per-launch flushed figure is measured beside the rotating one."""
    import torch

    c, d = device_case(case, prec, device)
    out, fn = residual_fn(c, d, prec, stream)
    set_bytes = sum(v.numel() * v.element_size() for v in d.values()) + out.numel() * out.element_size()
    n_sets = rotating_sets(set_bytes, l2_bytes(device))
    extra = []
    with torch.cuda.stream(stream):
        if n_sets:
            fns = [fn]
            for _ in range(n_sets - 1):
                dk = {k: v.clone() for k, v in d.items()}
                ok, fk = residual_fn(c, dk, prec, stream)
                extra.append((dk, ok))
                fns.append(fk)
            ms, wall, clocks, host_ms = timed_rotating(fns, steps, warmup, stream, dist, ws, sampler)
        else:
            ms, wall, clocks = timed_steps(fn, steps, warmup, stream, flush, dist, ws, sampler)
        if also_flushed or not n_sets:
            msf = ms if not n_sets else timed_steps(fn, min(steps, 500), warmup, stream, flush)[0]
    t = statistics.mean(ms) * 1e-3
    nbytes = algorithmic_bytes(c.physics, c.dim, prec, c.n_cells, c.n_verts, c.rule.n_q)
    row = {"physics": c.physics, "dim": c.dim, "prec": prec, "cells": c.n_cells, "verts": c.n_verts,
           "ms_per_launch": round(statistics.mean(ms), 6), "ms_median": round(statistics.median(ms), 6),
           "timing": (f"back to back over {n_sets} resident input copies ({n_sets * set_bytes / 1e6:.0f} MB, "
                      "inputs larger than L2), one event pair around the timed steps") if n_sets else
                     "one launch at a time after an L2 flush, CUDA events around each launch",
           "cells_per_s": c.n_cells / t, "alg_bytes_per_launch": nbytes, "alg_gbs": nbytes / t / 1e9,
           "hbm_frac_of_measured": nbytes / t / 1e9 / peak,
           "paper_model_gflops": perfmodel.flops_per_cell(c.dim, c.rule.n_q, c.n_comp) * c.n_cells / t / 1e9}
    if n_sets:
        row["host_enqueue_ms_per_step"] = round(host_ms, 6)
    if also_flushed or not n_sets:
        row["ms_per_launch_flushed"] = round(statistics.mean(msf), 6)
        row["ms_median_flushed"] = round(statistics.median(msf), 6)
    torch.cuda.synchronize()
    for _, ok in extra:  # every copy gives the same element vectors
        if not torch.equal(ok, out):
            raise RuntimeError("an input copy gave different element vectors")
    del extra
    if c.physics == "laplacian":
        row["counted_gflops"] = perfmodel.collapsed_laplacian_flops(c.dim, c.rule.n_q) * c.n_cells / t / 1e9
    if oracle_mod is not None:
        torch.cuda.synchronize()
        row["rel_maxnorm_err_vs_oracle"] = rel_err(out, oracle_timed(row, c.n_cells,
                                                                     lambda: oracle_mod.residual_for(c)))
        row["tolerance"] = TOL[prec]
        if c is not case:
            # against the float64 data of the workload itself: the float32 storage of the
            # values included (the line above compares on identical, rounded inputs)
            row["rel_maxnorm_err_vs_oracle_fp64_inputs"] = rel_err(out, oracle_mod.residual_for(case))
    return row, ms, wall, clocks


def measure_geometry_path(case, prec, device, stream, flush, steps, warmup, peak, oracle_mod=None):
    """The paper's layout: J^{-1} and det J precomputed once per mesh (not timed), then the
    residual from conn, u, K and the geometry (timed)."""
    import torch

    import paper_1607_04245_gb300 as fem

    c, d0 = device_case(case, prec, device)
    q = c.rule
    dt = fem.value_dtype(prec)
    res = {}

    def make(i):
        d = d0 if i == 0 else {k: v.clone() for k, v in d0.items()}
        with torch.cuda.stream(stream):
            geom = fem.fem_precompute_geometry(d["coords"], d["conn"], prec=prec, stream=stream)
        out = torch.empty((c.dim + 1, c.n_cells), dtype=dt, device=device)
        if i == 0:
            res["out"] = out
        return fem.fem_integrate_laplacian_geom(d["conn"], c.n_verts, d["u"], d["K"], q.points, q.weights, geom,
                                                out=out, prec=prec, stream=stream, prepare=True), (out,)

    sb = _nbytes([d0["conn"], d0["u"], d0["K"]]) + (c.dim * c.dim + 1 + c.dim + 1) * c.n_cells * (
        8 if prec == "fp64" else 4)  # the timed step's inputs, geometry and outputs
    ms, note, extra = timed_copies(make, sb, device, stream, flush, steps, warmup)
    out = res["out"]
    t = statistics.mean(ms) * 1e-3
    s = 8 if prec == "fp64" else 4
    nb = c.dim + 1
    nbytes = nb * 4 * c.n_cells + q.n_q * s * c.n_cells + (c.dim * c.dim + 1) * s * c.n_cells + nb * s * c.n_cells \
        + s * c.n_verts
    row = {"physics": "laplacian_precomputed_geometry", "dim": c.dim, "prec": prec, "cells": c.n_cells,
           "ms_per_launch": round(statistics.mean(ms), 6), "timing": note, **extra, "cells_per_s": c.n_cells / t,
           "alg_bytes_per_launch": nbytes, "alg_gbs": nbytes / t / 1e9, "hbm_frac_of_measured": nbytes / t / 1e9 / peak,
           "alg_bytes_per_cell": "conn 16 + K 4s + geom 10s + out 4s + (V/C) u s (s = value bytes); geometry "
                                 "precomputed once per mesh, not timed"}
    if oracle_mod is not None:
        torch.cuda.synchronize()
        row["rel_maxnorm_err_vs_oracle"] = rel_err(out, oracle_timed(row, c.n_cells,
                                                                     lambda: oracle_mod.residual_for(c)))
    return row


def measure_transposed(case, prec, device, stream, flush, steps, warmup, peak, oracle_mod=None,
                       configs=((32, 1), (32, 4), (32, 16), (64, 1), (64, 4), (64, 16), (128, 1), (128, 4), (128, 16),
                                (256, 1), (256, 4), (256, 16))):
    """The paper's thread-transposition kernel on its own data layout (J^{-1}, det J and
    the element coefficients u_e per cell): a sweep over cells per batch and batches per
    block (the analogue of the paper's Table 2). Timed: the kernel; also timed: the
    closure u -> u_e that a new u costs (the paper performs it on the host)."""
    import torch

    import paper_1607_04245_gb300 as fem

    c, d = device_case(case, prec, device)
    q = c.rule
    dt = fem.value_dtype(prec)
    s = 8 if prec == "fp64" else 4
    nb = c.dim + 1
    nbytes = nb * s * c.n_cells + q.n_q * s * c.n_cells + (c.dim * c.dim + 1) * s * c.n_cells + nb * s * c.n_cells
    with torch.cuda.stream(stream):
        geom = fem.fem_precompute_geometry(d["coords"], d["conn"], prec=prec, stream=stream)
        ue = fem.fem_element_values(d["conn"], c.n_verts, d["u"], prec=prec, stream=stream)
        out = torch.empty((nb, c.n_cells), dtype=dt, device=device)
        sweep = {}
        for cpb, bpb in configs:
            if prec == "fp64" and cpb > 128:
                continue
            fn = lambda: fem.fem_integrate_laplacian_transposed(ue, d["K"], q.points, q.weights, geom, cpb, bpb,
                                                                out=out, prec=prec, stream=stream)
            ms, _, _ = timed_steps(fn, steps, warmup, stream, flush)
            t = statistics.mean(ms) * 1e-3
            sweep[f"{cpb}x{bpb}"] = {"ms": round(statistics.mean(ms), 6), "cells_per_s": c.n_cells / t,
                                     "alg_gbs": nbytes / t / 1e9, "hbm_frac_of_measured": nbytes / t / 1e9 / peak}
        closure = lambda: fem.fem_element_values(d["conn"], c.n_verts, d["u"], ue=ue, prec=prec, stream=stream)
        ms_c, _, _ = timed_steps(closure, steps, warmup, stream, flush)
    best = min(sweep, key=lambda k: sweep[k]["ms"])
    row = {"physics": "laplacian_thread_transposition", "dim": c.dim, "prec": prec, "cells": c.n_cells,
           "alg_bytes_per_cell": "u_e 4s + K 4s + geom 10s + out 4s (s = value bytes); geometry once per mesh",
           "best": best, "best_ms": sweep[best]["ms"], "best_cells_per_s": sweep[best]["cells_per_s"],
           "best_hbm_frac_of_measured": sweep[best]["hbm_frac_of_measured"],
           "closure_ms": round(statistics.mean(ms_c), 6), "sweep_cells_per_batch_x_batches": sweep}
    if oracle_mod is not None:
        fem.fem_integrate_laplacian_transposed(ue, d["K"], q.points, q.weights, geom, 64, 4, out=out, prec=prec,
                                               stream=stream)
        torch.cuda.synchronize()
        row["rel_maxnorm_err_vs_oracle"] = rel_err(out, oracle_timed(row, c.n_cells,
                                                                     lambda: oracle_mod.residual_for(c)))
    return row


def measure_adjoint(case, prec, device, stream, flush, steps, warmup, peak, oracle_mod=None):
    import torch

    import paper_1607_04245_gb300 as fem

    c, d0 = device_case(case, prec, device)
    q = c.rule
    dt = fem.value_dtype(prec)
    res = {}

    def make(i):
        d = d0 if i == 0 else {k: v.clone() for k, v in d0.items()}
        with torch.cuda.stream(stream):
            ptr, idx = fem.fem_build_node2cell(d["conn"], c.n_verts, stream=stream)
        dK = torch.empty((q.n_q, c.n_cells), dtype=dt, device=device)
        du = torch.empty(c.n_verts, dtype=dt, device=device)
        scratch = torch.empty((c.dim + 1, c.n_cells), dtype=dt, device=device)
        if i == 0:
            res["dK"], res["du"] = dK, du
        return fem.fem_adjoint_laplacian(d["coords"], d["conn"], d["u"], d["K"], q.points, q.weights, d["adj"], ptr,
                                         idx, dK=dK, du=du, scratch=scratch, prec=prec, stream=stream,
                                         prepare=True), (dK, du)

    sz = 8 if prec in ("fp64", "fp64_df") else 4
    sb = _nbytes(d0.values()) + (q.n_q + c.dim + 1) * c.n_cells * sz + c.n_verts * sz \
        + 4 * ((c.dim + 1) * c.n_cells + c.n_verts + 1)  # inputs, dK, scratch, du, vertex-to-cell lists
    ms, note, extra = timed_copies(make, sb, device, stream, flush, steps, warmup)
    dK, du = res["dK"], res["du"]
    t = statistics.mean(ms) * 1e-3
    nbytes = adjoint_bytes(c.dim, prec, c.n_cells, c.n_verts, q.n_q)
    row = {"physics": "laplacian_adjoint", "dim": c.dim, "prec": prec, "cells": c.n_cells,
           "ms_per_step": round(statistics.mean(ms), 6), "timing": note, **extra, "cells_per_s": c.n_cells / t,
           "alg_bytes_per_step": nbytes, "alg_gbs": nbytes / t / 1e9, "hbm_frac_of_measured": nbytes / t / 1e9 / peak,
           "kernels_per_step": 2}
    if oracle_mod is not None:
        torch.cuda.synchronize()
        rK, ru = oracle_timed(row, c.n_cells, lambda: oracle_mod.adjoint_for(c))
        row["rel_err_dK"] = rel_err(dK, rK)
        row["rel_err_du"] = rel_err(du, ru)
        row["tolerance"] = TOL[prec]
        if c is not case:  # against the unrounded float64 u, K and lambda
            rK64, ru64 = oracle_mod.adjoint_for(case)
            row["rel_err_dK_fp64_inputs"] = rel_err(dK, rK64)
            row["rel_err_du_fp64_inputs"] = rel_err(du, ru64)
    return row


def measure_reaction(case, prec, device, stream, flush, steps, warmup, peak, oracle_mod=None, drift=1.0):
    """Reaction-diffusion with a P1 auxiliary field and its gradient (Eqs. 2 and 8):
    f1 = a grad u, f0 = c u + drift grad a . grad u, on the case's mesh."""
    import torch

    import paper_1607_04245_gb300 as fem

    c, d = device_case(case, prec, device)
    a_np, c_np = workloads.reaction_inputs(c)
    if prec != "fp64":
        a_np, c_np = (x.astype(np.float32).astype(np.float64) for x in (a_np, c_np))
    dt = fem.value_dtype(prec)
    a_d = torch.from_numpy(a_np).to(device=device, dtype=dt)
    c_d = torch.from_numpy(np.ascontiguousarray(c_np)).to(device=device, dtype=dt)
    q = c.rule
    d0 = dict(d, a=a_d, c=c_d)
    res = {}

    def make(i):
        dd = d0 if i == 0 else {k: v.clone() for k, v in d0.items()}
        out = torch.empty((c.dim + 1, c.n_cells), dtype=dt, device=device)
        if i == 0:
            res["out"] = out
        return fem.fem_integrate_reaction_diffusion(dd["coords"], dd["conn"], dd["u"], dd["a"], q.points, q.weights,
                                                    c=dd["c"], a_space=1, drift=drift, out=out, prec=prec,
                                                    stream=stream, prepare=True), (out,)

    sb = _nbytes(d0.values()) + (c.dim + 1) * c.n_cells * (8 if prec == "fp64" else 4)
    ms, note, extra = timed_copies(make, sb, device, stream, flush, steps, warmup)
    out = res["out"]
    t = statistics.mean(ms) * 1e-3
    s = 8 if prec == "fp64" else 4
    nb = c.dim + 1
    nbytes = nb * 4 * c.n_cells + q.n_q * s * c.n_cells + nb * s * c.n_cells + (c.dim * 8 + 2 * s) * c.n_verts
    row = {"physics": "reaction_diffusion_p1_grad_a", "dim": c.dim, "prec": prec, "cells": c.n_cells,
           "drift": drift, "ms_per_launch": round(statistics.mean(ms), 6), "timing": note, **extra,
           "cells_per_s": c.n_cells / t,
           "alg_bytes_per_launch": nbytes, "alg_gbs": nbytes / t / 1e9, "hbm_frac_of_measured": nbytes / t / 1e9 / peak,
           "alg_bytes_per_cell": "conn 4(d+1) + c n_q s + out (d+1) s + (V/C)(coords 8d + u s + a s)"}
    if oracle_mod is not None:
        torch.cuda.synchronize()
        ref = oracle_timed(row, c.n_cells, lambda: oracle_mod.reaction_diffusion(
            c.mesh.coords, c.mesh.conn, c.u, a_np, 1, c_np, q.points, q.weights, drift=drift))
        row["rel_maxnorm_err_vs_oracle"] = rel_err(out, ref)
        row["tolerance"] = TOL[prec]
        if prec != "fp64":
            a64, c64 = workloads.reaction_inputs(case)
            row["rel_maxnorm_err_vs_oracle_fp64_inputs"] = rel_err(out, oracle_mod.reaction_diffusion(
                case.mesh.coords, case.mesh.conn, case.u, a64, 1, c64, q.points, q.weights, drift=drift))
    return row


def measure_prepared(case, device, stream, flush, steps, warmup, peak, oracle_mod=None):
    """The mixed-form Laplacian from prepared vertex records (fem_prepare_vertices once per
    mesh, timed separately; fem_integrate_laplacian_prepared timed like the headline): one
    32-byte record load per vertex instead of three coordinate gathers and three splits."""
    import torch

    import paper_1607_04245_gb300 as fem

    c, d = device_case(case, "mixed", device)
    q = c.rule
    with torch.cuda.stream(stream):
        rec = fem.fem_prepare_vertices(d["coords"], stream=stream)
        ms_prep, _, _ = timed_steps(lambda: fem.fem_prepare_vertices(d["coords"], rec=rec, stream=stream), steps,
                                    warmup, stream, flush)
    res = {}

    def make(i):
        dd = dict(d, rec=rec) if i == 0 else {k: v.clone() for k, v in dict(d, rec=rec).items()}
        out = torch.empty((c.dim + 1, c.n_cells), dtype=torch.float32, device=device)
        if i == 0:
            res["out"] = out
        return fem.fem_integrate_laplacian_prepared(dd["coords"], dd["rec"], dd["conn"], dd["u"], dd["K"], q.points,
                                                    q.weights, out=out, stream=stream, prepare=True), (out,)

    sb = _nbytes(list(d.values()) + [rec]) + (c.dim + 1) * c.n_cells * 4
    ms, note, extra = timed_copies(make, sb, device, stream, flush, steps, warmup)
    out = res["out"]
    t = statistics.mean(ms) * 1e-3
    C, V, nb = c.n_cells, c.n_verts, c.dim + 1
    R = 8 if c.dim == 3 else 4
    nbytes = nb * 4 * C + q.n_q * 4 * C + nb * 4 * C + (R * 4 + 4) * V
    row = {"physics": "laplacian_prepared_vertex_records", "dim": c.dim, "prec": "mixed", "cells": C,
           "ms_per_launch": round(statistics.mean(ms), 6), "timing": note, **extra,
           "cells_per_s": C / t, "alg_bytes_per_launch": nbytes, "alg_gbs": nbytes / t / 1e9,
           "hbm_frac_of_measured": nbytes / t / 1e9 / peak,
           "prepare_ms_per_mesh": round(statistics.mean(ms_prep), 6),
           "alg_bytes_per_cell": "conn 4(d+1) + K 4 n_q + out 4(d+1) + (V/C)(record 4R + u 4), R = 8 (3D) or 4 (2D)",
           "kernel": "lap_rec_kernel (the pair kernel with one 32-byte record load per vertex, no splits)"}
    if oracle_mod is not None:
        torch.cuda.synchronize()
        row["rel_maxnorm_err_vs_oracle"] = rel_err(out, oracle_timed(row, C, lambda: oracle_mod.residual_for(c)))
    return row


POINTWISE_SRC = {
    "laplacian": "for (int i = 0; i < DIM; ++i) f1[i] = a[0] * grad_u[i];",
    # the oracle's "nonlinear" physics: kappa(u, x) = (p0 + p1 u + p2 u^2)(1 + p3 (x_0 + 2 x_1 + 3 x_2))
    "nonlinear": ("T s = T(0);\nfor (int i = 0; i < DIM; ++i) s += T(i + 1) * x[i];\n"
                  "const T kappa = (T(1.3) + T(-0.7) * u[0] + T(0.45) * u[0] * u[0]) * (T(1) + T(0.35) * s);\n"
                  "for (int i = 0; i < DIM; ++i) f1[i] = kappa * grad_u[i];"),
}
POINTWISE_PARAMS = (1.3, -0.7, 0.45, 0.35)


def measure_pointwise(case, physics, prec, device, stream, flush, steps, warmup, peak, oracle_mod=None):
    """User physics compiled at run time (fem_integrate_pointwise, Sec. 5): the Laplacian
    written as a source string, or the nonlinear kappa(u, x) grad u of Sec. 2, on the
    headline mesh. The compilation happens once, before the timed steps."""
    import torch

    import paper_1607_04245_gb300 as fem

    c, d = device_case(case, prec, device)
    q = c.rule
    dt = fem.value_dtype(prec)
    coef = d["K"][None].contiguous() if physics == "laplacian" else None
    out = torch.empty((c.dim + 1, c.n_cells), dtype=dt, device=device)
    t0 = time.perf_counter()
    fem.fem_integrate_pointwise(d["coords"], d["conn"][:, :0].contiguous(), d["u"], None if coef is None else
                                coef[:, :, :0].contiguous(), q.points, q.weights, f1=POINTWISE_SRC[physics],
                                prec=prec)
    compile_s = time.perf_counter() - t0
    d0 = dict(d, coef=coef) if coef is not None else dict(d)
    d0.pop("K", None)

    def make(i):
        dd = d0 if i == 0 else {k: v.clone() for k, v in d0.items()}
        o = out if i == 0 else torch.empty_like(out)
        return fem.fem_integrate_pointwise(dd["coords"], dd["conn"], dd["u"], dd.get("coef"), q.points, q.weights,
                                           f1=POINTWISE_SRC[physics], out=o, prec=prec, stream=stream,
                                           prepare=True), (o,)

    ms, note, extra = timed_copies(make, _nbytes(d0.values()) + _nbytes([out]), device, stream, flush, steps, warmup)
    t = statistics.mean(ms) * 1e-3
    s = 8 if prec == "fp64" else 4
    nb, C, V = c.dim + 1, c.n_cells, c.n_verts
    ncoef = 1 if coef is not None else 0
    nbytes = nb * 4 * C + ncoef * q.n_q * s * C + nb * s * C + (c.dim * 8 + s) * V
    row = {"physics": f"pointwise_{physics}", "dim": c.dim, "prec": prec, "cells": C,
           "ms_per_launch": round(statistics.mean(ms), 6), "timing": note, **extra, "cells_per_s": C / t,
           "alg_bytes_per_launch": nbytes, "alg_gbs": nbytes / t / 1e9, "hbm_frac_of_measured": nbytes / t / 1e9 / peak,
           "compile_s": round(compile_s, 3),
           "alg_bytes_per_cell": "conn 4(d+1) + coef n_coef n_q s + out (d+1) s + (V/C)(coords 8d + u s)",
           "kernel": "fem_pointwise_kernel (NVRTC, one cell per thread, per-point evaluation of Eq. 2)"}
    if oracle_mod is not None:
        torch.cuda.synchronize()
        if physics == "laplacian":
            ref = oracle_timed(row, C, lambda: oracle_mod.residual_for(c))
        else:
            ref = oracle_timed(row, C, lambda: oracle_mod.pointwise("nonlinear", c.mesh.coords, c.mesh.conn, c.u, None,
                                                                    q.points, q.weights, params=POINTWISE_PARAMS))
        row["rel_maxnorm_err_vs_oracle"] = rel_err(out, ref)
        row["tolerance"] = TOL[prec]
    return row


def measure_pcg(case, device, stream, peak, prec="fp64", rtol=1e-8, max_iter=5000, reps=2):
    """The matrix-free Jacobi-PCG solve with the assembled float64 operator (Eq. 2, E^T of
    the element residuals; prec "fp64_df": the residual in the double-float form) on the
    case's mesh and coefficient, boundary held at a linear g. Per iteration (all on the
    device, a CUDA graph WHILE loop): one residual launch, one vertex gather, the vector
    updates and three dot products."""
    import torch

    import paper_1607_04245_gb300 as fem

    c, d = device_case(case, prec, device)
    q = c.rule
    fixed_np, x0_np = workloads.dirichlet_problem(c)
    ptr, idx = fem.fem_build_node2cell(d["conn"], c.n_verts)
    fixed = torch.from_numpy(fixed_np).to(device)
    x0 = torch.from_numpy(x0_np).to(device)
    work = torch.empty(max(1, int(fem.binding.lib().fem_pcg_work_bytes(c.dim, c.n_cells, c.n_verts,
                                                                         fem.binding.precision(prec)))),
                       dtype=torch.uint8, device=device)
    times, iters, resid = [], 0, 0.0
    for _ in range(reps + 1):
        x = x0.clone()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, iters, resid = fem.fem_pcg_laplacian(d["coords"], d["conn"], d["K"], q.points, q.weights, ptr, idx, fixed,
                                                x, max_iter=max_iter, rtol=rtol, work=work, prec=prec,
                                                stream=stream)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    t = statistics.median(times[1:])  # the first solve warms up
    C, V, nb = c.n_cells, c.n_verts, c.dim + 1
    # per iteration: residual + gather (lists, element vectors, result) + mask, 3 dots,
    # the update of x, r, z and the new direction (float64 vectors of V entries)
    per_it = (algorithmic_bytes("laplacian", c.dim, "fp64", C, V, q.n_q)
              + (V + 1) * 4 + nb * C * 4 + nb * C * 8 + V * 8
              + V * (1 + 16) + 3 * V * 16 + V * (7 * 8 + 3 * 8) + V * 24)
    return {"physics": "pcg_laplacian", "dim": c.dim, "prec": prec, "cells": C, "verts": V, "rtol": rtol,
            "iterations": iters, "rel_residual": resid, "ms_per_solve": t * 1e3, "us_per_iteration": t / iters * 1e6,
            "alg_bytes_per_iteration": per_it, "alg_gbs": per_it * iters / t / 1e9,
            "hbm_frac_of_measured": per_it * iters / t / 1e9 / peak,
            "timing": "host wall clock around the whole solve (two host synchronisations per solve; the "
                      "iterations run as a device-side graph loop); median of 2 solves after one warm-up; L2 not "
                      "flushed between iterations"}


def measure_pcg_elasticity(device, stream, prec="fp64_df", rtol=1e-8, max_iter=20000, reps=2, refined=False):
    """The device-loop Jacobi-PCG for linear elasticity on the 3D elasticity workload mesh
    (2^21 tets), boundary held at a linear displacement, zero load."""
    import torch

    import paper_1607_04245_gb300 as fem

    case = workloads.elasticity_case(3)
    c, d = device_case(case, prec, device)
    q = c.rule
    x = c.mesh.coords
    fixed_np = np.any((np.abs(x) < 1e-14) | (np.abs(x - x.max(axis=1, keepdims=True)) < 1e-14), axis=0)
    g = np.stack([0.1 * x[0] + 0.2 * x[1], -0.1 * x[2], 0.05 * x[0] + 0.3 * x[1]])
    x0_np = np.where(fixed_np[None, :], g, 0.0)
    ptr, idx = fem.fem_build_node2cell(d["conn"], c.n_verts)
    fixed = torch.from_numpy(fixed_np.astype(np.uint8)).to(device)
    x0 = torch.from_numpy(x0_np).to(device=device, dtype=fem.value_dtype(prec))
    work = torch.empty(max(1, int(fem.binding.lib().fem_pcg_elasticity_work_bytes(
        c.dim, c.n_cells, c.n_verts, fem.binding.precision(prec)))), dtype=torch.uint8, device=device)
    if refined:
        K64 = lambda a: torch.from_numpy(np.ascontiguousarray(getattr(case, a))).to(device=device, dtype=torch.float64)
        lam64, mu64 = K64("lam"), K64("mu")
        x064 = torch.from_numpy(x0_np).to(device)
        times, res = [], None
        for _ in range(reps + 1):
            xs = x064.clone()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res = fem.fem_pcg_elasticity_refined(d["coords"], d["conn"], lam64, mu64, q.points, q.weights, ptr, idx,
                                                 fixed, xs, max_outer=30, max_inner=20000, inner_rtol=1e-4,
                                                 rtol=rtol, residual_prec="fp64_df", stream=stream)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
        t = statistics.median(times[1:])
        return {"physics": "pcg_elasticity_refined", "dim": c.dim, "residual_prec": "fp64_df", "cells": c.n_cells,
                "verts": c.n_verts, "unknowns": c.dim * c.n_verts, "rtol": rtol, "outer_steps": res[1],
                "inner_iterations": res[2], "rel_residual": res[3], "ms_per_solve": t * 1e3,
                "timing": "host wall clock around the whole solve; median of 2 solves after one warm-up"}
    times, iters, resid = [], 0, 0.0
    for _ in range(reps + 1):
        xs = x0.clone()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, iters, resid = fem.fem_pcg_elasticity(d["coords"], d["conn"], d["lam"], d["mu"], q.points, q.weights,
                                                 ptr, idx, fixed, xs, max_iter=max_iter, rtol=rtol, work=work,
                                                 prec=prec, stream=stream)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    t = statistics.median(times[1:])
    return {"physics": "pcg_elasticity", "dim": c.dim, "prec": prec, "cells": c.n_cells, "verts": c.n_verts,
            "unknowns": c.dim * c.n_verts, "rtol": rtol, "iterations": iters, "rel_residual": resid,
            "ms_per_solve": t * 1e3, "us_per_iteration": t / max(iters, 1) * 1e6,
            "timing": "host wall clock around the whole solve; median of 2 solves after one warm-up"}


def measure_pcg_refined(case, device, stream, residual_prec="fp64", rtol=1e-8, inner_rtol=1e-4, reps=2):
    """The same solve by mixed-precision iterative refinement: float64 iterate, residuals
    in residual_prec, corrections by the FP32-mixed PCG (the headline kernel as its
    operator). Reported beside the float64 PCG on the same problem: time, outer and inner
    iterations, the final relative residual (float64) and the difference to the float64
    PCG's solution."""
    import torch

    import paper_1607_04245_gb300 as fem

    c, d = device_case(case, "fp64", device)
    q = c.rule
    fixed_np, x0_np = workloads.dirichlet_problem(c)
    ptr, idx = fem.fem_build_node2cell(d["conn"], c.n_verts)
    fixed = torch.from_numpy(fixed_np).to(device)
    x0 = torch.from_numpy(x0_np).to(device)
    work = torch.empty(max(1, int(fem.binding.lib().fem_pcg_refined_work_bytes(c.dim, c.n_cells, c.n_verts,
                                                                                 q.n_q))),
                       dtype=torch.uint8, device=device)
    times, outer, inner, resid, x = [], 0, 0, 0.0, None
    for _ in range(reps + 1):
        x = x0.clone()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, outer, inner, resid = fem.fem_pcg_laplacian_refined(
            d["coords"], d["conn"], d["K"], q.points, q.weights, ptr, idx, fixed, x, max_outer=30, max_inner=5000,
            inner_rtol=inner_rtol, rtol=rtol, work=work, residual_prec=residual_prec, stream=stream)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    t = statistics.median(times[1:])
    x64 = x0.clone()
    fem.fem_pcg_laplacian(d["coords"], d["conn"], d["K"], q.points, q.weights, ptr, idx, fixed, x64, max_iter=5000,
                          rtol=rtol, prec="fp64", stream=stream)
    torch.cuda.synchronize()
    diff = ((x - x64).abs().max() / x64.abs().max()).item()
    return {"physics": "pcg_laplacian_refined", "dim": c.dim, "residual_prec": residual_prec, "cells": c.n_cells,
            "verts": c.n_verts, "rtol": rtol, "inner_rtol": inner_rtol, "outer_steps": outer,
            "inner_iterations": inner, "rel_residual": resid, "ms_per_solve": t * 1e3,
            "rel_maxnorm_diff_vs_fp64_pcg": diff,
            "timing": "host wall clock around the whole solve; median of 2 solves after one warm-up"}


def measure_fields(case, prec, device, stream, flush, steps, warmup, peak, oracle_mod=None, n_fields=8):
    """n_fields nodal fields on one mesh and coefficient in one launch (the cell geometry
    computed once per cell and reused for every field)."""
    import torch

    import paper_1607_04245_gb300 as fem

    c, d = device_case(case, prec, device)
    rng = np.random.default_rng(2024)
    U = rng.uniform(-1.0, 1.0, (n_fields, c.n_verts))
    if prec != "fp64":
        U = U.astype(np.float32).astype(np.float64)
    dt = fem.value_dtype(prec)
    U_d = torch.from_numpy(U).to(device=device, dtype=dt)
    q = c.rule
    out = torch.empty((n_fields, c.dim + 1, c.n_cells), dtype=dt, device=device)
    d0 = dict(d, U=U_d)
    d0.pop("u", None)

    def make(i):
        dd = d0 if i == 0 else {k: v.clone() for k, v in d0.items()}
        o = out if i == 0 else torch.empty_like(out)
        return fem.fem_integrate_laplacian_fields(dd["coords"], dd["conn"], dd["U"], dd["K"], q.points, q.weights,
                                                  out=o, prec=prec, stream=stream, prepare=True), (o,)

    ms, note, extra = timed_copies(make, _nbytes(d0.values()) + _nbytes([out]), device, stream, flush, steps, warmup)
    t = statistics.mean(ms) * 1e-3
    sz = 8 if prec == "fp64" else 4
    C, V, nb = c.n_cells, c.n_verts, c.dim + 1
    nbytes = nb * 4 * C + q.n_q * sz * C + c.dim * 8 * V + n_fields * (sz * V + nb * sz * C)
    row = {"physics": "laplacian_fields", "dim": c.dim, "prec": prec, "cells": C, "fields": n_fields,
           "ms_per_launch": round(statistics.mean(ms), 6), "timing": note, **extra,
           "field_cells_per_s": n_fields * C / t,
           "alg_bytes_per_launch": nbytes, "alg_gbs": nbytes / t / 1e9, "hbm_frac_of_measured": nbytes / t / 1e9 / peak,
           "alg_bytes_per_cell": "conn 4(d+1) + K n_q s + (V/C) coords 8d + F ((V/C) u s + out (d+1) s)"}
    if oracle_mod is not None:
        torch.cuda.synchronize()
        refs = oracle_timed(row, n_fields * C, lambda: [oracle_mod.laplacian(c.mesh.coords, c.mesh.conn, U[f], c.K,
                                                                              q.points, q.weights)
                                                         for f in range(n_fields)])
        row["oracle_field_cells_per_s"] = row.pop("oracle_cells_per_s")
        row["rel_maxnorm_err_vs_oracle"] = max(rel_err(out[f], refs[f]) for f in range(n_fields))
        row["tolerance"] = TOL[prec]
    return row


def measure_e2e(case, prec, device, steps, warmup):
    """Same metric through the host-buffer API: H2D of all inputs, kernel, D2H of the result."""
    import torch

    from paper_1607_04245_gb300.host import HostIntegrator

    c = case if prec in ("fp64", "fp64_df") else case.rounded_to_f32()
    import paper_1607_04245_gb300 as fem

    dt = fem.value_dtype(prec)
    hi = HostIntegrator(device)
    coords_h = hi.pinned("coords", c.mesh.coords, torch.float64)
    conn_h = hi.pinned("conn", c.mesh.conn, torch.int32)
    u_h = hi.pinned("u", c.u, dt)
    K_h = hi.pinned("K", c.K, dt)
    step = lambda: hi.laplacian(coords_h, conn_h, u_h, K_h, c.rule.points, c.rule.weights, prec=prec)
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    hi.h2d_bytes = hi.d2h_bytes = 0
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(hi.stream)
    for _ in range(steps):
        step()
    b.record(hi.stream)
    b.synchronize()
    t = a.elapsed_time(b) * 1e-3 / steps
    return {"value": c.n_cells / t, "unit": "cells/s", "h2d_bytes_per_step": hi.h2d_bytes // steps,
            "d2h_bytes_per_step": hi.d2h_bytes // steps, "ms_per_step": t * 1e3}


def measure_serving(device, n_requests, seed=0):
    """Serving stream: n requests (residual or adjoint, 2D/3D Laplacian and elasticity,
    log-uniform 1e3..1e6 cells, fresh seeded meshes), FP32-mixed. First all requests at
    t = 0 (saturation: the service capacity in requests/s), then Poisson arrivals at the
    highest of 85/70/55/40 % of that capacity whose backlog stays bounded; p50/p99 latency
    from arrival to observed completion. The saturation stream runs five times and each
    Poisson stream three times, after one warm-up run through each loop; the median run is
    reported beside all runs. Both loops are measured on the same requests: the native one
    (fem_serve_run, the whole stream in one call; reported first) and the Python one
    (serving.Scheduler, one native launch call per request)."""
    from paper_1607_04245_gb300.serving import (GpuExecutor, NativeScheduler, Scheduler, make_request,
                                                poisson_arrivals)

    t_gen = time.time()
    specs = workloads.cases.serving_specs(n_requests, seed=seed)
    reqs = [make_request(sp["rid"], workloads.cases.serving_case(sp), sp["kind"], "mixed") for sp in specs]
    t_gen = time.time() - t_gen
    ex = GpuExecutor(device, capacity=2 << 30, n_slots=16)

    def reset(arrivals):
        for r, a in zip(reqs, arrivals):
            r.arrival, r.status = float(a), "pending"

    # warm-up: every request once through each loop (the first device access to each pinned
    # host block is slower than the later ones, and the native loop's first run sets up its
    # own state: it served at a quarter of its rate)
    for loop in (Scheduler, NativeScheduler):
        reset([0.0] * len(reqs))
        loop(ex).run(reqs)
    h2d = sum(r.input_bytes for r in reqs)
    d2h = sum(sum(t.numel() * t.element_size() for t in r.result.values()) for r in reqs)
    link = host_link_rates(device)
    link_s = max(h2d / link["h2d_gbs"], d2h / link["d2h_gbs"], (h2d + d2h) / link["both_gbs"]) / 1e9

    def curve(make):
        # the loop is host-bound and the host is shared, so the saturation stream is run five
        # times (the Poisson streams three) and the median run is reported
        sats = []
        for _ in range(5):
            reset([0.0] * len(reqs))
            sats.append(make().run(reqs))
        sat = sorted(sats, key=lambda x: x.req_per_s)[2]
        # the operating curve: Poisson arrivals at 85/70/55/40 % of the saturation rate, every
        # fraction measured; the sustained rate is the highest fraction whose backlog stays
        # bounded (served rate within 3 % of the offered rate in the median run)
        sweep, st, rate, p99_runs = [], None, None, None
        for frac in (0.85, 0.70, 0.55, 0.40):
            r_off = frac * sat.req_per_s
            runs = []
            for _ in range(3):
                reset(poisson_arrivals(len(reqs), r_off, seed=seed + 1))
                runs.append(make().run(reqs, arrival_rate=r_off))
            med = sorted(runs, key=lambda x: x.p99_ms)[1]
            bounded = med.req_per_s >= 0.97 * r_off
            sweep.append({"fraction": frac, "offered_req_per_s": r_off, "served_req_per_s": med.req_per_s,
                          "p50_ms": med.p50_ms, "p99_ms": med.p99_ms, "bounded_backlog": bounded,
                          "p99_ms_of_3_runs": sorted(x.p99_ms for x in runs)})
            if bounded and st is None:
                st, rate, p99_runs = med, r_off, sweep[-1]["p99_ms_of_3_runs"]
        if st is None:
            st, rate, p99_runs = med, r_off, sweep[-1]["p99_ms_of_3_runs"]
        # what bounds the saturation rate: the bytes each request moves across the host link
        # against this box's measured link rates, and the host time per request
        bound = {"h2d_bytes": h2d, "d2h_bytes": d2h, "served_h2d_gbs": h2d / sat.makespan_s / 1e9,
                 "served_d2h_gbs": d2h / sat.makespan_s / 1e9, "link": link,
                 "link_floor_s": link_s, "link_fraction_of_makespan": link_s / sat.makespan_s,
                 "makespan_s": sat.makespan_s, "makespan_us_per_request": sat.makespan_s / len(reqs) * 1e6,
                 "reading": "link_fraction_of_makespan near 1: the host link bounds the rate; well below 1: the "
                            "per-request host work (admission, launch, polling) or the device does"}
        return {"saturation": {"req_per_s": sat.req_per_s, "cells_per_s": sat.cells_per_s, "p50_ms": sat.p50_ms,
                               "p99_ms": sat.p99_ms, "makespan_s": sat.makespan_s, "failed": sat.n_failed,
                               "req_per_s_of_5_runs": sorted(x.req_per_s for x in sats)},
                "poisson": {"arrival_rate_req_per_s": rate, "req_per_s": st.req_per_s, "cells_per_s": st.cells_per_s,
                            "p50_ms": st.p50_ms, "p99_ms": st.p99_ms, "mean_ms": st.mean_ms,
                            "max_inflight": st.max_inflight, "rejected": st.n_rejected, "failed": st.n_failed,
                            "makespan_s": st.makespan_s, "cells": st.cells, "p99_ms_of_3_runs": p99_runs},
                "rate_sweep": sweep, "saturation_bound": bound}

    native = curve(lambda: NativeScheduler(ex))
    python_loop = curve(lambda: Scheduler(ex))
    kinds = {}
    for sp in specs:
        k = f"{sp['physics']}{sp['dim']}d_{sp['kind']}"
        kinds[k] = kinds.get(k, 0) + 1
    out = {"requests": n_requests, "generation_s": round(t_gen, 2), "mix": kinds,
           "arena_bytes": ex.arena.capacity, "slots": ex.n_slots,
           "loop": "native: fem_serve_run serves the whole stream in one call"}
    out.update(native)
    out["python_loop"] = dict(python_loop, loop="serving.Scheduler: Python admission and polling, one native "
                                                "launch call per request")
    return out


def host_link_rates(device, nbytes=64 << 20):
    """Host<->device copy rates of this machine (GB/s) between page-locked host memory and the
    device: host to device, device to host, and both directions at once (two streams);
    best of 3, CUDA events."""
    import torch

    h = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    h2 = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    d = torch.empty(nbytes, dtype=torch.uint8, device=device)
    d2 = torch.empty(nbytes, dtype=torch.uint8, device=device)
    s1, s2 = torch.cuda.Stream(device=device), torch.cuda.Stream(device=device)

    def best(fn):
        t = None
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            t = dt if t is None else min(t, dt)
        return t

    def both():
        with torch.cuda.stream(s1):
            d.copy_(h, non_blocking=True)
        with torch.cuda.stream(s2):
            h2.copy_(d2, non_blocking=True)

    return {"h2d_gbs": nbytes / best(lambda: d.copy_(h, non_blocking=True)) / 1e9,
            "d2h_gbs": nbytes / best(lambda: h2.copy_(d2, non_blocking=True)) / 1e9,
            "both_gbs": 2 * nbytes / best(both) / 1e9, "bytes": nbytes}


def cpu_model() -> str:
    """The host CPU as /proc/cpuinfo names it (model name on x86; implementer/part on Arm)."""
    import platform

    info = {}
    try:
        for line in open("/proc/cpuinfo"):
            if ":" in line:
                k, v = line.split(":", 1)
                info.setdefault(k.strip(), v.strip())
    except OSError:
        pass
    name = info.get("model name") or (
        f"implementer {info.get('CPU implementer', '?')} part {info.get('CPU part', '?')}")
    return f"{platform.machine()}, {os.cpu_count()} logical CPUs, {name}"


def cpu_baseline(case, min_seconds=10.0, max_reps=200, single_seconds=4.0):
    """The oracle on the host cores: all threads over the full workload (about
    min_seconds), then one thread on a slice of it (about single_seconds)."""
    import oracle

    oracle.build()
    threads = oracle.num_threads()
    reps, t0 = 0, time.perf_counter()
    while reps < max_reps:
        oracle.residual_for(case)
        reps += 1
        if time.perf_counter() - t0 >= min_seconds:
            break
    dt = time.perf_counter() - t0
    # one thread: the first S cells, S sized from the all-thread rate
    rate_all = case.n_cells * reps / dt
    S = int(min(case.n_cells, max(4096, rate_all / max(1, threads) * single_seconds / 2)))
    m, q = case.mesh, case.rule
    conn = np.ascontiguousarray(m.conn[:, :S])
    K = np.ascontiguousarray(case.K[:, :S])
    oracle.set_threads(1)
    try:
        reps1, t1 = 0, time.perf_counter()
        while True:
            oracle.laplacian(m.coords, conn, case.u, K, q.points, q.weights)
            reps1 += 1
            if time.perf_counter() - t1 >= single_seconds:
                break
        dt1 = time.perf_counter() - t1
    finally:
        oracle.set_threads(threads)
    return {"value": rate_all, "unit": "cells/s", "cores": threads, "kind": "oracle",
            "sample": f"the full {case.n_cells}-cell workload x {reps} repetitions ({dt:.1f} s, float64, "
                      f"OpenMP over cells)",
            "single_thread": {"value": S * reps1 / dt1, "unit": "cells/s", "cores": 1,
                              "sample": f"the first {S} cells x {reps1} repetitions ({dt1:.1f} s)"},
            "cpu": cpu_model()}


# ----------------------------------------------------------------------------- arms


def run_reference(args):
    """The CPU oracle timed as it stands on the host cores (rank 0 only)."""
    rank, _, ws = dist_env()
    if rank != 0:
        return 0
    import oracle

    oracle.build()
    case = workloads.laplacian_cube_case(HEADLINE_CELLS).rounded_to_f32()
    m = case.mesh
    # calibrate, then size each step so the whole run stays around a minute
    t0 = time.perf_counter()
    oracle.residual_for(case)
    rate = case.n_cells / (time.perf_counter() - t0)
    budget = 60.0 / max(1, args.steps + args.warmup)
    S = int(min(case.n_cells, max(4096, rate * budget)))
    S -= S % 4
    nslices = max(1, min(8, case.n_cells // S))
    slices = []
    for i in range(nslices):
        a = i * S
        conn = np.ascontiguousarray(m.conn[:, a:a + S])
        K = np.ascontiguousarray(case.K[:, a:a + S])
        slices.append((conn, K))
    q = case.rule

    def step(i):
        conn, K = slices[i % nslices]
        oracle.laplacian(m.coords, conn, case.u, K, q.points, q.weights)

    for i in range(args.warmup):
        step(i)
    t0 = time.perf_counter()
    for i in range(args.steps):
        step(i)
    dt = time.perf_counter() - t0
    value = S * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "cells": HEADLINE_CELLS, "sample_cells_per_step": S,
                       "form": "float64 CPU oracle on float32-rounded inputs"},
            "cpu_baseline": {"value": value, "unit": "cells/s", "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": f"{S} cells per step (slices of the {HEADLINE_CELLS}-cell workload)"},
            "e2e": {"value": value, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line))
    return 0


def run_ours(args):
    import torch

    import paper_1607_04245_gb300 as fem

    rank, local_rank, ws = dist_env()
    if ws != args.gpus:
        ws = max(ws, 1)
    torch.cuda.set_device(local_rank)
    device = torch.device("cuda", local_rank)
    dist = dist_init(ws, "nccl")
    from paper_1607_04245_gb300 import binding

    binding.lib()
    peak, peak_kind = load_peaks()
    import oracle

    oracle.build()
    stream = torch.cuda.Stream(device=device)
    flush = make_flush(device)
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(device).uuid)
    except Exception:
        pass

    case = workloads.laplacian_cube_case(HEADLINE_CELLS)

    # headline: FP32-mixed residual
    row, ms, wall, clocks = measure_residual(case, "mixed", device, stream, flush, args.steps, args.warmup, peak,
                                             oracle if rank == 0 else None, dist, ws, ClockSampler(uuid),
                                             also_flushed=True)
    t_max = max_over_ranks(dist, ws, sum(ms) * 1e-3, device)
    ms_per_step = t_max / args.steps * 1e3
    value = weak_scaling_value(ws, case.n_cells, args.steps, t_max)

    fp64_steps = max(20, args.steps // 20)  # at least 20 back-to-back steps per row
    row64, _, _, _ = measure_residual(case, "fp64", device, stream, flush, fp64_steps, args.warmup, peak,
                                      oracle if rank == 0 else None)

    if rank != 0:
        barrier(dist, ws)
        return 0

    nbytes = row["alg_bytes_per_launch"]
    achieved = nbytes / (row["ms_per_launch"] * 1e-3) / 1e9
    traffic = recorded_traffic("lap3d_mixed")
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic,
                "traffic_kind": "recorded: ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch of the "
                                "same kernel sources (profiles/dram_traffic.txt, keyed by a hash of the sources; "
                                "null once they change), not measured in this run",
                "peak_kind": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"
                if peak_kind == "measured" else "fallback 6800 GB/s",
                "kernel": HEADLINE_KERNEL,
                "alg_bytes_per_launch": nbytes,
                "alg_bytes_per_cell": "conn 16 + K 16 + out 16 + (V/C)(coords 24 + u 4)"}

    fp64_inst = sum(FP64_INST_PER_CELL_LAP3D.values()) * case.n_cells
    fp64_flops = (2 * FP64_INST_PER_CELL_LAP3D["dfma"] + FP64_INST_PER_CELL_LAP3D["dadd"] +
                  FP64_INST_PER_CELL_LAP3D["dmul"]) * case.n_cells
    t64 = row64["ms_per_launch"] * 1e-3
    sm_mhz = (clocks or {}).get("sm_mhz") or 2070.0
    peak_inst = FP64_NOMINAL_TFLOPS / 2 * (sm_mhz / 2070.0)  # T instructions/s at the sampled clock
    roofline_fp64 = {"bound": "alu", "achieved": fp64_inst / t64 / 1e12, "peak": peak_inst,
                     "unit": "T float64 instructions/s", "frac": fp64_inst / t64 / 1e12 / peak_inst,
                     "achieved_tflops": fp64_flops / t64 / 1e12,
                     "peak_kind": f"nominal {FP64_NOMINAL_TFLOPS} TFLOP/s float64 = 2 FMA instructions/clock/SM, "
                                  f"at the sampled {sm_mhz:.0f} MHz",
                     "kernel": "lap_staged_kernel<3, FP64, NQ=4>",
                     "inst_per_cell": FP64_INST_PER_CELL_LAP3D}

    probe = measure_fp64_fma_rate(device)
    roofline_fp64_measured = dict(roofline_fp64, peak=probe["fma_per_s"] / 1e12,
                                  frac=fp64_inst / t64 / probe["fma_per_s"],
                                  peak_kind="measured in this run: float64 FMA instructions/s of fem_probe kind 0 "
                                            f"({probe['threads']} threads x 8 independent FMA chains, best of 3)")

    rows = {"fp64": row64}
    # float64 values with float32-pair arithmetic: float64-class error, float32-pipe speed
    row_df, _, _, _ = measure_residual(case, "fp64_df", device, stream, flush, fp64_steps, args.warmup, peak,
                                       oracle if rank == 0 else None)
    rows["fp64_df"] = row_df
    # --rows all | none | comma-separated row-name prefixes (e.g. "lap3d_fields8,elast3d")
    picked = None if args.rows in ("all", "none") else [x for x in args.rows.split(",") if x]
    want = lambda name: args.rows == "all" or (picked is not None and any(name.startswith(x) for x in picked))
    def put(name, fn):
        """Measure one optional row; a row that fails is recorded with its error and does not
        cost the bench line."""
        try:
            rows[name] = fn()
        except Exception as exc:  # noqa: BLE001 -- reported in the line and on stderr
            print(f"bench: row {name} failed: {exc!r}", file=sys.stderr)
            rows[name] = {"error": repr(exc)[:300]}

    rsteps = max(20, args.steps // 50)
    common = (device, stream, flush, rsteps, args.warmup, peak, oracle)
    if want("fp32_ablation"):
        put("fp32_ablation", lambda: measure_residual(case, "fp32", *common)[0])
    for prec in ("mixed", "fp64"):
        if want(f"lap3d_precomputed_geometry_{prec}"):
            put(f"lap3d_precomputed_geometry_{prec}", lambda: measure_geometry_path(case, prec, *common))
    for prec in ("fp32", "fp64"):
        if want(f"lap3d_thread_transposition_{prec}"):
            put(f"lap3d_thread_transposition_{prec}", lambda: measure_transposed(case, prec, *common))
    if want("lap2d_8192_fp64"):
        put("lap2d_8192_fp64", lambda: measure_residual(workloads.laplacian_square_case(), "fp64", *common)[0])
    for dim in (2, 3):
        if not any(want(f"elast{dim}d_{prec}") for prec in ("mixed", "fp64", "fp64_df")):
            continue
        el = workloads.elasticity_case(dim)
        for prec in ("mixed", "fp64", "fp64_df"):
            if want(f"elast{dim}d_{prec}"):
                put(f"elast{dim}d_{prec}", lambda: measure_residual(el, prec, *common)[0])
    if any(want(f"adjoint3d_{prec}") for prec in ("mixed", "fp64", "fp64_df")):
        adj = workloads.adjoint_case(HEADLINE_CELLS)
        for prec in ("mixed", "fp64", "fp64_df"):
            if want(f"adjoint3d_{prec}"):
                put(f"adjoint3d_{prec}", lambda: measure_adjoint(adj, prec, *common))
    for prec in ("mixed", "fp64"):
        if want(f"reaction3d_grad_a_{prec}"):
            put(f"reaction3d_grad_a_{prec}", lambda: measure_reaction(case, prec, *common))
    if want("lap3d_prepared_mixed"):
        put("lap3d_prepared_mixed", lambda: measure_prepared(case, *common))
    for prec in ("mixed", "fp64"):
        for phys in ("laplacian", "nonlinear"):
            if want(f"pointwise_{phys}3d_{prec}"):
                put(f"pointwise_{phys}3d_{prec}", lambda: measure_pointwise(case, phys, prec, *common))
    for prec in ("fp64", "fp64_df"):
        if want(f"pcg_lap3d_{prec}"):
            put(f"pcg_lap3d_{prec}", lambda: measure_pcg(case, device, stream, peak, prec))
    for prec in ("fp64_df", "mixed"):
        if want(f"pcg_elast3d_{prec}"):
            put(f"pcg_elast3d_{prec}", lambda: measure_pcg_elasticity(device, stream, prec))
    if want("pcg_elast3d_refined"):
        put("pcg_elast3d_refined", lambda: measure_pcg_elasticity(device, stream, "fp64", refined=True))
    for rprec in ("fp64", "fp64_df"):
        if want(f"pcg_refined_lap3d_{rprec}"):
            put(f"pcg_refined_lap3d_{rprec}", lambda: measure_pcg_refined(case, device, stream, rprec))
    for prec in ("mixed", "fp64"):
        if want(f"lap3d_fields8_{prec}"):
            put(f"lap3d_fields8_{prec}", lambda: measure_fields(case, prec, *common))

    def sweep():
        out = {}
        for e in range(16, 24):
            sc = workloads.laplacian_cube_case(1 << e)
            r = measure_residual(sc, "mixed", device, stream, flush, max(20, rsteps // 2), args.warmup, peak)[0]
            out[str(1 << e)] = {"cells_per_s": r["cells_per_s"], "alg_gbs": r["alg_gbs"],
                                "hbm_frac_of_measured": r["hbm_frac_of_measured"], "ms": r["ms_per_launch"]}
        return out

    if want("sweep_lap3d_mixed"):
        put("sweep_lap3d_mixed", sweep)
    if want("serving") and args.serving_requests > 0:
        put("serving", lambda: measure_serving(device, args.serving_requests))

    try:
        e2e = measure_e2e(case, "mixed", device, max(20, args.steps // 100), 3)
    except Exception as exc:  # noqa: BLE001 -- reported in the line and on stderr
        print(f"bench: e2e failed: {exc!r}", file=sys.stderr)
        e2e = {"error": repr(exc)[:300]}
    # every measured launch's device-side status: a bounded wait that gave up or a mesh error
    # would make the timed work incomplete (0 = FEM_OK)
    device_status = fem.fem_device_error()
    if device_status != 0:
        print(f"bench: fem_device_error() = {device_status} after the measured launches", file=sys.stderr)

    line = {"metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "ms_median": row["ms_median"],
            "ms_per_launch_flushed": row["ms_per_launch_flushed"], "ms_median_flushed": row["ms_median_flushed"],
            "host_enqueue_ms_per_step": row.get("host_enqueue_ms_per_step"),
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "cells": case.n_cells, "verts": case.n_verts,
                       "form": "fp32_mixed (float32 values, float64 coordinates split to float32 pairs, "
                               "compensated quadrature sum, float64 fallback for badly shaped cells)",
                       "l2": "inputs larger than L2: " + row["timing"] + "; ms_per_launch_flushed: one launch "
                             "at a time after an L2 flush (read of a 512 MiB buffer), events around each launch",
                       "parallelism": f"replicas x{ws}"},
            "hbm_gbs": row["alg_gbs"], "hbm_frac_of_measured_peak": row["hbm_frac_of_measured"],
            "hbm_frac_of_nominal_8tbs": row["alg_gbs"] / 8000.0,
            "paper_model_gflops": row["paper_model_gflops"], "counted_gflops": row.get("counted_gflops"),
            "rel_maxnorm_err_vs_oracle": row.get("rel_maxnorm_err_vs_oracle"),
            "rel_maxnorm_err_vs_oracle_fp64_inputs": row.get("rel_maxnorm_err_vs_oracle_fp64_inputs"),
            "fp64": {"cells_per_s": row64["cells_per_s"], "ms_per_launch": row64["ms_per_launch"],
                     "alg_gbs": row64["alg_gbs"], "hbm_frac_of_measured": row64["hbm_frac_of_measured"],
                     "rel_maxnorm_err_vs_oracle": row64.get("rel_maxnorm_err_vs_oracle")},
            "speedup_fp32_mixed_over_fp64": row["cells_per_s"] / row64["cells_per_s"],
            "fp64_df": {"cells_per_s": rows["fp64_df"]["cells_per_s"], "ms_per_launch": rows["fp64_df"]["ms_per_launch"],
                        "rel_maxnorm_err_vs_oracle": rows["fp64_df"].get("rel_maxnorm_err_vs_oracle"),
                        "speedup_over_fp64": rows["fp64_df"]["cells_per_s"] / row64["cells_per_s"],
                        "form": "float64 values, float32-pair arithmetic on the float32 pipe"},
            "roofline": roofline, "roofline_fp64": roofline_fp64, "roofline_fp64_measured": roofline_fp64_measured,
            "cpu_baseline": cpu_baseline(case) if (ws == 1 and not args.no_cpu_baseline) else None,
            "e2e": e2e, "gpu_launches": args.steps,
            "clocks": clocks, "rows": rows,
            "served_p99_ms": rows.get("serving", {}).get("poisson", {}).get("p99_ms"),
            "device_status": device_status}
    print(json.dumps(line))
    barrier(dist, ws)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--rows", default="all",
                    help="all, none, or comma-separated row-name prefixes to measure beside the headline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=500)
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
