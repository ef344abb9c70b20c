#!/usr/bin/env python3
"""Benchmark: D3Q19 + dynamic-IB lattice updates per second on GB300.

Workload (one step = the whole hot path: MLS interpolation at markers and
hydrodynamic probes, structure forces + update + spreading, fused
stream/wall/collide sweep): the largest single-GPU configuration, a rigid
sphere (radius 8, 10242 markers) settling in a closed 160 x 160 x 480 box
(12.3 M cells), tau 0.7, FP32 populations.  The line also carries the
96^3 deformable-capsule Couette cell (tau 0.8, shear rate 1e-4, capsule
radius 10, 2562 markers, Ca 0.05) measured the same way, under
"capsule96".  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl lbib|reference]

Multi-GPU runs (torchrun, one process per GPU) are independent replicas of
the workload (the method has no exchange between separate runs); the
value is the total over ranks divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "D3Q19+IB MLUPS & % HBM peak; served runs/h, p50/p99 latency vs plain"
UNIT = "MLUPS"
FALLBACK_HBM_GBS = 6800.0
# the end-to-end leg runs at least this many steps: a run's set-up (fields
# from the host, mesh upload, graph capture) is paid once per run
E2E_MIN_STEPS = 300


WORKLOADS = {
    "capsule96": "capsule_shear_96^3_Ca0.05_fp32",
    "settling": "settling_sphere_160x160x480_fp32",
    "couette_fp64": "couette_rigid_sphere_32^3_fp64",
    "capsule96_fp64": "capsule_shear_96^3_Ca0.05_fp64",
    "capsule96_fp16": "capsule_shear_96^3_Ca0.05_fp16dev",
    "capsule96_bf16": "capsule_shear_96^3_Ca0.05_bf16dev",
    "settling_fp16": "settling_sphere_160x160x480_fp16dev",
    "settling_bf16": "settling_sphere_160x160x480_bf16dev",
}
# storage of the populations per workload suffix: (precision, bytes per value, C++ type)
STORAGE = {"fp64": ("PREC_FP64", 8, "double"), "fp32": ("PREC_FP32", 4, "float"),
           "fp16": ("PREC_FP16_DEV", 2, "__half"), "bf16": ("PREC_BF16_DEV", 2, "__nv_bfloat16")}


def storage(name):
    suffix = name.rsplit("_", 1)[-1]
    return STORAGE[suffix] if suffix in STORAGE else STORAGE["fp32"]


def workload_case(name="capsule96"):
    from paper_2207_06029_gb300 import workloads as W
    prec = getattr(W, storage(name)[0])
    if name.startswith("settling"):
        return W.case_settling(precision=prec)
    if name == "couette_fp64":
        return W.case_couette_sphere(precision=W.PREC_FP64)
    return W.case_capsule_shear(n=96, tau=0.8, shear_rate=1e-4, radius=10.0, level=4, Ca=0.05, Eb=0.01, kv=1.0,
                                precision=prec)


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def sweep_source_hash():
    """Hash of the source k_sweep compiles from: the node routines
    (sweep_cell.cuh), sweep.cu up to the end of k_sweep and the device header
    up to the body view (the molecule, storage conversions and lattice
    parameters)."""
    csrc = os.path.join(ROOT, "paper_2207_06029_gb300", "csrc")
    cell = open(os.path.join(csrc, "sweep_cell.cuh")).read()
    sweep = open(os.path.join(csrc, "sweep.cu")).read()
    dev = open(os.path.join(csrc, "lbib_device.cuh")).read()
    sweep = sweep[:sweep.index("// The nodes inside the box")]
    dev = dev[:dev.index("struct BodyView")]
    return hashlib.sha256((cell + sweep + dev).encode()).hexdigest()[:16]


SWEEP_PROFILES = {"capsule96": "sweep_fp32_capsule96.md", "settling": "sweep_fp32_settling.md",
                  "couette_fp64": "sweep_fp64_capsule96.md", "capsule96_fp64": "sweep_fp64_capsule96.md"}


def profile_figure(workload, key):
    """A figure (`key: value`) of the workload's committed ncu summary, if
    that was taken on the current sweep source; else None."""
    path = os.path.join(ROOT, "profiles", SWEEP_PROFILES[workload])
    try:
        txt = open(path).read()
    except OSError:
        return None
    m = re.search(key + r":\s*([0-9.eE+]+)", txt)
    s = re.search(r"sweep_source_sha:\s*([0-9a-f]+)", txt)
    if not m or not s or s.group(1) != sweep_source_hash():
        return None
    return float(m.group(1))


def ncu_traffic(workload="capsule96"):
    """DRAM bytes per sweep launch of the workload from its committed ncu
    summary, if that was taken on the current sweep source; else None."""
    if workload not in ("capsule96", "settling"):
        return None  # summaries of DRAM traffic exist for the FP32 lattices
    path = os.path.join(ROOT, "profiles", SWEEP_PROFILES[workload])
    try:
        txt = open(path).read()
    except OSError:
        return None
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    s = re.search(r"sweep_source_sha:\s*([0-9a-f]+)", txt)
    if not m or not s or s.group(1) != sweep_source_hash():
        return None
    return float(m.group(1))


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for name, val in zip(names, parts[3:7]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def torch_allocator(torch):
    """Device allocation through PyTorch's caching allocator."""
    from paper_2207_06029_gb300 import lbib
    live = {}

    def _alloc(nbytes, user):
        t = torch.empty(int(nbytes), dtype=torch.uint8, device="cuda")
        live[t.data_ptr()] = t
        return t.data_ptr()

    def _free(ptr, user):
        live.pop(ptr, None)

    return lbib.ALLOC_FN(_alloc), lbib.FREE_FN(_free), live


def run_gpu(args, rank, world, workload=None):
    import torch

    from paper_2207_06029_gb300 import lbib
    workload = workload or args.workload

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    # a dedicated stream: the library's kernels, the timing events and the
    # L2 flush are all ordered on it
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    case = workload_case(workload)
    alloc_fn, free_fn, live = torch_allocator(torch)
    params = lbib.make_params(case.n, case.tau, bc=case.bc, wall_u=case.wall_u, precision=case.precision,
                              stream=stream.cuda_stream)
    params.alloc, params.free = alloc_fn, free_fn
    h = lbib.lbib_create(params)
    rho0, u0 = case.initial_fields()
    lbib.lbib_set_fields(h, rho0, u0.reshape(-1))
    b = case.bodies[0]
    lbib.lbib_add_body(h, b.verts, b.tris, lbib.make_body_params(**b.kwargs()))
    ncell = case.ncell

    lbib.lbib_step(h, args.warmup)
    if args.autotune:
        tuned = lbib.lbib_autotune(h, 20)  # launch configuration (untimed; advances the run)
    else:
        tuned = (0, 0, 1, 0, 0)
    if args.overlap != "auto":
        lbib.lbib_set_overlap(h, 1 if args.overlap == "on" else 0)
    tuned = lbib.lbib_get_launch_config(h)  # the five choices above and the IB kernels' blocks per SM
    lbib.lbib_sync(h)
    lbib.lbib_set_output(h, -1)  # no macroscopic-field output inside the timed loop
    # the launch configuration is final: capture the six phase graphs of the
    # timed step (one per phase of the buffer rotation) before timing
    lbib.lbib_step(h, 12)
    lbib.lbib_sync(h)
    # L2 flush between timed steps: write a buffer larger than the 129 MB L2,
    # then read another one, so that the write-back of the flush's dirty
    # lines happens before the step and the step starts on a cold, clean L2
    flush_w = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    flush_r = torch.ones(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    flush_acc = torch.empty((), dtype=torch.float32, device="cuda")

    def flush():
        flush_w.zero_()
        torch.sum(flush_r, dim=0, out=flush_acc)

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    stops = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    _, launches0 = lbib.lbib_counters(h)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev) as clk:
        for k in range(args.steps):
            flush()
            starts[k].record(stream)
            lbib.lbib_step(h, 1)
            stops[k].record(stream)
        torch.cuda.synchronize()
    lbib.lbib_sync(h)
    if world > 1:
        torch.distributed.barrier()
    ms = sum(s.elapsed_time(e) for s, e in zip(starts, stops))
    _, launches1 = lbib.lbib_counters(h)
    # stage breakdown: the same steps with the library's CUDA-event timing
    # of each stage (the events add a few microseconds per step, so this
    # loop is kept out of the timed one)
    nprof_steps = min(args.steps, 100)
    lbib.lbib_profile(h, 1)
    lbib.lbib_get_profile(h)
    for k in range(nprof_steps):
        flush()
        lbib.lbib_step(h, 1)
    mls_ms, struct_ms, sweep_ms, step_ms, nprof = lbib.lbib_get_profile(h)
    # the sweep kernel alone (one whole-lattice k_sweep launch per step, no
    # concurrent IB work), timed by CUDA events on the stream it runs on:
    # the roofline of the dominant kernel
    lbib.lbib_set_overlap(h, 0)
    lbib.lbib_get_profile(h)
    for k in range(nprof_steps):
        flush()
        lbib.lbib_step(h, 1)
    _, _, iso_sweep_ms, _, iso_n = lbib.lbib_get_profile(h)
    lbib.lbib_profile(h, 0)
    lbib.lbib_destroy(h)
    live.clear()

    # end to end through the public API with host buffers: create from host
    # fields, upload the mesh, K steps each followed by a read of the markers
    # into pinned host memory, and the fields at the end.  The steps run in
    # chunks of ten through lbib_step_markers, which queues the copy of
    # every step's markers behind it into a pinned ring; the host reads a
    # chunk's markers (a finite check of every value) while the next chunk
    # runs.
    import numpy as np
    import ctypes as C
    chunk = 10
    nvb = b.verts.shape[0]
    Xb = [torch.empty((chunk, nvb, 3), dtype=torch.float64, pin_memory=True) for _ in range(2)]
    Vb = [torch.empty((chunk, nvb, 3), dtype=torch.float64, pin_memory=True) for _ in range(2)]
    Fb = [torch.empty((chunk, nvb, 3), dtype=torch.float64, pin_memory=True) for _ in range(2)]
    ready = [torch.cuda.Event() for _ in range(2)]
    Xh = Xb[0][0]
    rho_h = torch.empty(ncell, dtype=torch.float64, pin_memory=True)
    u_h = torch.empty(3 * ncell, dtype=torch.float64, pin_memory=True)
    rho_in = torch.from_numpy(rho0).pin_memory()
    u_in = torch.from_numpy(np.ascontiguousarray(u0.reshape(-1))).pin_memory()
    e2e_steps = max(args.steps, E2E_MIN_STEPS)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    p2 = lbib.make_params(case.n, case.tau, bc=case.bc, wall_u=case.wall_u, precision=case.precision,
                          stream=stream.cuda_stream)
    p2.alloc, p2.free = alloc_fn, free_fn
    h2 = lbib.lbib_create(p2)
    # the launch configuration tuned above, through the public setters
    lbib.lbib_set_sweep_config(h2, tuned[3], tuned[0], tuned[1], tuned[4])
    lbib.lbib_set_overlap(h2, tuned[2])
    lbib.lbib_set_ib_blocks(h2, tuned[5])
    L = lbib.load()
    L.lbib_set_fields(h2, C.c_void_p(rho_in.data_ptr()), C.c_void_p(u_in.data_ptr()), 0)
    lbib.lbib_add_body(h2, b.verts, b.tris, lbib.make_body_params(**b.kwargs()))
    t_setup = time.perf_counter()
    finite = True

    def consume(j, n):
        nonlocal finite
        ready[j].synchronize()
        finite = finite and bool(np.isfinite(Xb[j][:n].numpy()).all() and np.isfinite(Fb[j][:n].numpy()).all())

    done, c, prev = 0, 0, None
    while done < e2e_steps:
        j, n = c % 2, min(chunk, e2e_steps - done)
        lbib.lbib_step_markers(h2, n, 0, Xb[j], Vb[j], Fb[j])
        ready[j].record(stream)
        if prev is not None:
            consume(*prev)
        prev = (j, n)
        done += n
        c += 1
    consume(*prev)
    L.lbib_get_fields(h2, C.c_void_p(rho_h.data_ptr()), C.c_void_p(u_h.data_ptr()), 0)
    t1 = time.perf_counter()
    if not finite:
        raise RuntimeError("non-finite markers in the end-to-end run")
    lbib.lbib_destroy(h2)
    live.clear()
    e2e_s = t1 - t0
    e2e_setup_s = t_setup - t0
    h2d = (rho0.nbytes + u0.nbytes + b.verts.nbytes + b.tris.nbytes) / e2e_steps
    d2h = 3 * Xh.numel() * 8 + (rho_h.numel() + u_h.numel()) * 8 / e2e_steps
    return {"ms": ms, "sweep_ms": sweep_ms, "mls_ms": mls_ms, "struct_ms": struct_ms, "nprof": nprof,
            "step_ms": step_ms, "iso_sweep_us": 1e3 * iso_sweep_ms / max(iso_n, 1), "tuned": tuned,
            "launches": launches1 - launches0,
            "clocks": clk.summary(), "ncell": ncell, "e2e_s": e2e_s, "e2e_steps": e2e_steps, "h2d": h2d,
            "e2e_setup_s": e2e_setup_s,
            "d2h": d2h, "nv": int(b.verts.shape[0]), "nt": int(b.tris.shape[0])}


def device_fields(torch, case):
    """Initial density and velocity of a case as CUDA tensors (set without
    the library's host staging buffer)."""
    rho, u = case.initial_fields()
    return (torch.from_numpy(rho).cuda(), torch.from_numpy(np.ascontiguousarray(u.reshape(-1))).cuda())


def large_sweep_leg(args):
    """The same whole-lattice sweep measured the same way (overlap off, L2
    written and read clean before each step, CUDA events on the stream) on
    the 160x160x480 settling lattice, where the launch ramp is a small part
    of the kernel: the sweep's roofline on a lattice large enough to stream."""
    import torch

    from paper_2207_06029_gb300 import lbib
    stream = torch.cuda.current_stream()
    case = workload_case("settling")
    alloc_fn, free_fn, live = torch_allocator(torch)
    params = lbib.make_params(case.n, case.tau, bc=case.bc, wall_u=case.wall_u, precision=case.precision,
                              stream=stream.cuda_stream)
    params.alloc, params.free = alloc_fn, free_fn
    h = lbib.lbib_create(params)
    rho, u = device_fields(torch, case)
    lbib.lbib_set_fields(h, rho, u)
    b = case.bodies[0]
    lbib.lbib_add_body(h, b.verts, b.tris, lbib.make_body_params(**b.kwargs()))
    lbib.lbib_step(h, 3)
    lbib.lbib_set_output(h, -1)
    lbib.lbib_set_overlap(h, 0)
    flush_w = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    flush_r = torch.ones(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    acc = torch.empty((), dtype=torch.float32, device="cuda")
    lbib.lbib_profile(h, 1)
    lbib.lbib_get_profile(h)
    n = 10
    for _ in range(n):
        flush_w.zero_()
        torch.sum(flush_r, dim=0, out=acc)
        lbib.lbib_step(h, 1)
    _, _, sweep_ms, _, nprof = lbib.lbib_get_profile(h)
    lbib.lbib_profile(h, 0)
    lbib.lbib_destroy(h)
    live.clear()
    us = 1e3 * sweep_ms / max(nprof, 1)
    peak, kind = hbm_peak()
    achieved = 152.0 * case.ncell / (us * 1e-6) / 1e9
    return {"workload": "settling sphere 160x160x480 (12.3 M cells), fp32", "kernel": "k_sweep<float,float>",
            "sweep_us": us, "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": ncu_traffic("settling"), "peak_source": kind, "launches_timed": nprof}


def batch_leg(args):
    """64 capsule-in-shear cases of uneven cubic lattices (48^3..112^3)
    advanced together by the batch launches, six steps per graph launch."""
    import torch

    from paper_2207_06029_gb300 import lbib
    from paper_2207_06029_gb300 import workloads as W
    cases, params = W.case_batch(count=args.batch_count, precision=W.PREC_FP32)
    stream = torch.cuda.current_stream()
    ctxs = []
    for case in cases:
        ctx = lbib.Context(case.n, case.tau, bc=case.bc, wall_u=case.wall_u, precision=case.precision,
                           stream=stream.cuda_stream)
        rho, u = device_fields(torch, case)
        lbib.lbib_set_fields(ctx.h, rho, u)
        for bd in case.bodies:
            ctx.add_body(bd.verts, bd.tris, **bd.kwargs())
        ctxs.append(ctx)
    torch.cuda.synchronize()
    batch = lbib.Batch(ctxs, stream=stream.cuda_stream)
    if args.batch_mode == "persistent":  # the persistent kernel, sweep tiles of 4096 cells
        batch.set_config(256, 1, 16)
        batch.set_persistent(1)
        tuned = (-1, 1, 16)
    elif args.batch_mode == "split":  # one sweep launch per lattice
        batch.set_config(0, 1, 4)
        tuned = (0, 1, 4)
    else:
        tuned = batch.autotune(2) if args.autotune else (256, 0, 4)
    batch.step(12)
    batch.sync()
    steps = max(6, (args.batch_steps // 6) * 6)
    _, l0 = batch.counters()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    batch.step(steps + 1)  # six-step graph launches plus the field-storing last step
    e1.record(stream)
    torch.cuda.synchronize()
    batch.sync()
    _, l1 = batch.counters()
    ms = e0.elapsed_time(e1)
    cells = sum(c.ncell for c in cases)
    out = {"workload": f"{len(cases)} capsule-in-shear cases, cubic N~U{{48..112}}, radius N/10, 642/2562 markers, "
                       "fp32",
           "value": cells * (steps + 1) / (ms * 1e-3) / 1e6, "unit": UNIT, "steps": steps + 1,
           "ms_per_step": ms / (steps + 1), "cells": cells, "markers": sum(len(c.bodies[0].verts) for c in cases),
           "launches_per_step": (l1 - l0) / (steps + 1),
           "autotuned": {"sweep": ("persistent kernel, six steps a launch, sweep tiles of "
                                   f"{256 * tuned[2]} cells" if tuned[0] == -1 else
                                   "one launch per lattice" if tuned[0] == 0 else
                                   f"batched, {tuned[0]} threads, {tuned[2]} cells per thread"),
                         "lattice_order": ["as given", "largest first"][tuned[1]]},
           "hbm_frac_sweep_bytes": cells * 152.0 * (steps + 1) / (ms * 1e-3) / 1e9 / hbm_peak()[0],
           "parameters": {"Ca": list(W.BATCH_CA), "Eb": list(W.BATCH_EB), "mass_ratio": list(W.BATCH_MASS_RATIOS)},
           "inputs": "larger than L2 (6.2 GB of populations per step)"}
    batch.close()
    for ctx in ctxs:
        ctx.close()
    return out


SERVE_STREAMS = {
    # the serving configuration as stated: Poisson 4/s, cubic N 32..192,
    # 2000..30000 steps, capsules (N >= 48) in the validated parameter box
    "stated": dict(count=64, seed=4, rate=4.0, n_range=(32, 192), step_range=(2000, 30000)),
    # the same stream with the capsule parameter box as stated (Ca 0.005..0.3,
    # Eb 0..0.05, mass ratio 0.5/1/2) and capsules from N = 32: runs that
    # diverge fail with LBIB_EDIVERGED and leave the batch
    "stated_full": dict(count=64, seed=4, rate=4.0, n_range=(32, 192), step_range=(2000, 30000),
                          capsule_min_n=32),
    # many small lattices, where one run alone leaves the GPU idle
    "small": dict(count=64, seed=9, rate=40.0, n_range=(32, 64), step_range=(500, 2000)),
}


def serve_leg(args, mode, precision, max_active=64, batch_cells=0, stream_kind="stated", batch_order=0):
    """A seeded Poisson stream of capsule-in-shear and settling-sphere runs
    through the serving engine; latency from submission to completion.  The
    step counts of the stated streams are scaled by args.serve_steps_scale."""
    from paper_2207_06029_gb300 import lbib
    from paper_2207_06029_gb300 import workloads as W
    kw = dict(SERVE_STREAMS[stream_kind])
    if stream_kind.startswith("stated"):
        scale = getattr(args, "serve_steps_scale", 1.0)
        kw["step_range"] = tuple(max(1, int(round(scale * x))) for x in kw["step_range"])
    if stream_kind == "stated_full":
        kw.update(Ca_range=W.FULL_CA, Eb_range=W.FULL_EB, mass_ratios=W.FULL_MASS_RATIOS)
    stream = W.serve_stream(precision=precision, **kw)
    server = lbib.lbib_serve_create(hbm_budget=150 << 30, chunk_steps=500, max_active=max_active, mode=mode,
                                    batch_cells=batch_cells, batch_order=batch_order)
    reqs = [(t, lbib.request_from_case(case, steps), case, steps) for t, case, steps in stream]
    t0 = time.perf_counter()
    ids = []
    for t, req, case, steps in reqs:
        now = time.perf_counter() - t0
        if t > now:
            time.sleep(t - now)
        ids.append(lbib.lbib_serve_submit(server, req))
    lat, failed = [], []
    for rid, (t, req, case, steps) in zip(ids, reqs):
        rc, state = lbib.lbib_serve_wait(server, rid, 600.0)
        h, times, rc = lbib.lbib_serve_take(server, rid)
        if h is not None:
            lbib.lbib_destroy(h)
        if rc:
            failed.append({"request": case.name, "steps": steps, "code": rc, "error": times["error"]})
        else:
            lat.append(times["latency_s"])
    makespan = time.perf_counter() - t0
    stats = lbib.lbib_serve_stats(server)
    lbib.lbib_serve_destroy(server)
    lat = sorted(lat)
    pct = lambda q: lat[min(len(lat) - 1, int(round(q * (len(lat) - 1))))] if lat else None
    codes = {}
    for f in failed:
        codes[str(f["code"])] = codes.get(str(f["code"]), 0) + 1
    return {"runs": len(lat), "failed": len(failed), "failed_by_code": codes, "makespan_s": makespan,
            "runs_per_h": len(lat) / makespan * 3600.0, "p50_s": pct(0.5), "p99_s": pct(0.99),
            "mlups": stats["cell_updates"] / makespan / 1e6,
            "busy_mlups": stats["cell_updates"] / max(stats["busy_s"], 1e-9) / 1e6,
            "chunks": stats["chunks"], "batch_rebuilds": stats["rebuilds"], "peak_bytes": stats["peak_bytes"]}


def max_over_ranks(values, device):
    """Element-wise maximum of per-rank timings over all ranks (the slowest
    rank sets the whole job's time)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def job_mlups(cells_per_rank, steps, world, ms):
    """Whole-job throughput of independent replicas: the cell updates of all
    ranks over the slowest rank's time."""
    return cells_per_rank * steps * world / (ms * 1e-3) / 1e6


def cpu_baseline(seconds=12.0, min_steps=2, workload="capsule96"):
    """The FP64 oracle on the same workload, on the host cores, for a bounded
    number of steps (about `seconds` of CPU work)."""
    import oracle
    case = workload_case(workload)
    s = oracle.Sim(case.n, case.tau, bc=case.bc, wall_u=case.wall_u.ravel())
    s.set_fields(*case.initial_fields())
    b = case.bodies[0]
    s.add_body(b.verts, b.tris, **b.kwargs())
    steps = 0
    t0 = time.perf_counter()
    while steps < min_steps or time.perf_counter() - t0 < seconds:
        assert s.step(1) == 0
        steps += 1
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": case.ncell * steps / dt / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{steps} steps of the {WORKLOADS[workload]} case (FP64 oracle, OpenMP over z-planes)"}


def cpu_baseline_one_core(seconds=6.0, workload="capsule96"):
    """The same sample on one host core: a fresh process (the oracle's
    OpenMP team is sized when its library loads) with OMP_NUM_THREADS=1."""
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-sample", str(seconds),
                        "--workload", workload], env=env, capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        return {"error": r.stderr.strip().splitlines()[-1] if r.stderr.strip() else f"exit {r.returncode}"}
    return json.loads(r.stdout.strip().splitlines()[-1])


def measured_line(args, r, world, ms, workload):
    """The JSON line's figures for one measured workload (run_gpu's result r,
    the slowest rank's timed milliseconds ms)."""
    value = job_mlups(r["ncell"], args.steps, world, ms)
    peak, peak_kind = hbm_peak()
    fp64 = workload.endswith("fp64")
    _, elem, ctype = storage(workload)
    bytes_per_cell = 38.0 * elem  # 19 reads + 19 writes of one stored value per cell
    bytes_per_launch = bytes_per_cell * r["ncell"]
    achieved = bytes_per_launch / (r["iso_sweep_us"] * 1e-6) / 1e9
    concurrent_s = r["sweep_ms"] * 1e-3 / max(r["nprof"], 1)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {8: "f64", 4: "fp32", 2: "fp32 (fp16/bf16 storage)"}[elem], "data": "synthetic",
        "config": {"workload": WORKLOADS[workload], "cells": r["ncell"], "markers": r["nv"], "triangles": r["nt"],
                   "parallelism": f"replicas{world}", "l2": "flushed between timed steps (256 MiB write, then 256 MiB read)",
                   "fields_output": "off in the timed loop (e2e reads them)",
                   "autotuned": {"sweep_block": list(r["tuned"][:2]), "overlap": bool(r["tuned"][2]),
                                 "sweep_row_tiles": bool(r["tuned"][3]), "far_field_blocks_per_sm": r["tuned"][4],
                                 "ib_blocks_per_sm": r["tuned"][5]},
                   "populations": ("fp64 deviations f_i - w_i, fp64 arithmetic" if fp64 else
                                   f"{ctype} deviations f_i - w_i, fp32 arithmetic; marker positions and rigid "
                                   "states fp64")},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": ncu_traffic(workload),
                     "kernel": ("k_sweep_tile<{0},{1}> (shared-memory row tiles, 128-bit loads/stores)"
                                if r["tuned"][3] else "k_sweep<{0},{1}>").format(ctype, "double" if fp64 else "float"),
                     "peak_source": peak_kind, "sweep_us": r["iso_sweep_us"],
                     "sweep_in_step_us": 1e6 * concurrent_s,
                     "sweep_in_step_frac": bytes_per_launch / concurrent_s / 1e9 / peak,
                     "mls_us_per_step": 1e3 * r["mls_ms"] / max(r["nprof"], 1),
                     "structure_us_per_step": 1e3 * r["struct_ms"] / max(r["nprof"], 1),
                     "step_us_per_step": 1e3 * r["step_ms"] / max(r["nprof"], 1),
                     "note": f"achieved = {bytes_per_cell:.0f} B/cell x cells / the mean CUDA-event duration of the whole-lattice "
                             "k_sweep launch (one per step, overlap off, L2 flushed before each step); "
                             "sweep_in_step_* and the stage times come from a profiled loop of the tuned step, "
                             "where the sweep runs as two launches, the far field concurrently with the IB "
                             "stage"},
        "e2e": {"value": r["ncell"] * r["e2e_steps"] * world / r["e2e_s"] / 1e6, "unit": UNIT,
                "h2d_bytes_per_step": int(r["h2d"]), "d2h_bytes_per_step": int(r["d2h"]),
                "steps": r["e2e_steps"], "setup_ms": 1e3 * r["e2e_setup_s"],
                "note": "context creation from host fields, mesh upload and graph capture included; the markers "
                        "of every step staged on the device behind the step, copied to pinned host buffers after "
                        "each chunk of ten steps and checked on the host while the next chunk runs; the fields "
                        "read at the end"},
        "gpu_launches": r["launches"],
        "clocks": r["clocks"],
    }
    if fp64:
        # the FP64 sweep issues its arithmetic on GB300's narrow FP64 pipe:
        # its roofline is the measured FP64 FMA rate, the FP64 operations per
        # cell counted by ncu (committed summary) times the cells per launch
        flop_cell = profile_figure(workload, "fp64_flop_per_cell")
        inst_cell = profile_figure(workload, "fp64_inst_per_cell")
        from paper_2207_06029_gb300 import lbib
        fma64 = lbib.lbib_measure_fma(True)
        # the pipe issues one FP64 instruction per slot: 2 flops as an FMA,
        # 1 as an add or a multiply; the peak for the sweep's mix
        peak = fma64 / 1e12 * (flop_cell / inst_cell / 2.0 if flop_cell and inst_cell else 1.0)
        hbm = line["roofline"]
        line["roofline"] = {"bound": "alu", "unit": "TFLOP/s", "peak": peak,
                            "peak_source": "measured FP64 FMA rate (lbib_measure_fma) x the sweep's flop per "
                                           "FP64 instruction / 2 (ncu instruction counts, committed summary)",
                            "fma_tflops": fma64 / 1e12,
                            "flop_per_cell": flop_cell, "kernel": hbm["kernel"], "sweep_us": r["iso_sweep_us"],
                            "achieved": (flop_cell * r["ncell"] / (r["iso_sweep_us"] * 1e-6) / 1e12
                                         if flop_cell else None),
                            "traffic": None, "hbm_view": {k: hbm[k] for k in ("achieved", "peak", "unit", "frac")}}
        for k in ("sweep_in_step_us", "mls_us_per_step", "structure_us_per_step", "step_us_per_step"):
            line["roofline"][k] = hbm[k]
        line["roofline"]["frac"] = (line["roofline"]["achieved"] / line["roofline"]["peak"]
                                    if flop_cell else None)
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="lbib", choices=["lbib", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="settling", choices=sorted(WORKLOADS))
    ap.add_argument("--no-extra", dest="extra", action="store_false",
                    help="skip the 96^3 capsule figure beside the settling workload")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="keep the default launch configuration")
    ap.add_argument("--no-batch", dest="batch", action="store_false", help="skip the batched-lattices leg")
    ap.add_argument("--batch-steps", type=int, default=60)
    ap.add_argument("--batch-count", type=int, default=64, help="lattices in the batched leg")
    ap.add_argument("--batch-mode", default="auto", choices=["auto", "persistent", "split"],
                    help="batched leg: autotuned launch configuration, the persistent kernel, or one sweep "
                         "launch per lattice")
    ap.add_argument("--batch-only", action="store_true",
                    help="only run the batched leg and print its figures (a diagnostic line)")
    ap.add_argument("--no-serve", dest="serve", action="store_false", help="skip the serving leg")
    ap.add_argument("--serve-steps-scale", type=float, default=0.25,
                    help="step counts of the stated serving stream (2000..30000) times this (1: full length, "
                         "about 90 s a leg)")
    ap.add_argument("--overlap", default="auto", choices=["auto", "on", "off"],
                    help="far-field sweep concurrent with the IB stage (auto: as tuned)")
    ap.add_argument("--cpu-sample", type=float, default=0.0,
                    help="only time the oracle for this many seconds on the host and print its figure")
    args = ap.parse_args()
    if args.cpu_sample > 0:
        print(json.dumps(cpu_baseline(args.cpu_sample, workload=args.workload)))
        return
    if args.warmup < 3:
        args.warmup = 3

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))

    if args.impl == "reference":
        # the reference arm is the FP64 oracle on the host cores (rank 0 only)
        if rank != 0:
            return
        import oracle
        case = workload_case(args.workload)
        s = oracle.Sim(case.n, case.tau, bc=case.bc, wall_u=case.wall_u.ravel())
        s.set_fields(*case.initial_fields())
        b = case.bodies[0]
        s.add_body(b.verts, b.tris, **b.kwargs())
        assert s.step(min(args.warmup, 5)) == 0  # untimed warm-up steps
        ksteps = max(1, min(args.steps, 40))
        t0 = time.perf_counter()
        assert s.step(ksteps) == 0
        dt = time.perf_counter() - t0
        val = case.ncell * ksteps / dt / 1e6
        cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
        line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
                "steps": ksteps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / ksteps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": {"workload": WORKLOADS[args.workload], "cells": case.ncell},
                "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                                 "sample": f"{ksteps} steps of the {WORKLOADS[args.workload]} case"},
                "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    if args.batch_only:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        torch.cuda.set_stream(torch.cuda.Stream())
        print(json.dumps({"batch": batch_leg(args)}))
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    r = run_gpu(args, rank, world)
    import torch
    ms_all = [r["ms"]]
    if world > 1:
        ms_max, r["e2e_s"] = max_over_ranks([r["ms"], r["e2e_s"]], "cuda")
        ms_all = [ms_max]
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    ms = ms_all[0]
    line = measured_line(args, r, world, ms, args.workload)
    if rank == 0 and world == 1 and args.workload == "settling" and args.extra:
        # the 96^3 capsule, measured the same way, as a second figure
        rc = run_gpu(args, rank, world, "capsule96")
        lc = measured_line(args, rc, world, rc["ms"], "capsule96")
        line["capsule96"] = {k: lc[k] for k in ("value", "unit", "ms_per_step", "config", "roofline", "e2e",
                                               "gpu_launches", "clocks")}
    if rank == 0 and world == 1 and args.workload == "capsule96":
        line["roofline_large_lattice"] = large_sweep_leg(args)
    if args.batch and rank == 0 and world == 1:
        line["batch"] = batch_leg(args)
    if args.serve and rank == 0 and world == 1:
        from paper_2207_06029_gb300 import lbib
        from paper_2207_06029_gb300 import workloads as W
        lo, hi = (max(1, int(round(args.serve_steps_scale * x))) for x in SERVE_STREAMS["stated"]["step_range"])
        stream = (f"64 requests, Poisson 4/s, half capsule-in-shear half settling sphere, cubic N~U{{32..192}}, "
                  f"steps~U{{{lo}..{hi}}} (the stated 2000..30000 x {args.serve_steps_scale:g}), budget 150 GB")
        line["serve"] = {
            "stream": stream + "; capsules N >= 48 in the validated parameter box",
            "plain_fp32": serve_leg(args, lbib.LBIB_SERVE_PLAIN, W.PREC_FP32),
            "batched_fp32_oldest_1M": serve_leg(args, lbib.LBIB_SERVE_BATCHED, W.PREC_FP32, batch_cells=1 << 20,
                                                batch_order=lbib.LBIB_SERVE_OLDEST),
            "batched_fp16_dev_oldest_1M": serve_leg(args, lbib.LBIB_SERVE_BATCHED, W.PREC_FP16_DEV,
                                                    batch_cells=1 << 20, batch_order=lbib.LBIB_SERVE_OLDEST),
            "full_box_stream": stream + "; capsules from N = 32 in the stated box (Ca 0.005..0.3, Eb 0..0.05, "
                                        "mass ratio 0.5/1/2): diverging runs fail with LBIB_EDIVERGED (-4)",
            "full_box_batched_fp32_oldest_1M": serve_leg(args, lbib.LBIB_SERVE_BATCHED, W.PREC_FP32,
                                                         batch_cells=1 << 20, batch_order=lbib.LBIB_SERVE_OLDEST,
                                                         stream_kind="stated_full"),
            "small_stream": "64 requests, Poisson 40/s, same mix, cubic N~U{32..64} (capsules 48..64), "
                            "steps~U{500..2000}",
            "small_batched_fp32": serve_leg(args, lbib.LBIB_SERVE_BATCHED, W.PREC_FP32, stream_kind="small"),
            "small_plain_fp32": serve_leg(args, lbib.LBIB_SERVE_PLAIN, W.PREC_FP32, stream_kind="small"),
        }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds, workload=args.workload)
        line["cpu_baseline"]["one_core"] = cpu_baseline_one_core(workload=args.workload)
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
