#!/usr/bin/env python
"""Benchmark of the assembly-free deflated FE hot path on one GB300.

One step = one topology iteration of the method on the 128x64x64 voided
cantilever (524,288 hex8 elements, 1,635,075 DOFs), inputs resident in HBM:
set the element moduli, build the coarse problem W^T K W and its factor,
solve K u = f to relative residual 1e-6 with FP32 inner deflated PCG inside
FP64 iterative refinement, compliance J = f^T u, the strain-energy
sensitivity field, and the level-set update at volume fraction 0.9.  The
moduli are reset at the start of every step, so every step does the same work.

Timing: W untimed warm-up steps, then K steps each bracketed by CUDA events on
torch's current stream (every library call returns after its own stream has
finished), an L2 flush (write of 512 MB) between timed steps, max over ranks.
`e2e` repeats the step through the same C-ABI calls with host numpy buffers
(host-to-device copies of the moduli and loads, device-to-host copies of u,
J and the field inside the timed region).

Three more legs run at N = 1 after the timed steps: "levelset" (20 steps of
compliance-constrained volume minimisation on the 384x192x192 mesh, warm
started), "batched" (the 96x48x48
mesh with 8 load cases in one multi-RHS solve, against one case at a time and
against the FP64 path) and "serve" (256 requests of mixed mesh sizes through
the serving loop under a 60 GB budget: saturated solves/s, and p50/p99 latency
at 0.8 x that rate).  `cpu_baseline` times the CPU oracle on a bounded sample.

    python bench.py [--steps K] [--warmup W] [--impl ours|reference]
                    [--no-serve] [--no-batched] [--no-levelset] [--no-cpu-baseline]

Under torchrun (N > 1) every rank solves its own replica (independent
problems, no collective on the data path): weak scaling.  `ms_per_step` is
the slowest rank's time per step; `value` is the whole job's time per step,
that time divided by N.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "dCG solve ms & GDOF/s matvec at rel-res 1e-6, mixed vs FP64 on GB300; serve p50/p99"
VOLUME_FRACTION = 0.9
UNIT = "ms per topology step (dCG solve to rel-res 1e-6 + coarse setup + J + sensitivity + level-set)"
# DRAM bytes (read + write) per launch of the FP32 apply kernel, each from one ncu capture of the kernel at that
# size (summarised under profiles/), keyed by mesh and CTA shape (warps, planes, async staging); any other shape
# reports null.
# FP32 operations of the modal hex8 apply per element (x/y butterflies 18, z butterfly 21, modal forces 42,
# transposed z 30, y 12 and x 15 stages: 138 operations, 9 of them FMAs counted twice), and the FP32 peak from the
# unit counts: SMs (read from the device) x 128 FP32 lanes x 2 flops per FMA x the maximum SM clock.
STENCIL_FLOPS_PER_ELEMENT = 147
FP32_LANES_PER_SM = 128
_SM_COUNT = {"n": None, "source": "nominal GB300 (no device queried)"}


def device_sm_count(dev=None) -> int:
    """Number of SMs of the device the bench runs on (queried once; 152 on a
    GB300 when no device can be asked, e.g. in CPU tests)."""
    if _SM_COUNT["n"] is None:
        try:
            import torch
            if torch.cuda.is_available():
                _SM_COUNT["n"] = int(torch.cuda.get_device_properties(dev or 0).multi_processor_count)
                _SM_COUNT["source"] = "torch.cuda.get_device_properties().multi_processor_count"
        except Exception:  # pragma: no cover
            pass
        if _SM_COUNT["n"] is None:
            _SM_COUNT["n"] = 152
    return _SM_COUNT["n"]


def sm_max_mhz() -> float:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return float(json.load(open(p)).get("sm_max_mhz", 2070.0))
    return 2070.0


def fp32_peak_tflops(sms: int, mhz: float) -> float:
    return sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12


def alu_roofline(n_elements: int, ms: float) -> dict:
    """The ALU side of the stencil's roofline: algorithmic FP32 flops per launch
    over the launch time, against the FP32 peak of the unit counts."""
    sms, mhz = device_sm_count(), sm_max_mhz()
    peak = fp32_peak_tflops(sms, mhz)
    tf = STENCIL_FLOPS_PER_ELEMENT * n_elements / (ms * 1e-3) / 1e12
    return {"bound": "alu", "flops_per_launch": STENCIL_FLOPS_PER_ELEMENT * n_elements,
            "achieved": round(tf, 2), "peak": round(peak, 1), "unit": "TFLOP/s",
            "frac": round(tf / peak, 4), "sm_count": sms, "sm_count_source": _SM_COUNT["source"],
            "peak_source": f"derived: {sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 flops x {mhz:g} MHz"}


# The FP32 stencil variants the autotuner chooses from (afd_stencil_async).
STENCIL_NAMES = {0: "stencil2_kernel<TY,{mode},register prefetch>", 1: "stencil2_kernel<TY,{mode},cp.async ring>",
                 2: "st3_kernel<TY,{mode}> (packed bands)"}
STENCIL_DRAM_BYTES = {
    (128, 64, 64, 8, 4, 0): 9197824, (128, 64, 64, 8, 4, 1): 9204992, (128, 64, 64, 8, 4, 2): 8667392,
    (128, 64, 64, 8, 6, 0): 9197568, (128, 64, 64, 8, 6, 1): 9205248, (128, 64, 64, 8, 6, 2): 8667392,
    (128, 64, 64, 8, 8, 0): 9197568, (128, 64, 64, 8, 8, 1): 9205248, (128, 64, 64, 8, 8, 2): 8667648,
    (128, 64, 64, 8, 12, 0): 9199104, (128, 64, 64, 8, 12, 1): 9205504, (128, 64, 64, 8, 12, 2): 8667648,
    (384, 192, 192, 8, 12, 1): 378244608, (384, 192, 192, 8, 12, 2): 363241984}
# The same for the stencil of the inner DPCG iteration (ST_APPLY_DOT), captured inside a mixed solve of the
# 128x64x64 workload in every shape of 8 warps the autotuner may pick (the reads of p_old, z, E and the mask;
# the writes of p and q stay in L2 until after the launch).
STENCIL_DOT_DRAM_BYTES = {
    (128, 64, 64, 8, 4, 0): 15789568, (128, 64, 64, 8, 4, 1): 15791616, (128, 64, 64, 8, 4, 2): 15809280,
    (128, 64, 64, 8, 6, 0): 15789312, (128, 64, 64, 8, 6, 1): 15792640, (128, 64, 64, 8, 6, 2): 15806464,
    (128, 64, 64, 8, 8, 0): 15789824, (128, 64, 64, 8, 8, 1): 15793152, (128, 64, 64, 8, 8, 2): 15812096,
    (128, 64, 64, 8, 12, 0): 15789056, (128, 64, 64, 8, 12, 1): 15791616, (128, 64, 64, 8, 12, 2): 15804672}


def rank_info():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms.  Samples
    are time-stamped as they arrive; only those between begin() and stop()
    (plus the first one after) describe the timed region."""

    FIELDS = "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active," \
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown," \
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.t_begin = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
            t0 = time.monotonic()   # wait for the first sample, so the timed region is covered
            while not self.lines and time.monotonic() - t0 < 3.0 and self.proc.poll() is None:
                time.sleep(0.01)
        except Exception:
            self.proc = None

    def begin(self):
        self.t_begin = time.monotonic()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        t_end = time.monotonic()
        time.sleep(0.1)   # the sample that covers the end of the region
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        tb = self.t_begin if self.t_begin is not None else 0.0
        inside = [ln for t, ln in self.lines if tb <= t <= t_end]
        after = [ln for t, ln in self.lines if t > t_end][:1]
        for ln in inside + after:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def run_ours(args):
    import torch

    import paper_2203_15115_gb300 as afd
    from synthetic import cantilever_128x64x64_voids

    rank, world, local = rank_info()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    afd.lib()
    w = cantilever_128x64x64_voids()
    dev = torch.device("cuda", local)
    E_d = torch.from_numpy(w.E).to(dev)
    f_d = torch.from_numpy(w.f).to(dev)
    m_d = torch.from_numpy(w.fixed).to(dev)
    s_d = torch.empty((1, w.nx * w.ny * w.nz), dtype=torch.float32, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    mesh = afd.Mesh(w.nx, w.ny, w.nz, precision=afd.AFD_MIXED, group=w.group)
    mesh.set_loads_bcs(f_d, m_d)
    last = {}

    def step():
        mesh.set_element_moduli(E_d)
        st = mesh.solve(w.tol)
        J = mesh.compliance()
        mesh.sensitivity(afd.AFD_SENS_STRAIN_ENERGY, s_d)
        tau = mesh.levelset_update(afd.AFD_SENS_STRAIN_ENERGY, [1.0], VOLUME_FRACTION)
        last.update(stats=st[0], J=float(J[0]), tau=tau)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    times = []
    l0 = afd.afd_kernel_launches(mesh.h)
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.begin()
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        s0.record()
        step()
        s1.record()
        torch.cuda.synchronize()
        times.append(s0.elapsed_time(s1))
    torch.cuda.synchronize()
    launches = (afd.afd_kernel_launches(mesh.h) - l0) // max(1, args.steps)
    clk = clocks.stop()
    ms = max_over_ranks(float(np.mean(times)), world, dev)
    value = whole_job_ms_per_step(ms, world)

    # stencil roofline: FP32 matvec on the solver's stream, same launch geometry
    u32 = torch.randn((1, mesh.ndof), dtype=torch.float32, device=dev)
    y32 = torch.empty_like(u32)
    afd.afd_time_stiffness(mesh.h, afd.AFD_F32, 1, u32, y32, 20)
    mv_ms = afd.afd_time_stiffness(mesh.h, afd.AFD_F32, 1, u32, y32, 200)
    u64 = torch.randn((1, mesh.ndof), dtype=torch.float64, device=dev)
    y64 = torch.empty_like(u64)
    afd.afd_time_stiffness(mesh.h, afd.AFD_F64, 1, u64, y64, 5)
    mv64_ms = afd.afd_time_stiffness(mesh.h, afd.AFD_F64, 1, u64, y64, 20)
    nn = (w.nx + 1) * (w.ny + 1) * (w.nz + 1)
    ne = w.nx * w.ny * w.nz
    bytes32 = 2 * 3 * nn * 4 + 4 * ne + nn          # read u, write y, read E, read fixed bits
    peak, peak_kind = measured_peaks()
    achieved = bytes32 / (mv_ms * 1e-3) / 1e9
    shape = (afd.afd_stencil_warps(mesh.h), afd.afd_stencil_depth(mesh.h), afd.afd_stencil_async(mesh.h))
    traffic = STENCIL_DRAM_BYTES.get((w.nx, w.ny, w.nz) + shape)
    # the step's dominant kernel: the FP32 stencil of the inner DPCG iteration (beta and the stopping test from
    # the partials, p = z + W mu + beta p formed on load, q = K p, p.q), each launch bracketed by CUDA events on
    # the mesh's stream, over 200 iterations continuing a solve of the step's design
    mesh.set_element_moduli(E_d)
    mesh.solve(w.tol)
    kt = afd.afd_time_dpcg_kernels(mesh.h, 200)
    it_ms = kt["stencil_us"] * 1e-3
    bytes_dot = 4 * 3 * nn * 4 + 4 * ne + nn        # read p_old, z, E, fixed bits; write p, q
    achieved_dot = bytes_dot / (it_ms * 1e-3) / 1e9
    traffic_dot = STENCIL_DOT_DRAM_BYTES.get((w.nx, w.ny, w.nz) + shape)

    # HBM roofline on the largest mesh of the method (384x192x192, 43 M DOFs): the
    # same FP32 apply, 400 MB of algorithmic traffic per launch, well above L2
    roofline_large = large_mesh_roofline(afd, torch, dev, peak, peak_kind)

    # pure FP64 path on the same workload (the comparison the metric names)
    m64 = afd.Mesh(w.nx, w.ny, w.nz, precision=afd.AFD_FP64, group=w.group)
    m64.set_loads_bcs(f_d, m_d)
    m64.set_element_moduli(E_d)
    m64.solve(w.tol)
    torch.cuda.synchronize()
    fp64 = []
    for _ in range(2):
        m64.set_element_moduli(E_d)
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st64 = m64.solve(w.tol)
        fp64.append((time.perf_counter() - t0) * 1e3)
    m64.close()

    # the same mixed solve with the inner iterations as one persistent cooperative kernel (option), timed
    # like the default CUDA-graph path below
    mp = afd.Mesh(w.nx, w.ny, w.nz, precision=afd.AFD_MIXED, group=w.group, persistent=1)
    mp.set_loads_bcs(f_d, m_d)
    mp.set_element_moduli(E_d)
    mp.solve(w.tol)
    pers = []
    for _ in range(3):
        mp.set_element_moduli(E_d)
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        stp = mp.solve(w.tol)
        pers.append((time.perf_counter() - t0) * 1e3)
    mp.close()

    # mixed solve alone (coarse setup included), for the comparison
    solve_ms = []
    for _ in range(3):
        mesh.set_element_moduli(E_d)
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        stm = mesh.solve(w.tol)
        solve_ms.append((time.perf_counter() - t0) * 1e3)

    # end to end through the C ABI with host buffers
    E_h, f_h, fix_h = w.E.copy(), w.f.copy(), w.fixed.copy()
    u_h = np.zeros_like(f_h)
    s_h = np.zeros((1, ne), np.float32)
    e2e = []
    for i in range(max(2, args.steps // 2) + 1):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mesh.set_loads_bcs(f_h, fix_h)
        mesh.set_element_moduli(E_h)
        mesh.solve(w.tol, u_out=u_h)
        J_h = mesh.compliance()
        mesh.sensitivity(afd.AFD_SENS_STRAIN_ENERGY, s_h)
        mesh.levelset_update(afd.AFD_SENS_STRAIN_ENERGY, [1.0], VOLUME_FRACTION)
        if i > 0:
            e2e.append((time.perf_counter() - t0) * 1e3)
    h2d = E_h.nbytes + f_h.nbytes + fix_h.nbytes
    d2h = u_h.nbytes + s_h.nbytes + J_h.nbytes

    out = {
        "metric": METRIC,
        "value": round(value, 4),
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms, 4),
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 inner / f64 refinement",
        "data": "synthetic (seeded spherical voids)",
        "config": {"workload": w.name, "elements": ne, "dofs": 3 * nn, "group": mesh.options.group or "auto",
                   "stencil_planes_per_cta": afd.afd_stencil_depth(mesh.h),
                   "stencil_warps_per_cta": afd.afd_stencil_warps(mesh.h),
                   "stencil_async_staging": afd.afd_stencil_async(mesh.h),
                   "inner_solver": "persistent cooperative kernel" if mesh.options.persistent else "CUDA-graph chunks",
                   "tol": w.tol, "volume_fraction": VOLUME_FRACTION, "l2": "flushed (512 MB write) between timed steps",
                   "parallelism": f"replicas x{world}"},
        "solve": {"mixed_ms": round(float(np.median(solve_ms)), 3), "fp64_ms": round(float(np.median(fp64)), 3),
                  "mixed_iters": stm[0]["iters"], "mixed_refine_steps": stm[0]["refine_steps"],
                  "fp64_iters": st64[0]["iters"], "mixed_rel_residual": stm[0]["rel_residual"],
                  "fp64_rel_residual": st64[0]["rel_residual"],
                  "speedup_mixed_vs_fp64": round(float(np.median(fp64)) / float(np.median(solve_ms)), 3),
                  "mixed_persistent_kernel_ms": round(float(np.median(pers)), 3),
                  "mixed_persistent_kernel_iters": stp[0]["iters"]},
        "matvec": {"f32_ms": round(mv_ms, 5), "f32_gdofs": round(3 * nn / (mv_ms * 1e-3) / 1e9, 3),
                   "f64_ms": round(mv64_ms, 5), "f64_gdofs": round(3 * nn / (mv64_ms * 1e-3) / 1e9, 3)},
        "roofline": {"kernel": STENCIL_NAMES[afd.afd_stencil_async(mesh.h)].format(mode="ST_APPLY_DOT") +
                               " (inner DPCG iteration: p formed on load, q = K p, p.q; FP32, packed float2)",
                     "bound": "hbm",
                     "achieved": round(achieved_dot, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved_dot / peak, 4), "traffic": traffic_dot,
                     "peak_source": peak_kind, "bytes_per_launch": bytes_dot,
                     "launch_us": round(kt["stencil_us"], 3),
                     "alu": alu_roofline(ne, it_ms),
                     "other_iteration_kernels_us": {k: round(kt[k], 3) for k in
                                                    ("update_us", "coarse_rhs_us", "coarse_step_us")}},
        "roofline_apply": {"kernel": STENCIL_NAMES[afd.afd_stencil_async(mesh.h)].format(mode="ST_APPLY") +
                                     " (K u alone, FP32, packed float2)", "bound": "hbm",
                           "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                           "frac": round(achieved / peak, 4), "traffic": traffic,
                           "peak_source": peak_kind, "bytes_per_launch": bytes32,
                           "alu": alu_roofline(ne, mv_ms)},
        "roofline_384x192x192": roofline_large,
        "e2e": {"value": round(float(np.median(e2e)), 3), "unit": UNIT, "buffers": "host (numpy)",
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches),
        "clocks": clk,
        "last_step": {k: v for k, v in last.items() if k != "stats"},
    }
    if world == 1 and args.batched:
        out["next_rows"] = next_rows_leg(afd, torch, dev, mesh, w, peak, peak_kind)
    mesh.close()
    if world == 1 and args.batched:
        out["batched"] = batched_leg(afd, torch, dev, flush)
    if world == 1 and args.levelset:
        out["levelset"] = levelset_leg(afd, torch, dev)
        out["constrained"] = constrained_leg(afd, torch, dev)
    if world == 1 and args.serve:
        del flush
        torch.cuda.empty_cache()
        out["serve"] = serve_leg(afd)
    if rank == 0 and world == 1 and args.cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(w)
    if world > 1:
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


def large_mesh_roofline(afd, torch, dev, peak, peak_kind, n=384):
    """FP32 stiffness apply on an n x n/2 x n/2 all-solid mesh (the 20-iteration
    level-set workload's size), timed with CUDA events on the mesh's stream
    over 50 launches per CTA shape after warm-up; the best shape is reported."""
    nx, ny, nz = n, n // 2, n // 2
    mesh = afd.Mesh(nx, ny, nz)
    mesh.set_element_moduli(torch.ones(nx * ny * nz, dtype=torch.float64, device=dev))
    u = torch.randn((1, mesh.ndof), dtype=torch.float32, device=dev)
    y = torch.empty_like(u)
    best = None
    for staging in (0, 1, 2):
        for warps, planes in ((8, 4), (8, 6), (8, 8), (8, 12), (16, 8), (16, 16)):
            afd.afd_set_stencil_shape(mesh.h, warps, planes, staging)
            afd.afd_time_stiffness(mesh.h, afd.AFD_F32, 1, u, y, 5)
            ms = afd.afd_time_stiffness(mesh.h, afd.AFD_F32, 1, u, y, 50)
            if best is None or ms < best[0]:
                best = (ms, warps, planes, staging)
    mesh.close()
    del u, y
    nn = (nx + 1) * (ny + 1) * (nz + 1)
    b = 2 * 3 * nn * 4 + 4 * nx * ny * nz + nn
    ach = b / (best[0] * 1e-3) / 1e9
    return {"kernel": STENCIL_NAMES[best[3]].format(mode="ST_APPLY") + " (K u, FP32)", "bound": "hbm",
            "achieved": round(ach, 1),
            "peak": peak, "unit": "GB/s", "frac": round(ach / peak, 4), "frac_of_nominal_8TBs": round(ach / 8000.0, 4),
            "peak_source": peak_kind, "bytes_per_launch": b, "ms_per_launch": round(best[0], 5),
            "gdofs": round(3 * nn / (best[0] * 1e-3) / 1e9, 2), "warps": best[1], "planes": best[2],
            "async_staging": best[3], "traffic": STENCIL_DRAM_BYTES.get((nx, ny, nz) + best[1:]),
            "alu": alu_roofline(nx * ny * nz, best[0])}


def max_over_ranks(x: float, world: int, device=None) -> float:
    """The largest value over all ranks: a job's step time is its slowest
    rank's.  Works on any process group (NCCL with a device, gloo on CPU)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_ms_per_step(ms_max: float, world: int) -> float:
    """Replicas: every rank completes one step per ms_max, so the whole job
    completes `world` steps in that time."""
    return ms_max / max(world, 1)


def percentile(xs, q):
    return float(np.percentile(np.asarray(xs, dtype=np.float64), q)) if len(xs) else None


def serve_leg(afd, n_requests: int = 256, slots: int = 8, budget: float = 60e9, tol: float = 1e-6):
    """The serving stream (meshes nx x nx/2 x nx/2, nx in {32,...,160}, 10-40 %
    seeded voids, cantilever loads) through the library's serving loop under a
    60 GB device budget.  A burst (all requests at t = 0) gives the saturated
    solves/s; the stream's Poisson arrivals, rescaled to 0.8 x that rate, give
    the latency percentiles.  Latency = submit to completion, measured by the
    server.  Inputs are generated before the timed region."""
    from synthetic import serving_request_inputs, serving_stream

    reqs = serving_stream(n_requests, rate_per_s=50.0)
    inputs = [serving_request_inputs(r) for r in reqs]

    def make_server(n_slots):
        srv = afd.Server(max_slots=n_slots, budget_bytes=budget)
        first = {}
        for r, x in zip(reqs, inputs):
            first.setdefault(r["nx"], (r, x))
        warm = [srv.submit(r["nx"], r["ny"], r["nz"], x[0], x[1], x[2], tol) for r, x in first.values()]
        for rid in warm:
            srv.wait(rid, want_u=False)
        return srv

    def run(srv, scale):
        t0 = time.perf_counter()
        ids = []
        for r, (E, f, fx) in zip(reqs, inputs):
            if scale is not None:
                dt = t0 + r["arrival_s"] * scale - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
            ids.append(srv.submit(r["nx"], r["ny"], r["nz"], E, f, fx, tol))
        lat, failed, worst, busy = [], 0, 0.0, 0.0
        for rid in ids:
            rc, st, J, l, _ = srv.wait(rid, want_u=False)
            if rc != afd.AFD_OK or not (st["rel_residual"] <= tol):
                failed += 1
            worst = max(worst, st["rel_residual"])
            busy += st["ms"]
            lat.append(l)
        wall = time.perf_counter() - t0
        # each request's solve time is measured in its own slot, from the call's entry to the end of its
        # stream's work; their sum above the wall time means the slots' solves ran at the same time
        return {"requests": len(ids), "wall_s": round(wall, 3), "solves_per_s": round(len(ids) / wall, 2),
                "p50_ms": round(percentile(lat, 50), 2), "p99_ms": round(percentile(lat, 99), 2),
                "failed": failed, "max_rel_residual": worst, "sum_solve_s": round(busy * 1e-3, 3),
                "sum_solve_over_wall": round(busy * 1e-3 / wall, 3)}

    srv = make_server(slots)
    burst = run(srv, None)
    rate = 0.8 * burst["solves_per_s"]
    poisson = run(srv, 50.0 / rate)
    poisson["offered_rate_per_s"] = round(rate, 2)
    srv.close()
    srv1 = make_server(1)
    burst1 = run(srv1, None)
    srv1.close()
    dofs = [3 * (r["nx"] + 1) * (r["ny"] + 1) * (r["nz"] + 1) for r in reqs]
    return {"slots": slots, "budget_gb": budget / 1e9, "tol": tol, "mean_dofs": int(np.mean(dofs)),
            "burst": burst, "poisson_0.8x": poisson, "burst_one_slot": burst1,
            "burst_speedup_vs_one_slot": round(burst["solves_per_s"] / burst1["solves_per_s"], 3)}


def levelset_leg(afd, torch, dev):
    """The 20-step compliance-constrained volume minimisation on the 384x192x192
    mesh (43 M DOFs): solid start, 2 % of the volume removed per step by the
    AL-weighted strain-energy level set, each solve warm-started from the
    previous design's displacement, J <= 1.6 J_0.  Timed end to end on the host
    clock (every library call returns after its stream has finished)."""
    from synthetic import levelset_384x192x192

    w = levelset_384x192x192(group=0)
    m = afd.Mesh(w.nx, w.ny, w.nz, group=0)
    m.set_element_moduli(torch.from_numpy(w.E).to(dev))
    m.set_loads_bcs(torch.from_numpy(w.f).to(dev), torch.from_numpy(w.fixed).to(dev))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist = afd.run_volume_minimisation(m, steps=20, dv=0.02, j_factor=1.6, tol=w.tol)
    total = time.perf_counter() - t0
    group = afd.afd_stencil_warps(m.h), afd.afd_stencil_depth(m.h)
    m.close()
    return {"workload": w.name, "dofs": w.ndof, "steps": 20, "total_s": round(total, 3),
            "solve_ms": [round(h["ms"], 1) for h in hist], "inner_iters": [h["iters"] for h in hist],
            "max_rel_residual": max(h["rel_residual"] for h in hist),
            "J_over_J0_final": round(hist[-1]["J"] / hist[0]["J"], 5), "constraint_J_le": "1.6 J0",
            "volume_fraction_final": round(hist[-1]["volume_fraction"], 4),
            "stencil_warps_planes": list(group)}


def next_rows_leg(afd, torch, dev, mesh, w, peak, peak_kind):
    """The widened rows on GB300: the casting scan (Sec. 3.7) of a 384x192x192
    level-set field, an HBM-bound kernel (4 B read + 4 B written per element),
    timed with CUDA events over 20 calls per axis; and the adjoint p-norm stress
    sensitivity (Eq. 3.3: d sigma_PN/du, the adjoint solve to 1e-6, T_sigma) on
    the benchmark mesh, timed on the host clock; and the modal analysis of the
    benchmark mesh (its 4 lowest modes to a relative residual of 1e-6, lumped
    mass) with the eigenvalue sensitivity of Eq. 3.4, and the linear buckling
    of its solved state (2 load factors to 1e-6) with Eq. 3.5's field, both
    timed on the host clock."""
    nx, ny, nz = 384, 192, 192
    keys = torch.rand(nx * ny * nz, dtype=torch.float32, device=dev)
    cast = {}
    for axis, parting in ((2, 96), (1, 0), (0, 192)):
        afd.afd_casting_scan(keys, nx, ny, nz, axis, parting)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(20):
            afd.afd_casting_scan(keys, nx, ny, nz, axis, parting)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 20
        b = 8 * nx * ny * nz
        cast["xyz"[axis]] = {"ms": round(ms, 4), "GB/s": round(b / (ms * 1e-3) / 1e9, 1),
                             "frac": round(b / (ms * 1e-3) / 1e9 / peak, 4)}
    del keys
    out = torch.empty((1, w.nx * w.ny * w.nz), dtype=torch.float32, device=dev)
    mesh.solve(w.tol)
    mesh.stress_sensitivity(8.0, w.tol, out)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = mesh.stress_sensitivity(8.0, w.tol, out)
    torch.cuda.synchronize()
    adj_ms = (time.perf_counter() - t0) * 1e3
    # linear buckling of the solved state (load case 0), 2 factors to 1e-6, with Eq. 3.5's field
    bsens = torch.empty((2, w.nx * w.ny * w.nz), dtype=torch.float32, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    blam, binfo = mesh.buckling(2, tol=1e-6, max_iter=200)
    mesh.buckling_sensitivity(bsens)
    torch.cuda.synchronize()
    buck_ms = (time.perf_counter() - t0) * 1e3
    n_modes = 4
    tsens = torch.empty((n_modes, w.nx * w.ny * w.nz), dtype=torch.float32, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lam, info = mesh.modal(n_modes, rho=1.0, tol=1e-6, max_iter=200)
    mesh.eigen_sensitivity(tsens)
    torch.cuda.synchronize()
    modal_ms = (time.perf_counter() - t0) * 1e3
    return {"casting_scan_384x192x192": {"bytes_per_call": 8 * nx * ny * nz, "peak": peak, "peak_source": peak_kind,
                                         "per_axis": cast},
            "stress_sensitivity_128x64x64": {"p": 8.0, "ms": round(adj_ms, 3), "adjoint_iters": st[0]["iters"],
                                             "adjoint_rel_residual": st[0]["rel_residual"]},
            "modal_128x64x64": {"n_modes": n_modes, "tol": 1e-6, "ms": round(modal_ms, 1),
                                "lobpcg_steps": info["steps"], "inner_iters": info["solve_iters"],
                                "lambda": [float(x) for x in lam]},
            "buckling_128x64x64": {"n_modes": 2, "tol": 1e-6, "ms": round(buck_ms, 1),
                                   "lobpcg_steps": binfo["steps"], "inner_iters": binfo["solve_iters"],
                                   "load_factors": [float(x) for x in blam]}}


def constrained_leg(afd, torch, dev, max_fea: int = 40):
    """The algorithm of Sec. 3.8 on the solid 128x64x64 cantilever: minimise
    the volume with hard constraints J <= 1.5 J_0 and sigma_PN <= 2 sigma_0
    (p = 8), volume steps of 0.05 halved on violation, each analysis a mixed
    solve to 1e-6 warm-started, plus the adjoint stress sensitivity.  Timed on
    the host clock over at most `max_fea` analyses."""
    from synthetic import clamp_face_x0, edge_load

    nx, ny, nz = 128, 64, 64
    m = afd.Mesh(nx, ny, nz, group=16)
    m.set_loads_bcs(edge_load(nx, ny, nz)[None], clamp_face_x0(nx, ny, nz))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = afd.run_constrained_topology(m, np.ones(nx * ny * nz), compliance=1.5, stress=2.0, p=8.0, dv0=0.05,
                                       v_min=0.3, max_fea=max_fea, tol=1e-6)
    total = time.perf_counter() - t0
    m.close()
    h = res["history"]
    return {"workload": "cantilever_128x64x64_solid", "constraints": "J <= 1.5 J0, sigma_PN(p=8) <= 2 sigma0 (hard)",
            "total_s": round(total, 3), "analyses": res["fea"], "stop": res["stop"],
            "final_volume_fraction": round(res["volume_fraction"], 4),
            "final_J_over_J0": round(max(x["J"] for x in h if x["v"] == res["volume_fraction"] and not x["violated"])
                                     / res["reference"]["J"], 5),
            "violations": sum(1 for x in h if x["violated"]), "ms_per_analysis": round(total * 1e3 / res["fea"], 1)}


def batched_leg(afd, torch, dev, flush, reps: int = 3):
    """The 96x48x48 multi-load workload: 8 load cases in one multi-RHS solve
    (coarse set-up, mixed dCG to 1e-6, compliance, von Mises and topological
    compliance fields for all 8) against 8 one-RHS solves and against the
    pure-FP64 batched solve."""
    from synthetic import multiload_96x48x48_voids

    w = multiload_96x48x48_voids()
    ne = w.nx * w.ny * w.nz
    E_d = torch.from_numpy(w.E).to(dev)
    f_d = torch.from_numpy(w.f).to(dev)
    m_d = torch.from_numpy(w.fixed).to(dev)
    s_d = torch.empty((w.n_rhs, ne), dtype=torch.float32, device=dev)

    def timed(fn):
        fn()
        out = []
        for _ in range(reps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = fn()
            torch.cuda.synchronize()
            out.append((time.perf_counter() - t0) * 1e3)
        return float(np.median(out)), r

    res = {}
    for name, prec in (("mixed", afd.AFD_MIXED), ("fp64", afd.AFD_FP64)):
        m = afd.Mesh(w.nx, w.ny, w.nz, precision=prec, group=w.group)
        m.set_loads_bcs(f_d, m_d)

        def step():
            m.set_element_moduli(E_d)
            st = m.solve(w.tol)
            m.compliance()
            m.sensitivity(afd.AFD_SENS_VON_MISES, s_d)
            m.sensitivity(afd.AFD_SENS_TJ, s_d)
            return st

        ms, st = timed(step)
        res[name] = {"ms": round(ms, 3), "max_iters": max(x["iters"] for x in st),
                     "max_rel_residual": max(x["rel_residual"] for x in st)}
        m.close()
    m1 = afd.Mesh(w.nx, w.ny, w.nz, precision=afd.AFD_MIXED, group=w.group)

    def one_by_one():
        for r in range(w.n_rhs):
            m1.set_loads_bcs(f_d[r:r + 1], m_d)
            m1.set_element_moduli(E_d)
            m1.solve(w.tol)
            m1.compliance()
            m1.sensitivity(afd.AFD_SENS_VON_MISES, s_d[r:r + 1])
            m1.sensitivity(afd.AFD_SENS_TJ, s_d[r:r + 1])

    ms1, _ = timed(one_by_one)
    m1.close()
    res["mixed_one_rhs_at_a_time"] = {"ms": round(ms1, 3)}
    res["batched_speedup_vs_one_at_a_time"] = round(ms1 / res["mixed"]["ms"], 3)
    res["mixed_speedup_vs_fp64"] = round(res["fp64"]["ms"] / res["mixed"]["ms"], 3)
    return {"workload": w.name, "n_rhs": w.n_rhs, "elements": ne, **res}


def oracle_step_sample(w, budget_s: float = 8.0):
    """One topology step of the oracle as it stands, on a bounded sample of the
    workload: CSR assembly, the set-up and a bounded number of iterations of
    its plain Jacobi-PCG (``fe.solve_pcg`` at two iteration caps gives the
    set-up and per-iteration cost), compliance, the strain-energy field and
    the level-set selection.  The solve is scaled to a full one by the
    oracle's own iteration count for this workload
    (oracle/reference_iterations.json).  Returns (ms per step or None, note)."""
    from oracle import fe, levelset, sensitivity

    t0 = time.perf_counter()
    K = fe.assemble(w.nx, w.ny, w.nz, w.E)
    t_asm = time.perf_counter() - t0
    f = w.f[0]
    m1 = 4
    t0 = time.perf_counter()
    fe.solve_pcg(K, f, w.fixed, rtol=w.tol, maxiter=m1)
    t1 = time.perf_counter() - t0
    # second cap sized from a rough per-iteration guess so the sample stays within budget_s
    guess = max(t1 / (m1 + 4), 1e-4)
    m2 = m1 + max(8, int(0.8 * budget_s / guess))
    t0 = time.perf_counter()
    u, _ = fe.solve_pcg(K, f, w.fixed, rtol=w.tol, maxiter=m2)
    t2 = time.perf_counter() - t0
    per_it = max(t2 - t1, 1e-9) / (m2 - m1)
    setup = max(t1 - m1 * per_it, 0.0)
    t0 = time.perf_counter()
    fe.compliance(f, u)
    s = sensitivity.strain_energy(w.nx, w.ny, w.nz, w.E, u)
    kept, _ = levelset.select_top(s, levelset.keep_count(VOLUME_FRACTION, s.size))
    levelset.apply_topology(kept, w.e_void)
    t_post = time.perf_counter() - t0
    ref = os.path.join(ROOT, "oracle", "reference_iterations.json")
    n_it = json.load(open(ref)).get(w.name, {}).get("iterations") if os.path.exists(ref) else None
    note = (f"{w.name}: CSR assembly {t_asm:.1f} s, PCG set-up {setup:.1f} s, {m2} Jacobi-PCG iterations "
            f"({per_it * 1e3:.1f} ms each), J + strain energy + selection {t_post:.1f} s")
    if n_it is None:
        return None, note + "; no stored iteration count"
    return (t_asm + setup + per_it * n_it + t_post) * 1e3, (
        note + f"; EXTRAPOLATED: the solve is scaled from the {m2} measured iterations to the {n_it} plain "
        f"Jacobi-PCG iterations the oracle needs to reach {w.tol:g} on this workload (measured once by "
        f"oracle/reference_iterations.py); the GPU path runs deflated PCG (about 230 inner iterations), so the "
        f"ratio is not a like-for-like solver comparison")


# The oracle's sparse products (scipy CSR) and vector updates (numpy) run on one thread.
ORACLE_THREADS = 1


def cpu_baseline(w, budget_s: float = 8.0):
    """The oracle timed on the host cores on a bounded sample (rank 0, N = 1)."""
    v, note = oracle_step_sample(w, budget_s)
    return {"value": None if v is None else round(v, 1), "unit": UNIT, "cores": ORACLE_THREADS,
            "affinity_cores": len(os.sched_getaffinity(0)),
            "kind": "oracle", "extrapolated": "measured set-up + sampled Jacobi-PCG iterations x stored iteration count",
            "sample": note}


def run_reference(args):
    """The reference arm: the CPU oracle as it stands, one bounded sample of the
    workload per step, on rank 0 only."""
    rank, world, _ = rank_info()
    if rank != 0:
        return
    from synthetic import cantilever_128x64x64_voids

    w = cantilever_128x64x64_voids()
    vals, note = [], ""
    # the PCG part of each sample shrinks with the number of steps, so that the
    # run stays within a few minutes (each sample also assembles K, ~5 s)
    budget = max(1.0, min(4.0, 60.0 / max(1, args.warmup + args.steps)))
    for i in range(args.warmup + args.steps):
        v, note = oracle_step_sample(w, budget_s=budget)
        if i >= args.warmup and v is not None:
            vals.append(v)
    v = round(float(np.median(vals)), 1) if vals else None
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": v, "higher_is_better": False,
                      "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded spherical voids)",
                      "config": {"workload": w.name},
                      "cpu_baseline": {"value": v, "unit": UNIT, "cores": ORACLE_THREADS,
                                       "affinity_cores": len(os.sched_getaffinity(0)),
                                       "kind": "oracle", "extrapolated": "measured set-up + sampled Jacobi-PCG "
                                       "iterations x stored iteration count", "sample": note},
                      "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}),
          flush=True)


def launch_summary(path: str):
    """Per-kernel launches, total time and share from an ncu launch list
    (``--metrics gpu__time_duration.sum --csv``) of ``bench.py --steps 1``:
    the launches of the one timed step, i.e. those after the first L2-flush
    fill (torch's fill kernel) up to the next torch kernel."""
    import csv

    rows = []
    with open(path) as fh:
        lines = [ln for ln in fh if ln.startswith('"')]
    for d in csv.DictReader(lines):
        if d.get("Metric Name") != "gpu__time_duration.sum":
            continue
        v = float(d["Metric Value"].replace(",", ""))
        unit = d.get("Metric Unit", "ns")
        scale = {"ns": 1e-3, "usecond": 1.0, "us": 1.0, "msecond": 1e3, "ms": 1e3, "nsecond": 1e-3}.get(unit, 1e-3)
        rows.append((d["Kernel Name"], v * scale))
    torch_k = lambda n: "at::" in n or "elementwise" in n or "FillFunctor" in n
    start = next((i for i, (n, _) in enumerate(rows) if torch_k(n)), -1)
    end = next((i for i in range(start + 1, len(rows)) if torch_k(rows[i][0])), len(rows))
    step = rows[start + 1:end]
    agg = {}
    for n, us in step:
        short = n.split("(")[0].replace("void ", "")
        c, t = agg.get(short, (0, 0.0))
        agg[short] = (c + 1, t + us)
    total = sum(t for _, t in agg.values())
    print(f"launches in the timed step: {len(step)}, total device time {total:.1f} us (serialised)")
    print(f"{'kernel':60s} {'launches':>8s} {'total us':>10s} {'share':>7s}")
    for k, (c, t) in sorted(agg.items(), key=lambda kv: -kv[1][1]):
        print(f"{k[:60]:60s} {c:8d} {t:10.1f} {t / total:7.1%}")


def profile_stencil(n: int, launches: int, warps: int = 0, planes: int = 0, staging: int = 0):
    """Apply K u on an n x n/2 x n/2 all-solid mesh (FP32, one RHS) `launches`
    times, in the CTA shape and plane staging given (0 = the size heuristic,
    register prefetch): a case for ncu captures of the stencil kernel (n >= 320
    is larger than L2)."""
    import torch

    import paper_2203_15115_gb300 as afd

    nx, ny, nz = n, n // 2, n // 2
    mesh = afd.Mesh(nx, ny, nz, stencil_warps=warps, stencil_planes=planes)
    mesh.set_element_moduli(np.ones(nx * ny * nz))
    if warps and planes:
        afd.afd_set_stencil_shape(mesh.h, warps, planes, staging)
    u = torch.randn((1, mesh.ndof), dtype=torch.float32, device="cuda")
    y = torch.empty_like(u)
    ms = afd.afd_time_stiffness(mesh.h, afd.AFD_F32, 1, u, y, launches)
    nn = (nx + 1) * (ny + 1) * (nz + 1)
    b = 2 * 3 * nn * 4 + 4 * nx * ny * nz + nn
    print(json.dumps({"mesh": [nx, ny, nz], "ms": ms, "GB/s": b / (ms * 1e-3) / 1e9, "bytes": b,
                      "warps": afd.afd_stencil_warps(mesh.h), "planes": afd.afd_stencil_depth(mesh.h),
                      "async_staging": afd.afd_stencil_async(mesh.h)}))
    mesh.close()


def profile_residual(launches: int):
    """K u on the 128x64x64 voided cantilever from FP64 data, `launches` times
    in double-float arithmetic (the refinement residual's kernel) and then in
    FP64: a case for ncu captures of the two (Sec. 3.5's FP64 residual)."""
    import torch

    import paper_2203_15115_gb300 as afd
    from synthetic import cantilever_128x64x64_voids

    w = cantilever_128x64x64_voids()
    mesh = afd.Mesh(w.nx, w.ny, w.nz, group=w.group)
    mesh.set_element_moduli(w.E)
    g = torch.Generator(device="cuda")
    g.manual_seed(3)
    u = torch.randn((1, mesh.ndof), dtype=torch.float64, device="cuda", generator=g)
    y = torch.empty_like(u)
    out = {"workload": w.name}
    for name, arith in (("f64_df", afd.AFD_F64_DF), ("f64", afd.AFD_F64)):
        out[name + "_us"] = round(afd.afd_time_stiffness(mesh.h, arith, 1, u, y, launches) * 1e3, 1)
    print(json.dumps(out))
    mesh.close()


def profile_solve(warps: int, planes: int, solves: int, staging: int = 0):
    """`solves` mixed solves of the 128x64x64 voided cantilever with the FP32
    stencil in a pinned CTA shape (no autotuning): the solver's kernels in
    their solve-time configuration, for ncu captures."""
    import torch

    import paper_2203_15115_gb300 as afd
    from synthetic import cantilever_128x64x64_voids

    w = cantilever_128x64x64_voids()
    mesh = afd.Mesh(w.nx, w.ny, w.nz, group=w.group, stencil_warps=warps or 8, stencil_planes=planes or 6)
    mesh.set_loads_bcs(w.f, w.fixed)
    afd.afd_set_stencil_shape(mesh.h, warps or 8, planes or 6, staging)
    for _ in range(solves):
        mesh.set_element_moduli(w.E)
        st = mesh.solve(w.tol)
    torch.cuda.synchronize()
    print(json.dumps({"workload": w.name, "iters": st[0]["iters"], "rel_residual": st[0]["rel_residual"],
                      "warps": afd.afd_stencil_warps(mesh.h), "planes": afd.afd_stencil_depth(mesh.h)}))
    mesh.close()


def profile_eigen(kind: str, calls: int):
    """`calls` eigen analyses of the 128x64x64 voided cantilever after one
    mixed solve (modal: 4 modes; buckling: 2 factors of the solved state; both
    to 1e-6), for ncu launch lists of the LOBPCG steps."""
    import torch

    import paper_2203_15115_gb300 as afd
    from synthetic import cantilever_128x64x64_voids

    w = cantilever_128x64x64_voids()
    mesh = afd.Mesh(w.nx, w.ny, w.nz, group=w.group)
    mesh.set_loads_bcs(w.f, w.fixed)
    mesh.set_element_moduli(w.E)
    out = []
    for _ in range(calls):
        mesh.solve(w.tol)
        t0 = time.perf_counter()
        lam, info = mesh.modal(4, tol=1e-6, max_iter=200) if kind == "modal" else mesh.buckling(2, tol=1e-6, max_iter=200)
        torch.cuda.synchronize()
        out.append({"ms": round((time.perf_counter() - t0) * 1e3, 1), "steps": info["steps"],
                    "inner_iters": info["solve_iters"], "values": [float(x) for x in lam]})
    print(json.dumps({"workload": w.name, "analysis": kind, "calls": out}))
    mesh.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-serve", dest="serve", action="store_false", help="skip the serving-stream leg")
    ap.add_argument("--no-batched", dest="batched", action="store_false", help="skip the 8-load-case leg")
    ap.add_argument("--no-levelset", dest="levelset", action="store_false",
                    help="skip the 20-step level-set leg on 384x192x192")
    ap.add_argument("--profile-stencil", type=int, default=0, metavar="NX",
                    help="only time the FP32 stencil on an NX x NX/2 x NX/2 mesh (for ncu)")
    ap.add_argument("--launch-summary", metavar="CSV", help="summarise an ncu launch list of one timed step")
    ap.add_argument("--profile-residual", action="store_true",
                    help="time (and let ncu capture) the double-float and FP64 K u of the refinement residual")
    ap.add_argument("--profile-solve", action="store_true",
                    help="only run --steps mixed solves of the 128x64x64 workload in a pinned stencil shape (for ncu)")
    ap.add_argument("--profile-eigen", choices=("modal", "buckling"),
                    help="only run --steps eigen analyses of the 128x64x64 workload (for ncu)")
    ap.add_argument("--stencil-warps", type=int, default=0, help="pinned FP32 stencil warps per CTA (profile modes)")
    ap.add_argument("--stencil-planes", type=int, default=0, help="pinned FP32 stencil planes per CTA (profile modes)")
    ap.add_argument("--stencil-async", type=int, default=0, choices=(0, 1, 2),
                    help="pinned FP32 stencil variant: 0 register prefetch, 1 cp.async ring, 2 packed bands "
                         "(profile modes)")
    args = ap.parse_args()
    if args.launch_summary:
        launch_summary(args.launch_summary)
    elif args.profile_stencil:
        profile_stencil(args.profile_stencil, max(1, args.steps), args.stencil_warps, args.stencil_planes, args.stencil_async)
    elif args.profile_residual:
        profile_residual(max(1, args.steps))
    elif args.profile_solve:
        profile_solve(args.stencil_warps, args.stencil_planes, max(1, args.steps), args.stencil_async)
    elif args.profile_eigen:
        profile_eigen(args.profile_eigen, max(1, args.steps))
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
