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

    python bench.py [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank solves its own replica (independent
problems, no collective on the data path): weak scaling.
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


def rank_info():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active," \
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown," \
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
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
    ms = float(np.mean(times))
    if world > 1:
        t = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())

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
        "value": round(ms, 4),
        "unit": "ms per topology step (mixed dCG solve to rel-res 1e-6 + coarse setup + J + sensitivity + level-set)",
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
                   "tol": w.tol, "volume_fraction": VOLUME_FRACTION, "l2": "flushed (512 MB write) between timed steps",
                   "parallelism": f"replicas x{world}"},
        "solve": {"mixed_ms": round(float(np.median(solve_ms)), 3), "fp64_ms": round(float(np.median(fp64)), 3),
                  "mixed_iters": stm[0]["iters"], "mixed_refine_steps": stm[0]["refine_steps"],
                  "fp64_iters": st64[0]["iters"], "mixed_rel_residual": stm[0]["rel_residual"],
                  "fp64_rel_residual": st64[0]["rel_residual"],
                  "speedup_mixed_vs_fp64": round(float(np.median(fp64)) / float(np.median(solve_ms)), 3)},
        "matvec": {"f32_ms": round(mv_ms, 5), "f32_gdofs": round(3 * nn / (mv_ms * 1e-3) / 1e9, 3),
                   "f64_ms": round(mv64_ms, 5), "f64_gdofs": round(3 * nn / (mv64_ms * 1e-3) / 1e9, 3)},
        "roofline": {"kernel": "stencil_kernel<float,32,8> (K u, FP32)", "bound": "hbm",
                     "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": None,
                     "peak_source": peak_kind, "bytes_per_launch": bytes32},
        "e2e": {"value": round(float(np.median(e2e)), 3), "unit": "ms per topology step, host buffers",
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches),
        "clocks": clk,
        "last_step": {k: v for k, v in last.items() if k != "stats"},
    }
    if rank == 0 and args.cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(w)
    mesh.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


def cpu_baseline(w, budget_s: float = 15.0):
    """The oracle as it stands on the host cores, on a bounded sample: CSR
    assembly plus as many plain Jacobi-PCG iterations as fit in the budget;
    scaled to a full solve by the oracle's own iteration count for this
    workload (oracle/reference_iterations.json)."""
    from oracle import fe

    cores = len(os.sched_getaffinity(0))
    t0 = time.perf_counter()
    K = fe.assemble(w.nx, w.ny, w.nz, w.E)
    t_asm = time.perf_counter() - t0
    fr = fe.free_dofs(w.fixed)
    A = K[fr][:, fr].tocsr()
    b = w.f[0][fr]
    dinv = 1.0 / A.diagonal()
    x = np.zeros_like(b)
    r = b.copy()
    z = dinv * r
    p = z.copy()
    rz = r @ z
    t1 = time.perf_counter()
    it = 0
    while time.perf_counter() - t1 < budget_s:
        q = A @ p
        a = rz / (p @ q)
        x += a * p
        r -= a * q
        z = dinv * r
        rzn = r @ z
        p = z + (rzn / rz) * p
        rz = rzn
        it += 1
    per_it = (time.perf_counter() - t1) / max(it, 1)
    ref = os.path.join(ROOT, "oracle", "reference_iterations.json")
    n_it = None
    if os.path.exists(ref):
        n_it = json.load(open(ref)).get(w.name, {}).get("iterations")
    if n_it is None:
        return {"value": None, "unit": "ms", "cores": cores, "kind": "oracle",
                "sample": f"assembly {t_asm:.1f} s + {it} PCG iterations at {per_it*1e3:.1f} ms; no stored count"}
    total_ms = (t_asm + per_it * n_it) * 1e3
    return {"value": round(total_ms, 1), "unit": "ms per solve (oracle FP64 Jacobi-PCG to 1e-6)", "cores": cores,
            "kind": "oracle",
            "sample": f"{w.name}: CSR assembly {t_asm:.1f} s + {it} Jacobi-PCG iterations in {budget_s:.0f} s "
                      f"({per_it*1e3:.1f} ms each), scaled to the oracle's {n_it} iterations to 1e-6"}


def run_reference(args):
    """The reference arm: the CPU oracle as it stands, one bounded sample per step."""
    rank, world, _ = rank_info()
    if rank != 0:
        return
    from synthetic import cantilever_128x64x64_voids

    w = cantilever_128x64x64_voids()
    vals = []
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(w, budget_s=10.0)
        if i >= args.warmup:
            vals.append(cb["value"])
    v = float(np.median([x for x in vals if x is not None])) if any(x is not None for x in vals) else None
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": cb["unit"], "n_gpus": world,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": v, "higher_is_better": False,
                      "config": {"workload": w.name}, "cpu_baseline": cb,
                      "e2e": {"value": v, "unit": cb["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}),
          flush=True)


def profile_stencil(n: int, launches: int):
    """Apply K u on an n x n/2 x n/2 all-solid mesh (FP32, one RHS) `launches`
    times: a case larger than L2 for ncu captures of the stencil kernel."""
    import torch

    import paper_2203_15115_gb300 as afd

    nx, ny, nz = n, n // 2, n // 2
    mesh = afd.Mesh(nx, ny, nz)
    mesh.set_element_moduli(np.ones(nx * ny * nz))
    u = torch.randn((1, mesh.ndof), dtype=torch.float32, device="cuda")
    y = torch.empty_like(u)
    ms = afd.afd_time_stiffness(mesh.h, afd.AFD_F32, 1, u, y, launches)
    nn = (nx + 1) * (ny + 1) * (nz + 1)
    b = 2 * 3 * nn * 4 + 4 * nx * ny * nz + nn
    print(json.dumps({"mesh": [nx, ny, nz], "ms": ms, "GB/s": b / (ms * 1e-3) / 1e9, "bytes": b}))
    mesh.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--profile-stencil", type=int, default=0, metavar="NX",
                    help="only time the FP32 stencil on an NX x NX/2 x NX/2 mesh (for ncu)")
    args = ap.parse_args()
    if args.profile_stencil:
        profile_stencil(args.profile_stencil, max(1, args.steps))
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
