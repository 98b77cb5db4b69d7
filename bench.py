#!/usr/bin/env python
"""Benchmark of the matrix-free CN-VMS CHNS hot path on one GB300 (or N replicas).

Workload: the 3D droplet on a uniform level-6 octree (64^3 trilinear hexes,
274,625 nodes x 6 unknowns = 1,647,750 DoF), droplet radius 0.15 at
(0.5, 0.5, 0.3), Cn 0.02, Re 100, We 50, Pe 1/Cn, Fr 1, density and viscosity
ratios 1e-2, dt 5e-4, synthetic initial data.

One timed step = one Crank-Nicolson step through the whole hot path: the FP64
residual, the nodal block-Jacobi build, FGMRES with the FP32 element J.w and
FP64 Gram-Schmidt, the FP64 Newton update, and the energy / mass diagnostics.

Reported value: Jacobian-apply throughput (GDoF/s = n_dof / mean J.w time) of
the FP32-bulk applies inside the timed CN steps, from CUDA events the library
records on the launching stream.  Also reported: seconds per CN step for the
FP32-bulk mixed path and the plain FP64 path at the same Newton tolerance, an
apply sweep over 100 seeded perturbation vectors (L2 flushed between applies),
the end-to-end rate through host buffers, and the oracle timed on the host.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1912_12453_gb300 import workloads as W  # noqa: E402

METRIC = "Jacobian-apply GDoF/s and s per CN step, FP32-mixed vs FP64 at equal residual"
WORKLOAD = "droplet3d_l6"
# FP32 operations per element of one 3D J.w apply, counted by ncu on the
# element kernel (thread-level FADD + FMUL + 2 x FFMA: 3.547e8 per 32,768
# elements of the level-6 droplet).
JV_FLOP_PER_ELEM_3D = 10825
# DRAM bytes of one J.w apply (element kernel + node gather) of the level-6
# droplet mesh, read + write, from one ncu capture with --cache-control none
# after an L2 flush.  Valid for the kernels as profiled; null for other meshes.
JV_TRAFFIC_PER_APPLY = {262144: 45_309_312 + 90_735_360}
# FP32 FMA-pipe peak measured on GB300 by paper_1912_12453_gb300/probes/fma_peak.cu
# (independent FMA chains on all SMs); the derived 152 x 128 x 2 x 2.07 GHz is 80.5.
FP32_PEAK_TFLOPS = 78.37
HBM_PEAK_FALLBACK = 6800.0


def log(*a):
    print("[bench]", *a, file=sys.stderr, flush=True)


def _measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi samples during a region (SM clock, limit, throttle reasons)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.idx)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def aggregate_replicas(dof_applies: float, jv_ms: float, t_region: float, world: int, device):
    """Whole-job totals of N independent replicas: the DoF-applies of all
    ranks summed, the J.w time and the timed region's length as the maximum
    over ranks (the slowest replica bounds the job)."""
    if world == 1:
        return dof_applies, jv_ms, t_region
    import torch
    import torch.distributed as dist
    t = torch.tensor([dof_applies, jv_ms, t_region], dtype=torch.float64, device=device)
    tm = t.clone()
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    dist.all_reduce(tm, op=dist.ReduceOp.MAX)
    return float(t[0]), float(tm[1]), float(tm[2])


def _gpu_index(local_rank: int) -> int:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v for v in vis.split(",") if v.strip()]
        try:
            return int(ids[local_rank])
        except (ValueError, IndexError):
            return local_rank
    return local_rank


def cpu_oracle_japply(wl, n_applies: int):
    """The oracle's J.w (single-threaded FP64 C++) on the full mesh."""
    from oracle import oracle as O
    om = O.OracleMesh(wl.leaves)
    U0 = W.initial_state(om.coords, wl).reshape(-1)
    w = W.perturbation(om.n_nodes, om.nf, 1)[0].reshape(-1)
    U1 = U0 + 1e-2 * w
    om.jacvec(wl.params, U1, U0, w)  # warm-up (page-in)
    t0 = time.perf_counter()
    for _ in range(n_applies):
        om.jacvec(wl.params, U1, U0, w)
    dt = (time.perf_counter() - t0) / n_applies
    return om.n_dof, dt


def run_reference(args, rank, world):
    """The oracle as the reference arm: each step is one J.w apply of the full
    workload on one host core (a bounded sample of the J.w applies the GPU
    arm runs)."""
    if rank != 0:
        return
    wl = W.workload(WORKLOAD)
    from oracle import oracle as O
    om = O.OracleMesh(wl.leaves)
    U0 = W.initial_state(om.coords, wl).reshape(-1)
    w = W.perturbation(om.n_nodes, om.nf, 1)[0].reshape(-1)
    U1 = U0 + 1e-2 * w
    for _ in range(args.warmup):
        om.jacvec(wl.params, U1, U0, w)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        om.jacvec(wl.params, U1, U0, w)
    T = time.perf_counter() - t0
    value = om.n_dof * args.steps / T / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GDoF/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * T / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": "3D droplet, uniform octree level 6 (64^3 hexes, "
                                                   "1,647,750 DoF)", "l2": "host"},
        "cpu_baseline": {"kind": "oracle", "value": value, "unit": "GDoF/s", "cores": 1,
                         "sample": f"{args.steps} oracle J.w applies of the full mesh, one host thread"},
        "e2e": {"value": value, "unit": "GDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--apply-vectors", type=int, default=100)
    ap.add_argument("--fp64-steps", type=int, default=None, help="timed FP64 CN steps (default: --steps)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-applies", type=int, default=2)
    ap.add_argument("--newton-rtol", type=float, default=1e-9)
    ap.add_argument("--precond-steps", type=int, default=5,
                    help="CN steps one preconditioner build serves (1: rebuilt every step); with the "
                         "defaults one rebuild falls inside the 5 timed steps")
    ap.add_argument("--workload", default=WORKLOAD,
                    help="droplet3d_l6 (the metric's configuration), droplet2d_l5 or bubble3d_l5_9")
    ap.add_argument("--krylov-max-it", type=int, default=400)
    ap.add_argument("--krylov-restart", type=int, default=64)
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import torch.distributed as dist
    from paper_1912_12453_gb300 import build, chns

    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        dist.barrier()
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    wl = W.workload(args.workload)
    prm = wl.params
    mesh = chns.Mesh(wl.leaves)
    n_dof = mesh.n_dof
    U0h = W.initial_state(mesh.coords, wl).reshape(-1)
    U0 = torch.from_numpy(U0h).to(dev)
    chns.init_mu(mesh, prm, U0)

    # ---- apply sweep: J.w over seeded perturbation vectors, L2 flushed
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2
    nvec = args.apply_vectors
    wv = W.perturbation(mesh.n_nodes, mesh.nf, 1)[0].reshape(-1)
    U1 = U0 + 1e-2 * torch.from_numpy(wv).to(dev)
    rng = np.random.default_rng(W.PERTURB_SEED + 1)

    def sweep(precision, op="jacvec"):
        dt_ = torch.float32 if precision == "fp32" else torch.float64
        y = torch.empty(n_dof, dtype=dt_, device=dev)
        times = []
        for r in range(nvec + 3):
            w = torch.from_numpy(rng.uniform(-1, 1, n_dof)).to(dev, dt_)
            flush.fill_(float(r))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if op == "jacvec":
                chns.jacvec(mesh, prm, U1, U0, w, out=y, precision=precision)
            else:
                chns.residual(mesh, prm, U1, U0, out=y)
            e1.record(stream)
            e1.synchronize()
            if r >= 3:
                times.append(e0.elapsed_time(e1))
        return float(np.mean(times)), float(np.median(times))

    log(f"mesh: {mesh.n_elem} elements, {n_dof} DoF, {mesh.n_colours} colours")
    jv32_mean, jv32_med = sweep("fp32")
    log(f"apply sweep fp32 J.w {jv32_mean:.3f} ms")
    jv64_mean, jv64_med = sweep("fp64", "jacvec") if nvec > 0 else (None, None)
    res64_mean, _ = sweep("fp64", "residual") if nvec > 0 else (None, None)
    log(f"apply sweep fp64 J.w {jv64_mean} ms, residual {res64_mean} ms")

    # ---- CN steps, FP32-bulk mixed (timed region)
    opts32 = chns.SolverOpts.make(precision="fp32", newton_rtol=args.newton_rtol, krylov_rtol=1e-3,
                                  krylov_restart=args.krylov_restart, krylov_max_it=args.krylov_max_it,
                                  reuse_preconditioner=args.precond_steps)
    opts64 = chns.SolverOpts.make(precision="fp64", newton_rtol=args.newton_rtol, krylov_rtol=1e-3,
                                  krylov_restart=args.krylov_restart, krylov_max_it=args.krylov_max_it,
                                  reuse_preconditioner=args.precond_steps)
    Ua = U0.clone()
    Ub = torch.empty_like(Ua)
    for _ in range(args.warmup):
        st = chns.step(mesh, prm, Ua, Ub, opts32)
        log("warm-up fp32 step", {k: st[k] for k in ("newton_its", "krylov_its_total", "seconds")})
        Ua, Ub = Ub, Ua
    Ua.copy_(U0)
    barrier()
    launches0 = chns.kernel_launches()
    stats32 = []
    with ClockSampler(_gpu_index(local_rank)) as clk:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("timed")
        e0.record(stream)
        for _ in range(args.steps):
            stats32.append(chns.step(mesh, prm, Ua, Ub, opts32))
            Ua, Ub = Ub, Ua
        e1.record(stream)
        barrier()
        torch.cuda.nvtx.range_pop()
    step32_ms = e0.elapsed_time(e1) / args.steps
    log("fp32 steps", [{k: st[k] for k in ("newton_its", "krylov_its_total", "seconds")} for st in stats32])
    launches = chns.kernel_launches() - launches0
    U32 = Ua.clone()
    jv_ms = sum(s["jacvec_ms"] for s in stats32)
    jv_calls = sum(s["jacvec_calls"] for s in stats32)
    dof_applies = float(n_dof) * jv_calls
    t_region = step32_ms * args.steps / 1e3
    dof_applies_all, jv_ms_max, t_region = aggregate_replicas(dof_applies, jv_ms, t_region, world, dev)
    value = dof_applies_all / (jv_ms_max / 1e3) / 1e9

    # ---- CN steps, plain FP64 (same tolerance, same start)
    k64 = args.fp64_steps if args.fp64_steps is not None else args.steps
    stats64 = []
    step64_ms = None
    if k64 > 0:
        Ua.copy_(U0)
        chns.step(mesh, prm, Ua, Ub, opts64)  # warm-up
        Ua.copy_(U0)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k64):
            stats64.append(chns.step(mesh, prm, Ua, Ub, opts64))
            log("fp64 step", {k: stats64[-1][k] for k in ("newton_its", "krylov_its_total", "seconds")})
            Ua, Ub = Ub, Ua
        e1.record(stream)
        barrier()
        step64_ms = e0.elapsed_time(e1) / k64
        U64 = Ua.clone()
        diff = float(torch.linalg.vector_norm(U32 - U64) / torch.linalg.vector_norm(U64)) if k64 == args.steps else None
    else:
        diff = None

    # ---- end to end through host buffers: H2D of U_n, the step, D2H of U_{n+1}
    host_in = torch.from_numpy(U0h.copy()).pin_memory()
    host_out = torch.empty(n_dof, dtype=torch.float64).pin_memory()
    Ud = torch.empty(n_dof, dtype=torch.float64, device=dev)
    chns.init_mu(mesh, prm, U0)  # host_in holds mu from the device projection
    host_in.copy_(U0.cpu())
    barrier()
    e_calls = 0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        Ud.copy_(host_in, non_blocking=True)
        st = chns.step(mesh, prm, Ud, Ub, opts32)
        host_out.copy_(Ub, non_blocking=True)
        torch.cuda.current_stream().synchronize()
        host_in.copy_(host_out)
        e_calls += st["jacvec_calls"]
    barrier()
    t_e2e = time.perf_counter() - t0
    e2e_value = float(n_dof) * e_calls / t_e2e / 1e9 * world

    # ---- roofline of the dominant kernel (the FP32 element J.w)
    peaks = _measured_peaks()
    jv_apply_ms = jv_ms / max(jv_calls, 1)
    roof = None
    if JV_FLOP_PER_ELEM_3D:
        ach = JV_FLOP_PER_ELEM_3D * mesh.n_elem / (jv_apply_ms / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": ach / FP32_PEAK_TFLOPS,
                "traffic": JV_TRAFFIC_PER_APPLY.get(mesh.n_elem) if mesh.dim == 3 else None,
                "per": f"one J.w apply (element kernel over {mesh.n_elem} leaves + node gather, "
                       f"{JV_FLOP_PER_ELEM_3D} flop/element)",
                "kernel": "k_element<3,float,J.w> + k_gather_nodes<3,float>",
                "peak_source": "measured FP32 FMA pipe (probes/fma_peak.cu)",
                "hbm_gbs_achieved": (JV_TRAFFIC_PER_APPLY.get(mesh.n_elem, 0) / (jv_apply_ms / 1e3) / 1e9)
                if mesh.dim == 3 else None}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        log("cpu baseline: oracle J.w")
        nd, t_cpu = cpu_oracle_japply(wl, args.cpu_applies)
        cpu = {"value": nd / t_cpu / 1e9, "unit": "GDoF/s", "cores": 1, "kind": "oracle",
               "sample": f"{args.cpu_applies} oracle J.w applies of the full mesh ({nd} DoF), one host thread"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GDoF/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step32_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "3D droplet, uniform octree level 6 (64^3 hexes, 274,625 nodes, "
                                   "1,647,750 DoF), Cn 0.02, Re 100, We 50, ratios 1e-2, dt 5e-4",
                       "precision": "FP32 element J.w + FP32 block-Jacobi inside FP64 Newton / FP64 Gram-Schmidt",
                       "newton_rtol": args.newton_rtol,
                       "krylov": f"FGMRES({args.krylov_restart})",
                       "preconditioner": f"nodal block-Jacobi + Galerkin coarse space (uniform level "
                                         f"min(3, coarsest leaf - 1)), built once per {args.precond_steps} CN steps "
                                         f"({sum(1 for s_ in stats32 if s_['precond_ms'] > 0)} builds inside the timed steps)",
                       "l2": "step working set (Krylov basis 31 x 13 MB) > L2; apply sweep flushes L2",
                       "parallelism": f"replicas x{world}"},
            "cn_step": {
                "fp32_mixed": {"s_per_step": step32_ms / 1e3,
                               "newton_its": [s["newton_its"] for s in stats32],
                               "krylov_its": [s["krylov_its_total"] for s in stats32],
                               "res_rel": [s["res_final"] / s["res0"] for s in stats32],
                               "jacvec_ms_per_apply": jv_apply_ms,
                               "residual_ms": sum(s["residual_ms"] for s in stats32) / max(1, sum(s["residual_calls"] for s in stats32)),
                               "precond_ms_per_step": float(np.mean([s["precond_ms"] for s in stats32]))},
                "fp64": None if not stats64 else {
                    "s_per_step": step64_ms / 1e3,
                    "newton_its": [s["newton_its"] for s in stats64],
                    "krylov_its": [s["krylov_its_total"] for s in stats64],
                    "res_rel": [s["res_final"] / s["res0"] for s in stats64],
                    "jacvec_ms_per_apply": sum(s["jacvec_ms"] for s in stats64) / max(1, sum(s["jacvec_calls"] for s in stats64))},
                "speedup_fp32_mixed_over_fp64": (step64_ms / step32_ms) if step64_ms else None,
                "rel_diff_fp32_vs_fp64_solution": diff,
            },
            "apply_sweep": {"vectors": nvec, "jacvec_fp32_ms": jv32_mean, "jacvec_fp32_GDoFs": n_dof / jv32_mean / 1e6,
                            "jacvec_fp64_ms": jv64_mean,
                            "jacvec_fp64_GDoFs": (n_dof / jv64_mean / 1e6) if jv64_mean else None,
                            "residual_fp64_ms": res64_mean,
                            "residual_fp64_GDoFs": (n_dof / res64_mean / 1e6) if res64_mean else None},
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "GDoF/s", "h2d_bytes_per_step": n_dof * 8,
                    "d2h_bytes_per_step": n_dof * 8},
            "gpu_launches": int(launches),
            "clocks": clk.summary(),
            "peaks": {"hbm_gbs": peaks.get("hbm_gbs"), "fp32_fma_tflops_measured": FP32_PEAK_TFLOPS},
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
