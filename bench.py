#!/usr/bin/env python
"""Benchmark of the matrix-free CN-VMS CHNS hot path on one GB300 (or N replicas).

Headline workload: the 3D droplet on a uniform level-6 octree (64^3 trilinear
hexes, 274,625 nodes x 6 unknowns = 1,647,750 DoF), droplet radius 0.15 at
(0.5, 0.5, 0.3), Cn 0.02, Re 100, We 50, Pe 1/Cn, Fr 1, density and viscosity
ratios 1e-2, dt 5e-4, synthetic initial data.

One timed step = one Crank-Nicolson step through the whole hot path: the FP64
residual, the preconditioner (rebuilt once per --precond-steps steps, inside
the timed steps), FGMRES with the FP32 element J.w, FP32 Krylov basis and
Gram-Schmidt (block sums in float, the sum over blocks in double), the FP64
Newton update, and the energy / mass diagnostics.

Reported value: Jacobian-apply throughput (GDoF/s = n_dof / mean J.w time) of
the FP32-bulk applies inside the timed CN steps, from CUDA events the library
records on the launching stream.  Also reported: seconds per CN step for the
FP32-bulk mixed path and the plain FP64 path at the same Newton tolerance
(with per-field differences of the two solutions), an apply sweep over 100
seeded perturbation vectors (L2 flushed between applies), the end-to-end rate
through host buffers, the same step comparison on further workloads
(--extra, default the adaptive 3D bubble), and the oracle timed on the host
cores (single thread and all cores).

--profile-applies N only builds the mesh and runs N operator applies (for a
profiler; no JSON line).
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import platform
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
DESCRIPTION = {
    "droplet2d_l5": "2D droplet, uniform quadtree level 5 (32^2 quads, 1,089 nodes, 5,445 DoF), Cn 0.04, Re 35, "
                    "We 125, ratios 0.1, dt 1e-3",
    "droplet3d_l6": "3D droplet, uniform octree level 6 (64^3 hexes, 274,625 nodes, 1,647,750 DoF), Cn 0.02, "
                    "Re 100, We 50, ratios 1e-2, dt 5e-4",
    "bubble3d_l5_9": "3D rising bubble, adaptive octree levels 5-9 in |phi| < 0.9, 2:1 balanced, hanging nodes, "
                     "Cn 0.01, Re 35, We 1, ratios 1e-3 / 1e-2, dt 2.5e-4",
    "merge3d_l6_10": "3D merging droplets, adaptive octree levels 6-10 in |phi| < 0.9, Cn 0.005, Re 100, We 10, "
                     "ratios 1e-3 / 1e-2, dt 1e-4",
}
# FP32 operations per leaf of one J.w apply of the element kernel, counted by
# ncu on k_element<3, float, J.w> (thread-level FADD + FMUL + 2 x FFMA).  The
# kernel does the same arithmetic for every leaf of every 3D mesh (hanging
# corners only add gather loads), so the count holds for any 3D mesh while the
# kernel is unchanged.
JV_FLOP_PER_LEAF = {3: 10825}
# DRAM bytes (read + write) of one J.w apply, element kernel + node gather,
# from one ncu capture of the named workload; valid for that mesh only.
JV_TRAFFIC_PER_APPLY = {"droplet3d_l6": 45_309_312 + 90_735_360}
# Algorithmic bytes of one FP32 J.w apply per node (read U~, dU and w, write y)
JV_ALG_BYTES_PER_NODE = {3: 4 * (6 + 4 + 6 + 6), 2: 4 * (5 + 3 + 5 + 5)}


def log(*a):
    print("[bench]", *a, file=sys.stderr, flush=True)


def _measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def measure_fma_peaks():
    """FP32 / FP64 FMA-pipe peaks of this GPU, measured now (libchns_peak.so)."""
    from paper_1912_12453_gb300 import build
    L = ctypes.CDLL(build.PEAK_OUT)
    L.chns_peak_fma.restype = ctypes.c_int
    L.chns_peak_fma.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    f32, f64 = ctypes.c_double(), ctypes.c_double()
    if L.chns_peak_fma(ctypes.byref(f32), ctypes.byref(f64)) != 0:
        raise RuntimeError("FMA peak probe failed")
    return f32.value, f64.value


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


# ---------------------------------------------------------------- the oracle on the host

def host_info():
    model = platform.processor() or platform.machine()
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model, "arch": platform.machine()}


def _oracle_inputs(wl):
    from oracle import oracle as O
    om = O.OracleMesh(wl.leaves)
    U0 = W.initial_state(om.coords, wl).reshape(-1)
    w = W.perturbation(om.n_nodes, om.nf, 1)[0].reshape(-1)
    return om, U0 + 1e-2 * w, U0, w


def _time_applies(fn, repeats, warmup):
    for _ in range(warmup):
        fn()
    ts = []
    for _ in range(repeats):
        t0 = time.perf_counter()
        fn()
        ts.append(time.perf_counter() - t0)
    return ts


def cpu_baseline(wl_main, threads):
    """The oracle as it stands, on the host cores: J.w applies of the
    headline mesh on one thread and on all cores (median of 20 after 3
    warm-ups on all cores; 3 after 1 on one thread, the single-thread apply
    taking seconds), J.w applies of the 2D droplet (median of 20 after 3,
    one thread), and one oracle CN step of the 2D droplet (one thread,
    sparse direct Newton to 1e-10)."""
    out = dict(host_info())
    om, U1, U0, w = _oracle_inputs(wl_main)
    ts1 = _time_applies(lambda: om.jacvec(wl_main.params, U1, U0, w), 3, 1)
    tsn = _time_applies(lambda: om.jacvec_threads(wl_main.params, U1, U0, w, threads), 20, 3)
    out["main"] = {"workload": wl_main.name, "n_dof": om.n_dof,
                   "jacvec_1thread_s": float(np.median(ts1)), "jacvec_1thread_GDoFs": om.n_dof / np.median(ts1) / 1e9,
                   "jacvec_allcores_s": float(np.median(tsn)), "jacvec_allcores_GDoFs": om.n_dof / np.median(tsn) / 1e9,
                   "threads": threads, "repeats": {"1thread": 3, "allcores": 20}}
    wl1 = W.workload("droplet2d_l5")
    o1, V1, V0, w1 = _oracle_inputs(wl1)
    t1 = _time_applies(lambda: o1.jacvec(wl1.params, V1, V0, w1), 20, 3)
    r1 = _time_applies(lambda: o1.residual(wl1.params, V1, V0), 20, 3)
    Ui = o1.init_mu(wl1.params, V0)
    t0 = time.perf_counter()
    _, st = o1.step(wl1.params, Ui, rtol=1e-10)
    out["droplet2d_l5"] = {"n_dof": o1.n_dof, "jacvec_1thread_s": float(np.median(t1)),
                           "residual_1thread_s": float(np.median(r1)),
                           "cn_step_1thread_s": time.perf_counter() - t0, "cn_step_newton_its": st["newton_its"]}
    out["main_cn_step"] = ("not run: the oracle's Newton uses a sparse direct factorisation of the full Jacobian, "
                           "which for the 1.65M-DoF 3D mesh exceeds the benchmark's few-minute cap")
    return out, om.n_dof / np.median(tsn) / 1e9


def run_reference(args, rank, world):
    """The oracle as the reference arm: each step is one J.w apply of the
    headline workload on all host cores (the oracle's element loop, elements
    grouped by its own colouring)."""
    if rank != 0:
        return
    wl = W.workload(WORKLOAD)
    threads = os.cpu_count() or 1
    om, U1, U0, w = _oracle_inputs(wl)
    for _ in range(args.warmup):
        om.jacvec_threads(wl.params, U1, U0, w, threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        om.jacvec_threads(wl.params, U1, U0, w, threads)
    T = time.perf_counter() - t0
    value = om.n_dof * args.steps / T / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GDoF/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * T / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": DESCRIPTION[WORKLOAD], "l2": "host"},
        "cpu_baseline": {"kind": "oracle", "value": value, "unit": "GDoF/s", "cores": threads,
                         "sample": f"{args.steps} oracle J.w applies of the full mesh ({om.n_dof} DoF), "
                                   f"{threads} host threads", **host_info()},
        "e2e": {"value": value, "unit": "GDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU side

def field_diffs(a, b, nf, dim):
    """Per-field relative 2-norm differences of two states (v, p, phi, mu)."""
    import torch
    A = a.reshape(-1, nf)
    B = b.reshape(-1, nf)
    names = [f"v{i + 1}" for i in range(dim)] + ["p", "phi", "mu"]
    out = {}
    for k, n in enumerate(names):
        den = float(torch.linalg.vector_norm(B[:, k]))
        out[n] = float(torch.linalg.vector_norm(A[:, k] - B[:, k])) / den if den > 0 else None
    return out


def compare_steps(chns, wl, mesh, U0, steps, opts32, opts64, dev, barrier, legs=("fp32_mixed", "fp64")):
    """FP32-bulk mixed vs plain FP64 CN steps from the same state, both to the
    same Newton tolerance: seconds per step (CUDA events), iteration counts,
    per-field solution differences."""
    import torch
    out = {}
    finals = {}
    for name, opts in (("fp32_mixed", opts32), ("fp64", opts64)):
        if name not in legs:
            continue
        Ua, Ub = U0.clone(), torch.empty_like(U0)
        try:
            chns.step(mesh, wl.params, Ua, Ub, opts)  # warm-up (builds graphs and the preconditioner)
            Ua.copy_(U0)
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            stats = []
            e0.record()
            for _ in range(steps):
                stats.append(chns.step(mesh, wl.params, Ua, Ub, opts))
                Ua, Ub = Ub, Ua
            e1.record()
            barrier()
        except chns.ChnsError as ex:
            out[name] = {"error": str(ex)}
            log(name, wl.name, "failed:", ex)
            continue
        ms = e0.elapsed_time(e1) / steps
        finals[name] = Ua.clone()
        out[name] = {"s_per_step": ms / 1e3, "newton_its": [s["newton_its"] for s in stats],
                     "krylov_its": [s["krylov_its_total"] for s in stats],
                     "res_rel": [s["res_final"] / s["res0"] for s in stats],
                     "jacvec_ms_per_apply": sum(s["jacvec_ms"] for s in stats) / max(1, sum(s["jacvec_calls"] for s in stats)),
                     "precond_ms_per_step": float(np.mean([s["precond_ms"] for s in stats])),
                     "fp64_newton_its": [s["fp64_newton_its"] for s in stats]}
        log(name, wl.name, f"{ms:.1f} ms/step", out[name]["newton_its"], out[name]["krylov_its"])
    if len(finals) == 2:
        out["speedup_fp32_mixed_over_fp64"] = out["fp64"]["s_per_step"] / out["fp32_mixed"]["s_per_step"]
        out["rel_diff_fp32_vs_fp64_per_field"] = field_diffs(finals["fp32_mixed"], finals["fp64"], mesh.nf, mesh.dim)
    out["steps"] = steps
    return out


def remesh_leg(chns, wl, mesh, U, steps, opts32, dev, barrier, shift_cells=4):
    """Remesh around the interface of a state (Sec. 4 "Intergrid transfers":
    marks from the corner test on phi, adaptation passes with 2:1 balance, a
    new mesh, the Q1 transfer of the state), project mu on the new mesh, then
    CN steps there, the first one included (it builds the preconditioner and
    tunes the J.w schedule): the paper's own measurement is the time for 5
    steps including remeshing.  The state is U with phi replaced by the
    profile of the spheres moved by shift_cells finest cells along the last
    axis (a stand-in for several steps of rise, so that the remesh refines and
    coarsens).  Host stages timed by the wall clock, the steps by CUDA events."""
    import torch
    level_min, level_max = int(wl.leaves.level.min()), int(wl.leaves.level.max())
    dim = mesh.dim
    h = shift_cells / float(1 << wl.leaves.max_level)
    moved = [W.Sphere(tuple(c + (h if k == dim - 1 else 0.0) for k, c in enumerate(sp.center)), sp.radius)
             for sp in wl.spheres]
    Um = U.detach().clone().view(-1, mesh.nf)
    Um[:, dim + 1] = torch.from_numpy(W.phi_profile(mesh.coords, moved, wl.params.Cn, wl.bubble)).to(dev)
    barrier()
    t0 = time.perf_counter()
    src = mesh.leaves()
    U_host = Um.to("cpu", torch.float64).numpy()
    t1 = time.perf_counter()
    new_leaves, passes = chns.leaves_remesh(src, mesh.coords_int, U_host, level_min, level_max, 0.9, mesh.nf)
    t2 = time.perf_counter()
    nm = chns.Mesh(new_leaves, mesh.lo, mesh.hi)
    t3 = time.perf_counter()
    Un = torch.from_numpy(chns.leaves_transfer(src, mesh.coords_int, U_host, nm.coords_int, mesh.nf)
                          .reshape(-1)).to(dev)
    barrier()
    t4 = time.perf_counter()
    chns.init_mu(nm, wl.params, Un)
    barrier()
    t5 = time.perf_counter()
    Ub = torch.empty_like(Un)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stats = []
    e0.record()
    for _ in range(steps):
        stats.append(chns.step(nm, wl.params, Un, Ub, opts32))
        Un, Ub = Ub, Un
    e1.record()
    barrier()
    steps_s = e0.elapsed_time(e1) / 1e3
    out = {"level_min": level_min, "level_max": level_max, "phi_band": 0.9, "passes": passes,
           "leaves_before": mesh.n_elem, "leaves_after": nm.n_elem, "n_dof_after": nm.n_dof,
           "host_threads": os.cpu_count(),
           "state": f"phi of the spheres moved by {shift_cells} finest cells along the last axis",
           "seconds": {"download": t1 - t0, "marks_adapt_balance": t2 - t1, "mesh_create": t3 - t2,
                       "transfer_upload": t4 - t3, "remesh_total": t4 - t0, "mu_projection": t5 - t4},
           "steps_after": steps, "steps_after_s": steps_s,
           "newton_its": [s_["newton_its"] for s_ in stats],
           "krylov_its": [s_["krylov_its_total"] for s_ in stats],
           f"{steps}_steps_including_remesh_s": (t5 - t0) + steps_s}
    log(wl.name, "remesh", f"{t4 - t0:.2f} s", f"{passes} passes", f"{mesh.n_elem} -> {nm.n_elem} leaves,",
        f"mu {t5 - t4:.2f} s, {steps} steps {steps_s:.2f} s")
    nm.close()
    return out


def compare_batch_steps(chns, n, steps, opts32, opts64, dev, barrier):
    """The batched workload: n independent droplet / bubble instances of
    uneven size and parameters (2D quadtrees to levels 6-9, 3D octrees to
    levels 5-7) fused into one union mesh per dimension and advanced
    together; FP32-bulk vs FP64 batch steps from the same state."""
    import torch
    wls = W.batched_workloads(n)
    meshes = [chns.Mesh(w.leaves) for w in wls]
    U0 = []
    for m, w in zip(meshes, wls):
        u = torch.from_numpy(W.initial_state(m.coords, w).reshape(-1)).to(dev)
        chns.init_mu(m, w.params, u)
        U0.append(u)
    batch = chns.Batch(meshes, [w.params for w in wls])
    out = {"instances": n, "dims": {"2": sum(1 for w in wls if w.params.dim == 2),
                                    "3": sum(1 for w in wls if w.params.dim == 3)},
           "leaves": int(sum(m.n_elem for m in meshes)), "n_dof": int(sum(m.n_dof for m in meshes)),
           "steps": steps}
    for name, opts in (("fp32_mixed", opts32), ("fp64", opts64)):
        Ua = [u.clone() for u in U0]
        Ub = [torch.empty_like(u) for u in U0]
        try:
            batch.step(Ua, Ub, opts)  # warm-up: graphs, hierarchy, preconditioner
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            stats = []
            e0.record()
            for _ in range(steps):
                stats.append(batch.step(Ua, Ub, opts))
                Ua, Ub = Ub, Ua
            e1.record()
            barrier()
        except chns.ChnsError as ex:
            out[name] = {"error": str(ex)}
            log("batch", name, "failed:", ex)
            continue
        ms = e0.elapsed_time(e1) / steps
        worst = max(st[i]["res_final"] / st[i]["res0"] for st in stats for i in range(n) if st[i]["res0"] > 0)
        # J.w rate: per dimension group (the instances of a group share its counters)
        jv = {}
        for i, w in enumerate(wls):
            d = w.params.dim
            g = jv.setdefault(d, {"dof": 0, "ms": 0.0, "calls": 0})
            g["dof"] += meshes[i].n_dof
        for d, g in jv.items():
            i0 = next(i for i, w in enumerate(wls) if w.params.dim == d)
            g["ms"] = sum(st[i0]["jacvec_ms"] for st in stats)
            g["calls"] = sum(st[i0]["jacvec_calls"] for st in stats)
        out[name] = {"s_per_step": ms / 1e3,
                     "newton_its_per_group": [[st[i]["newton_its"] for st in stats] for i in
                                              sorted({next(j for j, w in enumerate(wls) if w.params.dim == d)
                                                      for d in jv})],
                     "krylov_its_per_group": [[st[i]["krylov_its_total"] for st in stats] for i in
                                              sorted({next(j for j, w in enumerate(wls) if w.params.dim == d)
                                                      for d in jv})],
                     "worst_instance_res_rel": worst,
                     "jacvec_GDoFs": sum(g["dof"] * g["calls"] for g in jv.values()) /
                                     max(1e-9, sum(g["ms"] for g in jv.values()) / 1e3) / 1e9}
        log("batch", name, f"{ms:.1f} ms/step", out[name]["newton_its_per_group"], out[name]["krylov_its_per_group"])
    if "s_per_step" in out.get("fp64", {}) and "s_per_step" in out.get("fp32_mixed", {}):
        out["speedup_fp32_mixed_over_fp64"] = out["fp64"]["s_per_step"] / out["fp32_mixed"]["s_per_step"]
    batch.close()
    for m in meshes:
        m.close()
    return out


def profile_applies(args):
    """Mesh, initial state, then --profile-applies operator applies with an L2
    flush before each: a short command for a profiler to capture."""
    import torch
    from paper_1912_12453_gb300 import build, chns
    build.build()
    wl = W.workload(args.workload)
    mesh = chns.Mesh(wl.leaves)
    if args.profile_schedule >= 0:
        mesh.jacvec_schedule(args.profile_schedule)
    U0 = torch.from_numpy(W.initial_state(mesh.coords, wl).reshape(-1)).cuda()
    U1 = U0 + 1e-2 * torch.from_numpy(W.perturbation(mesh.n_nodes, mesh.nf, 1)[0].reshape(-1)).cuda()
    dt = torch.float32 if args.profile_precision == "fp32" else torch.float64
    w = torch.from_numpy(W.perturbation(mesh.n_nodes, mesh.nf, 2)[1].reshape(-1)).to("cuda", dt)
    y = torch.empty_like(w)
    F = torch.empty_like(U0)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    for r in range(args.profile_applies):
        flush.fill_(float(r))
        chns.jacvec(mesh, wl.params, U1, U0, w, out=y, precision=args.profile_precision)
        if args.profile_residual:
            chns.residual(mesh, wl.params, U1, U0, out=F)
    torch.cuda.synchronize()
    log(f"{args.profile_applies} applies on {mesh.n_elem} elements ({mesh.n_dof} DoF) done")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--apply-vectors", type=int, default=100)
    ap.add_argument("--fp64-steps", type=int, default=None, help="timed FP64 CN steps (default: --steps)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--newton-rtol", type=float, default=1e-9)
    ap.add_argument("--precond-steps", type=int, default=5,
                    help="CN steps one preconditioner build serves (1: rebuilt every step); with the "
                         "defaults one rebuild falls inside the 5 timed steps")
    ap.add_argument("--workload", default=WORKLOAD, help="headline workload (droplet3d_l6)")
    ap.add_argument("--extra", default="bubble3d_l5_9,batched64",
                    help="comma-separated further workloads for the FP32-vs-FP64 step comparison "
                         "(bubble3d_l5_9, merge3d_l6_10, batchedN = N batched instances; empty: none)")
    ap.add_argument("--extra-steps", type=int, default=2)
    ap.add_argument("--extra-legs", default="fp32,fp64", help="precisions timed on the extra workloads")
    ap.add_argument("--remesh-steps", type=int, default=5,
                    help="after the steps of an adaptive extra workload: remesh its state, then this many FP32 "
                         "CN steps on the new mesh (0: no remesh)")
    ap.add_argument("--preconditioner", default="multigrid", choices=["multigrid", "two_level"])
    ap.add_argument("--mg-omega", type=float, default=0.4)
    ap.add_argument("--mg-smooth", type=int, default=1)
    ap.add_argument("--autotune", type=int, default=1, help="1: autotune the FP32 J.w schedule per mesh")
    ap.add_argument("--krylov-max-it", type=int, default=400)
    ap.add_argument("--krylov-restart", type=int, default=64)
    ap.add_argument("--profile-applies", type=int, default=0)
    ap.add_argument("--profile-precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--profile-residual", action="store_true")
    ap.add_argument("--profile-schedule", type=int, default=-1, help="FP32 J.w schedule to profile (-1: default)")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.profile_applies:
        profile_applies(args)
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

    fp32_peak, fp64_peak = measure_fma_peaks()
    log(f"FMA peaks: FP32 {fp32_peak:.2f} TFLOP/s, FP64 {fp64_peak:.3f} TFLOP/s")

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
    jv32_mean, _ = sweep("fp32") if nvec > 0 else (None, None)
    jv64_mean, _ = sweep("fp64", "jacvec") if nvec > 0 else (None, None)
    res64_mean, _ = sweep("fp64", "residual") if nvec > 0 else (None, None)
    log(f"apply sweep: fp32 J.w {jv32_mean} ms, fp64 J.w {jv64_mean} ms, fp64 residual {res64_mean} ms")

    # ---- CN steps, FP32-bulk mixed (timed region)
    pc_kw = dict(preconditioner=args.preconditioner, mg_omega=args.mg_omega, mg_smooth=args.mg_smooth)
    opts32 = chns.SolverOpts.make(precision="fp32", newton_rtol=args.newton_rtol, krylov_rtol=1e-3,
                                  krylov_restart=args.krylov_restart, krylov_max_it=args.krylov_max_it,
                                  reuse_preconditioner=args.precond_steps, autotune=bool(args.autotune), **pc_kw)
    opts64 = chns.SolverOpts.make(precision="fp64", newton_rtol=args.newton_rtol, krylov_rtol=1e-3,
                                  krylov_restart=args.krylov_restart, krylov_max_it=args.krylov_max_it,
                                  reuse_preconditioner=args.precond_steps, **pc_kw)
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
    diff = None
    fp64_error = None
    if k64 > 0:
        try:
            Ua.copy_(U0)
            chns.step(mesh, prm, Ua, Ub, opts64)  # warm-up
            Ua.copy_(U0)
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(k64):
                stats64.append(chns.step(mesh, prm, Ua, Ub, opts64))
                Ua, Ub = Ub, Ua
            e1.record(stream)
            barrier()
            step64_ms = e0.elapsed_time(e1) / k64
            log("fp64 steps", [{k: st[k] for k in ("newton_its", "krylov_its_total", "seconds")} for st in stats64])
            if k64 == args.steps:
                diff = field_diffs(U32, Ua, mesh.nf, mesh.dim)
        except chns.ChnsError as ex:
            fp64_error = str(ex)
            stats64 = []
            log("fp64 steps failed:", ex)

    # ---- end to end through host buffers: H2D of U_n, the step, D2H of U_{n+1}
    host_in = torch.from_numpy(U0h.copy()).pin_memory()
    host_out = torch.empty(n_dof, dtype=torch.float64).pin_memory()
    Ud = torch.empty(n_dof, dtype=torch.float64, device=dev)
    host_in.copy_(U0.cpu())  # mu from the device projection
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
    fpl = JV_FLOP_PER_LEAF.get(mesh.dim)
    if fpl:
        ach = fpl * mesh.n_elem / (jv_apply_ms / 1e3) / 1e12
        traffic = JV_TRAFFIC_PER_APPLY.get(args.workload)
        alg_bytes = JV_ALG_BYTES_PER_NODE[mesh.dim] * mesh.n_nodes
        roof = {"bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s", "frac": ach / fp32_peak,
                "traffic": traffic,
                "per": f"one J.w apply inside the timed CN steps (element kernel over {mesh.n_elem} leaves + node "
                       f"gather), {fpl} FP32 flop per leaf (ncu count of the element kernel)",
                "kernel": "k_element<3,float,J.w> + k_gather_nodes<3,float>",
                "peak_source": "FP32 FMA pipe measured in this run (libchns_peak.so), of measured",
                "algorithmic_bytes_per_apply": alg_bytes,
                "hbm_gbs_algorithmic": alg_bytes / (jv_apply_ms / 1e3) / 1e9,
                "hbm_frac_algorithmic": alg_bytes / (jv_apply_ms / 1e3) / 1e9 / peaks["hbm_gbs"]
                if peaks.get("hbm_gbs") else None}

    # ---- further workloads: FP32-bulk vs FP64 steps at the same tolerance
    extra = {}
    for name in [x for x in args.extra.split(",") if x]:
        if name.startswith("batched"):
            try:
                extra[name] = compare_batch_steps(chns, int(name[len("batched"):] or 64), args.extra_steps,
                                                  opts32, opts64, dev, barrier)
                extra[name]["workload"] = ("batched droplet / bubble instances (2D quadtrees levels 6-9, 3D "
                                           "octrees levels 5-7, radii U[0.1, 0.25], density ratios log-U[1e-3, 1], "
                                           "viscosity ratios log-U[1e-2, 1], Cn 0.02), one union mesh per dimension")
            except Exception as ex:
                extra[name] = {"error": f"{type(ex).__name__}: {ex}"}
                log(name, "failed:", ex)
            torch.cuda.empty_cache()
            continue
        try:
            wx = W.workload(name)
            mx = chns.Mesh(wx.leaves)
            Ux = torch.from_numpy(W.initial_state(mx.coords, wx).reshape(-1)).to(dev)
            chns.init_mu(mx, wx.params, Ux)
            log(f"{name}: {mx.n_elem} leaves, {mx.n_dof} DoF, {mx.n_hanging} hanging nodes")
            legs = tuple({"fp32": "fp32_mixed", "fp64": "fp64"}[x] for x in args.extra_legs.split(","))
            r = compare_steps(chns, wx, mx, Ux, args.extra_steps, opts32, opts64, dev, barrier, legs)
            r.update({"workload": DESCRIPTION.get(name, name), "leaves": mx.n_elem, "n_dof": mx.n_dof,
                      "hanging_nodes": mx.n_hanging, "newton_rtol": args.newton_rtol})
            if args.remesh_steps > 0 and len(set(wx.leaves.level.tolist())) > 1:
                try:
                    r["remesh"] = remesh_leg(chns, wx, mx, Ux, args.remesh_steps, opts32, dev, barrier)
                except Exception as ex:
                    r["remesh"] = {"error": f"{type(ex).__name__}: {ex}"}
                    log(name, "remesh failed:", ex)
            extra[name] = r
            mx.close()
            del Ux
            torch.cuda.empty_cache()
        except Exception as ex:  # report, do not hide: the line says what failed
            extra[name] = {"error": f"{type(ex).__name__}: {ex}"}
            log(name, "failed:", ex)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        log("cpu baseline: oracle applies and a 2D CN step")
        threads = os.cpu_count() or 1
        detail, val_all = cpu_baseline(wl, threads)
        cpu = {"value": val_all, "unit": "GDoF/s", "cores": threads, "kind": "oracle",
               "sample": f"oracle J.w of the full {args.workload} mesh on {threads} host threads, median of 20 "
                         f"after 3 warm-ups; details (single thread, 2D droplet applies and CN step) in 'detail'",
               "detail": detail}

    if rank == 0:
        steps_first = {"newton_its": [s["newton_its"] for s in stats32],
                       "krylov_its": [s["krylov_its_total"] for s in stats32],
                       "res_rel": [s["res_final"] / s["res0"] for s in stats32],
                       "jacvec_ms_per_apply": jv_apply_ms,
                       "residual_ms": sum(s["residual_ms"] for s in stats32) / max(1, sum(s["residual_calls"] for s in stats32)),
                       "precond_ms_per_step": float(np.mean([s["precond_ms"] for s in stats32])),
                       "s_per_step": step32_ms / 1e3}
        basis_mb = (args.krylov_restart + 1) * n_dof * 4 / 1e6
        line = {
            "metric": METRIC, "value": value, "unit": "GDoF/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step32_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": DESCRIPTION[args.workload],
                       "precision": "FP32 element J.w, FP32 Krylov basis and Gram-Schmidt (products and block sums "
                                    "in float, the sum over blocks in double), FP32 preconditioner, inside an FP64 "
                                    "Newton iteration (FP64 residual and update)",
                       "newton_rtol": args.newton_rtol,
                       "krylov": f"FGMRES({args.krylov_restart})",
                       "preconditioner": (f"geometric multigrid V-cycle over the octree levels (coarsest uniform "
                                          f"level 2 solved by a dense inverse), {args.mg_smooth} damped block-Jacobi "
                                          f"sweep(s) omega {args.mg_omega}"
                                          if args.preconditioner == "multigrid" else
                                          "nodal block-Jacobi + Galerkin coarse space (uniform level min(3, coarsest "
                                          "leaf - 1))") +
                                         f"; built once per {args.precond_steps} CN steps "
                                         f"({sum(1 for s_ in stats32 if s_['precond_ms'] > 0)} builds inside the timed steps)",
                       "jacvec_schedule": chns.JACVEC_VARIANTS[stats32[-1]["jacvec_variant"]],
                       "l2": f"inputs larger than L2: the step's Krylov basis is {args.krylov_restart + 1} x "
                             f"{n_dof * 4 / 1e6:.1f} MB = {basis_mb:.0f} MB of floats; the apply sweep flushes L2 "
                             f"(256 MB write) before every apply",
                       "parallelism": f"replicas x{world}"},
            "cn_step": {
                "fp32_mixed": steps_first,
                "fp64": {"error": fp64_error} if fp64_error else None if not stats64 else {
                    "s_per_step": step64_ms / 1e3,
                    "newton_its": [s["newton_its"] for s in stats64],
                    "krylov_its": [s["krylov_its_total"] for s in stats64],
                    "res_rel": [s["res_final"] / s["res0"] for s in stats64],
                    "jacvec_ms_per_apply": sum(s["jacvec_ms"] for s in stats64) / max(1, sum(s["jacvec_calls"] for s in stats64))},
                "speedup_fp32_mixed_over_fp64": (step64_ms / step32_ms) if step64_ms else None,
                "rel_diff_fp32_vs_fp64_per_field": diff,
            },
            "apply_sweep": {"vectors": nvec, "jacvec_fp32_ms": jv32_mean,
                            "jacvec_fp32_GDoFs": n_dof / jv32_mean / 1e6 if jv32_mean else None,
                            "jacvec_fp64_ms": jv64_mean,
                            "jacvec_fp64_GDoFs": (n_dof / jv64_mean / 1e6) if jv64_mean else None,
                            "residual_fp64_ms": res64_mean,
                            "residual_fp64_GDoFs": (n_dof / res64_mean / 1e6) if res64_mean else None},
            "extra_workloads": extra,
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "GDoF/s", "h2d_bytes_per_step": n_dof * 8,
                    "d2h_bytes_per_step": n_dof * 8},
            "gpu_launches": int(launches),
            "clocks": clk.summary(),
            "peaks": {"hbm_gbs": peaks.get("hbm_gbs"), "fp32_fma_tflops_measured_now": fp32_peak,
                      "fp64_fma_tflops_measured_now": fp64_peak},
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
