"""Profiling driver: a few operator applies of one workload, nothing else.

Builds the mesh, forms the initial state, then runs ``--applies`` J.w applies
in the chosen precision (and optionally FP64 residuals), with an L2 flush
between applies.  Meant to run under ``ncu`` with few launches, e.g.

  python -m paper_1912_12453_gb300.profile_apply --workload droplet3d_l6 --applies 3
"""
from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="droplet3d_l6")
    ap.add_argument("--applies", type=int, default=3)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--residual", action="store_true", help="also run FP64 residual applies")
    args = ap.parse_args()

    import torch
    from paper_1912_12453_gb300 import build, chns, workloads as W
    build.build()
    wl = W.workload(args.workload)
    mesh = chns.Mesh(wl.leaves)
    U0 = torch.from_numpy(W.initial_state(mesh.coords, wl).reshape(-1)).cuda()
    U1 = U0 + 1e-2 * torch.from_numpy(W.perturbation(mesh.n_nodes, mesh.nf, 1)[0].reshape(-1)).cuda()
    dt = torch.float32 if args.precision == "fp32" else torch.float64
    w = torch.from_numpy(W.perturbation(mesh.n_nodes, mesh.nf, 2)[1].reshape(-1)).to("cuda", dt)
    y = torch.empty_like(w)
    F = torch.empty_like(U0)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    for r in range(args.applies):
        flush.fill_(float(r))
        chns.jacvec(mesh, wl.params, U1, U0, w, out=y, precision=args.precision)
        if args.residual:
            chns.residual(mesh, wl.params, U1, U0, out=F)
    torch.cuda.synchronize()
    print(f"{args.applies} applies on {mesh.n_elem} elements ({mesh.n_dof} DoF) done")


if __name__ == "__main__":
    main()
