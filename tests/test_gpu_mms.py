"""The manufactured-solution study of Sec. 5.1 through the product path.

chns_step advances the 2D manufactured solution (Re = 10, We = 1, Cn = 1,
Pe = 3, Fr = 1, rho-/rho+ = 0.85) with the nodal forcing at t_{k+1/2} and
the exact wall velocities / pinned pressure at t_{k+1}, as in the paper's
spatial study: time step 1e-3 to t = 0.2 on uniform quadtrees of levels
5..8 (h = 1/32 .. 1/256, bracketing the paper's 1/50 .. 1/175).  Errors are
L2 norms of the nodal error in the Q1 mass metric (the consistent mass
matrix of a uniform grid, a Kronecker product of 1D mass matrices).

Pins: the phi rate of the finest pair lies in the band of the paper's Table
tab:spatial_error_table (tests/golden/mms_spatial_table.txt, +-0.25), the
velocity rates of the two finer pairs are at least 1.5 (the table's v rates
run from 1.6 to 2.1; h = 1/32 is pre-asymptotic for v), and every phi rate is
above 1.8.  The ratio of phi's error to the table's (interpolated as C h^2
through its h = 1/100 value) is printed: the absolute values depend on
conventions the paper does not fix (measured: about 1/5).
"""
import math
import os

import numpy as np
import pytest

from paper_1912_12453_gb300 import workloads as W

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden():
    rows = []
    with open(os.path.join(GOLDEN, "mms_spatial_table.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            tok = line.split()
            n, d = tok[0].split("/")
            rows.append((float(n) / float(d), float(tok[5]), None if tok[6] == "-" else float(tok[6])))
    return rows


def _mass_norm(E, coords_int, level):
    """sqrt(e^T M e) for nodal values E (n_nodes,) on a uniform level-`level` grid."""
    n = 1 << level
    h = 1.0 / n
    G = np.zeros((n + 1, n + 1))
    G[coords_int[:, 1], coords_int[:, 0]] = E
    m1 = np.zeros((n + 1, n + 1))
    for e in range(n):
        m1[e:e + 2, e:e + 2] += h / 6 * np.array([[2.0, 1.0], [1.0, 2.0]])
    return math.sqrt(float(np.sum(G * (m1 @ G @ m1.T))))


def test_mms_spatial_rates_through_chns_step():
    pytest.importorskip("sympy")
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1912_12453_gb300 import build, chns
    from tests.mms import mms_functions
    build.build()
    prm = W.Params(2, 1e-3, 1.0, 10.0, 1.0, 3.0, 1.0, 0.85, 0.5)
    exact, forc = mms_functions(2, prm)
    dt, T = 1e-3, 0.2
    nsteps = int(round(T / dt))
    levels = (5, 6, 7, 8)
    errs = []
    for lev in levels:
        mesh = chns.Mesh(W.uniform_leaves(2, lev))
        X = mesh.coords
        U = torch.from_numpy(exact(X, 0.0).reshape(-1).copy()).cuda()
        V = torch.empty_like(U)
        opts = chns.SolverOpts.make(precision="fp32", newton_rtol=1e-10, newton_atol=1e-14, krylov_rtol=1e-3,
                                    newton_max_it=30, reuse_preconditioner=20, preconditioner="multigrid")
        t = 0.0
        for k in range(nsteps):
            f = torch.from_numpy(forc(X, t + dt / 2).reshape(-1).copy()).cuda()
            g = torch.from_numpy(exact(X, t + dt).reshape(-1).copy()).cuda()
            chns.step(mesh, prm, U, V, opts, forcing=f, bc=g)
            U, V = V, U
            t += dt
        E = U.cpu().numpy().reshape(-1, mesh.nf) - exact(X, t)
        ci = mesh.coords_int >> (mesh.max_level - lev)
        errs.append([_mass_norm(E[:, k], ci, lev) for k in range(mesh.nf)])
        mesh.close()
    errs = np.array(errs)
    rates = np.log2(errs[:-1] / errs[1:])
    print("MMS errors (v1, v2, p, phi, mu) per level", levels, "\n", errs, "\nrates\n", rates)
    gold = _golden()
    gr = [r for _, _, r in gold if r is not None]
    assert min(gr) - 0.25 < rates[-1, 3] < max(gr) + 0.25, rates
    # h = 1/32 is pre-asymptotic for v; the two finer pairs are in the table's range
    assert np.all(rates[1:, 0:2] > 1.5), rates
    assert np.all(rates[:, 3] > 1.8), rates
    # absolute phi errors next to the table's, as C h^2 through its h = 1/100
    # entry (reported, not asserted: the paper's absolute values depend on
    # conventions it does not fix)
    h100, e100 = [(h, e) for h, e, _ in gold if abs(h - 0.01) < 1e-12][0]
    print("phi error / table's C h^2:", [float(e / (e100 * ((1.0 / (1 << lev)) / h100) ** 2))
                                        for lev, e in zip(levels, errs[:, 3])])
