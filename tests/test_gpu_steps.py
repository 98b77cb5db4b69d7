"""Multi-step runs against the oracle: the 2D droplet workload (uniform
quadtree level 5, 5,445 DoF) for its 10 Crank-Nicolson steps, on the plain
FP64 path and the FP32-bulk mixed path, each GPU trajectory compared after
every step with the oracle's own trajectory (sparse direct Newton to 1e-14).

At the workload's Newton tolerance (1e-10): the GPU state is a root of the
oracle's residual to that tolerance, every field lies within the first-order
bound 2 ||J^-1|| (||F(U_gpu)|| + ||F(U_ref)||) of the oracle's state
(||J^-1|| by power iteration on the oracle's sparse Jacobian; a residual of
1e-10 moves the solution by up to that much), and phi is conserved.  Solved
to 1e-14: v, phi and mu match the oracle to 1e-9 (relative, per field) and
the pressure lies within the same first-order bound.
"""
import numpy as np
import pytest

from paper_1912_12453_gb300 import workloads as W
from tests.harness import Pair

pytestmark = pytest.mark.gpu


def _inv_norm(J, seed=0, its=25):
    import scipy.sparse.linalg as spla
    lu = spla.splu(J.tocsc())
    x = np.random.default_rng(seed).standard_normal(J.shape[0])
    for _ in range(its):
        x = lu.solve(lu.solve(x), trans="T")
        x /= np.linalg.norm(x)
    return float(np.linalg.norm(lu.solve(x)))


@pytest.fixture(scope="module")
def trajectory():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1912_12453_gb300 import build
    build.build()
    wl = W.workload("droplet2d_l5")
    p = Pair(wl.leaves)
    U0 = p.om.init_mu(wl.params, W.initial_state(p.om.coords, wl))
    ref = [U0]
    for _ in range(wl.steps):
        U, _ = p.om.step(wl.params, ref[-1], rtol=1e-14, atol=1e-16)
        ref.append(U)
    return wl, p, ref


@pytest.mark.parametrize("rtol", [1e-10, 1e-14])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_ten_steps_match_oracle(trajectory, precision, rtol):
    import torch
    wl, p, ref = trajectory
    prm = wl.params
    assert wl.steps == 10 and wl.newton_rtol == 1e-10
    opts = p.chns.SolverOpts.make(precision=precision, newton_rtol=rtol, newton_atol=1e-16,
                                  krylov_rtol=1e-6, newton_max_it=30)
    cur = p.to_gpu(ref[0])
    nxt = torch.empty_like(cur)
    prev_o = ref[0]
    dim, nf = p.om.dim, p.nf
    for k in range(1, wl.steps + 1):
        st = p.chns.step(p.gm, prm, cur, nxt, opts)
        got = p.to_oracle(nxt)
        # converged to the requested tolerance, measured by the oracle
        F0 = np.linalg.norm(p.om.residual(prm, prev_o, prev_o))
        Fg = np.linalg.norm(p.om.residual(prm, got, prev_o))
        assert Fg <= max(1.05 * rtol * F0, 1e-15), (k, Fg / F0)
        # against the oracle's trajectory
        d = (got - ref[k]).reshape(-1, nf)
        r = ref[k].reshape(-1, nf)
        if rtol <= 1e-14:
            for f in list(range(dim)) + [dim + 1, dim + 2]:
                assert np.linalg.norm(d[:, f]) <= 1e-9 * np.linalg.norm(r[:, f]), (k, f)
        # ||F(U_gpu; U_ref^{k-1})||: the GPU state's residual against the
        # oracle's previous state (the trajectories may differ by that much)
        Fgr = np.linalg.norm(p.om.residual(prm, got, ref[k - 1]))
        Fr = np.linalg.norm(p.om.residual(prm, ref[k], ref[k - 1]))
        bound = 2.0 * _inv_norm(p.om.jacobian(prm, ref[k], ref[k - 1])) * (Fgr + Fr)
        assert np.linalg.norm(d) <= bound + 1e-9 * np.linalg.norm(r), k
        assert abs(st["mass_new"] - st["mass_old"]) < 1e-12
        prev_o = got
        cur, nxt = nxt, cur
