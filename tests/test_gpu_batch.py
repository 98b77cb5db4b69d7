"""Batched CN steps (instances fused into union meshes) against the oracle's
steps of each instance and against one-instance GPU steps."""
import numpy as np
import pytest

from paper_1912_12453_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _instances():
    out = []
    specs = [
        (W.band_leaves(2, 3, 6, [W.Sphere((0.45, 0.55), 0.2)], 0.03), 2, 0.1, 0.1, False),
        (W.uniform_leaves(2, 4), 2, 0.5, 0.3, True),
        (W.half_refined_leaves(3, 2), 3, 0.05, 0.2, False),
        (W.band_leaves(3, 2, 4, [W.Sphere((0.5, 0.45, 0.4), 0.25)], 0.04), 3, 0.3, 1.0, True),
        (W.uniform_leaves(2, 3), 2, 1e-2, 1e-1, True),
    ]
    for leaves, dim, rr, er, bubble in specs:
        g = (0.0, -1.0, 0.0) if dim == 2 else (0.0, 0.0, -1.0)
        prm = W.Params(dim, 1e-3, 0.05, 30.0, 20.0, 20.0, 1.0, rr, er, gravity=g)
        wl = W.Workload("b", leaves, prm, [W.Sphere((0.5, 0.45, 0.4)[:dim], 0.22)], bubble)
        out.append(wl)
    return out


_REFS = {}


@pytest.mark.parametrize("preconditioner", ["two_level", "multigrid"])
def test_batch_step_matches_single_steps(preconditioner):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1912_12453_gb300 import build, chns
    build.build()
    from oracle import oracle as O
    wls = _instances()
    meshes = [chns.Mesh(w.leaves) for w in wls]
    # initial states from the oracle (mu by its L2 projection), in GPU order
    oms, maps, U0o, U0 = [], [], [], []
    for m, w in zip(meshes, wls):
        om = O.OracleMesh(w.leaves)
        g_of_o = W.match_nodes(m.coords_int, om.coords_int)
        u0 = om.init_mu(w.params, W.initial_state(om.coords, w)).reshape(-1)
        ug = np.empty((m.n_nodes, m.nf))
        ug[g_of_o] = u0.reshape(-1, m.nf)
        oms.append(om)
        maps.append(g_of_o)
        U0o.append(u0)
        U0.append(torch.from_numpy(ug.reshape(-1)).cuda())
    opts = chns.SolverOpts.make(precision="fp32", newton_rtol=1e-13, newton_atol=1e-16, krylov_rtol=1e-6,
                                newton_max_it=30, preconditioner=preconditioner)
    single = []
    for m, w, u in zip(meshes, wls, U0):
        out = torch.empty_like(u)
        chns.step(m, w.params, u, out, opts)
        single.append(out)
    batch = chns.Batch(meshes, [w.params for w in wls])
    outs = [torch.empty_like(u) for u in U0]
    stats = batch.step(U0, outs, opts)
    for i, (m, w) in enumerate(zip(meshes, wls)):
        # the oracle's Newton root of the instance's own step (sparse direct solves)
        om, g_of_o, u0 = oms[i], maps[i], U0o[i]
        if i not in _REFS:  # the oracle's root does not depend on the preconditioner
            _REFS[i] = om.step(w.params, u0, rtol=1e-14, atol=1e-16)[0]
        ref = _REFS[i]
        got = outs[i].cpu().numpy().reshape(-1, m.nf)[g_of_o]
        F0o = np.linalg.norm(om.residual(w.params, u0, u0))
        assert np.linalg.norm(om.residual(w.params, got.reshape(-1), u0)) <= 1.05e-13 * F0o, i
        dr = got - ref.reshape(-1, m.nf)
        for k in [f for f in range(m.nf) if f != m.dim]:
            assert np.linalg.norm(dr[:, k]) <= 1e-9 * max(np.linalg.norm(ref.reshape(-1, m.nf)[:, k]), 1e-12) + 1e-13, (i, k)
        # a root of the instance's own residual, and the same state as the single step
        F0 = chns.residual(m, w.params, U0[i], U0[i]).norm().item()
        Fb = chns.residual(m, w.params, outs[i], U0[i]).norm().item()
        assert Fb <= 1e-10 * F0, (i, Fb, F0)
        d = (outs[i] - single[i]).reshape(-1, m.nf).cpu().numpy()
        r = single[i].reshape(-1, m.nf).cpu().numpy()
        for k in [f for f in range(m.nf) if f != m.dim]:
            assert np.linalg.norm(d[:, k]) <= 1e-8 * max(np.linalg.norm(r[:, k]), 1e-12) + 1e-13, (i, k)
        e, mass, _ = chns.energy_mass(m, w.params, outs[i])
        assert abs(stats[i]["mass_new"] - mass) <= 1e-13 * max(1.0, abs(mass))
        assert abs(stats[i]["mass_new"] - stats[i]["mass_old"]) < 1e-11
    batch.close()


def test_batch_of_64_instances_converges_and_matches_oracle():
    """The batched workload: 64 independent droplet / bubble instances (35 in
    2D, 29 in 3D, levels up to 9 / 7, density ratios down to 1e-3) advanced
    by one FP32-bulk CN step with the multigrid preconditioner.  Every
    instance must reach its own Newton tolerance, and the three smallest
    instances (2D, a few thousand DoF, within reach of the oracle's direct
    solver) must match the oracle's Newton root."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from oracle import oracle as O
    from paper_1912_12453_gb300 import build, chns
    build.build()
    wls = W.batched_workloads(64)
    meshes = [chns.Mesh(w.leaves) for w in wls]
    sample = sorted(range(len(wls)), key=lambda i: wls[i].leaves.n)[:3]
    U0 = []
    oracle_side = {}
    for i, (m, w) in enumerate(zip(meshes, wls)):
        if i in sample:  # initial state from the oracle for the sampled instances
            om = O.OracleMesh(w.leaves)
            g_of_o = W.match_nodes(m.coords_int, om.coords_int)
            u0 = om.init_mu(w.params, W.initial_state(om.coords, w)).reshape(-1)
            ug = np.empty((m.n_nodes, m.nf))
            ug[g_of_o] = u0.reshape(-1, m.nf)
            oracle_side[i] = (om, g_of_o, u0)
            U0.append(torch.from_numpy(ug.reshape(-1)).cuda())
        else:
            u = torch.from_numpy(W.initial_state(m.coords, w).reshape(-1)).cuda()
            chns.init_mu(m, w.params, u)
            U0.append(u)
    batch = chns.Batch(meshes, [w.params for w in wls])
    outs = [torch.empty_like(u) for u in U0]
    opts = chns.SolverOpts.make(precision="fp32", newton_rtol=1e-12, newton_atol=1e-16, krylov_rtol=1e-6,
                                newton_max_it=40, preconditioner="multigrid")
    stats = batch.step(U0, outs, opts)
    for i, (m, w) in enumerate(zip(meshes, wls)):
        F0 = chns.residual(m, w.params, U0[i], U0[i]).norm().item()
        Fb = chns.residual(m, w.params, outs[i], U0[i]).norm().item()
        assert Fb <= 1.05e-12 * F0, (i, Fb, F0)
        assert abs(stats[i]["mass_new"] - stats[i]["mass_old"]) < 1e-11
    for i in sample:
        om, g_of_o, u0 = oracle_side[i]
        w = wls[i]
        ref, _ = om.step(w.params, u0, rtol=1e-14, atol=1e-16)
        got = outs[i].cpu().numpy().reshape(-1, meshes[i].nf)[g_of_o]
        F0o = np.linalg.norm(om.residual(w.params, u0, u0))
        Fg = np.linalg.norm(om.residual(w.params, got.reshape(-1), u0))
        assert Fg <= 1.05e-12 * F0o, i
        # every field within the first-order bound 2 ||J^-1|| (||F(U_gpu)|| +
        # ||F(U_ref)||) (a 1e-12 residual moves the weakly determined
        # pressure direction by up to that much)
        Fr = np.linalg.norm(om.residual(w.params, ref, u0))
        bound = 2.0 * _inv_norm(om.jacobian(w.params, ref, u0)) * (Fg + Fr)
        assert np.linalg.norm(got.reshape(-1) - ref) <= bound + 1e-12 * np.linalg.norm(ref), i
    batch.close()


def _inv_norm(J, seed=0, its=25):
    """||J^-1||_2 by power iteration on J^-T J^-1 (sparse LU)."""
    import scipy.sparse.linalg as spla
    lu = spla.splu(J.tocsc())
    x = np.random.default_rng(seed).standard_normal(J.shape[0])
    for _ in range(its):
        x = lu.solve(lu.solve(x), trans="T")
        x /= np.linalg.norm(x)
    return float(np.linalg.norm(lu.solve(x)))
