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


def test_batch_step_matches_single_steps():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1912_12453_gb300 import build, chns
    build.build()
    wls = _instances()
    meshes = [chns.Mesh(w.leaves) for w in wls]
    U0 = []
    for m, w in zip(meshes, wls):
        u = torch.from_numpy(W.initial_state(m.coords, w).reshape(-1)).cuda()
        chns.init_mu(m, w.params, u)
        U0.append(u)
    opts = chns.SolverOpts.make(precision="fp32", newton_rtol=1e-13, newton_atol=1e-16, krylov_rtol=1e-6,
                                newton_max_it=30)
    single = []
    for m, w, u in zip(meshes, wls, U0):
        out = torch.empty_like(u)
        chns.step(m, w.params, u, out, opts)
        single.append(out)
    batch = chns.Batch(meshes, [w.params for w in wls])
    outs = [torch.empty_like(u) for u in U0]
    stats = batch.step(U0, outs, opts)
    from oracle import oracle as O
    for i, (m, w) in enumerate(zip(meshes, wls)):
        # the oracle's Newton root of the instance's own step (sparse direct solves)
        om = O.OracleMesh(w.leaves)
        g_of_o = W.match_nodes(m.coords_int, om.coords_int)
        u0 = U0[i].cpu().numpy().reshape(-1, m.nf)[g_of_o].reshape(-1)
        ref, _ = om.step(w.params, u0, rtol=1e-14, atol=1e-16)
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
