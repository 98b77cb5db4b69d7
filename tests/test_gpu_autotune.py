"""The FP32 J.w schedules the autotuner chooses among.

Every schedule must give the oracle's J.w to the FP32 tolerance (1e-5,
relative 2-norm) on uniform and hanging-node meshes; the autotuner must
time all of them, keep the fastest, and leave the CN step unchanged (the
schedules differ only in the summation order of a node's contributions).
"""
import numpy as np
import pytest

from paper_1912_12453_gb300 import workloads as W
from tests.harness import Pair, physical_state, rel

pytestmark = pytest.mark.gpu
N_SCHEDULES = 7


@pytest.fixture(scope="module")
def pairs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1912_12453_gb300 import build
    build.build()
    return {"u2_l4": Pair(W.uniform_leaves(2, 4)),
            "band2": Pair(W.band_leaves(2, 3, 6, [W.Sphere((0.45, 0.55), 0.2)], 0.03)),
            "u3_l3": Pair(W.uniform_leaves(3, 3)),
            "band3": Pair(W.band_leaves(3, 2, 5, [W.Sphere((0.5, 0.45, 0.4), 0.25)], 0.04))}


@pytest.mark.parametrize("name", ["u2_l4", "band2", "u3_l3", "band3"])
@pytest.mark.parametrize("variant", list(range(N_SCHEDULES)))
def test_every_schedule_matches_oracle(pairs, name, variant):
    import torch
    p = pairs[name]
    wl = W.workload("droplet2d_l5" if p.om.dim == 2 else "droplet3d_l6")
    Uo, Un = physical_state(p.om, wl)
    w = W.perturbation(p.om.n_nodes, p.nf, 2)[1]
    ref = p.om.jacvec(wl.params, Un, Uo, w)
    p.gm.jacvec_schedule(variant)
    got = p.chns.jacvec(p.gm, wl.params, p.to_gpu(Un), p.to_gpu(Uo), p.to_gpu(w, torch.float32), precision="fp32")
    assert rel(p.to_oracle(got), ref) <= 1e-5
    p.gm.jacvec_schedule(0)


def test_autotuner_times_every_schedule_and_keeps_the_step(pairs):
    import torch
    from paper_1912_12453_gb300 import chns
    wl = W.workload("droplet3d_l6")
    leaves = W.band_leaves(3, 3, 5, [W.Sphere((0.5, 0.45, 0.4), 0.25)], 0.04)
    outs = []
    for tune in (False, True):
        mesh = chns.Mesh(leaves)
        U0 = torch.from_numpy(W.initial_state(mesh.coords, wl).reshape(-1)).cuda()
        chns.init_mu(mesh, wl.params, U0)
        out = torch.empty_like(U0)
        st = chns.step(mesh, wl.params, U0, out, chns.SolverOpts.make(
            precision="fp32", newton_rtol=1e-12, newton_atol=1e-16, krylov_rtol=1e-6, newton_max_it=30,
            autotune=tune))
        cur, times = mesh.jacvec_schedule()
        if tune:
            assert all(t > 0 for t in times), times
            assert times[cur] == min(times) and st["jacvec_variant"] == cur
        else:
            assert cur == 0 and all(t < 0 for t in times)
        outs.append(out.reshape(-1, mesh.nf))
        mesh.close()
    for k in (0, 1, 2, 4, 5):
        assert float((outs[0][:, k] - outs[1][:, k]).norm()) <= 1e-9 * float(outs[0][:, k].norm()) + 1e-14
