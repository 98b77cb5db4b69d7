"""The NS <-> CH block iteration of Sec. 3.1 (Fig. flowchart_block) against
the coupled Newton solve.

Both solve the same discrete CN step; the block iteration alternates Newton
on (v, p) with phi, mu frozen and Newton on (phi, mu) with v, p frozen, until
a block iteration changes no entry by more than block_tol.  Its result must
agree with the coupled root to within the block tolerance (the paper's 1e-4),
and to 1e-8 in v, phi, mu when block_tol is tight; the coupled residual of a
tight block-iteration result must be small.
"""
import numpy as np
import pytest

from paper_1912_12453_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1912_12453_gb300 import build, chns
    build.build()
    return chns


@pytest.mark.parametrize("name", ["droplet2d_l5", "band3"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_block_iteration_reaches_the_coupled_root(env, name, precision):
    import torch
    chns = env
    if name == "droplet2d_l5":
        wl = W.workload(name)
        leaves, prm = wl.leaves, wl.params
    else:
        wl = W.workload("droplet3d_l6")
        leaves, prm = W.band_leaves(3, 3, 5, [W.Sphere((0.5, 0.45, 0.4), 0.25)], 0.04), wl.params
        wl = W.Workload("band3", leaves, prm, [W.Sphere((0.5, 0.5, 0.3), 0.15)], False)
    mesh = chns.Mesh(leaves)
    U0 = torch.from_numpy(W.initial_state(mesh.coords, wl).reshape(-1)).cuda()
    chns.init_mu(mesh, prm, U0)
    base = dict(precision=precision, newton_rtol=1e-12, newton_atol=1e-15, krylov_rtol=1e-8, newton_max_it=30)
    coupled = torch.empty_like(U0)
    chns.step(mesh, prm, U0, coupled, chns.SolverOpts.make(**base))
    for tol, close in ((1e-4, 1e-4), (1e-10, 1e-8)):
        out = torch.empty_like(U0)
        st = chns.step(mesh, prm, U0, out, chns.SolverOpts.make(block_iteration=True, block_tol=tol, **base))
        assert st["block_its"] >= 2
        d = (out - coupled).reshape(-1, mesh.nf).abs().max(0).values.cpu().numpy()
        dim = mesh.dim
        fields = list(range(dim)) + [dim + 1, dim + 2]
        assert np.all(d[fields] <= close), (tol, d)
        if tol == 1e-10:
            assert st["res_final"] <= 1e-8 * st["res0"], st
        assert abs(st["mass_new"] - st["mass_old"]) < 1e-11
