"""Remeshing on a device mesh (Sec. 4, "Intergrid transfers"): the leaves a
mesh returns, a remesh of a device state around a moved interface against the
oracle's remesh and transfer, and one Crank-Nicolson step on the new mesh
against the oracle's step from the oracle's transferred state."""
import numpy as np
import pytest

from paper_1912_12453_gb300 import workloads as W
from tests.harness import Pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1912_12453_gb300 import build
    build.build()


@pytest.mark.parametrize("dim", [2, 3])
def test_mesh_leaves_round_trip(dim):
    from paper_1912_12453_gb300 import chns
    L = W.band_leaves(dim, 2, 5, [W.Sphere((0.5, 0.4, 0.5)[:dim], 0.2)], 0.03)
    m = chns.Mesh(L)
    got = m.leaves()
    assert np.array_equal(got.level, L.level) and np.array_equal(got.anchor, L.anchor.astype(np.uint32))
    assert got.max_level == L.max_level and got.dim == dim


def test_remesh_then_step_matches_the_oracle():
    import torch
    from oracle import remesh as R
    from oracle.oracle import OracleMesh
    from paper_1912_12453_gb300 import chns
    dim, base, top, Cn = 2, 3, 7, 0.02
    prm = W.Params(2, 1e-3, Cn, 35.0, 125.0, 1 / Cn, 1.0, 0.1, 0.1)
    L = W.band_leaves(dim, base, top, [W.Sphere((0.5, 0.35), 0.18)], Cn)
    p = Pair(L)
    x = p.om.coords
    U = np.zeros((p.om.n_nodes, dim + 3))
    U[:, dim + 1] = W.phi_profile(x, [W.Sphere((0.5, 0.35 + 3 / 32), 0.18)], Cn, True)
    U[:, dim + 2] = 0.5 * (U[:, dim + 1] ** 3 - U[:, dim + 1])
    wall = W.boundary_mask(p.om.coords_int, L.max_level)
    U[:, 1] = np.where(wall, 0.0, 0.05 * np.sin(np.pi * x[:, 0]) * np.sin(np.pi * x[:, 1]))
    new_mesh, gUn, passes = chns.remesh(p.gm, p.to_gpu(U), base, top)
    ora, opasses, margin = R.remesh(L, p.om.coords_int, U, base, top)
    assert margin > 1e-9 and passes == opasses >= 1
    got = new_mesh.leaves()
    assert np.array_equal(got.level, ora.level) and np.array_equal(got.anchor, ora.anchor)
    on = OracleMesh(ora)
    Uo = R.transfer(L, p.om.coords_int, U, on.coords_int)
    g_of_o = W.match_nodes(new_mesh.coords_int, on.coords_int)
    Ug = gUn.double().cpu().numpy().reshape(new_mesh.n_nodes, -1)[g_of_o]
    assert np.max(np.abs(Ug - Uo)) < 1e-14
    # one CN step on the new mesh from the transferred state
    opts = chns.SolverOpts.make(precision="fp64", newton_rtol=1e-14, newton_atol=1e-16, krylov_rtol=1e-6,
                                newton_max_it=30)
    out = torch.empty_like(gUn)
    chns.step(new_mesh, prm, gUn, out, opts)
    Ugs = out.double().cpu().numpy().reshape(new_mesh.n_nodes, -1)[g_of_o].reshape(-1)
    Uos, _ = on.step(prm, Uo.reshape(-1), rtol=1e-14, atol=1e-16)
    F0 = np.linalg.norm(on.residual(prm, Uo.reshape(-1), Uo.reshape(-1)))
    assert np.linalg.norm(on.residual(prm, Ugs, Uo.reshape(-1))) <= 1e-12 * F0
    d, r = (Ugs - Uos).reshape(-1, dim + 3), Uos.reshape(-1, dim + 3)
    for f in list(range(dim)) + [dim + 1, dim + 2]:
        assert np.linalg.norm(d[:, f]) <= 1e-9 * np.linalg.norm(r[:, f]), f
