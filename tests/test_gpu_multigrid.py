"""The geometric multigrid preconditioner over the octree levels.

A preconditioner changes the Krylov path, not the Newton root: a CN step with
the multigrid V-cycle must reach the same state as the oracle's Newton root
(v, phi, mu to 1e-9; the pressure by the first-order bound of its weakly
determined direction), on uniform and adaptive (hanging-node) meshes, with
the FP64 and the FP32-bulk operators, with and without graphs, and with
several smoothing settings.
"""
import numpy as np
import pytest

from paper_1912_12453_gb300 import workloads as W
from tests.harness import Pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1912_12453_gb300 import build
    build.build()


def _meshes():
    # oracle-compared meshes stay small: the oracle's Newton factorises the
    # full Jacobian with a sparse direct solver (a 3D mesh of ~10k DoF takes
    # tens of seconds per step on one core)
    return {
        "u2_l5": W.uniform_leaves(2, 5),
        "band2": W.band_leaves(2, 3, 6, [W.Sphere((0.45, 0.55), 0.2)], 0.03),
        "u3_l3": W.uniform_leaves(3, 3),
        "front3": W.half_refined_leaves(3, 2),
        "band3s": W.band_leaves(3, 2, 4, [W.Sphere((0.5, 0.45, 0.4), 0.2)], 0.04),
    }


@pytest.fixture(scope="module")
def pairs():
    return {k: Pair(v) for k, v in _meshes().items()}


_REFS = {}


def _oracle_root(p, name, prm, wl):
    """The oracle's initial state, Newton root and ||J^-1|| (computed once per mesh)."""
    if name not in _REFS:
        U0 = p.om.init_mu(prm, W.initial_state(p.om.coords, wl))
        ref, _ = p.om.step(prm, U0, rtol=1e-14, atol=1e-16)
        _REFS[name] = (U0, ref, _inv_norm(p.om.jacobian(prm, ref, U0)))
    return _REFS[name]


@pytest.fixture(scope="module")
def band3():
    """An adaptive 3D mesh too large for the oracle's direct solver (8,940
    leaves, hanging faces and edges): GPU-only comparisons."""
    from paper_1912_12453_gb300 import chns
    return chns.Mesh(W.band_leaves(3, 3, 5, [W.Sphere((0.5, 0.45, 0.4), 0.25)], 0.04))


def _inv_norm(J, seed=0, its=25):
    import scipy.sparse.linalg as spla
    lu = spla.splu(J.tocsc())
    x = np.random.default_rng(seed).standard_normal(J.shape[0])
    for _ in range(its):
        x = lu.solve(lu.solve(x), trans="T")
        x /= np.linalg.norm(x)
    return float(np.linalg.norm(lu.solve(x)))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name", ["u2_l5", "band2", "u3_l3", "front3", "band3s"])
def test_multigrid_step_matches_oracle(pairs, name, precision):
    import torch
    p = pairs[name]
    wl = W.workload("droplet2d_l5" if p.om.dim == 2 else "droplet3d_l6")
    prm = wl.params
    U0, ref, inv_norm = _oracle_root(p, name, prm, wl)
    t0 = p.to_gpu(U0)
    out = torch.empty_like(t0)
    opts = p.chns.SolverOpts.make(precision=precision, newton_rtol=1e-14, newton_atol=1e-16,
                                  krylov_rtol=1e-10 if precision == "fp64" else 1e-6, newton_max_it=30,
                                  preconditioner="multigrid")
    st = p.chns.step(p.gm, prm, t0, out, opts)
    got = p.to_oracle(out)
    F0 = np.linalg.norm(p.om.residual(prm, U0, U0))
    Fg = np.linalg.norm(p.om.residual(prm, got, U0))
    Fr = np.linalg.norm(p.om.residual(prm, ref, U0))
    assert Fg <= 1e-13 * F0
    d = (got - ref).reshape(-1, p.nf)
    r = ref.reshape(-1, p.nf)
    dim = p.om.dim
    for k in list(range(dim)) + [dim + 1, dim + 2]:
        assert np.linalg.norm(d[:, k]) <= 1e-9 * max(np.linalg.norm(r[:, k]), 1e-30) + 1e-14, k
    bound = 2.0 * inv_norm * (Fg + Fr)
    assert np.linalg.norm(d) <= bound + 1e-9 * np.linalg.norm(r)
    assert st["newton_its"] >= 1


def _band3_state(mesh):
    import torch
    from paper_1912_12453_gb300 import chns
    wl = W.workload("droplet3d_l6")
    U0 = torch.from_numpy(W.initial_state(mesh.coords, wl).reshape(-1)).cuda()
    chns.init_mu(mesh, wl.params, U0)
    return wl, U0


@pytest.mark.parametrize("kw", [dict(mg_smooth=2, mg_omega=0.5), dict(mg_coarsest=1), dict(use_graph=False)])
def test_multigrid_settings_reach_the_same_root(band3, kw):
    import torch
    from paper_1912_12453_gb300 import chns
    wl, U0 = _band3_state(band3)
    outs = []
    for extra in ({}, kw):
        out = torch.empty_like(U0)
        chns.step(band3, wl.params, U0, out, chns.SolverOpts.make(
            precision="fp32", newton_rtol=1e-14, newton_atol=1e-16, krylov_rtol=1e-6, newton_max_it=30,
            preconditioner="multigrid", **extra))
        outs.append(out.reshape(-1, band3.nf))
    for k in (0, 1, 2, 4, 5):
        assert float((outs[0][:, k] - outs[1][:, k]).norm()) <= 1e-9 * float(outs[0][:, k].norm()) + 1e-14


def test_multigrid_cuts_krylov_iterations(band3):
    """On the adaptive 3D mesh the V-cycle needs fewer FGMRES iterations than
    the two-level preconditioner for the same Newton solve."""
    import torch
    from paper_1912_12453_gb300 import chns
    wl, U0 = _band3_state(band3)
    its = {}
    for pcn in ("two_level", "multigrid"):
        out = torch.empty_like(U0)
        st = chns.step(band3, wl.params, U0, out, chns.SolverOpts.make(
            precision="fp32", newton_rtol=1e-9, krylov_rtol=1e-3, preconditioner=pcn))
        its[pcn] = st["krylov_its_total"]
    assert its["multigrid"] < its["two_level"], its
