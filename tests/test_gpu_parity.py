"""CUDA path against the oracle, element by element, on seeded inputs.

Tolerances (norm-wise relative 2-norm): FP64 apply 1e-12, FP32-bulk apply
1e-5, converged step 1e-9.
"""
import numpy as np
import pytest

from paper_1912_12453_gb300 import workloads as W
from tests.harness import Pair, rel, random_state, physical_state

pytestmark = pytest.mark.gpu

TOL64, TOL32, TOLSTEP = 1e-12, 1e-5, 1e-9


def _params(dim, **kw):
    base = dict(dt=1e-2, Cn=0.3, Re=7.0, We=3.0, Pe=5.0, Fr=2.0, rho_ratio=0.3, eta_ratio=0.6)
    base.update(kw)
    g = (0.6, -0.8, 0.0) if dim == 2 else (0.48, -0.6, 0.64)
    return W.Params(dim, gravity=g, **base)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1912_12453_gb300 import build
    build.build()


def _meshes():
    return {
        "u2_l1": W.uniform_leaves(2, 1),
        "u2_l3": W.uniform_leaves(2, 3),
        "hang2": W.tiny_leaves(2, "hang"),
        "front2": W.half_refined_leaves(2, 3),
        "band2": W.band_leaves(2, 3, 6, [W.Sphere((0.45, 0.55), 0.2)], 0.03),
        "u3_l1": W.uniform_leaves(3, 1),
        "u3_l2": W.uniform_leaves(3, 2),
        "hang3": W.tiny_leaves(3, "hang"),
        "front3": W.half_refined_leaves(3, 2),
        "band3": W.band_leaves(3, 2, 5, [W.Sphere((0.5, 0.45, 0.4), 0.25)], 0.04),
    }


MESHES = list(_meshes().keys())


@pytest.fixture(scope="module")
def pairs():
    return {k: Pair(v) for k, v in _meshes().items()}


@pytest.mark.parametrize("name", MESHES)
def test_mesh_nodes_match_oracle(pairs, name):
    p = pairs[name]
    assert p.gm.n_nodes == p.om.n_nodes
    assert p.gm.n_hanging == p.om.n_hanging
    assert p.gm.n_dof == p.om.n_dof


@pytest.mark.parametrize("name", MESHES)
@pytest.mark.parametrize("with_data", [False, True])
def test_residual_fp64(pairs, name, with_data):
    p = pairs[name]
    dim = p.om.dim
    prm = _params(dim)
    Un = random_state(p.om.n_nodes, p.nf, 1)
    Uo = random_state(p.om.n_nodes, p.nf, 2)
    f = random_state(p.om.n_nodes, p.nf, 3) if with_data else None
    g = random_state(p.om.n_nodes, p.nf, 4) if with_data else None
    ref = p.om.residual(prm, Un, Uo, f, g)
    got = p.chns.residual(p.gm, prm, p.to_gpu(Un), p.to_gpu(Uo),
                          None if f is None else p.to_gpu(f), None if g is None else p.to_gpu(g))
    assert rel(p.to_oracle(got), ref) <= TOL64


@pytest.mark.parametrize("name", MESHES)
def test_jacvec_fp64(pairs, name):
    p = pairs[name]
    prm = _params(p.om.dim)
    Un = random_state(p.om.n_nodes, p.nf, 5)
    Uo = random_state(p.om.n_nodes, p.nf, 6)
    w = random_state(p.om.n_nodes, p.nf, 7, -1, 1)
    ref = p.om.jacvec(prm, Un, Uo, w)
    got = p.chns.jacvec(p.gm, prm, p.to_gpu(Un), p.to_gpu(Uo), p.to_gpu(w))
    assert rel(p.to_oracle(got), ref) <= TOL64


@pytest.mark.parametrize("name", MESHES)
def test_jacvec_fp32_bulk(pairs, name):
    import torch
    p = pairs[name]
    wl = W.workload("droplet2d_l5" if p.om.dim == 2 else "droplet3d_l6")
    prm = wl.params
    Uo, Un = physical_state(p.om, wl)
    w = W.perturbation(p.om.n_nodes, p.nf, 2)[1]
    ref = p.om.jacvec(prm, Un, Uo, w)
    got = p.chns.jacvec(p.gm, prm, p.to_gpu(Un), p.to_gpu(Uo), p.to_gpu(w, torch.float32), precision="fp32")
    assert rel(p.to_oracle(got), ref) <= TOL32


@pytest.mark.parametrize("name", MESHES)
def test_mesh_check(pairs, name):
    """Host-side validator: colours with disjoint expanded footprints, exact
    node gather lists, well-formed hanging constraints."""
    pairs[name].gm.check()


def _float_exact_states(n_nodes, nf, seed, amp, damp):
    """(U_new, U_old) whose CN average and increment are exact float32 values:
    the FP32 path then sees exactly the oracle's inputs, and only its
    arithmetic differs."""
    rng = np.random.default_rng(seed)
    ut = rng.uniform(-amp, amp, (n_nodes, nf)).astype(np.float32).astype(np.float64)
    dl = rng.uniform(-damp, damp, (n_nodes, nf)).astype(np.float32).astype(np.float64)
    return ut + 0.5 * dl, ut - 0.5 * dl


@pytest.mark.parametrize("name", ["hang2", "band2", "hang3", "front3"])
def test_tau_floor_regime(pairs, name):
    """States where the tau_m radicand falls below 4/dt^2 at some Gauss points
    (dt = 0.2, Pe = 0.5, Re = 50, |phi| up to 1.1 so the phi* clip is active
    too): both sides floor the same Gauss points, and the residual and J.w
    (FP64 and FP32-bulk) match the oracle at the standard tolerances.  The
    floor makes J.w jump where a radicand crosses 4/dt^2, so the FP32 path
    could take the other branch at a Gauss point within its rounding of the
    threshold; the oracle shows every radicand of these states at least
    1e-4 (relative) away from it."""
    import torch
    p = pairs[name]
    prm = _params(p.om.dim, dt=0.2, Pe=0.5, Re=50.0)
    Un, Uo = _float_exact_states(p.om.n_nodes, p.nf, 21, 1.1, 0.05)
    w = np.random.default_rng(23).uniform(-1, 1, p.om.n_dof).astype(np.float32).astype(np.float64)
    n_ref = p.om.tau_floor_count(prm, Un, Uo)
    n_gpu = p.chns.tau_floor_count(p.gm, prm, p.to_gpu(Un), p.to_gpu(Uo))
    assert n_ref > 0 and n_gpu == n_ref
    assert n_ref < p.om.n_elem << p.om.dim  # and not all of them: both branches are exercised
    assert p.om.tau_floor_margin(prm, Un, Uo) > 1e-4
    ref = p.om.residual(prm, Un, Uo)
    got = p.chns.residual(p.gm, prm, p.to_gpu(Un), p.to_gpu(Uo))
    assert rel(p.to_oracle(got), ref) <= TOL64
    refj = p.om.jacvec(prm, Un, Uo, w)
    gotj = p.chns.jacvec(p.gm, prm, p.to_gpu(Un), p.to_gpu(Uo), p.to_gpu(w))
    assert rel(p.to_oracle(gotj), refj) <= TOL64
    gotj32 = p.chns.jacvec(p.gm, prm, p.to_gpu(Un), p.to_gpu(Uo), p.to_gpu(w, torch.float32), precision="fp32")
    assert rel(p.to_oracle(gotj32), refj) <= TOL32


@pytest.mark.parametrize("name", ["hang2", "band2", "hang3", "band3"])
def test_tau_floor_counts_in_an_extreme_regime(pairs, name):
    """About half of all Gauss points floored (dt = 1, Pe = 0.05, Re = 1e4,
    |phi| up to 1.5): the same points on both sides, and the residual at the
    FP64 tolerance.  (J.w is not compared here: with 1/Pe = 20 and random
    nodal data on leaves down to h = 1/32 its terms cancel strongly and the
    two evaluation orders differ by a few 1e-12.)"""
    p = pairs[name]
    prm = _params(p.om.dim, dt=1.0, Pe=0.05, Re=1e4)
    Un = random_state(p.om.n_nodes, p.nf, 11, -1.5, 1.5)
    Uo = random_state(p.om.n_nodes, p.nf, 12, -1.5, 1.5)
    n_ref = p.om.tau_floor_count(prm, Un, Uo)
    assert n_ref > (p.om.n_elem << p.om.dim) // 5
    assert p.chns.tau_floor_count(p.gm, prm, p.to_gpu(Un), p.to_gpu(Uo)) == n_ref
    ref = p.om.residual(prm, Un, Uo)
    got = p.chns.residual(p.gm, prm, p.to_gpu(Un), p.to_gpu(Uo))
    assert rel(p.to_oracle(got), ref) <= TOL64


@pytest.mark.parametrize("name", ["u2_l3", "band3"])
def test_tau_floor_absent_in_the_workload_regime(pairs, name):
    """The droplet parameters and smooth states floor no Gauss point."""
    p = pairs[name]
    wl = W.workload("droplet2d_l5" if p.om.dim == 2 else "droplet3d_l6")
    Uo, Un = physical_state(p.om, wl)
    assert p.om.tau_floor_count(wl.params, Un, Uo) == 0
    assert p.chns.tau_floor_count(p.gm, wl.params, p.to_gpu(Un), p.to_gpu(Uo)) == 0


@pytest.mark.parametrize("name", ["hang2", "band2", "hang3", "band3"])
def test_energy_mass(pairs, name):
    p = pairs[name]
    prm = _params(p.om.dim)
    U = random_state(p.om.n_nodes, p.nf, 8)
    ref = p.om.energy_mass(prm, U)
    got = p.chns.energy_mass(p.gm, prm, p.to_gpu(U))
    for a, b in zip(got, ref):
        assert abs(a - b) <= 1e-12 * max(1.0, abs(b))


@pytest.mark.parametrize("name", ["band2", "front3"])
def test_init_mu(pairs, name):
    p = pairs[name]
    prm = _params(p.om.dim)
    U = random_state(p.om.n_nodes, p.nf, 9, -1, 1)
    ref = p.om.init_mu(prm, U)
    t = p.to_gpu(U)
    p.chns.init_mu(p.gm, prm, t)
    assert rel(p.to_oracle(t), ref) <= 1e-10


def _inv_norm(J, seed=0, its=25):
    """||J^{-1}||_2 by power iteration on J^{-T} J^{-1} (sparse LU)."""
    import scipy.sparse.linalg as spla
    lu = spla.splu(J.tocsc())
    x = np.random.default_rng(seed).standard_normal(J.shape[0])
    for _ in range(its):
        x = lu.solve(lu.solve(x), trans="T")
        x /= np.linalg.norm(x)
    return float(np.linalg.norm(lu.solve(x)))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name", ["band2", "front3"])
def test_step_matches_oracle(pairs, name, precision):
    """One CN step from the droplet's initial state.

    The GPU state must be a root of the oracle's residual (to 1e-13 of the
    initial residual), v, phi and mu must match the oracle's Newton root to
    1e-9, and the whole state (pressure included) must lie within the
    first-order bound ||J^-1|| (||F(U_gpu)|| + ||F(U_ref)||): the PSPG block
    scales the pressure by tau_m/(rho We), so ||J^-1|| reaches ~1e8 along a
    pressure direction and rounding-level residuals move p that far.
    """
    import torch
    p = pairs[name]
    wl = W.workload("droplet2d_l5" if p.om.dim == 2 else "droplet3d_l6")
    prm = wl.params
    U0 = W.initial_state(p.om.coords, wl)
    U0 = p.om.init_mu(prm, U0)
    ref, st = p.om.step(prm, U0, rtol=1e-14, atol=1e-16)
    t0 = p.to_gpu(U0)
    out = torch.empty_like(t0)
    opts = p.chns.SolverOpts.make(precision=precision, newton_rtol=1e-14, newton_atol=1e-16,
                                  krylov_rtol=1e-10 if precision == "fp64" else 1e-6, newton_max_it=30)
    stats = p.chns.step(p.gm, prm, t0, out, opts)
    assert stats["newton_its"] >= 1
    got = p.to_oracle(out)
    F0 = np.linalg.norm(p.om.residual(prm, U0, U0))
    Fg = np.linalg.norm(p.om.residual(prm, got, U0))
    Fr = np.linalg.norm(p.om.residual(prm, ref, U0))
    assert Fg <= 1e-13 * F0
    d = (got - ref).reshape(-1, p.nf)
    r = ref.reshape(-1, p.nf)
    dim = p.om.dim
    for k in list(range(dim)) + [dim + 1, dim + 2]:
        assert np.linalg.norm(d[:, k]) <= TOLSTEP * max(np.linalg.norm(r[:, k]), 1e-30) + 1e-14, k
    bound = 2.0 * _inv_norm(p.om.jacobian(prm, ref, U0)) * (Fg + Fr)
    assert np.linalg.norm(d) <= bound + TOLSTEP * np.linalg.norm(r)
    assert abs(stats["mass_new"] - stats["mass_old"]) < 1e-12


@pytest.mark.parametrize("name", ["droplet2d_l5", "droplet3d_l6", "bubble3d_l5_9"])
def test_workload_applies_match_oracle(name):
    """The full-size meshes of the workloads (the 2D droplet, the uniform
    level-6 3D droplet the benchmark times, and the adaptive 3D bubble with
    hanging nodes, 1.4M leaves), in the launch configuration the benchmark
    uses: residual and J.w at the initial state plus a seeded perturbation,
    every entry compared."""
    import torch
    from oracle import oracle as O
    from paper_1912_12453_gb300 import chns
    wl = W.workload(name)
    p = Pair(wl.leaves)
    assert p.gm.n_hanging == p.om.n_hanging and p.gm.n_nodes == p.om.n_nodes
    Uo, Un = physical_state(p.om, wl)
    w = W.perturbation(p.om.n_nodes, p.nf, 2)[1]
    ref = p.om.residual(wl.params, Un, Uo)
    got = chns.residual(p.gm, wl.params, p.to_gpu(Un), p.to_gpu(Uo))
    assert rel(p.to_oracle(got), ref) <= TOL64
    refj = p.om.jacvec(wl.params, Un, Uo, w)
    gotj = chns.jacvec(p.gm, wl.params, p.to_gpu(Un), p.to_gpu(Uo), p.to_gpu(w))
    assert rel(p.to_oracle(gotj), refj) <= TOL64
    gotj32 = chns.jacvec(p.gm, wl.params, p.to_gpu(Un), p.to_gpu(Uo), p.to_gpu(w, torch.float32),
                         precision="fp32")
    assert rel(p.to_oracle(gotj32), refj) <= TOL32


@pytest.fixture(scope="module")
def largest():
    import os
    wl = W.workload("merge3d_l6_10")
    p = Pair(wl.leaves)
    Uo, Un = physical_state(p.om, wl)
    w = W.perturbation(p.om.n_nodes, p.nf, 2)[1]
    refj = p.om.jacvec_threads(wl.params, Un, Uo, w, os.cpu_count() or 1)
    return wl, p, Uo, Un, w, refj


@pytest.mark.parametrize("schedule", [0, 5, 6])
def test_largest_workload_applies_match_oracle(largest, schedule):
    """The largest workload (two merging droplets, octree levels 6-10, 6.98M
    leaves, 771k hanging nodes, 39.6M DoF): FP64 and FP32-bulk J.w at the
    initial state plus a seeded perturbation, every entry compared with the
    oracle's J.w (run on all host cores), for the default FP32 schedule and
    the two register budgets the autotuner picks on the uniform workload."""
    import torch
    from paper_1912_12453_gb300 import chns
    wl, p, Uo, Un, w, refj = largest
    assert p.gm.n_hanging == p.om.n_hanging and p.gm.n_nodes == p.om.n_nodes
    if schedule == 0:
        gotj = chns.jacvec(p.gm, wl.params, p.to_gpu(Un), p.to_gpu(Uo), p.to_gpu(w))
        assert rel(p.to_oracle(gotj), refj) <= TOL64
    p.gm.jacvec_schedule(schedule)
    gotj32 = chns.jacvec(p.gm, wl.params, p.to_gpu(Un), p.to_gpu(Uo), p.to_gpu(w, torch.float32),
                         precision="fp32")
    assert rel(p.to_oracle(gotj32), refj) <= TOL32

