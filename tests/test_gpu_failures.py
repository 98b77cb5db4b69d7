"""Failure detection through the C ABI: every error is a status code, the
GPU context stays usable, and the next call on the same mesh succeeds.

Faults are made on the host (non-finite input, iteration caps, an injected
Krylov breakdown); nothing here makes a kernel fault, trap or hang.
"""
import numpy as np
import pytest

from paper_1912_12453_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NONFINITE, NEWTON, KRYLOV = 4, 5, 6


@pytest.fixture(scope="module")
def setup():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1912_12453_gb300 import build, chns
    build.build()
    wl = W.workload("droplet2d_l5")
    mesh = chns.Mesh(wl.leaves)
    U0 = torch.from_numpy(W.initial_state(mesh.coords, wl).reshape(-1)).cuda()
    chns.init_mu(mesh, wl.params, U0)
    return chns, wl, mesh, U0


def _good_step(chns, wl, mesh, U0):
    import torch
    out = torch.empty_like(U0)
    st = chns.step(mesh, wl.params, U0, out, chns.SolverOpts.make(newton_rtol=1e-10))
    assert st["res_final"] <= 1e-10 * st["res0"]
    return out


def test_nan_input_gives_nonfinite(setup):
    import torch
    chns, wl, mesh, U0 = setup
    bad = U0.clone()
    bad[7 * mesh.nf + mesh.dim + 1] = float("nan")
    out = torch.empty_like(U0)
    with pytest.raises(chns.ChnsError) as ei:
        chns.step(mesh, wl.params, bad, out, chns.SolverOpts.make())
    assert ei.value.status == NONFINITE
    _good_step(chns, wl, mesh, U0)


def test_newton_cap_gives_newton_error(setup):
    import torch
    chns, wl, mesh, U0 = setup
    out = torch.empty_like(U0)
    opts = chns.SolverOpts.make(newton_rtol=1e-14, newton_atol=0.0, newton_max_it=1, krylov_rtol=1e-2)
    with pytest.raises(chns.ChnsError) as ei:
        chns.step(mesh, wl.params, U0, out, opts)
    assert ei.value.status == NEWTON and "Newton reached 1" in str(ei.value)
    _good_step(chns, wl, mesh, U0)


def test_krylov_cap_one_iteration_stalls_newton(setup):
    """krylov_max_it = 1: each correction is one FGMRES iteration; Newton
    cannot reach a tight tolerance in two iterations and reports it."""
    import torch
    chns, wl, mesh, U0 = setup
    out = torch.empty_like(U0)
    opts = chns.SolverOpts.make(newton_rtol=1e-12, newton_max_it=2, krylov_max_it=1)
    with pytest.raises(chns.ChnsError) as ei:
        chns.step(mesh, wl.params, U0, out, opts)
    assert ei.value.status == NEWTON
    _good_step(chns, wl, mesh, U0)


@pytest.mark.parametrize("use_graph", [True, False])
def test_injected_krylov_breakdown(setup, monkeypatch, use_graph):
    import torch
    chns, wl, mesh, U0 = setup
    out = torch.empty_like(U0)
    monkeypatch.setenv("CHNS_INJECT", "krylov")
    with pytest.raises(chns.ChnsError) as ei:
        chns.step(mesh, wl.params, U0, out, chns.SolverOpts.make(use_graph=use_graph))
    assert ei.value.status == KRYLOV and "breakdown" in str(ei.value)
    monkeypatch.delenv("CHNS_INJECT")
    _good_step(chns, wl, mesh, U0)


def test_graphs_and_plain_launches_give_the_same_step(setup):
    import torch
    chns, wl, mesh, U0 = setup
    outs = []
    for g in (True, False):
        out = torch.empty_like(U0)
        chns.step(mesh, wl.params, U0, out, chns.SolverOpts.make(precision="fp32", newton_rtol=1e-10,
                                                                 use_graph=g))
        outs.append(out)
    assert torch.equal(outs[0], outs[1])


def test_invalid_options_rejected(setup):
    import torch
    chns, wl, mesh, U0 = setup
    out = torch.empty_like(U0)
    for kw in (dict(krylov_restart=0), dict(krylov_restart=65), dict(krylov_max_it=0), dict(newton_max_it=-1)):
        with pytest.raises(chns.ChnsError) as ei:
            chns.step(mesh, wl.params, U0, out, chns.SolverOpts.make(**kw))
        assert ei.value.status == 1
    bad = W.Params(2, 1e-3, 0.0, 35.0, 125.0, 25.0, 1.0, 0.1, 0.1)  # Cn = 0
    with pytest.raises(chns.ChnsError) as ei:
        chns.residual(mesh, bad, U0, U0)
    assert ei.value.status == 1
