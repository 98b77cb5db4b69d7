"""The allocation-free diagnostics entry point against the allocating one.

chns_energy_mass_noalloc serves callers that may not allocate device memory
while running (work issued during a CUDA graph capture, hosts whose device
memory belongs to a pool fixed at start-up).  It must give the same energy,
phi integral and light-phase volume as chns_energy_mass, call after call,
although its scratch is one fixed array shared by all calls.  This file runs
last so that a failure here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest

from paper_1912_12453_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_noalloc_energy_mass_matches_allocating_entry_point():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1912_12453_gb300 import build, chns
    build.build()
    L = chns.lib()
    leaves = W.band_leaves(3, 3, 5, [W.Sphere((0.5, 0.45, 0.4), 0.22)], 0.04)
    mesh = chns.Mesh(leaves)
    prm = W.Params(3, 1e-3, 0.04, 10.0, 3.0, 25.0, 1.0, 0.1, 0.2, gravity=(0.0, 0.0, -1.0))
    cprm = chns.Params.of(prm)
    rng = np.random.default_rng(42)
    out3 = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for call in range(2):
        U = torch.from_numpy(rng.uniform(-1.2, 1.2, mesh.n_dof)).to("cuda")
        e, m, b = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        assert L.chns_energy_mass(mesh.handle, ctypes.byref(cprm), U.data_ptr(), ctypes.byref(e),
                                  ctypes.byref(m), ctypes.byref(b), stream.cuda_stream or None) == 0
        assert L.chns_energy_mass_noalloc(mesh.handle, ctypes.byref(cprm), U.data_ptr(), out3.data_ptr(),
                                          stream.cuda_stream or None) == 0, L.chns_last_error()
        got = out3.cpu().numpy()
        ref = np.array([e.value, m.value, b.value])
        assert np.all(np.abs(got - ref) <= 1e-12 * np.maximum(1.0, np.abs(ref))), (call, got, ref)


def test_noalloc_rejects_meshes_beyond_its_scratch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1912_12453_gb300 import chns
    L = chns.lib()
    mesh = chns.Mesh(W.uniform_leaves(3, 7))  # 2,097,152 leaves: exactly at the limit
    prm = chns.Params.of(W.Params(3, 1e-3, 0.04, 10.0, 3.0, 25.0, 1.0, 0.1, 0.2))
    U = torch.zeros(mesh.n_dof, dtype=torch.float64, device="cuda")
    out3 = torch.zeros(3, dtype=torch.float64, device="cuda")
    assert L.chns_energy_mass_noalloc(mesh.handle, ctypes.byref(prm), U.data_ptr(), out3.data_ptr(), None) == 0
    mesh.close()
    big = W.build_leaves(3, 7, 8, lambda l, lo, hi: (lo[:, 0] < 1e-9) & (lo[:, 1] < 1e-9) & (lo[:, 2] < 1e-9))
    mesh2 = chns.Mesh(big)
    U2 = torch.zeros(mesh2.n_dof, dtype=torch.float64, device="cuda")
    s = L.chns_energy_mass_noalloc(mesh2.handle, ctypes.byref(prm), U2.data_ptr(), out3.data_ptr(), None)
    assert s == 1 and b"too large" in L.chns_last_error()


def test_noalloc_checks_parameters_like_the_allocating_entry_point():
    """Both entry points accept and reject the same parameters: Cn = 0 or
    Fr = 0 is an argument error (status 1), not a NaN in out3."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1912_12453_gb300 import chns
    L = chns.lib()
    mesh = chns.Mesh(W.uniform_leaves(2, 3))
    U = torch.zeros(mesh.n_dof, dtype=torch.float64, device="cuda")
    out3 = torch.zeros(3, dtype=torch.float64, device="cuda")
    for bad in (dict(Cn=0.0), dict(Fr=0.0)):
        kw = dict(dt=1e-3, Cn=0.04, Re=10.0, We=3.0, Pe=25.0, Fr=1.0, rho_ratio=0.1, eta_ratio=0.2)
        kw.update(bad)
        prm = chns.Params.of(W.Params(2, **kw))
        e, m, b = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        assert L.chns_energy_mass(mesh.handle, ctypes.byref(prm), U.data_ptr(), ctypes.byref(e), ctypes.byref(m),
                                  ctypes.byref(b), None) == 1
        assert L.chns_energy_mass_noalloc(mesh.handle, ctypes.byref(prm), U.data_ptr(), out3.data_ptr(),
                                          None) == 1

