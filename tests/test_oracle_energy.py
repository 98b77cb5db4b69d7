"""Energy and mass over CN steps of the oracle (property checks, Sec. 3.3).

The discrete scheme is not proven energy stable once the VMS terms and the
phi* clip enter, so this is a property check on the 2D droplet (1,024 leaves):

- without gravity (1/Fr = 0) the energy functional (Eq. energy_functional)
  decreases at every step;
- the integral of phi is conserved to round-off at every step (Prop.
  mass_conservation), with gravity on.

With gravity on, the energy as read here (gravity potential (1/Fr) int rho z
outside the 1/(Cn We) factor) decreases for the first steps and then grows
by ~1e-4 relative per step, on level-5 and level-6 meshes alike: the
potential term changes through the diffusive flux of phi, which the
momentum equation's gravity work does not balance.
"""
import dataclasses

import numpy as np

from oracle.oracle import OracleMesh
from paper_1912_12453_gb300 import workloads as W


def _run(Fr, steps):
    wl = W.workload("droplet2d_l5")
    prm = dataclasses.replace(wl.params, Fr=Fr)
    om = OracleMesh(wl.leaves)
    U = om.init_mu(prm, W.initial_state(om.coords, wl).reshape(-1))
    E, M, _ = om.energy_mass(prm, U)
    Es, Ms = [E], [M]
    for _ in range(steps):
        U, _ = om.step(prm, U, rtol=1e-10)
        E, M, _ = om.energy_mass(prm, U)
        Es.append(E)
        Ms.append(M)
    return np.array(Es), np.array(Ms)


def test_energy_decreases_without_gravity():
    Es, Ms = _run(1e12, 8)
    assert np.all(np.diff(Es) < 0), np.diff(Es)
    assert np.abs(Ms - Ms[0]).max() <= 1e-12 * abs(Ms[0])


def test_mass_conserved_with_gravity():
    Es, Ms = _run(1.0, 4)
    assert np.abs(Ms - Ms[0]).max() <= 1e-12 * abs(Ms[0])
    assert np.all(np.diff(Es)[:4] < 0)  # the early steps still dissipate
