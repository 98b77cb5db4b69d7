"""Python side of the CHNS oracle (test infrastructure only).

Loads ``liboracle.so`` (plain FP64 C++, built from ``chns_oracle.cpp`` by
``oracle/build.py``) and adds the pieces that are naturally written with a
library primitive:

* Newton's method on F(U^{k+1}; U^k) = 0 (Sec. 3.5): J dU = -F, U += dU,
  started from U^k, stopped when ||F||_2 <= rtol ||F(U^k)||_2 (or atol).  The
  linear solves use a sparse direct factorisation of the exact Jacobian
  assembled element by element, so no Krylov method or preconditioner is
  involved.
* the initial chemical potential: the L2 projection M mu0 = (N, psi'(phi0)) +
  Cn^2 (grad N, grad phi0), i.e. the chemical-potential row with U^{k+1} = U^k.

Only the test suite, the smoke check and the benchmark's CPU-baseline leg
import this module.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "chns_oracle.cpp")
_lib = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-pthread", "-o", _LIB_PATH, _SRC]
        subprocess.check_call(cmd)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        L.oracle_mesh_create.restype = vp
        L.oracle_mesh_create.argtypes = [i32, i64, vp, vp, i32, vp, vp, ctypes.c_char_p, i32]
        L.oracle_mesh_destroy.argtypes = [vp]
        L.oracle_mesh_info.argtypes = [vp, vp]
        L.oracle_mesh_nodes.argtypes = [vp, vp, vp]
        L.oracle_mesh_P.restype = i64
        L.oracle_mesh_P.argtypes = [vp, vp, vp, vp]
        L.oracle_residual.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.oracle_jacvec.argtypes = [vp, vp, vp, vp, vp, vp]
        L.oracle_jacobian_coo.restype = i64
        L.oracle_jacobian_coo.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.oracle_energy_mass.argtypes = [vp, vp, vp, vp]
        L.oracle_tau_floor_count.restype = i64
        L.oracle_tau_floor_count.argtypes = [vp, vp, vp, vp, vp]
        L.oracle_jacvec_threads.argtypes = [vp, vp, vp, vp, vp, vp, i32]
        _lib = L
    return _lib


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data


def _params_array(params) -> np.ndarray:
    t = params.as_tuple() if hasattr(params, "as_tuple") else tuple(params)
    return np.ascontiguousarray(np.asarray(t, dtype=np.float64))


def _vec(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1))


class OracleMesh:
    """Independent nodes are numbered in canonical order (z, y, x)."""

    def __init__(self, leaves, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)):
        L = lib()
        self.dim = leaves.dim
        self.max_level = leaves.max_level
        self.nf = self.dim + 3
        lev = np.ascontiguousarray(leaves.level, dtype=np.uint8)
        anc = np.ascontiguousarray(leaves.anchor, dtype=np.uint32)
        lo_a = np.asarray(lo, dtype=np.float64)
        hi_a = np.asarray(hi, dtype=np.float64)
        self.lo, self.hi = lo_a, hi_a
        err = ctypes.create_string_buffer(256)
        h = L.oracle_mesh_create(self.dim, lev.shape[0], _p(lev), _p(anc), self.max_level,
                                 _p(lo_a), _p(hi_a), err, 256)
        if not h:
            raise ValueError("oracle mesh: " + err.value.decode())
        self._h = ctypes.c_void_p(h)
        info = np.zeros(5, dtype=np.int64)
        L.oracle_mesh_info(self._h, _p(info))
        self.n_nodes, self.n_dof, self.n_hanging, self.origin, self.n_elem = (int(x) for x in info)
        self.coords_int = np.zeros((self.n_nodes, self.dim), dtype=np.int64)
        self.on_wall = np.zeros(self.n_nodes, dtype=np.uint8)
        L.oracle_mesh_nodes(self._h, _p(self.coords_int), _p(self.on_wall))
        scale = (hi_a[: self.dim] - lo_a[: self.dim]) / float(1 << self.max_level)
        self.coords = lo_a[: self.dim] + self.coords_int * scale

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.oracle_mesh_destroy(h)
            self._h = None

    # constrained rows ------------------------------------------------------
    def constrained_rows(self) -> np.ndarray:
        rows = []
        nf = self.nf
        wall = np.nonzero(self.on_wall)[0]
        for k in range(self.dim):
            rows.append(wall * nf + k)
        rows.append(np.array([self.origin * nf + self.dim]))
        return np.sort(np.concatenate(rows))

    def P(self):
        n = lib().oracle_mesh_P(self._h, None, None, None)
        start = np.zeros(self.n_elem * (1 << self.dim) + 1, dtype=np.int64)
        node = np.zeros(n, dtype=np.int64)
        w = np.zeros(n, dtype=np.float64)
        lib().oracle_mesh_P(self._h, _p(start), _p(node), _p(w))
        return start, node, w

    # operators -------------------------------------------------------------
    def residual(self, params, Un, Uo, f=None, g=None) -> np.ndarray:
        prm = _params_array(params)
        Un, Uo = _vec(Un), _vec(Uo)
        f = None if f is None else _vec(f)
        g = None if g is None else _vec(g)
        F = np.zeros(self.n_dof)
        lib().oracle_residual(self._h, _p(prm), _p(Un), _p(Uo), _p(f), _p(g), _p(F))
        return F

    def jacvec(self, params, Un, Uo, w) -> np.ndarray:
        prm = _params_array(params)
        Un, Uo, w = _vec(Un), _vec(Uo), _vec(w)
        y = np.zeros(self.n_dof)
        lib().oracle_jacvec(self._h, _p(prm), _p(Un), _p(Uo), _p(w), _p(y))
        return y

    def jacvec_threads(self, params, Un, Uo, w, n_threads: int) -> np.ndarray:
        """jacvec on ``n_threads`` host threads (elements grouped by colour)."""
        prm = _params_array(params)
        Un, Uo, w = _vec(Un), _vec(Uo), _vec(w)
        y = np.zeros(self.n_dof)
        lib().oracle_jacvec_threads(self._h, _p(prm), _p(Un), _p(Uo), _p(w), _p(y), int(n_threads))
        return y

    def tau_floor_count(self, params, Un, Uo) -> int:
        """Gauss points whose tau_m radicand is raised to 4/dt^2."""
        prm = _params_array(params)
        return int(lib().oracle_tau_floor_count(self._h, _p(prm), _p(_vec(Un)), _p(_vec(Uo)), None))

    def tau_floor_margin(self, params, Un, Uo) -> float:
        """Smallest |radicand dt^2/4 - 1| over all Gauss points: the distance
        of the closest one from the floor decision."""
        prm = _params_array(params)
        m = ctypes.c_double()
        lib().oracle_tau_floor_count(self._h, _p(prm), _p(_vec(Un)), _p(_vec(Uo)), ctypes.byref(m))
        return float(m.value)

    def jacobian(self, params, Un, Uo):
        import scipy.sparse as sp
        prm = _params_array(params)
        Un, Uo = _vec(Un), _vec(Uo)
        n = lib().oracle_jacobian_coo(self._h, _p(prm), _p(Un), _p(Uo), None, None, None)
        I = np.zeros(n, dtype=np.int64)
        J = np.zeros(n, dtype=np.int64)
        V = np.zeros(n)
        lib().oracle_jacobian_coo(self._h, _p(prm), _p(Un), _p(Uo), _p(I), _p(J), _p(V))
        return sp.csr_matrix((V, (I, J)), shape=(self.n_dof, self.n_dof))

    def energy_mass(self, params, U):
        prm = _params_array(params)
        U = _vec(U)
        out = np.zeros(3)
        lib().oracle_energy_mass(self._h, _p(prm), _p(U), _p(out))
        return float(out[0]), float(out[1]), float(out[2])

    # solvers ---------------------------------------------------------------
    def step(self, params, Uk, rtol=1e-10, atol=1e-14, max_it=25, f=None, g=None, guess=None):
        """One CN step: Newton on F(U; U^k) = 0 from U^k (or ``guess``)."""
        import scipy.sparse.linalg as spla
        Uk = _vec(Uk)
        U = Uk.copy() if guess is None else _vec(guess).copy()
        F = self.residual(params, U, Uk, f, g)
        r0 = np.linalg.norm(self.residual(params, Uk, Uk, f, g))
        hist = [float(np.linalg.norm(F))]
        its = 0
        while hist[-1] > max(rtol * r0, atol) and its < max_it:
            J = self.jacobian(params, U, Uk)
            dU = spla.spsolve(J.tocsc(), -F)
            U = U + dU
            F = self.residual(params, U, Uk, f, g)
            hist.append(float(np.linalg.norm(F)))
            its += 1
        if hist[-1] > max(rtol * r0, atol):
            raise RuntimeError(f"oracle Newton did not converge: {hist}")
        return U, {"newton_its": its, "res0": r0, "history": hist}

    def init_mu(self, params, U) -> np.ndarray:
        """Return U with mu replaced by the L2 projection of psi'(phi) - Cn^2 lap phi."""
        import scipy.sparse.linalg as spla
        U = _vec(U).copy()
        nf, dim = self.nf, self.dim
        imu = np.arange(self.n_nodes) * nf + dim + 2
        J = self.jacobian(params, U, U).tocsc()
        M = -2.0 * J[imu][:, imu]        # the mu-mu block of the mu row is -M/2
        F = self.residual(params, U, U)
        U[imu] += spla.spsolve(M.tocsc(), F[imu])
        return U
