"""Python binding of libchns (ctypes): argument marshalling only.

Every computation runs in the CUDA kernels of ``libchns.so``; this module
passes torch CUDA tensors' device pointers and the current CUDA stream.  If
the library is not built, ``lib()`` raises: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libchns.so")

CHNS_FP64 = 0
CHNS_FP32_BULK = 1
CHNS_PC_TWO_LEVEL = 0
CHNS_PC_MULTIGRID = 1
# FP32 J.w schedules the autotuner chooses among (StepStats.jacvec_variant)
JACVEC_VARIANTS = ["element-local buffer + node gather, 128-thread blocks, 6/SM",
                   "element-local buffer + node gather, 256-thread blocks, 3/SM",
                   "element-local buffer + node gather, 64-thread blocks, 12/SM",
                   "element-local buffer + node gather, 128-thread blocks, 8/SM (at most 64 registers)",
                   "element colours, in-place adds into y, 128-thread blocks",
                   "element-local buffer + node gather, 128-thread blocks, 5/SM (at most 102 registers)",
                   "element-local buffer + node gather, 128-thread blocks, 4/SM (at most 128 registers)"]
STATUS = {0: "CHNS_OK", 1: "CHNS_ERR_ARG", 2: "CHNS_ERR_MESH", 3: "CHNS_ERR_CUDA",
          4: "CHNS_ERR_NONFINITE", 5: "CHNS_ERR_NEWTON", 6: "CHNS_ERR_KRYLOV",
          8: "CHNS_ERR_OOM"}

EXPORTS = ["chns_mesh_create", "chns_mesh_info", "chns_mesh_node_coords", "chns_mesh_destroy",
           "chns_residual", "chns_jacvec", "chns_init_mu", "chns_step", "chns_energy_mass",
           "chns_batch_create", "chns_batch_step", "chns_batch_destroy", "chns_last_error",
           "chns_kernel_launches", "chns_energy_mass_noalloc", "chns_tau_floor_count",
           "chns_mesh_check", "chns_mesh_jacvec_schedule", "chns_mesh_leaves", "chns_leaves_adapt",
           "chns_leaves_transfer", "chns_leaves_mark_interface", "chns_leaves_remesh", "chns_leaves_free"]


class ChnsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("dt", ctypes.c_double), ("Cn", ctypes.c_double),
                ("Re", ctypes.c_double), ("We", ctypes.c_double), ("Pe", ctypes.c_double),
                ("Fr", ctypes.c_double), ("rho_ratio", ctypes.c_double), ("eta_ratio", ctypes.c_double),
                ("C_I", ctypes.c_double), ("gravity", ctypes.c_double * 3)]

    @classmethod
    def of(cls, p) -> "Params":
        """From any object with the fields of workloads.Params."""
        return cls(int(p.dim), p.dt, p.Cn, p.Re, p.We, p.Pe, p.Fr, p.rho_ratio, p.eta_ratio, p.C_I,
                   (ctypes.c_double * 3)(*p.gravity))


class SolverOpts(ctypes.Structure):
    _fields_ = [("newton_rtol", ctypes.c_double), ("newton_atol", ctypes.c_double),
                ("newton_max_it", ctypes.c_int), ("krylov_rtol", ctypes.c_double),
                ("krylov_restart", ctypes.c_int), ("krylov_max_it", ctypes.c_int),
                ("precision", ctypes.c_int), ("reuse_preconditioner", ctypes.c_int),
                ("coarse_level", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("preconditioner", ctypes.c_int), ("mg_coarsest", ctypes.c_int), ("mg_smooth", ctypes.c_int),
                ("mg_omega", ctypes.c_double), ("block_iteration", ctypes.c_int), ("block_tol", ctypes.c_double),
                ("block_max_it", ctypes.c_int), ("autotune", ctypes.c_int)]

    @classmethod
    def make(cls, precision="fp64", newton_rtol=1e-10, newton_atol=1e-13, newton_max_it=20,
             krylov_rtol=1e-4, krylov_restart=64, krylov_max_it=600, reuse_preconditioner=1,
             coarse_level=-1, use_graph=True, preconditioner="two_level", mg_coarsest=-1, mg_smooth=1,
             mg_omega=0.4, block_iteration=False, block_tol=1e-4, block_max_it=50, autotune=False):
        prec = CHNS_FP64 if precision == "fp64" else CHNS_FP32_BULK
        pcn = {"two_level": CHNS_PC_TWO_LEVEL, "multigrid": CHNS_PC_MULTIGRID}[preconditioner]
        return cls(newton_rtol, newton_atol, newton_max_it, krylov_rtol, krylov_restart, krylov_max_it,
                   prec, int(reuse_preconditioner), int(coarse_level), int(bool(use_graph)), pcn,
                   int(mg_coarsest), int(mg_smooth), float(mg_omega), int(bool(block_iteration)),
                   float(block_tol), int(block_max_it), int(bool(autotune)))


class StepStats(ctypes.Structure):
    _fields_ = [("newton_its", ctypes.c_int), ("krylov_its_total", ctypes.c_int),
                ("res0", ctypes.c_double), ("res_final", ctypes.c_double),
                ("energy_old", ctypes.c_double), ("energy_new", ctypes.c_double),
                ("mass_old", ctypes.c_double), ("mass_new", ctypes.c_double),
                ("seconds", ctypes.c_double), ("jacvec_ms", ctypes.c_double),
                ("jacvec_calls", ctypes.c_int), ("residual_ms", ctypes.c_double),
                ("residual_calls", ctypes.c_int), ("precond_ms", ctypes.c_double),
                ("fp64_newton_its", ctypes.c_int), ("block_its", ctypes.c_int), ("jacvec_variant", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libchns.so is not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, i32, st = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int
        L.chns_last_error.restype = ctypes.c_char_p
        L.chns_kernel_launches.restype = ctypes.c_uint64
        L.chns_kernel_launches.argtypes = []
        L.chns_mesh_create.restype = st
        L.chns_mesh_create.argtypes = [i32, i64, vp, vp, i32, vp, vp, ctypes.POINTER(vp)]
        L.chns_mesh_info.restype = st
        L.chns_mesh_info.argtypes = [vp, vp, vp, vp, vp]
        L.chns_mesh_node_coords.restype = st
        L.chns_mesh_node_coords.argtypes = [vp, vp]
        L.chns_mesh_destroy.argtypes = [vp]
        L.chns_mesh_destroy.restype = None
        L.chns_residual.restype = st
        L.chns_residual.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
        L.chns_jacvec.restype = st
        L.chns_jacvec.argtypes = [vp, vp, vp, vp, vp, vp, i32, vp]
        L.chns_init_mu.restype = st
        L.chns_init_mu.argtypes = [vp, vp, vp, vp]
        L.chns_step.restype = st
        L.chns_step.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.chns_energy_mass.restype = st
        L.chns_energy_mass.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.chns_tau_floor_count.restype = st
        L.chns_tau_floor_count.argtypes = [vp, vp, vp, vp, vp, vp]
        L.chns_mesh_check.restype = st
        L.chns_mesh_check.argtypes = [vp]
        L.chns_mesh_jacvec_schedule.restype = st
        L.chns_mesh_jacvec_schedule.argtypes = [vp, i32, vp, vp]
        L.chns_energy_mass_noalloc.restype = st
        L.chns_energy_mass_noalloc.argtypes = [vp, vp, vp, vp, vp]
        L.chns_batch_create.restype = st
        L.chns_batch_create.argtypes = [i32, vp, vp, ctypes.POINTER(vp)]
        L.chns_batch_step.restype = st
        L.chns_batch_step.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.chns_batch_destroy.argtypes = [vp]
        L.chns_batch_destroy.restype = None
        L.chns_mesh_leaves.restype = st
        L.chns_mesh_leaves.argtypes = [vp, vp, vp]
        L.chns_leaves_adapt.restype = st
        L.chns_leaves_adapt.argtypes = [i32, i32, i64, vp, vp, vp, vp, vp, vp]
        L.chns_leaves_transfer.restype = st
        L.chns_leaves_transfer.argtypes = [i32, i32, i64, vp, vp, i64, vp, i32, vp, i64, vp, vp]
        L.chns_leaves_mark_interface.restype = st
        L.chns_leaves_mark_interface.argtypes = [i32, i32, i64, vp, vp, i64, vp, i32, vp, i32,
                                                 ctypes.c_double, i32, i32, i64, vp, vp, vp]
        L.chns_leaves_remesh.restype = st
        L.chns_leaves_remesh.argtypes = [i32, i32, i64, vp, vp, i64, vp, i32, vp, i32, ctypes.c_double,
                                         i32, i32, vp, vp, vp, vp]
        L.chns_leaves_free.restype = None
        L.chns_leaves_free.argtypes = [vp]
        _lib = L
    return _lib


def _check(status: int):
    if status != 0:
        raise ChnsError(status, lib().chns_last_error().decode())


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


def _stream(stream=None) -> Optional[int]:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream or None


class Mesh:
    """A library-owned mesh built from octree leaves (host arrays)."""

    def __init__(self, leaves, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)):
        L = lib()
        self.dim = int(leaves.dim)
        self.max_level = int(leaves.max_level)
        self.nf = self.dim + 3
        lev = np.ascontiguousarray(leaves.level, dtype=np.uint8)
        anc = np.ascontiguousarray(leaves.anchor, dtype=np.uint32)
        self._lo = (ctypes.c_double * 3)(*lo)
        self._hi = (ctypes.c_double * 3)(*hi)
        h = ctypes.c_void_p()
        _check(L.chns_mesh_create(self.dim, lev.shape[0], lev.ctypes.data, anc.ctypes.data, self.max_level,
                                  ctypes.addressof(self._lo), ctypes.addressof(self._hi), ctypes.byref(h)))
        self._h = h
        nn, nd, nh = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        nc = ctypes.c_int()
        _check(L.chns_mesh_info(h, ctypes.byref(nn), ctypes.byref(nd), ctypes.byref(nc), ctypes.byref(nh)))
        self.n_nodes, self.n_dof, self.n_colours, self.n_hanging = nn.value, nd.value, nc.value, nh.value
        self.n_elem = int(lev.shape[0])
        self.coords_int = np.zeros((self.n_nodes, self.dim), dtype=np.int64)
        _check(L.chns_mesh_node_coords(h, self.coords_int.ctypes.data))
        lo_a = np.asarray(lo[: self.dim], dtype=np.float64)
        hi_a = np.asarray(hi[: self.dim], dtype=np.float64)
        self.lo, self.hi = tuple(lo), tuple(hi)
        self.coords = lo_a + self.coords_int * ((hi_a - lo_a) / float(1 << self.max_level))

    def leaves(self) -> "Leaves":
        """The leaves the mesh was built from (Morton order)."""
        lev = np.zeros(self.n_elem, dtype=np.uint8)
        anc = np.zeros((self.n_elem, self.dim), dtype=np.uint32)
        _check(lib().chns_mesh_leaves(self._h, lev.ctypes.data, anc.ctypes.data))
        return Leaves(self.dim, self.max_level, lev, anc)

    @property
    def handle(self):
        return self._h

    def jacvec_schedule(self, variant: int = -1):
        """Fix (variant >= 0) or read the FP32 J.w schedule; returns (current, times_ms)."""
        cur = ctypes.c_int()
        times = (ctypes.c_double * 7)()
        _check(lib().chns_mesh_jacvec_schedule(self._h, int(variant), ctypes.byref(cur), times))
        return cur.value, list(times)

    def check(self):
        """Host-side validation of colouring, gather lists and hanging constraints."""
        _check(lib().chns_mesh_check(self._h))

    def close(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.chns_mesh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Leaves:
    """A leaf list: level[n] (uint8) and anchor[n, dim] (uint32), Morton order."""

    def __init__(self, dim: int, max_level: int, level, anchor):
        self.dim, self.max_level = int(dim), int(max_level)
        self.level = np.ascontiguousarray(level, dtype=np.uint8)
        self.anchor = np.ascontiguousarray(np.asarray(anchor, dtype=np.uint32).reshape(-1, self.dim))

    @property
    def n(self) -> int:
        return int(self.level.shape[0])


def _leaf_arrays(leaves):
    lev = np.ascontiguousarray(leaves.level, dtype=np.uint8)
    anc = np.ascontiguousarray(leaves.anchor, dtype=np.uint32)
    return lev, anc


def _take_leaves(dim, max_level, n, lp, ap) -> Leaves:
    try:
        m = n.value
        lev = np.ctypeslib.as_array(ctypes.cast(lp, ctypes.POINTER(ctypes.c_uint8)), shape=(m,)).copy()
        anc = np.ctypeslib.as_array(ctypes.cast(ap, ctypes.POINTER(ctypes.c_uint32)), shape=(m * dim,)).copy()
    finally:
        lib().chns_leaves_free(lp)
        lib().chns_leaves_free(ap)
    return Leaves(dim, max_level, lev, anc)


def _field(U, xyz, nf):
    U = np.ascontiguousarray(U, dtype=np.float64).reshape(-1)
    xyz = np.ascontiguousarray(xyz, dtype=np.int64)
    if U.shape[0] != xyz.shape[0] * nf:
        raise ValueError("field size does not match the node count")
    return U, xyz


def leaves_adapt(leaves, mark=None) -> Leaves:
    """One split / merge pass by marks (+1, -1, 0), then 2:1 balance (host)."""
    lev, anc = _leaf_arrays(leaves)
    mk = None if mark is None else np.ascontiguousarray(mark, dtype=np.int8)
    if mk is not None and mk.shape[0] != lev.shape[0]:
        raise ValueError("one mark per leaf")
    n, lp, ap = ctypes.c_int64(), ctypes.c_void_p(), ctypes.c_void_p()
    _check(lib().chns_leaves_adapt(leaves.dim, leaves.max_level, lev.shape[0], lev.ctypes.data, anc.ctypes.data,
                                   None if mk is None else mk.ctypes.data, ctypes.byref(n), ctypes.byref(lp),
                                   ctypes.byref(ap)))
    return _take_leaves(leaves.dim, leaves.max_level, n, lp, ap)


def leaves_transfer(leaves, xyz, U, points, nf: Optional[int] = None) -> np.ndarray:
    """Values at integer points of the nodal Q1 field U (host, [n_nodes, nf])."""
    nf = int(nf if nf is not None else leaves.dim + 3)
    lev, anc = _leaf_arrays(leaves)
    U, xyz = _field(U, xyz, nf)
    pts = np.ascontiguousarray(points, dtype=np.int64)
    out = np.zeros((pts.shape[0], nf), dtype=np.float64)
    _check(lib().chns_leaves_transfer(leaves.dim, leaves.max_level, lev.shape[0], lev.ctypes.data,
                                      anc.ctypes.data, xyz.shape[0], xyz.ctypes.data, nf, U.ctypes.data,
                                      pts.shape[0], pts.ctypes.data, out.ctypes.data))
    return out


def leaves_mark_interface(src, xyz, U, leaves, level_min: int, level_max: int, phi_band: float = 0.9,
                          nf: Optional[int] = None, phi_index: Optional[int] = None) -> np.ndarray:
    """Interface marks (+1, -1, 0) of a leaf list against the phi of U on src (host)."""
    nf = int(nf if nf is not None else src.dim + 3)
    phi_index = int(phi_index if phi_index is not None else src.dim + 1)
    slev, sanc = _leaf_arrays(src)
    lev, anc = _leaf_arrays(leaves)
    U, xyz = _field(U, xyz, nf)
    mark = np.zeros(lev.shape[0], dtype=np.int8)
    _check(lib().chns_leaves_mark_interface(src.dim, src.max_level, slev.shape[0], slev.ctypes.data,
                                            sanc.ctypes.data, xyz.shape[0], xyz.ctypes.data, nf, U.ctypes.data,
                                            phi_index, float(phi_band), int(level_min), int(level_max),
                                            lev.shape[0], lev.ctypes.data, anc.ctypes.data, mark.ctypes.data))
    return mark


def leaves_remesh(src, xyz, U, level_min: int, level_max: int, phi_band: float = 0.9,
                  nf: Optional[int] = None, phi_index: Optional[int] = None):
    """Leaves refined to level_max around the interface of U's phi and
    coarsened to level_min elsewhere, 2:1 balanced (host).  Returns
    (Leaves, passes)."""
    nf = int(nf if nf is not None else src.dim + 3)
    phi_index = int(phi_index if phi_index is not None else src.dim + 1)
    slev, sanc = _leaf_arrays(src)
    U, xyz = _field(U, xyz, nf)
    n, lp, ap, passes = ctypes.c_int64(), ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_int()
    _check(lib().chns_leaves_remesh(src.dim, src.max_level, slev.shape[0], slev.ctypes.data, sanc.ctypes.data,
                                    xyz.shape[0], xyz.ctypes.data, nf, U.ctypes.data, phi_index,
                                    float(phi_band), int(level_min), int(level_max), ctypes.byref(n),
                                    ctypes.byref(lp), ctypes.byref(ap), ctypes.byref(passes)))
    return _take_leaves(src.dim, src.max_level, n, lp, ap), passes.value


def remesh(mesh: Mesh, U, level_min: int, level_max: int, phi_band: float = 0.9):
    """Remesh around the interface of the device state U and transfer U:
    returns (new Mesh, new device state, passes).  The octree work and the
    interpolation run in the library on the host; U is copied to the host and
    the transferred state back to U's device."""
    import torch
    src = mesh.leaves()
    U_host = U.detach().to("cpu", torch.float64).numpy()
    new_leaves, passes = leaves_remesh(src, mesh.coords_int, U_host, level_min, level_max, phi_band, mesh.nf)
    new_mesh = Mesh(new_leaves, mesh.lo, mesh.hi)
    U_new = leaves_transfer(src, mesh.coords_int, U_host, new_mesh.coords_int, mesh.nf)
    return new_mesh, torch.from_numpy(U_new.reshape(-1)).to(U.device), passes


def residual(mesh: Mesh, params, U_new, U_old, forcing=None, bc=None, out=None, stream=None):
    import torch
    if out is None:
        out = torch.empty_like(U_new)
    prm = Params.of(params)
    _check(lib().chns_residual(mesh.handle, ctypes.byref(prm), _ptr(U_new), _ptr(U_old), _ptr(forcing),
                               _ptr(bc), _ptr(out), _stream(stream)))
    return out


def jacvec(mesh: Mesh, params, U_new, U_old, w, out=None, precision="fp64", stream=None):
    import torch
    prec = CHNS_FP64 if precision == "fp64" else CHNS_FP32_BULK
    want = torch.float64 if prec == CHNS_FP64 else torch.float32
    if w.dtype != want:
        raise ValueError(f"w must be {want} for precision {precision}")
    if out is None:
        out = torch.empty_like(w)
    prm = Params.of(params)
    _check(lib().chns_jacvec(mesh.handle, ctypes.byref(prm), _ptr(U_new), _ptr(U_old), _ptr(w), _ptr(out),
                             prec, _stream(stream)))
    return out


def init_mu(mesh: Mesh, params, U, stream=None):
    prm = Params.of(params)
    _check(lib().chns_init_mu(mesh.handle, ctypes.byref(prm), _ptr(U), _stream(stream)))
    return U


def step(mesh: Mesh, params, U_n, out, opts: Optional[SolverOpts] = None, U_nm1=None, forcing=None, bc=None,
         stream=None, stats=True):
    prm = Params.of(params)
    o = opts or SolverOpts.make()
    s = StepStats() if stats else None
    _check(lib().chns_step(mesh.handle, ctypes.byref(prm), ctypes.byref(o), _ptr(U_n), _ptr(U_nm1),
                           _ptr(forcing), _ptr(bc), _ptr(out), ctypes.byref(s) if s is not None else None,
                           _stream(stream)))
    return s.as_dict() if s is not None else None


def energy_mass(mesh: Mesh, params, U, stream=None):
    prm = Params.of(params)
    e, m, b = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().chns_energy_mass(mesh.handle, ctypes.byref(prm), _ptr(U), ctypes.byref(e), ctypes.byref(m),
                                  ctypes.byref(b), _stream(stream)))
    return e.value, m.value, b.value


def tau_floor_count(mesh: Mesh, params, U_new, U_old, stream=None) -> int:
    prm = Params.of(params)
    c = ctypes.c_int64()
    _check(lib().chns_tau_floor_count(mesh.handle, ctypes.byref(prm), _ptr(U_new), _ptr(U_old), ctypes.byref(c),
                                      _stream(stream)))
    return int(c.value)


def kernel_launches() -> int:
    return int(lib().chns_kernel_launches())


def energy_mass_noalloc(mesh: Mesh, params, U, out3, stream=None):
    """Allocation-free diagnostics: out3 is a CUDA float64 tensor of 3 entries."""
    prm = Params.of(params)
    _check(lib().chns_energy_mass_noalloc(mesh.handle, ctypes.byref(prm), _ptr(U), _ptr(out3),
                                          _stream(stream)))
    return out3


class Batch:
    def __init__(self, meshes: Sequence[Mesh], params: Sequence):
        self.meshes = list(meshes)
        n = len(self.meshes)
        arr = (ctypes.c_void_p * n)(*[m.handle.value for m in self.meshes])
        prm = (Params * n)(*[Params.of(p) for p in params])
        h = ctypes.c_void_p()
        _check(lib().chns_batch_create(n, arr, prm, ctypes.byref(h)))
        self._h = h

    def step(self, U_n, out, opts: Optional[SolverOpts] = None, U_nm1=None, stream=None):
        n = len(self.meshes)
        o = opts or SolverOpts.make()
        a = (ctypes.c_void_p * n)(*[_ptr(u) for u in U_n])
        c = (ctypes.c_void_p * n)(*[_ptr(u) for u in out])
        b = (ctypes.c_void_p * n)(*[_ptr(u) for u in U_nm1]) if U_nm1 is not None else None
        st = (StepStats * n)()
        _check(lib().chns_batch_step(self._h, ctypes.byref(o), a, b, c, st, _stream(stream)))
        return [s.as_dict() for s in st]

    def close(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.chns_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
