"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This module holds no arithmetic of the method itself (no weak form, no
stabilisation, no solver).  It produces only what a user would hand to the
solver:

* linear octrees / quadtrees as (level, anchor) leaf lists in Morton order,
  built top-down by refining every octant that meets the diffuse-interface band
  of one or more spheres (the refinement rule of Sec. 4, "Refinement"), then
  2:1 balanced across faces, edges and corners (Sec. 4, "2:1 Balancing");
* the initial fields of the droplet / bubble workloads sampled at node
  coordinates (tanh interface profile, Sec. 5);
* uniform random perturbation vectors from a fixed seed.

Nodal data are produced in *canonical order*: nodes sorted lexicographically by
their integer coordinates (z, then y, then x).  Each side maps canonical order
to its own node numbering by matching integer coordinates.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

PERTURB_SEED = 20191226


# --------------------------------------------------------------------------
# octree construction
# --------------------------------------------------------------------------

def _offsets(dim: int) -> np.ndarray:
    rng = (-1, 0, 1)
    if dim == 2:
        off = [(a, b) for b in rng for a in rng if (a, b) != (0, 0)]
    else:
        off = [(a, b, c) for c in rng for b in rng for a in rng if (a, b, c) != (0, 0, 0)]
    return np.asarray(off, dtype=np.int64)


def _key(coords: np.ndarray, level: int) -> np.ndarray:
    """Linear key of integer octant coordinates at one level (x fastest)."""
    k = np.zeros(coords.shape[0], dtype=np.int64)
    for ax in range(coords.shape[1] - 1, -1, -1):
        k = (k << level) | coords[:, ax]
    return k


def _unkey(keys: np.ndarray, level: int, dim: int) -> np.ndarray:
    mask = (1 << level) - 1
    out = np.empty((keys.shape[0], dim), dtype=np.int64)
    k = keys.copy()
    for ax in range(dim):
        out[:, ax] = k & mask
        k >>= level
    return out


def _children(coords: np.ndarray, dim: int) -> np.ndarray:
    n = coords.shape[0]
    ch = np.empty((n << dim, dim), dtype=np.int64)
    for c in range(1 << dim):
        bits = np.array([(c >> ax) & 1 for ax in range(dim)], dtype=np.int64)
        ch[c::1 << dim] = 2 * coords + bits
    return ch


def morton_keys(anchor: np.ndarray, max_level: int) -> np.ndarray:
    """Morton (Z-order) key of integer anchors at ``max_level`` (x = lowest bit)."""
    dim = anchor.shape[1]
    key = np.zeros(anchor.shape[0], dtype=np.uint64)
    a = anchor.astype(np.uint64)
    for b in range(max_level + 1):
        for ax in range(dim):
            key |= ((a[:, ax] >> np.uint64(b)) & np.uint64(1)) << np.uint64(dim * b + ax)
    return key


@dataclasses.dataclass
class Leaves:
    """A linear octree: leaves in Morton order."""
    dim: int
    max_level: int
    level: np.ndarray    # uint8 [n]
    anchor: np.ndarray   # uint32 [n, dim], integer corner at max_level resolution

    @property
    def n(self) -> int:
        return int(self.level.shape[0])


def build_leaves(dim: int, base_level: int, max_level: int, refine=None) -> Leaves:
    """Top-down refinement then 2:1 balance.

    ``refine(level, lo, hi) -> bool mask`` decides, for octants of one level
    given their physical boxes in the unit cube, which ones are split.  Every
    octant below ``base_level`` is split.
    """
    assert 1 <= base_level <= max_level <= 20
    refined: Dict[int, np.ndarray] = {}
    # levels below base: everything refined
    for l in range(base_level):
        n = 1 << l
        g = np.stack(np.meshgrid(*([np.arange(n, dtype=np.int64)] * dim), indexing="ij"), -1)
        refined[l] = np.unique(_key(g.reshape(-1, dim), l))
    for l in range(base_level, max_level):
        parents = _unkey(refined[l - 1], l - 1, dim)
        cand = _children(parents, dim)
        if refine is None or cand.shape[0] == 0:
            refined[l] = np.zeros(0, dtype=np.int64)
            continue
        h = 1.0 / (1 << l)
        lo = cand * h
        mask = np.asarray(refine(l, lo, lo + h), dtype=bool)
        refined[l] = np.unique(_key(cand[mask], l))
    # 2:1 balance (faces, edges and corners): every same-level neighbour of a
    # refined octant must exist, i.e. its parent must be refined.
    off = _offsets(dim)
    for l in range(max_level - 1, 0, -1):
        r = refined.get(l)
        if r is None or r.shape[0] == 0:
            continue
        c = _unkey(r, l, dim)
        nb = (c[:, None, :] + off[None, :, :]).reshape(-1, dim)
        inside = np.all((nb >= 0) & (nb < (1 << l)), axis=1)
        par = np.concatenate([nb[inside] >> 1, c >> 1])
        refined[l - 1] = np.union1d(refined[l - 1], _key(par, l - 1))
    # leaves: children of refined octants that are not refined themselves
    lev_list: List[np.ndarray] = []
    anc_list: List[np.ndarray] = []
    for l in range(1, max_level + 1):
        par = refined.get(l - 1)
        if par is None or par.shape[0] == 0:
            continue
        ch = _children(_unkey(par, l - 1, dim), dim)
        kch = _key(ch, l)
        r = refined.get(l, np.zeros(0, dtype=np.int64))
        keep = ~np.isin(kch, r, assume_unique=False)
        ch = ch[keep]
        lev_list.append(np.full(ch.shape[0], l, dtype=np.uint8))
        anc_list.append((ch << (max_level - l)).astype(np.uint32))
    level = np.concatenate(lev_list)
    anchor = np.concatenate(anc_list)
    order = np.argsort(morton_keys(anchor, max_level), kind="stable")
    return Leaves(dim, max_level, level[order], np.ascontiguousarray(anchor[order]))


def uniform_leaves(dim: int, level: int) -> Leaves:
    return build_leaves(dim, level, level, None)


@dataclasses.dataclass
class Sphere:
    center: Tuple[float, ...]
    radius: float


def band_refiner(spheres: Sequence[Sphere], half_width: float):
    """Refine octants that meet the shell |r - R| < half_width of any sphere."""
    def refine(level, lo, hi):
        hit = np.zeros(lo.shape[0], dtype=bool)
        for s in spheres:
            c = np.asarray(s.center[: lo.shape[1]], dtype=np.float64)
            near = np.clip(c, lo, hi)
            dmin = np.sqrt(((near - c) ** 2).sum(1))
            far = np.where(np.abs(lo - c) > np.abs(hi - c), lo, hi)
            dmax = np.sqrt(((far - c) ** 2).sum(1))
            hit |= (dmin < s.radius + half_width) & (dmax > s.radius - half_width)
        return hit
    return refine


def interface_half_width(Cn: float, phi_band: float = 0.9) -> float:
    """Distance from the interface at which |tanh(d / (sqrt(2) Cn))| = phi_band."""
    return math.sqrt(2.0) * Cn * math.atanh(phi_band)


def band_leaves(dim, base_level, max_level, spheres, Cn, phi_band=0.9) -> Leaves:
    return build_leaves(dim, base_level, max_level,
                        band_refiner(spheres, interface_half_width(Cn, phi_band)))


def tiny_leaves(dim: int, kind: str) -> Leaves:
    """Meshes of a few leaves: '1' (root split once per axis is not allowed:
    a single level-0 leaf is represented as level 0), '4' (uniform level 1 in
    2D / '8' in 3D) and 'hang' (level 1 with the first child refined once)."""
    if kind == "uniform1":
        return uniform_leaves(dim, 1)
    if kind == "hang":
        max_level = 2
        lev, anc = [], []
        for c in range(1 << dim):
            bits = [(c >> ax) & 1 for ax in range(dim)]
            if c == 0:
                for cc in range(1 << dim):
                    b2 = [(cc >> ax) & 1 for ax in range(dim)]
                    lev.append(2)
                    anc.append(b2)
            else:
                lev.append(1)
                anc.append([2 * b for b in bits])
        anc = np.asarray(anc, dtype=np.uint32)
        lev = np.asarray(lev, dtype=np.uint8)
        order = np.argsort(morton_keys(anc, max_level), kind="stable")
        return Leaves(dim, max_level, lev[order], np.ascontiguousarray(anc[order]))
    raise ValueError(kind)


def half_refined_leaves(dim: int, level: int) -> Leaves:
    """Uniform ``level`` with the octants in x < 1/2 refined once more: a
    straight refinement front of hanging nodes across the whole domain."""
    def refine(l, lo, hi):
        return hi[:, 0] <= 0.5 + 1e-12
    return build_leaves(dim, level, level + 1, refine)


# --------------------------------------------------------------------------
# node sets in canonical order
# --------------------------------------------------------------------------

def canonical_order(coords_int: np.ndarray) -> np.ndarray:
    """Permutation sorting integer node coordinates by (z, y, x)."""
    keys = tuple(coords_int[:, ax] for ax in range(coords_int.shape[1]))
    return np.lexsort(keys)


def match_nodes(coords_a: np.ndarray, coords_b: np.ndarray) -> np.ndarray:
    """Index map m with coords_a[m[i]] == coords_b[i] (exact integer match)."""
    oa = canonical_order(coords_a)
    ob = canonical_order(coords_b)
    if coords_a.shape != coords_b.shape or not np.array_equal(coords_a[oa], coords_b[ob]):
        raise ValueError("node sets differ")
    m = np.empty(coords_b.shape[0], dtype=np.int64)
    m[ob] = oa
    return m


# --------------------------------------------------------------------------
# physical parameters and initial data of the workloads
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Params:
    dim: int
    dt: float
    Cn: float
    Re: float
    We: float
    Pe: float
    Fr: float
    rho_ratio: float
    eta_ratio: float
    C_I: float = 6.0
    gravity: Tuple[float, float, float] = (0.0, -1.0, 0.0)

    def as_tuple(self):
        return (self.dim, self.dt, self.Cn, self.Re, self.We, self.Pe, self.Fr,
                self.rho_ratio, self.eta_ratio, self.C_I) + tuple(self.gravity)


@dataclasses.dataclass
class Workload:
    name: str
    leaves: Leaves
    params: Params
    spheres: List[Sphere]
    bubble: bool                  # True: light phase (phi = -1) inside the spheres
    velocity: Optional[str] = None  # None: fluid at rest; "merge": droplets approach
    steps: int = 1
    newton_rtol: float = 1e-10


def phi_profile(xyz: np.ndarray, spheres: Sequence[Sphere], Cn: float, bubble: bool) -> np.ndarray:
    """tanh interface profile; phi = +1 in the reference fluid outside bubbles,
    phi = +1 inside droplets.  Several spheres: the one nearest the point."""
    d = np.full(xyz.shape[0], np.inf)
    for s in spheres:
        c = np.asarray(s.center[: xyz.shape[1]])
        r = np.sqrt(((xyz - c) ** 2).sum(1))
        sd = r - s.radius
        d = np.where(np.abs(sd) < np.abs(d), sd, d)
    arg = d / (math.sqrt(2.0) * Cn)
    return np.tanh(arg) if bubble else np.tanh(-arg)


def initial_state(xyz: np.ndarray, wl: Workload) -> np.ndarray:
    """U^0 per node (canonical order given by ``xyz``): v, p = 0, phi, mu = 0.
    The chemical potential is left at zero; the solver projects it."""
    dim = wl.params.dim
    nf = dim + 3
    U = np.zeros((xyz.shape[0], nf))
    phi = phi_profile(xyz, wl.spheres, wl.params.Cn, wl.bubble)
    U[:, dim + 1] = phi
    if wl.velocity == "merge":
        U[:, 0] = -0.5 * np.sign(xyz[:, 0] - 0.5) * (1.0 + phi) / 2.0
        on_wall = np.any((xyz <= 0.0) | (xyz >= 1.0), axis=1)
        U[on_wall, :dim] = 0.0
    return U


def perturbation(n_nodes: int, nf: int, count: int = 1, seed: int = PERTURB_SEED) -> np.ndarray:
    """``count`` vectors uniform in [-1, 1], shape (count, n_nodes, nf)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=(count, n_nodes, nf))


def boundary_mask(xyz_int: np.ndarray, max_level: int) -> np.ndarray:
    top = 1 << max_level
    return np.any((xyz_int == 0) | (xyz_int == top), axis=1)


# the five workloads ---------------------------------------------------------

def workload(name: str) -> Workload:
    if name == "droplet2d_l5":
        p = Params(2, 1e-3, 0.04, 35.0, 125.0, 1 / 0.04, 1.0, 0.1, 0.1)
        return Workload(name, uniform_leaves(2, 5), p, [Sphere((0.5, 0.3), 0.15)], False,
                        steps=10, newton_rtol=1e-10)
    if name == "droplet3d_l6":
        p = Params(3, 5e-4, 0.02, 100.0, 50.0, 1 / 0.02, 1.0, 1e-2, 1e-2, gravity=(0.0, 0.0, -1.0))
        return Workload(name, uniform_leaves(3, 6), p, [Sphere((0.5, 0.5, 0.3), 0.15)], False,
                        steps=5, newton_rtol=1e-9)
    if name == "bubble3d_l5_9":
        p = Params(3, 2.5e-4, 0.01, 35.0, 1.0, 100.0, 1.0, 1e-3, 1e-2, gravity=(0.0, 0.0, -1.0))
        sp = [Sphere((0.5, 0.5, 0.25), 0.125)]
        return Workload(name, band_leaves(3, 5, 9, sp, 0.01), p, sp, True, steps=20, newton_rtol=1e-9)
    if name == "merge3d_l6_10":
        p = Params(3, 1e-4, 0.005, 100.0, 10.0, 200.0, 1.0, 1e-3, 1e-2, gravity=(0.0, 0.0, -1.0))
        sp = [Sphere((0.4, 0.5, 0.5), 0.1), Sphere((0.6, 0.5, 0.5), 0.1)]
        return Workload(name, band_leaves(3, 6, 10, sp, 0.005), p, sp, False, velocity="merge",
                        steps=5, newton_rtol=1e-9)
    raise KeyError(name)


def batched_workloads(n: int = 64, seed: int = 7) -> List[Workload]:
    """Independent droplet/bubble instances of uneven size and parameters."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        dim = 2 if rng.random() < 0.5 else 3
        top = int(rng.integers(6, 10)) if dim == 2 else int(rng.integers(5, 8))
        base = top - 2  # coarsest leaves at level >= 3: the coarse space of a union is level >= 2
        R = float(rng.uniform(0.1, 0.25))
        rho_r = float(10 ** rng.uniform(-3, 0))
        eta_r = float(10 ** rng.uniform(-2, 0))
        bubble = bool(rng.random() < 0.5)
        c = tuple(float(x) for x in rng.uniform(0.3, 0.7, size=dim))
        g = (0.0, -1.0, 0.0) if dim == 2 else (0.0, 0.0, -1.0)
        p = Params(dim, 5e-4, 0.02, 35.0, 10.0, 1 / 0.02, 1.0, rho_r, eta_r, gravity=g)
        sp = [Sphere(c, R)]
        out.append(Workload(f"inst{i}", band_leaves(dim, base, top, sp, 0.02), p, sp, bubble,
                            steps=10, newton_rtol=1e-9))
    return out
