"""Remeshing oracle (test infrastructure only): plain, brute-force Python for
small leaf sets.

Sec. 4 of the paper remeshes every few steps: the octree is refined again
around the current interface ("Refinement": an octant whose corner tests see
the surface is refined), 2:1 balanced ("2:1 Balancing": neighbouring octants
differ by at most one level), meshed, and the fields move to the new mesh by
interpolation between parents and children ("Intergrid transfers").  This
module restates those steps without any search structure:

* ``apply_marks``: +1 splits a leaf, -1 merges a family whose members are all
  leaves marked -1, 0 keeps it;
* ``balance``: while some leaf touches (closed boxes, across a face, an edge or
  a corner) a leaf at least two levels finer, split every such leaf.  Each of
  those splits is forced in any balanced refinement, so the fixed point is
  the coarsest balanced refinement;
* ``transfer``: for each point, the first leaf whose closed box holds it, its
  corner values through the oracle mesh's own hanging-node constraint matrix
  P, and the multilinear shape functions of that leaf;
* ``mark_interface`` / ``remesh``: the corner test on the transferred phi
  (|phi| <= band at a corner, or corners of both signs: the leaf aims at
  level_max, otherwise at level_min), alternated with adaptation passes.

Only the test suite imports this module.
"""
from __future__ import annotations

from typing import Optional

import numpy as np

from . import oracle as _oracle


class OLeaves:
    """A leaf list (level[n], anchor[n, dim]) in Morton order."""

    def __init__(self, dim, max_level, level, anchor):
        self.dim, self.max_level = int(dim), int(max_level)
        self.level = np.ascontiguousarray(level, dtype=np.uint8)
        self.anchor = np.ascontiguousarray(np.asarray(anchor, dtype=np.uint32).reshape(-1, self.dim))

    @property
    def n(self):
        return int(self.level.shape[0])


def morton_key(a, dim, max_level):
    """Bits of the anchor interleaved, x lowest."""
    k = 0
    for b in range(max_level + 1):
        for ax in range(dim):
            k |= ((int(a[ax]) >> b) & 1) << (dim * b + ax)
    return k


def _sorted(dim, max_level, octs):
    octs = sorted(set(octs), key=lambda o: morton_key(o[1], dim, max_level))
    return OLeaves(dim, max_level, [o[0] for o in octs], [list(o[1]) for o in octs])


def _octs(leaves):
    return [(int(l), tuple(int(x) for x in a)) for l, a in zip(leaves.level, leaves.anchor)]


def _children(o, dim, max_level):
    l, a = o
    h = 1 << (max_level - l - 1)
    return [(l + 1, tuple(a[k] + (h if (c >> k) & 1 else 0) for k in range(dim))) for c in range(1 << dim)]


def _parent(o, dim, max_level):
    l, a = o
    ps = 1 << (max_level - l + 1)
    return (l - 1, tuple(x // ps * ps for x in a))


def apply_marks(leaves, mark):
    dim, ml = leaves.dim, leaves.max_level
    octs = _octs(leaves)
    where = {o: i for i, o in enumerate(octs)}
    out = []
    for i, o in enumerate(octs):
        m = int(mark[i]) if mark is not None else 0
        if m > 0 and o[0] < ml:
            out.extend(_children(o, dim, ml))
        elif m < 0 and o[0] > 0:
            p = _parent(o, dim, ml)
            fam = _children(p, dim, ml)
            if all(f in where and int(mark[where[f]]) < 0 for f in fam):
                out.append(p)
            else:
                out.append(o)
        else:
            out.append(o)
    return _sorted(dim, ml, out)


def touching(leaves):
    """Boolean matrix: closed boxes of leaves i != j intersect."""
    a = leaves.anchor.astype(np.int64)
    s = (np.int64(1) << (leaves.max_level - leaves.level.astype(np.int64)))
    lo, hi = a, a + s[:, None]
    t = np.all((lo[:, None, :] <= hi[None, :, :]) & (lo[None, :, :] <= hi[:, None, :]), axis=2)
    np.fill_diagonal(t, False)
    return t


def is_balanced(leaves):
    lv = leaves.level.astype(np.int64)
    return not np.any(touching(leaves) & (np.abs(lv[:, None] - lv[None, :]) > 1))


def balance(leaves):
    dim, ml = leaves.dim, leaves.max_level
    while True:
        lv = leaves.level.astype(np.int64)
        bad = np.any(touching(leaves) & (lv[None, :] >= lv[:, None] + 2), axis=1)
        if not bad.any():
            return leaves
        octs = _octs(leaves)
        out = []
        for i, o in enumerate(octs):
            out.extend(_children(o, dim, ml) if bad[i] else [o])
        leaves = _sorted(dim, ml, out)


def adapt(leaves, mark=None):
    """One adaptation pass: marks, then 2:1 balance."""
    return balance(apply_marks(leaves, mark))


def transfer(leaves, xyz, U, points, nf: Optional[int] = None):
    """Values at integer points of the nodal field U (rows: the nodes with
    integer coordinates xyz) on the leaf list."""
    dim, ml = leaves.dim, leaves.max_level
    nf = nf if nf is not None else dim + 3
    om = _oracle.OracleMesh(leaves)
    U = np.asarray(U, dtype=np.float64).reshape(-1, nf)
    row = {tuple(int(v) for v in c): i for i, c in enumerate(np.asarray(xyz))}
    Uo = np.array([U[row[tuple(int(v) for v in c)]] for c in om.coords_int])
    start, node, w = om.P()
    a = leaves.anchor.astype(np.int64)
    s = np.int64(1) << (ml - leaves.level.astype(np.int64))
    nc = 1 << dim
    out = np.zeros((len(points), nf))
    for j, x in enumerate(np.asarray(points, dtype=np.int64)):
        inside = np.nonzero(np.all((a <= x) & (x <= a + s[:, None]), axis=1))[0]
        if inside.size == 0:
            raise ValueError("point outside the leaves")
        e = int(inside[0])
        t = (x - a[e]) / float(s[e])
        for c in range(nc):
            N = 1.0
            for k in range(dim):
                N *= t[k] if (c >> k) & 1 else 1.0 - t[k]
            r = e * nc + c
            uc = np.zeros(nf)
            for q in range(start[r], start[r + 1]):
                uc += w[q] * Uo[node[q]]
            out[j] += N * uc
    return out


def leaf_corners(leaves):
    """Integer corners of every leaf, [n * 2^dim, dim] (corner c: bit k = +s on axis k)."""
    dim, ml = leaves.dim, leaves.max_level
    a = leaves.anchor.astype(np.int64)
    s = np.int64(1) << (ml - leaves.level.astype(np.int64))
    off = np.array([[(c >> k) & 1 for k in range(dim)] for c in range(1 << dim)], dtype=np.int64)
    return (a[:, None, :] + off[None, :, :] * s[:, None, None]).reshape(-1, dim)


def mark_interface(src, xyz, U, leaves, level_min, level_max, band=0.9, phi_index=None, nf=None):
    """Marks of ``leaves`` and the smallest distance of a corner |phi| from
    the band (the margin of the comparisons)."""
    dim = src.dim
    nf = nf if nf is not None else dim + 3
    phi_index = phi_index if phi_index is not None else dim + 1
    pts, back = np.unique(leaf_corners(leaves), axis=0, return_inverse=True)
    phi = transfer(src, xyz, U, pts, nf)[:, phi_index][back.reshape(-1)].reshape(leaves.n, 1 << dim)
    near = np.any(np.abs(phi) <= band, axis=1)
    both = np.any(phi > 0, axis=1) & np.any(phi < 0, axis=1)
    target = np.where(near | both, level_max, level_min)
    lv = leaves.level.astype(np.int64)
    mark = np.where(lv < target, 1, np.where(lv > target, -1, 0)).astype(np.int8)
    return mark, float(np.min(np.abs(np.abs(phi) - band)))


def remesh(src, xyz, U, level_min, level_max, band=0.9, phi_index=None, nf=None):
    """Alternate marks (against the source field) and adaptation passes until
    nothing is marked or a pass changes nothing.  Returns (leaves, passes,
    margin)."""
    cur = OLeaves(src.dim, src.max_level, src.level, src.anchor)
    passes, margin = 0, np.inf
    for _ in range(2 * src.max_level + 2):
        mark, mg = mark_interface(src, xyz, U, cur, level_min, level_max, band, phi_index, nf)
        margin = min(margin, mg)
        if not mark.any():
            break
        nxt = adapt(cur, mark)
        if np.array_equal(nxt.level, cur.level) and np.array_equal(nxt.anchor, cur.anchor):
            break
        cur = nxt
        passes += 1
    return cur, passes, margin
