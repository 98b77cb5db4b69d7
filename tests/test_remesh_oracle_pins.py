"""Pins of the remeshing oracle (oracle/remesh.py) against what the paper and
the mathematics fix, independent of the library: hand-worked adaptations and
a hand-worked remesh, the oracle mesh's separate C++ balance validation,
refinement and minimality of the balanced tree, exact reproduction of Q1
fields through hanging constraints, conservation of the phi integral under
refinement, and the round trip refine -> coarsen.  (Sec. 4, "Refinement",
"2:1 Balancing", "Intergrid transfers".)"""
import numpy as np
import pytest

from oracle import remesh as R
from oracle.oracle import OracleMesh
from paper_1912_12453_gb300 import workloads as W


def _uniform(dim, level, max_level):
    U = W.uniform_leaves(dim, level)
    return R.OLeaves(dim, max_level, U.level, U.anchor.astype(np.uint32) << (max_level - level))


def _idx(leaves, level, anchor):
    hit = [i for i, o in enumerate(R._octs(leaves)) if o == (level, tuple(anchor))]
    assert len(hit) == 1
    return hit[0]


def test_hand_worked_adaptation_2d():
    """Resolution 2^4, four level-1 leaves.  Split (0,0): 7 leaves.  Split
    its child (4,4): the four level-3 leaves touch (8,8), a corner of the three
    other level-1 leaves, which the balance splits: 4 + 3 + 12 = 19.  Merging
    the level-3 family back gives the uniform level-2 grid, in Morton order."""
    L0 = _uniform(2, 1, 4)
    A = R.adapt(L0, np.array([1 if o == (1, (0, 0)) else 0 for o in R._octs(L0)], np.int8))
    assert A.n == 7
    m = np.zeros(A.n, np.int8)
    m[_idx(A, 2, (4, 4))] = 1
    B = R.adapt(A, m)
    assert B.n == 19 and np.bincount(B.level, minlength=4).tolist() == [0, 0, 15, 4]
    C = R.adapt(B, np.where(B.level == 3, -1, 0).astype(np.int8))
    U = _uniform(2, 2, 4)
    assert np.array_equal(C.level, U.level) and np.array_equal(C.anchor, U.anchor)


def test_hand_worked_adaptation_3d():
    """Resolution 2^3, eight level-1 leaves.  Split (0,0,0), then its child
    (2,2,2): its eight level-3 leaves touch the box centre, a corner of the
    seven other level-1 leaves, which all split: 8 + 7 + 56 = 71."""
    L0 = _uniform(3, 1, 3)
    m = np.zeros(8, np.int8)
    m[_idx(L0, 1, (0, 0, 0))] = 1
    A = R.adapt(L0, m)
    assert A.n == 15
    m = np.zeros(A.n, np.int8)
    m[_idx(A, 2, (2, 2, 2))] = 1
    B = R.adapt(A, m)
    assert B.n == 71 and np.bincount(B.level, minlength=4).tolist() == [0, 0, 63, 8]


def test_no_balance_work_without_contact():
    """Split (0,0) of four level-1 leaves, then its child at the origin: the
    level-3 leaves fill [0, 4]^2 and touch only level-2 leaves, so the balance
    adds nothing: 3 + 3 + 4 = 10 leaves (a pin against over-refinement)."""
    L0 = _uniform(2, 1, 4)
    A = R.adapt(L0, np.array([1 if o == (1, (0, 0)) else 0 for o in R._octs(L0)], np.int8))
    m = np.zeros(A.n, np.int8)
    m[_idx(A, 2, (0, 0))] = 1
    B = R.adapt(A, m)
    assert B.n == 10 and np.bincount(B.level, minlength=4).tolist() == [0, 3, 3, 4]


def test_merge_rules():
    L0 = _uniform(2, 2, 2)
    fam = [_idx(L0, 2, a) for a in [(0, 0), (1, 0), (0, 1), (1, 1)]]
    m = np.zeros(16, np.int8)
    m[fam[:3]] = -1
    B = R.adapt(L0, m)
    assert np.array_equal(B.level, L0.level) and np.array_equal(B.anchor, L0.anchor)
    m[fam[3]] = -1
    A = R.adapt(L0, m)
    assert A.n == 13 and int(A.level[0]) == 1 and tuple(A.anchor[0]) == (0, 0)
    # marks at the limits are ignored
    assert R.adapt(L0, np.ones(16, np.int8)).n == 16
    root = R.OLeaves(2, 2, [0], [[0, 0]])
    assert R.adapt(root, np.array([-1], np.int8)).n == 1


@pytest.mark.parametrize("dim,base,top", [(2, 3, 6), (3, 2, 4)])
def test_balanced_refinement_is_valid_and_minimal(dim, base, top):
    """Random marks on a band mesh: the result tiles the box, refines the
    marked tree, passes the oracle mesh's own balance check, and every family
    finer than the marked tree could not merge without breaking the balance."""
    sp = [W.Sphere((0.45, 0.55, 0.5)[:dim], 0.22)]
    Lw = W.band_leaves(dim, base, top - 1, sp, 0.03)
    cur = R.OLeaves(dim, top, Lw.level, Lw.anchor.astype(np.uint32) << 1)
    rng = np.random.default_rng(7)
    for _ in range(2):
        u = rng.uniform(size=cur.n)
        mark = np.where(u < 0.15, 1, np.where(u > 0.5, -1, 0)).astype(np.int8)
        marked = R.apply_marks(cur, mark)
        bal = R.adapt(cur, mark)
        s = 1 << (top - bal.level.astype(np.int64))
        assert int((s.astype(np.float64) ** dim).sum()) == (1 << (top * dim))   # tiles the box
        keys = [R.morton_key(a, dim, top) for a in bal.anchor]
        assert keys == sorted(keys)
        OracleMesh(bal)
        # refines the marked tree: each balanced leaf lies in a marked leaf of level <= its own
        ma = marked.anchor.astype(np.int64)
        ms = np.int64(1) << (top - marked.level.astype(np.int64))
        for a, l in zip(bal.anchor.astype(np.int64), bal.level.astype(np.int64)):
            inside = np.all((ma <= a) & (a < ma + ms[:, None]), axis=1)
            assert inside.sum() == 1 and marked.level[np.argmax(inside)] <= l
        # minimal
        octs = R._octs(bal)
        have, mk = set(octs), set(R._octs(marked))
        a_all = bal.anchor.astype(np.int64)
        seen = set()
        for o in octs:
            if o[0] == 0:
                continue
            p = R._parent(o, dim, top)
            if p in seen:
                continue
            seen.add(p)
            fam = R._children(p, dim, top)
            if not all(f in have for f in fam) or any(f in mk for f in fam):
                continue
            plo = np.asarray(p[1], dtype=np.int64)
            phi_ = plo + (np.int64(1) << (top - p[0]))
            touch = np.all((a_all <= phi_) & (plo <= a_all + s[:, None]), axis=1)
            assert np.any(touch & (bal.level.astype(np.int64) >= p[0] + 2)), p
        cur = bal


def _q1(xyz, max_level, nf, dim):
    x = xyz.astype(np.float64) / (1 << max_level)
    U = np.zeros((xyz.shape[0], nf))
    for k in range(nf):
        f = 1.0 + 0.3 * (k + 1) * x[:, 0] - 0.7 * x[:, 1] + (0.5 + k) * x[:, 0] * x[:, 1]
        if dim == 3:
            f += 0.25 * x[:, 2] - (1.5 - 0.1 * k) * x[:, 0] * x[:, 1] * x[:, 2] + 0.4 * x[:, 1] * x[:, 2]
        U[:, k] = f
    return U


@pytest.mark.parametrize("dim", [2, 3])
def test_transfer_reproduces_q1_fields(dim):
    sp = [W.Sphere((0.4, 0.6, 0.5)[:dim], 0.2)]
    L = W.band_leaves(dim, 2, 5 if dim == 2 else 4, sp, 0.03)
    om = OracleMesh(L)
    assert om.n_hanging > 0
    nf = dim + 3
    U = _q1(om.coords_int, L.max_level, nf, dim)
    pts = np.random.default_rng(5).integers(0, (1 << L.max_level) + 1, size=(300, dim))
    assert np.max(np.abs(R.transfer(L, om.coords_int, U, pts, nf) - _q1(pts, L.max_level, nf, dim))) < 1e-13
    # at the nodes themselves: the identity, exactly
    assert np.array_equal(R.transfer(L, om.coords_int, U, om.coords_int, nf), U)


@pytest.mark.parametrize("dim", [2, 3])
def test_refinement_conserves_phi_and_round_trips(dim):
    sp = [W.Sphere((0.4, 0.6, 0.5)[:dim], 0.2)]
    L = W.band_leaves(dim, 2, 5 if dim == 2 else 4, sp, 0.03)
    om = OracleMesh(L)
    nf = dim + 3
    params = W.Params(dim, 1e-3, 0.05, 10.0, 1.0, 20.0, 1.0, 0.1, 0.1)
    U = np.random.default_rng(21).uniform(-1, 1, size=(om.n_nodes, nf))
    fine = R.adapt(L, np.where(L.level < L.max_level, 1, 0).astype(np.int8))
    of = OracleMesh(fine)
    Uf = R.transfer(L, om.coords_int, U, of.coords_int, nf)
    m0 = om.energy_mass(params, U.reshape(-1))[1]
    m1 = of.energy_mass(params, Uf.reshape(-1))[1]
    assert abs(m1 - m0) <= 1e-13 * max(1.0, abs(m0))
    Ub = R.transfer(fine, of.coords_int, Uf, om.coords_int, nf)
    assert np.array_equal(Ub, U)


def _linear_interface():
    """Resolution 2^4, uniform level 2 (size 4), phi = x - 0.3 at the nodes."""
    L = _uniform(2, 2, 4)
    om = OracleMesh(L)
    U = np.zeros((om.n_nodes, 5))
    U[:, 3] = om.coords_int[:, 0] / 16.0 - 0.3
    return L, om, U


def test_hand_worked_marks():
    """phi = x - 0.3, band 0.1: the columns x in [0, 1/4] (phi = -0.05 at
    x = 1/4) and [1/4, 1/2] (sign change) meet the interface and aim at
    level 3 (+1); the columns x >= 1/2 (phi >= 0.2) aim at level 1 (-1)."""
    L, om, U = _linear_interface()
    mark, margin = R.mark_interface(L, om.coords_int, U, L, 1, 3, band=0.1)
    left = L.anchor[:, 0] < 8
    assert np.all(mark[left] == 1) and np.all(mark[~left] == -1)
    assert margin > 0.04
    # phi = x - 0.32: at x = 1/4 |phi| = 0.07, inside a band of 0.1 and
    # outside one of 0.06 (the first column then has phi < 0 at every corner)
    U[:, 3] -= 0.02
    first = L.anchor[:, 0] < 4
    mark, _ = R.mark_interface(L, om.coords_int, U, L, 1, 3, band=0.1)
    assert np.all(mark[first] == 1)
    mark, _ = R.mark_interface(L, om.coords_int, U, L, 1, 3, band=0.06)
    assert np.all(mark[first] == -1) and np.all(mark[left & ~first] == 1)


def test_hand_worked_remesh():
    """Same field, levels 1..3.  Pass 1 splits the 8 left leaves into 32
    level-3 leaves and merges the right half into two level-1 leaves, which
    the balance splits again (they touch level-3 leaves at x = 1/2): 32 + 8 =
    40.  Pass 2 marks the column x in [0, 1/8] for merging (phi <= -0.175)
    but its families reach into x in [1/8, 1/4], which stays; the right half
    would merge but the balance undoes it: nothing changes, one pass."""
    L, om, U = _linear_interface()
    new, passes, margin = R.remesh(L, om.coords_int, U, 1, 3, band=0.1)
    assert passes == 1 and new.n == 40
    assert np.bincount(new.level, minlength=4).tolist() == [0, 0, 8, 32]
    assert np.all(new.level[new.anchor[:, 0] < 8] == 3) and np.all(new.level[new.anchor[:, 0] >= 8] == 2)
