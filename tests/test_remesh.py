"""Remeshing (Sec. 4, "Refinement", "2:1 Balancing", "Intergrid transfers"):
the library's host calls against the brute-force oracle, and the oracle
pinned by hand-worked examples, the oracle mesh's own balance validation,
exactness of the Q1 interpolation and the conservation of the phi integral
under refinement.  No GPU."""
import numpy as np
import pytest

from oracle import remesh as R
from oracle.oracle import OracleMesh
from paper_1912_12453_gb300 import chns, workloads as W


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1912_12453_gb300 import build
    build.build()
    chns.lib()


def _same(a, b):
    return a.n == b.n and np.array_equal(a.level, b.level) and np.array_equal(a.anchor, b.anchor)


def _find(leaves, level, anchor):
    hit = np.nonzero((leaves.level == level) & np.all(leaves.anchor == np.asarray(anchor), axis=1))[0]
    assert hit.size == 1
    return int(hit[0])


# ---------------------------------------------------------------- adaptation

def test_worked_example_2d():
    """Quadtree of resolution 2^4, four level-1 leaves (size 8).
    1) Split the leaf at the origin: 3 + 4 = 7 leaves, no balance work.
    2) Split its child at (4, 4) (size 4): four level-3 leaves fill [4, 8]^2.
       They touch the point (8, 8), a corner of the three other level-1 leaves,
       two levels coarser: the balance splits all three, 4 + 3 + 12 = 19.
    3) Merge the four level-3 leaves: 16 level-2 leaves (the balance splits
       stay)."""
    for adapt in (chns.leaves_adapt, R.adapt):
        L0 = chns.Leaves(2, 4, [1, 1, 1, 1], [[0, 0], [8, 0], [0, 8], [8, 8]])
        A = adapt(L0, np.array([1, 0, 0, 0], np.int8))
        assert A.n == 7 and sorted(A.level.tolist()) == [1, 1, 1, 2, 2, 2, 2]
        m = np.zeros(A.n, np.int8)
        m[_find(A, 2, (4, 4))] = 1
        B = adapt(A, m)
        assert B.n == 19 and np.bincount(B.level, minlength=4).tolist() == [0, 0, 15, 4]
        C = adapt(B, np.where(B.level == 3, -1, 0).astype(np.int8))
        assert C.n == 16 and set(C.level.tolist()) == {2}
        # 16 leaves of level 2 in Morton order are the uniform level-2 grid
        U = W.uniform_leaves(2, 2)
        assert np.array_equal(C.anchor, U.anchor.astype(np.uint32) << 2)


def test_worked_example_3d():
    """Octree of resolution 2^3, eight level-1 leaves (size 4).  Split the
    leaf at the origin, then its child at (2, 2, 2): eight level-3 leaves fill
    [2, 4]^3 and touch the box centre, a corner of the seven other level-1
    leaves: all seven split.  8 + 7 + 56 = 71 leaves."""
    U1 = W.uniform_leaves(3, 1)
    for adapt in (chns.leaves_adapt, R.adapt):
        L0 = chns.Leaves(3, 3, U1.level, U1.anchor.astype(np.uint32) << 2)
        m = np.zeros(8, np.int8)
        m[_find(L0, 1, (0, 0, 0))] = 1
        A = adapt(L0, m)
        assert A.n == 15
        m = np.zeros(A.n, np.int8)
        m[_find(A, 2, (2, 2, 2))] = 1
        B = adapt(A, m)
        assert B.n == 71 and np.bincount(B.level, minlength=4).tolist() == [0, 0, 63, 8]


def test_merge_needs_the_whole_family():
    """-1 on three of four siblings merges nothing; on all four it merges."""
    U = W.uniform_leaves(2, 2)
    L0 = chns.Leaves(2, 2, U.level, U.anchor)
    fam = [_find(L0, 2, a) for a in [(0, 0), (1, 0), (0, 1), (1, 1)]]
    for adapt in (chns.leaves_adapt, R.adapt):
        m = np.zeros(16, np.int8)
        m[fam[:3]] = -1
        assert _same(adapt(L0, m), L0)
        m[fam[3]] = -1
        A = adapt(L0, m)
        assert A.n == 13 and A.level[0] == 1
        # marks at the limits are ignored: +1 at max_level, -1 at level 0
        assert _same(adapt(L0, np.ones(16, np.int8)), L0)
        root = chns.Leaves(2, 2, [0], [[0, 0]])
        assert _same(adapt(root, np.array([-1], np.int8)), root)


def _random_marks(leaves, seed, p_split=0.15, p_merge=0.5):
    rng = np.random.default_rng(seed)
    u = rng.uniform(size=leaves.n)
    return np.where(u < p_split, 1, np.where(u > 1 - p_merge, -1, 0)).astype(np.int8)


@pytest.mark.parametrize("dim,base,top,passes", [(2, 3, 7, 4), (3, 2, 5, 2)])
def test_adapt_matches_the_oracle(dim, base, top, passes):
    """Seeded random marks on a band mesh, several passes: the library's
    leaf lists equal the oracle's exactly; every result is accepted by the
    oracle mesh (its own balance check) and is minimal: merging any family the
    balance created breaks the balance."""
    sp = [W.Sphere((0.45, 0.55, 0.5)[:dim], 0.22)]
    L = W.band_leaves(dim, base, top - 1, sp, 0.03)
    cur = chns.Leaves(dim, top, L.level, L.anchor.astype(np.uint32) << 1)
    for k in range(passes):
        m = _random_marks(cur, 100 + k)
        lib = chns.leaves_adapt(cur, m)
        ora = R.adapt(R.OLeaves(dim, top, cur.level, cur.anchor), m)
        assert _same(lib, ora), (dim, k)
        assert R.is_balanced(ora)
        OracleMesh(ora)  # raises if the oracle's validation rejects the balance
        _check_minimal(R.apply_marks(cur, m), ora)
        cur = lib


def _check_minimal(marked, bal):
    """Every family of ``bal`` that is finer than the marked tree there
    exists only because merging it would break the balance: some leaf that
    touches the parent's closed box is two or more levels finer than it."""
    dim, ml = bal.dim, bal.max_level
    octs = R._octs(bal)
    have = set(octs)
    mk = set(R._octs(marked))
    a = bal.anchor.astype(np.int64)
    s = np.int64(1) << (ml - bal.level.astype(np.int64))
    seen = set()
    for o in octs:
        if o[0] == 0:
            continue
        p = R._parent(o, dim, ml)
        if p in seen:
            continue
        seen.add(p)
        fam = R._children(p, dim, ml)
        if not all(f in have for f in fam) or any(f in mk for f in fam):
            continue  # not a complete family, or one the marks asked for
        plo = np.asarray(p[1], dtype=np.int64)
        phi_ = plo + (np.int64(1) << (ml - p[0]))
        touch = np.all((a <= phi_) & (plo <= a + s[:, None]), axis=1)
        assert np.any(touch & (bal.level.astype(np.int64) >= p[0] + 2)), p


def test_adapt_rejects_bad_input():
    with pytest.raises(chns.ChnsError, match="CHNS_ERR_MESH"):
        chns.leaves_adapt(chns.Leaves(2, 2, [1, 1, 1, 1], [[2, 0], [0, 0], [0, 2], [2, 2]]))
    with pytest.raises(chns.ChnsError, match="CHNS_ERR_MESH"):
        chns.leaves_adapt(chns.Leaves(2, 2, [1, 1, 1], [[0, 0], [2, 0], [0, 2]]))
    with pytest.raises(ValueError):
        chns.leaves_adapt(chns.Leaves(2, 2, [0], [[0, 0]]), np.zeros(2, np.int8))


# ---------------------------------------------------------------- transfer

def _hanging_mesh(dim):
    sp = [W.Sphere((0.4, 0.6, 0.5)[:dim], 0.2)]
    return W.band_leaves(dim, 2, 5 if dim == 2 else 4, sp, 0.03)


def _q1_field(xyz, max_level, nf, dim):
    """A field in Q1 on every leaf: affine plus x y (2D) / x y z terms; these
    are also linear along every edge and face diagonal-free, so hanging-node
    means reproduce them."""
    x = xyz.astype(np.float64) / (1 << max_level)
    U = np.zeros((xyz.shape[0], nf))
    for k in range(nf):
        c = 0.3 * (k + 1)
        f = 1.0 + c * x[:, 0] - 0.7 * x[:, 1] + (0.5 + k) * x[:, 0] * x[:, 1]
        if dim == 3:
            f += 0.25 * x[:, 2] - (1.5 - 0.1 * k) * x[:, 0] * x[:, 1] * x[:, 2] + 0.4 * x[:, 1] * x[:, 2]
        U[:, k] = f
    return U


@pytest.mark.parametrize("dim", [2, 3])
def test_transfer_reproduces_q1_fields(dim):
    """Oracle and library: a field in Q1 on each leaf (hanging constraints
    included) is reproduced exactly at arbitrary points."""
    L = _hanging_mesh(dim)
    om = OracleMesh(L)
    assert om.n_hanging > 0
    nf = dim + 3
    U = _q1_field(om.coords_int, L.max_level, nf, dim)
    rng = np.random.default_rng(5)
    pts = rng.integers(0, (1 << L.max_level) + 1, size=(300, dim))
    exact = _q1_field(pts, L.max_level, nf, dim)
    lib = chns.leaves_transfer(L, om.coords_int, U, pts, nf)
    ora = R.transfer(L, om.coords_int, U, pts, nf)
    assert np.max(np.abs(lib - exact)) < 1e-13
    assert np.max(np.abs(ora - exact)) < 1e-13


@pytest.mark.parametrize("dim", [2, 3])
def test_transfer_matches_the_oracle(dim):
    """A random nodal field (not in Q1 globally) at random points and at the
    nodes of an adapted mesh: library and oracle agree to rounding."""
    L = _hanging_mesh(dim)
    om = OracleMesh(L)
    nf = dim + 3
    U = np.random.default_rng(9).uniform(-1, 1, size=(om.n_nodes, nf))
    perm = np.random.default_rng(10).permutation(om.n_nodes)   # any node order works
    xyz, Up = om.coords_int[perm], U[perm]
    new = R.adapt(L, _random_marks(L, 11, 0.3, 0.3))
    pts = np.concatenate([OracleMesh(new).coords_int,
                          np.random.default_rng(12).integers(0, (1 << L.max_level) + 1, size=(200, dim))])
    lib = chns.leaves_transfer(L, xyz, Up, pts, nf)
    ora = R.transfer(L, xyz, Up, pts, nf)
    assert np.max(np.abs(lib - ora)) < 1e-14
    # at the source nodes the transfer is the identity, exactly
    same = chns.leaves_transfer(L, xyz, Up, om.coords_int, nf)
    assert np.array_equal(same, U)


@pytest.mark.parametrize("dim", [2, 3])
def test_refinement_conserves_phi_and_coarsening_round_trips(dim):
    """Refinement only: the transferred field is the same piecewise-Q1
    function, so the phi integral (2^d Gauss rule, exact for Q1) is unchanged
    to rounding.  Coarsening back then returns the original nodal values
    (parents' corners are nodes of the children).  A coarsening of a field
    that is not Q1 on the parent changes the integral (the mass defect the
    paper notes for coarsening)."""
    L = _hanging_mesh(dim)
    om = OracleMesh(L)
    nf = dim + 3
    params = W.Params(dim, 1e-3, 0.05, 10.0, 1.0, 20.0, 1.0, 0.1, 0.1)
    rng = np.random.default_rng(21)
    U = rng.uniform(-1, 1, size=(om.n_nodes, nf))
    fine = chns.leaves_adapt(L, np.where(L.level < L.max_level, 1, 0).astype(np.int8))
    of = OracleMesh(fine)
    Uf = chns.leaves_transfer(L, om.coords_int, U, of.coords_int, nf)
    m0 = om.energy_mass(params, U.reshape(-1))[1]
    m1 = of.energy_mass(params, Uf.reshape(-1))[1]
    assert abs(m1 - m0) <= 1e-13 * max(1.0, abs(m0))
    # back: merge every family of the refined leaves that was split above
    back = chns.leaves_adapt(fine, np.where(np.isin(R_keys(fine), R_child_keys(L, fine)), -1, 0).astype(np.int8))
    assert _same(back, chns.Leaves(dim, L.max_level, L.level, L.anchor))
    Ub = chns.leaves_transfer(fine, of.coords_int, Uf, om.coords_int, nf)
    assert np.array_equal(Ub, U)
    # coarsening a random (non-Q1) fine field changes the phi integral
    Ur = rng.uniform(-1, 1, size=(of.n_nodes, nf))
    Uc = chns.leaves_transfer(fine, of.coords_int, Ur, om.coords_int, nf)
    mr = of.energy_mass(params, Ur.reshape(-1))[1]
    mc = om.energy_mass(params, Uc.reshape(-1))[1]
    assert abs(mc - mr) > 1e-6


def R_keys(leaves):
    return np.array([R.morton_key(a, leaves.dim, leaves.max_level) * 64 + int(l)
                     for l, a in zip(leaves.level, leaves.anchor)])


def R_child_keys(coarse, fine):
    """Keys of the fine leaves that are children of a split coarse leaf."""
    split = {tuple(int(x) for x in a) + (int(l),) for l, a in zip(coarse.level, coarse.anchor)
             if l < coarse.max_level}
    out = []
    for l, a in zip(fine.level, fine.anchor):
        p = R._parent((int(l), tuple(int(x) for x in a)), fine.dim, fine.max_level)
        if p[1] + (p[0],) in split:
            out.append(R.morton_key(a, fine.dim, fine.max_level) * 64 + int(l))
    return np.array(out)


def test_transfer_errors():
    L = _hanging_mesh(2)
    om = OracleMesh(L)
    U = np.zeros((om.n_nodes, 5))
    with pytest.raises(chns.ChnsError, match="CHNS_ERR_ARG"):
        chns.leaves_transfer(L, om.coords_int, U, np.array([[0, (1 << L.max_level) + 1]]))
    with pytest.raises(chns.ChnsError, match="CHNS_ERR_MESH"):   # a node missing from the list
        chns.leaves_transfer(L, om.coords_int[1:], U[1:], om.coords_int[:1])
    with pytest.raises(ValueError):
        chns.leaves_transfer(L, om.coords_int, U[:-1], om.coords_int[:1])


# ---------------------------------------------------------------- remeshing

def _moved_bubble(dim):
    """A band mesh around a bubble, and on its nodes the phi of the bubble
    moved by 3/32 (the state the next remesh sees)."""
    Cn = 0.02
    sp0 = [W.Sphere((0.5, 0.35, 0.5)[:dim], 0.18)]
    base, top = (3, 7) if dim == 2 else (2, 5)
    L = W.band_leaves(dim, base, top, sp0, Cn)
    om = OracleMesh(L)
    x = om.coords
    sp1 = [W.Sphere((0.5, 0.35 + 3 / 32, 0.5)[:dim], 0.18)]
    U = np.zeros((om.n_nodes, dim + 3))
    U[:, dim + 1] = W.phi_profile(x, sp1, Cn, True)
    U[:, 0] = 0.1 * x[:, 1]
    return L, om, U, base, top


@pytest.mark.parametrize("dim", [2, 3])
def test_remesh_matches_the_oracle(dim):
    """Remesh around the moved interface: identical leaf lists and pass counts,
    the comparisons of |phi| with the band decided with room to spare, every
    leaf whose corners see the interface at the finest level, and the new
    state the oracle's transfer of the old one."""
    L, om, U, base, top = _moved_bubble(dim)
    lib, passes = chns.leaves_remesh(L, om.coords_int, U, base, top)
    ora, opasses, margin = R.remesh(L, om.coords_int, U, base, top)
    assert margin > 1e-9
    assert _same(lib, ora) and passes == opasses and passes >= 1
    assert not _same(lib, L)
    on = OracleMesh(ora)
    # no leaf is left below its target; a leaf left above it is one whose
    # family cannot merge (not all leaves marked -1, or the merged parent
    # would touch a leaf two levels finer)
    m, _ = R.mark_interface(L, om.coords_int, U, ora, base, top)
    assert not (m > 0).any() and (m < 0).any()
    octs = R._octs(ora)
    where = {o: i for i, o in enumerate(octs)}
    a = ora.anchor.astype(np.int64)
    s = np.int64(1) << (ora.max_level - ora.level.astype(np.int64))
    for i in np.nonzero(m < 0)[0]:
        p = R._parent(octs[i], dim, ora.max_level)
        fam = R._children(p, dim, ora.max_level)
        if all(f in where and m[where[f]] < 0 for f in fam):
            plo = np.asarray(p[1], dtype=np.int64)
            phi_ = plo + (np.int64(1) << (ora.max_level - p[0]))
            touch = np.all((a <= phi_) & (plo <= a + s[:, None]), axis=1)
            assert np.any(touch & (ora.level.astype(np.int64) >= p[0] + 2))
    phi = R.transfer(L, om.coords_int, U, R.leaf_corners(ora))[:, dim + 1].reshape(ora.n, -1)
    near = np.any(np.abs(phi) <= 0.9, axis=1) | (np.any(phi > 0, axis=1) & np.any(phi < 0, axis=1))
    assert np.all(ora.level[near] == top)
    Un = chns.leaves_transfer(L, om.coords_int, U, on.coords_int)
    assert np.max(np.abs(Un - R.transfer(L, om.coords_int, U, on.coords_int))) < 1e-14


def test_remesh_marks_match_the_oracle():
    L, om, U, base, top = _moved_bubble(2)
    lib = chns.leaves_mark_interface(L, om.coords_int, U, L, base, top)
    ora, _ = R.mark_interface(L, om.coords_int, U, L, base, top)
    assert np.array_equal(lib, ora) and (lib == 1).any() and (lib == -1).any()
    Un = U.copy()
    Un[3, 3] = np.nan
    with pytest.raises(chns.ChnsError, match="CHNS_ERR_NONFINITE"):
        chns.leaves_mark_interface(L, om.coords_int, Un, L, base, base)


def test_remesh_of_a_settled_mesh_changes_nothing():
    """The band mesh of the generator, with the phi it was built for: the
    interface leaves are already at the finest level; remeshing with
    level_min at the base level only coarsens leaves the generator kept finer
    than the corner test needs, and a second remesh is a fixed point."""
    L, om, U, base, top = _moved_bubble(2)
    a, _ = chns.leaves_remesh(L, om.coords_int, U, base, top)
    oa = OracleMesh(a)
    Ua = chns.leaves_transfer(L, om.coords_int, U, oa.coords_int)
    b, passes = chns.leaves_remesh(a, oa.coords_int, Ua, base, top)
    assert passes == 0 and _same(a, b)


def test_hand_worked_remesh_library():
    """The library on the hand-worked case of the oracle pins: phi = x - 0.3
    on a uniform level-2 quadtree (resolution 2^4), band 0.1, levels 1..3:
    marks +1 on the columns x < 1/2 and -1 on the others; remeshing gives 32
    level-3 leaves on the left half and 8 level-2 leaves on the right, in one
    pass."""
    U2 = W.uniform_leaves(2, 2)
    L = chns.Leaves(2, 4, U2.level, U2.anchor.astype(np.uint32) << 2)
    om = OracleMesh(L)
    U = np.zeros((om.n_nodes, 5))
    U[:, 3] = om.coords_int[:, 0] / 16.0 - 0.3
    mark = chns.leaves_mark_interface(L, om.coords_int, U, L, 1, 3, 0.1)
    left = L.anchor[:, 0] < 8
    assert np.all(mark[left] == 1) and np.all(mark[~left] == -1)
    new, passes = chns.leaves_remesh(L, om.coords_int, U, 1, 3, 0.1)
    assert passes == 1 and new.n == 40
    assert np.all(new.level[new.anchor[:, 0] < 8] == 3) and np.all(new.level[new.anchor[:, 0] >= 8] == 2)
    U[:, 3] -= 0.02   # |phi| = 0.07 at x = 1/4: inside a band of 0.1, outside one of 0.06
    first = L.anchor[:, 0] < 4
    assert np.all(chns.leaves_mark_interface(L, om.coords_int, U, L, 1, 3, 0.1)[first] == 1)
    mark = chns.leaves_mark_interface(L, om.coords_int, U, L, 1, 3, 0.06)
    assert np.all(mark[first] == -1) and np.all(mark[left & ~first] == 1)


@pytest.mark.parametrize("seed", range(12))
def test_random_trees_match_the_oracle(seed):
    """Seeded random trees (2D and 3D, root-only to level 6, several
    adaptation passes with random split / merge rates), then a remesh around
    a random bubble with random level bounds, and a transfer at random
    points: the library equals the oracle (leaf lists, pass counts exactly;
    values to rounding)."""
    rng = np.random.default_rng(1000 + seed)
    dim = 3 if seed % 3 == 0 else 2
    top = int(rng.integers(3, 7 if dim == 2 else 5))
    base = int(rng.integers(0, top))
    if base == 0:
        cur = chns.Leaves(dim, top, [0], [[0] * dim])
    else:
        U = W.uniform_leaves(dim, base)
        cur = chns.Leaves(dim, top, U.level, U.anchor.astype(np.uint32) << (top - base))
    for _ in range(int(rng.integers(1, 5))):
        u = rng.uniform(size=cur.n)
        m = np.where(u < rng.uniform(0, 0.5), 1, np.where(u > 1 - rng.uniform(0, 0.9), -1, 0)).astype(np.int8)
        lib = chns.leaves_adapt(cur, m)
        ora = R.adapt(R.OLeaves(dim, top, cur.level, cur.anchor), m)
        assert _same(lib, ora)
        cur = lib
        if cur.n > 2500:
            break
    om = OracleMesh(cur)
    c, r, Cn = rng.uniform(0.2, 0.8, size=dim), rng.uniform(0.1, 0.3), rng.uniform(0.01, 0.08)
    U = np.zeros((om.n_nodes, dim + 3))
    U[:, dim + 1] = W.phi_profile(om.coords, [W.Sphere(tuple(c), r)], Cn, bool(seed % 2))
    lmin = int(rng.integers(0, top))
    lmax = int(rng.integers(lmin, top + 1))
    lib, p1 = chns.leaves_remesh(cur, om.coords_int, U, lmin, lmax)
    ora, p2, margin = R.remesh(R.OLeaves(dim, top, cur.level, cur.anchor), om.coords_int, U, lmin, lmax)
    if margin > 1e-12:
        assert _same(lib, ora) and p1 == p2
    pts = rng.integers(0, (1 << top) + 1, size=(40, dim))
    assert np.max(np.abs(chns.leaves_transfer(cur, om.coords_int, U, pts) - R.transfer(cur, om.coords_int, U, pts))) < 1e-13
