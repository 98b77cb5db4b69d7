"""The library's mesh builder on the CPU.

The host code of ``csrc/mesh.cpp`` (validation, node numbering, hanging-node
constraints, element and node colourings, gather lists) is built with host
stand-ins for its CUDA runtime calls (``tests/host/cuda_host_stub.cpp``) and
checked against the oracle mesh: the independent node set, the hanging nodes
and their parents, the wall nodes; the library's own validation (colours
with disjoint expanded footprints, exact gather lists) passes on every mesh,
including remeshed ones; unbalanced and untiled leaf lists are rejected.
No GPU."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import remesh as R
from oracle.oracle import OracleMesh
from paper_1912_12453_gb300 import chns, workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1912_12453_gb300", "csrc")


def _cuda_include():
    for base in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if base and os.path.exists(os.path.join(base, "include", "cuda_runtime.h")):
            return os.path.join(base, "include")
    return None


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    inc = _cuda_include()
    if shutil.which("g++") is None or inc is None:
        pytest.skip("g++ or the CUDA headers are missing")
    out = str(tmp_path_factory.mktemp("meshhost") / "mesh_host")
    cmd = ["g++", "-O2", "-std=c++17", "-pthread", "-I", os.path.join(ROOT, "include"), "-I", CSRC, "-I", inc,
           os.path.join(CSRC, "mesh.cpp"), os.path.join(ROOT, "tests", "host", "cuda_host_stub.cpp"),
           os.path.join(ROOT, "tests", "host", "mesh_host_main.cpp"), "-o", out]
    subprocess.check_call(cmd)
    return out


def _run(exe, leaves, tmp_path):
    src, dst = str(tmp_path / "leaves.bin"), str(tmp_path / "mesh.bin")
    with open(src, "wb") as f:
        f.write(np.int64(leaves.level.shape[0]).tobytes())
        f.write(np.int32(leaves.dim).tobytes())
        f.write(np.int32(leaves.max_level).tobytes())
        f.write(np.ascontiguousarray(leaves.level, np.uint8).tobytes())
        f.write(np.ascontiguousarray(leaves.anchor, np.uint32).tobytes())
    subprocess.check_call([exe, src, dst])
    raw = open(dst, "rb").read()
    st, val = np.frombuffer(raw[:8], np.int32)
    out = {"status": int(st), "validate": int(val)}
    if st != 0 or val != 0:
        return out
    dim, n = leaves.dim, leaves.level.shape[0]
    q = np.frombuffer(raw[8:], np.int64)
    n_nodes, n_hang, n_col, origin, n_wall = (int(x) for x in q[:5])
    k = 5
    xyz = q[k:k + n_nodes * dim].reshape(n_nodes, dim)
    k += n_nodes * dim
    nrec = int(q[k])
    k += 1
    rec = q[k:k + nrec].reshape(-1, 5 * dim)
    k += nrec
    cs = q[k:k + n_col + 1]
    hang = {}
    for r in rec:
        corner = tuple(int(v) for v in r[:dim])
        par = [tuple(int(v) for v in r[dim * (b + 1):dim * (b + 2)]) for b in range(4)]
        hang[corner] = tuple(sorted(p for p in par if p[0] >= 0))
    out.update(n_nodes=n_nodes, n_hang=n_hang, n_colours=n_col, origin=origin, n_wall=n_wall, xyz=xyz,
               hang=hang, colour_start=cs, n=n)
    return out


def _oracle_hanging(leaves, om):
    """corner coordinates -> sorted parent coordinates, from the oracle's P."""
    start, node, w = om.P()
    dim = leaves.dim
    nc = 1 << dim
    out = {}
    s = np.int64(1) << (leaves.max_level - leaves.level.astype(np.int64))
    for e in range(leaves.level.shape[0]):
        for c in range(nc):
            r = e * nc + c
            if start[r + 1] - start[r] <= 1:
                continue
            corner = tuple(int(leaves.anchor[e, a]) + (int(s[e]) if (c >> a) & 1 else 0) for a in range(dim))
            par = tuple(sorted(tuple(int(v) for v in om.coords_int[node[t]]) for t in range(start[r], start[r + 1])))
            assert set(w[start[r]:start[r + 1]]) <= {0.5, 0.25}
            out[corner] = par
    return out


def _meshes():
    cases = [("uniform2d", W.uniform_leaves(2, 4)), ("uniform3d", W.uniform_leaves(3, 3)),
             ("hang2", W.tiny_leaves(2, "hang")), ("hang3", W.tiny_leaves(3, "hang")),
             ("band2d", W.band_leaves(2, 3, 7, [W.Sphere((0.45, 0.55), 0.2)], 0.02)),
             ("band3d", W.band_leaves(3, 2, 5, [W.Sphere((0.45, 0.55, 0.5), 0.2)], 0.03))]
    for i, wl in enumerate(W.batched_workloads(64)):
        if wl.leaves.level.shape[0] < 20000:
            cases.append((f"batched{i}", wl.leaves))
        if len(cases) >= 8:
            break
    return cases


@pytest.mark.parametrize("name,leaves", _meshes(), ids=[c[0] for c in _meshes()])
def test_builder_matches_the_oracle_mesh(exe, tmp_path, name, leaves):
    got = _run(exe, leaves, tmp_path)
    assert got["status"] == 0 and got["validate"] == 0, got
    om = OracleMesh(leaves)
    assert got["n_nodes"] == om.n_nodes and got["n_hang"] == om.n_hanging
    assert {tuple(r) for r in got["xyz"].tolist()} == {tuple(r) for r in om.coords_int.tolist()}
    assert got["hang"] == _oracle_hanging(leaves, om)
    assert tuple(got["xyz"][got["origin"]]) == (0,) * leaves.dim
    assert got["n_wall"] == int(om.on_wall.sum())
    cs = got["colour_start"]
    assert cs[0] == 0 and cs[-1] == got["n"] and np.all(np.diff(cs) > 0)
    if len(set(leaves.level.tolist())) == 1:
        assert got["n_colours"] == 1 << leaves.dim


def test_builder_accepts_remeshed_and_adapted_leaves(exe, tmp_path):
    """Leaf lists produced by the library's remeshing are valid meshes for its
    builder (balanced, tiled, colourable) and agree with the oracle mesh."""
    sp0 = [W.Sphere((0.5, 0.35), 0.18)]
    L = W.band_leaves(2, 3, 7, sp0, 0.02)
    om = OracleMesh(L)
    U = np.zeros((om.n_nodes, 5))
    U[:, 3] = W.phi_profile(om.coords, [W.Sphere((0.5, 0.45), 0.18)], 0.02, True)
    new, passes = chns.leaves_remesh(L, om.coords_int, U, 3, 7)
    assert passes >= 1
    rng = np.random.default_rng(3)
    adapted = chns.leaves_adapt(new, rng.integers(-1, 2, size=new.n).astype(np.int8))
    for leaves in (new, adapted):
        got = _run(exe, leaves, tmp_path)
        assert got["status"] == 0 and got["validate"] == 0
        on = OracleMesh(leaves)
        assert got["n_nodes"] == on.n_nodes and got["n_hang"] == on.n_hanging
        assert got["hang"] == _oracle_hanging(leaves, on)


def test_builder_rejects_unbalanced_and_untiled_leaves(exe, tmp_path):
    # a level-3 family touching three level-1 leaves at the box centre
    octs = [(1, (4, 0)), (1, (0, 4)), (1, (4, 4)), (2, (0, 0)), (2, (2, 0)), (2, (0, 2))]
    octs += [(3, (2 + dx, 2 + dy)) for dx in (0, 1) for dy in (0, 1)]
    unbal = R._sorted(2, 3, octs)
    assert _run(exe, unbal, tmp_path)["status"] == 2
    # the same corner in 3D
    octs = [(1, (x, y, z)) for x in (0, 4) for y in (0, 4) for z in (0, 4) if (x, y, z) != (0, 0, 0)]
    octs += [(2, (x, y, z)) for x in (0, 2) for y in (0, 2) for z in (0, 2) if (x, y, z) != (2, 2, 2)]
    octs += [(3, (2 + dx, 2 + dy, 2 + dz)) for dx in (0, 1) for dy in (0, 1) for dz in (0, 1)]
    assert _run(exe, R._sorted(3, 3, octs), tmp_path)["status"] == 2
    # a missing leaf, and leaves out of Morton order
    U = W.uniform_leaves(2, 2)
    gap = chns.Leaves(2, 2, U.level[1:], U.anchor[1:])
    assert _run(exe, gap, tmp_path)["status"] == 2
    swapped = chns.Leaves(2, 2, U.level, U.anchor[[1, 0] + list(range(2, 16))])
    assert _run(exe, swapped, tmp_path)["status"] == 2


@pytest.mark.parametrize("seed", range(10))
def test_builder_on_random_balanced_trees(exe, tmp_path, seed):
    """Seeded random balanced trees (random split / merge passes from a
    uniform level, 2D and 3D): the builder's output agrees with the oracle
    mesh and passes the library's own validation."""
    rng = np.random.default_rng(2000 + seed)
    dim = 3 if seed % 3 == 0 else 2
    top = int(rng.integers(2, 7 if dim == 2 else 5))
    base = int(rng.integers(1, top + 1))
    U = W.uniform_leaves(dim, base)
    cur = chns.Leaves(dim, top, U.level, U.anchor.astype(np.uint32) << (top - base))
    for _ in range(int(rng.integers(0, 5))):
        u = rng.uniform(size=cur.n)
        m = np.where(u < rng.uniform(0, 0.4), 1, np.where(u > 1 - rng.uniform(0, 0.8), -1, 0)).astype(np.int8)
        cur = chns.leaves_adapt(cur, m)
        if cur.n > 3000:
            break
    got = _run(exe, cur, tmp_path)
    assert got["status"] == 0 and got["validate"] == 0
    om = OracleMesh(cur)
    assert got["n_nodes"] == om.n_nodes and got["n_hang"] == om.n_hanging
    assert {tuple(r) for r in got["xyz"].tolist()} == {tuple(r) for r in om.coords_int.tolist()}
    assert got["hang"] == _oracle_hanging(cur, om)


# ---------------------------------------------------------------- AddressSanitizer builds

def _asan_build(tmp_path_factory, name, sources):
    inc = _cuda_include()
    if shutil.which("g++") is None or inc is None:
        pytest.skip("g++ or the CUDA headers are missing")
    out = str(tmp_path_factory.mktemp("asan") / name)
    cmd = ["g++", "-O1", "-g", "-fsanitize=address", "-fno-omit-frame-pointer", "-std=c++17", "-pthread",
           "-I", os.path.join(ROOT, "include"), "-I", CSRC, "-I", inc] + sources + ["-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("no AddressSanitizer runtime: " + r.stderr[-200:])
    return out


@pytest.fixture(scope="module")
def asan_mesh(tmp_path_factory):
    return _asan_build(tmp_path_factory, "mesh_host_asan",
                       [os.path.join(CSRC, "mesh.cpp"), os.path.join(ROOT, "tests", "host", "cuda_host_stub.cpp"),
                        os.path.join(ROOT, "tests", "host", "mesh_host_main.cpp")])


@pytest.fixture(scope="module")
def asan_octree(tmp_path_factory):
    return _asan_build(tmp_path_factory, "octree_host_asan",
                       [os.path.join(CSRC, "mesh.cpp"), os.path.join(CSRC, "octree.cpp"),
                        os.path.join(ROOT, "tests", "host", "cuda_host_stub.cpp"),
                        os.path.join(ROOT, "tests", "host", "octree_host_main.cpp")])


def _asan_env():
    env = dict(os.environ)
    env["ASAN_OPTIONS"] = "detect_leaks=0:abort_on_error=0:exitcode=86"
    return env


def test_mesh_builder_under_address_sanitizer(asan_mesh, tmp_path):
    """The builder's host code reads and writes only inside its arrays on
    uniform, banded, batched and random adapted trees, and on rejected ones."""
    cases = [m for _, m in _meshes()]
    rng = np.random.default_rng(5)
    cur = chns.Leaves(3, 5, W.uniform_leaves(3, 2).level, W.uniform_leaves(3, 2).anchor.astype(np.uint32) << 3)
    for _ in range(3):
        cur = chns.leaves_adapt(cur, rng.integers(-1, 2, size=cur.n).astype(np.int8))
    cases.append(cur)
    octs = [(1, (4, 0)), (1, (0, 4)), (1, (4, 4)), (2, (0, 0)), (2, (2, 0)), (2, (0, 2))]
    octs += [(3, (2 + dx, 2 + dy)) for dx in (0, 1) for dy in (0, 1)]
    cases.append(R._sorted(2, 3, octs))
    for leaves in cases:
        src, dst = str(tmp_path / "l.bin"), str(tmp_path / "m.bin")
        with open(src, "wb") as f:
            f.write(np.int64(leaves.level.shape[0]).tobytes() + np.int32(leaves.dim).tobytes()
                    + np.int32(leaves.max_level).tobytes() + np.ascontiguousarray(leaves.level, np.uint8).tobytes()
                    + np.ascontiguousarray(leaves.anchor, np.uint32).tobytes())
        r = subprocess.run([asan_mesh, src, dst], capture_output=True, text=True, env=_asan_env())
        assert r.returncode == 0 and "AddressSanitizer" not in r.stderr, r.stderr[-2000:]


def _leaf_bytes(leaves):
    return (np.int64(leaves.level.shape[0]).tobytes() + np.int32(leaves.dim).tobytes()
            + np.int32(leaves.max_level).tobytes() + np.ascontiguousarray(leaves.level, np.uint8).tobytes()
            + np.ascontiguousarray(leaves.anchor, np.uint32).tobytes())


def test_remeshing_under_address_sanitizer(asan_octree, tmp_path):
    """The remeshing calls (adapt, remesh, transfer) built with
    AddressSanitizer stay inside their arrays and give the shared library's
    results (leaf lists bit for bit, values to rounding)."""
    src, dst = str(tmp_path / "i.bin"), str(tmp_path / "o.bin")

    def run(mode, payload):
        with open(src, "wb") as f:
            f.write(payload)
        r = subprocess.run([asan_octree, mode, src, dst], capture_output=True, text=True, env=_asan_env())
        assert r.returncode == 0 and "AddressSanitizer" not in r.stderr, r.stderr[-2000:]
        return open(dst, "rb").read()

    for dim, base, top in [(2, 3, 7), (3, 2, 5)]:
        sp = [W.Sphere((0.5, 0.35, 0.5)[:dim], 0.18)]
        L = W.band_leaves(dim, base, top, sp, 0.02 if dim == 2 else 0.03)
        om = OracleMesh(L)
        nf = dim + 3
        # adapt with random marks
        mark = np.random.default_rng(dim).integers(-1, 2, size=L.n).astype(np.int8)
        raw = run("adapt", _leaf_bytes(L) + mark.tobytes())
        st, m = np.frombuffer(raw[:4], np.int32)[0], int(np.frombuffer(raw[4:12], np.int64)[0])
        lib = chns.leaves_adapt(L, mark)
        assert st == 0 and m == lib.n
        assert np.array_equal(np.frombuffer(raw[12:12 + m], np.uint8), lib.level)
        assert np.array_equal(np.frombuffer(raw[12 + m:], np.uint32).reshape(-1, dim), lib.anchor)
        # remesh around a moved bubble
        U = np.zeros((om.n_nodes, nf))
        U[:, dim + 1] = W.phi_profile(om.coords, [W.Sphere((0.5, 0.45, 0.5)[:dim], 0.18)], 0.02, True)
        field = (np.int64(om.n_nodes).tobytes() + np.int32(nf).tobytes()
                 + np.ascontiguousarray(om.coords_int, np.int64).tobytes() + U.tobytes())
        raw = run("remesh", _leaf_bytes(L) + field + np.int32(base).tobytes() + np.int32(top).tobytes()
                  + np.float64(0.9).tobytes())
        st, m = np.frombuffer(raw[:4], np.int32)[0], int(np.frombuffer(raw[4:12], np.int64)[0])
        passes = int(np.frombuffer(raw[12:16], np.int32)[0])
        new, lp = chns.leaves_remesh(L, om.coords_int, U, base, top)
        assert st == 0 and m == new.n and passes == lp
        assert np.array_equal(np.frombuffer(raw[16:16 + m], np.uint8), new.level)
        # transfer to the new mesh's nodes and to the box corners
        pts = np.concatenate([OracleMesh(new).coords_int, np.zeros((1, dim), np.int64),
                              np.full((1, dim), 1 << L.max_level, np.int64)])
        raw = run("transfer", _leaf_bytes(L) + field + np.int64(pts.shape[0]).tobytes()
                  + np.ascontiguousarray(pts, np.int64).tobytes())
        assert np.frombuffer(raw[:4], np.int32)[0] == 0
        got = np.frombuffer(raw[4:], np.float64).reshape(-1, nf)
        # (the two builds may contract multiply-adds differently)
        assert np.max(np.abs(got - chns.leaves_transfer(L, om.coords_int, U, pts))) <= 1e-14
