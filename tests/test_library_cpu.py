"""Host-side checks of the C ABI library (no GPU compute)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1912_12453_gb300 import chns, workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1912_12453_gb300 import build
    build.build()
    return chns.lib()


def _header_functions():
    src = open(os.path.join(ROOT, "include", "chns.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(chns_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol(L):
    names = _header_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(L, n), n
    assert sorted(chns.EXPORTS) == names


def test_abi_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors have the sizes and field offsets the C compiler gives."""
    import subprocess
    checks = {"chns_params": chns.Params, "chns_solver_opts": chns.SolverOpts,
              "chns_step_stats": chns.StepStats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "chns.h"', "int main(void){"]
    for cname, cls in checks.items():
        lines.append(f'printf("%zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("%zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0;}")
    src = tmp_path / "abi.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "abi"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    exp = []
    for cls in checks.values():
        exp.append(ctypes.sizeof(cls))
        exp.extend(getattr(cls, f).offset for f, _ in cls._fields_)
    assert out == exp


def _create(L, dim, lev, anc, max_level):
    h = ctypes.c_void_p()
    lev = np.ascontiguousarray(lev, dtype=np.uint8)
    anc = np.ascontiguousarray(anc, dtype=np.uint32)
    s = L.chns_mesh_create(dim, lev.shape[0], lev.ctypes.data, anc.ctypes.data, max_level, None, None,
                           ctypes.byref(h))
    return s, L.chns_last_error().decode()


def test_invalid_arguments_rejected_on_host(L):
    s, msg = _create(L, 4, [1], [[0, 0]], 1)
    assert s == 1 and "dim" in msg
    assert L.chns_mesh_info(None, None, None, None, None) == 1
    # an empty leaf list, and a leaf level beyond max_level
    s, msg = _create(L, 2, np.zeros(0, dtype=np.uint8), np.zeros((0, 2), dtype=np.uint32), 2)
    assert s == 1 and "no leaves" in msg
    s, msg = _create(L, 2, [3], [[0, 0]], 2)
    assert s == 2
    assert L.chns_mesh_check(None) == 1
    assert L.chns_mesh_jacvec_schedule(None, 0, None, None) == 1


def test_unsorted_leaves_rejected(L):
    lv = W.uniform_leaves(2, 2)
    anc = lv.anchor[::-1].copy()
    s, msg = _create(L, 2, lv.level[::-1], anc, 2)
    assert s == 2 and "Morton" in msg


def test_gap_rejected(L):
    lv = W.uniform_leaves(2, 2)
    s, msg = _create(L, 2, lv.level[:-1], lv.anchor[:-1], 2)
    assert s == 2


def test_unbalanced_rejected(L):
    # a level-1 quadrant next to level-3 leaves (two levels apart)
    lev, anc = [], []
    for c in range(4):
        b = [(c >> a) & 1 for a in range(2)]
        if c == 0:
            for cc in range(4):
                b2 = [(cc >> a) & 1 for a in range(2)]
                if cc == 3:
                    for ccc in range(4):
                        b3 = [(ccc >> a) & 1 for a in range(2)]
                        lev.append(3)
                        anc.append([2 + b3[0], 2 + b3[1]])
                else:
                    lev.append(2)
                    anc.append([2 * b2[0], 2 * b2[1]])
        else:
            lev.append(1)
            anc.append([4 * b[0], 4 * b[1]])
    anc = np.array(anc, dtype=np.uint32)
    lev = np.array(lev, dtype=np.uint8)
    o = np.argsort(W.morton_keys(anc, 3), kind="stable")
    s, msg = _create(L, 2, lev[o], anc[o], 3)
    assert s == 2 and "balanced" in msg


def test_generated_octrees_are_balanced_and_sorted():
    for L_ in (W.band_leaves(3, 3, 6, [W.Sphere((0.5, 0.5, 0.3), 0.2)], 0.02),
               W.band_leaves(2, 3, 8, [W.Sphere((0.4, 0.6), 0.2)], 0.01)):
        keys = W.morton_keys(L_.anchor, L_.max_level)
        assert np.all(np.diff(keys.astype(np.int64)) > 0)
        vol = np.sum(1.0 / (1 << (L_.dim * L_.level.astype(np.int64))))
        assert abs(vol - 1.0) < 1e-12


def test_batched_workload_generator():
    """64 independent instances from one seed: both dimensions, levels 6-9 in
    2D and 5-7 in 3D, parameters in the stated ranges, every octree sorted,
    tiling the box and 2:1 balanced (checked by its own neighbour search)."""
    wls = W.batched_workloads(64)
    assert len(wls) == 64
    dims = [w.params.dim for w in wls]
    assert 0 < dims.count(2) < 64
    for w in wls:
        L = w.leaves
        top = int(L.level.max())
        assert (6 <= top <= 9) if L.dim == 2 else (5 <= top <= 7)
        assert 1e-3 <= w.params.rho_ratio <= 1.0 and 1e-2 <= w.params.eta_ratio <= 1.0
        assert 0.1 <= w.spheres[0].radius <= 0.25
        keys = W.morton_keys(L.anchor, L.max_level).astype(np.int64)
        assert np.all(np.diff(keys) > 0)
        vol = np.sum(1.0 / (1 << (L.dim * L.level.astype(np.int64))))
        assert abs(vol - 1.0) < 1e-12
    # 2:1 balance of the six smallest instances by brute force: the level of
    # every max-level cell next to a leaf's corners differs from the leaf's by
    # at most one
    import itertools
    for w in sorted(wls, key=lambda w: w.leaves.n)[:6]:
        L = w.leaves
        size = 1 << L.max_level
        lev = L.level.astype(np.int64)
        anc = L.anchor.astype(np.int64)
        lookup = {}
        for a, l in zip(anc, lev):
            s = 1 << (L.max_level - l)
            for off in itertools.product(range(s), repeat=L.dim):
                lookup[tuple(a + np.array(off))] = l
        assert len(lookup) == size ** L.dim
        for a, l in zip(anc, lev):
            s = 1 << (L.max_level - l)
            for off in itertools.product((-1, 0, s), repeat=L.dim):
                q = tuple(a + np.array(off))
                if all(0 <= x < size for x in q):
                    assert abs(lookup[q] - l) <= 1
