"""Mutation test of the remeshing oracle's pins: one plausible mistake at a
time is planted in a copy of ``oracle/remesh.py`` (a strict contact test, a
wrong balance threshold, a wrong parent, merging on any sibling, swapped
shape functions, hanging constraints dropped, an "or" for the sign test, a
swapped target level, a miscounted pass, a transposed Morton key) and the
oracle-only pins (``tests/test_remesh_oracle_pins.py``) run on the copy;
every mistake must make a pin fail.  The repository itself is not changed."""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

M = [
 ("touch_strict", "t = np.all((lo[:, None, :] <= hi[None, :, :]) & (lo[None, :, :] <= hi[:, None, :]), axis=2)",
  "t = np.all((lo[:, None, :] < hi[None, :, :]) & (lo[None, :, :] < hi[:, None, :]), axis=2)"),
 ("balance_threshold", "bad = np.any(touching(leaves) & (lv[None, :] >= lv[:, None] + 2), axis=1)",
  "bad = np.any(touching(leaves) & (lv[None, :] >= lv[:, None] + 1), axis=1)"),
 ("parent_size", "ps = 1 << (max_level - l + 1)", "ps = 1 << (max_level - l)"),
 ("merge_any", "if all(f in where and int(mark[where[f]]) < 0 for f in fam):",
  "if any(f in where and int(mark[where[f]]) < 0 for f in fam):"),
 ("shape_swap", "N *= t[k] if (c >> k) & 1 else 1.0 - t[k]", "N *= 1.0 - t[k] if (c >> k) & 1 else t[k]"),
 ("no_hanging", "for q in range(start[r], start[r + 1]):", "for q in range(start[r], start[r] + 1):"),
 ("sign_or", "both = np.any(phi > 0, axis=1) & np.any(phi < 0, axis=1)",
  "both = np.any(phi > 0, axis=1) | np.any(phi < 0, axis=1)"),
 ("target_swap", "target = np.where(near | both, level_max, level_min)",
  "target = np.where(near | both, level_min, level_max)"),
 ("passes_count", "        cur = nxt\n        passes += 1", "        cur = nxt\n        passes += 2"),
 ("morton_axes", "k |= ((int(a[ax]) >> b) & 1) << (dim * b + ax)",
  "k |= ((int(a[ax]) >> b) & 1) << (dim * b + dim - 1 - ax)"),
 ("children_half", "h = 1 << (max_level - l - 1)", "h = 1 << (max_level - l)"),
 ("band_strict", "near = np.any(np.abs(phi) <= band, axis=1)", "near = np.any(np.abs(phi) <= 0.5 * band, axis=1)"),
]


def _run(mut):
    name, a, b = mut
    d = tempfile.mkdtemp(prefix="rmut_")
    try:
        ign = shutil.ignore_patterns("*.so", "__pycache__", "_build", "*.o", "csrc")
        for sub in ("oracle", "tests", "paper_1912_12453_gb300"):
            shutil.copytree(os.path.join(ROOT, sub), os.path.join(d, sub), ignore=ign)
        p = os.path.join(d, "oracle", "remesh.py")
        s = open(p).read()
        if s.count(a) != 1:
            return name, None, "pattern not found once"
        open(p, "w").write(s.replace(a, b, 1))
        r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_remesh_oracle_pins.py", "-x", "-q",
                            "-p", "no:cacheprovider"], cwd=d, capture_output=True, text=True, timeout=600)
        failed = [l for l in r.stdout.splitlines() if l.startswith("FAILED")]
        return name, r.returncode != 0, failed[:1]
    finally:
        shutil.rmtree(d, ignore_errors=True)


@pytest.mark.slow
def test_every_planted_remesh_mistake_is_caught():
    with cf.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        res = list(ex.map(_run, M))
    bad = [(n, why) for n, caught, why in res if caught is not True]
    assert not bad, bad
    assert len(res) == len(M) >= 12
