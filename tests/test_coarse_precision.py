"""The coarse operator of the two-level preconditioner may be inverted in FP32.

A_c = P^T J P (P: trilinear interpolation of all fields from the nodes of the
uniform coarse level to the mesh nodes; J: the oracle's FP64 Jacobian of the
CN-VMS form, Sec. 3.4, at a droplet state) is ill-conditioned (cond ~ 1e8)
along a single pressure direction.  The FP32 path inverts A_c with the
in-place Gauss-Jordan elimination with partial pivoting that the library runs
on the GPU; here the same steps, in float32 with numpy, are checked against the
FP64 inverse: the applied inverse must be accurate per field to well below the
Krylov tolerances (1e-3), with the dominant direction itself also resolved.
CPU only (oracle + numpy).
"""
import numpy as np
import scipy.sparse as sp

from oracle.oracle import OracleMesh
from paper_1912_12453_gb300 import workloads as W


def gauss_jordan_inplace(A):
    """Inverse by in-place Gauss-Jordan with partial pivoting, in A's dtype."""
    a = A.copy()
    n = a.shape[0]
    piv = np.zeros(n, dtype=np.int64)
    one = a.dtype.type(1)
    for k in range(n):
        p = k + int(np.argmax(np.abs(a[k:, k])))
        piv[k] = p
        if p != k:
            a[[k, p], :] = a[[p, k], :]
        d = one / a[k, k]
        a[k, :] *= d
        a[k, k] = d
        col = a[:, k].copy()
        col[k] = 0
        a -= np.outer(col, a[k, :])      # rows i != k (col[k] = 0 leaves row k)
        a[:, k] = -col * d
        a[k, k] = d
    for k in range(n - 1, -1, -1):
        if piv[k] != k:
            a[:, [k, piv[k]]] = a[:, [piv[k], k]]
    return a


def coarse_operator(level=4, Lc=2):
    wl = W.workload("droplet3d_l6")
    om = OracleMesh(W.uniform_leaves(3, level))
    U0 = om.init_mu(wl.params, W.initial_state(om.coords, wl).reshape(-1))
    U1 = U0 + 1e-2 * W.perturbation(om.n_nodes, om.nf, 1)[0].reshape(-1)
    J = om.jacobian(wl.params, U1, U0)
    nf, nc1 = om.nf, (1 << Lc) + 1
    pos = om.coords * (1 << Lc)
    b = np.clip(np.floor(pos).astype(np.int64), 0, nc1 - 2)
    t = pos - b
    rows, cols, vals = [], [], []
    for c in range(8):
        idx = np.zeros(om.n_nodes, dtype=np.int64)
        w = np.ones(om.n_nodes)
        for a in range(2, -1, -1):
            idx = idx * nc1 + b[:, a] + ((c >> a) & 1)
        for a in range(3):
            w *= t[:, a] if (c >> a) & 1 else 1 - t[:, a]
        for q in range(nf):
            rows.append(np.arange(om.n_nodes) * nf + q)
            cols.append(idx * nf + q)
            vals.append(w)
    P = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(om.n_dof, nc1 ** 3 * nf))
    return (P.T @ (J @ P)).toarray(), nf


def test_gauss_jordan_matches_lapack_inverse():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((40, 40))
    A[0, 0] = 1e-12  # forces a pivot interchange
    X = gauss_jordan_inplace(A)
    assert np.abs(X @ A - np.eye(40)).max() < 1e-11
    assert np.abs(X - np.linalg.inv(A)).max() <= 1e-12 * np.abs(np.linalg.inv(A)).max()


def test_fp32_coarse_inverse_is_accurate_per_field():
    Ac, nf = coarse_operator()
    s = np.linalg.svd(Ac, compute_uv=False)
    assert s[0] / s[-1] > 1e6  # the ill-conditioned case this decision is about
    X64 = np.linalg.inv(Ac)
    X32 = gauss_jordan_inplace(Ac.astype(np.float32)).astype(np.float64)
    vmin = np.linalg.svd(Ac)[2][-1]
    rng = np.random.default_rng(5)
    for _ in range(3):
        r = rng.standard_normal(Ac.shape[0])
        z64, z32 = X64 @ r, X32 @ r
        d = z32 - z64
        assert abs(vmin @ d) <= 1e-4 * abs(vmin @ z64)
        dp, zp = d - vmin * (vmin @ d), z64 - vmin * (vmin @ z64)
        for q in range(nf):
            assert np.linalg.norm(dp[q::nf]) <= 1e-4 * np.linalg.norm(zp[q::nf]), q
