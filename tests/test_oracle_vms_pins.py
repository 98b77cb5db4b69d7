"""Hand-linearised Jacobian of the fully discrete VMS form (Sec. 3.4) at
states where every coefficient is constant in space, compared with the
oracle's exact (dual-number) Jacobian.

At these states the strong residual R_m is a nonzero constant, the flow moves
(v~ != 0) and the flux J or the phase gradient is nonzero, so the
stabilisation terms (cross-stress, Reynolds-stress, SUPG-like, PSPG, flux
and grad-div terms) and the capillary terms all contribute to J.  Every
perturbation is a combination of N_b, d_l N_b and d_i d_j N_b with constant
coefficients, so each block is a sum of tensor products of the 1D Q1 element
matrices.  The linearisation below is derived by hand from the printed weak
form; it shares nothing with the oracle's code.
"""
import numpy as np
import pytest

from paper_1912_12453_gb300 import workloads as W
from oracle import oracle as O


def _fem1d(n, h):
    M = np.zeros((n + 1, n + 1))
    K = np.zeros_like(M)
    C = np.zeros_like(M)  # C[a, b] = int phi_a' phi_b
    for e in range(n):
        idx = [e, e + 1]
        M[np.ix_(idx, idx)] += h / 6 * np.array([[2, 1], [1, 2]])
        K[np.ix_(idx, idx)] += 1 / h * np.array([[1, -1], [-1, 1]])
        C[np.ix_(idx, idx)] += np.array([[-0.5, -0.5], [0.5, 0.5]])
    return {(0, 0): M, (1, 0): C, (0, 1): C.T, (1, 1): K}


class Ops:
    """int (d^test N_a)(d^trial N_b) on a uniform grid, canonical node order."""

    def __init__(self, dim, n):
        self.dim = dim
        self.f = _fem1d(n, 1.0 / n)
        self.cache = {}

    def __call__(self, test=(), trial=()):
        key = (tuple(test), tuple(sorted(trial)))
        if key not in self.cache:
            out = None
            for a in reversed(range(self.dim)):  # z slowest
                m = self.f[(1 if a in test else 0, 1 if a in trial else 0)]
                out = m if out is None else np.kron(out, m)
            self.cache[key] = out
        return self.cache[key]


class Lin:
    """Perturbation c0 N_b + sum_l c1[l] d_l N_b + sum_{i<j} c2[i,j] d_i d_j N_b."""

    def __init__(self, dim, c0=0.0, c1=None, c2=None):
        self.dim = dim
        self.c0 = float(c0)
        self.c1 = np.zeros(dim) if c1 is None else np.asarray(c1, dtype=float).copy()
        self.c2 = np.zeros((dim, dim)) if c2 is None else np.asarray(c2, dtype=float).copy()

    def __add__(self, o):
        return Lin(self.dim, self.c0 + o.c0, self.c1 + o.c1, self.c2 + o.c2)

    def __sub__(self, o):
        return self + (-1.0) * o

    def __rmul__(self, s):
        return Lin(self.dim, s * self.c0, s * self.c1, s * self.c2)

    def test_N(self, ops):       # (N_a, X)
        r = self.c0 * ops()
        for l in range(self.dim):
            r = r + self.c1[l] * ops((), (l,))
        for i in range(self.dim):
            for j in range(i + 1, self.dim):
                r = r + self.c2[i, j] * ops((), (i, j))
        return r

    def test_dN(self, j, ops):   # (d_j N_a, X)
        r = self.c0 * ops((j,), ())
        for l in range(self.dim):
            r = r + self.c1[l] * ops((j,), (l,))
        for i in range(self.dim):
            for k in range(i + 1, self.dim):
                r = r + self.c2[i, k] * ops((j,), (i, k))
        return r


def zero(dim):
    return Lin(dim)


def expected_blocks(dim, prm, st, ops, clipped=False):
    """Jacobian blocks J[(row field), (col field)] (n x n each), hand derived.

    State: v^{k+1} = a, v^k = b (constants), p^{k+1} = p^k = q.x,
    phi^{k+1} = phi^k = c + k.x, mu^{k+1} = mu^k = m.x; phi is constant
    (k = 0) unless rho_r = eta_r = 1, so rho, eta, tau_m, tau_c and R_m are
    constants.
    """
    a, b, q, c, kk, m = st["a"], st["b"], st["q"], st["c"], st["k"], st["m"]
    dt, We, Re, Fr, Pe, Cn, CI = prm.dt, prm.We, prm.Re, prm.Fr, prm.Pe, prm.Cn, prm.C_I
    g = np.asarray(prm.gravity[:dim])
    alpha, beta = 0.5 * (1 - prm.rho_ratio), 0.5 * (1 + prm.rho_ratio)
    gamma, xi = 0.5 * (1 - prm.eta_ratio), 0.5 * (1 + prm.eta_ratio)
    jc = 0.5 * (prm.rho_ratio - 1)
    G = 4.0 / st["h"] ** 2
    vb = 0.5 * (a + b)
    dv = a - b
    if clipped:  # phi^{k+1} > 1 everywhere: phi* = 1, rho = eta = 1, no derivative
        rho, eta = 1.0, 1.0
        alpha = gamma = 0.0
        eta_grad = np.zeros(dim)
    else:
        rho = alpha * c + beta
        eta = gamma * c + xi
        eta_grad = gamma * kk
    # constant coefficients need a constant rho (alpha = 0 or phi constant) and
    # an eta that does not enter tau (C_I = 0) or is constant
    assert np.all(kk == 0) or clipped or (alpha == 0 and (gamma == 0 or CI == 0))
    J = jc * m
    R = rho * dv / dt + q / We - rho * g / Fr          # constant strong momentum residual
    rad = 4 / dt ** 2 + G * vb @ vb + G * (vb @ J) / (rho * Pe) + CI * (eta / (rho * Re)) ** 2 * dim * G * G
    assert rad >= 4 / dt ** 2
    tau = rad ** -0.5
    tau_c = 1.0 / (dim * G * tau)
    nf = dim + 3
    ip, iphi, imu = dim, dim + 1, dim + 2
    blocks = {}
    for col in range(nf):
        # perturbations of the primitive fields along N_b in field `col`
        d_vt = [Lin(dim, 0.5 if col == i else 0.0) for i in range(dim)]   # v~
        d_dv = [Lin(dim, 1.0 if col == i else 0.0) for i in range(dim)]   # v^{k+1} - v^k
        d_pt = Lin(dim, 0.5 if col == ip else 0.0)
        d_phin = Lin(dim, 1.0 if col == iphi else 0.0)                    # phi^{k+1}
        d_phit = Lin(dim, 0.5 if col == iphi else 0.0)
        d_mut = Lin(dim, 0.5 if col == imu else 0.0)

        def grad(L, l):
            return Lin(dim, 0.0, np.eye(dim)[l] * L.c0)

        def hess(L, i, j):
            c2 = np.zeros((dim, dim))
            c2[min(i, j), max(i, j)] = L.c0
            return Lin(dim, 0.0, None, c2)

        d_rho = alpha * d_phin
        d_eta = gamma * d_phin
        d_J = [jc * grad(d_mut, i) for i in range(dim)]
        # rad = 4/dt^2 + G v.v + G v.J/(rho Pe) + CI (eta/(rho Re))^2 dim G^2
        d_rad = zero(dim)
        for i in range(dim):
            d_rad = d_rad + (2 * G * vb[i]) * d_vt[i]
            d_rad = d_rad + (G / (rho * Pe)) * (J[i] * d_vt[i] + vb[i] * d_J[i])
        d_rad = d_rad - (G * (vb @ J) / (rho ** 2 * Pe)) * d_rho
        visc = eta / (rho * Re)
        d_rad = d_rad + (CI * dim * G * G * 2 * visc) * ((1 / (rho * Re)) * d_eta - (eta / (rho ** 2 * Re)) * d_rho)
        d_tau = (-0.5 * tau ** 3) * d_rad
        d_tau_over_rho = (1 / rho) * d_tau - (tau / rho ** 2) * d_rho
        # d R_i at this state (grad v~ = 0, Hessian of phi~ = 0, grad eta = 0)
        d_R = []
        for i in range(dim):
            r = (dv[i] / dt - g[i] / Fr) * d_rho + (rho / dt) * d_dv[i]
            for j in range(dim):
                r = r + (rho * vb[j] + J[j] / Pe) * grad(d_vt[i], j)
                if j != i:
                    r = r + (Cn / We * kk[j]) * hess(d_phit, i, j)
            r = r + (1 / We) * grad(d_pt, i)
            for k in range(dim):
                r = r - (eta_grad[k] / Re) * grad(d_vt[i], k)           # -(1/Re) d_k eta d_k v_i
            d_R.append(r)
        d_Rc = zero(dim)
        for i in range(dim):
            d_Rc = d_Rc + grad(d_vt[i], i)
        rows = {}
        for i in range(dim):
            A = (rho / dt) * d_dv[i] + (dv[i] / dt) * d_rho              # (w, rho dv/dt)
            T = zero(dim)
            for j in range(dim):
                A = A + (rho * vb[j]) * grad(d_vt[i], j)                  # (w, rho v.grad v)
                A = A - (tau * R[j]) * grad(d_vt[i], j)                   # -(w, tau R_j d_j v_i)
                A = A + (J[j] / Pe) * grad(d_vt[i], j)                    # (1/Pe)(w, J.grad v)
            A = A - (g[i] / Fr) * d_rho                                   # -(w, rho g/Fr)
            blk = A.test_N(ops)
            for j in range(dim):
                X = (tau * R[i]) * d_vt[j] + vb[j] * (R[i] * d_tau + tau * d_R[i])       # (d_j w, v_j tau R_i)
                X = X - (R[j] * R[i]) * ((2 * tau / rho) * d_tau - (tau ** 2 / rho ** 2) * d_rho) \
                    - (tau ** 2 / rho) * (R[i] * d_R[j] + R[j] * d_R[i])                 # -(d_j w, tau^2/rho R_j R_i)
                X = X + (1 / Pe) * ((tau * R[i] / rho) * d_J[j] + J[j] * R[i] * d_tau_over_rho
                                    + (J[j] * tau / rho) * d_R[i])                       # (1/Pe)(d_j w, J_j tau/rho R_i)
                X = X - (Cn / We) * (kk[j] * grad(d_phit, i) + kk[i] * grad(d_phit, j))  # -(Cn/We)(d_j w, d_i phi d_j phi)
                X = X + (eta / Re) * grad(d_vt[i], j)                                    # (1/Re)(d_j w, eta d_j v_i)
                if j == i:
                    X = X - (1 / We) * d_pt + (rho * tau_c / We) * d_Rc                  # p and grad-div
                blk = blk + X.test_dN(j, ops)
            rows[i] = blk
        # continuity
        blk = d_Rc.test_N(ops)
        for i in range(dim):
            blk = blk + (R[i] * d_tau_over_rho + (tau / rho) * d_R[i]).test_dN(i, ops)
        rows[ip] = blk
        # Cahn-Hilliard and chemical potential (phi constant: c == phi~)
        if np.all(kk == 0):
            blk = ((1 / dt) * d_phin).test_N(ops)
            for i in range(dim):
                blk = blk + (-c * d_vt[i] - vb[i] * d_phit + (1 / (Pe * Cn)) * grad(d_mut, i)).test_dN(i, ops)
            rows[iphi] = blk
            blk = ((3 * c * c - 1) * d_phit - d_mut).test_N(ops)
            for i in range(dim):
                blk = blk + (Cn ** 2 * grad(d_phit, i)).test_dN(i, ops)
            rows[imu] = blk
        for r, B in rows.items():
            blocks[(r, col)] = B
    return blocks


def _run(dim, prm, st, lev=2, clipped=False, rows_only=None):
    n = 1 << lev
    st = dict(st, h=1.0 / n)
    m = O.OracleMesh(W.uniform_leaves(dim, lev))
    x = m.coords
    Un = np.zeros((m.n_nodes, m.nf))
    Uo = np.zeros_like(Un)
    Un[:, :dim] = st["a"]
    Uo[:, :dim] = st["b"]
    for U in (Un, Uo):
        U[:, dim] = x @ st["q"]
        U[:, dim + 1] = st["c"] + x @ st["k"]
        U[:, dim + 2] = x @ st["m"]
    Jm = m.jacobian(prm, Un, Uo).toarray()
    ops = Ops(dim, n)
    exp = expected_blocks(dim, prm, st, ops, clipped)
    constrained = np.zeros(m.n_dof, dtype=bool)
    constrained[m.constrained_rows()] = True
    nf = m.nf
    worst = 0.0
    for (r, c), B in exp.items():
        if rows_only is not None and r not in rows_only:
            continue
        rows = ~constrained[r::nf]
        got = Jm[r::nf, c::nf][rows]
        ref = B[rows]
        scale = max(1.0, np.max(np.abs(ref)))
        err = np.max(np.abs(got - ref)) / scale
        assert err < 1e-11, (r, c, err)
        worst = max(worst, err)
    return worst


@pytest.mark.parametrize("dim", [2, 3])
def test_vms_jacobian_moving_flow_with_flux(dim):
    """phi constant, rho_r != 1: R_m = rho dv/dt + grad p/We - rho g/Fr != 0,
    v~ != 0 and J = (rho_r - 1)/2 grad mu != 0."""
    prm = W.Params(dim, 0.05, 0.3, 7.0, 3.0, 5.0, 2.0, 0.3, 0.6,
                   gravity=(0.6, -0.8, 0.0) if dim == 2 else (0.48, -0.6, 0.64))
    st = dict(a=np.array([0.7, -0.4, 0.3][:dim]), b=np.array([0.2, 0.5, -0.6][:dim]),
              q=np.array([0.9, -1.3, 0.5][:dim]), c=0.35, k=np.zeros(dim),
              m=np.array([-1.1, 0.8, 1.7][:dim]))
    _run(dim, prm, st)


@pytest.mark.parametrize("dim", [2, 3])
def test_vms_jacobian_capillary(dim):
    """rho_r = eta_r = 1 and a linear phase field: the Korteweg term of R_m and
    the capillary stress term of the momentum rows contribute."""
    prm = W.Params(dim, 0.05, 0.3, 7.0, 3.0, 5.0, 2.0, 1.0, 1.0,
                   gravity=(0.6, -0.8, 0.0) if dim == 2 else (0.48, -0.6, 0.64))
    st = dict(a=np.array([0.7, -0.4, 0.3][:dim]), b=np.array([0.2, 0.5, -0.6][:dim]),
              q=np.array([0.9, -1.3, 0.5][:dim]), c=0.1, k=np.array([0.5, -0.3, 0.2][:dim]),
              m=np.array([-1.1, 0.8, 1.7][:dim]))
    _run(dim, prm, st)


@pytest.mark.parametrize("dim", [2, 3])
def test_vms_jacobian_clipped_phase(dim):
    """phi^{k+1} > 1 everywhere with a nonzero gradient: the phi* clip makes
    rho = eta = 1 constant, so grad eta = 0 even though grad phi != 0."""
    prm = W.Params(dim, 0.05, 0.3, 7.0, 3.0, 5.0, 2.0, 0.3, 0.6,
                   gravity=(0.6, -0.8, 0.0) if dim == 2 else (0.48, -0.6, 0.64))
    st = dict(a=np.array([0.7, -0.4, 0.3][:dim]), b=np.array([0.2, 0.5, -0.6][:dim]),
              q=np.array([0.9, -1.3, 0.5][:dim]), c=1.5, k=np.array([0.3, 0.2, 0.1][:dim]),
              m=np.array([-1.1, 0.8, 1.7][:dim]))
    _run(dim, prm, st, clipped=True, rows_only=set(range(dim + 1)))


@pytest.mark.parametrize("dim", [2, 3])
def test_vms_jacobian_viscosity_gradient(dim):
    """rho_r = 1, eta_r != 1, linear phi, C_I = 0: grad eta != 0 enters the
    strong residual, -(1/Re) d_k eta d_k v_i; the continuity rows (PSPG) see it
    with constant coefficients."""
    prm = W.Params(dim, 0.05, 0.3, 7.0, 3.0, 5.0, 2.0, 1.0, 0.4, C_I=0.0,
                   gravity=(0.6, -0.8, 0.0) if dim == 2 else (0.48, -0.6, 0.64))
    st = dict(a=np.array([0.7, -0.4, 0.3][:dim]), b=np.array([0.2, 0.5, -0.6][:dim]),
              q=np.array([0.9, -1.3, 0.5][:dim]), c=0.1, k=np.array([0.5, -0.3, 0.2][:dim]),
              m=np.array([-1.1, 0.8, 1.7][:dim]))
    _run(dim, prm, st, rows_only={dim})
