"""Manufactured solution of Sec. 5.1 and its forcing (test helper).

The exact fields are the ones printed in Eq. manufac_exact (a 3D variant
adds z-dependence to p, phi and mu, keeps v_3 = 0, and still satisfies
div v = 0, v.n = 0 and zero normal derivatives of phi and mu on the walls).
The forcing is the strong residual of the continuous equations (Sec. 2) in
the convective form used by the time-discrete scheme (Sec. 3.1), derived
symbolically here, independently of any weak-form code.
"""
import numpy as np


def mms_functions(dim, prm):
    import sympy as sp
    x, y, z, t = sp.symbols("x y z t")
    X = [x, y, z][:dim]
    pi = sp.pi
    if dim == 2:
        v = [sp.sin(pi * x) * sp.cos(pi * y) * sp.sin(t), -sp.cos(pi * x) * sp.sin(pi * y) * sp.sin(t)]
        p = sp.sin(pi * x) * sp.sin(pi * y) * sp.cos(t)
        phi = sp.cos(pi * x) * sp.cos(pi * y) * sp.sin(t)
    else:
        v = [sp.sin(pi * x) * sp.cos(pi * y) * sp.sin(t), -sp.cos(pi * x) * sp.sin(pi * y) * sp.sin(t),
             sp.Integer(0)]
        p = sp.sin(pi * x) * sp.sin(pi * y) * sp.sin(pi * z) * sp.cos(t)
        phi = sp.cos(pi * x) * sp.cos(pi * y) * sp.cos(pi * z) * sp.sin(t)
    mu = phi
    rr, er = prm.rho_ratio, prm.eta_ratio
    rho = (1 - rr) / 2 * phi + (1 + rr) / 2
    eta = (1 - er) / 2 * phi + (1 + er) / 2
    J = [(rr - 1) / 2 * sp.diff(mu, X[i]) for i in range(dim)]
    g = prm.gravity
    fv = []
    for i in range(dim):
        e = (rho * sp.diff(v[i], t)
             + sum(rho * v[j] * sp.diff(v[i], X[j]) for j in range(dim))
             + sum(J[j] * sp.diff(v[i], X[j]) for j in range(dim)) / prm.Pe
             + prm.Cn / prm.We * sum(sp.diff(sp.diff(phi, X[i]) * sp.diff(phi, X[j]), X[j]) for j in range(dim))
             + sp.diff(p, X[i]) / prm.We
             - sum(sp.diff(eta * sp.diff(v[i], X[j]), X[j]) for j in range(dim)) / prm.Re
             - rho * g[i] / prm.Fr)
        fv.append(e)
    fp = sum(sp.diff(v[i], X[i]) for i in range(dim))
    fphi = (sp.diff(phi, t) + sum(sp.diff(v[i] * phi, X[i]) for i in range(dim))
            - sum(sp.diff(mu, X[i], 2) for i in range(dim)) / (prm.Pe * prm.Cn))
    fmu = -mu + phi ** 3 - phi - prm.Cn ** 2 * sum(sp.diff(phi, X[i], 2) for i in range(dim))
    fe = sp.lambdify(X + [t], v + [p, phi, mu], "numpy")
    ff = sp.lambdify(X + [t], fv + [fp, fphi, fmu], "numpy")

    def ev(fn, xyz, tt):
        vals = fn(*[xyz[:, i] for i in range(dim)], tt)
        return np.stack([np.broadcast_to(np.asarray(q, dtype=float), xyz.shape[0]) for q in vals], 1)

    return (lambda xyz, tt: ev(fe, xyz, tt)), (lambda xyz, tt: ev(ff, xyz, tt))
