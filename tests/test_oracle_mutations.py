"""Mutation test of the oracle's pins: one plausible mistake at a time (a
flipped sign, a dropped term, a swapped index, a wrong weight, a broken dual
number rule, a missing clip or floor) is planted in a copy of the oracle, and
the pin tests run on the copy; every planted mistake must make a pin fail.
The repository itself is not changed.  The mutants run in parallel, each in
its own temporary copy (oracle, tests, the input generators).
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

M = [
 ("pspg_sign", "s += T(dNa[i]) * tau_m / rho * Rm[i]; // +(d_i q", "s = s - T(dNa[i]) * tau_m / rho * Rm[i]; // +(d_i q"),
 ("cross_sign", "s = s - T(Na) * cross;", "s += T(Na) * cross;"),
 ("drop_capil_Rm", "+ T(P.Cn / P.We) * capil +", "+"),
 ("visc_no_eta", "s += T(dNa[k]) * eta * dvt[i][k] / T(P.Re);", "s += T(dNa[k]) * dvt[i][k] / T(P.Re);"),
 ("J_sign", "T(0.5 * (P.rho_r - 1.0)) * dmut[i]", "T(0.5 * (1.0 - P.rho_r)) * dmut[i]"),
 ("tau_c_GG", "T tau_c = T(1.0) / (T(trG) * tau_m);", "T tau_c = T(1.0) / (T(GG) * tau_m);"),
 ("p_not_avg", "T pt = T(0.5) * (pn.u + po.u)", "T pt = pn.u"),
 ("psi_sign", "T dpsi = phit * phit * phit - phit;", "T dpsi = phit * phit * phit + phit;"),
 ("ch_adv_sign", "s = s - T(dNa[i]) * vt[i] * phit;", "s += T(dNa[i]) * vt[i] * phit;"),
 ("capil_index", "capil += ddphit[i][j] * dphit[j];", "capil += ddphit[i][j] * dphit[i];"),
 ("conv_index_Rm", "conv += vt[j] * dvt[i][j];\n        flux", "conv += vt[j] * dvt[j][i];\n        flux"),
 ("drop_gravity_weak", "s = s - T(Na) * rho * T(P.g[i] / P.Fr);", ""),
 ("graddiv_no_rho", "s += T(dNa[i]) * rho * tau_c * Rc / T(P.We);", "s += T(dNa[i]) * tau_c * Rc / T(P.We);"),
 ("supg_transpose", "s += T(dNa[j]) * vt[j] * tau_m * Rm[i];", "s += T(dNa[j]) * vt[i] * tau_m * Rm[j];"),
 ("tau_vGJ_sign", "+ vGJ / (rho * T(P.Pe))", "- vGJ / (rho * T(P.Pe))"),
 ("Rm_dt_no_rho", "Rm[i] = rho * dv[i] / T(dt)", "Rm[i] = dv[i] / T(dt)"),
 ("hang_weight", "double w = 1.0 / (double)it->second.size();", "double w = 0.5;"),
 ("dual_sqrt", "return Dual(s, a.d / (2.0 * s));", "return Dual(s, a.d / s);"),
 ("deta_noclip", "deta[k] = inside ? T(gamma) * phin.du[k] : T(0.0);", "deta[k] = T(gamma) * phin.du[k];"),
 ("no_floor", "      rad = T(4.0 / (dt * dt));\n      if (floors)", "      if (floors)"),
 ("mu_Cn", "s += T(P.Cn * P.Cn) * T(dNa[i]) * dphit[i];", "s += T(P.Cn) * T(dNa[i]) * dphit[i];"),
 ("ch_mob", "dmut[i] / T(P.Pe * P.Cn);", "dmut[i] / T(P.Pe);"),
 ("energy_kin", "E += detJ * (0.5 * rho * v2", "E += detJ * (rho * v2"),
 ("visc_Rm_sign", "- visc_t / T(P.Re)", "+ visc_t / T(P.Re)"),
 ("Jflux_weak_drop", "s += T(Na) * flux / T(P.Pe);", ""),
 ("tau2_sign", "s = s - T(dNa[j]) * tau_m * tau_m / rho * Rm[j] * Rm[i];", "s += T(dNa[j]) * tau_m * tau_m / rho * Rm[j] * Rm[i];"),
 ("J_tau_term_drop", "s += T(dNa[j]) * J[j] * tau_m / rho * Rm[i] / T(P.Pe);", ""),
 ("C_I_drop", "T(P.C_I) * visc * visc * T(GG)", "visc * visc * T(GG)"),
 ("phis_no_clip", "bool inside = std::fabs(val(phin.u)) <= 1.0;", "bool inside = true;"),
 ("rho_old_phi", "T rho = T(alpha) * phis + T(beta);\n    T eta", "T rho = T(alpha) * phio.u + T(beta);\n    T eta"),
]


def _run(mut):
    name, a, b = mut
    d = tempfile.mkdtemp(prefix="mut_")
    try:
        ign = shutil.ignore_patterns("*.so", "__pycache__", "_build", "*.o", "csrc")
        for sub in ("oracle", "tests", "paper_1912_12453_gb300"):
            shutil.copytree(os.path.join(ROOT, sub), os.path.join(d, sub), ignore=ign)
        p = os.path.join(d, "oracle", "chns_oracle.cpp")
        s = open(p).read()
        if s.count(a) < 1:
            return name, None, "pattern not found"
        open(p, "w").write(s.replace(a, b, 1))
        r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle_vms_pins.py", "tests/test_oracle_pins.py",
                            "-x", "-q", "-m", "not gpu", "-p", "no:cacheprovider"],
                           cwd=d, capture_output=True, text=True, timeout=600)
        failed = [l for l in r.stdout.splitlines() if l.startswith("FAILED")]
        return name, r.returncode != 0, failed[:1]
    finally:
        shutil.rmtree(d, ignore_errors=True)


@pytest.mark.slow
def test_every_planted_mistake_is_caught():
    with cf.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        res = list(ex.map(_run, M))
    bad = [(n, why) for n, caught, why in res if caught is not True]
    assert not bad, bad
    assert len(res) == len(M) >= 30
