"""Mutation sweep of the oracle pins (run by hand: python tests/oracle_mutation_sweep.py).

Plants one plausible mistake at a time in a copy of the oracle (a flipped
sign, a dropped term, a swapped index, a wrong weight) and runs the oracle
pin tests on the copy; every planted mistake must make some pin fail.
Nothing is changed in the repository itself.
"""
import os, shutil, subprocess, sys, tempfile
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
 ("no_floor", "if (val(rad) < 4.0 / (dt * dt)) rad = T(4.0 / (dt * dt));", ""),
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
which = sys.argv[1:] or [m[0] for m in M]
res = {}
for name, a, b in M:
    if name not in which: continue
    d = tempfile.mkdtemp(prefix='mut_')
    for sub in ['oracle','tests','paper_1912_12453_gb300']:
        shutil.copytree(os.path.join(ROOT,sub), os.path.join(d,sub), ignore=shutil.ignore_patterns('*.so','__pycache__'))
    p = os.path.join(d,'oracle','chns_oracle.cpp'); s = open(p).read()
    assert s.count(a) >= 1, name
    open(p,'w').write(s.replace(a,b,1))
    r = subprocess.run([sys.executable,'-m','pytest','tests/test_oracle_vms_pins.py','tests/test_oracle_pins.py','-x','-q','-m','not gpu','-p','no:cacheprovider'],cwd=d,capture_output=True,text=True)
    last = [l for l in r.stdout.splitlines() if l.startswith('FAILED')]
    res[name] = (r.returncode, last[:1])
    print(name, 'CAUGHT' if r.returncode!=0 else 'MISSED', last[:1], flush=True)
    shutil.rmtree(d)
missed = [k for k, v in res.items() if v[0] == 0]
print(f"{len(res) - len(missed)}/{len(res)} planted mistakes caught", "missed: " + ", ".join(missed) if missed else "")
sys.exit(1 if missed else 0)
