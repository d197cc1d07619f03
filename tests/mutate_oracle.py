"""Mutation check of the oracle's pins (run by hand, not collected by pytest):
plants plausible mistakes, one at a time, into temporary copies of
oracle/fdtd_oracle.c and reports whether the CPU pin suites fail on each.
A mistake no pin catches is either an equivalent change or a gap in the
pins.  Takes a few minutes:

    python tests/mutate_oracle.py [name ...]
"""
import os
import shutil
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = open(os.path.join(ROOT, "oracle", "fdtd_oracle.c")).read()

# name: (text in the oracle, the mistake put in its place)
MUTANTS = {
 'h_curl_sign': ('Hx[q] += g->db[0][q] * (tz - ty);', 'Hx[q] += g->db[0][q] * (ty - tz);'),
 'explicit_loss': ('*ca = (1.0 - a) / (1.0 + a);', '*ca = 1.0 - 2.0 * a;'),
 'cb_no_loss_div': ('*cb = dt / (e * dx) / (1.0 + a);', '*cb = dt / (e * dx);'),
 'cpml_kappa_inv': ('*b = bb; *c = cc; *ki = 1.0 / kap;', '*b = bb; *c = cc; *ki = kap;'),
 'cpml_b_half': ('exp(-(sig / kap + alp) * g->dt / ORC_EPS0)', 'exp(-(sig / kap + alp) * g->dt / (2.0 * ORC_EPS0))'),
 'cpml_c_sign': ('sig * (bb - 1.0) / (sig * kap + kap * kap * alp)', 'sig * (1.0 - bb) / (sig * kap + kap * kap * alp)'),
 'debye_beta': ('beta[p] = 2.0 * ORC_EPS0 * deps[p] * m * dt / (2.0 * tau[p] + dt);', 'beta[p] = ORC_EPS0 * deps[p] * m * dt / (2.0 * tau[p] + dt);'),
 'debye_kk': ('kk[p] = deps[p] > 0 ? (2.0 * tau[p] - dt) / (2.0 * tau[p] + dt) : 0.0;', 'kk[p] = deps[p] > 0 ? (2.0 * tau[p] - dt) / (2.0 * tau[p]) : 0.0;'),
 'debye_cj_sign': ('cj[p] = -dt * (1.0 + kk[p]) / D;', 'cj[p] = dt * (1.0 + kk[p]) / D;'),
 'avg_eps_two_cells': ('eps[0][q] = 0.25 * (cell_eps(g, i, j - 1, k - 1) + cell_eps(g, i, j, k - 1) +\n                                        cell_eps(g, i, j - 1, k) + cell_eps(g, i, j, k));',
                       'eps[0][q] = 0.5 * (cell_eps(g, i, j - 1, k - 1) + cell_eps(g, i, j, k));'),
 'ex_curl_index': ('real ty = term(Hz[q] - Hz[q - sy], g->psi[EX][1]', 'real ty = term(Hz[q + sy] - Hz[q], g->psi[EX][1]'),
 'source_sign': ('g->src_coef[s] = r32(g, -cbq / dx);', 'g->src_coef[s] = r32(g, cbq / dx);'),
 'probe_v_sign': ('            v -= g->f[p->axis][IDX(g, q[0], q[1], q[2])] * dx;', '            v += g->f[p->axis][IDX(g, q[0], q[1], q[2])] * dx;'),
 'probe_i_term': ('return dx * (Hy[IDX(g, i, j, k)] - Hy[IDX(g, i - 1, j, k)] - Hx[IDX(g, i, j, k)] + Hx[IDX(g, i, j - 1, k)]);',
                  'return dx * (Hy[IDX(g, i, j, k)] - Hy[IDX(g, i - 1, j, k)] - Hx[IDX(g, i, j, k)]);'),
 'wire_factor_inv': ('return log(g->dx / (ORC_R0_FRAC * g->dx)) / log(g->dx / a);', 'return log(g->dx / a) / log(g->dx / (ORC_R0_FRAC * g->dx));'),
 'owire_scatter_sign': ('g->f[S->comp[e]][S->q[e]] -= (double)S->ws[e] * g->oI[s];', 'g->f[S->comp[e]][S->q[e]] += (double)S->ws[e] * g->oI[s];'),
 'owire_net_sign': ('net[g->osegs[s].b] += g->oI[s];', 'net[g->osegs[s].b] -= g->oI[s];'),
 'owire_no_relax': ('g->oQ[m] += g->dt * net[m] - (double)nd->cs / (double)nd->K * (Vn + V);', 'g->oQ[m] += g->dt * net[m];'),
 'owire_lattice_pi': ('(w00 * w11 + w10 * w01) / M_PI);', '(w00 * w11 + w10 * w01) / 4.0);'),
 'junction_floating': ('if (on_axis_wire(&g->wires[w], g->onodes[m].p)) g->onodes[m].grounded = 1;', 'if (0 && on_axis_wire(&g->wires[w], g->onodes[m].p)) g->onodes[m].grounded = 1;'),
 'r0_wrong': ('const double r0 = exp(-0.57721566490153286) / (2.0 * sqrt(2.0));', 'const double r0 = 0.23;'),
 'vb_no_twelfth': ('double wt = dd[c] * (w1 * w2 + (d1 == d2 ? 1.0 : -1.0) * dd[v1] * dd[v2] / 12.0);', 'double wt = dd[c] * (w1 * w2);'),
 'lump_cap_no_dx': ('return add_lump(g, i, j, k, axis, capacitance / g->dx, resistance > 0 ? 1.0 / (resistance * g->dx) : 0.0);',
                    'return add_lump(g, i, j, k, axis, capacitance, resistance > 0 ? 1.0 / (resistance * g->dx) : 0.0);'),
 'lump_res_no_dx': ('return add_lump(g, i, j, k, axis, capacitance / g->dx, resistance > 0 ? 1.0 / (resistance * g->dx) : 0.0);',
                    'return add_lump(g, i, j, k, axis, capacitance / g->dx, resistance > 0 ? 1.0 / resistance : 0.0);'),
 'vsource_sign': ('if (g->srcs[s].hard) g->hard_coef[s] = r32(g, -1.0 / dx);', 'if (g->srcs[s].hard) g->hard_coef[s] = r32(g, 1.0 / dx);'),
 'vsource_r_current': ('return push_src(g, i, j, k, axis, volt, n, 1.0 / r_internal, 0);', 'return push_src(g, i, j, k, axis, volt, n, r_internal, 0);'),
 'cpml_sigma_max': ('sigma_max = 0.8 * (order + 1.0) / (eta0 * g->dx);', 'sigma_max = 0.2 * (order + 1.0) / (eta0 * g->dx);'),
 'debye_be': ('be[p] = beta[p] / dt;', 'be[p] = beta[p];'),
 'owire_gather_weight': ('S->wg[e] = r32(g, S->W[e] * dx / S->dl);', 'S->wg[e] = r32(g, S->W[e]);'),
 'owire_series_r': ('double k = 0.5 * dt * (S->R / (Lp * S->dl) + S->nu);', 'double k = 0.5 * dt * (S->R / Lp + S->nu);'),
 'owire_cpml_nu_linear': ('S->nu += S->t[q] * S->t[q] * cpml_rate(g, q, S->c[q]);', 'S->nu += fabs(S->t[q]) * cpml_rate(g, q, S->c[q]);'),
 'owire_no_nu': ('S->nu += S->t[q] * S->t[q] * cpml_rate(g, q, S->c[q]);', 'S->nu += 0.0 * cpml_rate(g, q, S->c[q]);'),
 'owire_node_K': ('double K = lam / (2.0 * M_PI * nd->dlm);', 'double K = lam / nd->dlm;'),
}
PINS = ["tests/test_oracle_pins.py", "tests/test_debye_pins.py", "tests/test_owire_pins.py", "tests/test_lumped_pins.py",
        "tests/test_wire_path_pins.py", "tests/test_golden.py", "tests/test_owire_stability.py"]


def check(name, old, new, work):
    if SRC.count(old) != 1:
        raise SystemExit(f"{name}: the text to replace is not unique in the oracle (edit the mutant)")
    d = os.path.join(work, name)
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(d, "oracle"),
                    ignore=shutil.ignore_patterns("_build", "__pycache__"))
    with open(os.path.join(d, "oracle", "fdtd_oracle.c"), "w") as f:
        f.write(SRC.replace(old, new))
    shutil.copytree(os.path.join(ROOT, "tests"), os.path.join(d, "tests"), ignore=shutil.ignore_patterns("__pycache__"))
    os.symlink(os.path.join(ROOT, "paper_2207_06908_gb300"), os.path.join(d, "paper_2207_06908_gb300"))
    shutil.copy(os.path.join(ROOT, "pytest.ini"), d)
    r = subprocess.run([sys.executable, "-m", "pytest", *PINS, "-m", "not gpu", "-q", "-x", "-p", "no:cacheprovider"],
                       cwd=d, capture_output=True, text=True, timeout=1800)
    first = next((l for l in r.stdout.splitlines() if l.startswith(("FAILED", "ERROR"))), "")
    return r.returncode != 0, first


def main(names):
    todo = {k: v for k, v in MUTANTS.items() if not names or k in names}
    caught = 0
    with tempfile.TemporaryDirectory() as work:
        for name, (old, new) in todo.items():
            t0 = time.time()
            ok, first = check(name, old, new, work)
            caught += ok
            print(f"{name:24s} {'caught' if ok else 'SURVIVED':9s} {time.time() - t0:5.1f} s  {first[:100]}", flush=True)
    print(f"{caught} of {len(todo)} caught")


if __name__ == "__main__":
    main(sys.argv[1:])
