"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a copy of oracle.c (on the CPU, in a
temporary directory), builds it, and runs the pin suite against that build
in a child process: the suite has to fail.  The unmodified build has to
pass.  This checks the pins themselves, not the CUDA path.
"""
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTANTS = {
    "changeover_denominator_sign": ("2.0 * y2 - 2.0 * y + 1.0", "2.0 * y2 - 2.0 * y - 1.0"),
    "quintic_coefficient": ("(10.0 - 15.0 * y + 6.0 * y * y)", "(10.0 - 15.0 * y + 5.0 * y * y)"),
    "sun_velocity_sign": ("double ux = vx[i] + P[0] / Mstar;", "double ux = vx[i] - P[0] / Mstar;"),
    "rcrit_mu_without_mi": ("double mu = G * (Mstar + m[i]);", "double mu = G * Mstar;"),
    "hill_radius_exponent": ("a * cbrt(m[i] / (3.0 * Mstar))", "a * sqrt(m[i] / (3.0 * Mstar))"),
    "velocity_term_dropped_dt": ("t2 = n2 * dt * sqrt(v2)", "t2 = n2 * sqrt(v2)"),
    "pair_radius_index": ("0.5 * (ai + aj)", "0.5 * (ai + ai)"),
    "pair_radius_mode0_min": ("return (rci > rcj) ? rci : rcj;", "return (rci < rcj) ? rci : rcj;"),
    "kick_offset_sign": ("double dx = x[j] - x[i], dy = y[j] - y[i], dz = z[j] - z[i];\n            double r2",
                         "double dx = x[i] - x[j], dy = y[j] - y[i], dz = z[j] - z[i];\n            double r2"),
    "kick_changeover_argument": ("K = oracle_changeover((r / rcij - 0.1) / 0.9, form);",
                                 "K = oracle_changeover(r / rcij, form);"),
    "kick_mass_index": ("double f = G * m[j] * K / (r2 * r);", "double f = G * m[i] * K / (r2 * r);"),
    "kick_inverse_square": ("double f = G * m[j] * K / (r2 * r);", "double f = G * m[j] * K / r2;"),
    "kick_missing_changeover": ("double f = G * m[j] * K / (r2 * r);", "double f = G * m[j] / (r2 * r);"),
    "encounter_squared_distance": ("            if (r < rcij) {\n                if (cnt < cap)",
                                   "            if (r * r < rcij) {\n                if (cnt < cap)"),
    "sun_velocity_sign_y": ("double uy = vy[i] + P[1] / Mstar;", "double uy = vy[i] - P[1] / Mstar;"),
    "stumpff_doubling": ("s3 = (s2 + s0 * s3) * 0.25;", "s3 = (s2 + s1 * s3) * 0.25;"),
    "stumpff_series": ("(1.0 - z / 20.0 * (1.0 - z / 42.0", "(1.0 - z / 20.0 * (1.0 - z / 40.0"),
    "kepler_g_sign": ("double g = r0 * G1 + eta * G2;", "double g = r0 * G1 - eta * G2;"),
    "kepler_fdot": ("double fd = -mu * G1 / (r * r0);", "double fd = -mu * G1 / (r0 * r0);"),
    "hc_drift_no_mass_division": ("x[i] += tau * P[0] / Mstar;", "x[i] += tau * P[0];"),
    "drift_full_hc_halves": ("Mstar, 0.5 * dt);\n    #pragma omp parallel for reduction(+:bad)\n    for (int i = 0; i < N; i++) {\n        double s[6]",
                             "Mstar, dt);\n    #pragma omp parallel for reduction(+:bad)\n    for (int i = 0; i < N; i++) {\n        double s[6]"),
    "step_full_kick": ("mode, form, n_big, 0.5 * dt, ax, ay, az);\n        bad +=",
                       "mode, form, n_big, dt, ax, ay, az);\n        bad +="),
    "energy_sun_term": ("/ (2.0 * Mstar));", "/ (2.0));"),
    "energy_pair_term_mass": ("nadd(&e, -G * m[i] * m[j] / sqrt", "nadd(&e, -G * m[i] * m[i] / sqrt"),
    "tp2_either_test_particle": ("return n_big >= 0 && i >= n_big && j >= n_big;",
                                 "return n_big >= 0 && (i >= n_big || j >= n_big);"),
    "tp2_encounters_not_skipped": ("            if (tp_pair(n_big, i, j)) continue;\n            double dx = x[j] - x[i], dy = y[j] - y[i], dz = z[j] - z[i];\n            double r = sqrt(dx * dx + dy * dy + dz * dz);\n            double rcij = oracle_pair_rcrit(mode, m[i], m[j], a[i], a[j], rc[i], rc[j], n1, Mstar);\n            if (r < rcij) {",
                                   "            double dx = x[j] - x[i], dy = y[j] - y[i], dz = z[j] - z[i];\n            double r = sqrt(dx * dx + dy * dy + dz * dz);\n            double rcij = oracle_pair_rcrit(mode, m[i], m[j], a[i], a[j], rc[i], rc[j], n1, Mstar);\n            if (r < rcij) {"),
    "angular_momentum_component": ("nadd(&lz, m[i] * (x[i] * vy[i] - y[i] * vx[i]));",
                                   "nadd(&lz, m[i] * (x[i] * vy[i] + y[i] * vx[i]));"),
    # close-encounter level
    "groups_count_every_member": ("if (label[v] == v) ngroups++;", "ngroups++;"),
    "level1_central_sign": ("double c = -g->G * g->Mstar / (r2 * r);", "double c = g->G * g->Mstar / (r2 * r);"),
    "level1_weight_is_K": ("w *= 1.0 - oracle_changeover(", "w *= oracle_changeover("),
    "level1_offset_sign": ("double dx = xj[0] - xi[0], dy", "double dx = xi[0] - xj[0], dy"),
    "level1_mass_index": ("double f = g->G * g->m[bj] * w", "double f = g->G * g->m[bi] * w"),
    "level1_tp_pairs_kept": ("if (j == i || tp_pair(g->n_big, bi, bj) || bs_ghost", "if (j == i || bs_ghost"),
    "midpoint_step_factor": ("zn[q] = zp[q] + 2.0 * H * fz[q];", "zn[q] = zp[q] + H * fz[q];"),
    "extrapolation_in_h_not_h2": ("double cf = (nkj * nkj) / (nk * nk - nkj * nkj);",
                                  "double cf = nkj / (nk - nkj);"),
    "members_also_kepler_drifted": ("        if (label[i] >= 0) continue;\n", ""),
    "bs_no_step_growth": ("        if (acc_col <= BS_GROW_COL) frac *= 2.0;\n", ""),
    "bs_first_frac_no_velocity": ("(f * fabs(dt)) * (f * fabs(dt)) * v2 > r2", "(f * fabs(dt)) * (f * fabs(dt)) > r2"),
    "bs_kepler_completion_full_dt": ("oracle_kepler(G * Mstar, yv + 6 * k, (1.0 - done) * dt, 50);",
                                     "oracle_kepler(G * Mstar, yv + 6 * k, dt, 50);"),
    "bs_kepler_completion_skipped": ("        for (int k = 0; k < n; k++) oracle_kepler(G * Mstar, yv + 6 * k, (1.0 - done) * dt, 50);\n", ""),
    # mergers and removal
    "merge_once_only": ("        merges++;\n    }\n}", "        merges++;\n        return merges;\n    }\n}"),
    "merger_plain_average": ("yv[6 * fi + c] = (mt > 0.0) ? (mi * u + mj * w) / mt : 0.5 * (u + w);",
                             "yv[6 * fi + c] = 0.5 * (u + w);"),
    "merger_radius_sum": ("R[bi] = cbrt(R[bi] * R[bi] * R[bi] + R[bj] * R[bj] * R[bj]);", "R[bi] = R[bi] + R[bj];"),
    "merger_overlap_one_radius": ("double rr = R[g->mem[i]] + R[g->mem[j]];", "double rr = R[g->mem[i]];"),
    "merger_survivor_higher_index": ("        ghost[fj] = 1;\n", "        ghost[fi] = 1;\n"),
    "ghost_feels_no_central_body": ("        double c = -g->G * g->Mstar / (r2 * r);",
                                    "        double c = bs_ghost(g, i) ? 0.0 : -g->G * g->Mstar / (r2 * r);"),
    "ghosts_still_pull": ("|| bs_ghost(g, i) || bs_ghost(g, j)) continue;", ") continue;"),
    "removal_outer_uses_inner": ("(r_out > 0.0 && r2 > r_out * r_out)", "(r_out > 0.0 && r2 > r_in * r_in)"),
    "prediction_not_used_by_the_step": ("        int64_t npr = oracle_predicted_pairs(", "        int64_t npr = 0 * oracle_predicted_pairs("),
    "prediction_keeps_test_particle_pairs": ("            if (tp_pair(n_big, i, j)) continue;\n            double dx = x[j] - x[i], dy = y[j] - y[i], dz = z[j] - z[i];\n            double r = sqrt(dx * dx + dy * dy + dz * dz);\n            double rcij = oracle_pair_rcrit(mode, m[i], m[j], a[i], a[j], rc[i], rc[j], n1, Mstar);\n            if (r < rcij || r >= PREDICT_RANGE",
                                             "            double dx = x[j] - x[i], dy = y[j] - y[i], dz = z[j] - z[i];\n            double r = sqrt(dx * dx + dy * dy + dz * dz);\n            double rcij = oracle_pair_rcrit(mode, m[i], m[j], a[i], a[j], rc[i], rc[j], n1, Mstar);\n            if (r < rcij || r >= PREDICT_RANGE"),
    "prediction_unclamped": ("            if (t > thi) t = thi;\n", ""),
    "prediction_wrong_sign": ("            double t = uu > 0.0 ? -du / uu : 0.0;",
                              "            double t = uu > 0.0 ? du / uu : 0.0;"),
    "prediction_range": ("if (r < rcij || r >= PREDICT_RANGE * rcij) continue;", "if (r < rcij || r >= 1.1 * rcij) continue;"),
    # intermediate levels
    "levels_weight_drops_level0_keep": ("for (int k = 0; k < l && k <= L; k++)", "for (int k = 1; k < l && k <= L; k++)"),
    "levels_radius_power": ("for (int k = 0; k < l; k++) p *= s;", "for (int k = 1; k < l; k++) p *= s;"),
    "levels_last_factor_is_keep": ("if (l <= L) w *= oracle_changeover(", "if (l <= L) w *= 1.0 - oracle_changeover("),
    "levels_full_first_kick": ("        ml_kick(c, l, n, mem, 0.5 * h);\n        for (int i = 0; i < n; i++) { root[i]",
                               "        ml_kick(c, l, n, mem, h);\n        for (int i = 0; i < n; i++) { root[i]"),
    "levels_substep_not_divided": ("double h = T / c->s;", "double h = T;"),
    "levels_bs_weight_level": ("double w = oracle_ml_weight(q, rcij, g->nlev + 1,", "double w = oracle_ml_weight(q, rcij, g->nlev,"),
    "levels_subgroup_radius": ("double rcl = oracle_ml_radius(rcij, l, s);", "double rcl = oracle_ml_radius(rcij, l + 1, s);"),
    "levels_kick_weight_level": ("oracle_ml_weight(q, rcij, l, L, s, form)", "oracle_ml_weight(q, rcij, l + 1, L, s, form)"),
    "levels_members_not_drifted": ("            if (inpair[i]) continue;\n", "            if (!inpair[i]) continue;\n"),
    "levels_kick_mass_index": ("double f = G * m[bj] * oracle_ml_weight", "double f = G * m[bi] * oracle_ml_weight"),
    "levels_bs_skip_radius_one_level_deeper": ("if (q >= oracle_ml_radius(rcij, g->nlev, g->nsub)) continue;",
                                               "if (q >= oracle_ml_radius(rcij, g->nlev + 1, g->nsub)) continue;"),
    "levels_weight_radius_uses_level0": ("w *= 1.0 - oracle_changeover((q / oracle_ml_radius(rc, k, s) - 0.1) / 0.9, form);",
                                         "w *= 1.0 - oracle_changeover((q / oracle_ml_radius(rc, 0, s) - 0.1) / 0.9, form);"),
    "levels_prediction_dropped": ("    if (q2 >= rout * rout) return 0;\n", "    return 0;\n"),
    "levels_prediction_range": ("rout = 1.5 * rcl;", "rout = 1.1 * rcl;"),
    "levels_second_kick_dropped": ("&c->merges, c->L, c->s, NULL, NULL);\n        }\n        ml_kick(c, l, n, mem, 0.5 * h);\n",
                                   "&c->merges, c->L, c->s, NULL, NULL);\n        }\n"),
    "levels_tp_pairs_kicked": ("                if (j == i || signbit(m[bj]) || tp_pair(n_big, bi, bj)) continue;",
                               "                if (j == i || signbit(m[bj])) continue;"),
    "levels_ghosts_in_subgroups": ("    if (signbit(m[bi]) || signbit(m[bj]) || tp_pair(n_big, bi, bj)) return 0;",
                                   "    if (tp_pair(n_big, bi, bj)) return 0;"),
    "levels_kick_offset_sign": ("                double dx = x[bj] - x[bi], dy = y[bj] - y[bi], dz = z[bj] - z[bi];\n                double q2",
                                "                double dx = x[bi] - x[bj], dy = y[bj] - y[bi], dz = z[bj] - z[bi];\n                double q2"),
    "dead_pairs_grouped": ("        if (dead && (dead[pairs[2 * p]] || dead[pairs[2 * p + 1]])) continue;\n", ""),
}


def _build(src_text, d):
    c = os.path.join(d, "m.c")
    so = os.path.join(d, "m.so")
    with open(c, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-shared", "-fPIC", c, "-o", so, "-lm"],
                   check=True, capture_output=True)
    return so


def _run_pins(so):
    env = dict(os.environ, ORACLE_LIB=so)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                        os.path.join(ROOT, "tests", "test_oracle_bs.py"),
                        os.path.join(ROOT, "tests", "test_oracle_merge.py"),
                        os.path.join(ROOT, "tests", "test_oracle_levels.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name):
    old, new = MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) == 1, f"mutation site for {name} not unique / not found"
    with tempfile.TemporaryDirectory() as d:
        so = _build(text.replace(old, new), d)
        assert _run_pins(so) != 0, f"pins did not catch mutant {name}"


def test_unmutated_build_passes_pins():
    with tempfile.TemporaryDirectory() as d:
        so = _build(open(SRC).read(), d)
        assert _run_pins(so) == 0
