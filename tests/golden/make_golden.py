"""Writes tests/golden/oracle_disc24.json from the CPU oracle only.

The fixture is a 24-body disc (seed 24) with three planted close pairs:
one at ~0.5 r_crit (changeover region), one at ~0.05 r_crit (K = 0) and
one just outside r_crit.  It stores the oracle's critical radii, kick
accelerations, encounter pairs and the state after one level-0 step, after
one step with the close-encounter level and after one step with two
intermediate levels of three sub-steps above it (Sect. 1), so a later
change of the oracle's arithmetic shows up as a diff of this file.

Run:  python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2309_08217_gb300 import discs  # noqa: E402


def build_case():
    d = discs.disc_uniform(24, 24, a_min=0.9, a_max=1.2, m_total=24 * 3e-7)
    arr = oracle.disc_arrays(d)
    a, rc = oracle.rcrit(*arr, G=d.G, Mstar=d.Mstar, dt=d.dt, n1=3.0, n2=0.4)
    # planted pairs: body i is moved next to body j along a fixed direction
    u = np.array([0.6, 0.0, 0.8])
    for i, j, frac in [(1, 0, 0.5), (3, 2, 0.05), (5, 4, 1.02)]:
        rcij = oracle.pair_rcrit(1, arr[6][i], arr[6][j], a[i], a[j], rc[i], rc[j], 3.0, 1.0)
        for c in range(3):
            arr[c][i] = arr[c][j] + frac * rcij * u[c]
    return d, arr


def main():
    d, arr = build_case()
    G, M = d.G, d.Mstar
    out = {"source": "tests/golden/make_golden.py (CPU oracle only)",
           "G": G, "Mstar": M, "dt": d.dt, "n1": 3.0, "n2": 0.4,
           "state": [a.tolist() for a in arr]}
    a, rc = oracle.rcrit(*arr, G=G, Mstar=M, dt=d.dt, n1=3.0, n2=0.4)
    out["a"] = a.tolist()
    out["rcrit_eq1"] = rc.tolist()
    for mode in (0, 1):
        for form in (0, 1):
            acc = oracle.kick_acc(arr[0], arr[1], arr[2], arr[6], a, rc, G, M, 3.0, mode, form)
            out[f"acc_mode{mode}_form{form}"] = acc.tolist()
        pairs, band = oracle.encounters(arr[0], arr[1], arr[2], arr[6], a, rc, 3.0, M, mode)
        out[f"pairs_mode{mode}"] = pairs.tolist()
    st = oracle.disc_arrays(d)
    st = [np.array(v) for v in out["state"]]
    bad = oracle.step(st, G, M, d.dt, 3.0, 0.4, 1, 0, 1)
    out["after_one_step_mode1_form0"] = [v.tolist() for v in st]
    out["kepler_failures"] = bad
    # the same step with the close-encounter level (Bulirsch-Stoer groups, tolerance 1e-12)
    st = [np.array(v) for v in out["state"]]
    forced = [0]
    out["kepler_failures_bs"] = oracle.step(st, G, M, d.dt, 3.0, 0.4, 1, 0, 1, bs_tol=1e-12, forced=forced)
    out["bs_forced"] = forced[0]
    out["after_one_step_bs_mode1_form0"] = [v.tolist() for v in st]
    # the same step with 2 intermediate levels of 3 sub-steps above Bulirsch-Stoer
    st = [np.array(v) for v in out["state"]]
    forced = [0]
    out["kepler_failures_levels"] = oracle.step(st, G, M, d.dt, 3.0, 0.4, 1, 0, 1, bs_tol=1e-12, forced=forced,
                                                n_levels=2, n_sub=3)
    out["levels_forced"] = forced[0]
    out["after_one_step_levels2_3_mode1_form0"] = [v.tolist() for v in st]
    out["energy"] = oracle.energy([np.array(v) for v in out["state"]], G, M).tolist()
    with open(os.path.join(HERE, "oracle_disc24.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
