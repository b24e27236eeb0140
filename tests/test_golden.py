"""The oracle against its stored fixture and the paper's printed constants.

Floats are compared to a few ulp (the C library's cbrt may differ in the
last place between machines); pair lists exactly.
"""
import json
import os

import numpy as np

import oracle
from paper_2309_08217_gb300 import discs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_paper_constants_are_the_defaults():
    c = json.load(open(os.path.join(GOLD, "paper_constants.json")))
    d = discs.disc_uniform(8, 1)
    assert (d.n1, d.n2) == (c["n1"], c["n2"])          # Sect. 1, after Eq. (1)


def test_oracle_reproduces_stored_fixture():
    g = json.load(open(os.path.join(GOLD, "oracle_disc24.json")))
    arr = [np.array(v) for v in g["state"]]
    G, M, dt = g["G"], g["Mstar"], g["dt"]
    a, rc = oracle.rcrit(*arr, G=G, Mstar=M, dt=dt, n1=g["n1"], n2=g["n2"])
    assert np.allclose(a, g["a"], rtol=1e-14, atol=0)
    assert np.allclose(rc, g["rcrit_eq1"], rtol=1e-14, atol=0)
    for mode in (0, 1):
        for form in (0, 1):
            acc = oracle.kick_acc(arr[0], arr[1], arr[2], arr[6], a, rc, G, M, 3.0, mode, form)
            assert np.allclose(acc, np.array(g[f"acc_mode{mode}_form{form}"]), rtol=1e-13, atol=0)
        pairs, _ = oracle.encounters(arr[0], arr[1], arr[2], arr[6], a, rc, 3.0, M, mode)
        assert pairs.tolist() == g[f"pairs_mode{mode}"]
    # the planted pairs: (0,1) at 0.5 r_crit and (2,3) at 0.05 r_crit are encounters
    assert g["pairs_mode1"] == [[0, 1], [2, 3]]
    st = [np.array(v) for v in g["state"]]
    assert oracle.step(st, G, M, dt, 3.0, 0.4, 1, 0, 1) == 0
    for v, w in zip(st, g["after_one_step_mode1_form0"]):
        assert np.allclose(v, np.array(w), rtol=1e-13, atol=1e-18)
    # with the close-encounter level the planted pairs (0,1), (2,3) are two groups
    st = [np.array(v) for v in g["state"]]
    forced = [0]
    assert oracle.step(st, G, M, dt, 3.0, 0.4, 1, 0, 1, bs_tol=1e-12, forced=forced) == 0
    assert forced[0] == 0 == g["bs_forced"]
    for v, w in zip(st, g["after_one_step_bs_mode1_form0"]):
        assert np.allclose(v, np.array(w), rtol=1e-12, atol=1e-18)
    moved = [np.abs(np.array(u) - np.array(w)).max()
             for u, w in zip(g["after_one_step_bs_mode1_form0"], g["after_one_step_mode1_form0"])]
    assert max(moved) > 1e-9          # the level changes the planted pairs' motion
    # with 2 intermediate levels of 3 sub-steps (Sect. 1's hierarchy)
    st = [np.array(v) for v in g["state"]]
    forced = [0]
    assert oracle.step(st, G, M, dt, 3.0, 0.4, 1, 0, 1, bs_tol=1e-12, forced=forced, n_levels=2, n_sub=3) == 0
    assert forced[0] == 0 == g["levels_forced"]
    for v, w in zip(st, g["after_one_step_levels2_3_mode1_form0"]):
        assert np.allclose(v, np.array(w), rtol=1e-12, atol=1e-18)
    moved = [np.abs(np.array(u) - np.array(w)).max()
             for u, w in zip(g["after_one_step_levels2_3_mode1_form0"], g["after_one_step_bs_mode1_form0"])]
    assert max(moved) > 1e-12         # the pair at 0.5 r_crit is outside r_crit / 3: level-1 kicks instead
