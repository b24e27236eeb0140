"""Pins of the oracle's intermediate levels (Sect. 1: symplectic levels with
smaller steps between the kick and the Bulirsch-Stoer integrator).  None of
these calls the CUDA path.

* the weights of the levels are a partition of unity of the pair force:
  sum_{l=0}^{L+1} W_l(q) = 1 for every separation (a dropped or repeated
  factor breaks it), W_0 = K_0 is the kick's weight, every W_l >= 0;
* the radii: level l's weights end exactly at r_crit / s^l -- the
  Bulirsch-Stoer share is 1 inside 0.1 r_crit / s^L and 0 beyond r_crit / s^L,
  the shares of levels >= 1 vanish beyond r_crit;
* a group whose pairs stay beyond r_crit sees no level force: L levels of s
  sub-steps are s^0 + ... Kepler drifts adding up to one Kepler drift over dt;
* a tight binary deep inside 0.1 r_crit / s^L is all Bulirsch-Stoer: the
  recursion (s^L pieces of dt / s^L) gives the single Bulirsch-Stoer drift
  over dt (the level-1 drift without intermediate levels) to its tolerance;
* a flyby that stays outside the subgroups converges to that same drift as
  the sub-step shrinks (leapfrog on the (1 - K_0) force);
* a slow pair inside r_crit,1 (a subgroup on level 2, the Bulirsch-Stoer
  level) gets the same pair impulse as the single Bulirsch-Stoer drift, to
  the splitting error of the level-1 kicks.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2309_08217_gb300 import discs

G = discs.G_GAUSS
TOL = 1e-12


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("L,s", [(0, 2), (1, 2), (1, 4), (2, 3), (3, 2), (2, 5)])
def test_level_weights_partition_of_unity(form, L, s):
    rc = 0.37
    for q in np.linspace(1e-4, 1.3 * rc, 997):
        w = [oracle.ml_weight(q, rc, l, L, s, form) for l in range(L + 2)]
        assert min(w) >= 0.0
        assert abs(sum(w) - 1.0) < 4e-16 * (L + 2)
        assert w[0] == oracle.changeover((q / rc - 0.1) / 0.9, form)


def _kick_K(q, rc, form):
    y = (q / rc - 0.1) / 0.9
    if y <= 0:
        return 0.0
    if y >= 1:
        return 1.0
    return y * y / (2 * y * y - 2 * y + 1) if form == 0 else y ** 3 * (10 - 15 * y + 6 * y * y)


@pytest.mark.parametrize("L,s", [(1, 2), (2, 3), (3, 4)])
def test_level_radii(L, s):
    rc = 0.5
    rL = rc / s ** L
    assert oracle.ml_radius(rc, L, s) == rL
    bs = L + 1
    assert oracle.ml_weight(0.0999 * rL, rc, bs, L, s, 0) == 1.0
    assert oracle.ml_weight(0.1001 * rL, rc, bs, L, s, 0) < 1.0
    assert oracle.ml_weight(0.9999 * rL, rc, bs, L, s, 0) > 0.0
    assert oracle.ml_weight(1.0001 * rL, rc, bs, L, s, 0) == 0.0
    for l in range(1, L + 1):
        assert oracle.ml_weight(1.0001 * rc, rc, l, L, s, 0) == 0.0
        # between the radii of levels l and l - 1 level l's share is the rest of level l - 1's
        rl = rc / s ** l
        q = 1.5 * rl if 1.5 * rl < 0.999 * rc / s ** (l - 1) else 0.5 * (rl + rc / s ** (l - 1))
        keep = 1.0
        for k in range(l):
            keep *= 1.0 - _kick_K(q, rc / s ** k, 0)
        assert oracle.ml_weight(q, rc, l, L, s, 0) == pytest.approx(keep, rel=1e-14)


def _state(pos, vel, m):
    return [np.array([p[c] for p in pos], float) for c in range(3)] + \
           [np.array([v[c] for v in vel], float) for c in range(3)] + [np.array(m, float)]


def _kepler_all(arr, dt):
    for b in range(len(arr[6])):
        st, status = oracle.kepler(G, [arr[c][b] for c in range(6)], dt)
        assert status == 0
        for c in range(6):
            arr[c][b] = st[c]


def _rel(a, b):
    return max(np.abs(a[c] - b[c]).max() / np.abs(b[c]).max() for c in range(6))


@pytest.mark.parametrize("L,s", [(1, 3), (2, 2), (2, 3)])
def test_far_group_is_one_kepler_drift(L, s):
    vc = math.sqrt(G)
    pos = [(1.0, 0.0, 0.0), (0.0, 1.2, 0.01), (-0.9, 0.1, -0.02)]
    vel = [(0.0, vc, 0.0), (-vc / math.sqrt(1.2), 0.0, 0.0), (0.0, -vc / math.sqrt(0.9), 1e-4)]
    m = [1e-6, 2e-6, 1.5e-6]
    arr = _state(pos, vel, m)
    ref = [a.copy() for a in arr]
    _kepler_all(ref, 7.0)
    a_osc, rc = np.ones(3), np.full(3, 0.05)
    f, bad = oracle.ml_group(arr, [0, 1, 2], a_osc, rc, G, 1.0, 3.0, 0, 0, 7.0, TOL, L, s)
    assert f == 0 and bad == 0
    assert _rel(arr, ref) < 1e-13


def _binary(d, m, Gc):
    """A circular binary of separation d about (1, 0, 0) on a circular orbit."""
    vc = math.sqrt(Gc)
    w = math.sqrt(Gc * 2 * m / d ** 3)
    c0 = np.array([1.0, 0.0, 0.0])
    u = np.array([0.6, 0.0, 0.8]); vp = np.array([0.0, 1.0, 0.0])
    pos = [c0 + 0.5 * d * u, c0 - 0.5 * d * u]
    vel = [np.array([0, vc, 0]) + 0.5 * d * w * vp, np.array([0, vc, 0]) - 0.5 * d * w * vp]
    return _state(pos, vel, [m, m])


@pytest.mark.parametrize("L,s", [(1, 2), (2, 3), (3, 2)])
def test_deep_binary_is_all_bulirsch_stoer(L, s):
    """Separation 1e-3 au, r_crit 0.2 au: inside 0.1 r_crit / s^L for every
    case.  About one binary period over dt."""
    m, d, dt = 3e-4, 1e-3, 0.5
    a_osc, rc = np.ones(2), np.full(2, 0.2)
    arr = _binary(d, m, G)
    ref = [a.copy() for a in arr]
    assert oracle.bs_group(ref, [0, 1], a_osc, rc, G, 1.0, 3.0, 0, 0, dt, TOL) == 0
    f, bad = oracle.ml_group(arr, [0, 1], a_osc, rc, G, 1.0, 3.0, 0, 0, dt, TOL, L, s)
    assert f == 0 and bad == 0
    # the pair's own motion (1e-3 au, 0.02 au/day) to ~1e-9 of itself
    for c in range(6):
        scale = d if c < 3 else d * math.sqrt(G * 2 * m / d ** 3)
        assert np.abs(arr[c] - ref[c]).max() < 1e-9 * scale, c


def _flyby(q_min, rc, m, dt):
    """Two bodies near (1, 0, 0) (masses m, 2 m) passing each other at q_min
    (z offset) with relative speed 2 rc / dt along y, closest at mid-step."""
    vc = math.sqrt(G)
    u = 2.0 * rc / dt
    pos = [(1.0, 0.0, 0.0), (1.0, -0.5 * u * dt, q_min)]
    vel = [(0.0, vc, 0.0), (0.0, vc + u, 0.0)]
    return _state(pos, vel, [m, 2 * m])


def test_flyby_converges_as_the_substep_shrinks():
    """L = 1 with s = 4 .. 64 sub-steps: 1.5 r_crit / s < 0.85 r_crit, so no
    subgroup forms and level 1 is leapfrog on the (1 - K_0) force; its error
    in the velocities stays below 0.5 / s^2 of the pair impulse (a symmetric
    pass: in fact it falls faster) and goes to zero."""
    rc0, m, dt = 0.02, 1e-5, 10.0
    a_osc, rc = np.ones(2), np.full(2, rc0)
    base = _flyby(0.85 * rc0, rc0, m, dt)
    ref = [a.copy() for a in base]
    oracle.bs_group(ref, [0, 1], a_osc, rc, G, 1.0, 3.0, 0, 0, dt, TOL)
    # impulse of the (1 - K_0) force on body 0 over the drift
    free = [a.copy() for a in base]
    _kepler_all(free, dt)
    dv = np.array([ref[3 + c][0] - free[3 + c][0] for c in range(3)])
    assert np.linalg.norm(dv) > 1e-6            # the level-1 force matters here
    errs = {}
    for s in (4, 8, 16, 32, 64):
        arr = [a.copy() for a in base]
        f, bad = oracle.ml_group(arr, [0, 1], a_osc, rc, G, 1.0, 3.0, 0, 0, dt, TOL, 1, s)
        assert f == 0 and bad == 0
        errs[s] = max(np.abs(arr[3 + c] - ref[3 + c]).max() for c in range(3)) / np.linalg.norm(dv)
        assert errs[s] < 0.5 / s ** 2, (s, errs)
    assert errs[64] < 1e-5


def test_slow_pair_inside_level1_radius():
    """q = 0.3 r_crit, s = 2: inside r_crit,1 = 0.5 r_crit, so the pair is a
    subgroup on the Bulirsch-Stoer level with weight (1 - K_0)(1 - K_1), the
    level-1 kicks carrying (1 - K_0) K_1.  The pair impulse over dt equals the
    single Bulirsch-Stoer drift's to the kicks' splitting error
    (dt / binary period ~ 1/40)."""
    rc0, m, dt, q = 0.02, 1e-5, 1.0, 0.006
    a_osc, rc = np.ones(2), np.full(2, rc0)
    vc = math.sqrt(G)
    base = _state([(1.0, 0.0, 0.0), (1.0, q, 0.0)], [(0.0, vc, 0.0), (-vc * q, vc, 0.0)], [m, 2 * m])
    ref = [a.copy() for a in base]
    oracle.bs_group(ref, [0, 1], a_osc, rc, G, 1.0, 3.0, 0, 0, dt, TOL)
    free = [a.copy() for a in base]
    _kepler_all(free, dt)
    dv = np.array([ref[3 + c][0] - free[3 + c][0] for c in range(3)])
    for L in (1, 2):
        arr = [a.copy() for a in base]
        f, bad = oracle.ml_group(arr, [0, 1], a_osc, rc, G, 1.0, 3.0, 0, 0, dt, TOL, L, 2)
        assert f == 0 and bad == 0
        got = np.array([arr[3 + c][0] - free[3 + c][0] for c in range(3)])
        assert np.linalg.norm(got - dv) < 2e-3 * np.linalg.norm(dv), L


def test_step_without_groups_ignores_the_levels():
    """No encounter pairs and no predicted entries: the levels change nothing."""
    d = discs.disc_uniform(150, 2, a_min=0.8, a_max=1.6)
    arr = oracle.disc_arrays(d)
    a, rc = oracle.rcrit(*arr, G=d.G, Mstar=d.Mstar, dt=d.dt, n1=3.0, n2=0.4)
    pairs, _ = oracle.encounters(arr[0], arr[1], arr[2], arr[6], a, rc, 3.0, d.Mstar, 1)
    assert len(pairs) == 0 and len(oracle.predicted_pairs(arr, a, rc, 3.0, d.Mstar, 1, d.dt)) == 0
    ref = [v.copy() for v in arr]
    oracle.step(ref, d.G, d.Mstar, d.dt, 3.0, 0.4, 1, 0, 1, bs_tol=TOL)
    oracle.step(arr, d.G, d.Mstar, d.dt, 3.0, 0.4, 1, 0, 1, bs_tol=TOL, n_levels=2, n_sub=3)
    for c in range(7):
        assert np.array_equal(arr[c], ref[c])


@pytest.mark.parametrize("mode,form,L,s", [(1, 0, 1, 2), (1, 1, 2, 3), (0, 0, 3, 2), (1, 0, 2, 4)])
@pytest.mark.parametrize("n_big", [-1, 2])
def test_kick_plus_levels_plus_bulirsch_stoer_is_newton(mode, form, L, s, n_big):
    """K_0 (the kick) + the level-l shares + the Bulirsch-Stoer share minus its
    central term = the whole Newtonian pair force, for pairs spread from deep
    inside r_crit / s^L to beyond r_crit; in test-particle mode 2 the pairs of
    two test particles have no share anywhere."""
    rng = np.random.default_rng(7 + mode + 2 * form + 3 * L)
    n = 8
    x = 1.0 + 0.02 * rng.standard_normal(n)
    y = 0.02 * rng.standard_normal(n)
    z = 0.005 * rng.standard_normal(n)
    m = rng.uniform(1e-7, 1e-5, n)
    a = rng.uniform(0.98, 1.02, n)
    rc = rng.uniform(0.005, 0.03, n)
    x[1], y[1], z[1] = x[0] + 2e-4, y[0] - 1e-4, z[0]        # one pair deep inside every radius
    for l in range(1, min(L, 3) + 1):                        # one pair in the band of level l (with a big body)
        i, j = (l - 1) % 2, 2 * l + 1
        rcij = oracle.pair_rcrit(mode, m[i], m[j], a[i], a[j], rc[i], rc[j], 3.0, 1.0)
        sep = 0.6 * rcij / s ** (l - 1)                      # inside r_crit,(l-1), outside r_crit,l for s >= 2
        x[j], y[j], z[j] = x[i] + 0.6 * sep, y[i] + 0.8 * sep, z[i]
    mem = np.arange(n)
    k = oracle.kick_acc(x, y, z, m, a, rc, G, 1.0, 3.0, mode, form, n_big=n_big)
    levels = sum(oracle.ml_level_acc(x, y, z, m, a, rc, mem, G, 1.0, 3.0, mode, form, l, L, s, n_big=n_big)
                 for l in range(1, L + 1))
    bs = oracle.bs_acc_ml(x, y, z, m, a, rc, mem, G, 1.0, 3.0, mode, form, L, s, n_big=n_big)
    pos = np.stack([x, y, z])
    central = -G * pos / np.linalg.norm(pos, axis=0) ** 3
    newton = np.zeros((3, n))
    for i in range(n):
        for j in range(n):
            if i != j and not (n_big >= 0 and i >= n_big and j >= n_big):
                d = pos[:, j] - pos[:, i]
                newton[:, i] += G * m[j] * d / np.linalg.norm(d) ** 3
    got = k + levels + bs - central
    assert np.abs(got - newton).max() <= 1e-13 * np.abs(newton).max()
    # the pairs span every level: some inside 0.1 r_crit / s^L, some between levels, some beyond r_crit
    r = np.linalg.norm(pos[:, :, None] - pos[:, None, :], axis=0)
    rcij = np.array([[oracle.pair_rcrit(mode, m[i], m[j], a[i], a[j], rc[i], rc[j], 3.0, 1.0)
                      for j in range(n)] for i in range(n)])
    q = (r / rcij)[~np.eye(n, dtype=bool)]
    assert (q < 0.1 / s ** L).any() and ((q > 1.0 / s ** L) & (q < 1.0)).any() and (q > 1).any()
    for l in range(1, L + 1):       # every level carries part of the force
        assert np.abs(oracle.ml_level_acc(x, y, z, m, a, rc, mem, G, 1.0, 3.0, mode, form, l, L, s,
                                          n_big=n_big)).max() > 0.0


@pytest.mark.parametrize("level,s", [(1, 2), (1, 4), (2, 3)])
def test_subgroup_pairs_against_brute_force(level, s):
    """The pairs a level-l group forms its subgroups from: inside r_crit / s^l,
    or within 1.5 r_crit / s^l and entering r_crit / s^l on the straight-line
    relative motion within h (a dense time grid stands in for the closed form);
    a ghost (m = -0.0) and, in test-particle mode 2, two test particles never
    pair."""
    rng = np.random.default_rng(11 + level + s)
    n = 60
    h = 6.0 / s ** level
    rcl = 0.01 / s ** level
    sx, sv = 2.5 * rcl, rcl / h                         # a cloud a few r_crit,l wide, crossing r_crit,l in ~h
    arr = [1.0 + sx * rng.standard_normal(n), sx * rng.standard_normal(n), 0.3 * sx * rng.standard_normal(n),
           0.01 + sv * rng.standard_normal(n), 0.017 + sv * rng.standard_normal(n),
           0.3 * sv * rng.standard_normal(n), rng.uniform(1e-7, 1e-6, n)]
    arr[6][5] = -0.0                                    # a ghost
    a, rc = np.ones(n), np.full(n, 0.01)
    mem = np.arange(n)
    n_big = 40
    got = {tuple(p) for p in oracle.ml_subpairs(arr, mem, a, rc, 3.0, 1.0, 0, level, s, h, n_big=n_big)}
    x = np.stack(arr[:3], 1); v = np.stack(arr[3:6], 1)
    ts = np.linspace(0.0, h, 4001)
    want, edge, inside, entering = set(), 0, 0, 0
    for i in range(n):
        for j in range(i + 1, n):
            if i == 5 or j == 5 or (i >= n_big and j >= n_big):
                continue
            d = x[j] - x[i]
            r = np.linalg.norm(d)
            if r < rcl:
                want.add((i, j)); inside += 1
                continue
            if r >= 1.5 * rcl:
                continue
            path = np.linalg.norm(d[None, :] + (v[j] - v[i])[None, :] * ts[:, None], axis=1)
            if abs(path.min() / rcl - 1) < 1e-6:
                edge += 1
                continue
            if path.min() < rcl:
                want.add((i, j)); entering += 1
    assert inside >= 3 and entering >= 3
    assert want <= got and len(got - want) <= edge
    assert all(5 not in p for p in got) and all(not (p[0] >= n_big and p[1] >= n_big) for p in got)


@pytest.mark.parametrize("L,s", [(1, 2), (1, 4), (2, 3), (3, 2)])
def test_hybrid_step_with_levels_resolves_a_close_flyby(L, s):
    """The close flyby of two planets (0.004 au at closest, inside the
    changeover region) over 120 days against an independent DOP853
    integration of the heliocentric equations of motion: with intermediate
    levels the step follows the true motion to ~1e-5 au at dt = 6 d (without
    the close-encounter level the error is ~3e-2 au), and the error falls
    with the step."""
    from tests.test_oracle_bs import _flyby, _truth
    T = 120.0
    ref = _truth(_flyby(), T)
    errs = {}
    for dt in (6.0, 1.5):
        arr = _flyby()
        forced = [0]
        assert oracle.step(arr, G, 1.0, dt, 3.0, 0.4, 1, 0, int(round(T / dt)), bs_tol=TOL, forced=forced,
                           n_levels=L, n_sub=s) == 0
        assert forced[0] == 0
        errs[dt] = np.abs(np.stack(arr[:3], 1) - ref).max()
    assert errs[6.0] < 1e-4
    assert errs[1.5] < errs[6.0] / 3.0
