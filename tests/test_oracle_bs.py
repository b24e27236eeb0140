"""Pins of the oracle's close-encounter level (Sect. 1: level 1 of the hybrid
integrator, a Bulirsch-Stoer integration of each group of encounter pairs
under the central body and the (1 - K) part of the members' pair forces).

None of these calls the CUDA path.  What fixes each part:

* groups: connected components, against the transitive closure of the pair
  graph worked out with boolean matrix products;
* the level-1 force: kick (K part) + level 1 (1 - K part) - central term is
  Newton's pair force for every pair of a group, and test-particle pairs
  (mode 2) have none;
* the integrator: Kepler's equation solved by 40-digit bisection for massless
  members; the closed-form circular orbit of two bodies about each other;
  energy and angular momentum of a three-body group with K = 0; time
  reversal;
* the hybrid step: a close flyby of two planets against an independent
  high-accuracy integration of the heliocentric equations of motion (scipy
  DOP853), where the step without the level is wrong at the 1e-2 au level.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2309_08217_gb300 import discs

G = discs.G_GAUSS


# ------------------------------------------------------------- groups ---
def _closure_components(N, pairs):
    A = np.eye(N, dtype=bool)
    for i, j in pairs:
        A[i, j] = A[j, i] = True
    while True:
        B = (A.astype(np.int64) @ A.astype(np.int64)) > 0
        if np.array_equal(A, B):
            break
        A = B
    touched = np.zeros(N, bool)
    for i, j in pairs:
        touched[i] = touched[j] = True
    label = np.full(N, -1)
    for v in range(N):
        if touched[v]:
            label[v] = int(np.argmax(A[v]))       # smallest index reachable from v
    return label


@pytest.mark.parametrize("seed", range(8))
def test_groups_are_the_transitive_closure(seed):
    rng = np.random.default_rng(seed)
    N = int(rng.integers(2, 40))
    npairs = int(rng.integers(0, 2 * N))
    pairs = []
    for _ in range(npairs):
        i, j = sorted(rng.choice(N, 2, replace=False))
        pairs.append((int(i), int(j)))
    label, ng = oracle.groups(N, pairs)
    ref = _closure_components(N, pairs)
    assert np.array_equal(label, ref)
    assert ng == len({v for v in ref if v >= 0})


def test_groups_chain_and_empty():
    label, ng = oracle.groups(6, [])
    assert ng == 0 and np.all(label == -1)
    # a chain listed from its far end joins into one group rooted at 0
    label, ng = oracle.groups(6, [(4, 5), (3, 4), (2, 3), (0, 2)])
    assert ng == 1 and label.tolist() == [0, -1, 0, 0, 0, 0]


# ---------------------------------------------------- the level-1 force ---
@pytest.mark.parametrize("mode,form", [(0, 0), (1, 0), (1, 1)])
def test_kick_plus_level1_is_newton(mode, form):
    """K (kick) + (1 - K) (level 1) = the whole pair force, for pairs spread
    over K = 0, the changeover region and K = 1."""
    rng = np.random.default_rng(3 + mode + 2 * form)
    n = 6
    x = 1.0 + 0.02 * rng.standard_normal(n)
    y = 0.02 * rng.standard_normal(n)
    z = 0.005 * rng.standard_normal(n)
    m = rng.uniform(1e-7, 1e-5, n)
    a = rng.uniform(0.98, 1.02, n)
    rc = rng.uniform(0.005, 0.03, n)
    mem = np.arange(n)
    k = oracle.kick_acc(x, y, z, m, a, rc, G, 1.0, 3.0, mode, form)
    lv = oracle.bs_acc(x, y, z, m, a, rc, mem, G, 1.0, 3.0, mode, form)
    pos = np.stack([x, y, z])
    central = -G * pos / np.linalg.norm(pos, axis=0) ** 3
    newton = np.zeros((3, n))
    for i in range(n):
        for j in range(n):
            if i != j:
                d = pos[:, j] - pos[:, i]
                newton[:, i] += G * m[j] * d / np.linalg.norm(d) ** 3
    got = k + lv - central
    assert np.abs(got - newton).max() <= 1e-13 * np.abs(newton).max()
    # the test draws pairs on both sides of the changeover region
    r = np.linalg.norm(pos[:, :, None] - pos[:, None, :], axis=0)
    rcij = np.array([[oracle.pair_rcrit(mode, m[i], m[j], a[i], a[j], rc[i], rc[j], 3.0, 1.0)
                      for j in range(n)] for i in range(n)])
    q = (r / rcij)[~np.eye(n, dtype=bool)]
    assert (q < 1).any() and (q > 1).any()


def test_level1_test_particle_pairs_have_no_force():
    x = np.array([1.0, 1.001, 1.002]); y = np.array([0.0, 0.001, -0.001]); z = np.zeros(3)
    m = np.array([1e-5, 1e-9, 1e-9]); a = np.ones(3); rc = np.full(3, 0.1)
    mem = [0, 1, 2]
    tp = oracle.bs_acc(x, y, z, m, a, rc, mem, G, 1.0, 3.0, 0, 0, n_big=1)
    pos = np.stack([x, y, z])
    central = -G * pos / np.linalg.norm(pos, axis=0) ** 3
    # test particles 1 and 2 feel only body 0 (K = 0 at these distances)
    for i in (1, 2):
        d = pos[:, 0] - pos[:, i]
        assert np.allclose(tp[:, i] - central[:, i], G * m[0] * d / np.linalg.norm(d) ** 3,
                           rtol=1e-13, atol=0)
    full = oracle.bs_acc(x, y, z, m, a, rc, mem, G, 1.0, 3.0, 0, 0, n_big=-1)
    assert np.allclose(tp[:, 0], full[:, 0], rtol=1e-15, atol=0)   # body 0 feels both


# ------------------------------------------------------ the integrator ---
def _two_massless(s0, s1_far):
    arr = [np.array([s0[c], s1_far[c]]) for c in range(6)] + [np.zeros(2)]
    return arr


@pytest.mark.parametrize("e,dt", [(0.1, 40.0), (0.6, 150.0)])
def test_bs_massless_members_follow_kepler(e, dt):
    mpmath = pytest.importorskip("mpmath")
    from tests.test_oracle_pins import _mp_state_elliptic, _rotate
    mpmath.mp.dps = 40
    mu, a = G, 1.7
    n = math.sqrt(mu / a ** 3)
    ss0, ss1 = [], []
    for k, (M0, rot) in enumerate([(1.0, (0.3, 1.1, 0.4)), (2.2, (0.1, 0.5, 2.0))]):
        ss0.append(_rotate(_mp_state_elliptic(mpmath.mpf(mu), mpmath.mpf(a), mpmath.mpf(e),
                                              mpmath.mpf(M0)), *rot))
        ss1.append(_rotate(_mp_state_elliptic(mpmath.mpf(mu), mpmath.mpf(a), mpmath.mpf(e),
                                              mpmath.mpf(M0) + mpmath.mpf(n) * dt), *rot))
    arr = [np.array([ss0[0][c], ss0[1][c]]) for c in range(6)] + [np.zeros(2)]
    forced = oracle.bs_group(arr, [0, 1], np.ones(2), np.full(2, 10.0), G, 1.0, 3.0, 0, 0, dt, 1e-13)
    assert forced == 0
    for k in range(2):
        got = np.array([arr[c][k] for c in range(6)])
        assert np.abs(got[:3] - ss1[k][:3]).max() <= 1e-11 * np.abs(ss1[k][:3]).max()
        assert np.abs(got[3:] - ss1[k][3:]).max() <= 1e-11 * np.abs(ss1[k][3:]).max()


def test_bs_two_bodies_circular_about_each_other():
    """A negligible central mass: the pair turns rigidly at w = sqrt(G (m1 + m2) / d^3)
    about its centre of mass, which drifts at the centre-of-mass velocity."""
    Gc, m, d = 1.0, 1e-3, 0.01
    Ms = 1e-20
    w = math.sqrt(Gc * 2 * m / d ** 3)
    c0 = np.array([1.0, 0.5, 0.2]); V = np.array([0.01, -0.02, 0.005])
    u = np.array([0.6, 0.8, 0.0]); wv = np.array([0.0, 0.0, 1.0])
    vperp = np.cross(wv, u)
    r0 = [c0 + 0.5 * d * u, c0 - 0.5 * d * u]
    v0 = [V + 0.5 * d * w * vperp, V - 0.5 * d * w * vperp]
    arr = [np.array([r0[0][c], r0[1][c]]) for c in range(3)] + \
          [np.array([v0[0][c], v0[1][c]]) for c in range(3)] + [np.full(2, m)]
    t = 0.1
    forced = oracle.bs_group(arr, [0, 1], np.ones(2), np.full(2, 1.0), Gc, Ms, 3.0, 0, 0, t, 1e-13)
    assert forced == 0
    ut = math.cos(w * t) * u + math.sin(w * t) * vperp
    ct = c0 + V * t
    for k, sgn in enumerate((1.0, -1.0)):
        pos = np.array([arr[c][k] for c in range(3)])
        vel = np.array([arr[c][k] for c in range(3, 6)])
        want_p = ct + sgn * 0.5 * d * ut
        want_v = V + sgn * 0.5 * d * w * np.cross(wv, ut)
        assert np.abs(pos - want_p).max() <= 1e-12 * np.linalg.norm(want_p)
        assert np.abs(vel - want_v).max() <= 1e-10 * np.linalg.norm(want_v)


def _three_close(seed=5, spread=0.02):
    """Three bodies of a few Earth masses about 0.02 au apart near 1 au."""
    rng = np.random.default_rng(seed)
    pos, vel = discs.elements_to_cartesian(G * np.ones(3), np.array([1.0, 1.004, 0.997]),
                                           np.array([0.01, 0.02, 0.015]), np.array([0.001, 0.002, 0.0]),
                                           np.array([0.1, 0.1, 0.1]), np.array([0.2, 0.2, 0.2]),
                                           np.array([0.0, spread, -spread]))
    m = rng.uniform(1e-6, 5e-6, 3)
    return [pos[0].copy(), pos[1].copy(), pos[2].copy(), vel[0].copy(), vel[1].copy(), vel[2].copy(), m]


def _level1_energy(arr, Ms=1.0):
    x = np.stack(arr[:3]); v = np.stack(arr[3:6]); m = arr[6]
    E = 0.5 * (m * (v ** 2).sum(0)).sum() - (G * Ms * m / np.linalg.norm(x, axis=0)).sum()
    for i in range(len(m)):
        for j in range(i + 1, len(m)):
            E -= G * m[i] * m[j] / np.linalg.norm(x[:, i] - x[:, j])
    L = (m * np.cross(x.T, v.T).T).sum(1)
    return E, L


def test_bs_group_with_k_zero_conserves_energy_and_momentum():
    """With K = 0 (r_crit far beyond the group) level 1 is the three-body
    problem about a fixed central mass: E and L are constants of motion.
    (The error control is relative to each member's heliocentric |x| and |v|,
    so a tight binary inside a group keeps its internal energy less well:
    members about 0.02 au apart keep E to 1e-13 here.)"""
    arr = _three_close()
    E0, L0 = _level1_energy(arr)
    for _ in range(5):
        assert oracle.bs_group(arr, [0, 1, 2], np.ones(3), np.full(3, 100.0), G, 1.0, 3.0, 0, 0,
                               30.0, 1e-13) == 0
    E1, L1 = _level1_energy(arr)
    assert abs(E1 / E0 - 1) < 1e-12
    assert np.abs(L1 - L0).max() < 1e-12 * np.linalg.norm(L0)


def test_bs_time_reversal():
    arr = _three_close(9)
    start = [a.copy() for a in arr]
    a_osc, rc = np.ones(3), np.full(3, 0.01)           # a changeover region inside the group
    assert oracle.bs_group(arr, [0, 1, 2], a_osc, rc, G, 1.0, 3.0, 0, 0, 25.0, 1e-13) == 0
    moved = max(np.abs(arr[c] - start[c]).max() for c in range(3))
    assert moved > 1e-3
    assert oracle.bs_group(arr, [0, 1, 2], a_osc, rc, G, 1.0, 3.0, 0, 0, -25.0, 1e-13) == 0
    for c in range(6):
        assert np.abs(arr[c] - start[c]).max() <= 1e-11 * np.abs(start[c]).max()


def test_bs_forced_acceptance_is_reported():
    # a negative tolerance is never met: every sub-step halves down to the
    # floor, and the attempt limit then covers the rest of the drift at once
    arr = _three_close(2)
    assert oracle.bs_group(arr, [0, 1, 2], np.ones(3), np.full(3, 100.0), G, 1.0, 3.0, 0, 0,
                           30.0, -1.0) == 1
    assert all(np.isfinite(c).all() for c in arr)


# ------------------------------------------------------ the hybrid step ---
def _flyby():
    """Planet 0 on a circular orbit at 1 au; planet 1 starts 0.05 au behind it
    along the track, 0.004 au further out, 1.2e-3 au/day faster: a close
    flyby inside the three-mutual-Hill-radius changeover region."""
    m = np.array([3e-6, 3e-6])
    x0 = np.array([1.0, 0.0, 0.0]); v0 = np.array([0.0, math.sqrt(G * (1 + m[0])), 0.0])
    x1 = x0 + np.array([0.004, -0.05, 0.0]); v1 = v0 + np.array([0.0, 1.2e-3, 0.0])
    xs, vh = np.stack([x0, x1]), np.stack([v0, v1])
    vb = vh - (m[:, None] * vh).sum(0) / (1 + m.sum())
    return [xs[:, 0].copy(), xs[:, 1].copy(), xs[:, 2].copy(),
            vb[:, 0].copy(), vb[:, 1].copy(), vb[:, 2].copy(), m]


def _truth(arr, T):
    solve_ivp = pytest.importorskip("scipy.integrate").solve_ivp
    x = np.stack(arr[:3], 1); vb = np.stack(arr[3:6], 1); m = arr[6]
    vh = vb + (m[:, None] * vb).sum(0)          # M* = 1: v_hel = v_bary + P / M*

    def f(t, s):
        r = s[:6].reshape(2, 3); v = s[6:].reshape(2, 3)
        acc = np.zeros((2, 3))
        for i in range(2):      # heliocentric equations of motion
            acc[i] -= G * (1 + m[i]) * r[i] / np.linalg.norm(r[i]) ** 3
            j = 1 - i
            d = r[j] - r[i]
            acc[i] += G * m[j] * (d / np.linalg.norm(d) ** 3 - r[j] / np.linalg.norm(r[j]) ** 3)
        return np.concatenate([v.ravel(), acc.ravel()])

    sol = solve_ivp(f, (0.0, T), np.concatenate([x.ravel(), vh.ravel()]), method="DOP853",
                    rtol=1e-13, atol=1e-16)
    return sol.y[:6, -1].reshape(2, 3)


def test_hybrid_step_resolves_a_close_flyby():
    T = 120.0
    ref = _truth(_flyby(), T)
    errs = {}
    for dt in (6.0, 1.5):
        for tol in (0.0, 1e-12):
            arr = _flyby()
            forced = [0]
            assert oracle.step(arr, G, 1.0, dt, 3.0, 0.4, 1, 0, int(round(T / dt)), bs_tol=tol,
                               forced=forced) == 0
            assert forced[0] == 0
            errs[dt, tol] = np.abs(np.stack(arr[:3], 1) - ref).max()
    # without the level the flyby's inner part is missing: wrong at 1e-2 au
    assert errs[6.0, 0.0] > 1e-2 and errs[1.5, 0.0] > 1e-2
    # with it the step follows the true motion, better than first order in dt
    assert errs[6.0, 1e-12] < 1e-3 * errs[6.0, 0.0]
    assert errs[1.5, 1e-12] < errs[6.0, 1e-12] / 6.0


def test_hybrid_step_without_encounters_is_the_level0_step():
    from tests.test_oracle_pins import _two_planets
    a, b = _two_planets(), _two_planets()
    assert oracle.step(a, G, 1.0, 6.0, 3.0, 0.4, 1, 0, 50) == 0
    assert oracle.step(b, G, 1.0, 6.0, 3.0, 0.4, 1, 0, 50, bs_tol=1e-12) == 0
    for u, v in zip(a, b):
        assert np.array_equal(u, v)


# ------------------------------------------------- predicted entries ---
def test_predicted_pairs_against_brute_force():
    """Pairs outside r_crit (but within 1.5 r_crit) whose straight-line
    relative motion over the drift enters r_crit: a dense grid of times
    t in [0, dt] stands in for the closed-form closest approach."""
    d = discs.disc_uniform(2000, 21, a_min=0.97, a_max=1.03)
    arr = oracle.disc_arrays(d)
    a, rc = oracle.rcrit(*arr, G=d.G, Mstar=d.Mstar, dt=d.dt)
    got = {tuple(p) for p in oracle.predicted_pairs(arr, a, rc, 3.0, d.Mstar, 1, d.dt)}
    x = np.stack(arr[:3], 1); v = np.stack(arr[3:6], 1); m = arr[6]
    ts = np.linspace(0.0, d.dt, 4001)
    want, near_edge = set(), 0
    for i in range(d.N):
        dd = x[i + 1:] - x[i]
        r = np.linalg.norm(dd, axis=1)
        for k in np.nonzero(r < 2.0 * 0.02)[0]:
            j = i + 1 + k
            rcij = oracle.pair_rcrit(1, m[i], m[j], a[i], a[j], rc[i], rc[j], 3.0, d.Mstar)
            if not (rcij <= r[k] < 1.5 * rcij):
                continue
            path = np.linalg.norm(dd[k][None, :] + (v[j] - v[i])[None, :] * ts[:, None], axis=1)
            if abs(path.min() / rcij - 1) < 1e-6:
                near_edge += 1          # the grid cannot decide these
                continue
            if path.min() < rcij:
                want.add((i, j))
    got_clear = {p for p in got}
    assert len(want) >= 3
    assert want <= got_clear and len(got_clear - want) <= near_edge


def test_step_size_control_trace():
    """The sub-step control on a case its rules decide by hand: two massless
    bodies in free space (straight lines, so every column extrapolates the
    exact motion and column 1 is accepted), 0.01 au apart with relative speed
    8 x 0.01 au / dt.  The first sub-step is the largest binary fraction with
    f dt |v_ij| <= r_ij: dt/8; each acceptance by column <= 2 doubles the next,
    clipped to what is left: dt/8, dt/4, dt/2, dt/8 -- four sub-steps, no
    rejections, and the exact straight-line end state."""
    dt = 8.0
    x0 = [np.array([1.0, 1.01]), np.zeros(2), np.zeros(2)]
    v0 = [np.zeros(2), np.array([0.0, 0.01]), np.zeros(2)]
    arr = [a.copy() for a in x0 + v0] + [np.zeros(2)]
    f, accepted, attempts = oracle.bs_group_counted(arr, [0, 1], np.ones(2), np.zeros(2), 1.0, 1e-20, 3.0, 1, 0,
                                                   dt, 1e-12)
    assert (f, accepted, attempts) == (0, 4, 4)
    for c in range(3):
        np.testing.assert_allclose(arr[c], x0[c] + v0[c] * dt, rtol=0, atol=1e-15)
        np.testing.assert_allclose(arr[3 + c], v0[c], rtol=0, atol=1e-15)


def test_attempt_limit_completes_the_remaining_time_on_kepler_orbits():
    """A tolerance no column can meet (except where the columns agree to the
    last bit): the sub-steps are halved to the floor (dt 2^-30) and accepted
    there as forced, 4,096 attempts pass, and the
    members drift the rest of dt on their Kepler orbits (straight lines in
    free space).  Momentum is conserved by both parts, so the centre of mass
    ends at c0 + V dt exactly as a uniform motion -- a completion over the
    whole dt instead of the remainder would overshoot by V times the time
    already integrated."""
    Gc, Ms, dt = 1.0, 1e-20, 8.0
    m = np.array([1e-3, 2e-3])
    V = np.array([0.05, -0.02, 0.01])
    x0 = np.array([[1.0, 2.0, 0.5], [1.01, 2.0, 0.5]])
    v0 = np.array([V + [0.0, 0.001, 0.0], V - [0.0, 0.0005, 0.0]])
    arr = [x0[:, c].copy() for c in range(3)] + [v0[:, c].copy() for c in range(3)] + [m.copy()]
    f, accepted, attempts = oracle.bs_group_counted(arr, [0, 1], np.ones(2), np.full(2, 1.0), Gc, Ms, 3.0, 0, 0,
                                                   dt, 1e-300)
    assert f == 1 and attempts == 4096 and 0 < accepted < 4096
    c0 = (m[:, None] * x0).sum(0) / m.sum()
    cend = np.array([(m * arr[c]).sum() / m.sum() for c in range(3)])
    vcm = (m[:, None] * v0).sum(0) / m.sum()
    assert np.abs(cend - (c0 + vcm * dt)).max() < 1e-10      # rounding of 4,096 forced sub-steps: ~1e-12


def test_predicted_pairs_of_two_test_particles_are_dropped():
    """Test-particle mode 2: a pair of two test particles is never an entry
    (it has no force), while the same disc without the mode has such pairs."""
    d = discs.disc_uniform(2000, 21, a_min=0.97, a_max=1.03)
    arr = oracle.disc_arrays(d)
    a, rc = oracle.rcrit(*arr, G=d.G, Mstar=d.Mstar, dt=d.dt)
    n_big = 1000
    every = oracle.predicted_pairs(arr, a, rc, 3.0, d.Mstar, 1, d.dt)
    tp = oracle.predicted_pairs(arr, a, rc, 3.0, d.Mstar, 1, d.dt, n_big=n_big)
    both = [(i, j) for i, j in every if i >= n_big and j >= n_big]
    assert len(both) >= 1
    assert {tuple(p) for p in tp} == {tuple(p) for p in every} - set(both)


def _fast_pass():
    """Two Earth-mass planets near 1 au: planet 1 starts 1.3 r_crit behind
    planet 0 (three mutual Hill radii), 0.3 r_crit outward, 0.01 au/day
    faster -- it passes at 0.3 r_crit and leaves r_crit again within 10 days."""
    m = np.array([3e-6, 3e-6])
    rc = 3.0 * (2 * 3e-6 / 3.0) ** (1 / 3)
    b, v = 0.3 * rc, 0.01
    s0 = math.sqrt((1.3 * rc) ** 2 - b ** 2)
    x0 = np.array([1.0, 0.0, 0.0]); v0 = np.array([0.0, math.sqrt(G * (1 + m[0])), 0.0])
    x1 = x0 + np.array([b, -s0, 0.0]); v1 = v0 + np.array([0.0, v, 0.0])
    xs, vh = np.stack([x0, x1]), np.stack([v0, v1])
    vb = vh - (m[:, None] * vh).sum(0) / (1 + m.sum())
    return [xs[:, 0].copy(), xs[:, 1].copy(), xs[:, 2].copy(), vb[:, 0].copy(), vb[:, 1].copy(), vb[:, 2].copy(), m]


def test_a_pass_within_one_step_is_grouped_by_its_predicted_entry():
    """With dt = 12 d the pair is outside r_crit at both step starts, so only
    the predicted entry (R10) puts it into a group: the step then follows the
    independent DOP853 integration 5x better than without the level, where
    the whole pass keeps only its K part."""
    T, dt = 24.0, 12.0
    ref = _truth(_fast_pass(), T)
    errs = {}
    for tol in (0.0, 1e-12):
        arr = _fast_pass()
        forced = [0]
        assert oracle.step(arr, G, 1.0, dt, 3.0, 0.4, 1, 0, 2, bs_tol=tol, forced=forced) == 0
        assert forced[0] == 0
        errs[tol] = np.abs(np.stack(arr[:3], 1) - ref).max()
    assert errs[1e-12] < 0.3 * errs[0.0]
