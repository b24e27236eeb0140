"""The intermediate levels of the changeover on the GPU (genga_step with
bs_tol > 0 and n_levels > 0) against the oracle's recursion.

Both sides take the same subgroup decisions (correctly rounded comparisons)
and integrate with the same algorithm, so the states agree to the rounding
differences of the two FP64 evaluations carried through the levels, as for
the Bulirsch-Stoer level alone: 1e-10 of each body's |x| and |v| with FP64
kicks, 1e-9 with FP32 kicks.  On these cases the levels move the states by
1e-7 (planted pairs) to 1e-3 (the swarm) from the drift without levels, so
the bar tests the level path itself.  Cases: planted orbiting pairs at 0.05
to 1.1 of the changeover scale for (L, s) = (1, 2), (1, 4), (2, 3), (3, 2);
a planet with 80 bodies around it (groups wider than a warp, in test-particle
mode 2 too); mergers at the deepest level; a batch of systems; without groups
the levels change nothing; invalid settings are rejected.
"""
import numpy as np
import pytest

import oracle
from paper_2309_08217_gb300 import discs
from tests.gpu_cases import check_merged, orbiting_pairs_disc, planted_disc
from tests.test_gpu_bs import _rel_state, _swarm

pytestmark = pytest.mark.gpu

TOL_BS = 1e-12


def _params(g, d, precision, L, s, n_big=-1, r_in=0.0, r_out=0.0):
    return g.make_params(G=d.G, Mstar=d.Mstar, dt=d.dt, n1=3.0, n2=0.4,
                         rcrit_mode=g.GENGA_RCRIT_MUTUAL_HILL, changeover=g.GENGA_K_CHAMBERS,
                         precision=precision, n_big=n_big, bs_tol=TOL_BS, r_in=r_in, r_out=r_out,
                         n_levels=L, n_sub=s)


@pytest.fixture(scope="module")
def ctx(genga):
    c = genga.Context(20_000)
    yield c
    c.close()


def _oracle_step(d, steps, L, s, n_big=-1, radius=None, dead=None, merges=None):
    arr = oracle.disc_arrays(d)
    forced = [0]
    assert oracle.step(arr, d.G, d.Mstar, d.dt, 3.0, 0.4, 1, 0, steps, n_big=n_big, bs_tol=TOL_BS, forced=forced,
                       radius=radius, dead=dead, merges=merges, n_levels=L, n_sub=s) == 0
    assert forced[0] == 0
    return arr


@pytest.mark.parametrize("L,s", [(1, 2), (1, 4), (2, 3), (3, 2)])
@pytest.mark.parametrize("precision", [0, 1])
def test_step_parity(genga, ctx, precision, L, s):
    d = orbiting_pairs_disc(800, 17)
    st = genga.DeviceSystem.from_disc(d)
    genga.genga_step(ctx, st, _params(genga, d, precision, L, s), 3)
    assert genga.genga_get_status(ctx) == genga.GENGA_OK
    ref = _oracle_step(d, 3, L, s)
    assert _rel_state(st.numpy(), ref) < (1e-10 if precision == 0 else 1e-9)


@pytest.mark.parametrize("n_big", [-1, 1])
def test_large_group_parity(genga, ctx, n_big):
    d = _swarm()
    st = genga.DeviceSystem.from_disc(d)
    genga.genga_step(ctx, st, _params(genga, d, 0, 2, 2, n_big=n_big), 2)
    assert genga.genga_get_status(ctx) == genga.GENGA_OK
    ref = _oracle_step(d, 2, 2, 2, n_big=n_big)
    assert _rel_state(st.numpy(), ref) < 1e-10


def test_mergers_at_the_deepest_level(genga, ctx):
    """planted_disc's closest pair starts at rest relative to each other and
    falls in: it merges on the Bulirsch-Stoer level below two levels."""
    d = planted_disc(800, 17)
    R = np.full(d.N, 2e-5)
    st = genga.DeviceSystem.from_disc(d, radius=R)
    genga.genga_step(ctx, st, _params(genga, d, 0, 2, 2), 3)
    assert genga.genga_get_status(ctx) == genga.GENGA_OK
    Ro, dead, merges = R.copy(), np.zeros(d.N, np.int32), [0]
    ref = _oracle_step(d, 3, 2, 2, radius=Ro, dead=dead, merges=merges)
    got = st.numpy()
    assert merges[0] >= 1 and dead[1] == 1
    assert np.array_equal(np.signbit(got[6]), dead == 1)
    np.testing.assert_allclose(got[6], ref[6], rtol=1e-15, atol=0)
    np.testing.assert_allclose(st.radius_numpy(), Ro, rtol=1e-14, atol=0)
    check_merged(got, ref, dead, 1e-10, {1: 0}, m0=d.m, dt=d.dt)


def test_batched_step_parity(genga):
    sizes = [900, 333, 1200]
    parts = [orbiting_pairs_disc(n, 90 + k) for k, n in enumerate(sizes)]
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    arrays = [np.concatenate([p.arrays()[c] for p in parts]) for c in range(7)]
    c = genga.Context(4000)
    st = genga.DeviceSystem.from_arrays(arrays)
    genga.genga_step_batched(c, st, offsets, _params(genga, parts[0], 1, 1, 3), 3)
    assert genga.genga_get_status(c) == genga.GENGA_OK
    got = st.numpy()
    for k, d in enumerate(parts):
        lo, hi = int(offsets[k]), int(offsets[k + 1])
        ref = _oracle_step(d, 3, 1, 3)
        assert _rel_state([g[lo:hi] for g in got], ref) < 1e-9, f"system {k}"
    c.close()


def test_graph_replay_equals_step_by_step(genga):
    """16 steps: the captured graph (with its level launches) against the
    same steps launched one by one -- bit for bit."""
    d = orbiting_pairs_disc(1500, 71)
    a, b = genga.Context(1500), genga.Context(1500)
    genga.genga_set_step_graphs(b, False)
    sa, sb = genga.DeviceSystem.from_disc(d), genga.DeviceSystem.from_disc(d)
    p = _params(genga, d, 1, 2, 3)
    genga.genga_step(a, sa, p, 16)
    genga.genga_step(b, sb, p, 16)
    assert genga.genga_get_status(a) == genga.GENGA_OK and genga.genga_get_status(b) == genga.GENGA_OK
    ga, gb = sa.numpy(), sb.numpy()
    for c in range(7):
        assert np.array_equal(ga[c], gb[c])
    a.close()
    b.close()


def test_without_groups_the_levels_change_nothing(genga, ctx):
    d = discs.disc_uniform(150, 2, a_min=0.8, a_max=1.6)
    s0, s1 = genga.DeviceSystem.from_disc(d), genga.DeviceSystem.from_disc(d)
    genga.genga_step(ctx, s0, _params(genga, d, 0, 0, 2), 2)
    genga.genga_step(ctx, s1, _params(genga, d, 0, 3, 4), 2)
    assert genga.genga_get_status(ctx) == genga.GENGA_OK
    g0, g1 = s0.numpy(), s1.numpy()
    for c in range(7):
        assert np.array_equal(g0[c], g1[c])


@pytest.mark.parametrize("L,s,tol", [(4, 2, TOL_BS), (1, 1, TOL_BS), (1, 17, TOL_BS), (-1, 2, TOL_BS), (1, 2, 0.0)])
def test_invalid_level_settings_rejected(genga, ctx, L, s, tol):
    d = planted_disc(10, 1)
    st = genga.DeviceSystem.from_disc(d)
    p = _params(genga, d, 0, L, s)
    p.bs_tol = tol
    with pytest.raises(genga.GengaError):
        genga.genga_step(ctx, st, p, 1)


def test_tune_levels_times_candidates_without_touching_the_state(genga, ctx):
    d = orbiting_pairs_disc(1500, 5)
    st = genga.DeviceSystem.from_disc(d)
    before = st.numpy()
    p = _params(genga, d, 1, 0, 2)
    cand = [(0, 2), (1, 2), (2, 3)]
    best, ms = genga.genga_tune_levels(ctx, st, p, cand, 4)
    assert genga.genga_get_status(ctx) == genga.GENGA_OK
    assert best in cand and len(ms) == 3 and all(m > 0.0 for m in ms)
    assert ms[cand.index(best)] == min(ms)
    after = st.numpy()
    for c in range(7):
        assert np.array_equal(before[c], after[c])
    # the tuned setting steps on like the oracle
    p.n_levels, p.n_sub = best
    genga.genga_step(ctx, st, p, 2)
    assert genga.genga_get_status(ctx) == genga.GENGA_OK
    assert _rel_state(st.numpy(), _oracle_step(d, 2, best[0], best[1])) < 1e-9
    with pytest.raises(genga.GengaError):
        genga.genga_tune_levels(ctx, st, p, [(1, 2), (4, 2)], 2)


def test_tune_levels_skips_candidates_that_raise_a_status(genga, ctx):
    # every trial meets the head-on singularity (no radii): a forced sub-step in
    # each candidate, so the fastest comes back and the status stays raised
    d = planted_disc(800, 17)
    st = genga.DeviceSystem.from_disc(d)
    p = _params(genga, d, 1, 0, 2)
    codes = []
    best, ms = genga.genga_tune_levels(ctx, st, p, [(0, 2), (1, 2)], 3, codes=codes)
    assert len(codes) == 2 and all(k != genga.GENGA_OK for k in codes) and genga.GENGA_ERR_BS in codes
    assert ms[[(0, 2), (1, 2)].index(best)] == min(ms)
    assert genga.genga_get_status(ctx) != genga.GENGA_OK
    # a dense swarm: a candidate whose trial raised a status is never the one chosen
    dsw = discs.workload("swarm4k")
    c = genga.Context(dsw.N)
    ssw = genga.DeviceSystem.from_disc(dsw)
    codes = []
    cand = [(0, 2), (2, 4)]
    best, ms = genga.genga_tune_levels(c, ssw, _params(genga, dsw, 1, 0, 2), cand, 4, codes=codes)
    assert codes[1] == 0 and codes[cand.index(best)] == 0
    assert genga.genga_get_status(c) == genga.GENGA_OK
    c.close()


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-9)])
def test_swarm4k_parity(genga, precision, tol):
    """The benchmark's dense case: a planet with 80 planetesimals around it in
    a 4,000-body disc (one 85-member group), 2 levels of 4 sub-steps, 2 steps."""
    d = discs.workload("swarm4k")
    c = genga.Context(d.N)
    st = genga.DeviceSystem.from_disc(d)
    genga.genga_step(c, st, _params(genga, d, precision, 2, 4), 2)
    assert genga.genga_get_status(c) == genga.GENGA_OK
    assert _rel_state(st.numpy(), _oracle_step(d, 2, 2, 4)) < tol
    c.close()


@pytest.mark.parametrize("L,s", [(1, 3), (2, 2)])
def test_kick_then_drift_parity(genga, ctx, L, s):
    """genga_kick then genga_drift with levels against the oracle's kick and
    drift of the groups of the kick's pairs and predicted entries."""
    d = orbiting_pairs_disc(800, 17)
    st = genga.DeviceSystem.from_disc(d)
    p = _params(genga, d, 0, L, s)
    genga.genga_kick(ctx, st, p, 0.5 * d.dt)
    genga.genga_drift(ctx, st, p, d.dt)
    assert genga.genga_get_status(ctx) == genga.GENGA_OK
    arr = oracle.disc_arrays(d)
    a, rc = oracle.rcrit(*arr, G=d.G, Mstar=d.Mstar, dt=d.dt)
    pairs, _ = oracle.encounters(arr[0], arr[1], arr[2], arr[6], a, rc, 3.0, d.Mstar, 1)
    pred = oracle.predicted_pairs(arr, a, rc, 3.0, d.Mstar, 1, d.dt)
    oracle.kick(arr, d.G, d.Mstar, d.dt, 3.0, 0.4, 1, 0, 0.5 * d.dt)
    bad, forced = oracle.drift_groups(arr, a, rc, np.concatenate([pairs, pred]), d.G, d.Mstar, 3.0, 1, 0, d.dt,
                                      TOL_BS, n_levels=L, n_sub=s)
    assert bad == 0 and forced == 0
    assert _rel_state(st.numpy(), arr) < 1e-10


def test_disc40k_drift_with_levels(genga):
    """The 40,000-body benchmark disc in the benchmark's launch configuration:
    an FP32 kick of length 0 (the pair lists of the state, velocities
    unchanged), then the drift with 2 levels of 3 sub-steps, against the
    oracle's lists and level drift of the same state -- every body."""
    d = discs.workload("disc40k")
    c = genga.Context(d.N)
    st = genga.DeviceSystem.from_disc(d)
    p = _params(genga, d, 1, 2, 3)
    genga.genga_kick(c, st, p, 0.0)
    genga.genga_drift(c, st, p, d.dt)
    assert genga.genga_get_status(c) == genga.GENGA_OK
    c.close()
    arr = oracle.disc_arrays(d)
    a, rc = oracle.rcrit(*arr, G=d.G, Mstar=d.Mstar, dt=d.dt)
    pairs, _ = oracle.encounters(arr[0], arr[1], arr[2], arr[6], a, rc, 3.0, d.Mstar, 1)
    pred = oracle.predicted_pairs(arr, a, rc, 3.0, d.Mstar, 1, d.dt)
    assert len(pairs) > 50
    bad, forced = oracle.drift_groups(arr, a, rc, np.concatenate([pairs, pred]), d.G, d.Mstar, 3.0, 1, 0, d.dt,
                                      TOL_BS, n_levels=2, n_sub=3)
    assert bad == 0 and forced == 0
    got = st.numpy()
    members = np.unique(np.concatenate([pairs, pred]).ravel())
    others = np.setdiff1d(np.arange(d.N), members)
    assert _rel_state(got, arr, others) < 1e-12
    assert _rel_state(got, arr, members) < 1e-10
