"""The close-encounter level on the GPU (genga_drift / genga_step with
bs_tol > 0) against the oracle's groups and Bulirsch-Stoer integration.

Members of a group are integrated with the same algorithm and constants on
both sides, so the states agree to the rounding differences of the two FP64
evaluations (sqrt and division order, FMA contraction) carried through the
encounter: 1e-10 of each body's |x| and |v| for FP64 kicks after a few steps
(the bodies outside groups stay at the level-0 tolerance, 1e-12), and 1e-9
with FP32 kicks.  Cases: planted close pairs in a disc, a planet with a
swarm of 80 bodies around it (a group larger than a warp) with every pair
interacting and in test-particle mode 2, a close flyby of two planets,
a batch of systems, graphs against step-by-step launches, determinism.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2309_08217_gb300 import discs
from tests.gpu_cases import orbiting_pairs_disc, planted_disc

pytestmark = pytest.mark.gpu

TOL_BS = 1e-12


def _params(g, d, precision, n_big=-1, tol=TOL_BS, dt=None):
    return g.make_params(G=d.G, Mstar=d.Mstar, dt=d.dt if dt is None else dt, n1=3.0, n2=0.4,
                         rcrit_mode=g.GENGA_RCRIT_MUTUAL_HILL, changeover=g.GENGA_K_CHAMBERS,
                         precision=precision, n_big=n_big, bs_tol=tol)


def _rel_state(got, ref, idx=None):
    """max over bodies of |dx|/|x| and |dv|/|v| (optionally over idx only)."""
    g = np.stack(got[:6]); r = np.stack(ref[:6])
    if idx is not None:
        g, r = g[:, idx], r[:, idx]
    ep = np.sqrt(((g[:3] - r[:3]) ** 2).sum(0)) / np.sqrt((r[:3] ** 2).sum(0))
    ev = np.sqrt(((g[3:] - r[3:]) ** 2).sum(0)) / np.sqrt((r[3:] ** 2).sum(0))
    return max(ep.max(initial=0.0), ev.max(initial=0.0))


@pytest.fixture(scope="module")
def ctx(genga):
    c = genga.Context(20_000)
    yield c
    c.close()


def _members(d, n_big=-1):
    arr = oracle.disc_arrays(d)
    a, rc = oracle.rcrit(*arr, G=d.G, Mstar=d.Mstar, dt=d.dt)
    pairs, _ = oracle.encounters(arr[0], arr[1], arr[2], arr[6], a, rc, 3.0, d.Mstar, 1, n_big=n_big)
    label, ng = oracle.groups(d.N, pairs)
    return np.nonzero(label >= 0)[0], ng, pairs


@pytest.mark.parametrize("precision", [0, 1])
def test_kick_then_drift_parity(genga, ctx, precision):
    d = orbiting_pairs_disc(800, 17)
    mem, ng, pairs = _members(d)
    assert ng >= 3 and len(mem) >= 6
    s = genga.DeviceSystem.from_disc(d)
    p = _params(genga, d, precision)
    genga.genga_kick(ctx, s, p, 0.5 * d.dt)
    genga.genga_drift(ctx, s, p, d.dt)
    assert genga.genga_get_status(ctx) == genga.GENGA_OK
    arr = oracle.disc_arrays(d)
    a, rc = oracle.rcrit(*arr, G=d.G, Mstar=d.Mstar, dt=d.dt)
    # the drift's groups: the encounter pairs and the pairs predicted to enter r_crit
    pred = oracle.predicted_pairs(arr, a, rc, 3.0, d.Mstar, 1, d.dt)
    oracle.kick(arr, d.G, d.Mstar, d.dt, 3.0, 0.4, 1, 0, 0.5 * d.dt)
    bad, forced = oracle.drift_groups(arr, a, rc, np.concatenate([pairs, pred]), d.G, d.Mstar, 3.0, 1, 0,
                                      d.dt, TOL_BS)
    assert bad == 0 and forced == 0
    got = s.numpy()
    others = np.setdiff1d(np.arange(d.N), mem)
    tol_far = 1e-12 if precision == 0 else 1e-9
    assert _rel_state(got, arr, others) < tol_far
    assert _rel_state(got, arr, mem) < (1e-10 if precision == 0 else 1e-9)
    # the level moved the members differently from a Kepler drift
    arr0 = oracle.disc_arrays(d)
    oracle.kick(arr0, d.G, d.Mstar, d.dt, 3.0, 0.4, 1, 0, 0.5 * d.dt)
    oracle.drift(arr0, d.G, d.Mstar, d.dt)
    assert _rel_state(arr0, arr, mem) > 1e-8


@pytest.mark.parametrize("precision", [0, 1])
def test_step_parity(genga, ctx, precision):
    d = orbiting_pairs_disc(800, 17)
    s = genga.DeviceSystem.from_disc(d)
    genga.genga_step(ctx, s, _params(genga, d, precision), 3)
    assert genga.genga_get_status(ctx) == genga.GENGA_OK
    arr = oracle.disc_arrays(d)
    forced = [0]
    assert oracle.step(arr, d.G, d.Mstar, d.dt, 3.0, 0.4, 1, 0, 3, bs_tol=TOL_BS, forced=forced) == 0
    assert forced[0] == 0
    assert _rel_state(s.numpy(), arr) < (1e-10 if precision == 0 else 1e-9)


def _swarm(n_swarm=80, seed=3):
    """A planet of 10 Earth masses at 1 au in a 300-body disc, with n_swarm
    planetesimals inside 0.05 au of it (its changeover radius with them is
    about 0.065 au): one group of n_swarm + 1 bodies.  The planet is body 0."""
    d = orbiting_pairs_disc(300, seed)
    arr = [a.copy() for a in d.arrays()]
    rng = np.random.default_rng(seed)
    G = d.G
    mp = 3.0e-5
    pos = np.array([1.0, 0.0, 0.0]); vel = np.array([0.0, math.sqrt(G * (1 + mp)), 0.0])
    arr[0][0], arr[1][0], arr[2][0] = pos
    arr[3][0], arr[4][0], arr[5][0] = vel
    arr[6][0] = mp
    for k in range(1, n_swarm + 1):
        u = rng.normal(size=3); u /= np.linalg.norm(u)
        r = rng.uniform(0.01, 0.05)
        for c in range(3):
            arr[c][k] = pos[c] + r * u[c]
            arr[3 + c][k] = vel[c] + 3e-4 * rng.normal()
    d2 = d.copy()
    for dst, src in zip(d2.arrays(), arr):
        dst[:] = src
    return d2


@pytest.mark.parametrize("n_big", [-1, 1])
def test_large_group_parity(genga, ctx, n_big):
    d = _swarm()
    mem, ng, _ = _members(d, n_big)
    assert 0 in mem and len(mem) >= 60          # a group wider than one warp
    s = genga.DeviceSystem.from_disc(d)
    genga.genga_step(ctx, s, _params(genga, d, 0, n_big=n_big), 2)
    assert genga.genga_get_status(ctx) == genga.GENGA_OK
    arr = oracle.disc_arrays(d)
    forced = [0]
    assert oracle.step(arr, d.G, d.Mstar, d.dt, 3.0, 0.4, 1, 0, 2, n_big=n_big, bs_tol=TOL_BS,
                       forced=forced) == 0
    assert forced[0] == 0
    assert _rel_state(s.numpy(), arr) < 1e-10


def test_flyby_parity(genga, ctx):
    from tests.test_oracle_bs import _flyby
    arr0 = _flyby()
    s = genga.DeviceSystem.from_arrays([a.copy() for a in arr0])
    p = genga.make_params(G=discs.G_GAUSS, Mstar=1.0, dt=6.0, precision=0, bs_tol=TOL_BS)
    genga.genga_step(ctx, s, p, 20)
    assert genga.genga_get_status(ctx) == genga.GENGA_OK
    ref = [a.copy() for a in arr0]
    assert oracle.step(ref, discs.G_GAUSS, 1.0, 6.0, 3.0, 0.4, 1, 0, 20, bs_tol=TOL_BS) == 0
    assert _rel_state(s.numpy(), ref) < 1e-10


def test_batched_step_parity(genga):
    sizes = [900, 333, 1200]
    parts = [orbiting_pairs_disc(n, 90 + k) for k, n in enumerate(sizes)]
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    arrays = [np.concatenate([p.arrays()[c] for p in parts]) for c in range(7)]
    c = genga.Context(4000)
    s = genga.DeviceSystem.from_arrays(arrays)
    genga.genga_step_batched(c, s, offsets, _params(genga, parts[0], 1), 3)
    assert genga.genga_get_status(c) == genga.GENGA_OK
    got = s.numpy()
    for k, d in enumerate(parts):
        lo, hi = int(offsets[k]), int(offsets[k + 1])
        ref = oracle.disc_arrays(d)
        assert oracle.step(ref, d.G, d.Mstar, d.dt, 3.0, 0.4, 1, 0, 3, bs_tol=TOL_BS) == 0
        assert _rel_state([g[lo:hi] for g in got], ref) < 1e-9, f"system {k}"
    c.close()


def test_graph_steps_equal_step_by_step_and_deterministic(genga):
    d = orbiting_pairs_disc(1500, 71)
    a, b = genga.Context(1500), genga.Context(1500)
    genga.genga_set_step_graphs(b, False)
    for c in (a, b):
        genga.genga_set_kernel_variant(c, 0)
    sa, sb = genga.DeviceSystem.from_disc(d), genga.DeviceSystem.from_disc(d)
    p = _params(genga, d, 1)
    genga.genga_step(a, sa, p, 12)
    for _ in range(12):
        genga.genga_step(b, sb, p, 1)
    assert genga.genga_get_status(a) == genga.GENGA_OK and genga.genga_get_status(b) == genga.GENGA_OK
    assert np.array_equal(sa.numpy(), sb.numpy())
    # the same calls on a fresh context give the same bits
    c = genga.Context(1500)
    genga.genga_set_kernel_variant(c, 0)
    sc = genga.DeviceSystem.from_disc(d)
    genga.genga_step(c, sc, p, 12)
    assert np.array_equal(sa.numpy(), sc.numpy())
    for x in (a, b, c):
        x.close()


def test_head_on_collision_forces_a_substep(genga, ctx):
    """planted_disc's closest pair starts at rest relative to each other and
    falls straight in: the integration meets the r = 0 singularity, which
    both sides report as a forced sub-step (no mergers in this path)."""
    d = planted_disc(800, 17)
    s = genga.DeviceSystem.from_disc(d)
    genga.genga_step(ctx, s, _params(genga, d, 0), 2)
    assert genga.genga_get_status(ctx) == genga.GENGA_ERR_BS
    assert all(np.isfinite(c).all() for c in s.numpy())
    arr = oracle.disc_arrays(d)
    forced = [0]
    oracle.step(arr, d.G, d.Mstar, d.dt, 3.0, 0.4, 1, 0, 2, bs_tol=TOL_BS, forced=forced)
    assert forced[0] >= 1


def test_level1_off_is_the_level0_drift(genga, ctx):
    d = orbiting_pairs_disc(500, 8)
    s1, s2 = genga.DeviceSystem.from_disc(d), genga.DeviceSystem.from_disc(d)
    p_on, p_off = _params(genga, d, 0), _params(genga, d, 0, tol=0.0)
    genga.genga_kick(ctx, s1, p_off, 0.0)            # a list of this state, then drift without the level
    genga.genga_drift(ctx, s1, p_off, d.dt)
    arr = oracle.disc_arrays(d)
    oracle.drift(arr, d.G, d.Mstar, d.dt)
    assert _rel_state(s1.numpy(), arr) < 1e-12
    genga.genga_kick(ctx, s2, p_on, 0.0)
    genga.genga_drift(ctx, s2, p_on, d.dt)
    assert genga.genga_get_status(ctx) == genga.GENGA_OK
    assert not np.array_equal(s1.numpy(), s2.numpy())


def test_invalid_tolerance_rejected(genga, ctx):
    d = planted_disc(10, 1)
    s = genga.DeviceSystem.from_disc(d)
    for bad in (-1e-12, 1e-15, float("nan"), float("inf")):
        with pytest.raises(genga.GengaError):
            genga.genga_drift(ctx, s, _params(genga, d, 0, tol=bad), 1.0)


@pytest.mark.parametrize("precision", [0, 1])
def test_step_parity_eq1_radius_quintic_weight(genga, ctx, precision):
    """The level with the per-body Eq. (1) radius (velocity term included)
    and the quintic changeover, at dt = 1 d."""
    d = orbiting_pairs_disc(600, 29)
    dt = 1.0
    s = genga.DeviceSystem.from_disc(d)
    p = genga.make_params(G=d.G, Mstar=d.Mstar, dt=dt, n1=3.0, n2=0.4, rcrit_mode=genga.GENGA_RCRIT_EQ1,
                          changeover=genga.GENGA_K_QUINTIC, precision=precision, bs_tol=TOL_BS)
    genga.genga_step(ctx, s, p, 3)
    assert genga.genga_get_status(ctx) == genga.GENGA_OK
    arr = oracle.disc_arrays(d)
    forced = [0]
    assert oracle.step(arr, d.G, d.Mstar, dt, 3.0, 0.4, 0, 1, 3, bs_tol=TOL_BS, forced=forced) == 0
    assert forced[0] == 0
    assert _rel_state(s.numpy(), arr) < (1e-10 if precision == 0 else 1e-9)


@pytest.mark.parametrize("n_swarm", [23, 24, 30])
def test_group_sizes_around_the_cluster_threshold(genga, ctx, n_swarm):
    """Groups of 24 members run on one warp, of 25 and more on a cluster of
    CTAs (the same workspace path with cluster barriers and reductions):
    both against the oracle's Bulirsch-Stoer steps, and bitwise repeatable."""
    d = _swarm(n_swarm=n_swarm, seed=5)
    mem, ng, pairs = _members(d)
    label, _ = oracle.groups(d.N, pairs)
    assert int((label == label[0]).sum()) == n_swarm + 1   # the planet's group
    arr = oracle.disc_arrays(d)
    forced = [0]
    assert oracle.step(arr, d.G, d.Mstar, d.dt, 3.0, 0.4, 1, 0, 2, bs_tol=TOL_BS, forced=forced) == 0
    assert forced[0] == 0
    got = []
    for _ in range(2):  # fresh contexts: the same spatial order and plans
        c = genga.Context(d.N)
        s = genga.DeviceSystem.from_disc(d)
        genga.genga_step(c, s, _params(genga, d, 0), 2)
        assert genga.genga_get_status(c) == genga.GENGA_OK
        got.append(np.stack(s.numpy()))
        c.close()
    assert np.array_equal(got[0], got[1])
    assert _rel_state(list(got[0]), arr) < 1e-10
