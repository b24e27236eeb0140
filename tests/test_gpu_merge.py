"""Perfect mergers, removal radii and compaction on the GPU (genga_step with
bs_tol > 0 and physical radii; params r_in / r_out; genga_compact) against
the oracle's step with the same switches.

The merged masses, radii and the set of ghosts (mass -0.0) must be
identical; positions and velocities of the live bodies agree to 1e-10 of |x|
and |v| (FP64 kick) as in the other close-encounter tests.  A merged ghost
keeps the state of the sub-step that detected the overlap, which can flip
with rounding, so its state is checked against the bound that follows from
that (gpu_cases.check_merged: within 2 v_rel dt and 2 v_rel of the oracle's
ghost, v_rel the pair's relative speed before the merger); removed bodies
match the oracle like live ones.  Compaction keeps the
survivors' order and moves an id array along.
"""
import numpy as np
import pytest

import oracle
from tests.gpu_cases import check_merged, planted_disc
from tests.test_gpu_bs import _rel_state, _swarm

pytestmark = pytest.mark.gpu

TOL_BS = 1e-12


def _params(g, d, precision=0, n_big=-1, r_in=0.0, r_out=0.0):
    return g.make_params(G=d.G, Mstar=d.Mstar, dt=d.dt, n1=3.0, n2=0.4, precision=precision, n_big=n_big,
                         bs_tol=TOL_BS, r_in=r_in, r_out=r_out)


@pytest.fixture(scope="module")
def ctx(genga):
    c = genga.Context(4096)
    yield c
    c.close()


def _run_both(genga, ctx, d, R, steps, precision=0, n_big=-1, r_in=0.0, r_out=0.0):
    import torch
    s = genga.DeviceSystem.from_disc(d, radius=R)
    ids = torch.arange(d.N, dtype=torch.int32, device="cuda")
    genga.genga_step(ctx, s, _params(genga, d, precision, n_big, r_in, r_out), steps)
    assert genga.genga_get_status(ctx) == genga.GENGA_OK
    got = s.numpy()
    got_R = s.radius_numpy()
    arr = oracle.disc_arrays(d)
    Ro = np.array(R, dtype=np.float64).copy()
    dead = np.zeros(d.N, np.int32)
    merges, forced = [0], [0]
    assert oracle.step(arr, d.G, d.Mstar, d.dt, 3.0, 0.4, 1, 0, steps, n_big=n_big, bs_tol=TOL_BS, forced=forced,
                       radius=Ro, dead=dead, r_in=r_in, r_out=r_out, merges=merges) == 0
    assert forced[0] == 0
    return s, ids, got, got_R, arr, Ro, dead, merges[0]


def test_head_on_pair_merges(genga, ctx):
    """planted_disc's closest pair starts at rest relative to each other and
    falls in during the second step: with radii it merges instead of meeting
    the singularity."""
    d = planted_disc(800, 17)
    R = np.full(d.N, 2e-5)
    s, ids, got, got_R, arr, Ro, dead, merges = _run_both(genga, ctx, d, R, 3)
    assert merges >= 1 and dead[1] == 1 and dead[0] == 0
    assert np.array_equal(np.signbit(got[6]), dead == 1)
    np.testing.assert_allclose(got[6], arr[6], rtol=1e-15, atol=0)
    np.testing.assert_allclose(got_R, Ro, rtol=1e-14, atol=0)
    check_merged(got, arr, dead, 1e-10, {1: 0}, m0=d.m, dt=d.dt)
    # compaction drops exactly the ghosts, in order, with the ids
    n = genga.genga_compact(ctx, s, ids)
    assert n == d.N - int(dead.sum())
    keep = np.nonzero(dead == 0)[0]
    assert np.array_equal(ids[:n].cpu().numpy(), keep)
    after = s.numpy()
    for c in range(7):
        assert np.array_equal(after[c], got[c][keep])
    assert np.array_equal(s.radius_numpy(), got_R[keep])


def test_removal_radii(genga, ctx):
    d = planted_disc(1500, 5, a_min=0.5, a_max=3.0)
    R = np.full(d.N, 1e-6)
    s, ids, got, got_R, arr, Ro, dead, merges = _run_both(genga, ctx, d, R, 2, precision=1, r_in=0.62, r_out=2.8)
    assert dead.sum() >= 4
    assert np.array_equal(np.signbit(got[6]), dead == 1)
    assert np.array_equal(got_R == 0.0, dead == 1)
    assert _rel_state(got, arr) < 1e-9
    n = genga.genga_compact(ctx, s, ids)
    assert np.array_equal(ids[:n].cpu().numpy(), np.nonzero(dead == 0)[0])
    # the compacted system steps on like the oracle's compacted one
    p = _params(genga, d, 1, r_in=0.62, r_out=2.8)
    genga.genga_step(ctx, s, p, 1)
    assert genga.genga_get_status(ctx) == genga.GENGA_OK
    keep = dead == 0
    arr2 = [a[keep].copy() for a in arr]
    R2, dead2 = Ro[keep].copy(), np.zeros(int(keep.sum()), np.int32)
    assert oracle.step(arr2, d.G, d.Mstar, d.dt, 3.0, 0.4, 1, 0, 1, bs_tol=TOL_BS, radius=R2, dead=dead2,
                       r_in=0.62, r_out=2.8) == 0
    assert _rel_state(s.numpy(), arr2) < 1e-9


@pytest.mark.parametrize("n_big", [-1, 1])
def test_swarm_mergers_large_group(genga, ctx, n_big):
    """The planet with 80 bodies around it, with a planet radius of 0.02 au:
    the bodies inside it at the first sub-step and those that reach it merge
    into it (body 0, the lowest index); a group wider than a warp."""
    d = _swarm()
    R = np.full(d.N, 1e-6)
    R[0] = 0.02
    s, ids, got, got_R, arr, Ro, dead, merges = _run_both(genga, ctx, d, R, 2, n_big=n_big)
    assert merges >= 5 and dead[0] == 0
    assert np.array_equal(np.signbit(got[6]), dead == 1)
    np.testing.assert_allclose(got[6], arr[6], rtol=1e-14, atol=0)
    np.testing.assert_allclose(got_R, Ro, rtol=1e-13, atol=0)
    # every ghost fell into the planet (the swarm bodies' radii are 1e-6 au)
    check_merged(got, arr, dead, 1e-10, {int(k): 0 for k in np.nonzero(dead)[0]}, m0=d.m, dt=d.dt)


def test_no_radius_no_mergers(genga, ctx):
    """Without radii the same state keeps every body (and meets the head-on
    singularity as a forced sub-step)."""
    d = planted_disc(800, 17)
    s = genga.DeviceSystem.from_disc(d)
    genga.genga_step(ctx, s, _params(genga, d), 3)
    assert genga.genga_get_status(ctx) == genga.GENGA_ERR_BS
    assert np.all(s.numpy()[6] > 0)


def test_invalid_radii_rejected(genga, ctx):
    d = planted_disc(10, 1)
    s = genga.DeviceSystem.from_disc(d)
    for bad in (float("nan"), float("inf")):
        with pytest.raises(genga.GengaError):
            genga.genga_drift(ctx, s, _params(genga, d, r_out=bad), 1.0)


@pytest.mark.parametrize("pattern", ["none", "all", "ends", "every_other"])
def test_compaction_edge_cases(genga, ctx, pattern):
    import torch
    d = planted_disc(2500, 3)
    s = genga.DeviceSystem.from_disc(d, radius=np.full(d.N, 1e-6))
    ghost = np.zeros(d.N, bool)
    if pattern == "all":
        ghost[:] = True
    elif pattern == "ends":
        ghost[[0, 1, d.N - 1]] = True
    elif pattern == "every_other":
        ghost[::2] = True
    m = s.tensors[6]
    m[torch.as_tensor(np.nonzero(ghost)[0], device="cuda")] = -0.0
    before = s.numpy()
    ids = torch.arange(d.N, dtype=torch.int32, device="cuda")
    n = genga.genga_compact(ctx, s, ids)
    keep = np.nonzero(~ghost)[0]
    assert n == len(keep) == s.N
    assert np.array_equal(ids[:n].cpu().numpy(), keep)
    after = s.numpy()
    for c in range(7):
        assert np.array_equal(after[c], before[c][keep])
    if n:   # the compacted system steps on normally
        genga.genga_step(ctx, s, _params(genga, d, 1), 1)
        assert genga.genga_get_status(ctx) == genga.GENGA_OK


def test_batched_mergers_and_removal(genga):
    """Three systems in one batched call, each with a head-on pair that merges
    and removal radii: every system as the oracle steps it alone (ghosts
    marked in place; batched mode has no compaction)."""
    sizes = [800, 500, 1100]
    parts = [planted_disc(n, 17 + 3 * k) for k, n in enumerate(sizes)]
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    arrays = [np.concatenate([p.arrays()[c] for p in parts]) for c in range(7)]
    R = np.full(int(offsets[-1]), 2e-5)
    c = genga.Context(4000)
    s = genga.DeviceSystem.from_arrays(arrays, radius=R)
    p = _params(genga, parts[0], 1, r_in=0.72, r_out=2.9)
    genga.genga_step_batched(c, s, offsets, p, 3)
    assert genga.genga_get_status(c) == genga.GENGA_OK
    got, got_R = s.numpy(), s.radius_numpy()
    total_ghosts = 0
    for k, d in enumerate(parts):
        lo, hi = int(offsets[k]), int(offsets[k + 1])
        ref = oracle.disc_arrays(d)
        Rk, dead = R[lo:hi].copy(), np.zeros(d.N, np.int32)
        assert oracle.step(ref, d.G, d.Mstar, d.dt, 3.0, 0.4, 1, 0, 3, bs_tol=TOL_BS, radius=Rk, dead=dead,
                           r_in=0.72, r_out=2.9) == 0
        gk = [g[lo:hi] for g in got]
        assert np.array_equal(np.signbit(gk[6]), dead == 1), f"system {k}"
        np.testing.assert_allclose(gk[6], ref[6], rtol=1e-15, atol=0)
        np.testing.assert_allclose(got_R[lo:hi], Rk, rtol=1e-14, atol=0)
        # the head-on pair (0, 1) merges into body 0; the other ghosts are removed bodies
        merged = {1: 0} if dead[1] and not dead[0] and ref[6][0] > d.m[0] else {}
        check_merged(gk, ref, dead, 1e-9, merged, m0=d.m, dt=d.dt)
        total_ghosts += int(dead.sum())
    assert total_ghosts >= 3
    c.close()
