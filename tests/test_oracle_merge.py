"""Pins of the oracle's perfect mergers and removal radii (Sect. 2: collisions
are perfect mergers; bodies are removed inside an inner or beyond an outer
heliocentric distance).  None of these calls the CUDA path.

* a head-on collision in free space (negligible central mass): the survivor
  (the lower index) carries the total mass, moves with the centre of mass,
  whose motion is uniform, and has the equal-density radius; the absorbed
  body is a ghost (mass -0.0) marked dead;
* the overlap test: two bodies on a circular orbit about each other merge when
  the radii add up to more than their separation and not otherwise;
* removal: exactly the live bodies beyond r_out or inside r_in after the drift
  are marked dead, with m = -0.0;
* ghosts are inert: a step with a ghost in the arrays gives the other bodies
  bit for bit the state of the same step without it.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2309_08217_gb300 import discs

G = discs.G_GAUSS


def _pair(r0, r1, v0, v1, m):
    return [np.array([r0[c], r1[c]]) for c in range(3)] + \
           [np.array([v0[c], v1[c]]) for c in range(3)] + [np.array(m, dtype=float)]


def test_head_on_merger_in_free_space():
    Gc, Ms = 1.0, 1e-20
    m = [3e-3, 1e-3]
    c0 = np.array([1.0, 2.0, 0.5]); V = np.array([0.02, -0.01, 0.03])
    u = np.array([0.0, 0.6, 0.8])
    d0 = 0.02
    # at rest relative to each other: they fall straight in
    r0 = c0 + m[1] / sum(m) * d0 * u
    r1 = c0 - m[0] / sum(m) * d0 * u
    arr = _pair(r0, r1, V, V, m)
    R = np.array([2e-3, 1e-3])
    dead = np.zeros(2, np.int32)
    merges = [0]
    T = 1.5   # free-fall time from d0 to contact is about 0.99 for G(m0+m1) = 4e-3
    forced = oracle.bs_group(arr, [0, 1], np.ones(2), np.full(2, 1.0), Gc, Ms, 3.0, 0, 0, T, 1e-13,
                             radius=R, dead=dead, merges=merges)
    assert forced == 0 and merges[0] == 1
    assert dead.tolist() == [0, 1]
    assert arr[6][0] == pytest.approx(4e-3, rel=1e-15) and arr[6][1] == 0.0 and np.signbit(arr[6][1])
    assert R[0] == pytest.approx((2e-3 ** 3 + 1e-3 ** 3) ** (1 / 3), rel=1e-14) and R[1] == 0.0
    pos = np.array([arr[c][0] for c in range(3)])
    vel = np.array([arr[c][0] for c in range(3, 6)])
    assert np.abs(pos - (c0 + V * T)).max() < 1e-11
    assert np.abs(vel - V).max() < 1e-11


@pytest.mark.parametrize("scale,merge", [(0.99, False), (1.01, True)])
def test_overlap_test_on_a_circular_binary(scale, merge):
    Gc, m, d = 1.0, 1e-3, 0.01
    w = math.sqrt(Gc * 2 * m / d ** 3)
    c0 = np.array([1.0, 0.5, 0.2])
    u = np.array([0.6, 0.8, 0.0]); vp = np.array([-0.8, 0.6, 0.0])
    arr = _pair(c0 + 0.5 * d * u, c0 - 0.5 * d * u, 0.5 * d * w * vp, -0.5 * d * w * vp, [m, m])
    R = np.full(2, 0.5 * scale * d)
    dead = np.zeros(2, np.int32)
    merges = [0]
    oracle.bs_group(arr, [0, 1], np.ones(2), np.full(2, 1.0), Gc, 1e-20, 3.0, 0, 0, 0.05, 1e-13,
                    radius=R, dead=dead, merges=merges)
    assert merges[0] == (1 if merge else 0)
    assert dead.tolist() == ([0, 1] if merge else [0, 0])
    if merge:   # the survivor sits at the centre of mass, at rest
        assert np.abs(np.array([arr[c][0] for c in range(3)]) - c0).max() < 1e-13
        assert np.abs(np.array([arr[c][0] for c in range(3, 6)])).max() < 1e-13


def test_removal_radii_mark_exactly_the_bodies_outside():
    d = discs.disc_uniform(300, 9, a_min=0.5, a_max=3.0)
    arr = oracle.disc_arrays(d)
    dead = np.zeros(d.N, np.int32)
    R = np.full(d.N, 1e-6)
    r_in, r_out = 0.62, 2.8
    oracle.step(arr, d.G, d.Mstar, d.dt, 3.0, 0.4, 1, 0, 1, bs_tol=1e-12, radius=R, dead=dead,
                r_in=r_in, r_out=r_out)
    r2 = arr[0] ** 2 + arr[1] ** 2 + arr[2] ** 2
    want = (r2 < r_in * r_in) | (r2 > r_out * r_out)
    assert want.sum() >= 4 and (~want).sum() > 200
    assert np.array_equal(dead.astype(bool), want)
    assert np.all(arr[6][want] == 0.0) and np.all(np.signbit(arr[6][want])) and np.all(arr[6][~want] > 0.0)
    assert np.all(R[want] == 0.0)


def test_ghosts_are_inert():
    d = discs.disc_uniform(120, 4, a_min=0.8, a_max=1.4)
    arr = [a.copy() for a in oracle.disc_arrays(d)]
    # a ghost (massless, dead) right next to body 7, inserted at index 40
    ghost = [arr[c][7] + (1e-5 if c == 0 else 0.0) for c in range(6)] + [0.0]
    with_g = [np.insert(arr[c], 40, ghost[c]) for c in range(7)]
    dead_g = np.zeros(d.N + 1, np.int32); dead_g[40] = 1
    dead = np.zeros(d.N, np.int32)
    Rg = np.full(d.N + 1, 1e-7); Rg[40] = 0.0
    R = np.full(d.N, 1e-7)
    for st, dd, rr in ((arr, dead, R), (with_g, dead_g, Rg)):
        assert oracle.step(st, d.G, d.Mstar, d.dt, 3.0, 0.4, 1, 0, 3, bs_tol=1e-12, radius=rr, dead=dd) == 0
    keep = np.r_[0:40, 41:d.N + 1]
    for c in range(7):
        assert np.array_equal(with_g[c][keep], arr[c])
    assert dead_g[40] == 1 and dead_g[keep].sum() == 0


def test_simultaneous_overlaps_all_merge_after_one_substep():
    """Three bodies overlapping at once, drifted over a time short enough for
    a single accepted sub-step: the search repeats until no pair overlaps, so
    both mergers happen after that sub-step -- one survivor (the lowest index)
    with the total mass, the mass-weighted velocity and the equal-density
    radius of all three."""
    Gc, Ms = 1.0, 1e-20
    m = [3e-3, 1e-3, 2e-3]
    pos = [np.array([1.0, 2.0, 0.5]), np.array([1.0005, 2.0, 0.5]), np.array([1.0, 2.0006, 0.5])]
    vel = [np.array([0.01, 0.0, 0.0]), np.array([0.0, 0.02, 0.0]), np.array([0.0, 0.0, -0.03])]
    arr = [np.array([p[c] for p in pos]) for c in range(3)] + [np.array([v[c] for v in vel]) for c in range(3)] + \
          [np.array(m)]
    R = np.array([1e-3, 1e-3, 1e-3])
    dead = np.zeros(3, np.int32)
    merges = [0]
    forced = oracle.bs_group(arr, [0, 1, 2], np.ones(3), np.full(3, 1.0), Gc, Ms, 3.0, 0, 0, 1e-6, 1e-12,
                             radius=R, dead=dead, merges=merges)
    assert forced == 0 and merges[0] == 2 and dead.tolist() == [0, 1, 1]
    assert arr[6][0] == pytest.approx(6e-3, rel=1e-15) and np.all(np.signbit(arr[6][1:]))
    vcm = sum(mi * v for mi, v in zip(m, vel)) / sum(m)
    assert np.abs(np.array([arr[c][0] for c in range(3, 6)]) - vcm).max() < 1e-9
    assert R[0] == pytest.approx(3 ** (1 / 3) * 1e-3, rel=1e-14)


def test_a_ghost_moves_on_its_kepler_orbit():
    """Two massless bodies overlapping at t = 0 near the Sun merge after the
    first accepted sub-step (no pair force ever acts: m = 0); the absorbed one
    then feels the central body only (R24), so at the end of the drift it is
    where the Kepler solution of its initial state puts it."""
    vc = math.sqrt(G)
    arr = _pair([1.0, 0.0, 0.0], [1.0 + 5e-6, 1e-6, 0.0], [0.0, vc, 0.0], [1e-4, 1.02 * vc, 2e-4], [0.0, 0.0])
    x1 = [arr[c][1] for c in range(6)]
    R = np.array([1e-5, 1e-5])
    dead = np.zeros(2, np.int32)
    merges = [0]
    dt = 10.0
    forced = oracle.bs_group(arr, [0, 1], np.ones(2), np.full(2, 1.0), G, 1.0, 3.0, 0, 0, dt, 1e-12,
                             radius=R, dead=dead, merges=merges)
    assert forced == 0 and merges[0] == 1 and dead.tolist() == [0, 1]
    want, status = oracle.kepler(G, x1, dt)
    assert status == 0
    got = np.array([arr[c][1] for c in range(6)])
    assert np.abs(got[:3] - want[:3]).max() < 1e-11 and np.abs(got[3:] - want[3:]).max() < 1e-12
