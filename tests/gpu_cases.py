"""Seeded inputs shared by the GPU parity tests (no method arithmetic here:
bodies are only placed; the oracle computes everything else)."""
import numpy as np

from paper_2309_08217_gb300 import discs


def planted_disc(N, seed, fracs=(0.05, 0.5, 0.9, 1.1, 0.3), mass_scale=1.0, a_min=0.7, a_max=3.0):
    """An equal-mass disc (2.5 Earth masses in total) with close pairs planted
    at fixed fractions of the three-mutual-Hill-radius scale
    3 (2m/3)^(1/3) a, so the changeover region, K = 0 and the r_crit
    boundary are all exercised."""
    d = discs.disc_uniform(N, seed, a_min=a_min, a_max=a_max, m_total=2.5 * discs.M_EARTH * mass_scale)
    arr = [a.copy() for a in d.arrays()]
    rng = np.random.default_rng(seed + 77)
    m = arr[6][0]
    npl = min(len(fracs), N // 2)
    for k in range(npl):
        i, j = 2 * k + 1, 2 * k
        r = np.sqrt(arr[0][j] ** 2 + arr[1][j] ** 2 + arr[2][j] ** 2)
        scale = 3.0 * (2 * m / 3.0) ** (1 / 3) * r
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        for c in range(3):
            arr[c][i] = arr[c][j] + fracs[k] * scale * u[c]
        for c in range(3, 6):
            arr[c][i] = arr[c][j]
    d2 = d.copy()
    for dst, src in zip(d2.arrays(), arr):
        dst[:] = src
    return d2


def orbiting_pairs_disc(N, seed, fracs=(0.05, 0.5, 0.9, 1.1, 0.3)):
    """planted_disc with each planted pair set on a circular orbit about its
    centre of mass (relative speed sqrt(G (m_i + m_j) / r) perpendicular to the
    separation), so the close pairs revolve instead of falling onto each other."""
    d = planted_disc(N, seed, fracs)
    arr = [a.copy() for a in d.arrays()]
    rng = np.random.default_rng(seed + 91)
    npl = min(len(fracs), N // 2)
    for k in range(npl):
        i, j = 2 * k + 1, 2 * k
        sep = np.array([arr[c][i] - arr[c][j] for c in range(3)])
        r = np.linalg.norm(sep)
        w = rng.normal(size=3)
        w -= w @ sep / r ** 2 * sep
        w /= np.linalg.norm(w)
        vrel = np.sqrt(d.G * (arr[6][i] + arr[6][j]) / r)
        mi, mj = arr[6][i], arr[6][j]
        for c in range(3):   # relative velocity split so the pair's momentum is unchanged
            arr[3 + c][i] += mj / (mi + mj) * vrel * w[c]
            arr[3 + c][j] -= mi / (mi + mj) * vrel * w[c]
    d2 = d.copy()
    for dst, src in zip(d2.arrays(), arr):
        dst[:] = src
    return d2


def check_merged(got, ref, dead, tol=1e-10, survivors=None, m0=None, dt=None):
    """Parity of a state with perfect mergers.

    Live bodies agree with the oracle to `tol` of |x| and |v|, and so do
    ghosts without a survivor (bodies removed by the removal radii: they move
    on as massless bodies on both sides).

    A merged ghost keeps the state of the accepted Bulirsch-Stoer sub-step
    that detected its overlap, and which sub-step that is can flip with the
    rounding of the tolerance test.  Up to that sub-step both sides follow the
    same trajectory; after it the ghost moves as a massless body.  So two
    valid ghost states differ by what the partner's attraction does to the
    ghost over at most one sub-step (h <= dt): a displacement below
    v_rel h and a velocity change below v_rel, v_rel the pair's relative
    speed before the merger.  The oracle's end state gives v_rel: the survivor
    moves with the pair's centre of mass, so v_rel = |v_ghost - v_survivor| *
    m_survivor / (m_survivor - m_ghost), with the ghost's initial mass m0.
    Each ghost listed in `survivors` ({ghost: survivor}) must lie within
    2 v_rel dt and 2 v_rel of the oracle's ghost (a factor 2 for the
    rounding of the two integrations and the curvature of the paths)."""
    live = np.nonzero(dead == 0)[0]
    g = np.stack(got[:6]); r = np.stack(ref[:6])
    survivors = survivors or {}
    plain = np.array(sorted(set(live.tolist()) | (set(np.nonzero(dead != 0)[0].tolist()) - set(survivors))),
                     dtype=np.int64)
    ep = np.sqrt(((g[:3, plain] - r[:3, plain]) ** 2).sum(0)) / np.sqrt((r[:3, plain] ** 2).sum(0))
    ev = np.sqrt(((g[3:, plain] - r[3:, plain]) ** 2).sum(0)) / np.sqrt((r[3:, plain] ** 2).sum(0))
    assert max(ep.max(initial=0.0), ev.max(initial=0.0)) < tol
    ghosts = np.nonzero(dead != 0)[0]
    assert np.all(np.isfinite(g[:, ghosts]))
    if survivors:
        assert m0 is not None and dt is not None
    for gh, sv in survivors.items():
        assert dead[gh] != 0 and dead[sv] == 0
        ms = ref[6][sv]
        vrel = np.linalg.norm(r[3:, gh] - r[3:, sv]) * ms / (ms - m0[gh])
        dx = np.linalg.norm(g[:3, gh] - r[:3, gh])
        dv = np.linalg.norm(g[3:, gh] - r[3:, gh])
        assert dx <= 2 * vrel * abs(dt) and dv <= 2 * vrel, (gh, sv, dx, dv, vrel)
