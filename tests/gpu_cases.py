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


def check_merged(got, ref, dead, tol=1e-10, survivors=None):
    """Parity of a state with perfect mergers.  The live bodies agree with the
    oracle to `tol` of |x| and |v|.  A ghost keeps the state it had when the
    overlap was detected, at the end of an accepted Bulirsch-Stoer sub-step,
    and which sub-step that is can flip with the rounding of the tolerance
    test (a one-ulp change of one input coordinate moves the oracle's own
    ghost by its pre-merge relative speed times a sub-step), so a ghost is
    only checked to be finite and, for merged pairs given as
    {ghost: survivor}, to stay within 0.01 au and 1e-3 au/day of its survivor."""
    live = np.nonzero(dead == 0)[0]
    g = np.stack(got[:6]); r = np.stack(ref[:6])
    ep = np.sqrt(((g[:3, live] - r[:3, live]) ** 2).sum(0)) / np.sqrt((r[:3, live] ** 2).sum(0))
    ev = np.sqrt(((g[3:, live] - r[3:, live]) ** 2).sum(0)) / np.sqrt((r[3:, live] ** 2).sum(0))
    assert max(ep.max(initial=0.0), ev.max(initial=0.0)) < tol
    ghosts = np.nonzero(dead != 0)[0]
    assert np.all(np.isfinite(g[:, ghosts]))
    for gh, sv in (survivors or {}).items():
        assert np.linalg.norm(g[:3, gh] - g[:3, sv]) < 0.01 and np.linalg.norm(g[3:, gh] - g[3:, sv]) < 1e-3
