"""Seeded synthetic planetesimal discs: the inputs of every workload.

This module only draws orbital elements and turns them into the state arrays
that both the CUDA path and the CPU oracle consume.  It holds none of the
method's arithmetic (no kick, changeover, critical radius or drift); it
imports only numpy, so the oracle tests and the GPU tests can share it.

Units: au, solar masses, days; G is the Gaussian gravitational constant
squared (k^2).  Coordinates are democratic-heliocentric: heliocentric
positions and barycentric velocities (the coordinate set of the hybrid
symplectic step the paper builds on, Sect. 1).

Workloads (the paper's own initial conditions are not public in a form we can
use, so these seeded discs stand in for them; shapes follow Sect. 2):

* ``disc_uniform``  -- equal-mass bodies, a ~ U(a_min, a_max)
* ``disc_powerlaw`` -- equal-mass bodies, surface density ~ a^-1.5
                       (inverse-CDF sampling of dN/da ~ a^-0.5)
* ``embryo_disc``   -- a few embryos plus many planetesimals
* ``giants_disc``   -- four giant planets plus an outer planetesimal belt
* ``batch_of_discs``-- many independent discs of log-uniform size
* ``planet_swarm``  -- a planet with a dense swarm around it inside a disc
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List

import numpy as np

G_GAUSS = 2.959122082855911e-4  # au^3 Msun^-1 day^-2
M_EARTH = 3.0034896e-6          # Msun


@dataclass
class Disc:
    """State of one system: N bodies orbiting a central mass ``Mstar``.

    x, y, z    heliocentric positions [au], float64[N]
    vx, vy, vz barycentric velocities [au/day], float64[N]
    m          masses [Msun], float64[N]
    """
    name: str
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    vx: np.ndarray
    vy: np.ndarray
    vz: np.ndarray
    m: np.ndarray
    Mstar: float = 1.0
    G: float = G_GAUSS
    dt: float = 6.0
    n1: float = 3.0
    n2: float = 0.4
    meta: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return int(self.m.shape[0])

    def arrays(self):
        return (self.x, self.y, self.z, self.vx, self.vy, self.vz, self.m)

    def copy(self) -> "Disc":
        return Disc(self.name, *(a.copy() for a in self.arrays()), Mstar=self.Mstar,
                    G=self.G, dt=self.dt, n1=self.n1, n2=self.n2, meta=dict(self.meta))

    def subset(self, n: int) -> "Disc":
        """First n bodies (heavy bodies come first in every generator)."""
        return Disc(self.name + f"[:{n}]", *(a[:n].copy() for a in self.arrays()),
                    Mstar=self.Mstar, G=self.G, dt=self.dt, n1=self.n1, n2=self.n2,
                    meta=dict(self.meta))


def rayleigh(rng: np.random.Generator, sigma: float, n: int) -> np.ndarray:
    """Rayleigh deviates by inversion: sigma * sqrt(-2 ln(1-u))."""
    u = rng.random(n)
    return sigma * np.sqrt(-2.0 * np.log1p(-u))


def _solve_kepler_equation(M: np.ndarray, e: np.ndarray) -> np.ndarray:
    """Eccentric anomaly from the mean anomaly (elliptic orbits), Newton."""
    E = np.where(e < 0.8, M, np.pi * np.ones_like(M))
    for _ in range(60):
        f = E - e * np.sin(E) - M
        E = E - f / (1.0 - e * np.cos(E))
    return E


def elements_to_cartesian(mu, a, e, inc, Omega, omega, M):
    """Heliocentric position/velocity from Keplerian elements (elliptic)."""
    a = np.asarray(a, float)
    e = np.asarray(e, float)
    E = _solve_kepler_equation(np.mod(M, 2 * np.pi), e)
    cE, sE = np.cos(E), np.sin(E)
    sq = np.sqrt(1.0 - e * e)
    n = np.sqrt(mu / a ** 3)
    xo = a * (cE - e)
    yo = a * sq * sE
    fac = n * a / (1.0 - e * cE)
    vxo = -sE * fac
    vyo = sq * cE * fac
    cO, sO = np.cos(Omega), np.sin(Omega)
    cw, sw = np.cos(omega), np.sin(omega)
    ci, si = np.cos(inc), np.sin(inc)
    # rotation R_z(Omega) R_x(inc) R_z(omega) applied to (xo, yo, 0)
    r11 = cO * cw - sO * sw * ci
    r12 = -cO * sw - sO * cw * ci
    r21 = sO * cw + cO * sw * ci
    r22 = -sO * sw + cO * cw * ci
    r31 = sw * si
    r32 = cw * si
    pos = np.stack([r11 * xo + r12 * yo, r21 * xo + r22 * yo, r31 * xo + r32 * yo])
    vel = np.stack([r11 * vxo + r12 * vyo, r21 * vxo + r22 * vyo, r31 * vxo + r32 * vyo])
    return pos, vel


def _assemble(name, m, a, e, inc, Omega, omega, M, Mstar, G, dt, meta) -> Disc:
    mu = G * (Mstar + m)  # heliocentric two-body orbit of each body
    pos, vhel = elements_to_cartesian(mu, a, e, inc, Omega, omega, M)
    # barycentric velocities: v_bary = v_hel - sum_j m_j v_hel_j / (Mstar + sum_j m_j)
    vsun = -(vhel * m).sum(axis=1) / (Mstar + m.sum())
    vbar = vhel + vsun[:, None]
    return Disc(name, pos[0].copy(), pos[1].copy(), pos[2].copy(),
                vbar[0].copy(), vbar[1].copy(), vbar[2].copy(), m.astype(np.float64),
                Mstar=Mstar, G=G, dt=dt, meta=meta)


def _angles(rng, n):
    return (rng.uniform(0.0, 2 * np.pi, n), rng.uniform(0.0, 2 * np.pi, n),
            rng.uniform(0.0, 2 * np.pi, n))


def disc_uniform(N: int, seed: int, a_min=0.7, a_max=3.0, m_total=2.5 * M_EARTH,
                 sig_e=0.01, sig_i=0.005, dt=6.0, name=None) -> Disc:
    """N equal-mass bodies, a uniform in [a_min, a_max]."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(a_min, a_max, N)
    e = rayleigh(rng, sig_e, N)
    inc = rayleigh(rng, sig_i, N)
    Om, om, M = _angles(rng, N)
    m = np.full(N, m_total / N)
    return _assemble(name or f"uniform-N{N}-s{seed}", m, a, e, inc, Om, om, M, 1.0, G_GAUSS, dt,
                     {"seed": seed, "kind": "uniform"})


def disc_powerlaw(N: int, seed: int, a_min=0.5, a_max=4.0, m_total=5.0 * M_EARTH,
                  sig_e=0.01, sig_i=0.005, dt=6.0, name=None) -> Disc:
    """N equal-mass bodies, surface density ~ a^-1.5 on [a_min, a_max].

    dN/da ~ a * a^-1.5 = a^-0.5, whose inverse CDF is
    a = (sqrt(a_min) + u (sqrt(a_max) - sqrt(a_min)))^2.
    """
    rng = np.random.default_rng(seed)
    u = rng.random(N)
    a = (np.sqrt(a_min) + u * (np.sqrt(a_max) - np.sqrt(a_min))) ** 2
    e = rayleigh(rng, sig_e, N)
    inc = rayleigh(rng, sig_i, N)
    Om, om, M = _angles(rng, N)
    m = np.full(N, m_total / N)
    return _assemble(name or f"powerlaw-N{N}-s{seed}", m, a, e, inc, Om, om, M, 1.0, G_GAUSS, dt,
                     {"seed": seed, "kind": "powerlaw"})


def embryo_disc(n_emb=25, n_pl=6600, seed=2, a_min=0.5, a_max=4.0, m_emb=0.05 * M_EARTH,
                m_pl_total=2.5 * M_EARTH, dt=6.0) -> Disc:
    """Embryos (first n_emb bodies) plus equal-mass planetesimals."""
    rng = np.random.default_rng(seed)
    N = n_emb + n_pl
    a = rng.uniform(a_min, a_max, N)
    e = rayleigh(rng, 0.01, N)
    inc = rayleigh(rng, 0.005, N)
    Om, om, M = _angles(rng, N)
    m = np.concatenate([np.full(n_emb, m_emb), np.full(n_pl, m_pl_total / n_pl)])
    return _assemble(f"embryos{n_emb}+pl{n_pl}-s{seed}", m, a, e, inc, Om, om, M, 1.0, G_GAUSS, dt,
                     {"seed": seed, "kind": "embryo"})


def giants_disc(n_pl=100_000, seed=5, dt=36.5) -> Disc:
    """Four giants at 5.5/8/11.5/15 au plus a belt of n_pl planetesimals
    (35 Earth masses in total, uniform surface density on 16-30 au)."""
    rng = np.random.default_rng(seed)
    mg = np.array([1.0e-3, 2.9e-4, 4.4e-5, 5.2e-5])
    ag = np.array([5.5, 8.0, 11.5, 15.0])
    eg = rng.uniform(0.0, 0.01, 4)
    ig = rng.uniform(0.0, 0.01, 4)
    Omg, omg, Mg = _angles(rng, 4)
    u = rng.random(n_pl)
    ap = np.sqrt(16.0 ** 2 + u * (30.0 ** 2 - 16.0 ** 2))
    ep = rayleigh(rng, 0.01, n_pl)
    ip = rayleigh(rng, 0.005, n_pl)
    Omp, omp, Mp = _angles(rng, n_pl)
    m = np.concatenate([mg, np.full(n_pl, 35.0 * M_EARTH / n_pl)])
    cat = np.concatenate
    return _assemble(f"giants4+pl{n_pl}-s{seed}", m, cat([ag, ap]), cat([eg, ep]), cat([ig, ip]),
                     cat([Omg, Omp]), cat([omg, omp]), cat([Mg, Mp]), 1.0, G_GAUSS, dt,
                     {"seed": seed, "kind": "giants"})


def batch_sizes(D=256, seed=4, n_lo=1000, n_hi=16000) -> np.ndarray:
    """Disc sizes drawn log-uniform in [n_lo, n_hi]."""
    rng = np.random.default_rng(seed)
    return np.floor(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi), D))).astype(np.int64)


def batch_of_discs(D=256, seed=4, n_lo=1000, n_hi=16000) -> List[Disc]:
    """D independent planetesimal discs (2.5 Earth masses each, 0.5-4 au)."""
    sizes = batch_sizes(D, seed, n_lo, n_hi)
    out = []
    for d, n in enumerate(sizes):
        out.append(disc_uniform(int(n), seed * 1_000_000 + d, a_min=0.5, a_max=4.0,
                                m_total=2.5 * M_EARTH, name=f"batch{d}-N{n}"))
    return out


# Named workloads: the sizes, distributions and seeds of the benchmark and test configurations.
def planet_swarm(n_disc=4000, n_swarm=80, seed=6, m_planet=10 * M_EARTH, r_lo=0.01, r_hi=0.05,
                 sigma_v=3e-4) -> Disc:
    """A planet on a circular orbit at 1 au (body 0) with n_swarm planetesimals
    placed 0.01-0.05 au from it in random directions, moving with the planet
    plus a Gaussian velocity dispersion sigma_v (au/day), followed by a
    uniform disc of n_disc planetesimals on 0.7-3 au: one dense
    close-encounter group of a protoplanet and its feeding zone (Sect. 2's
    embryo runs) inside an ordinary disc."""
    d = disc_uniform(n_disc, seed)
    rng = np.random.default_rng(seed + 1000)
    n = 1 + n_swarm + n_disc
    arr = [np.zeros(n) for _ in range(7)]
    pos = np.array([1.0, 0.0, 0.0])
    vel = np.array([0.0, np.sqrt(G_GAUSS * (1.0 + m_planet)), 0.0])
    for c in range(3):
        arr[c][0] = pos[c]
        arr[3 + c][0] = vel[c]
    arr[6][0] = m_planet
    m_pl = d.m[0]
    for k in range(1, n_swarm + 1):
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        r = rng.uniform(r_lo, r_hi)
        for c in range(3):
            arr[c][k] = pos[c] + r * u[c]
            arr[3 + c][k] = vel[c] + sigma_v * rng.normal()
        arr[6][k] = m_pl
    for c, src in enumerate(d.arrays()):
        arr[c][1 + n_swarm:] = src
    return Disc(f"swarm-N{n}-s{seed}", *arr, Mstar=1.0, G=G_GAUSS, dt=6.0,
                meta={"seed": seed, "kind": "planet_swarm", "n_swarm": n_swarm})


def workload(name: str):
    if name == "disc2048":        # 2,048 planetesimals, 0.7-3.0 au, 2.5 Earth masses
        return disc_uniform(2048, 1)
    if name == "embryo6625":      # 25 embryos + 6,600 planetesimals
        return embryo_disc(25, 6600, 2)
    if name == "disc40k":         # 40,000 planetesimals, Sigma ~ a^-1.5 on 0.5-4 au
        return disc_powerlaw(40_000, 3)
    if name == "batch256":        # 256 discs of 1k-16k bodies
        return batch_of_discs(256, 4)
    if name == "giants100k":      # 4 giants + 100,000 planetesimals
        return giants_disc(100_000, 5)
    if name == "swarm4k":         # a 10 Earth-mass planet with 80 planetesimals around it + 4,000
        return planet_swarm(4000, 80, 6)
    raise KeyError(name)
