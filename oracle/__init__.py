"""CPU FP64 oracle of the GENGA long-range kick path (test infrastructure).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  Nothing in the product
package imports this module, and this module imports nothing from it.

The arithmetic lives in ``oracle.c`` (plain C, FP64, compensated sums in
index order).  This file compiles it with the host C compiler and wraps it
with numpy-friendly functions.  Each function cites the part of the paper
it follows (see the header of ``oracle.c``).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = C.POINTER(C.c_double)
_i64p = C.POINTER(C.c_int64)
_i32p = C.POINTER(C.c_int32)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (no fast-math, no FMA contraction)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    cc = os.environ.get("CC", "gcc")
    base = [cc, "-O2", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC", _SRC,
            "-o", _LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)   # no OpenMP: serial oracle
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        alt = os.environ.get("ORACLE_LIB")      # a mutated build, for the mutation test only
        if alt:
            lib = C.CDLL(alt)
        else:
            build()
            lib = C.CDLL(_LIB)
        i, d = C.c_int, C.c_double
        sig = {
            "oracle_threads": ([], i),
            "oracle_set_threads": ([i], None),
            "oracle_changeover": ([d, i], d),
            "oracle_momentum": ([i, _dp, _dp, _dp, _dp, _dp], None),
            "oracle_rcrit": ([i] + [_dp] * 7 + [d] * 5 + [_dp, _dp], None),
            "oracle_pair_rcrit": ([i, d, d, d, d, d, d, d, d], d),
            "oracle_kick_acc": ([i] + [_dp] * 6 + [d, d, d, i, i, i, i, _i64p] + [_dp] * 4, None),
            "oracle_kick": ([i] + [_dp] * 7 + [d] * 5 + [i, i, i, d] + [_dp] * 3, None),
            "oracle_encounters": ([i] + [_dp] * 6 + [d, d, i, i, _i32p, C.c_int64, d, _i32p,
                                                    C.c_int64, _i64p], C.c_int64),
            "oracle_kepler": ([d, _dp, d, i], i),
            "oracle_hc_drift": ([i] + [_dp] * 7 + [d, d], None),
            "oracle_drift": ([i] + [_dp] * 7 + [d, d, d, i], i),
            "oracle_step": ([i] + [_dp] * 7 + [d] * 5 + [i, i, i, i, i], i),
            "oracle_energy": ([i] + [_dp] * 7 + [d, d, i, _dp], None),
            "oracle_groups": ([i, C.c_int64, _i32p, _i32p], i),
            "oracle_predicted_pairs": ([i] + [_dp] * 9 + [d, d, i, i, d, _i32p, C.c_int64], C.c_int64),
            "oracle_bs_acc": ([i, _i32p] + [_dp] * 6 + [d, d, d, i, i, i, _dp], None),
            "oracle_bs_group": ([i, _i32p] + [_dp] * 9 + [d, d, d, i, i, i, d, d], i),
            "oracle_drift_groups": ([i] + [_dp] * 9 + [C.c_int64, _i32p, d, d, d, i, i, i, d, d, i,
                                                       C.POINTER(C.c_int)], i),
            "oracle_step_bs": ([i] + [_dp] * 7 + [d] * 5 + [i, i, i, i, d, i, C.POINTER(C.c_int)], i),
            "oracle_step_full": ([i] + [_dp] * 8 + [_i32p] + [d] * 5 + [i, i, i, i, d, d, d, i,
                                                                        C.POINTER(C.c_int), C.POINTER(C.c_int)], i),
            "oracle_bs_group_full": ([i, _i32p] + [_dp] * 10 + [_i32p, d, d, d, i, i, i, d, d,
                                                                  C.POINTER(C.c_int)], i),
            "oracle_ml_radius": ([d, i, i], d),
            "oracle_ml_weight": ([d, d, i, i, i, i], d),
            "oracle_bs_group_counted": ([i, _i32p] + [_dp] * 9 + [d, d, d, i, i, i, d, d, C.POINTER(C.c_int),
                                                                   C.POINTER(C.c_int)], i),
            "oracle_ml_level_acc": ([i, _i32p] + [_dp] * 6 + [d, d, d, i, i, i, i, i, i, _dp], None),
            "oracle_ml_subpairs": ([i, _i32p] + [_dp] * 9 + [d, d, i, i, i, i, d, _i32p, C.c_int64], C.c_int64),
            "oracle_bs_acc_ml": ([i, _i32p] + [_dp] * 6 + [d, d, d, i, i, i, i, i, _dp], None),
            "oracle_ml_group": ([i, _i32p] + [_dp] * 10 + [_i32p, d, d, d, i, i, i, d, d, i, i, i,
                                                             C.POINTER(C.c_int), C.POINTER(C.c_int)], i),
            "oracle_drift_groups_ml": ([i] + [_dp] * 10 + [_i32p, C.c_int64, _i32p, d, d, d, i, i, i, d, d, i, d, d,
                                                         i, i, C.POINTER(C.c_int), C.POINTER(C.c_int)], i),
            "oracle_step_ml": ([i] + [_dp] * 8 + [_i32p] + [d] * 5 + [i, i, i, i, d, d, d, i, i, i,
                                                                      C.POINTER(C.c_int), C.POINTER(C.c_int)], i),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def _p(a):
    return a.ctypes.data_as(_dp)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def threads() -> int:
    return int(_load().oracle_threads())


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


# ------------------------------------------------------------------ Sect. 1
def changeover(y, form: int = 0):
    """K(y): the changeover weight (Chambers 1999 form 0, quintic form 1)."""
    lib = _load()
    y = np.asarray(y, dtype=np.float64)
    out = np.array([lib.oracle_changeover(float(v), int(form)) for v in y.ravel()])
    return out.reshape(y.shape) if y.shape else float(out[0])


def momentum(vx, vy, vz, m):
    P = np.zeros(3)
    vx, vy, vz, m = map(_f64, (vx, vy, vz, m))
    _load().oracle_momentum(len(m), _p(vx), _p(vy), _p(vz), _p(m), _p(P))
    return P


def rcrit(x, y, z, vx, vy, vz, m, G, Mstar, dt, n1=3.0, n2=0.4):
    """Eq. (1): per-body osculating a_i and r_crit,i = max(n1 R_H,i, n2 dt v_i)."""
    arrs = [_f64(v) for v in (x, y, z, vx, vy, vz, m)]
    N = len(arrs[-1])
    a = np.zeros(N)
    rc = np.zeros(N)
    _load().oracle_rcrit(N, *map(_p, arrs), G, Mstar, dt, n1, n2, _p(a), _p(rc))
    return a, rc


def pair_rcrit(mode, mi, mj, ai, aj, rci, rcj, n1, Mstar):
    return float(_load().oracle_pair_rcrit(int(mode), mi, mj, ai, aj, rci, rcj, n1, Mstar))


def kick_acc(x, y, z, m, a, rc, G, Mstar, n1=3.0, mode=1, form=0, idx=None, with_abs=False, n_big=-1):
    """Sect. 1 long-range sum a_i = sum_{j!=i} G m_j K (x_j-x_i)/r^3 for i in idx
    (n_big >= 0: test-particle mode 2, no force between bodies >= n_big)."""
    arrs = [_f64(v) for v in (x, y, z, m, a, rc)]
    N = len(arrs[3])
    idx = np.arange(N, dtype=np.int64) if idx is None else np.ascontiguousarray(idx, np.int64)
    n = len(idx)
    ax, ay, az, ab = np.zeros(n), np.zeros(n), np.zeros(n), np.zeros(n)
    _load().oracle_kick_acc(N, *map(_p, arrs), G, Mstar, n1, int(mode), int(form), int(n_big), n,
                            idx.ctypes.data_as(_i64p), _p(ax), _p(ay), _p(az),
                            _p(ab) if with_abs else None)
    acc = np.stack([ax, ay, az])
    return (acc, ab) if with_abs else acc


def kick(disc_arrays, G, Mstar, dt, n1, n2, mode, form, tau, n_big=-1):
    """r_crit from the current state, then v += a tau (in place); returns acc."""
    x, y, z, vx, vy, vz, m = disc_arrays
    N = len(m)
    ax, ay, az = np.zeros(N), np.zeros(N), np.zeros(N)
    _load().oracle_kick(N, *map(_p, (x, y, z, vx, vy, vz, m)), G, Mstar, dt, n1, n2,
                        int(mode), int(form), int(n_big), tau, _p(ax), _p(ay), _p(az))
    return np.stack([ax, ay, az])


def encounters(x, y, z, m, a, rc, n1, Mstar, mode=1, band=1e-9, cap=None, n_big=-1):
    """Pairs i<j with r_ij < r_crit,ij (lexicographic) and the +-band pairs."""
    arrs = [_f64(v) for v in (x, y, z, m, a, rc)]
    N = len(arrs[3])
    lib = _load()
    cap = cap if cap is not None else max(16, 4 * N)
    bcap = max(16, N)
    pairs = np.zeros(2 * cap, np.int32)
    bpairs = np.zeros(2 * bcap, np.int32)
    bcount = np.zeros(1, np.int64)
    cnt = lib.oracle_encounters(N, *map(_p, arrs), n1, Mstar, int(mode), int(n_big),
                                pairs.ctypes.data_as(_i32p), cap, band,
                                bpairs.ctypes.data_as(_i32p), bcap, bcount.ctypes.data_as(_i64p))
    if cnt > cap or bcount[0] > bcap:
        return encounters(x, y, z, m, a, rc, n1, Mstar, mode, band,
                          cap=int(max(cnt, bcount[0], cap) * 2), n_big=n_big)
    return (pairs[: 2 * cnt].reshape(-1, 2).copy(),
            bpairs[: 2 * int(bcount[0])].reshape(-1, 2).copy())


def kepler(mu, xv, dt, max_iter=50):
    """Universal-variable two-body drift of one body; returns (state, status)."""
    s = _f64(np.array(xv, dtype=np.float64).copy())
    st = _load().oracle_kepler(mu, _p(s), dt, int(max_iter))
    return s, int(st)


def hc_drift(arrs, Mstar, tau):
    x, y, z, vx, vy, vz, m = arrs
    _load().oracle_hc_drift(len(m), *map(_p, (x, y, z, vx, vy, vz, m)), Mstar, tau)


def drift(arrs, G, Mstar, dt, max_iter=50):
    """HC(dt/2) Kepler(dt) HC(dt/2), in place; returns the non-converged count."""
    x, y, z, vx, vy, vz, m = arrs
    return int(_load().oracle_drift(len(m), *map(_p, (x, y, z, vx, vy, vz, m)), G, Mstar, dt,
                                    int(max_iter)))


def step(arrs, G, Mstar, dt, n1, n2, mode, form, nsteps, max_iter=50, n_big=-1, bs_tol=0.0,
         forced=None, radius=None, dead=None, r_in=0.0, r_out=0.0, merges=None, n_levels=0, n_sub=2):
    """nsteps of kick(dt/2) drift(dt) kick(dt/2), in place.  bs_tol > 0: the
    drift integrates the encounter groups of each step's first kick with the
    Bulirsch-Stoer level at that tolerance (forced: optional one-element list
    that accumulates the forced acceptances).  radius (per body, float64,
    updated) turns on perfect mergers inside that level, r_in / r_out (> 0)
    the removal radii; dead (per body, int32, updated) marks the bodies merged
    away or removed (they stay as massless ghosts); merges: optional
    one-element list that accumulates the mergers.  n_levels >= 1: that many
    intermediate levels of n_sub sub-steps between the kick and the
    Bulirsch-Stoer level.  Returns the Kepler cap count."""
    x, y, z, vx, vy, vz, m = arrs
    if radius is not None or dead is not None or r_in > 0.0 or r_out > 0.0 or n_levels > 0:
        assert bs_tol > 0.0
        if radius is not None or r_in > 0.0 or r_out > 0.0:
            assert dead is not None and dead.dtype == np.int32
        f, mg = C.c_int(0), C.c_int(0)
        rp = _p(radius) if radius is not None else None
        dp = dead.ctypes.data_as(_i32p) if dead is not None else None
        bad = int(_load().oracle_step_ml(len(m), *map(_p, (x, y, z, vx, vy, vz, m)), rp, dp, G, Mstar, dt, n1, n2,
                                         int(mode), int(form), int(n_big), int(max_iter), float(bs_tol),
                                         float(r_in), float(r_out), int(n_levels), int(n_sub), int(nsteps),
                                         C.byref(f), C.byref(mg)))
        if forced is not None:
            forced[0] += f.value
        if merges is not None:
            merges[0] += mg.value
        return bad
    if bs_tol <= 0.0:
        return int(_load().oracle_step(len(m), *map(_p, (x, y, z, vx, vy, vz, m)), G, Mstar, dt,
                                       n1, n2, int(mode), int(form), int(n_big), int(max_iter),
                                       int(nsteps)))
    f = C.c_int(0)
    bad = int(_load().oracle_step_bs(len(m), *map(_p, (x, y, z, vx, vy, vz, m)), G, Mstar, dt,
                                     n1, n2, int(mode), int(form), int(n_big), int(max_iter),
                                     float(bs_tol), int(nsteps), C.byref(f)))
    if forced is not None:
        forced[0] += f.value
    return bad


# ------------------------------------------- close-encounter level, Sect. 1
def groups(N, pairs):
    """Connected components of the encounter pairs: label[v] = smallest body
    of v's group, -1 for bodies in no pair; returns (label, number of groups)."""
    pairs = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
    label = np.zeros(max(N, 1), np.int32)
    ng = _load().oracle_groups(int(N), len(pairs), pairs.ctypes.data_as(_i32p),
                               label.ctypes.data_as(_i32p))
    return label[:N], int(ng)


def predicted_pairs(arrs, a, rc, n1, Mstar, mode, dt, n_big=-1):
    """Pairs i < j outside r_crit,ij but within 1.5 r_crit,ij whose straight-line
    relative motion over the coming drift of length dt enters r_crit,ij."""
    x, y, z, vx, vy, vz, m = [_f64(v) for v in arrs]
    a, rc = _f64(a), _f64(rc)
    N = len(m)
    cap = max(16, 4 * N)
    out = np.zeros(2 * cap, np.int32)
    n = _load().oracle_predicted_pairs(N, *map(_p, (x, y, z, vx, vy, vz, m, a, rc)), n1, Mstar, int(mode),
                                       int(n_big), float(dt), out.ctypes.data_as(_i32p), cap)
    assert n <= cap
    return out[: 2 * n].reshape(-1, 2).copy()


def bs_acc(x, y, z, m, a, rc, members, G, Mstar, n1, mode, form, n_big=-1):
    """Level-1 acceleration of each member of a group: the central body plus
    the (1 - K) part of the members' pair forces; shape (3, len(members))."""
    mem = np.ascontiguousarray(np.asarray(members, dtype=np.int32))
    out = np.zeros(3 * max(len(mem), 1))
    _load().oracle_bs_acc(len(mem), mem.ctypes.data_as(_i32p), *map(_p, map(_f64, (x, y, z, m, a, rc))),
                          G, Mstar, n1, int(mode), int(form), int(n_big), _p(out))
    return out[: 3 * len(mem)].reshape(-1, 3).T.copy()


def bs_group(arrs, members, a, rc, G, Mstar, n1, mode, form, dt, tol, n_big=-1, radius=None,
             dead=None, merges=None):
    """Bulirsch-Stoer integration of one group (ascending body indices) over
    dt under the central body and the (1 - K) part of the members' pair
    forces, in place; returns 1 if an acceptance was forced, else 0.  With
    radius (and dead, int32 per body) overlapping members merge after every
    accepted sub-step (m, radius and dead updated in place)."""
    x, y, z, vx, vy, vz, m = arrs
    mem = np.ascontiguousarray(np.asarray(members, dtype=np.int32))
    a, rc = _f64(a), _f64(rc)
    if radius is not None:
        assert dead is not None and dead.dtype == np.int32
        mg = C.c_int(0)
        f = int(_load().oracle_bs_group_full(len(mem), mem.ctypes.data_as(_i32p),
                                             *map(_p, (x, y, z, vx, vy, vz, m, a, rc, radius)),
                                             dead.ctypes.data_as(_i32p), G, Mstar, n1, int(mode), int(form),
                                             int(n_big), float(dt), float(tol), C.byref(mg)))
        if merges is not None:
            merges[0] += mg.value
        return f
    return int(_load().oracle_bs_group(len(mem), mem.ctypes.data_as(_i32p),
                                       *map(_p, (x, y, z, vx, vy, vz, m, a, rc)), G, Mstar, n1,
                                       int(mode), int(form), int(n_big), float(dt), float(tol)))


def ml_radius(rc, level, n_sub):
    """r_crit of level l: rc / n_sub^l."""
    return float(_load().oracle_ml_radius(float(rc), int(level), int(n_sub)))


def ml_weight(q, rc, level, n_levels, n_sub, form):
    """Share of the pair force at separation q (pair radius rc) that level
    `level` applies: K_l prod_{k<l}(1 - K_k) for level <= n_levels, the
    Bulirsch-Stoer share prod_{k<=n_levels}(1 - K_k) for level = n_levels + 1."""
    return float(_load().oracle_ml_weight(float(q), float(rc), int(level), int(n_levels), int(n_sub), int(form)))


def ml_level_acc(x, y, z, m, a, rc, members, G, Mstar, n1, mode, form, level, n_levels, n_sub, n_big=-1):
    """Level `level`'s share of the pair forces on each member (no central
    term), shape (3, n)."""
    mem = np.ascontiguousarray(np.asarray(members, dtype=np.int32))
    acc = np.zeros(3 * max(len(mem), 1))
    _load().oracle_ml_level_acc(len(mem), mem.ctypes.data_as(_i32p), *map(_p, [_f64(v) for v in (x, y, z, m, a, rc)]),
                                G, Mstar, n1, int(mode), int(form), int(n_big), int(level), int(n_levels), int(n_sub),
                                _p(acc))
    return acc[: 3 * len(mem)].reshape(-1, 3).T


def bs_acc_ml(x, y, z, m, a, rc, members, G, Mstar, n1, mode, form, n_levels, n_sub, n_big=-1):
    """The Bulirsch-Stoer level's acceleration of each member (central term
    plus the share prod_{k<=L}(1 - K_k) of the pair forces), shape (3, n)."""
    mem = np.ascontiguousarray(np.asarray(members, dtype=np.int32))
    acc = np.zeros(3 * max(len(mem), 1))
    _load().oracle_bs_acc_ml(len(mem), mem.ctypes.data_as(_i32p), *map(_p, [_f64(v) for v in (x, y, z, m, a, rc)]),
                             G, Mstar, n1, int(mode), int(form), int(n_big), int(n_levels), int(n_sub), _p(acc))
    return acc[: 3 * len(mem)].reshape(-1, 3).T


def ml_subpairs(arrs, members, a, rc, n1, Mstar, mode, level, n_sub, h, n_big=-1):
    """The member pairs that form the subgroups of level + 1 for a drift of h."""
    x, y, z, vx, vy, vz, m = [_f64(v) for v in arrs]
    mem = np.ascontiguousarray(np.asarray(members, dtype=np.int32))
    cap = max(16, len(mem) * len(mem))
    out = np.zeros(2 * cap, np.int32)
    n = _load().oracle_ml_subpairs(len(mem), mem.ctypes.data_as(_i32p), *map(_p, (x, y, z, vx, vy, vz, m)),
                                   *map(_p, (_f64(a), _f64(rc))), n1, Mstar, int(mode), int(n_big), int(level),
                                   int(n_sub), float(h), out.ctypes.data_as(_i32p), cap)
    return out[: 2 * n].reshape(-1, 2).copy()


def ml_group(arrs, members, a, rc, G, Mstar, n1, mode, form, dt, tol, n_levels, n_sub, n_big=-1,
             radius=None, dead=None, merges=None, max_iter=50):
    """One group (ascending body indices) over dt on level 1 with n_levels
    intermediate levels of n_sub symplectic sub-steps and the Bulirsch-Stoer
    level below them, in place; returns (forced, Kepler cap count)."""
    x, y, z, vx, vy, vz, m = arrs
    mem = np.ascontiguousarray(np.asarray(members, dtype=np.int32))
    a, rc = _f64(a), _f64(rc)
    mg, bad = C.c_int(0), C.c_int(0)
    rp = _p(radius) if radius is not None else None
    dp = dead.ctypes.data_as(_i32p) if dead is not None else None
    f = int(_load().oracle_ml_group(len(mem), mem.ctypes.data_as(_i32p), *map(_p, (x, y, z, vx, vy, vz, m, a, rc)),
                                    rp, dp, G, Mstar, n1, int(mode), int(form), int(n_big), float(dt), float(tol),
                                    int(n_levels), int(n_sub), int(max_iter), C.byref(mg), C.byref(bad)))
    if merges is not None:
        merges[0] += mg.value
    return f, bad.value


def bs_group_counted(arrs, members, a, rc, G, Mstar, n1, mode, form, dt, tol, n_big=-1):
    """bs_group without collisions; returns (forced, accepted sub-steps, attempts)."""
    x, y, z, vx, vy, vz, m = arrs
    mem = np.ascontiguousarray(np.asarray(members, dtype=np.int32))
    acc_, att_ = C.c_int(0), C.c_int(0)
    f = int(_load().oracle_bs_group_counted(len(mem), mem.ctypes.data_as(_i32p),
                                            *map(_p, (x, y, z, vx, vy, vz, m, _f64(a), _f64(rc))), G, Mstar, n1,
                                            int(mode), int(form), int(n_big), float(dt), float(tol),
                                            C.byref(acc_), C.byref(att_)))
    return f, acc_.value, att_.value


def drift_groups(arrs, a, rc, pairs, G, Mstar, n1, mode, form, dt, tol, n_big=-1, max_iter=50, n_levels=0,
                 n_sub=2):
    """HC(dt/2); Kepler for bodies outside the groups of `pairs`, the
    Bulirsch-Stoer level for each group (below n_levels intermediate levels of
    n_sub sub-steps); HC(dt/2).  In place; returns (Kepler cap count, groups
    with a forced acceptance)."""
    x, y, z, vx, vy, vz, m = arrs
    pairs = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
    a, rc = _f64(a), _f64(rc)
    f = C.c_int(0)
    if n_levels > 0:
        bad = int(_load().oracle_drift_groups_ml(len(m), *map(_p, (x, y, z, vx, vy, vz, m, a, rc)), None, None,
                                                 len(pairs), pairs.ctypes.data_as(_i32p), G, Mstar, n1, int(mode),
                                                 int(form), int(n_big), float(dt), float(tol), int(max_iter), 0.0, 0.0,
                                                 int(n_levels), int(n_sub), C.byref(f), None))
        return bad, f.value
    bad = int(_load().oracle_drift_groups(len(m), *map(_p, (x, y, z, vx, vy, vz, m, a, rc)),
                                          len(pairs), pairs.ctypes.data_as(_i32p), G, Mstar, n1,
                                          int(mode), int(form), int(n_big), float(dt), float(tol),
                                          int(max_iter), C.byref(f)))
    return bad, f.value


def energy(arrs, G, Mstar, n_big=-1):
    """(E, Lx, Ly, Lz) of the democratic-heliocentric Hamiltonian."""
    x, y, z, vx, vy, vz, m = [_f64(v) for v in arrs]
    out = np.zeros(4)
    _load().oracle_energy(len(m), *map(_p, (x, y, z, vx, vy, vz, m)), G, Mstar, int(n_big), _p(out))
    return out


def disc_arrays(disc):
    """Writable float64 copies of a Disc's seven state arrays."""
    return [np.array(a, dtype=np.float64, copy=True) for a in disc.arrays()]
