"""Parity at the workloads' full sizes, every body against the oracle.

* disc2048 (2,048 planetesimals, FP64 kick, dt = 6 d, three mutual Hill
  radii): 100 level-0 steps through genga_step against oracle.step, every
  body to 1e-12 of its position and velocity; then the FP64 accelerations
  (1e-13 per body) and the encounter list at the final state.
* disc40k (40,000 planetesimals, the benchmark's workload, in the launch
  configuration the benchmark times): the FP32 kick (2e-5 per body) and the
  FP64 kick (1e-13) on all 40,000 bodies, and the whole encounter list.
* batch256 (256 systems of 1,000-16,000 bodies in one batched call, as the
  benchmark runs it): the batched FP32 kick and 3 batched steps, checked
  system by system on 10 systems (the smallest and the largest N_d among
  them), every body.

The oracle sums every pair of each of these (about 2 s for a 40,000-body
kick on 16 cores), so nothing is sampled.
"""
import numpy as np
import pytest

import oracle
from paper_2309_08217_gb300 import discs

pytestmark = pytest.mark.gpu

TOL = {0: 1e-13, 1: 2e-5}


def _rel(got, ref):
    num = np.sqrt(((got - ref) ** 2).sum(0))
    den = np.sqrt((ref ** 2).sum(0))
    assert np.all(num[den == 0] == 0)
    return num[den > 0] / den[den > 0]


def _params(g, d, precision):
    return g.make_params(G=d.G, Mstar=d.Mstar, dt=d.dt, n1=3.0, n2=0.4, precision=precision)


def _oracle_acc_and_pairs(arr, d):
    a, rc = oracle.rcrit(*arr, G=d.G, Mstar=d.Mstar, dt=d.dt, n1=3.0, n2=0.4)
    acc = oracle.kick_acc(arr[0], arr[1], arr[2], arr[6], a, rc, d.G, d.Mstar, 3.0, 1, 0)
    pairs, band = oracle.encounters(arr[0], arr[1], arr[2], arr[6], a, rc, 3.0, d.Mstar, 1, band=1e-9)
    return acc, pairs, band


def _gpu_kick(g, ctx, s, p, N):
    import torch
    acc = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    g.genga_kick(ctx, s, p, 0.0, acc)
    assert g.genga_get_status(ctx) == g.GENGA_OK
    return acc.view(3, N).cpu().numpy()


def _gpu_pairs(g, ctx, s, p, N):
    import torch
    cap = 4 * N + 16
    pairs = torch.zeros(2 * cap, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    g.genga_encounters(ctx, s, p, pairs, cap, cnt)
    assert g.genga_get_status(ctx) == g.GENGA_OK
    n = int(cnt.item())
    return pairs[: 2 * n].view(-1, 2).cpu().numpy()


def _same_pairs(got, ref, band):
    assert np.all(got[:, 0] < got[:, 1])
    if len(got) > 1:
        keys = got[:, 0].astype(np.int64) * (1 << 32) + got[:, 1]
        assert np.all(np.diff(keys) > 0)
    gs, rs, bs = (set(map(tuple, a.tolist())) for a in (got, ref, band))
    assert gs - bs == rs - bs


def _per_body_state_err(got, ref):
    ep = np.sqrt(((np.stack(got[:3]) - np.stack(ref[:3])) ** 2).sum(0)) / np.sqrt((np.stack(ref[:3]) ** 2).sum(0))
    ev = np.sqrt(((np.stack(got[3:6]) - np.stack(ref[3:6])) ** 2).sum(0)) / np.sqrt((np.stack(ref[3:6]) ** 2).sum(0))
    return ep.max(), ev.max()


# ------------------------------------------------------------- disc2048 --
def test_disc2048_fp64_100_steps(genga):
    d = discs.workload("disc2048")
    ctx = genga.Context(d.N)
    p = _params(genga, d, genga.GENGA_FP64)
    s = genga.DeviceSystem.from_disc(d)
    genga.genga_step(ctx, s, p, 100)
    assert genga.genga_get_status(ctx) == genga.GENGA_OK
    got = s.numpy()
    ref = oracle.disc_arrays(d)
    assert oracle.step(ref, d.G, d.Mstar, d.dt, 3.0, 0.4, 1, 0, 100) == 0
    ep, ev = _per_body_state_err(got, ref)
    assert ep < 1e-12 and ev < 1e-12, (ep, ev)
    assert np.array_equal(got[6], ref[6])
    # the outputs at the final state: FP64 accelerations and the encounter list
    # (the oracle evaluates them on the GPU's final state, so the comparison
    # holds the kick alone, not the 100 steps' rounding differences)
    fin = discs.Disc("disc2048_t100", *[a.copy() for a in got], G=d.G, Mstar=d.Mstar, dt=d.dt)
    acc_ref, pr, band = _oracle_acc_and_pairs(oracle.disc_arrays(fin), fin)
    sf = genga.DeviceSystem.from_disc(fin)
    assert _rel(_gpu_kick(genga, ctx, sf, p, d.N), acc_ref).max() <= TOL[0]
    _same_pairs(_gpu_pairs(genga, ctx, sf, p, d.N), pr, band)
    ctx.close()


# -------------------------------------------------------------- disc40k --
@pytest.fixture(scope="module")
def disc40k_ref():
    d = discs.workload("disc40k")
    acc, pairs, band = _oracle_acc_and_pairs(oracle.disc_arrays(d), d)
    return d, acc, pairs, band


@pytest.fixture(scope="module")
def ctx40k(genga):
    c = genga.Context(40_000)
    yield c
    c.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_disc40k_every_body(genga, ctx40k, disc40k_ref, precision):
    d, ref, _, _ = disc40k_ref
    s = genga.DeviceSystem.from_disc(d)
    got = _gpu_kick(genga, ctx40k, s, _params(genga, d, precision), d.N)
    err = _rel(got, ref)
    assert err.size == d.N
    assert err.max() <= TOL[precision], f"max err {err.max():.3e} at body {err.argmax()}"


def test_disc40k_encounter_list(genga, ctx40k, disc40k_ref):
    d, _, pairs, band = disc40k_ref
    s = genga.DeviceSystem.from_disc(d)
    got = _gpu_pairs(genga, ctx40k, s, _params(genga, d, genga.GENGA_FP32), d.N)
    assert len(pairs) > 50            # the disc has encounters at t = 0
    _same_pairs(got, pairs, band)


# ------------------------------------------------------------- batch256 --
@pytest.fixture(scope="module")
def batch256(genga):
    ds = discs.workload("batch256")
    sizes = np.array([d.N for d in ds])
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    padded = int(sum((n + 1023) // 1024 * 1024 for n in sizes))
    arrays = [np.concatenate([d.arrays()[c] for d in ds]) for c in range(7)]
    order = np.argsort(sizes)
    picks = sorted(set([int(order[0]), int(order[-1])] + [int(k) for k in np.linspace(0, len(ds) - 1, 8).round()]))
    ctx = genga.Context(padded)
    yield ds, offsets, arrays, picks, ctx
    ctx.close()


def test_batch256_kick_system_by_system(genga, batch256):
    import torch
    ds, offsets, arrays, picks, ctx = batch256
    NT = int(offsets[-1])
    s = genga.DeviceSystem.from_arrays(arrays)
    p = _params(genga, ds[0], genga.GENGA_FP32)
    acc = torch.zeros(3 * NT, dtype=torch.float64, device="cuda")
    genga.genga_kick_batched(ctx, s, offsets, p, 0.0, acc)
    assert genga.genga_get_status(ctx) == genga.GENGA_OK
    got = acc.view(3, NT).cpu().numpy()
    assert len(picks) >= 8
    for k in picks:
        d = ds[k]
        lo, hi = int(offsets[k]), int(offsets[k + 1])
        arr = oracle.disc_arrays(d)
        a, rc = oracle.rcrit(*arr, G=d.G, Mstar=d.Mstar, dt=d.dt, n1=3.0, n2=0.4)
        ref = oracle.kick_acc(arr[0], arr[1], arr[2], arr[6], a, rc, d.G, d.Mstar, 3.0, 1, 0)
        err = _rel(got[:, lo:hi], ref)
        assert err.size == d.N and err.max() <= TOL[1], f"system {k} (N = {d.N}): {err.max():.3e}"


def test_batch256_three_steps_system_by_system(genga, batch256):
    ds, offsets, arrays, picks, ctx = batch256
    s = genga.DeviceSystem.from_arrays(arrays)
    p = _params(genga, ds[0], genga.GENGA_FP32)
    genga.genga_step_batched(ctx, s, offsets, p, 3)
    assert genga.genga_get_status(ctx) == genga.GENGA_OK
    got = s.numpy()
    for k in picks:
        d = ds[k]
        lo, hi = int(offsets[k]), int(offsets[k + 1])
        ref = oracle.disc_arrays(d)
        assert oracle.step(ref, d.G, d.Mstar, d.dt, 3.0, 0.4, 1, 0, 3) == 0
        ep, ev = _per_body_state_err([a[lo:hi] for a in got], ref)
        # FP32 pair terms (<= 2e-5 of a) over 3 steps: far below 1e-9 of the state
        assert ep < 1e-9 and ev < 1e-9, f"system {k} (N = {d.N}): {ep:.3e} {ev:.3e}"
