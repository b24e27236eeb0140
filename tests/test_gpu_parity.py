"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances (per body, err_i = |a_gpu - a_oracle| / |a_oracle|, max over i):
  FP64 kick  1e-13     FP32 kick  2e-5
The encounter list must equal the oracle's except for pairs whose distance is
within 1e-9 relative of r_crit,ij (either side), where both answers are valid.
Drift and step states are compared coordinate-wise, relative to the size of
the position / velocity vector.
"""
import numpy as np
import pytest

import oracle
from paper_2309_08217_gb300 import discs
from tests.gpu_cases import planted_disc

pytestmark = pytest.mark.gpu

TOL = {0: 1e-13, 1: 2e-5}   # precision -> per-body relative tolerance


def _params(g, d, precision, mode=1, form=0, maxit=50):
    return g.make_params(G=d.G, Mstar=d.Mstar, dt=d.dt, n1=3.0, n2=0.4, rcrit_mode=mode, changeover=form,
                         precision=precision, kepler_max_iter=maxit)


def _oracle_acc(d, mode=1, form=0, idx=None):
    arr = oracle.disc_arrays(d)
    a, rc = oracle.rcrit(*arr, G=d.G, Mstar=d.Mstar, dt=d.dt, n1=3.0, n2=0.4)
    acc = oracle.kick_acc(arr[0], arr[1], arr[2], arr[6], a, rc, d.G, d.Mstar, 3.0, mode, form, idx=idx)
    return acc, a, rc


def _gpu_acc(g, ctx, d, precision, mode=1, form=0):
    import torch
    s = g.DeviceSystem.from_disc(d)
    acc = torch.zeros(3 * max(d.N, 1), dtype=torch.float64, device="cuda")
    g.genga_kick(ctx, s, _params(g, d, precision, mode, form), 0.0, acc)
    assert g.genga_get_status(ctx) == g.GENGA_OK
    return acc[: 3 * d.N].view(3, d.N).cpu().numpy() if d.N else np.zeros((3, 0)), s


def _rel_err(got, ref):
    num = np.sqrt(((got - ref) ** 2).sum(0))
    den = np.sqrt((ref ** 2).sum(0))
    ok = den > 0
    assert np.all(num[~ok] == 0)
    return num[ok] / den[ok]


@pytest.fixture(scope="module")
def ctx(genga):
    c = genga.Context(120_000)
    yield c
    c.close()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("N", [1, 2, 3, 31, 33, 255, 1000, 1024, 3001])
def test_kick_parity_sizes(genga, ctx, precision, N):
    d = planted_disc(N, 100 + N)
    got, _ = _gpu_acc(genga, ctx, d, precision)
    ref, _, _ = _oracle_acc(d)
    if N == 1:
        assert np.all(got == 0)
        return
    err = _rel_err(got, ref)          # bodies with zero acceleration must match exactly
    if err.size:
        assert err.max() <= TOL[precision], f"max err {err.max():.3e} at body {err.argmax()}"


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("mode,form", [(0, 0), (0, 1), (1, 1)])
def test_kick_parity_modes(genga, ctx, precision, mode, form):
    d = planted_disc(1500, 7)
    got, _ = _gpu_acc(genga, ctx, d, precision, mode, form)
    ref, _, _ = _oracle_acc(d, mode, form)
    assert _rel_err(got, ref).max() <= TOL[precision]


def test_every_fp32_variant(genga, ctx):
    """Each FP32 pass variant the autotuner may pick meets the tolerance."""
    d = planted_disc(5000, 8)
    ref, _, _ = _oracle_acc(d)
    _, nvar = genga.genga_get_kernel_variant(ctx, d.N)
    assert nvar >= 2
    try:
        for v in range(nvar):
            genga.genga_set_kernel_variant(ctx, v)
            got, _ = _gpu_acc(genga, ctx, d, 1)
            assert _rel_err(got, ref).max() <= TOL[1], f"variant {v}"
    finally:
        genga.genga_set_kernel_variant(ctx, -1)
    with pytest.raises(genga.GengaError):
        genga.genga_set_kernel_variant(ctx, nvar)


def test_kick_embryos_mixed_masses(genga, ctx):
    d = discs.embryo_disc(25, 2000, seed=9)
    for precision in (0, 1):
        got, _ = _gpu_acc(genga, ctx, d, precision)
        ref, _, _ = _oracle_acc(d)
        assert _rel_err(got, ref).max() <= TOL[precision]


def test_kick_updates_velocity(genga, ctx):
    import torch
    d = planted_disc(700, 3)
    s = genga.DeviceSystem.from_disc(d)
    acc = torch.zeros(3 * d.N, dtype=torch.float64, device="cuda")
    genga.genga_kick(ctx, s, _params(genga, d, 0), 3.0, acc)
    assert genga.genga_get_status(ctx) == genga.GENGA_OK
    v = s.numpy()
    arr = oracle.disc_arrays(d)
    oracle.kick(arr, d.G, d.Mstar, d.dt, 3.0, 0.4, 1, 0, 3.0)
    for c in (3, 4, 5):
        assert np.allclose(v[c], arr[c], rtol=1e-13, atol=1e-18)
    for c in (0, 1, 2, 6):
        assert np.array_equal(v[c], d.arrays()[c])          # positions and masses untouched


def _encounter_sets(genga, ctx, d, mode, precision_for_pass=None):
    import torch
    s = genga.DeviceSystem.from_disc(d)
    cap = 4 * d.N + 16
    pairs = torch.zeros(2 * cap, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    genga.genga_encounters(ctx, s, _params(genga, d, 1, mode), pairs, cap, cnt)
    assert genga.genga_get_status(ctx) == genga.GENGA_OK
    n = int(cnt.item())
    got = pairs[: 2 * n].view(-1, 2).cpu().numpy()
    arr = oracle.disc_arrays(d)
    a, rc = oracle.rcrit(*arr, G=d.G, Mstar=d.Mstar, dt=d.dt, n1=3.0, n2=0.4)
    ref, band = oracle.encounters(arr[0], arr[1], arr[2], arr[6], a, rc, 3.0, d.Mstar, mode, band=1e-9)
    return got, ref, band


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("N", [2, 64, 1000, 3001])
def test_encounter_list(genga, ctx, mode, N):
    d = planted_disc(N, 200 + N)
    got, ref, band = _encounter_sets(genga, ctx, d, mode)
    # sorted, i < j, unique
    assert np.all(got[:, 0] < got[:, 1])
    if len(got) > 1:
        keys = got[:, 0].astype(np.int64) * (1 << 32) + got[:, 1]
        assert np.all(np.diff(keys) > 0)
    gs = set(map(tuple, got.tolist()))
    rs = set(map(tuple, ref.tolist()))
    bs = set(map(tuple, band.tolist()))
    assert gs - bs == rs - bs
    if mode == 1 and N >= 64:
        assert len(rs) >= 3          # the planted pairs at 0.05, 0.3, 0.5, 0.9 of the Hill scale


def test_last_encounters_matches_kick(genga, ctx):
    import torch
    d = planted_disc(2000, 5)
    s = genga.DeviceSystem.from_disc(d)
    genga.genga_kick(ctx, s, _params(genga, d, 1), 0.0, None)
    pairs = torch.zeros(2 * 64, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    genga.genga_last_encounters(ctx, pairs, 64, cnt)
    assert genga.genga_get_status(ctx) == genga.GENGA_OK
    got, ref, band = _encounter_sets(genga, ctx, d, 1)
    n = int(cnt.item())
    assert n == len(got)
    assert np.array_equal(pairs[: 2 * n].view(-1, 2).cpu().numpy(), got)


def test_encounter_capacity_overflow(genga, ctx):
    import torch
    d = planted_disc(1000, 11)
    s = genga.DeviceSystem.from_disc(d)
    pairs = torch.zeros(2, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    genga.genga_encounters(ctx, s, _params(genga, d, 1, 0), pairs, 1, cnt)   # mode 0: many pairs
    assert genga.genga_get_status(ctx) == genga.GENGA_ERR_CAPACITY
    assert int(cnt.item()) > 1
    assert genga.genga_get_status(ctx) == genga.GENGA_OK                     # status was cleared


def _rel_state_err(a, b):
    pa, pb = np.stack(a[:3]), np.stack(b[:3])
    va, vb = np.stack(a[3:6]), np.stack(b[3:6])
    ep = np.abs(pa - pb).max(0) / np.sqrt((pb ** 2).sum(0))
    ev = np.abs(va - vb).max(0) / np.sqrt((vb ** 2).sum(0))
    return ep.max(), ev.max()


@pytest.mark.parametrize("N", [1, 5, 1000])
def test_drift_parity(genga, ctx, N):
    d = planted_disc(N, 300 + N)
    s = genga.DeviceSystem.from_disc(d)
    genga.genga_drift(ctx, s, _params(genga, d, 0), d.dt * 7.0)
    assert genga.genga_get_status(ctx) == genga.GENGA_OK
    arr = oracle.disc_arrays(d)
    assert oracle.drift(arr, d.G, d.Mstar, d.dt * 7.0) == 0
    ep, ev = _rel_state_err(s.numpy(), arr)
    assert ep < 1e-13 and ev < 1e-13


def test_drift_eccentric_orbits(genga, ctx):
    rng = np.random.default_rng(5)
    n = 64
    mu = discs.G_GAUSS
    e = np.concatenate([np.linspace(0, 0.95, n // 2), rng.uniform(0, 0.5, n // 2)])
    pos, vel = discs.elements_to_cartesian(mu * (1 + 1e-9), rng.uniform(0.3, 30, n), e, rng.uniform(0, 1, n),
                                           rng.uniform(0, 6, n), rng.uniform(0, 6, n), rng.uniform(0, 6, n))
    arr = [pos[0], pos[1], pos[2], vel[0], vel[1], vel[2], np.full(n, 1e-9)]
    d = discs.Disc("ecc", *[a.copy() for a in arr])
    s = genga.DeviceSystem.from_disc(d)
    genga.genga_drift(ctx, s, _params(genga, d, 0), 200.0)
    assert genga.genga_get_status(ctx) == genga.GENGA_OK
    ref = oracle.disc_arrays(d)
    assert oracle.drift(ref, d.G, d.Mstar, 200.0) == 0
    ep, ev = _rel_state_err(s.numpy(), ref)
    assert ep < 1e-11 and ev < 1e-11


def test_kepler_iteration_cap_sets_status(genga, ctx):
    d = planted_disc(100, 1)
    s = genga.DeviceSystem.from_disc(d)
    genga.genga_drift(ctx, s, _params(genga, d, 0, maxit=1), 40.0)
    assert genga.genga_get_status(ctx) == genga.GENGA_ERR_KEPLER


@pytest.mark.parametrize("precision", [0, 1])
def test_step_parity(genga, ctx, precision):
    d = planted_disc(800, 17)
    s = genga.DeviceSystem.from_disc(d)
    genga.genga_step(ctx, s, _params(genga, d, precision), 3)
    assert genga.genga_get_status(ctx) == genga.GENGA_OK
    arr = oracle.disc_arrays(d)
    assert oracle.step(arr, d.G, d.Mstar, d.dt, 3.0, 0.4, 1, 0, 3) == 0
    ep, ev = _rel_state_err(s.numpy(), arr)
    if precision == 0:
        assert ep < 1e-12 and ev < 1e-12
    else:
        # velocities change by a*dt per step, a tiny fraction of v: FP32-force
        # errors (<= 2e-5 of a) stay far below 1e-9 of the state
        assert ep < 1e-9 and ev < 1e-9


def test_energy_parity(genga, ctx):
    d = planted_disc(3000, 21)
    s = genga.DeviceSystem.from_disc(d)
    E = genga.genga_energy(ctx, s, _params(genga, d, 0))
    ref = oracle.energy(oracle.disc_arrays(d), d.G, d.Mstar)
    assert abs(E[0] / ref[0] - 1) < 1e-13
    assert np.abs(np.array(E[1:]) - ref[1:]).max() < 1e-13 * np.linalg.norm(ref[1:])


def test_newton_third_law_fp64(genga, ctx):
    d = planted_disc(2048, 33)
    got, _ = _gpu_acc(genga, ctx, d, 0)
    m = d.m
    tot = (got * m).sum(1)
    assert np.all(np.abs(tot) <= 1e-13 * (np.abs(got) * m).sum())


def test_bitwise_determinism(genga, ctx):
    d = planted_disc(5000, 44)
    for precision in (0, 1):
        a1, _ = _gpu_acc(genga, ctx, d, precision)
        a2, _ = _gpu_acc(genga, ctx, d, precision)
        assert np.array_equal(a1, a2)


def test_nonfinite_input_sets_status(genga, ctx):
    import torch
    d = planted_disc(300, 2)
    d.x[5] = np.nan
    s = genga.DeviceSystem.from_disc(d)
    acc = torch.zeros(3 * d.N, dtype=torch.float64, device="cuda")
    genga.genga_kick(ctx, s, _params(genga, d, 1), 0.0, acc)
    assert genga.genga_get_status(ctx) == genga.GENGA_ERR_NONFINITE


def test_empty_system(genga, ctx):
    import torch
    s = genga.genga_system(0, None, None, None, None, None, None, None)
    p = genga.make_params(G=discs.G_GAUSS)
    genga.genga_kick(ctx, s, p, 1.0, None)
    genga.genga_drift(ctx, s, p, 1.0)
    genga.genga_step(ctx, s, p, 2)
    cnt = torch.full((1,), 7, dtype=torch.int32, device="cuda")
    genga.genga_encounters(ctx, s, p, None, 0, cnt)
    assert int(cnt.item()) == 0
    assert genga.genga_energy(ctx, s, p) == [0.0, 0.0, 0.0, 0.0]
    assert genga.genga_get_status(ctx) == genga.GENGA_OK


def test_invalid_arguments(genga, ctx):
    d = planted_disc(10, 1)
    s = genga.DeviceSystem.from_disc(d)
    bad = _params(genga, d, 1)
    bad.precision = 7
    with pytest.raises(genga.GengaError) as e:
        genga.genga_kick(ctx, s, bad, 0.0, None)
    assert e.value.code == genga.GENGA_ERR_INVALID_ARG
    small = genga.Context(5)
    with pytest.raises(genga.GengaError):
        genga.genga_kick(small, s, _params(genga, d, 1), 0.0, None)     # N > max_N
    small.close()


# ----------------------------------------------------- full-size workloads --
def _sampled_check(genga, ctx, d, precision, nsample=192, seed=0):
    got, _ = _gpu_acc(genga, ctx, d, precision)
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(d.N, size=min(nsample, d.N), replace=False))
    ref, _, _ = _oracle_acc(d, idx=idx)
    return _rel_err(got[:, idx], ref)


@pytest.mark.parametrize("precision", [0, 1])
def test_disc40k_sampled(genga, ctx, precision):
    """The 40,000-body power-law disc, in the launch configuration the
    benchmark times; 192 bodies are checked against the oracle one by one."""
    d = discs.workload("disc40k")
    err = _sampled_check(genga, ctx, d, precision)
    assert err.max() <= TOL[precision]


def test_giants100k_sampled_fp32(genga, ctx):
    d = discs.giants_disc(100_000, 5)
    idx_heavy = np.arange(4)
    got, _ = _gpu_acc(genga, ctx, d, 1)
    rng = np.random.default_rng(1)
    idx = np.concatenate([idx_heavy, np.sort(rng.choice(np.arange(4, d.N), 60, replace=False))])
    ref, _, _ = _oracle_acc(d, idx=idx)
    assert _rel_err(got[:, idx], ref).max() <= TOL[1]
