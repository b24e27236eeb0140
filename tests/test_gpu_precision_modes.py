"""The FP32 offset forms as precision modes: GENGA_FP32_HILO (hi/lo split,
the one-sided pass), GENGA_FP32_BLOCKREL (block-relative offsets, the mutual
pass) and GENGA_FP32 (the autotuner picks either), each against the FP64
oracle at the FP32 tolerance (per-body relative error <= 2e-5; encounter
list equal outside the 1e-9 band) on all 40,000 bodies of the throughput
disc, plus the combinations the block-relative mode does not take.
"""
import numpy as np
import pytest

import oracle
from paper_2309_08217_gb300 import discs
from tests.gpu_cases import planted_disc

pytestmark = pytest.mark.gpu

TOL32 = 2e-5


def _params(g, d, precision, **kw):
    return g.make_params(G=d.G, Mstar=d.Mstar, dt=d.dt, n1=3.0, n2=0.4, rcrit_mode=1, changeover=0,
                         precision=precision, **kw)


def _rel(got, ref):
    num = np.sqrt(((got - ref) ** 2).sum(0))
    den = np.sqrt((ref ** 2).sum(0))
    return num / den


def _kick(g, ctx, d, p):
    import torch
    s = g.DeviceSystem.from_disc(d)
    acc = torch.zeros(3 * d.N, dtype=torch.float64, device="cuda")
    g.genga_kick(ctx, s, p, 0.0, acc)
    assert g.genga_get_status(ctx) == g.GENGA_OK
    cap = 4 * d.N + 16
    pairs = torch.zeros(2 * cap, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    g.genga_last_encounters(ctx, pairs, cap, cnt)
    n = int(cnt.item())
    return acc.view(3, d.N).cpu().numpy(), pairs[: 2 * n].view(-1, 2).cpu().numpy()


@pytest.fixture(scope="module")
def disc40k_ref():
    d = discs.workload("disc40k")
    arr = oracle.disc_arrays(d)
    a, rc = oracle.rcrit(*arr, G=d.G, Mstar=d.Mstar, dt=d.dt, n1=3.0, n2=0.4)
    acc = oracle.kick_acc(arr[0], arr[1], arr[2], arr[6], a, rc, d.G, d.Mstar, 3.0, 1, 0)
    pairs, band = oracle.encounters(arr[0], arr[1], arr[2], arr[6], a, rc, 3.0, d.Mstar, 1, band=1e-9)
    return d, acc, pairs, band


@pytest.mark.parametrize("mode", ["GENGA_FP32_HILO", "GENGA_FP32_BLOCKREL", "GENGA_FP32"])
def test_fp32_mode_disc40k_every_body(genga, disc40k_ref, mode):
    d, ref, pairs, band = disc40k_ref
    c = genga.Context(d.N)
    got, gp = _kick(genga, c, d, _params(genga, d, getattr(genga, mode)))
    err = _rel(got, ref)
    assert err.size == d.N and err.max() <= TOL32, f"{mode}: {err.max():.3e}"
    gs, rs, bs = (set(map(tuple, a.tolist())) for a in (gp, pairs, band))
    assert gs - bs == rs - bs
    c.close()


def test_modes_run_their_own_pass(genga):
    """HILO times only one-sided variants, BLOCKREL only mutual ones, and a
    forced variant outside a mode's family is not used by that mode."""
    d = planted_disc(20000, 44)
    c = genga.Context(d.N)
    kinds = {v: genga.genga_kernel_variant_info(v)["kind"] for v in range(genga.genga_get_kernel_variant(c, 1)[1])}
    one_sided = [v for v, k in kinds.items() if k == 0]
    mutual = [v for v, k in kinds.items() if k == 1]
    _kick(genga, c, d, _params(genga, d, genga.GENGA_FP32_HILO))
    ms = genga.genga_tuning_times(c, d.N)
    assert all(ms[v] > 0 for v in one_sided) and all(ms[v] == 0 for v in mutual)
    _kick(genga, c, d, _params(genga, d, genga.GENGA_FP32_BLOCKREL))
    ms = genga.genga_tuning_times(c, d.N)
    assert all(ms[v] > 0 for v in mutual)
    # a forced one-sided variant is not taken by the block-relative mode:
    # its result is bitwise that of the mode's own tuned (mutual) variant
    a_blk, _ = _kick(genga, c, d, _params(genga, d, genga.GENGA_FP32_BLOCKREL))
    genga.genga_set_kernel_variant(c, one_sided[0])
    a_forced, _ = _kick(genga, c, d, _params(genga, d, genga.GENGA_FP32_BLOCKREL))
    assert np.array_equal(a_blk, a_forced)
    genga.genga_set_kernel_variant(c, -1)
    c.close()


def test_blockrel_steps(genga):
    """genga_step in the block-relative mode (captured step graphs) against
    the oracle's FP64 steps at the FP32 step tolerance of the parity tests."""
    d = planted_disc(6000, 45)
    ref = oracle.disc_arrays(d)
    assert oracle.step(ref, d.G, d.Mstar, d.dt, 3.0, 0.4, 1, 0, 8) == 0
    c = genga.Context(d.N)
    s = genga.DeviceSystem.from_disc(d)
    genga.genga_step(c, s, _params(genga, d, genga.GENGA_FP32_BLOCKREL), 8)
    assert genga.genga_get_status(c) == genga.GENGA_OK
    got = s.numpy()
    for comp in range(6):
        scale = np.sqrt(sum(ref[k] ** 2 for k in ((0, 1, 2) if comp < 3 else (3, 4, 5))))
        assert np.max(np.abs(got[comp] - ref[comp]) / scale) < 1e-9, f"component {comp}"
    c.close()


def test_blockrel_refuses_tp2(genga):
    d = planted_disc(3000, 46)
    c = genga.Context(2 * d.N)
    s = genga.DeviceSystem.from_disc(d)
    with pytest.raises(genga.GengaError):
        genga.genga_kick(c, s, _params(genga, d, genga.GENGA_FP32_BLOCKREL, n_big=5), 0.0, None)
    off = [0, d.N]
    with pytest.raises(genga.GengaError):
        genga.genga_kick_batched(c, s, off, _params(genga, d, genga.GENGA_FP32_BLOCKREL, n_big=5), 0.0, None)
    c.close()


@pytest.mark.parametrize("mode", ["GENGA_FP32_HILO", "GENGA_FP32_BLOCKREL", "GENGA_FP32"])
def test_modes_in_batched_mode(genga, mode):
    """Each FP32 mode in batched mode (the mutual pass over the systems of a
    batch for BLOCKREL): every system against the oracle run on it alone,
    kick and encounter list with global indices."""
    import torch
    sizes = [7000, 1, 0, 3001, 12000, 64, 2500]
    parts = [planted_disc(n, 300 + k) if n > 0 else None for k, n in enumerate(sizes)]
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    arrays = [np.concatenate([q.arrays()[comp] for q in parts if q is not None]) for comp in range(7)]
    NT = int(offsets[-1])
    c = genga.Context(NT + 8 * 1024)
    s = genga.DeviceSystem.from_arrays(arrays)
    p = _params(genga, parts[0], getattr(genga, mode))
    acc = torch.zeros(3 * NT, dtype=torch.float64, device="cuda")
    genga.genga_kick_batched(c, s, offsets, p, 0.0, acc)
    assert genga.genga_get_status(c) == genga.GENGA_OK
    cap = 4 * NT
    pairs = torch.zeros(2 * cap, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    genga.genga_last_encounters(c, pairs, cap, cnt)
    got_pairs = set(map(tuple, pairs[: 2 * int(cnt.item())].view(-1, 2).cpu().numpy().tolist()))
    got = acc.view(3, NT).cpu().numpy()
    want, band_all = set(), set()
    for k, d in enumerate(parts):
        if d is None or d.N < 2:
            continue
        arr = oracle.disc_arrays(d)
        a, rc = oracle.rcrit(*arr, G=d.G, Mstar=d.Mstar, dt=d.dt, n1=3.0, n2=0.4)
        ref = oracle.kick_acc(arr[0], arr[1], arr[2], arr[6], a, rc, d.G, d.Mstar, 3.0, 1, 0)
        err = _rel(got[:, offsets[k]:offsets[k + 1]], ref)
        assert err.max() <= TOL32, f"{mode} system {k}: {err.max():.3e}"
        pr, band = oracle.encounters(arr[0], arr[1], arr[2], arr[6], a, rc, 3.0, d.Mstar, 1, band=1e-9)
        o = int(offsets[k])
        want |= {(int(i) + o, int(j) + o) for i, j in pr}
        band_all |= {(int(i) + o, int(j) + o) for i, j in band}
    assert got_pairs - band_all == want - band_all
    c.close()
