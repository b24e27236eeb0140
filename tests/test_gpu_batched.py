"""Batched mode (genga_kick_batched / genga_step_batched) against the oracle.

Independent systems of uneven size are concatenated; each system must get
exactly the kick, encounter list and step it gets alone (FP32 kick tolerance
2e-5 per body against the FP64 oracle; encounter pairs with global indices).
"""
import numpy as np
import pytest

import oracle
from paper_2309_08217_gb300 import discs
from tests.gpu_cases import planted_disc

pytestmark = pytest.mark.gpu

SIZES = [700, 1, 0, 3001, 1500, 64]


def _batch(sizes, seed=60):
    parts = [planted_disc(n, seed + k) if n > 0 else None for k, n in enumerate(sizes)]
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    arrays = []
    for c in range(7):
        arrays.append(np.concatenate([p.arrays()[c] for p in parts if p is not None]))
    return parts, offsets, arrays


def _params(g, d):
    return g.make_params(G=d.G, Mstar=d.Mstar, dt=d.dt, precision=g.GENGA_FP32)


def _rel(got, ref):
    num = np.sqrt(((got - ref) ** 2).sum(0))
    den = np.sqrt((ref ** 2).sum(0))
    assert np.all(num[den == 0] == 0)
    return num[den > 0] / den[den > 0]


@pytest.fixture(scope="module")
def bctx(genga):
    c = genga.Context(40_000)
    yield c
    c.close()


def test_batched_kick_and_encounters(genga, bctx):
    import torch
    parts, offsets, arrays = _batch(SIZES)
    NT = int(offsets[-1])
    s = genga.DeviceSystem.from_arrays(arrays)
    p = _params(genga, parts[0])
    acc = torch.zeros(3 * NT, dtype=torch.float64, device="cuda")
    genga.genga_kick_batched(bctx, s, offsets, p, 0.0, acc)
    cap = 4 * NT
    pairs = torch.zeros(2 * cap, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    genga.genga_last_encounters(bctx, pairs, cap, cnt)
    assert genga.genga_get_status(bctx) == genga.GENGA_OK
    got = acc.view(3, NT).cpu().numpy()
    got_pairs = set(map(tuple, pairs[: 2 * int(cnt.item())].view(-1, 2).cpu().numpy().tolist()))
    want_pairs, band_pairs = set(), set()
    for k, d in enumerate(parts):
        if d is None:
            continue
        lo, hi = int(offsets[k]), int(offsets[k + 1])
        arr = oracle.disc_arrays(d)
        a, rc = oracle.rcrit(*arr, G=d.G, Mstar=d.Mstar, dt=d.dt, n1=3.0, n2=0.4)
        ref = oracle.kick_acc(arr[0], arr[1], arr[2], arr[6], a, rc, d.G, d.Mstar, 3.0, 1, 0)
        if d.N > 1:
            err = _rel(got[:, lo:hi], ref)
            if err.size:
                assert err.max() <= 2e-5, f"system {k}: {err.max():.3e}"
        else:
            assert np.all(got[:, lo:hi] == 0)
        pr, band = oracle.encounters(arr[0], arr[1], arr[2], arr[6], a, rc, 3.0, d.Mstar, 1)
        want_pairs |= {(i + lo, j + lo) for i, j in pr.tolist()}
        band_pairs |= {(i + lo, j + lo) for i, j in band.tolist()}
    assert got_pairs - band_pairs == want_pairs - band_pairs
    assert len(want_pairs) >= 3


def test_batched_step_matches_oracle(genga, bctx):
    parts, offsets, arrays = _batch([900, 2048, 333], seed=90)
    s = genga.DeviceSystem.from_arrays(arrays)
    p = _params(genga, parts[0])
    genga.genga_step_batched(bctx, s, offsets, p, 3)
    assert genga.genga_get_status(bctx) == genga.GENGA_OK
    got = s.numpy()
    for k, d in enumerate(parts):
        lo, hi = int(offsets[k]), int(offsets[k + 1])
        ref = oracle.disc_arrays(d)
        assert oracle.step(ref, d.G, d.Mstar, d.dt, 3.0, 0.4, 1, 0, 3) == 0
        for c in range(6):
            scale = np.abs(ref[c]).max()
            assert np.abs(got[c][lo:hi] - ref[c]).max() <= 1e-9 * scale, f"system {k} component {c}"


def test_batched_equals_single_system_calls(genga, bctx):
    """A batch of one system gives the same accelerations as genga_kick."""
    import torch
    d = planted_disc(2500, 5)
    s1 = genga.DeviceSystem.from_disc(d)
    s2 = genga.DeviceSystem.from_disc(d)
    p = _params(genga, d)
    a1 = torch.zeros(3 * d.N, dtype=torch.float64, device="cuda")
    a2 = torch.zeros(3 * d.N, dtype=torch.float64, device="cuda")
    genga.genga_kick(bctx, s1, p, 0.0, a1)
    genga.genga_kick_batched(bctx, s2, [0, d.N], p, 0.0, a2)
    assert genga.genga_get_status(bctx) == genga.GENGA_OK
    ref = oracle.kick_acc(*[a for a in (d.x, d.y, d.z, d.m)],
                          *oracle.rcrit(*oracle.disc_arrays(d), G=d.G, Mstar=d.Mstar, dt=d.dt), d.G, d.Mstar)
    for a in (a1, a2):
        assert _rel(a.view(3, d.N).cpu().numpy(), ref).max() <= 2e-5


def test_batched_argument_checks(genga, bctx):
    d = planted_disc(100, 1)
    s = genga.DeviceSystem.from_disc(d)
    p = _params(genga, d)
    for bad in ([0, 50], [1, 100], [0, 60, 50, 100]):
        with pytest.raises(genga.GengaError):
            genga.genga_kick_batched(bctx, s, bad, p, 0.0, None)
    p64 = genga.make_params(G=d.G, precision=genga.GENGA_FP64)
    with pytest.raises(genga.GengaError):
        genga.genga_kick_batched(bctx, s, [0, 100], p64, 0.0, None)


def test_batched_variant_is_tuned_per_layout(genga):
    """The first batched kick of a layout times every variant's batched pass
    (one-sided and mutual) and keeps the fastest; a second layout gets its own entry;
    the tuned kick still meets the oracle."""
    import torch
    c = genga.Context(40_000)
    for sizes, seed in (([9000, 1200, 5000, 300], 70), ([2500] * 6, 80)):
        parts, offsets, arrays = _batch(sizes, seed)
        assert genga.genga_batched_tuning(c, offsets)[0] == -1
        NT = int(offsets[-1])
        s = genga.DeviceSystem.from_arrays(arrays)
        acc = torch.zeros(3 * NT, dtype=torch.float64, device="cuda")
        genga.genga_kick_batched(c, s, offsets, _params(genga, parts[0]), 0.0, acc)
        assert genga.genga_get_status(c) == genga.GENGA_OK
        v, ms = genga.genga_batched_tuning(c, offsets)   # GENGA_FP32: one-sided and mutual variants
        assert 0 <= v < len(ms) and all(t > 0 for t in ms)
        assert ms[v] == min(ms)
        got = acc.view(3, NT).cpu().numpy()
        for k, d in enumerate(parts):
            arr = oracle.disc_arrays(d)
            a, rc = oracle.rcrit(*arr, G=d.G, Mstar=d.Mstar, dt=d.dt, n1=3.0, n2=0.4)
            ref = oracle.kick_acc(arr[0], arr[1], arr[2], arr[6], a, rc, d.G, d.Mstar, 3.0, 1, 0)
            assert _rel(got[:, offsets[k]:offsets[k + 1]], ref).max() <= 2e-5
    c.close()
