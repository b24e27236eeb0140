"""Test-particle mode 2 (genga_params.n_big) through the C ABI against the
oracle: bodies n_big.. feel the first n_big bodies but not each other, while
those feel everything.  Same tolerances as the plain kick (FP64 1e-13, FP32
2e-5 per body); encounter lists exact outside the 1e-9 band; n_big = -1 and
n_big >= N must give the plain kick."""
import numpy as np
import pytest

import oracle
from paper_2309_08217_gb300 import discs
from tests.gpu_cases import planted_disc

pytestmark = pytest.mark.gpu

TOL = {0: 1e-13, 1: 2e-5}


def _params(g, d, precision, n_big):
    return g.make_params(G=d.G, Mstar=d.Mstar, dt=d.dt, precision=precision, n_big=n_big)


def _rel(got, ref):
    num = np.sqrt(((got - ref) ** 2).sum(0))
    den = np.sqrt((ref ** 2).sum(0))
    assert np.all(num[den == 0] == 0)
    return num[den > 0] / den[den > 0]


def _oracle(d, n_big):
    arr = oracle.disc_arrays(d)
    a, rc = oracle.rcrit(*arr, G=d.G, Mstar=d.Mstar, dt=d.dt, n1=3.0, n2=0.4)
    acc = oracle.kick_acc(arr[0], arr[1], arr[2], arr[6], a, rc, d.G, d.Mstar, 3.0, 1, 0, n_big=n_big)
    pairs, band = oracle.encounters(arr[0], arr[1], arr[2], arr[6], a, rc, 3.0, d.Mstar, n_big=n_big)
    return acc, pairs, band


def _gpu(g, ctx, d, precision, n_big):
    import torch
    s = g.DeviceSystem.from_disc(d)
    acc = torch.zeros(3 * d.N, dtype=torch.float64, device="cuda")
    g.genga_kick(ctx, s, _params(g, d, precision, n_big), 0.0, acc)
    cap = 8 * d.N
    pairs = torch.zeros(2 * cap, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    g.genga_last_encounters(ctx, pairs, cap, cnt)
    assert g.genga_get_status(ctx) == g.GENGA_OK
    n = int(cnt.item())
    return acc.view(3, d.N).cpu().numpy(), pairs[: 2 * n].view(-1, 2).cpu().numpy()


def _same_pairs(got, ref, band):
    g = set(map(tuple, got.tolist()))
    r = set(map(tuple, ref.tolist()))
    b = set(map(tuple, band.tolist()))
    assert (g ^ r) <= b, f"differ outside the band: {sorted((g ^ r) - b)[:5]}"


@pytest.fixture(scope="module")
def ctx(genga):
    c = genga.Context(20_000)
    yield c
    c.close()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("n_big", [0, 1, 5, 700, 3001, -1])
def test_tp2_kick_and_encounters(genga, ctx, precision, n_big):
    d = planted_disc(3001, 600)
    got, gp = _gpu(genga, ctx, d, precision, n_big)
    ref, rp, band = _oracle(d, n_big)
    if n_big == 0:
        assert np.all(got == 0) and len(gp) == 0
        return
    assert _rel(got, ref).max() <= TOL[precision]
    _same_pairs(gp, rp, band)


def test_tp2_every_fp32_variant(genga, ctx):
    d = planted_disc(2500, 601)
    ref, _, _ = _oracle(d, 37)
    _, nvar = genga.genga_get_kernel_variant(ctx, d.N)
    try:
        for v in range(nvar):
            genga.genga_set_kernel_variant(ctx, v)
            got, _ = _gpu(genga, ctx, d, 1, 37)
            assert _rel(got, ref).max() <= TOL[1], f"variant {v}"
    finally:
        genga.genga_set_kernel_variant(ctx, -1)


def test_tp2_giants_and_planetesimals(genga):
    # the configuration of the paper's giant-planet runs: 4 giants, then
    # planetesimals that feel the giants only (a sample of 40k-body disc)
    d = discs.giants_disc(12_000, 5)
    ctx = genga.Context(d.N)
    try:
        for precision in (0, 1):
            got, gp = _gpu(genga, ctx, d, precision, 4)
            idx = np.concatenate([np.arange(4), np.arange(4, d.N, 97)])
            arr = oracle.disc_arrays(d)
            a, rc = oracle.rcrit(*arr, G=d.G, Mstar=d.Mstar, dt=d.dt, n1=3.0, n2=0.4)
            ref = oracle.kick_acc(arr[0], arr[1], arr[2], arr[6], a, rc, d.G, d.Mstar, 3.0, 1, 0, idx=idx, n_big=4)
            assert _rel(got[:, idx], ref).max() <= TOL[precision]
            assert all(min(p) < 4 for p in map(tuple, gp.tolist()))     # no planetesimal pair
    finally:
        ctx.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_tp2_step_and_energy(genga, ctx, precision):
    d = planted_disc(900, 602)
    s = genga.DeviceSystem.from_disc(d)
    p = _params(genga, d, precision, 60)
    E = genga.genga_energy(ctx, s, p)
    arr = oracle.disc_arrays(d)
    Eo = oracle.energy(arr, d.G, d.Mstar, n_big=60)
    assert abs(E[0] / Eo[0] - 1) < 1e-13
    genga.genga_step(ctx, s, p, 3)
    assert genga.genga_get_status(ctx) == genga.GENGA_OK
    assert oracle.step(arr, d.G, d.Mstar, d.dt, 3.0, 0.4, 1, 0, 3, n_big=60) == 0
    st = np.stack(s.numpy()[:6])
    ref = np.stack(arr[:6])
    ep = (np.abs(st[:3] - ref[:3]).max(0) / np.sqrt((ref[:3] ** 2).sum(0))).max()
    ev = (np.abs(st[3:] - ref[3:]).max(0) / np.sqrt((ref[3:] ** 2).sum(0))).max()
    lim = 1e-12 if precision == 0 else 1e-9
    assert ep < lim and ev < lim


def test_tp2_batched(genga):
    import torch
    sizes = [700, 3001, 1, 1500]
    parts = [planted_disc(n, 610 + k) for k, n in enumerate(sizes)]
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    arrays = [np.concatenate([q.arrays()[c] for q in parts]) for c in range(7)]
    ctx = genga.Context(8192)
    try:
        s = genga.DeviceSystem.from_arrays(arrays)
        NT = int(offsets[-1])
        acc = torch.zeros(3 * NT, dtype=torch.float64, device="cuda")
        genga.genga_kick_batched(ctx, s, offsets, _params(genga, parts[0], 1, 20), 0.0, acc)
        assert genga.genga_get_status(ctx) == genga.GENGA_OK
        got = acc.view(3, NT).cpu().numpy()
        for k, q in enumerate(parts):
            if q.N < 2:
                continue
            ref, _, _ = _oracle(q, 20)          # n_big counts within each system
            lo = int(offsets[k])
            assert _rel(got[:, lo:lo + q.N], ref).max() <= TOL[1]
    finally:
        ctx.close()


def test_tp2_noalloc(genga):
    import torch
    d = planted_disc(2000, 603)
    s = genga.DeviceSystem.from_disc(d)
    acc = torch.zeros(3 * d.N, dtype=torch.float64, device="cuda")
    genga.genga_kick_noalloc(s, _params(genga, d, 0, 11), 0.0, acc)
    torch.cuda.synchronize()
    ref, _, _ = _oracle(d, 11)
    assert _rel(acc.view(3, d.N).cpu().numpy(), ref).max() <= TOL[0]


def test_tp2_invalid_n_big(genga, ctx):
    d = planted_disc(100, 604)
    s = genga.DeviceSystem.from_disc(d)
    with pytest.raises(genga.GengaError):
        genga.genga_kick(ctx, s, _params(genga, d, 1, -2), 0.0, None)
