"""The FP64 pass variants (the one-sided pass and the mutual pass, each
unordered pair evaluated once with its terms added to both bodies) against
the oracle, every variant forced in turn.

Tolerance as for every FP64 kick: per-body relative error <= 1e-13 against
the FP64 oracle; the encounter list equal except pairs within 1e-9 of
r_crit,ij.  Sizes span one i-block, several blocks with a partial last one
and the 40,000-body workload; both r_crit modes and changeover forms over
planted close pairs, steps with the close-encounter level, bitwise
determinism, the autotuner's choice and the bounded-wait timeout.
"""
import numpy as np
import pytest

import oracle
from paper_2309_08217_gb300 import discs
from tests.gpu_cases import orbiting_pairs_disc, planted_disc

pytestmark = pytest.mark.gpu

TOL64 = 1e-13


def _variants(g):
    c = g.Context(16)
    n = g.genga_get_fp64_variant(c, 16)[1]
    c.close()
    return list(range(n))


def _params(g, d, mode=1, form=0, **kw):
    return g.make_params(G=d.G, Mstar=d.Mstar, dt=d.dt, n1=3.0, n2=0.4, rcrit_mode=mode, changeover=form,
                         precision=g.GENGA_FP64, **kw)


def _rel(got, ref):
    num = np.sqrt(((got - ref) ** 2).sum(0))
    den = np.sqrt((ref ** 2).sum(0))
    assert np.all(num[den == 0] == 0)
    return num[den > 0] / den[den > 0]


def _oracle(d, mode=1, form=0):
    arr = oracle.disc_arrays(d)
    a, rc = oracle.rcrit(*arr, G=d.G, Mstar=d.Mstar, dt=d.dt, n1=3.0, n2=0.4)
    acc = oracle.kick_acc(arr[0], arr[1], arr[2], arr[6], a, rc, d.G, d.Mstar, 3.0, mode, form)
    pairs, band = oracle.encounters(arr[0], arr[1], arr[2], arr[6], a, rc, 3.0, d.Mstar, mode, band=1e-9)
    return acc, pairs, band


def _kick(g, ctx, d, p):
    import torch
    s = g.DeviceSystem.from_disc(d)
    acc = torch.zeros(3 * max(d.N, 1), dtype=torch.float64, device="cuda")
    g.genga_kick(ctx, s, p, 0.0, acc)
    assert g.genga_get_status(ctx) == g.GENGA_OK
    cap = 4 * d.N + 16
    pairs = torch.zeros(2 * cap, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    g.genga_last_encounters(ctx, pairs, cap, cnt)
    assert g.genga_get_status(ctx) == g.GENGA_OK
    n = int(cnt.item())
    return acc[: 3 * d.N].view(3, d.N).cpu().numpy(), pairs[: 2 * n].view(-1, 2).cpu().numpy()


def _same_pairs(got, ref, band):
    assert np.all(got[:, 0] < got[:, 1])
    gs, rs, bs = (set(map(tuple, a.tolist())) for a in (got, ref, band))
    assert len(gs) == len(got)                      # no pair listed twice
    assert gs - bs == rs - bs


@pytest.fixture(scope="module")
def ctx64(genga):
    c = genga.Context(60_000)
    yield c
    genga.genga_set_fp64_variant(c, -1)
    c.close()


def test_fp64_variant_info(genga):
    vs = _variants(genga)
    assert len(vs) >= 2
    kinds = [genga.genga_fp64_variant_info(v)["kind"] for v in vs]
    assert kinds[0] == 0 and all(k == 1 for k in kinds[1:])
    for v in vs:
        info = genga.genga_fp64_variant_info(v)
        assert info["warps"] >= 1 and info["bodies_per_thread"] >= 1
    with pytest.raises(genga.GengaError):
        genga.genga_fp64_variant_info(len(vs))


@pytest.mark.parametrize("N", [1, 2, 63, 64, 65, 1000, 3001, 7000, 13000])
def test_fp64_variant_sizes(genga, ctx64, N):
    d = planted_disc(N, 900 + N)
    ref, pairs, band = _oracle(d)
    for v in _variants(genga):
        genga.genga_set_fp64_variant(ctx64, v)
        got, gp = _kick(genga, ctx64, d, _params(genga, d))
        if N == 1:
            assert np.all(got == 0)
            continue
        err = _rel(got, ref)
        assert err.max(initial=0.0) <= TOL64, f"variant {v}: max err {err.max(initial=0.0):.3e}"
        _same_pairs(gp, pairs, band)
    genga.genga_set_fp64_variant(ctx64, -1)


@pytest.mark.parametrize("mode,form", [(0, 0), (0, 1), (1, 1)])
def test_fp64_variant_modes(genga, ctx64, mode, form):
    d = planted_disc(9000, 78)
    ref, pairs, band = _oracle(d, mode, form)
    for v in _variants(genga):
        genga.genga_set_fp64_variant(ctx64, v)
        got, gp = _kick(genga, ctx64, d, _params(genga, d, mode, form))
        assert _rel(got, ref).max() <= TOL64, f"variant {v}"
        _same_pairs(gp, pairs, band)
    genga.genga_set_fp64_variant(ctx64, -1)


def test_fp64_variant_disc40k_every_body(genga, ctx64):
    d = discs.workload("disc40k")
    ref, pairs, band = _oracle(d)
    for v in _variants(genga):
        genga.genga_set_fp64_variant(ctx64, v)
        got, gp = _kick(genga, ctx64, d, _params(genga, d))
        err = _rel(got, ref)
        assert err.size == d.N and err.max() <= TOL64, f"variant {v}: {err.max():.3e}"
        _same_pairs(gp, pairs, band)
    genga.genga_set_fp64_variant(ctx64, -1)


def test_fp64_variant_embryos_and_determinism(genga, ctx64):
    d = discs.embryo_disc(25, 12000, seed=32)
    ref, _, _ = _oracle(d)
    for v in _variants(genga):
        genga.genga_set_fp64_variant(ctx64, v)
        a1, p1 = _kick(genga, ctx64, d, _params(genga, d))
        a2, p2 = _kick(genga, ctx64, d, _params(genga, d))
        assert np.array_equal(a1, a2) and np.array_equal(p1, p2), f"variant {v}"
        assert _rel(a1, ref).max() <= TOL64, f"variant {v}"
    genga.genga_set_fp64_variant(ctx64, -1)


def test_fp64_variant_steps_with_close_encounter_level(genga, ctx64):
    """Three FP64 steps with the close-encounter level (encounter pairs and
    predicted entries from the first kick of each step) against the oracle."""
    d = orbiting_pairs_disc(9000, 62)
    ref = oracle.disc_arrays(d)
    assert oracle.step(ref, d.G, d.Mstar, d.dt, 3.0, 0.4, 1, 0, 3, bs_tol=1e-12) == 0
    for v in _variants(genga):
        genga.genga_set_fp64_variant(ctx64, v)
        s = genga.DeviceSystem.from_disc(d)
        genga.genga_step(ctx64, s, _params(genga, d, bs_tol=1e-12), 3)
        assert genga.genga_get_status(ctx64) == genga.GENGA_OK
        got = s.numpy()
        for c in range(6):
            scale = np.sqrt(sum(ref[k] ** 2 for k in ((0, 1, 2) if c < 3 else (3, 4, 5))))
            assert np.max(np.abs(got[c] - ref[c]) / scale) < 1e-10, f"variant {v} component {c}"
    genga.genga_set_fp64_variant(ctx64, -1)


def test_fp64_autotuner_times_every_variant(genga):
    """The first FP64 kick at a size times every variant, keeps the fastest,
    and steps (through the step graphs) with it."""
    d = planted_disc(20000, 5)
    c = genga.Context(d.N)
    p = _params(genga, d)
    ref, _, _ = _oracle(d)
    got, _ = _kick(genga, c, d, p)
    assert _rel(got, ref).max() <= TOL64
    v, n = genga.genga_get_fp64_variant(c, d.N)
    ms = genga.genga_fp64_tuning_times(c, d.N)
    assert len(ms) == n and all(t > 0 for t in ms)
    assert 0 <= v < n and ms[v] == min(ms)
    s = genga.DeviceSystem.from_disc(d)
    genga.genga_step(c, s, p, 8)
    assert genga.genga_get_status(c) == genga.GENGA_OK
    assert np.all(np.isfinite(np.stack(s.numpy())))
    c.close()


def test_fp64_tp2_takes_the_one_sided_pass(genga, ctx64):
    """Test-particle mode 2 is not a mutual pass: a forced mutual FP64
    variant runs the one-sided pass there, with the mode-2 sum."""
    d = planted_disc(5000, 13)
    arr = oracle.disc_arrays(d)
    a, rc = oracle.rcrit(*arr, G=d.G, Mstar=d.Mstar, dt=d.dt, n1=3.0, n2=0.4)
    ref = oracle.kick_acc(arr[0], arr[1], arr[2], arr[6], a, rc, d.G, d.Mstar, 3.0, 1, 0, n_big=7)
    genga.genga_set_fp64_variant(ctx64, 1)
    got, _ = _kick(genga, ctx64, d, _params(genga, d, n_big=7))
    genga.genga_set_fp64_variant(ctx64, -1)
    assert _rel(got, ref).max() <= TOL64


def test_fp64_mutual_bounded_wait_times_out(genga):
    """The mutual FP64 pass's bounded waits: with the producers withholding
    their first stage, the consumers give up after about 1 ms and the status
    reads GENGA_ERR_TIMEOUT; the next kick then runs normally."""
    d = planted_disc(13000, 4)
    ref, _, _ = _oracle(d)
    c = genga.Context(d.N)
    genga.genga_set_fp64_variant(c, 1)
    p = _params(genga, d)
    got, _ = _kick(genga, c, d, p)
    assert _rel(got, ref).max() <= TOL64
    genga.genga_set_test_waits(c, 20, True)
    s = genga.DeviceSystem.from_disc(d)
    genga.genga_kick(c, s, p, 0.0, None)
    assert genga.genga_get_status(c) == genga.GENGA_ERR_TIMEOUT
    genga.genga_set_test_waits(c, 0, False)
    got, _ = _kick(genga, c, d, p)
    assert _rel(got, ref).max() <= TOL64
    c.close()


def test_fp64_mutual_at_100k_sampled(genga):
    """100,000 bodies (the partial rows grow for the mutual plans): each FP64
    variant on 256 sampled bodies against the oracle."""
    import torch
    d = discs.disc_powerlaw(100_000, 8)
    c = genga.Context(d.N)
    p = _params(genga, d)
    rng = np.random.default_rng(4)
    idx = np.sort(rng.choice(d.N, 256, replace=False))
    arr = oracle.disc_arrays(d)
    a, rc = oracle.rcrit(*arr, G=d.G, Mstar=d.Mstar, dt=d.dt, n1=3.0, n2=0.4)
    ref = oracle.kick_acc(arr[0], arr[1], arr[2], arr[6], a, rc, d.G, d.Mstar, 3.0, 1, 0, idx=idx)
    s = genga.DeviceSystem.from_disc(d)
    for v in _variants(genga):
        genga.genga_set_fp64_variant(c, v)
        acc = torch.zeros(3 * d.N, dtype=torch.float64, device="cuda")
        genga.genga_kick(c, s, p, 0.0, acc)
        assert genga.genga_get_status(c) == genga.GENGA_OK
        got = acc.view(3, d.N).cpu().numpy()[:, idx]
        assert _rel(got, ref).max() <= TOL64, f"variant {v}"
    c.close()
