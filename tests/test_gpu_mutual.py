"""The mutual FP32 pass (each unordered pair evaluated once, its terms added
to both bodies) against the oracle, every variant forced in turn.

Tolerance as for every FP32 kick: per-body relative error <= 2e-5 against
the FP64 oracle; the encounter list equal except pairs within 1e-9 of
r_crit,ij.  Sizes span one i-block, several blocks with a partial last one,
and the 40,000-body workload; the screened-pair path (planted close pairs,
both r_crit modes and changeover forms), predicted entries (a step with the
close-encounter level), bitwise determinism and the bounded-wait timeout.
"""
import numpy as np
import pytest

import oracle
from paper_2309_08217_gb300 import discs
from tests.gpu_cases import orbiting_pairs_disc, planted_disc

pytestmark = pytest.mark.gpu

TOL32 = 2e-5


def _mutual_variants(g):
    return [v for v in range(_num_variants(g)) if g.genga_kernel_variant_info(v)["kind"] == 1]


def _num_variants(g):
    c = g.Context(16)
    n = g.genga_get_kernel_variant(c, 16)[1]
    c.close()
    return n


def _params(g, d, mode=1, form=0, **kw):
    return g.make_params(G=d.G, Mstar=d.Mstar, dt=d.dt, n1=3.0, n2=0.4, rcrit_mode=mode, changeover=form,
                         precision=g.GENGA_FP32, **kw)


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
def mctx(genga):
    c = genga.Context(60_000)
    yield c
    genga.genga_set_kernel_variant(c, -1)
    c.close()


def test_variant_info(genga):
    kinds = [genga.genga_kernel_variant_info(v)["kind"] for v in range(_num_variants(genga))]
    assert 0 in kinds and 1 in kinds
    for v in range(len(kinds)):
        info = genga.genga_kernel_variant_info(v)
        assert info["warps"] >= 1 and info["bodies_per_thread"] >= 1


@pytest.mark.parametrize("N", [1, 2, 63, 64, 65, 1000, 3001, 7000, 13000])
def test_mutual_sizes(genga, mctx, N):
    d = planted_disc(N, 500 + N)
    ref, pairs, band = _oracle(d)
    for v in _mutual_variants(genga):
        genga.genga_set_kernel_variant(mctx, v)
        got, gp = _kick(genga, mctx, d, _params(genga, d))
        if N == 1:
            assert np.all(got == 0)
            continue
        err = _rel(got, ref)          # bodies with zero acceleration must match exactly
        assert err.max(initial=0.0) <= TOL32, f"variant {v}: max err {err.max(initial=0.0):.3e}"
        _same_pairs(gp, pairs, band)
    genga.genga_set_kernel_variant(mctx, -1)


@pytest.mark.parametrize("mode,form", [(0, 0), (0, 1), (1, 1)])
def test_mutual_modes(genga, mctx, mode, form):
    d = planted_disc(9000, 77)
    ref, pairs, band = _oracle(d, mode, form)
    for v in _mutual_variants(genga):
        genga.genga_set_kernel_variant(mctx, v)
        got, gp = _kick(genga, mctx, d, _params(genga, d, mode, form))
        assert _rel(got, ref).max() <= TOL32, f"variant {v}"
        _same_pairs(gp, pairs, band)
    genga.genga_set_kernel_variant(mctx, -1)


def test_mutual_disc40k_every_body(genga, mctx):
    d = discs.workload("disc40k")
    ref, pairs, band = _oracle(d)
    for v in _mutual_variants(genga):
        genga.genga_set_kernel_variant(mctx, v)
        got, gp = _kick(genga, mctx, d, _params(genga, d))
        err = _rel(got, ref)
        assert err.size == d.N and err.max() <= TOL32, f"variant {v}: {err.max():.3e}"
        _same_pairs(gp, pairs, band)
    genga.genga_set_kernel_variant(mctx, -1)


def test_mutual_embryos_and_determinism(genga, mctx):
    d = discs.embryo_disc(25, 12000, seed=31)
    ref, _, _ = _oracle(d)
    for v in _mutual_variants(genga):
        genga.genga_set_kernel_variant(mctx, v)
        a1, p1 = _kick(genga, mctx, d, _params(genga, d))
        a2, p2 = _kick(genga, mctx, d, _params(genga, d))
        assert np.array_equal(a1, a2) and np.array_equal(p1, p2), f"variant {v}"
        assert _rel(a1, ref).max() <= TOL32, f"variant {v}"
    genga.genga_set_kernel_variant(mctx, -1)


def test_mutual_steps_with_close_encounter_level(genga, mctx):
    """Steps with the close-encounter level: the first kick of a step lists
    the encounter pairs and the predicted entries that form the groups."""
    d = orbiting_pairs_disc(9000, 61)
    ref = oracle.disc_arrays(d)
    assert oracle.step(ref, d.G, d.Mstar, d.dt, 3.0, 0.4, 1, 0, 3, bs_tol=1e-12) == 0
    for v in _mutual_variants(genga):
        genga.genga_set_kernel_variant(mctx, v)
        s = genga.DeviceSystem.from_disc(d)
        genga.genga_step(mctx, s, _params(genga, d, bs_tol=1e-12), 3)
        assert genga.genga_get_status(mctx) == genga.GENGA_OK
        got = s.numpy()
        for c in range(6):
            scale = np.sqrt(sum(ref[k] ** 2 for k in ((0, 1, 2) if c < 3 else (3, 4, 5))))
            assert np.max(np.abs(got[c] - ref[c]) / scale) < 1e-9, f"variant {v} component {c}"
    genga.genga_set_kernel_variant(mctx, -1)


def test_forced_mutual_variant_in_tp2_mode(genga, mctx):
    """Test-particle mode 2 is not a mutual pass: a forced mutual variant
    runs the one-sided pass there, with the mode-2 sum."""
    d = planted_disc(5000, 12)
    arr = oracle.disc_arrays(d)
    a, rc = oracle.rcrit(*arr, G=d.G, Mstar=d.Mstar, dt=d.dt, n1=3.0, n2=0.4)
    ref = oracle.kick_acc(arr[0], arr[1], arr[2], arr[6], a, rc, d.G, d.Mstar, 3.0, 1, 0, n_big=7)
    genga.genga_set_kernel_variant(mctx, _mutual_variants(genga)[0])
    got, _ = _kick(genga, mctx, d, _params(genga, d, n_big=7))
    genga.genga_set_kernel_variant(mctx, -1)
    assert _rel(got, ref).max() <= TOL32


@pytest.mark.parametrize("kind", [0, 1])
def test_bounded_wait_times_out(genga, kind):
    """The failure path of the pipeline's bounded waits: with the test hook's
    producers withholding their first stage (no copy issued), the consumers'
    waits run out after about 1 ms, the kernel returns and the sticky status
    reads GENGA_ERR_TIMEOUT; the context then runs the next kick normally."""
    d = planted_disc(13000, 3)
    ref, _, _ = _oracle(d)
    c = genga.Context(d.N)
    v = [u for u in range(_num_variants(genga)) if genga.genga_kernel_variant_info(u)["kind"] == kind][0]
    genga.genga_set_kernel_variant(c, v)
    p = _params(genga, d)
    got, _ = _kick(genga, c, d, p)                 # fills the partial rows with finite values
    assert _rel(got, ref).max() <= TOL32
    genga.genga_set_test_waits(c, 20, True)        # 2^20 ns ~ 1 ms, producers hold
    s = genga.DeviceSystem.from_disc(d)
    genga.genga_kick(c, s, p, 0.0, None)
    assert genga.genga_get_status(c) == genga.GENGA_ERR_TIMEOUT
    genga.genga_set_test_waits(c, 0, False)
    got, _ = _kick(genga, c, d, p)
    assert _rel(got, ref).max() <= TOL32
    with pytest.raises(genga.GengaError):
        genga.genga_set_test_waits(c, 41, False)
    c.close()


def test_mutual_plan_grows_the_workspace(genga):
    """At 100,000 bodies a mutual plan needs more partial rows than a fresh
    context holds; the context enlarges them (and drops a captured step graph
    that used the old ones).  Each mutual variant, 256 sampled bodies against
    the oracle, then steps with the tuned variant through the step graphs."""
    import torch
    d = discs.disc_powerlaw(100_000, 7)
    c = genga.Context(d.N)
    p = _params(genga, d)
    rng = np.random.default_rng(3)
    idx = np.sort(rng.choice(d.N, 256, replace=False))
    arr = oracle.disc_arrays(d)
    a, rc = oracle.rcrit(*arr, G=d.G, Mstar=d.Mstar, dt=d.dt, n1=3.0, n2=0.4)
    ref = oracle.kick_acc(arr[0], arr[1], arr[2], arr[6], a, rc, d.G, d.Mstar, 3.0, 1, 0, idx=idx)
    s = genga.DeviceSystem.from_disc(d)
    for v in _mutual_variants(genga):
        genga.genga_set_kernel_variant(c, v)
        acc = torch.zeros(3 * d.N, dtype=torch.float64, device="cuda")
        genga.genga_kick(c, s, p, 0.0, acc)
        assert genga.genga_get_status(c) == genga.GENGA_OK
        got = acc.view(3, d.N).cpu().numpy()[:, idx]
        assert _rel(got, ref).max() <= TOL32, f"variant {v}"
    genga.genga_set_kernel_variant(c, -1)
    genga.genga_step(c, s, p, 8)
    assert genga.genga_get_status(c) == genga.GENGA_OK
    assert np.all(np.isfinite(np.stack(s.numpy())))
    c.close()


def test_mutual_200k_sampled(genga):
    """200,000 bodies (longer sums: the per-body error grows with N), each
    mutual variant on 512 sampled bodies against the oracle."""
    import torch
    d = discs.disc_powerlaw(200_000, 9)
    c = genga.Context(d.N)
    p = _params(genga, d)
    rng = np.random.default_rng(5)
    idx = np.sort(rng.choice(d.N, 512, replace=False))
    arr = oracle.disc_arrays(d)
    a, rc = oracle.rcrit(*arr, G=d.G, Mstar=d.Mstar, dt=d.dt, n1=3.0, n2=0.4)
    ref = oracle.kick_acc(arr[0], arr[1], arr[2], arr[6], a, rc, d.G, d.Mstar, 3.0, 1, 0, idx=idx)
    s = genga.DeviceSystem.from_disc(d)
    for v in _mutual_variants(genga):
        genga.genga_set_kernel_variant(c, v)
        acc = torch.zeros(3 * d.N, dtype=torch.float64, device="cuda")
        genga.genga_kick(c, s, p, 0.0, acc)
        assert genga.genga_get_status(c) == genga.GENGA_OK
        got = acc.view(3, d.N).cpu().numpy()[:, idx]
        assert _rel(got, ref).max() <= TOL32, f"variant {v}"
    c.close()
