"""genga_kick_noalloc: the FP64 kick for callers that cannot allocate device
memory (their scratch is a fixed array inside the library).

Through the C ABI it must give the oracle's accelerations within the FP64
parity tolerance (1e-13 per body), on two calls in a row -- the second call
finds the scratch holding the first call's contents -- and at the largest
size it accepts, where the last region of the scratch reaches the end of the
fixed array.  This file runs last so that a failure here cannot hide other
results; it also passes alone.
"""
import numpy as np
import pytest

import oracle
from paper_2309_08217_gb300 import discs
from tests.gpu_cases import planted_disc

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-13


def _rel(got, ref):
    num = np.sqrt(((got - ref) ** 2).sum(0))
    den = np.sqrt((ref ** 2).sum(0))
    assert np.all(num[den == 0] == 0)
    return num[den > 0] / den[den > 0]


def _oracle_acc(d, p, idx=None):
    arr = oracle.disc_arrays(d)
    a, rc = oracle.rcrit(*arr, G=d.G, Mstar=d.Mstar, dt=d.dt, n1=p.n1, n2=p.n2)
    return oracle.kick_acc(arr[0], arr[1], arr[2], arr[6], a, rc, d.G, d.Mstar, p.n1, p.rcrit_mode,
                           p.changeover, idx=idx, n_big=p.n_big)


@pytest.mark.parametrize("mode", [0, 1])
def test_noalloc_kick_matches_oracle_twice(genga, mode):
    import torch
    d = planted_disc(3001, 404)
    p = genga.make_params(G=d.G, Mstar=d.Mstar, dt=d.dt, rcrit_mode=mode, precision=genga.GENGA_FP64)
    ref = _oracle_acc(d, p)
    s = genga.DeviceSystem.from_disc(d)
    for call in range(2):
        out = torch.full((3 * d.N,), float("nan"), dtype=torch.float64, device="cuda")
        genga.genga_kick_noalloc(s, p, 0.0, out)
        torch.cuda.synchronize()
        got = out.view(3, d.N).cpu().numpy()
        assert np.all(np.isfinite(got)), f"call {call}"
        assert _rel(got, ref).max() <= TOL_FP64, f"call {call}"


def test_noalloc_kick_at_the_size_limit(genga):
    """N = GENGA_NOALLOC_MAX_N: every scratch region in use up to the end of
    the array; 512 sampled bodies (the first and last ones included) against
    the oracle, on two calls in a row."""
    import torch
    N = genga.GENGA_NOALLOC_MAX_N
    d = discs.disc_uniform(N, 65536)
    p = genga.make_params(G=d.G, Mstar=d.Mstar, dt=d.dt, precision=genga.GENGA_FP64)
    rng = np.random.default_rng(5)
    idx = np.unique(np.concatenate([[0, 1, N - 2, N - 1], rng.choice(N, 508, replace=False)]))
    ref = _oracle_acc(d, p, idx)
    s = genga.DeviceSystem.from_disc(d)
    for call in range(2):
        out = torch.full((3 * N,), float("nan"), dtype=torch.float64, device="cuda")
        genga.genga_kick_noalloc(s, p, 0.0, out)
        torch.cuda.synchronize()
        got = out.view(3, N).cpu().numpy()
        assert np.all(np.isfinite(got)), f"call {call}"
        assert _rel(got[:, idx], ref).max() <= TOL_FP64, f"call {call}"


def test_noalloc_velocity_update_and_limits(genga):
    import torch
    small = planted_disc(500, 9)
    p = genga.make_params(G=small.G, Mstar=small.Mstar, dt=small.dt, precision=genga.GENGA_FP64)
    b = genga.DeviceSystem.from_disc(small)
    genga.genga_kick_noalloc(b, p, 3.0, None)
    torch.cuda.synchronize()
    ref = oracle.disc_arrays(small)
    oracle.kick(ref, small.G, small.Mstar, small.dt, p.n1, p.n2, p.rcrit_mode, p.changeover, 3.0)
    vb = b.numpy()
    for c in (3, 4, 5):
        assert np.allclose(vb[c], ref[c], rtol=1e-14, atol=1e-20)
    # sizes above the fixed maximum and FP32 parameters are rejected
    big = genga.genga_system(genga.GENGA_NOALLOC_MAX_N + 1, *([b.c.x] * 7))
    with pytest.raises(genga.GengaError) as e:
        genga.genga_kick_noalloc(big, p, 0.0, None)
    assert e.value.code == genga.GENGA_ERR_INVALID_ARG
    p32 = genga.make_params(G=small.G, precision=genga.GENGA_FP32)
    with pytest.raises(genga.GengaError):
        genga.genga_kick_noalloc(b, p32, 0.0, None)
