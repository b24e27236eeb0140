"""genga_kick_noalloc: the FP64 kick for callers that cannot allocate device
memory (their scratch is a fixed array inside the library).

Through the C ABI it must give the accelerations genga_kick gives, within the
FP64 parity tolerance (1e-13 per body), on two calls in a row -- the second
call finds the scratch holding the first call's contents.  This file runs
last so that a failure here cannot hide other results; it also passes alone.
"""
import numpy as np
import pytest

from tests.gpu_cases import planted_disc

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-13


def _rel(got, ref):
    num = np.sqrt(((got - ref) ** 2).sum(0))
    den = np.sqrt((ref ** 2).sum(0))
    assert np.all(num[den == 0] == 0)
    return num[den > 0] / den[den > 0]


@pytest.mark.parametrize("mode", [0, 1])
def test_noalloc_kick_matches_genga_kick_twice(genga, mode):
    import torch
    d = planted_disc(3001, 404)
    p = genga.make_params(G=d.G, Mstar=d.Mstar, dt=d.dt, rcrit_mode=mode, precision=genga.GENGA_FP64)
    ctx = genga.Context(d.N)
    s = genga.DeviceSystem.from_disc(d)
    ref = torch.zeros(3 * d.N, dtype=torch.float64, device="cuda")
    genga.genga_kick(ctx, s, p, 0.0, ref)
    assert genga.genga_get_status(ctx) == genga.GENGA_OK
    ref = ref.view(3, d.N).cpu().numpy()
    for call in range(2):
        out = torch.full((3 * d.N,), float("nan"), dtype=torch.float64, device="cuda")
        genga.genga_kick_noalloc(s, p, 0.0, out)
        torch.cuda.synchronize()
        got = out.view(3, d.N).cpu().numpy()
        assert np.all(np.isfinite(got)), f"call {call}"
        assert _rel(got, ref).max() <= TOL_FP64, f"call {call}"
    ctx.close()


def test_noalloc_velocity_update_and_limits(genga):
    import torch
    small = planted_disc(500, 9)
    p = genga.make_params(G=small.G, Mstar=small.Mstar, dt=small.dt, precision=genga.GENGA_FP64)
    ctx = genga.Context(small.N)
    a = genga.DeviceSystem.from_disc(small)
    b = genga.DeviceSystem.from_disc(small)
    genga.genga_kick(ctx, a, p, 3.0, None)
    genga.genga_kick_noalloc(b, p, 3.0, None)
    torch.cuda.synchronize()
    va, vb = a.numpy(), b.numpy()
    for c in (3, 4, 5):
        assert np.allclose(vb[c], va[c], rtol=1e-14, atol=1e-20)
    ctx.close()
    # sizes above the fixed maximum and FP32 parameters are rejected
    big = genga.genga_system(genga.GENGA_NOALLOC_MAX_N + 1, *([a.c.x] * 7))
    with pytest.raises(genga.GengaError) as e:
        genga.genga_kick_noalloc(big, p, 0.0, None)
    assert e.value.code == genga.GENGA_ERR_INVALID_ARG
    p32 = genga.make_params(G=small.G, precision=genga.GENGA_FP32)
    with pytest.raises(genga.GengaError):
        genga.genga_kick_noalloc(a, p32, 0.0, None)
