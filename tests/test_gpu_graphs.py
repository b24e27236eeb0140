"""Captured step graphs: genga_step / genga_step_batched replay a CUDA graph of
four steps once the spatial order is fresh.  The graph holds the same kernels
in the same order as the step-by-step path, so the states must agree bit for
bit, across calls, after a parameter change (a new capture) and in batched
mode; the launch counter counts the replayed kernels."""
import numpy as np
import pytest

import oracle
from tests.gpu_cases import planted_disc

pytestmark = pytest.mark.gpu


def _pair(genga, n):
    a, b = genga.Context(n), genga.Context(n)
    genga.genga_set_step_graphs(b, False)
    for c in (a, b):                       # the same FP32 variant on both sides
        genga.genga_set_kernel_variant(c, 0)
    return a, b


def _params(genga, d, precision, dt=None):
    return genga.make_params(G=d.G, Mstar=d.Mstar, dt=d.dt if dt is None else dt, precision=precision)


@pytest.mark.parametrize("precision", [1, 0])
def test_graph_steps_bitwise_equal_step_by_step(genga, precision):
    n = 3001 if precision == 1 else 700
    d = planted_disc(n, 71)
    a, b = _pair(genga, n)
    sa, sb = genga.DeviceSystem.from_disc(d), genga.DeviceSystem.from_disc(d)
    p = _params(genga, d, precision)
    la0, lb0 = genga.genga_launch_count(a), genga.genga_launch_count(b)
    for k in (5, 9, 2):                    # 16 steps over calls of uneven length
        genga.genga_step(a, sa, p, k)
    for _ in range(16):
        genga.genga_step(b, sb, p, 1)
    assert genga.genga_get_status(a) == genga.GENGA_OK and genga.genga_get_status(b) == genga.GENGA_OK
    assert np.array_equal(sa.numpy(), sb.numpy())
    assert genga.genga_launch_count(a) - la0 == genga.genga_launch_count(b) - lb0
    a.close()
    b.close()


def test_graph_recaptured_on_parameter_change(genga):
    d = planted_disc(1500, 72)
    a, b = _pair(genga, 1500)
    sa, sb = genga.DeviceSystem.from_disc(d), genga.DeviceSystem.from_disc(d)
    for dt in (6.0, 3.0):
        p = _params(genga, d, 1, dt)
        genga.genga_step(a, sa, p, 12)
        genga.genga_step(b, sb, p, 12)
    assert np.array_equal(sa.numpy(), sb.numpy())
    # and against the oracle: 24 FP64-drift steps with the FP32 kick
    arr = oracle.disc_arrays(d)
    for dt in (6.0, 3.0):
        assert oracle.step(arr, d.G, d.Mstar, dt, 3.0, 0.4, 1, 0, 12) == 0
    got, ref = np.stack(sa.numpy()[:6]), np.stack(arr[:6])
    ep = (np.abs(got[:3] - ref[:3]).max(0) / np.sqrt((ref[:3] ** 2).sum(0))).max()
    ev = (np.abs(got[3:] - ref[3:]).max(0) / np.sqrt((ref[3:] ** 2).sum(0))).max()
    assert ep < 1e-8 and ev < 1e-8   # FP32-kick errors (<= 2e-5 of a) over 24 steps
    a.close()
    b.close()


def test_graph_batched_bitwise_equal(genga):
    sizes = [700, 3001, 1, 1500]
    parts = [planted_disc(n, 80 + k) for k, n in enumerate(sizes)]
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    arrays = [np.concatenate([q.arrays()[c] for q in parts]) for c in range(7)]
    a, b = _pair(genga, 8192)
    sa, sb = genga.DeviceSystem.from_arrays(arrays), genga.DeviceSystem.from_arrays(arrays)
    p = _params(genga, parts[0], 1)
    genga.genga_step_batched(a, sa, offsets, p, 13)
    for _ in range(13):
        genga.genga_step_batched(b, sb, offsets, p, 1)
    assert genga.genga_get_status(a) == genga.GENGA_OK and genga.genga_get_status(b) == genga.GENGA_OK
    assert np.array_equal(sa.numpy(), sb.numpy())
    a.close()
    b.close()
