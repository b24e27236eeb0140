"""bench.py's multi-rank host logic on CPU: two gloo ranks (one process per
GPU in a real run), replica discs, the max over ranks and the whole-job
(weak-scaling) value; the reference arm's non-zero ranks exit without work."""
import json
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, outdir):
    sys.path.insert(0, ROOT)
    import bench
    from paper_2309_08217_gb300 import discs
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    ms_local = 10.0 + 5.0 * rank                     # rank 1 is the slow one
    ms_max = bench.max_over_ranks(ms_local, dist, torch.device("cpu"))
    d = discs.disc_powerlaw(2000, bench.replica_seed(rank))
    pairs = 2 * d.N * (d.N - 1)
    out = {"rank": rank, "env": list(bench.dist_env()), "ms_max": ms_max,
           "value": bench.weak_value(ws, pairs, 7, ms_max), "pairs": pairs, "x0": float(d.x[0])}
    # the reference arm: ranks other than 0 return at once
    if rank != 0:
        class A:
            cpu_seconds, steps, warmup, gpus = 1.0, 1, 0, ws
        out["reference_rc"] = bench.run_reference(A())
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(outdir, f"rank{rank}.json"), "w") as f:
        json.dump(out, f)


def test_two_gloo_ranks(tmp_path):
    ws = 2
    mp.start_processes(_rank_main, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, start_method="spawn")
    r = [json.load(open(tmp_path / f"rank{k}.json")) for k in range(ws)]
    assert [x["env"] for x in r] == [[2, 0, 0], [2, 1, 1]]
    assert r[0]["ms_max"] == r[1]["ms_max"] == 15.0           # the slowest rank's time
    assert r[0]["value"] == r[1]["value"] == pytest.approx(2 * r[0]["pairs"] * 7 / 15e-3)
    assert r[0]["x0"] != r[1]["x0"]                            # independent replica discs
    assert r[1]["reference_rc"] == 0


def test_single_process_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5                    # no process group: identity
    assert bench.replica_seed(0) == 3                          # rank 0 runs the disc40k workload itself
    assert bench.weak_value(1, 1000, 10, 5.0) == pytest.approx(2e6)
