"""The multi-process path of bench.py on CPU: two gloo ranks, each timing its own replica.

The whole-job figure must take the slowest rank's time and count every rank's work, and
the reference arm must print from rank 0 only."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    # rank r ran its 10 steps in 100 (r + 1) ms; 268 band-applies per step and rank
    ms, value = bench.whole_job(100.0 * (rank + 1), 10, 268, ws, "cpu")
    worst = bench.max_over_ranks(rank + 0.5, ws, "cpu")
    out[rank] = (ms, value, worst)
    dist.barrier()
    dist.destroy_process_group()


def test_whole_job_value_uses_slowest_rank_and_all_units():
    ws = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(ws, _free_port(), out), nprocs=ws, join=True)
        res = dict(out)
    for r in range(ws):
        ms, value, worst = res[r]
        assert ms == pytest.approx(20.0)          # slowest rank: 200 ms / 10 steps
        assert value == pytest.approx(2 * 268 / 0.020)
        assert worst == pytest.approx(1.5)


def test_single_rank_needs_no_process_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job(50.0, 5, 268, 1, "cpu") == pytest.approx((10.0, 26800.0))
