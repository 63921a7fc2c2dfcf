"""The N > 1 path of bench.py (independent replicas, one per rank): the
whole-job figure is every rank's cells over the slowest rank's time, reduced
with torch.distributed. Two gloo ranks on the CPU."""
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


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        got = bench.aggregate_ranks(total_ms=100.0 + 50.0 * rank, cells=1000 * (rank + 1), ws=ws)
        out[rank] = got
    finally:
        dist.destroy_process_group()


def test_aggregate_two_ranks():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    procs = [ctx.Process(target=_rank, args=(r, ws, port, out)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(ws):
        total_ms, cells, value = out[r]
        assert total_ms == 150.0                     # the slowest rank's time
        assert cells == 3000.0                       # both ranks' cells
        assert value == pytest.approx(3000.0 / 0.150)


def test_aggregate_one_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_ranks(200.0, 500, 1) == (200.0, 500, 2500.0)
