"""The multi-process path of bench.py (one rank per GPU, each running its
own replica): the job's time is the slowest rank's and its units are the sum
over ranks.  Run here as two gloo ranks on CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms = [100.0, 150.0, 90.0][rank]
        units = [4, 4, 5][rank]
        q.put((rank, bench.combine_ranks(ms, units)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_combine_ranks_over_gloo(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want_ms = max([100.0, 150.0, 90.0][:world])
    want_units = float(sum([4, 4, 5][:world]))
    for r in range(world):
        assert got[r] == (want_ms, want_units), (r, got[r])


def test_combine_ranks_single_process():
    import bench
    assert bench.combine_ranks(12.5, 3) == (12.5, 3.0)
