"""The multi-GPU path of bench.py on CPU with the gloo backend (world size 2):
every rank takes its own contiguous shard of the sample stream (no data-path
collective) and the step time is the maximum over ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import bench
        first, count = bench.shard(rank, ws, 4096, 512)
        t = bench.max_over_ranks(10.0 + 5.0 * rank)
        # the shards as seen by everyone
        got = [None] * ws
        dist.all_gather_object(got, (first, count))
        q.put((rank, first, count, t, got))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("ws", [2])
def test_shards_and_max_time(ws):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(ws)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    shards = res[0][4]
    # equal per-rank work, contiguous, disjoint, covering the workload
    assert all(c == 2048 for _, c in shards)
    assert shards[0] == (0, 2048) and shards[1] == (2048, 2048)
    # every rank reports the slowest rank's time
    assert all(r[3] == 15.0 for r in res)


def test_single_rank_helpers():
    import bench
    assert bench.shard(0, 1, 4096, 512) == (0, 4096)
    # fewer samples than a batch per rank: every rank still gets one batch,
    # and every shard stays inside the workload's 4096 samples
    assert bench.shard(3, 16, 4096, 512) == (1536, 512)
    assert bench.shard(8, 16, 4096, 512) == (3584, 512)
    assert bench.shard(15, 16, 4096, 512) == (3584, 512)
    for r in range(16):
        first, count = bench.shard(r, 16, 4096, 512)
        assert 0 <= first and first + count <= 4096
    assert bench.max_over_ranks(3.5) == 3.5
