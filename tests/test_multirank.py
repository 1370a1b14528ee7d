"""The bench's multi-rank path on CPU: two gloo ranks (world size 2) take
disjoint tiles every step, and the timing reduction gives the maximum time
and the summed work over the ranks."""

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    w, r, _ = bench.dist_init()
    assert (w, r) == (ws, rank)
    mx, sm = bench.reduce_max_sum([1.0 + rank, 10.0 * rank], [100.0 + rank], w)
    bench.barrier(w)
    tiles = [bench.tile_index(i, w, r, 150) for i in range(6)]
    out.put((rank, mx, sm, tiles))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_tiles_and_reduce():
    mp = pytest.importorskip("torch.multiprocessing")
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, mx0, sm0, t0), (r1, mx1, sm1, t1) = res
    assert mx0 == mx1 == [2.0, 10.0] and sm0 == sm1 == [201.0]
    assert not set(t0) & set(t1)  # no tile is solved by both ranks
    assert sorted(t0 + t1) == list(range(12))
