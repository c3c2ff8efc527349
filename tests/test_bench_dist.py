"""The benchmark's multi-rank logic on CPU: two gloo ranks, weak-scaling seeds,
max-over-ranks timing and the summed ray count."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    import bench
    r, w, lr = bench.dist_env()
    dist = bench.dist_init(w, use_cuda=False)
    bench.barrier(dist)
    mx = bench.max_over_ranks(dist, 10.0 + rank)
    sm = bench.sum_over_ranks(dist, 1000.0 * (rank + 1))
    seed = bench.rank_seed(123, r)
    q.put((r, mx, sm, seed))
    dist.destroy_process_group()


def test_two_rank_reductions_and_seeds():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [11.0, 11.0]
    assert [r[2] for r in res] == [3000.0, 3000.0]
    assert res[0][3] == 123 and res[1][3] != res[0][3]
