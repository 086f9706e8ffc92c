"""The multi-rank path of bench.py on CPU: two gloo ranks (one process each,
rendezvous on 127.0.0.1) read their rank from the environment as torchrun
sets it, take the job's time as the maximum over the ranks, and report the
whole-job throughput of the independent replicas (weak scaling)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        env = bench.dist_env()
        t = bench.max_over_ranks(1.5 + rank, ws, "cpu")   # rank r took 1.5 + r s
        q.put((rank, env, t, bench.job_glups(ws, 524288, 100, t)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, env, t, value in res:
        assert env == (2, rank, rank)
        assert t == 2.5
        assert value == pytest.approx(2 * 524288 * 100 / 2.5 / 1e9)


def test_one_rank_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, 1, "cpu") == 3.25
    assert bench.job_glups(1, 1000, 10, 1e-3) == pytest.approx(1e-2)


def _shard_rank(rank, ws, port, n, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        lo, hi = bench.shard(n, rank, ws)
        total = bench.sum_over_ranks(hi - lo, ws, "cpu")
        shares = [None] * ws
        dist.all_gather_object(shares, (lo, hi))
        q.put((rank, (lo, hi), total, shares))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("ws,n", [(2, 256), (2, 7), (3, 256)])
def test_batch_instances_are_sharded_disjoint_and_covering(ws, n):
    """A batch's instances are independent problems: under torchrun each rank
    advances its own contiguous share of them (no data-path collective), the
    shares are disjoint and together cover every instance, and the job's node
    count is the sum over the ranks."""
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_rank, args=(r, ws, port, n, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    covered = []
    for rank, (lo, hi), total, shares in res:
        assert shares == [r[1] for r in res]  # every rank sees the same split
        assert total == n
        assert hi - lo in (n // ws, n // ws + 1)
        covered.extend(range(lo, hi))
    assert covered == list(range(n))
