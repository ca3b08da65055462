"""bench.py on several ranks (CPU, gloo, world size 2): every rank runs its own
copy of the workload with its own request ids (weak scaling, no data-path
exchange), and the reported time is the maximum over ranks while the work is
summed."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    maxima, sums = bench.reduce_over_ranks([1.0 + rank, 10.0 * (rank + 1)], [100.0 * (rank + 1)])
    ids = [p["request"] for p in bench.problems_for_rank(rank)]
    q.put((rank, maxima, sums, ids, bench.dist_env()))
    dist.destroy_process_group()


def test_two_rank_aggregation_and_sharding():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for rank, maxima, sums, ids, env in out:
        assert maxima == [2.0, 20.0]
        assert sums == [300.0]
        assert env == (rank, 2, rank)
    assert not set(out[0][3]) & set(out[1][3])


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_over_ranks([3.0], [4.0]) == ([3.0], [4.0])
