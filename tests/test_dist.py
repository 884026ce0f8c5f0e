"""The bench's multi-process logic on CPU: two gloo ranks (world_size 2).

Single-source BFS does not shard (replicas only): each rank runs its own
replica of the graph on its own roots, with no collective on the data path.
What is shared is host logic: disjoint root shards, the max over ranks of the
step time, and the gather of per-root rates for the whole-job figure."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    d = bench.Dist("cpu")
    roots = bench.shard_roots(list(range(100, 100 + 2 * 64)), d.rank, d.world, 64)
    rates = [float(rank + 1)] * 3
    allr = d.gather(rates)
    mx = d.max(10.0 * (rank + 1))
    d.barrier()
    q.put((rank, roots, allr, mx, bench.harmonic_mean(allr)))
    d.close()


def test_two_gloo_ranks_share_roots_and_reduce_times():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, r0, all0, mx0, hm0), (_, r1, all1, mx1, hm1) = out
    assert len(r0) == len(r1) == 64 and not set(r0) & set(r1)       # disjoint shards
    assert sorted(all0) == sorted(all1) == [1.0] * 3 + [2.0] * 3      # every rank sees all rates
    assert mx0 == mx1 == 20.0                                         # max over ranks
    assert abs(hm0 - 6 / (3 / 1.0 + 3 / 2.0)) < 1e-12
