"""bench.py's multi-rank plumbing on CPU: two gloo ranks (127.0.0.1).

With N GPUs every rank runs its own chain (replicas, no data-path
collective); the only cross-rank steps are the barrier around the timed
region and the max over ranks of the elapsed time.  Both run here over gloo.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, local = bench.dist_env()
    bench.barrier(w)
    got = bench.max_over_ranks(10.0 * (rank + 1), w)
    # the reference arm: every rank but 0 leaves without work
    class A:
        steps, warmup, gpus = 1, 0, world
    rc = bench.run_reference(A) if rank == 1 else None
    bench.barrier(w)
    dist.destroy_process_group()
    q.put((rank, w, r, got, rc))


def test_two_gloo_ranks_barrier_and_max():
    torch = pytest.importorskip("torch")
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1]
    for rank, w, r, got, rc in res:
        assert w == 2 and r == rank
        assert got == 20.0                       # max over ranks
    assert res[1][4] == 0                        # rank 1's reference arm: no work, exit 0


def test_single_rank_max_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    bench.barrier(1)
