"""Host logic of bench.py's multi-rank (replicas) path, on CPU with gloo.

With N ranks every rank solves its own copy of the workload; the bench line
reports the slowest rank's time and the pairs found by all ranks, and the
reference arm runs on rank 0 only.  These checks need no GPU."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = bench.rank_info()
    # rank r took 100 + 10 r ms for 30 + r converged pairs
    t, p = bench.combine_ranks(100.0 + 10 * rank, 30 + rank, world, torch.device("cpu"))
    ref = bench.run_reference(None, r, w) if r != 0 else "rank0"
    dist.barrier()
    dist.destroy_process_group()
    q.put((r, w, lr, t, p, ref))


@pytest.mark.parametrize("world", [2])
def test_replicas_combine(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rr, w, lr, t, p, ref) in enumerate(res):
        assert (rr, w, lr) == (r, world, r)
        assert t == 100.0 + 10 * (world - 1)                      # slowest rank
        assert p == sum(30 + k for k in range(world))              # all ranks' pairs
        assert ref == ("rank0" if r == 0 else None)                 # reference arm: rank 0 only


def test_single_rank_combine():
    sys.path.insert(0, ROOT)
    import torch
    import bench
    assert bench.combine_ranks(12.5, 30, 1, torch.device("cpu")) == (12.5, 30.0)
