"""The multi-GPU form of the single-range workload on CPU: two gloo ranks each
sieve their own block (no exchange on the data path); summing the counts and
taking the max of the step times across ranks reproduces the one-process
answer.  No GPU."""
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


def _worker(rank, world, port, units, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_1205_4883_gb300.workloads import rank_block
    lo, hi = rank_block(rank, units)
    c = torch.tensor([oracle.count(lo, hi, 1)], dtype=torch.int64)
    t = torch.tensor([0.5 + rank], dtype=torch.float64)  # a per-rank step time
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        q.put((int(c.item()), float(t.item())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_blocks_sum_to_the_whole():
    import oracle
    oracle.build()
    units = 3 * 10**6
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, units, q)) for r in range(2)]
    for p in procs:
        p.start()
    total, tmax = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert total == oracle.count(0, 2 * units)
    assert tmax == 1.5


def test_rank_blocks_tile_the_line():
    from paper_1205_4883_gb300.workloads import rank_block
    blocks = [rank_block(r, 10**12) for r in range(8)]
    assert blocks[0] == (0, 10**12)
    assert all(blocks[i][1] == blocks[i + 1][0] for i in range(7))
