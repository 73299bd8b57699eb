"""The multi-GPU split of the single-range workload, run through the library:
two gloo ranks, each sieving its own block of bench.py's per-rank split
(rank_block, scaled down to 10^9 integers per rank) with libgbsieve on the one
GPU this test has.  Their kernels never wait on each other (independent
ranges, no exchange on the data path), so sharing one GPU is sound.  The
counts summed over the ranks must equal the oracle's count of the union."""
import os
import socket

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU-only hosts
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

UNITS = 10**9


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import paper_1205_4883_gb300 as gb
    from paper_1205_4883_gb300.workloads import rank_block
    lo, hi = rank_block(rank, UNITS)
    torch.cuda.set_device(0)
    with gb.Sieve(world * UNITS) as sv:
        out = torch.zeros(1, dtype=torch.int64, device="cuda")
        sv.count_dev(lo, hi, out)
        c = torch.tensor([int(out.item())], dtype=torch.int64)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    if rank == 0:
        q.put(int(c.item()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_through_the_library_sum_to_the_oracle():
    import oracle
    import oracle_pool
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    total = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    # the oracle over the union [0, 2 * 10^9), in windows on every host core
    edges = list(range(0, 2 * UNITS, 10**8)) + [2 * UNITS]
    want = sum(oracle_pool.pmap(lambda ab: oracle.count(ab[0], ab[1], 1), list(zip(edges[:-1], edges[1:]))))
    assert total == want
