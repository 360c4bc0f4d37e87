"""Multi-rank bookkeeping of the benchmark on CPU: two gloo ranks (spawned
processes, 127.0.0.1) check that every rank decomposes its own stacks (no
collective on the data path), that the timed region is the slowest rank's
and that the whole-job rate counts every rank's stacks (weak scaling)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    seeds = bench.stack_seeds("fhd_1920x1080", rank, 4)
    gathered = [None] * world
    dist.all_gather_object(gathered, seeds)
    dist.barrier()
    ms = 100.0 * (rank + 1)            # rank 1 is the slow one
    slow = bench.slowest_rank_ms(ms, dist, "cpu")
    out.put((rank, gathered, slow, bench.whole_job_rate(4, 5, world, slow)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, gathered, slow, rate in res:
        a, b = gathered
        assert len(set(a)) == 4 and not set(a) & set(b)      # disjoint stacks per rank
        assert slow == 200.0                                  # the slowest rank's time
        assert rate == pytest.approx(2 * 4 * 5 / 0.2)         # every rank's stacks / slowest time
