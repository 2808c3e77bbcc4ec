"""The multi-rank path of bench.py on CPU (gloo, world size 2): every rank scores a disjoint
set of parts of the all-against-all (weak scaling, no data-path collective), and the timing
reductions (max over ranks) and work sums are correct."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    n_parts = bench.PARTS_PER_GPU * world
    seq = bench.part_sequence(n_parts, 11 * world)
    mine = seq[rank::world]
    t = bench.max_over_ranks(world, float(rank + 1), "cpu")
    s = bench.sum_over_ranks(world, float(10 * (rank + 1)), "cpu")
    out[rank] = (mine, t, s)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_partition_and_reductions():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    parts = [set(out[r][0]) for r in range(world)]
    assert parts[0].isdisjoint(parts[1])
    assert all(len(p) == 11 for p in parts)
    assert all(out[r][1] == 2.0 for r in range(world))        # max over ranks
    assert all(out[r][2] == 30.0 for r in range(world))       # sum over ranks
