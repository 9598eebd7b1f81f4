"""Host-side multi-GPU logic of the benchmark, run as two gloo ranks on the CPU: each rank
owns a disjoint block of slices (weak scaling, no collective on the data path), the step
time is the max over ranks, and the reference arm runs on rank 0 only."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    idx, seeds = bench.shard(rank, 4)
    gathered = [None] * world
    dist.all_gather_object(gathered, (idx, seeds))
    t = bench.reduce_max(10.0 + rank, world)
    ref = bench.run_reference(bench.parse_args(["--impl", "reference"])) if rank != 0 else "skip"
    out[rank] = (gathered, t, ref)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_shard_and_reduce():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn")
        res = dict(out)
    gathered, t0, _ = res[0]
    _, t1, ref1 = res[1]
    all_idx = sorted(i for idx, _ in gathered for i in idx)
    assert all_idx == list(range(8))                       # disjoint, complete
    seeds = [s for _, ss in gathered for s in ss]
    assert len(set(seeds)) == 8
    assert t0 == t1 == 11.0                                # max over ranks
    assert ref1 is None                                    # reference arm: rank 0 only
