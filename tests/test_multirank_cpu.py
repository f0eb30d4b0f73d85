"""Multi-rank host logic of bench.py on the CPU: two gloo ranks (127.0.0.1).

The path shards without any data exchange (replicas of the workload, or
disjoint instance shares); the only collective is the timing reduction: the
step time is the maximum over ranks.
"""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from paper_1807_11830_gb300 import synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local = [10.0 + rank, 3.0 - rank]  # per-rank step times
    agg = bench.max_over_ranks(local, world)
    dist.barrier()
    out[rank] = agg
    dist.destroy_process_group()


def test_timing_is_max_over_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        assert out[0] == out[1] == [11.0, 3.0]


def test_single_rank_identity():
    assert bench.max_over_ranks([1.5, 2.5], 1) == [1.5, 2.5]


@pytest.mark.parametrize("world", [2, 3, 8])
def test_lpt_shards_are_disjoint_complete_and_balanced(world):
    specs = synth.draw_mix(512)
    shares = [bench.shard_instances(specs, world, r) for r in range(world)]
    flat = sorted(i for sh in shares for i in sh)
    assert flat == list(range(len(specs)))
    loads = [sum(bench.instance_cost(specs[i]) for i in sh) for sh in shares]
    biggest = max(bench.instance_cost(sp) for sp in specs)
    assert max(loads) - min(loads) <= biggest  # LPT bound
