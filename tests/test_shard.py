"""The problem-level split of a batch over ranks (host logic), checked alone and
with world-size-2 gloo process groups on the CPU: every problem is solved by
exactly one rank, every rank computes the same split, and the busiest rank
carries at most the mean load plus the largest single problem."""

import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2411_00688_gb300.shard import lpt_shards  # noqa: E402


def _costs():
    from synth.configs import BatchConfig
    return [sp["H"] * sp["W"] for sp in BatchConfig().specs()]


def _check(costs, shards):
    flat = sorted(i for s in shards for i in s)
    assert flat == list(range(len(costs)))
    loads = [sum(costs[i] for i in s) for s in shards]
    assert max(loads) <= sum(costs) / len(shards) + max(costs)


def test_lpt_shards_cover_and_balance():
    costs = _costs()
    for world in (1, 2, 3, 4, 8):
        _check(costs, lpt_shards(costs, world))
    assert lpt_shards([5, 1, 1, 1, 1, 1], 2) == [[0], [1, 2, 3, 4, 5]]
    assert lpt_shards([], 3) == [[], [], []]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    from paper_2411_00688_gb300.shard import lpt_shards as split
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = split(_costs(), world)[rank]
        got = [None] * world
        dist.all_gather_object(got, mine)
        out[rank] = got
    finally:
        dist.destroy_process_group()


def test_ranks_agree_on_disjoint_shards_with_two_gloo_ranks():
    world, port = 2, _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    costs = _costs()
    assert out[0] == out[1]
    _check(costs, out[0])
