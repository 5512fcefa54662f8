"""Multi-GPU split of the batched workload (paper_1709_00302_gb300.shard), on the CPU.

The batched reductions are independent, so N ranks split the matrices and exchange no
data; the benchmark reduces only the step time (max over ranks) and the device status
words (sum).  These tests pin the partition (disjoint, complete, balanced, deterministic,
within LPT's 4/3 bound of the brute-force optimum on tiny inputs) and run the host side of
a two-rank job over gloo on 127.0.0.1.
"""
import itertools
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

import workloads
from paper_1709_00302_gb300 import shard


def test_flop_counts_are_the_papers():
    assert shard.sy2sb_flops(3) == pytest.approx(36.0)                 # 4 n^3 / 3
    assert shard.ge2gb_flops(6, 3) == pytest.approx(4 * (54 - 9))      # 4 (m n^2 - n^3 / 3)
    assert shard.ge2gb_flops(8, 8) == pytest.approx(8 * 8 ** 3 / 3)    # square: 8 n^3 / 3


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_lpt_partition_is_disjoint_complete_and_balanced(world):
    rng = np.random.default_rng(world)
    costs = list(rng.uniform(1.0, 100.0, size=257))
    parts, loads = shard.shard_lpt(costs, world)
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(costs)))
    assert all(p == sorted(p) for p in parts)
    for p, l in zip(parts, loads):
        assert l == pytest.approx(sum(costs[i] for i in p))
    assert max(loads) - min(loads) <= max(costs) + 1e-9
    assert shard.shard_lpt(costs, world) == (parts, loads)  # deterministic


def _best_makespan(costs, world):
    best = float("inf")
    for assign in itertools.product(range(world), repeat=len(costs)):
        loads = [0.0] * world
        for c, r in zip(costs, assign):
            loads[r] += c
        best = min(best, max(loads))
    return best


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("world", [2, 3])
def test_lpt_is_within_four_thirds_of_the_optimum(seed, world):
    costs = list(np.random.default_rng(seed).integers(1, 20, size=7).astype(float))
    _, loads = shard.shard_lpt(costs, world)
    assert max(loads) <= (4.0 / 3.0 - 1.0 / (3 * world)) * _best_makespan(costs, world) + 1e-9


def test_lpt_rejects_a_bad_world_and_handles_fewer_items_than_ranks():
    with pytest.raises(ValueError):
        shard.shard_lpt([1.0], 0)
    parts, loads = shard.shard_lpt([5.0, 1.0], 4)
    assert parts == [[0], [1], [], []] and loads == [5.0, 1.0, 0.0, 0.0]


def test_one_rank_keeps_the_whole_batch_in_order():
    sym, gen = workloads.batched_mix(50, 40, seed=3)
    si, gi = shard.batched_shard(sym, gen, 1, 0)
    assert si == list(range(50)) and gi == list(range(40))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        sym, gen = workloads.batched_mix(world * 1000, world * 1000, seed=0)
        si, gi = shard.batched_shard(sym, gen, world, rank)
        load = sum(shard.sy2sb_flops(sym[i][0]) for i in si) + sum(shard.ge2gb_flops(*gen[i][:2]) for i in gi)
        # the benchmark's host reductions: step time (here proportional to the load) and
        # the sum of the device status words (0 on every rank)
        t = torch.tensor([load * 1e-12], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        bad = torch.zeros(1, dtype=torch.float64)
        dist.all_reduce(bad, op=dist.ReduceOp.SUM)
        shares = [None] * world
        dist.all_gather_object(shares, (si, gi, load))
        if rank == 0:
            out.put((shares, float(t.item()), float(bad.item()), len(sym), len(gen)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_split_the_batch_over_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    env_keep = os.environ.get("MASTER_ADDR")
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    try:
        procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        shares, tmax, bad, ns, ng = out.get(timeout=120)
        for p in procs:
            p.join(timeout=60)
            assert p.exitcode == 0
    finally:
        if env_keep is None:
            os.environ.pop("MASTER_ADDR", None)
        else:
            os.environ["MASTER_ADDR"] = env_keep
    sym_sets = [set(s[0]) for s in shares]
    gen_sets = [set(s[1]) for s in shares]
    assert not (sym_sets[0] & sym_sets[1]) and not (gen_sets[0] & gen_sets[1])
    assert sym_sets[0] | sym_sets[1] == set(range(ns)) and gen_sets[0] | gen_sets[1] == set(range(ng))
    loads = [s[2] for s in shares]
    assert tmax == pytest.approx(max(loads) * 1e-12)
    assert bad == 0.0
    # both ranks hold about half the work and both kinds of matrix
    assert max(loads) / min(loads) < 1.001
    assert all(len(s[0]) > 0 and len(s[1]) > 0 for s in shares)
