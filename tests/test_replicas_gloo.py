"""The N > 1 host logic on the CPU: LPT split of the 64 seeded boxes, and the
max-over-ranks timing / whole-job rate over a world_size-2 gloo group."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import workloads as W
from paper_2110_03044_gb300.replicas import (lpt_partition, max_over_ranks, part_loads,
                                             sum_over_ranks, whole_job_rate)


def test_lpt_covers_every_box_once_within_graham_bound():
    weights = [int(np.prod(d)) for d in W.batched_box_dims()]
    for n in (1, 2, 3, 4, 8):
        parts = lpt_partition(weights, n)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(weights)))
        loads = part_loads(weights, parts)
        # OPT >= max(total / n, largest box); LPT <= 4/3 OPT
        opt_lb = max(sum(weights) / n, max(weights))
        assert max(loads) <= 4 / 3 * opt_lb + 1e-9
        assert sum(loads) == sum(weights)


def test_lpt_small_cases():
    assert lpt_partition([5, 4, 3, 3, 3], 2) in ([[0, 3], [1, 2, 4]], [[0, 2], [1, 3, 4]])
    assert lpt_partition([], 3) == [[], [], []]
    assert lpt_partition([7], 2) == [[0], []]
    with pytest.raises(ValueError):
        lpt_partition([1], 0)


def test_reductions_without_group_are_identity():
    assert max_over_ranks(3.5) == 3.5
    assert sum_over_ranks(2.0) == 2.0


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        weights = [int(np.prod(d)) for d in W.batched_box_dims()]
        mine = lpt_partition(weights, world)[rank]
        units = float(sum(weights[i] for i in mine))
        ms = 10.0 + 5.0 * rank  # the slower rank sets the time
        rate, tmax = whole_job_rate(units, ms)
        q.put((rank, mine, units, rate, tmax))
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_split_and_timing():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    weights = [int(np.prod(d)) for d in W.batched_box_dims()]
    assert sorted(out[0][1] + out[1][1]) == list(range(len(weights)))
    assert not set(out[0][1]) & set(out[1][1])
    total = float(sum(weights))
    for _, _, _, rate, tmax in out:
        assert tmax == 15.0
        assert rate == pytest.approx(total / 15e-3)
