"""Multi-rank host logic on CPU (gloo, world_size 2): box partitioning, the
max-over-ranks timing reduction, and a sharded run of independent boxes --
each rank advances its share of boxes with the FP64 oracle -- that must
equal the single-process run box for box."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1606_02862_gb300 import shard


def test_partition_covers_every_box_once_and_balances():
    rng = np.random.default_rng(0)
    costs = list(rng.uniform(1, 100, 64))
    for nranks in (1, 2, 3, 8):
        parts = shard.partition(costs, nranks)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(64))
        assert len(parts) == nranks
        assert shard.imbalance(costs, parts) < 1.1
    assert shard.partition([5.0], 4)[1:] == [[], [], []]
    with pytest.raises(ValueError):
        shard.partition([1.0], 0)


def test_reductions_without_process_group():
    assert shard.max_over_ranks([1.0, 2.5]) == [1.0, 2.5]
    assert shard.sum_over_ranks([3.0]) == [3.0]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _boxes():
    from paper_1606_02862_gb300 import workloads as W

    rng = np.random.default_rng(5)
    out = []
    for n, ppc in ((8, 2), (12, 1), (8, 3), (4, 4), (8, 1)):
        x = W.uniform_in_cells(rng, n, n, n, ppc)
        u = W.maxwellian(rng, x.shape[0], 0.2)
        out.append((n, x, u, np.full(x.shape[0], 0.01 / ppc)))
    return out


def _run_boxes(idx, steps=3):
    import oracle

    res = {}
    for i in idx:
        n, x, u, w = _boxes()[i]
        sp = oracle.Species(-1.0, 1.0, 2, x, u, w)
        st = oracle.State(n, n, n, 0.5 / np.sqrt(3.0), species=[sp], rho_bg=0.01)
        st.step(steps)
        res[i] = st.diagnostics()
    return res


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        costs = [shard.box_cost(b[0] ** 3, b[1].shape[0]) for b in _boxes()]
        parts = shard.partition(costs, world)
        mine = _run_boxes(parts[rank])
        # timing reduction: rank r reports r + 1
        mx = shard.max_over_ranks([rank + 1.0, -rank], dist)
        tot = shard.sum_over_ranks([sum(v[2] for v in mine.values())], dist)
        gathered = [None] * world
        dist.all_gather_object(gathered, {k: v.tolist() for k, v in mine.items()})
        if rank == 0:
            q.put({"parts": parts, "max": mx, "charge": tot[0], "results": gathered})
    finally:
        dist.destroy_process_group()


def test_sharded_boxes_match_single_process():
    import oracle

    oracle.build()
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out["max"] == [2.0, 0.0]
    merged = {}
    for part in out["results"]:
        for k, v in part.items():
            assert k not in merged
            merged[int(k)] = np.array(v)
    assert sorted(merged) == list(range(len(_boxes())))
    single = _run_boxes(range(len(_boxes())))
    for k, v in single.items():
        assert np.array_equal(merged[k], v)  # same code, same inputs: bitwise
    assert abs(out["charge"] - sum(v[2] for v in single.values())) < 1e-12
