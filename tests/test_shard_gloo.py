"""Batched sharding across ranks: world_size-2 gloo processes on CPU (no GPU).

Each rank computes its share of the instances on its own; the shares must be disjoint,
cover every instance and balance the N^3 work; the host-side gather of per-instance
results returns them in instance order.  In the factorizing test every rank runs the
CPU oracle's Algorithm 2 on its own small instances and the gathered iteration counts,
histories and factors match a single-process run over the whole batch."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2404_19163_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, sizes, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = shard.mine(sizes, rank, world)
    # stand-in per-instance result computed locally (instance index * 10 + rank id ignored)
    local = {i: i * 10 for i in mine}
    gathered = [None] * world
    dist.all_gather_object(gathered, {"rank": rank, "mine": mine, "res": local})
    if rank == 0:
        q.put(gathered)
    dist.barrier()
    dist.destroy_process_group()


def test_shards_cover_disjoint_balanced():
    g = np.random.default_rng(4)
    sizes = [int(x) for x in g.integers(256, 3073, 128)]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, sizes, q)) for r in range(2)]
    for p in procs:
        p.start()
    gathered = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    shares = [set(x["mine"]) for x in sorted(gathered, key=lambda x: x["rank"])]
    assert shares[0].isdisjoint(shares[1])
    assert shares[0] | shares[1] == set(range(128))
    merged = {}
    for x in gathered:
        merged.update(x["res"])
    assert [merged[i] for i in range(128)] == [i * 10 for i in range(128)]
    assert shard.imbalance(sizes, 2) < 1.02
    assert shard.imbalance(sizes, 8) < 1.1


def test_assign_single_rank_and_errors():
    assert shard.assign([5, 3, 9], 1) == [[2, 0, 1]]
    with pytest.raises(ValueError):
        shard.assign([1], 0)


def _factor_worker(rank, world, port, seeds, sizes, q):
    import oracle
    from paper_2404_19163_gb300 import synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local = {}
    for i in shard.mine(sizes, rank, world):
        S, Q, lam = synth.householder_spd(sizes[i], seed=seeds[i])
        Z, hist, it = oracle.refine(S, None, m=2, nmax=50)
        local[i] = {"iters": it, "hist": [float(h) for h in hist], "Z": Z, "rank": rank}
    res = shard.gather(local, len(sizes))
    if rank == 0:
        q.put(res)
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_factorizations_gather_in_instance_order():
    import oracle
    from paper_2404_19163_gb300 import synth
    g = np.random.default_rng(9)
    count = 11
    sizes = [int(x) for x in g.integers(6, 40, count)]
    seeds = [int(x) for x in g.integers(0, 10_000, count)]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_factor_worker, args=(r, 2, port, seeds, sizes, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert {r["rank"] for r in res} == {0, 1}            # both ranks did work
    for i in range(count):
        S, Q, lam = synth.householder_spd(sizes[i], seed=seeds[i])
        Z, hist, it = oracle.refine(S, None, m=2, nmax=50)
        assert res[i]["iters"] == it and res[i]["hist"] == [float(h) for h in hist]
        assert np.array_equal(res[i]["Z"], Z)
        assert res[i]["Z"].shape == (sizes[i], sizes[i])


def test_gather_rejects_missing_instances():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_gather_bad_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    msgs = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all("missing" in m for m in msgs)


def _gather_bad_worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        shard.gather({rank: rank}, 3)          # instance 2 is on no rank
        q.put("no error")
    except ValueError as e:
        q.put(str(e))
    dist.barrier()
    dist.destroy_process_group()
