"""Host logic of the multi-GPU path on CPU: two gloo ranks shard a scene by
object, each trains its share (with the oracle standing in for a GPU), and
the result equals training the whole scene in one process; the timing and
unit reductions are max and sum over ranks."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2302_01838_b300 import scenes, sharding


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _states(sc, ids):
    from oracle import vmap_step as vs
    return [vs.ObjectState(H=sc["objects"][k]["H"], pool=sc["objects"][k]["pool"],
                           center=np.asarray(sc["objects"][k]["center"], np.float64),
                           scale=float(sc["objects"][k]["scale"]), n_surface=sc["objects"][k]["n_surface"],
                           n_strat=sc["objects"][k]["n_strat"], stream=k, params=sc["objects"][k]["init"])
            for k in ids]


def _scene():
    sc = scenes.scene_small(seed=5, n_objects=5, rays=24)
    for k, o in enumerate(sc["objects"]):
        o["rays"] = 8 + 8 * k
    return sc


def _train(sc, ids, steps=2):
    from oracle import vmap_step as vs
    cfg = vs.Config(seed=sc["seed"], B=np.asarray(sc["B"], np.float64))
    st = _states(sc, ids)
    for _ in range(steps):
        vs.train_step(cfg, st, [sc["objects"][k]["rays"] for k in ids])
    return {k: s.params.copy() for k, s in zip(ids, st)}


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sc = _scene()
        objs = sc["objects"]
        costs = [sharding.object_cost(o["rays"], o["n_surface"] + o["n_strat"], o["H"]) for o in objs]
        mine = sharding.partition(costs, world)[rank]
        params = _train(sc, mine)
        gathered = [None] * world
        dist.all_gather_object(gathered, params)
        t = sharding.max_over_ranks(1.5 + rank)
        n = sharding.sum_over_ranks(sum(objs[k]["rays"] for k in mine))
        if rank == 0:
            merged = {}
            for g in gathered:
                merged.update(g)
            q.put((merged, t, n))
    finally:
        dist.destroy_process_group()


def test_partition_is_balanced_and_complete():
    costs = [sharding.object_cost(r, 22, h) for r, h in
             [(600, 32), (32, 32), (1200, 128), (100, 64), (50, 16), (400, 32), (64, 32)]]
    for world in (1, 2, 3, 4, 8):
        parts = sharding.partition(costs, world)
        assert sorted(k for p in parts for k in p) == list(range(len(costs)))
        loads = [sum(costs[k] for k in p) for p in parts]
        # greedy largest-first: no rank exceeds the mean load by more than the largest object
        assert max(loads) <= sum(costs) / world + max(costs)
    assert sharding.partition(costs, 2) == sharding.partition(costs, 2)


def test_two_gloo_ranks_equal_one_process():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    merged, t, n = q.get(timeout=240)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sc = _scene()
    whole = _train(sc, list(range(len(sc["objects"]))))
    assert sorted(merged) == sorted(whole)
    for k in whole:
        assert np.array_equal(merged[k], whole[k]), f"object {k} differs when sharded"
    assert t == 2.5
    assert n == sum(o["rays"] for o in sc["objects"])


def test_reductions_without_a_process_group():
    assert not dist.is_initialized()
    assert sharding.max_over_ranks(3.0) == 3.0 and sharding.sum_over_ranks(4) == 4.0
