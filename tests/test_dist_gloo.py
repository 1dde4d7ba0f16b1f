"""The multi-rank path on CPU: two gloo ranks split a batch of independent grids by LPT,
solve their shares, and time with a barrier and the maximum over ranks.

The GPU kernels do not run here; each rank solves its share with the oracle, which is
enough to check the orchestration (the split covers every grid exactly once, every rank
derives the same split without exchanging it, the gathered results equal one process
solving everything, and max_over_ranks / barrier behave).
"""
import json
import os
import socket

import numpy as np
import pytest

from paper_1904_07400_gb300 import dist as pdist

SPECS = [(8, 12, 1), (16, 8, 3), (12, 12, 2), (24, 16, 3), (10, 18, 1), (20, 20, 2), (6, 30, 3)]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _sigma(nx, ny, seed):
    rng = np.random.default_rng(seed)
    return rng.random((nx, ny))


def _solve(nx, ny, k, seed):
    from oracle.convolution import Solver
    s = Solver(nx, ny, k, 1.0 / nx, 1.0 / ny)
    fx, fy = s.forces(_sigma(nx, ny, seed))
    return fx, fy


def _rank_main(rank, world, port, out_path):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        costs = [pdist.solve_cost(nx, ny) for nx, ny, _ in SPECS]
        shards = pdist.shard_lpt(costs, world)
        mine = shards[rank]
        # every rank derived the same split on its own
        seen = [None] * world
        dist.all_gather_object(seen, shards)
        assert all(s == shards for s in seen)
        results = {i: [a.tolist() for a in _solve(*SPECS[i], seed=i)] for i in mine}
        gathered = [None] * world
        dist.all_gather_object(gathered, results)
        pdist.barrier(world)
        tmax = pdist.max_over_ranks(float(10 + rank), world)
        if rank == 0:
            merged = {}
            for g in gathered:
                for i, v in g.items():
                    assert i not in merged
                    merged[i] = v
            with open(out_path, "w") as f:
                json.dump({"tmax": tmax, "merged": {str(i): v for i, v in merged.items()},
                           "shards": shards}, f)
    finally:
        dist.destroy_process_group()


def test_shard_lpt_partition_and_balance():
    rng = np.random.default_rng(0)
    costs = list(rng.random(57) * 10)
    for world in (1, 2, 3, 8):
        shards = pdist.shard_lpt(costs, world)
        flat = sorted(i for s in shards for i in s)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in s) for s in shards]
        # LPT bound: no rank exceeds the mean load by more than the largest single item
        assert max(loads) <= sum(costs) / world + max(costs) + 1e-12
        assert pdist.shard_lpt(costs, world) == shards  # deterministic


def test_solve_cost_orders_the_batched_grids():
    from workloads import synthetic as syn
    specs = syn.batched_specs(256, seed=4)
    costs = [pdist.solve_cost(nx, ny) for nx, ny, _, _ in specs]
    shards = pdist.shard_lpt(costs, 8)
    loads = [sum(costs[i] for i in s) for s in shards]
    assert max(loads) / (sum(costs) / 8) < 1.02  # 256 grids balance to within 2 % on 8 ranks


def test_padded_period_matches_the_library():
    import ctypes
    from paper_1904_07400_gb300 import build, native
    build.build()
    lib = native.load()
    for n in (1, 2, 3, 5, 7, 17, 33, 64, 100, 128, 192, 384, 768, 1000, 4096):
        h = ctypes.c_void_p()
        assert lib.tdg_init(ctypes.byref(h), n, 2, 1, 1.0, 1.0, 1.0, 0, 0) == 0
        px = ctypes.c_int()
        lib.tdg_plan_info(h, ctypes.byref(px), None, None, None)
        assert px.value == pdist.padded_period(n), n
        lib.tdg_destroy(h)


def test_two_gloo_ranks_split_solve_and_time(tmp_path):
    import torch.multiprocessing as mp
    out = tmp_path / "rank0.json"
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(out)), nprocs=world, join=True,
                       start_method="spawn")
    res = json.loads(out.read_text())
    assert res["tmax"] == 11.0
    assert len(res["shards"]) == 2 and all(len(s) > 0 for s in res["shards"])
    merged = res["merged"]
    assert sorted(int(i) for i in merged) == list(range(len(SPECS)))
    for i, spec in enumerate(SPECS):
        fx, fy = _solve(*spec, seed=i)
        assert np.array_equal(np.asarray(merged[str(i)][0]), fx)
        assert np.array_equal(np.asarray(merged[str(i)][1]), fy)
