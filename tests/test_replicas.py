"""Sharding of independent networks over ranks (CPU, gloo, world size 2).

The multi-GPU path has no data-path collective: each rank solves its share of
the networks and the host gathers the results.  These tests run that host
logic as two gloo processes with the FP64 oracle standing in for a rank's
solver, and check that the sharded results equal the single-process ones, that
every network is solved exactly once, and that the timing reduction is a max.
"""
import os
import socket

import numpy as np
import pytest

from paper_1908_03301_gb300 import netgen, replicas


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def small_specs(count=9):
    specs = []
    for i in range(count):
        gen = netgen.rng(7000 + i)
        if i % 3 == 2:
            dims = (int(gen.integers(5, 9)),) * 3
        else:
            s = int(gen.integers(6, 24))
            dims = (s, s + i % 4)
        planes = netgen.lognormal_iid(dims, gen)
        if i % 4 == 1:
            planes = netgen.percolate(planes, 0.75, gen)
        specs.append((dims, planes))
    return specs


def oracle_solve(specs):
    import oracle

    return [oracle.solve(d, p, tol=1e-13).g_eff for d, p in specs]


# ---------------------------------------------------------------- pure host logic
def test_lpt_covers_every_index_once_and_balances():
    gen = np.random.default_rng(3)
    works = list(gen.lognormal(3.0, 1.5, size=97))
    for world in (1, 2, 3, 8):
        parts = replicas.lpt_assign(works, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(works)))
        loads = [sum(works[i] for i in p) for p in parts]
        # LPT bound: no rank exceeds the mean load by more than the largest item
        assert max(loads) <= sum(works) / world + max(works) + 1e-9
        assert replicas.lpt_assign(works, world) == parts  # deterministic


def test_lpt_more_ranks_than_networks():
    parts = replicas.lpt_assign([5.0, 1.0], 4)
    assert sorted(len(p) for p in parts) == [0, 0, 1, 1]
    assert parts[0] == [0]


def test_work_estimate_orders_by_unknowns_times_side():
    assert replicas.work_estimate((64, 64)) == 64 * 64 * 64
    assert replicas.work_estimate((16, 16, 16)) < replicas.work_estimate((128, 128))
    with pytest.raises(ValueError):
        replicas.my_share([(4, 4)], 2, 2)


def test_single_process_run_matches_direct():
    specs = small_specs(5)
    got = replicas.run_sharded(specs, oracle_solve, 0, 1)
    assert got == oracle_solve(specs)


def test_gather_rejects_missing_and_duplicates():
    with pytest.raises(RuntimeError):
        replicas.gather_results({0: 1.0}, 2)


# ---------------------------------------------------------------- two gloo ranks
def _worker(rank, world, port, out_dir):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        specs = small_specs()
        mine = replicas.my_share([d for d, _ in specs], rank, world)
        got = replicas.run_sharded(specs, oracle_solve, rank, world)
        tmax = replicas.max_over_ranks(1.5 + rank)
        np.save(os.path.join(out_dir, f"r{rank}.npy"),
                np.array(got + [tmax, float(len(mine))], dtype=np.float64))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_match_single_process(tmp_path):
    import torch.multiprocessing as mp

    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    specs = small_specs()
    want = oracle_solve(specs)
    counts = []
    for r in range(world):
        a = np.load(tmp_path / f"r{r}.npy")
        got, tmax, nmine = list(a[:-2]), a[-2], int(a[-1])
        # the oracle is deterministic for any thread count: equal bit for bit
        assert got == want
        assert tmax == 2.5
        counts.append(nmine)
    assert sum(counts) == len(specs) and min(counts) >= 1
