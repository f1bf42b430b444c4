"""Trials across ranks (host logic, CPU): the sharding covers every trial
once, and the global selection over two gloo ranks equals the selection
over the whole batch (least Phi, ties to the lowest trial index, optional
qualification mask)."""
import os

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1405_6104_gb300.shard import global_selection, shard_by_cost, shard_trials


def test_shard_covers_every_trial_once():
    for n in (0, 1, 7, 64, 65, 1000):
        for world in (1, 2, 3, 8):
            got = np.concatenate([shard_trials(n, world, r) for r in range(world)])
            assert np.array_equal(got, np.arange(n))
            sizes = [len(shard_trials(n, world, r)) for r in range(world)]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_trials(10, 2, 2)


def test_cost_sharding_covers_every_trial_and_balances():
    rng = np.random.default_rng(7)
    for n, world in ((32, 2), (32, 4), (33, 8), (5, 8), (0, 3)):
        # log-uniform atom counts (5k - 60k) x 5000 steps, as the uneven batch
        cost = np.exp(rng.uniform(np.log(5000), np.log(60000), n)).round() * 5000
        parts = [shard_by_cost(cost, world, r) for r in range(world)]
        got = np.sort(np.concatenate(parts))
        assert np.array_equal(got, np.arange(n))
        assert all(np.array_equal(p_, np.sort(p_)) for p_ in parts)
        loads = [cost[p_].sum() for p_ in parts]
        if n:
            assert max(loads) - min(loads) <= cost.max()
            # on these draws also no worse than contiguous blocks of equal count
            blocks = [cost[shard_trials(n, world, r)].sum() for r in range(world)]
            assert max(loads) <= max(blocks) + 1e-9
    with pytest.raises(ValueError):
        shard_by_cost([1.0, -1.0], 2, 0)


def test_selection_single_process():
    phi = np.array([3.0, 1.0, 2.0, 1.0])
    assert global_selection(phi, np.arange(4)) == (1, 1.0)
    assert global_selection(phi, np.arange(4), z_ok_local=[True, False, True, False]) == (2, 2.0)
    assert global_selection(phi, np.arange(4), z_ok_local=[False] * 4)[0] == -1


def _worker(rank, world, port, phi_all, ok_all, out, cost=None):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        tr = shard_trials(len(phi_all), world, rank) if cost is None else shard_by_cost(cost, world, rank)
        res = global_selection(phi_all[tr], tr, z_ok_local=ok_all[tr])
        out[rank] = res
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,uneven", [(2, False), (2, True)])
def test_global_selection_over_gloo_ranks(world, uneven):
    rng = np.random.default_rng(3)
    phi = rng.uniform(0, 10, 37)
    phi[[5, 30]] = phi.min() - 1.0  # a tie across the two ranks: the lower trial wins
    ok = rng.random(37) > 0.2
    ok[[5, 30]] = True
    want = global_selection(phi, np.arange(37), z_ok_local=ok)
    assert want == (5, float(phi[5]))
    port = 29500 + (os.getpid() % 1000)
    ctx = mp.get_context("spawn")
    with ctx.Manager() as man:
        out = man.dict()
        # uneven: trials of the uneven batch's sizes, sharded by atoms x steps
        cost = rng.integers(5000, 60000, 37) * 5000.0 if uneven else None
        procs = [ctx.Process(target=_worker, args=(r, world, port + int(uneven), phi, ok, out, cost))
                 for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        for r in range(world):
            assert tuple(out[r]) == want
