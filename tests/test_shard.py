"""Trials across ranks (host logic, CPU): the sharding covers every trial
once, and the global selection over two gloo ranks equals the selection
over the whole batch (least Phi, ties to the lowest trial index, optional
qualification mask)."""
import os

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1405_6104_gb300.shard import global_selection, shard_trials


def test_shard_covers_every_trial_once():
    for n in (0, 1, 7, 64, 65, 1000):
        for world in (1, 2, 3, 8):
            got = np.concatenate([shard_trials(n, world, r) for r in range(world)])
            assert np.array_equal(got, np.arange(n))
            sizes = [len(shard_trials(n, world, r)) for r in range(world)]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_trials(10, 2, 2)


def test_selection_single_process():
    phi = np.array([3.0, 1.0, 2.0, 1.0])
    assert global_selection(phi, np.arange(4)) == (1, 1.0)
    assert global_selection(phi, np.arange(4), z_ok_local=[True, False, True, False]) == (2, 2.0)
    assert global_selection(phi, np.arange(4), z_ok_local=[False] * 4)[0] == -1


def _worker(rank, world, port, phi_all, ok_all, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        tr = shard_trials(len(phi_all), world, rank)
        res = global_selection(phi_all[tr], tr, z_ok_local=ok_all[tr])
        out[rank] = res
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_global_selection_over_gloo_ranks(world):
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
        procs = [ctx.Process(target=_worker, args=(r, world, port, phi, ok, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        for r in range(world):
            assert tuple(out[r]) == want
