"""Trials across GPUs: the trials of the method are independent until the
final selection (Sec. "Results": the least functional over the trial paths
of an initial condition), so a multi-GPU run gives each rank its own trials
and exchanges one double per trial at the end (no collective on the data
path).

``shard_trials`` assigns global trial indices to ranks (contiguous blocks,
balanced to within one trial); ``shard_by_cost`` balances trials of uneven
cost (atoms x steps) instead; ``global_selection`` gathers (Phi, trial) of
every rank on the host and returns the global argmin, ties going to the
lowest trial index as in ``bias_functional``.  Both run on CPU; the process
group may use gloo or NCCL (CPU tensors then travel through gloo only)."""
from __future__ import annotations

import numpy as np


def shard_trials(n_trials: int, world: int, rank: int) -> np.ndarray:
    """Global trial indices of `rank` out of `world` ranks."""
    if world < 1 or not 0 <= rank < world or n_trials < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(n_trials, world)
    lo = rank * base + min(rank, extra)
    hi = lo + base + (1 if rank < extra else 0)
    return np.arange(lo, hi, dtype=np.int64)


def shard_by_cost(costs, world: int, rank: int) -> np.ndarray:
    """Global trial indices of `rank` when trial k costs costs[k] (e.g. its
    atoms x steps): trials in decreasing cost, ties by index, each to the
    rank with the least cost so far (ties to the lower rank).  Every rank's
    total is within the largest single cost of every other rank's; the
    indices come back ascending.  Deterministic: every rank computes the
    same assignment."""
    c = np.asarray(costs, np.float64)
    if world < 1 or not 0 <= rank < world or c.ndim != 1 or np.any(c < 0):
        raise ValueError("bad shard arguments")
    order = sorted(range(len(c)), key=lambda k: (-c[k], k))
    load = np.zeros(world)
    owner = np.empty(len(c), np.int64)
    for k in order:
        r = int(np.argmin(load))  # the first of equal loads
        owner[k] = r
        load[r] += c[k]
    return np.nonzero(owner == rank)[0].astype(np.int64)


def global_selection(phi_local, trials_local, group=None, z_ok_local=None):
    """(argmin trial, its Phi) over all ranks.  phi_local[k] is the functional
    of global trial trials_local[k]; z_ok_local (optional, bool) marks the
    trials that qualify (e.g. final z below a threshold).  Without a process
    group the local values are the whole batch."""
    phi = np.asarray(phi_local, np.float64)
    tr = np.asarray(trials_local, np.int64)
    ok = np.ones(len(phi), bool) if z_ok_local is None else np.asarray(z_ok_local, bool)
    key = np.where(ok, phi, np.inf)
    if group is not None or _dist_ready():
        import torch
        import torch.distributed as dist
        world = dist.get_world_size(group)
        # NCCL moves device tensors only; gloo host tensors
        dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" else None
        n = torch.tensor([len(key)], dtype=torch.int64, device=dev)
        sizes = [torch.zeros(1, dtype=torch.int64, device=dev) for _ in range(world)]
        dist.all_gather(sizes, n, group=group)
        m = int(max(s.item() for s in sizes))
        pad_k = np.full(m, np.inf)
        pad_t = np.full(m, -1, np.int64)
        pad_k[: len(key)] = key
        pad_t[: len(tr)] = tr
        gk = [torch.zeros(m, dtype=torch.float64, device=dev) for _ in range(world)]
        gt = [torch.zeros(m, dtype=torch.int64, device=dev) for _ in range(world)]
        dist.all_gather(gk, torch.from_numpy(pad_k).to(dev) if dev else torch.from_numpy(pad_k), group=group)
        dist.all_gather(gt, torch.from_numpy(pad_t).to(dev) if dev else torch.from_numpy(pad_t), group=group)
        key = np.concatenate([x.cpu().numpy() for x in gk])
        tr = np.concatenate([x.cpu().numpy() for x in gt])
        valid = tr >= 0
        key, tr = key[valid], tr[valid]
    if len(key) == 0 or not np.isfinite(key).any():
        return -1, np.inf
    best = np.min(key)
    idx = tr[key == best].min()
    return int(idx), float(best)


def _dist_ready() -> bool:
    try:
        import torch.distributed as dist
        return dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1
    except Exception:
        return False
