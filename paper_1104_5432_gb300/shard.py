"""Sharding of independent lattices over ranks (one GPU per rank).

A temperature scan or an ensemble (Sec. 2.2) is a set of independent
lattices: the sweeps need no exchange, so each rank advances its own subset
and only the per-lattice results are gathered at the end.  The paper's own
multi-GPU runs split one lattice over the two GPUs of a card with OpenMP
host threads; for independent lattices no halo exchange exists, so none is
built.

  partition(volumes, world)  greedy longest-processing-time split by volume
  sharded_run(items, worker) each rank runs worker(its items) and every
                             rank receives all results in item order; a
                             failure on any rank raises ShardError on all
                             ranks (reported through the gather itself, so
                             nobody waits for a result that never comes)
"""
from __future__ import annotations

from typing import Callable, List, Sequence


class ShardError(RuntimeError):
    pass


def partition(volumes: Sequence[int], world: int) -> List[List[int]]:
    """Indices of the items each rank runs, balancing the summed volume:
    items in decreasing volume (ties by index) go to the least loaded rank
    (ties by rank).  Every rank's list is in increasing index order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0] * world
    parts: List[List[int]] = [[] for _ in range(world)]
    for i in sorted(range(len(volumes)), key=lambda k: (-int(volumes[k]), k)):
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += int(volumes[i])
    return [sorted(p) for p in parts]


def sharded_run(items: Sequence, volumes: Sequence[int], worker: Callable[[List], List],
                group=None) -> List:
    """Run `worker` on this rank's share of `items` and return the results of
    ALL items, in item order, on every rank.

    worker(list_of_items) -> list of per-item results (same order).
    Uses torch.distributed when it is initialised (any backend), else runs
    everything locally."""
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return list(worker(list(items)))
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    parts = partition(volumes, world)
    mine = parts[rank]
    try:
        res = list(worker([items[i] for i in mine]))
        if len(res) != len(mine):
            raise ShardError(f"worker returned {len(res)} results for {len(mine)} items")
        payload = (True, res)
    except Exception as e:  # reported to every rank through the gather
        payload = (False, f"{type(e).__name__}: {e}")
    gathered = [None] * world
    dist.all_gather_object(gathered, payload, group=group)
    failed = [(r, g[1]) for r, g in enumerate(gathered) if not g[0]]
    if failed:
        msg = "; ".join(f"rank {r}: {m}" for r, m in failed)
        raise ShardError(f"sharded run failed on {len(failed)} rank(s): {msg}")
    out = [None] * len(items)
    for r, (_, res) in enumerate(gathered):
        for i, v in zip(parts[r], res):
            out[i] = v
    return out


def gpu_scan_worker(n_therm: int, n_meas: int, rmax: int, dtype: int = 0):
    """Worker for sharded_run: items are dicts with Ns, Nt, beta, seed; the
    rank's lattices form one batch handle, are thermalised, then measured
    after every sweep.  Returns per item (mean plaquette of the measured
    sweeps, <L>, <|L|>, <C(r)> for r = 0..rmax)."""
    def run(items):
        import numpy as np

        from . import su2

        if not items:
            return []
        lat = su2.Lattice([it["Ns"] for it in items], [it["Nt"] for it in items], dtype)
        betas = [it["beta"] for it in items]
        seeds = [it["seed"] for it in items]
        lat.batch_init(su2.HOT, seeds)
        lat.batch_heatbath(betas, n_therm, seeds, plaq=None)
        plaq, ps, cs = lat.batch_heatbath_measure(betas, n_meas, seeds, rmax)
        n = len(items)
        out = [dict(plaquette=float(plaq[l].mean()), polyakov=float(ps[0, l] / n_meas),
                    abs_polyakov=float(ps[1, l] / n_meas),
                    correlator=(cs[l] / n_meas).tolist()) for l in range(n)]
        lat.close()
        return out
    return run
