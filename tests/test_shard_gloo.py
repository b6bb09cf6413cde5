"""Multi-rank path on CPU: world_size-2 gloo process groups.

The lattices of a scan are independent, so ranks split them (partition by
volume) and gather the per-lattice results.  The worker here is the CPU
oracle standing in for the GPU library, which these CPU tests cannot run.
"""
import multiprocessing as mp
import os
import socket
import traceback
from datetime import timedelta

import numpy as np
import pytest

from paper_1104_5432_gb300 import shard


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


ITEMS = [dict(Ns=4, Nt=4, beta=2.2, seed=1), dict(Ns=2, Nt=4, beta=2.4, seed=2),
         dict(Ns=4, Nt=2, beta=0.8, seed=3), dict(Ns=6, Nt=2, beta=2.3, seed=4),
         dict(Ns=2, Nt=2, beta=3.0, seed=5)]
VOLS = [it["Ns"] ** 3 * it["Nt"] for it in ITEMS]


def oracle_worker(items):
    from oracle import oracle as O
    out = []
    for it in items:
        links = O.init(it["Ns"], it["Nt"], True, it["seed"])
        links, plaq, _ = O.heatbath(it["Ns"], it["Nt"], links, it["beta"], 2, it["seed"])
        m, a, _ = O.polyakov(it["Ns"], it["Nt"], links)
        out.append(dict(plaquette=float(plaq[-1]), polyakov=m, abs_polyakov=a))
    return out


def failing_worker(items):
    import torch.distributed as dist
    if dist.get_rank() == 1:
        raise ValueError("injected failure on this rank")
    return oracle_worker(items)


def _rank_main(rank, world, port, mode, q):
    import torch.distributed as dist
    try:
        os.environ["MASTER_ADDR"] = "127.0.0.1"
        os.environ["MASTER_PORT"] = str(port)
        dist.init_process_group("gloo", rank=rank, world_size=world,
                                timeout=timedelta(seconds=20))
        if mode == "ok":
            res = shard.sharded_run(ITEMS, VOLS, oracle_worker)
            q.put((rank, "ok", res))
        elif mode == "fail":
            try:
                shard.sharded_run(ITEMS, VOLS, failing_worker)
                q.put((rank, "no-error", None))
            except shard.ShardError as e:
                q.put((rank, "shard-error", str(e)))
        elif mode == "absent":
            if rank == 1:
                q.put((rank, "left", None))
                q.close()
                q.join_thread()  # flush the message before leaving
                os._exit(0)  # leaves between steps, before the gather
            try:
                shard.sharded_run(ITEMS, VOLS, oracle_worker)
                q.put((rank, "no-error", None))
            except Exception as e:
                q.put((rank, "error", type(e).__name__))
        dist.destroy_process_group()
    except Exception:
        q.put((rank, "crash", traceback.format_exc()))


def run_ranks(mode, world=2, timeout=120):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, mode, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(world):
        r, status, payload = q.get(timeout=timeout)
        out[r] = (status, payload)
    for p in procs:
        p.join(timeout=30)
        if p.is_alive():
            p.kill()
    return out


def test_partition_balances_and_covers():
    vols = [100, 10, 50, 50, 40, 5]
    parts = shard.partition(vols, 2)
    assert sorted(sum(parts, [])) == list(range(6))
    loads = [sum(vols[i] for i in p) for p in parts]
    # greedy LPT is within 4/3 of the best possible makespan
    assert max(loads) <= 4 / 3 * max(sum(vols) / 2, max(vols))
    assert parts == [[0, 4], [1, 2, 3, 5]]
    assert shard.partition([3, 3], 4) == [[0], [1], [], []]
    with pytest.raises(ValueError):
        shard.partition([1], 0)


def test_sharded_run_world2_equals_single_process():
    out = run_ranks("ok")
    ref = oracle_worker(ITEMS)
    for r in range(2):
        status, res = out[r]
        assert status == "ok", res
        assert len(res) == len(ITEMS)
        for a, b in zip(res, ref):
            assert a == b


def test_failure_on_one_rank_raises_on_all():
    out = run_ranks("fail")
    for r in range(2):
        status, msg = out[r]
        assert status == "shard-error", (status, msg)
        assert "rank 1" in msg and "injected failure" in msg


def test_rank_that_never_joins_ends_the_others_with_an_error():
    out = run_ranks("absent", timeout=150)
    assert out[1][0] == "left"
    assert out[0][0] == "error", out[0]
