"""Multi-rank host logic on CPU (gloo, world size 2): events are sharded over
ranks without overlap or gaps, and the report-time reduction of the ensemble
sums over ranks equals the sums over all events computed in one process."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2303_05599_gb300 import multi


def fake_obs(e, n_species=3):
    rng = np.random.default_rng(100 + e)
    o = {f: rng.uniform(0, 10, size=n_species) for f in multi.SUM_FIELDS + multi.MAX_FIELDS}
    o["n_active"] = rng.integers(1, 1000, size=n_species).astype(float)
    return o


def test_sharding_covers_every_event_once():
    for n in (1, 5, 64, 65):
        for world in (1, 2, 3, 8):
            got = sorted(sum((multi.shard_events(n, r, world) for r in range(world)), []))
            assert got == list(range(n))
            sizes = [len(multi.shard_events(n, r, world)) for r in range(world)]
            assert max(sizes) - min(sizes) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, n_events, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = [fake_obs(e) for e in multi.shard_events(n_events, rank, world)]
    res = multi.ensemble_reduce(mine, 3)
    q.put((rank, res))
    dist.barrier()
    dist.destroy_process_group()


def test_ensemble_reduce_over_two_gloo_ranks():
    n_events, world = 7, 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n_events, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    serial = multi.ensemble_reduce([fake_obs(e) for e in range(n_events)], 3)
    for r in range(world):
        for k in range(3):
            for key, v in serial[k].items():
                assert abs(results[r][k][key] - v) <= 1e-12 * max(1.0, abs(v)), (r, k, key)
