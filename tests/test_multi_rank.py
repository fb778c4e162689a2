"""Multi-rank host logic on CPU (gloo, world size 2): events are sharded over
ranks without overlap or gaps, and the report-time reduction of the ensemble
sums over ranks equals the sums over all events computed in one process.  A
NaN Casimir drift in one event of one rank reaches every rank's report."""
import math
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2303_05599_gb300 import multi


NAN_EVENT, NAN_SPECIES = 5, 1


def fake_obs(e, n_species=3, with_nan=False):
    rng = np.random.default_rng(100 + e)
    o = {f: rng.uniform(0, 10, size=n_species) for f in multi.SUM_FIELDS + multi.MAX_FIELDS}
    o["n_active"] = rng.integers(1, 1000, size=n_species).astype(float)
    if with_nan and e == NAN_EVENT:
        o["casimir2_dev"][NAN_SPECIES] = math.nan
    return o


def test_local_maxima_propagate_nan():
    obs = [fake_obs(e, with_nan=True) for e in range(7)]
    s, m = multi.local_sums(obs, 3)
    assert math.isnan(m[NAN_SPECIES, 0])
    assert np.isfinite(np.delete(m, NAN_SPECIES, axis=0)).all() and np.isfinite(m[:, 1]).all()
    # the NaN event may come first or last
    s2, m2 = multi.local_sums(obs[::-1], 3)
    assert math.isnan(m2[NAN_SPECIES, 0])


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
    mine_nan = [fake_obs(e, with_nan=True) for e in multi.shard_events(n_events, rank, world)]
    res_nan = multi.ensemble_reduce(mine_nan, 3)
    q.put((rank, (res, res_nan)))
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
                assert abs(results[r][0][k][key] - v) <= 1e-12 * max(1.0, abs(v)), (r, k, key)
    # the NaN event sits on rank 1 only; both ranks report a NaN maximum for
    # that species, and every other value as before
    assert NAN_EVENT in multi.shard_events(n_events, 1, world)
    for r in range(world):
        for k in range(3):
            for key, v in serial[k].items():
                got = results[r][1][k][key]
                if k == NAN_SPECIES and key == "casimir2_dev":
                    assert math.isnan(got), (r, k, key)
                else:
                    assert abs(got - v) <= 1e-12 * max(1.0, abs(v)), (r, k, key)
