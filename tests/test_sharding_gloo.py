"""Sample sharding across ranks, tested as world_size-2 gloo process groups on CPU: the
per-rank statistics merged on the host equal the unsharded ensemble's."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import ensemble_inputs as gen
from oracle import stats
from paper_2608_23786_gb300 import sharding


def test_shard_range_covers_all_samples():
    for M in (1, 7, 64, 65):
        for world in (1, 2, 3, 8):
            ranges = [sharding.shard_range(M, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == M
            for (a, b), (c, d) in zip(ranges, ranges[1:]):
                assert b == c
            sizes = [b - a for a, b in ranges]
            assert max(sizes) - min(sizes) <= 1


def test_merge_mean_var_equals_unsharded():
    u = gen.normal(3, (11, 3, 4, 4, 4))
    mean, var = stats.mean_var(u)
    parts = []
    for lo, hi in ((0, 4), (4, 5), (5, 11)):
        sub = u[lo:hi]
        mu = sub.mean(axis=0)
        m2 = ((sub - mu) ** 2).sum(axis=0)
        parts.append((hi - lo, mu, m2))
    n, mu, v = sharding.merge_mean_var(parts)
    assert n == 11
    np.testing.assert_allclose(mu, mean, rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(v, var, rtol=1e-13)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, M, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    u_all = gen.normal(5, (M, 3, 8, 8, 8))
    lo, hi = sharding.shard_range(M, rank, world)
    mine = u_all[lo:hi]
    mu, var = stats.mean_var(mine) if hi - lo > 1 else (mine.mean(0), np.zeros_like(mine[0]))
    n, gm, gv = sharding.merged_mean_var(hi - lo, mu, var)
    E = sharding.allgather_concat(stats.kinetic_energy(mine))
    R = sharding.allgather_concat(stats.restrict(mine, 4))
    if rank == 0:
        q.put((n, gm, gv, E, R))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("M", [6, 7])
def test_two_rank_gloo_statistics_match_unsharded(M):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, M, q)) for r in range(2)]
    for p in procs:
        p.start()
    n, gm, gv, E, R = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    u_all = gen.normal(5, (M, 3, 8, 8, 8))
    mean, var = stats.mean_var(u_all)
    assert n == M
    np.testing.assert_allclose(gm, mean, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(gv, var, rtol=1e-12)
    np.testing.assert_array_equal(E, stats.kinetic_energy(u_all))
    np.testing.assert_array_equal(R, stats.restrict(u_all, 4))
    # the gathered restrictions give the unsharded W1
    other = gen.normal(9, (M + 2, 3, 8, 8, 8))
    assert stats.w1_one_point(R, stats.restrict(other, 4), Q=4) == stats.w1_one_point(
        stats.restrict(u_all, 4), stats.restrict(other, 4), Q=4)
