"""World-size-2 gloo tests of the multi-rank host logic (no GPU).

Each rank evaluates its contiguous shard of the scenarios with the FP64
oracle and the ranks combine with shard.allreduce_candidates; the combined
flags and slacks must equal the unsharded evaluation, and the speculative
bisection run by rounds around that exchange (shard.sharded_search, decided
by the library's rrg_bisect_plan / rrg_bisect_decide) must give the
oracle's joint bisection over all scenarios.  The replica path's
bookkeeping (distinct seeds, MAX of the timed region) is checked the same way.
"""
import os
import socket

import numpy as np
import pytest

from paper_2510_08288_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import oracle as O
        from paper_2510_08288_gb300 import inputs
        p = inputs.fc3_params()
        N, H = 37, 120
        x_t = O.equilibrium(p, 100.0)
        d = O.sample_disturbances(5, 2, N, H, inputs.DIST_AMP)
        kap = np.linspace(0.0, 0.3, 13)
        k0, k1 = shard.shard_range(N, world, rank)
        dl = np.ascontiguousarray(d[:, :, k0:k1])
        c = O.cfg(H=H, N=k1 - k0, early_exit=0)
        a, s, _, _ = O.eval_candidates(p, c, x_t, 100.0, 250.0, kap, dl)
        a_all, s_all = shard.allreduce_candidates(a, s)
        t_max = shard.allreduce_max(float(rank) + 0.5)
        # the search by rounds: each round's kappas on this rank's shard, the
        # flags combined over the ranks
        cs = O.cfg(H=H, N=k1 - k0)
        ev = lambda kk: O.eval_candidates(p, cs, x_t, 100.0, 250.0, kk, dl)[:2]
        ks, fs, rounds = shard.sharded_search(ev, 12, 8)
        q.put((rank, a_all.tolist(), s_all.tolist(), t_max, shard.replica_seed(1, rank), (k0, k1),
               (ks, fs, rounds)))
    finally:
        dist.destroy_process_group()


def test_sharded_evaluation_equals_unsharded():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    world, port = 2, _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    from oracle import oracle as O
    from paper_2510_08288_gb300 import inputs
    p = inputs.fc3_params()
    N, H = 37, 120
    d = O.sample_disturbances(5, 2, N, H, inputs.DIST_AMP)
    a, s, _, _ = O.eval_candidates(p, O.cfg(H=H, N=N, early_exit=0), O.equilibrium(p, 100.0), 100.0, 250.0,
                                   np.linspace(0.0, 0.3, 13), d)
    k_o, f_o = O.bisect_joint(p, O.cfg(H=H, N=N), O.equilibrium(p, 100.0), 100.0, 250.0, 12, d)
    for rank, a_all, s_all, t_max, seed, rng, search in res:
        np.testing.assert_array_equal(np.array(a_all, dtype=np.uint8), a)
        np.testing.assert_array_equal(np.array(s_all), s)
        assert t_max == 1.5
        assert search[:2] == (k_o, f_o) and search[2] < 12
    assert res[0][4] != res[1][4]
    assert res[0][5] == (0, 19) and res[1][5] == (19, 37)


@pytest.mark.parametrize("N,world", [(1024, 2), (37, 2), (5, 4), (4, 4)])
def test_shard_ranges_partition(N, world):
    rs = [shard.shard_range(N, world, r) for r in range(world)]
    assert rs[0][0] == 0 and rs[-1][1] == N
    assert all(rs[i][1] == rs[i + 1][0] for i in range(world - 1))
    assert max(b - a for a, b in rs) - min(b - a for a, b in rs) <= 1


def test_shard_range_rejects_bad_ranks():
    with pytest.raises(ValueError):
        shard.shard_range(3, 4, 0)
    with pytest.raises(ValueError):
        shard.shard_range(8, 2, 2)
