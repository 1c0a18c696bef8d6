"""Trajectories split over ranks: each rank's (count, mean, M2), an
all-gather over two gloo ranks (CPU), and tc_merge_moments (host) give the
mean and standard error of the whole set (the Monte Carlo estimate of Section
"Batched Monte Carlo trajectory noise simulation")."""
import os
import socket
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _values():
    rng = np.random.default_rng(44)
    return rng.choice([-1.0, 1.0], size=8192, p=[0.3, 0.7]) + rng.normal(0, 0.01, 8192)


def _rank_main(rank, world, port, q):
    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2205_10091_b300 import native as nt

    x = np.array_split(_values(), world)[rank]
    # this rank's triple (computed here by numpy; on a GPU, tc_shard_moments)
    m = torch.tensor([len(x), x.mean(), ((x - x.mean()) ** 2).sum()], dtype=torch.float64)
    parts = [torch.empty_like(m) for _ in range(world)]
    dist.all_gather(parts, m)
    q.put((rank, nt.merge_moments(torch.stack(parts).numpy())))
    dist.destroy_process_group()


def test_two_gloo_ranks_merge_to_the_whole_set():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    x = _values()
    mean, se = x.mean(), x.std(ddof=1) / np.sqrt(len(x))
    assert res[0] == res[1]  # the same bits on every rank
    assert abs(res[0][0] - mean) <= 1e-14 and abs(res[0][1] - se) <= 1e-15


def test_merge_edge_cases():
    from paper_2205_10091_b300 import native as nt

    x = _values()
    parts = [(len(s), s.mean(), ((s - s.mean()) ** 2).sum()) for s in np.array_split(x, 5)]
    parts.insert(2, (0, 0.0, 0.0))  # an empty shard
    m, se = nt.merge_moments(parts)
    assert abs(m - x.mean()) <= 1e-14 and abs(se - x.std(ddof=1) / np.sqrt(len(x))) <= 1e-15
    assert nt.merge_moments([(1, 0.25, 0.0)]) == (0.25, 0.0)
    for bad in ([(0, 0.0, 0.0)], [(-1, 0.0, 0.0)], [(3, 0.0, -1.0)]):
        try:
            nt.merge_moments(bad)
            raise AssertionError("accepted %r" % (bad,))
        except nt.TcError as e:
            assert e.status == nt.TC_E_INVALID
