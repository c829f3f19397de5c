"""World-size-2 gloo tests of the multi-rank host path (CPU only)."""
import os
import socket

import numpy as np
import pytest

from paper_2107_07315_gb300 import shard


def test_assign_stars_lpt_complete_and_balanced():
    rng = np.random.default_rng(2107)
    counts = np.round(np.exp(rng.uniform(np.log(1e4), np.log(2e5), size=64))).astype(int)
    for ws in (1, 2, 4, 8):
        parts = shard.assign_stars(counts, ws)
        flat = sorted(s for p in parts for s in p)
        assert flat == list(range(64))
        loads = [counts[p].sum() for p in parts]
        assert max(loads) - min(loads) <= counts.max()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        counts = [50, 40, 30, 20, 10]
        mine = shard.assign_stars(counts, ws)[rank]
        pairs = float(sum(counts[s] for s in mine)) * 60.0
        t_ms = 10.0 + rank
        t, p = shard.reduce_timing(t_ms, pairs)
        q.put((rank, mine, t, p))
    finally:
        dist.destroy_process_group()


def test_two_rank_timing_reduction_gloo():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    stars = sorted(s for _, m, _, _ in res for s in m)
    assert stars == [0, 1, 2, 3, 4]
    for _, _, t, p in res:
        assert t == 11.0
        assert p == 150.0 * 60.0
