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


def _star_worker(rank, ws, port, q):
    import torch.distributed as dist

    import oracle
    from paper_2107_07315_gb300 import inputs as I

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        st, _, _, params = I.ensemble_state(nstars=5, seed=11, n_lo=300, n_hi=900, nr=64)
        mine = shard.assign_stars(params["N"], ws)[rank]
        rows = []
        for s_id in mine:
            sel = st["star"] == s_id
            sub = {k: (v[..., sel] if v is not None else None) for k, v in st.items()}
            rows.append(oracle.totals(sub))
        q.put((rank, shard.gather_star_totals(mine, rows, 5)))
    finally:
        dist.destroy_process_group()


def test_two_rank_star_totals_gather_equals_single_process():
    import torch.multiprocessing as mp

    import oracle
    from paper_2107_07315_gb300 import inputs as I

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_star_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=180) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # the single-process result: every star's totals in one place
    st, _, _, _ = I.ensemble_state(nstars=5, seed=11, n_lo=300, n_hi=900, nr=64)
    ref = np.zeros((5, 16))
    for s_id in range(5):
        sel = st["star"] == s_id
        ref[s_id] = oracle.totals({k: (v[..., sel] if v is not None else None) for k, v in st.items()})
    for _, got in res:
        assert np.array_equal(got, ref)
