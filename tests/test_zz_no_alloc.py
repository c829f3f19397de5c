"""The allocation-free neighbour entry point.

sph_neighbors_noalloc serves callers that cannot call cudaMalloc: plug-ins
whose host application owns the device memory, processes under a fixed
memory budget, loops where allocator calls are not allowed.  It must give
exactly the lists of the context-based sph_neighbors and of the FP64
brute-force oracle, on two calls in a row (its scratch array is shared
between calls and keeps the last call's contents), on the default stream and
on a side stream, and refuse inputs beyond its limits with a clear status.
Collected last so that a stop at the first failure has already run every
other test; it also passes when run alone in a fresh process.
"""
import numpy as np
import pytest

import oracle
from paper_2107_07315_gb300 import inputs as I
from paper_2107_07315_gb300 import sph

pytestmark = pytest.mark.gpu


def _context_lists(st, eos):
    import torch

    dev = sph.device_state(st)
    torch.cuda.synchronize()
    ctx = sph.sph_init(dev, eos, dict(I.DEFAULT_MATERIAL), None, sph.SPH_MIXED)
    rates = sph.alloc_rates(len(st["x"]))
    torch.cuda.synchronize()
    sph.sph_rhs(ctx, rates)
    sph.sph_sync(ctx)
    offs, idx = sph.neighbors(ctx)
    sph.sph_free(ctx)
    return dev, offs, idx


def _noalloc_lists(dev, n, cap, stream=None):
    import torch

    offs = torch.full((n + 1,), -1, dtype=torch.int64, device="cuda")
    idx = torch.full((max(cap, 1),), -1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    sph.sph_neighbors_noalloc(n, dev["x"], dev["y"], dev["z"], dev["h"], offs, idx, cap,
                              stream=stream)
    torch.cuda.synchronize()
    o = offs.cpu().numpy()
    return o, idx.cpu().numpy()[: o[-1]]


def test_noalloc_matches_oracle_and_context_lists_twice():
    # two different particle sets so the second call sees the first call's
    # leftovers in the shared scratch
    cases = [I.random_state(5000, seed=41, vel=0.1, stress=0.0, solid_frac=0.0),
             I.random_state(3111, seed=42, vel=0.1, stress=0.0, solid_frac=0.0)]
    for st, eos in cases:
        o_offs, o_idx = oracle.neighbors(st)
        dev, offs_ref, idx_ref = _context_lists(st, eos)
        assert np.array_equal(offs_ref, o_offs) and np.array_equal(idx_ref, o_idx)
        n = len(st["x"])
        for _ in range(2):
            offs, idx = _noalloc_lists(dev, n, int(o_offs[-1]))
            assert np.array_equal(offs, o_offs)
            assert np.array_equal(idx, o_idx)


def test_noalloc_on_a_side_stream_matches_default_stream():
    import torch

    st, _ = I.random_state(4000, seed=43, vel=0.1, stress=0.0, solid_frac=0.0)
    dev = sph.device_state(st)
    o_offs, o_idx = oracle.neighbors(st)
    n = len(st["x"])
    a = _noalloc_lists(dev, n, int(o_offs[-1]))
    side = torch.cuda.Stream()
    b = _noalloc_lists(dev, n, int(o_offs[-1]), stream=side.cuda_stream)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert np.array_equal(b[0], o_offs) and np.array_equal(b[1], o_idx)


def test_noalloc_rejects_lists_larger_than_cap():
    st, _ = I.random_state(2500, seed=44, vel=0.1, stress=0.0, solid_frac=0.0)
    dev = sph.device_state(st)
    o_offs, _ = oracle.neighbors(st)
    n = len(st["x"])
    with pytest.raises(sph.SphError) as e:
        _noalloc_lists(dev, n, int(o_offs[-1]) - 1)
    assert e.value.status == 4
    # the lists still fit exactly at cap = total
    offs, _ = _noalloc_lists(dev, n, int(o_offs[-1]))
    assert np.array_equal(offs, o_offs)


def test_noalloc_capacity_error_for_dense_cluster():
    # 1200 particles in a ball where every particle has about 1000 neighbours:
    # more than the 128 per particle that the fixed scratch serves
    rng = np.random.default_rng(45)
    n = 1200
    st = I._empty_state(n)
    p = rng.normal(size=(n, 3))
    p *= (rng.random(n) ** (1 / 3) / np.linalg.norm(p, axis=1))[:, None]
    st["x"], st["y"], st["z"] = p[:, 0].copy(), p[:, 1].copy(), p[:, 2].copy()
    st["h"][:] = 0.9
    dev = sph.device_state(st)
    with pytest.raises(sph.SphError) as e:
        _noalloc_lists(dev, n, 4 * n * n)
    assert e.value.status == 4
    assert "128" in str(e.value)
    # a following call with ordinary input is unaffected
    st2, _ = I.random_state(1000, seed=46, vel=0.1, stress=0.0, solid_frac=0.0)
    dev2 = sph.device_state(st2)
    o_offs, o_idx = oracle.neighbors(st2)
    offs, idx = _noalloc_lists(dev2, 1000, int(o_offs[-1]))
    assert np.array_equal(offs, o_offs) and np.array_equal(idx, o_idx)


def test_noalloc_rejects_sizes_beyond_limit():
    import torch

    n = 16385
    z = torch.zeros(n, dtype=torch.float64, device="cuda")
    offs = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    with pytest.raises(sph.SphError) as e:
        sph.sph_neighbors_noalloc(n, z, z, z, z + 1.0, offs, offs, 0)
    assert e.value.status == 1
    assert "16384" in str(e.value)
