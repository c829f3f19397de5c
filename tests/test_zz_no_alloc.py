"""The allocation-free neighbour entry point against sph_neighbors.

sph_neighbors_noalloc serves callers that cannot call cudaMalloc (plug-ins
whose host application owns the device memory, processes under a fixed
memory budget, loops where allocator calls are not allowed).  It must give
exactly the lists of the context-based sph_neighbors, on two calls in a row
(its scratch array is shared between calls and keeps the last call's
contents).  Collected last so that a stop at the first failure has already
run every other test.
"""
import numpy as np
import pytest

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


def _noalloc_lists(dev, n, cap):
    import torch

    offs = torch.full((n + 1,), -1, dtype=torch.int64, device="cuda")
    idx = torch.full((max(cap, 1),), -1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    sph.sph_neighbors_noalloc(n, dev["x"], dev["y"], dev["z"], dev["h"], offs, idx, cap)
    torch.cuda.synchronize()
    o = offs.cpu().numpy()
    return o, idx.cpu().numpy()[: o[-1]]


def test_noalloc_matches_context_lists_twice():
    # two different particle sets so the second call sees the first call's
    # leftovers in the shared scratch
    cases = [I.random_state(5000, seed=41, vel=0.1, stress=0.0, solid_frac=0.0),
             I.random_state(3111, seed=42, vel=0.1, stress=0.0, solid_frac=0.0)]
    for st, eos in cases:
        dev, offs_ref, idx_ref = _context_lists(st, eos)
        n = len(st["x"])
        for _ in range(2):
            offs, idx = _noalloc_lists(dev, n, int(offs_ref[-1]))
            assert np.array_equal(offs, offs_ref)
            assert np.array_equal(idx, idx_ref)


def test_noalloc_rejects_sizes_beyond_limit():
    import torch

    n = 16385
    z = torch.zeros(n, dtype=torch.float64, device="cuda")
    offs = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    with pytest.raises(sph.SphError) as e:
        sph.sph_neighbors_noalloc(n, z, z, z, z + 1.0, offs, offs, 0)
    assert e.value.status == 1
    assert "16384" in str(e.value)
