"""Failure paths through the C ABI, made without faulting the GPU.

* A bounded device-side wait that runs out: the sort's look-back is given a
  limit of zero rounds, so every sort tile after the first gives up and
  raises the timeout.  sph_sync reports SPH_ERR_TIMEOUT, no kernel consumes
  the invalid order, and after the default limit is restored the same
  context computes the oracle's right-hand side again.
* The same for the persistent launch: a step without a curve sort whose force
  items may not wait for the screening items reports the timeout, and the
  context then evaluates its current state as the oracle does.
* A checkpoint whose stored particle order points outside the particle range
  is refused on the host with SPH_ERR_BOUNDS before anything is copied; one
  with a repeated entry with SPH_ERR_ARG.
"""
import numpy as np
import pytest
import torch

import oracle
from _parity import TOL_MIXED, field_errors, stream
from paper_2107_07315_gb300 import inputs as I
from paper_2107_07315_gb300 import sph

pytestmark = pytest.mark.gpu
MAT = dict(I.DEFAULT_MATERIAL)


def _ctx(st, eos):
    dev = sph.device_state(st)
    torch.cuda.synchronize()
    ctx = sph.sph_init(dev, eos, MAT, None, sph.SPH_MIXED, None, stream=stream().cuda_stream)
    return ctx, dev


def _rhs(ctx, n):
    rates = sph.alloc_rates(n)
    torch.cuda.synchronize()
    sph.sph_rhs(ctx, rates)
    return rates


def test_sort_wait_timeout_is_reported_and_context_reusable():
    st, eos = I.random_state(3000, seed=61, vel=0.1, stress=0.05)   # 12 sort tiles
    n = len(st["x"])
    ctx, _ = _ctx(st, eos)
    _rhs(ctx, n)
    sph.sph_sync(ctx)
    sph.sph_set_wait_limit(ctx, 0)
    _rhs(ctx, n)
    with pytest.raises(sph.SphError) as e:
        sph.sph_sync(ctx)
    assert e.value.status == 5, e.value
    # the error was cleared by sph_sync; the default limit gives a valid RHS
    sph.sph_set_wait_limit(ctx, -1)
    rates = _rhs(ctx, n)
    sph.sph_sync(ctx)
    g = sph.to_numpy(rates)
    o = oracle.rhs(st, eos, MAT, None, scales=True)
    assert np.array_equal(g["ncount"], o["ncount"])
    errs = field_errors(g, o)
    for k, v in errs.items():
        assert v <= TOL_MIXED[k], (k, v)
    sph.sph_free(ctx)


def test_timeout_rhs_writes_nothing():
    # every kernel that reads the sorted order returns at entry: rates that
    # were poisoned before the timed-out right-hand side stay untouched
    st, eos = I.random_state(2000, seed=62, vel=0.1, stress=0.0, solid_frac=0.0)
    n = len(st["x"])
    ctx, _ = _ctx(st, eos)
    sph.sph_set_wait_limit(ctx, 0)
    rates = sph.alloc_rates(n)
    for v in rates.values():
        v.fill_(-7)
    torch.cuda.synchronize()
    sph.sph_rhs(ctx, rates)
    with pytest.raises(sph.SphError) as e:
        sph.sph_sync(ctx)
    assert e.value.status == 5
    g = sph.to_numpy(rates)
    for k, v in g.items():
        assert np.all(v == -7), k
    sph.sph_free(ctx)


def test_checkpoint_order_outside_range_is_a_bounds_error():
    st, eos, _, _ = I.cube_state(n_side=8)
    n = len(st["x"])
    ctx, dev = _ctx(st, eos)
    sph.sph_step(ctx, 1e-3, 2)
    sph.sph_sync(ctx)
    blob = sph.sph_get_state(ctx)
    before = sph.to_numpy(dev)
    perm = blob[len(blob) - 4 * n:].view(np.int32)
    bad = blob.copy()
    bad[len(bad) - 4 * n:].view(np.int32)[5] = n          # outside [0, n)
    with pytest.raises(sph.SphError) as e:
        sph.sph_set_state(ctx, bad)
    assert e.value.status == 7, e.value
    dup = blob.copy()
    dup[len(dup) - 4 * n:].view(np.int32)[5] = perm[6]      # a repeated entry
    with pytest.raises(sph.SphError) as e:
        sph.sph_set_state(ctx, dup)
    assert e.value.status == 1, e.value
    # nothing was copied, and the context goes on stepping
    after = sph.to_numpy(dev)
    for k in ("x", "vx", "u", "h"):
        assert np.array_equal(before[k], after[k])
    sph.sph_step(ctx, 1e-3, 1)
    sph.sph_sync(ctx)
    sph.sph_free(ctx)


def test_persistent_queue_wait_timeout_is_reported():
    # a step without a curve sort, so the only wait is the force items' wait
    # for the screening items of the persistent launch: with no polls allowed
    # the force items that start before the screening is done give up (the
    # 3000 particles make about 190 items, fewer than the resident blocks, so
    # every item starts at once)
    st, eos = I.random_state(3000, seed=63, vel=0.1, stress=0.05)
    n = len(st["x"])
    dev = sph.device_state(st)
    torch.cuda.synchronize()
    ctx = sph.sph_init(dev, eos, MAT, None, sph.SPH_MIXED, dict(persistent=1, sort_every=1000),
                       stream=stream().cuda_stream)
    assert sph.sph_stats(ctx)[25] > 0
    dt = 0.5 * I.cfl_dt(st, eos)
    sph.sph_step(ctx, dt, 1)
    sph.sph_sync(ctx)
    sph.sph_set_wait_limit(ctx, 0)
    sph.sph_step(ctx, dt, 1)
    with pytest.raises(sph.SphError) as e:
        sph.sph_sync(ctx)
    assert e.value.status == 5, e.value
    # default limit again: the context evaluates the current state correctly
    sph.sph_set_wait_limit(ctx, -1)
    rates = _rhs(ctx, n)
    sph.sph_sync(ctx)
    g = sph.to_numpy(rates)
    cur = sph.to_numpy(dev)
    o = oracle.rhs(cur, eos, MAT, None, scales=True)
    assert np.array_equal(g["ncount"], o["ncount"])
    for k, v in field_errors(g, o).items():
        assert v <= TOL_MIXED[k], (k, v)
    sph.sph_free(ctx)
