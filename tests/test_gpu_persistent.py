"""Persistent right-hand side (mixed precision): the exact screening, density,
equation of state and force pass of all particles of one star, or of a batch
of stars in one index space, as one launch over a global work queue of
particle blocks (screening items first, force items after them).

It runs the same block code, in the same order of sums, as the separate
launches, so the rates are the same bit for bit; against the oracle it holds
the mixed-precision tolerances, on a six-star batch too."""
import numpy as np
import pytest
import torch

import oracle
from _parity import TOL_MIXED, assert_close, assert_same_neighbors, gpu_rhs, stream
from paper_2107_07315_gb300 import inputs as I
from paper_2107_07315_gb300 import sph

pytestmark = pytest.mark.gpu
MAT = dict(I.DEFAULT_MATERIAL)
FIELDS = ("ax", "ay", "az", "dudt", "drhodt", "rho", "P", "D", "cs", "deps", "dR", "dS", "ncount")
KEYS = ("x", "y", "z", "vx", "vy", "vz", "u", "h", "S", "flags")


@pytest.fixture(scope="module")
def ensemble():
    return I.ensemble_state(nstars=6, seed=2107, scale_n=0.02, nr=512)


@pytest.mark.parametrize("lanes,screen", [(8, 4), (4, 4), (8, 8), (4, 8)])
def test_persistent_rates_equal_separate_launches(lanes, screen):
    st, eos = I.random_state(2500, seed=91, vel=0.2, stress=0.05)
    base = dict(lanes_per_particle=lanes, screen_lanes=screen)
    a, ca, _ = gpu_rhs(st, eos, MAT, None, sph.SPH_MIXED, dict(base, persistent=1))
    b, cb, _ = gpu_rhs(st, eos, MAT, None, sph.SPH_MIXED, base)
    assert sph.sph_stats(ca)[25] > 0 and sph.sph_stats(cb)[25] == 0
    for k in FIELDS:
        assert np.array_equal(a[k], b[k]), k
    o = oracle.rhs(st, eos, MAT, None, scales=True)
    assert_close(a, o, TOL_MIXED, label="persistent")


def test_persistent_ensemble_vs_oracle(ensemble):
    # six stars of uneven size in one index space, one persistent launch
    st, eos, met, _ = ensemble
    o = oracle.rhs(st, eos, MAT, met, scales=True)
    g, ctx, _ = gpu_rhs(st, eos, MAT, met, sph.SPH_MIXED, dict(persistent=1))
    assert sph.sph_stats(ctx)[25] > 0
    offs, idx = oracle.neighbors(st)
    assert_same_neighbors(ctx, offs, idx)
    assert_close(g, o, TOL_MIXED, label="persistent ensemble")


def _steps(st, eos, met, options, nsteps):
    dev = sph.device_state(st)
    torch.cuda.synchronize()
    ctx = sph.sph_init(dev, eos, MAT, met, sph.SPH_MIXED, options, stream=stream().cuda_stream)
    dt = 0.5 * I.cfl_dt(st, eos)
    sph.sph_step(ctx, dt, nsteps)
    sph.sph_sync(ctx)
    torch.cuda.synchronize()
    return sph.to_numpy(dev), sph.sph_stats(ctx)


def test_persistent_graph_steps_equal_separate_launches(ensemble):
    # graph-captured steps with curve sorts every 3 steps and candidate reuse
    st, eos, met, _ = ensemble
    base = dict(h_nmin=55, h_nmax=65, sort_every=3, use_graph=1)
    a, sa = _steps(st, eos, met, dict(base, persistent=1), 7)
    b, sb = _steps(st, eos, met, base, 7)
    for k in KEYS:
        assert np.array_equal(a[k], b[k]), k
    # screening and the two force kernels become one launch per right-hand side
    assert sa[3] == sb[3] - 2, (sa[3], sb[3])


def test_persistent_is_ignored_in_fp64():
    st, eos = I.random_state(800, seed=92, vel=0.2, stress=0.05)
    g, ctx, _ = gpu_rhs(st, eos, MAT, None, sph.SPH_FP64, dict(persistent=1))
    assert sph.sph_stats(ctx)[25] == 0
    with pytest.raises(sph.SphError):
        gpu_rhs(st, eos, MAT, None, sph.SPH_MIXED, dict(persistent=2))


def test_autotuner_chooses_between_persistent_and_separate():
    st, eos = I.random_state(2600, seed=93, vel=0.2, stress=0.05)
    opts = dict(lanes_per_particle=-1, persistent=-1)
    g, ctx, _ = gpu_rhs(st, eos, MAT, None, sph.SPH_MIXED, opts)
    s = sph.sph_stats(ctx)
    assert s[20] == 1 and s[26] > 0 and s[27] > 0
    assert (s[25] > 0) == (s[27] < s[26])
    o = oracle.rhs(st, eos, MAT, None, scales=True)
    assert_close(g, o, TOL_MIXED, label="tuned persistent")
    # a second context of this configuration takes the cached choice
    g2, ctx2, _ = gpu_rhs(st, eos, MAT, None, sph.SPH_MIXED, opts)
    s2 = sph.sph_stats(ctx2)
    assert s2[20] == 2 and (s2[25] > 0) == (s[25] > 0)
    for k in FIELDS:
        assert np.array_equal(g[k], g2[k]), k
