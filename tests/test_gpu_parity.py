"""CUDA path vs FP64 oracle, element by element, through the C ABI.

Neighbour lists are compared bit for bit in both precisions; rates within
the tolerances of tests/_parity.py.
"""
import numpy as np
import pytest

import oracle
from paper_2107_07315_gb300 import inputs as I
from paper_2107_07315_gb300 import sph

from _parity import (TOL_FP64, TOL_MIXED, assert_close, assert_same_neighbors, field_errors,
                     gpu_rhs)

pytestmark = pytest.mark.gpu
MAT = dict(I.DEFAULT_MATERIAL)
PREC = [(sph.SPH_FP64, TOL_FP64), (sph.SPH_MIXED, TOL_MIXED)]


def _check(state, eos, metric=None, mat=MAT, prec=sph.SPH_FP64, tol=TOL_FP64, options=None,
           label=""):
    o = oracle.rhs(state, eos, mat, metric, scales=True)
    g, ctx, _ = gpu_rhs(state, eos, mat, metric, prec, options)
    offs, idx = oracle.neighbors(state)
    assert_same_neighbors(ctx, offs, idx)
    errs = assert_close(g, o, tol, label=label)
    return errs, g, o, ctx


@pytest.mark.parametrize("prec,tol", PREC)
def test_cube_config0(prec, tol):
    # 16^3 lattice, h = 1.3, all solid, uniform-strain velocity (config 0)
    st, eos, _, _ = I.cube_state()
    st["S"][:] = 0.0
    errs, g, o, ctx = _check(st, eos, prec=prec, tol=tol, label="cube")
    assert int(g["ncount"].sum()) == 270984
    stats = sph.sph_stats(ctx)
    assert stats[0] == 270984


@pytest.mark.parametrize("prec,tol", PREC)
@pytest.mark.parametrize("seed,n,nstars", [(1, 1000, 1), (2, 1237, 1), (3, 2051, 3), (4, 777, 2)])
def test_random_states(prec, tol, seed, n, nstars):
    # varied h, mixed fluid/solid, random traceless S, several stars, ragged leaves
    st, eos = I.random_state(n, seed=seed, nstars=nstars, vel=0.2, stress=0.05)
    _check(st, eos, prec=prec, tol=tol, label="random %d" % seed)


@pytest.mark.parametrize("prec,tol", PREC)
@pytest.mark.parametrize("jaumann,yield_mode", [(1, 0), (0, 1)])
def test_material_options(prec, tol, jaumann, yield_mode):
    st, eos = I.random_state(900, seed=9, vel=0.3, stress=0.05, solid_frac=0.8)
    mat = dict(MAT, jaumann=jaumann, yield_mode=yield_mode, alpha_av=0.5, beta_av=1.0)
    _check(st, eos, mat=mat, prec=prec, tol=tol, label="options")


@pytest.mark.parametrize("prec,tol", PREC)
@pytest.mark.parametrize("pressure_form", [0, 1])
def test_star_with_metric(prec, tol, pressure_form):
    # 2e4-particle TOV star in its isotropic background, crust 5 %, l=0+l=2
    st, eos, met, _ = I.star_state(20000, seed=1, amp_l0=1e-3, amp_l2=1e-3)
    met = dict(met, pressure_form=pressure_form)
    _check(st, eos, metric=met, prec=prec, tol=tol, label="star")


@pytest.mark.parametrize("prec,tol", PREC)
def test_edge_single_and_pair(prec, tol):
    eos = dict(K=np.array([1.0]), Gamma=np.array([2.0]))
    # one particle: no neighbours, density = self term
    st = I._empty_state(1)
    st["h"][:] = 1.0
    st["m"][:] = 2.0
    g, ctx, _ = gpu_rhs(st, eos, MAT, None, prec)
    assert g["ncount"][0] == 0
    assert abs(g["D"][0] - 2.0 / np.pi) < tol["D"] * 2.0 / np.pi
    assert g["ax"][0] == 0.0
    # two particles exactly at the support boundary (not neighbours), then
    # just inside it
    for x1, expect in [(2.0, 0), (2.0 - 1e-12, 1)]:
        st = I._empty_state(2)
        st["x"][:] = [0.0, x1]
        st["h"][:] = [1.0, 1.0]
        st["m"][:] = 1.0
        st["type"][:] = [1, 0]
        st["mu"][:] = 0.5
        st["Y0"][:] = 0.1
        st["eps_break"][:] = 0.05
        g, ctx, _ = gpu_rhs(st, eos, MAT, None, prec)
        assert list(g["ncount"]) == [expect, expect]
        o = oracle.rhs(st, eos, MAT, None, scales=True)
        if prec == sph.SPH_FP64:
            assert_close(g, o, tol, label="pair")
        else:
            # At 2h(1 - 5e-13) the exact kernel gradient (~(2-q)^2) lies below
            # FP32 resolution; measure against the pair force's natural scale
            # m (P_a/D_a^2 + P_b/D_b^2) max|dW/dr| = m 2P/D^2 sigma/h.
            assert abs(g["D"][0] - o["D"][0]) <= tol["D"] * o["D"][0]
            fscale = 2 * o["P"][0] / o["D"][0] ** 2 / np.pi
            assert np.all(np.abs(g["ax"] - o["ax"]) <= tol["a"] * fscale)


@pytest.mark.parametrize("prec,tol", PREC)
def test_edge_coincident_and_lonely_star(prec, tol):
    # particles sharing a position (zero separation: W finite, grad W = 0)
    # and a star holding a single particle in a batch
    st, eos = I.random_state(300, seed=12, nstars=2, vel=0.1, stress=0.02)
    st["x"][5], st["y"][5], st["z"][5] = st["x"][6], st["y"][6], st["z"][6]
    st["star"][6] = st["star"][5]
    eos = dict(K=np.array([1.0, 1.2, 0.8]), Gamma=np.array([2.0, 1.9, 2.4]))
    st = {k: (np.concatenate([v, v[..., :1]], axis=-1) if v is not None else None)
          for k, v in st.items()}
    st["star"][-1] = 2
    st["x"][-1] = 500.0
    _check(st, eos, prec=prec, tol=tol, label="edge")


def test_empty_input():
    eos = dict(K=np.array([1.0]), Gamma=np.array([2.0]))
    st = I._empty_state(0)
    import torch

    dev = sph.device_state(st)
    ctx = sph.sph_init(dev, eos, MAT, None, sph.SPH_MIXED)
    sph.sph_rhs(ctx, sph.alloc_rates(0))
    sph.sph_step(ctx, 1e-3, 2)
    sph.sph_sync(ctx)
    torch.cuda.synchronize()


@pytest.mark.parametrize("prec", [sph.SPH_FP64, sph.SPH_MIXED])
def test_momentum_conserved_to_rounding(prec):
    st, eos = I.random_state(2000, seed=21, vel=0.3, stress=0.05)
    st["m"][:] = 1.0
    g, _, _ = gpu_rhs(st, eos, MAT, None, prec)
    eps = 1e-13 if prec == sph.SPH_FP64 else 1e-6
    for k in ("ax", "ay", "az"):
        assert abs(g[k].sum()) < eps * np.abs(g[k]).sum()


@pytest.mark.parametrize("prec", [sph.SPH_MIXED, sph.SPH_FP64])
@pytest.mark.parametrize("lanes,screen", [(4, 4), (8, 4), (4, 8), (8, 8)])
def test_lane_variants_agree(lanes, screen, prec):
    # every launch shape the autotuner may pick, in both precisions
    st, eos = I.random_state(1500, seed=31, vel=0.2, stress=0.05)
    opts = dict(lanes_per_particle=lanes, screen_lanes=screen, use_graph=1)
    tol = TOL_MIXED if prec == sph.SPH_MIXED else TOL_FP64
    _check(st, eos, prec=prec, tol=tol, options=opts, label="lanes")


def test_capacity_error_is_reported():
    st, eos, _, _ = I.cube_state(n_side=8)
    dev = sph.device_state(st)
    ctx = sph.sph_init(dev, eos, MAT, None, sph.SPH_MIXED, dict(max_neighbors=16))
    rates = sph.alloc_rates(len(st["x"]))
    sph.sph_rhs(ctx, rates)
    with pytest.raises(sph.SphError) as e:
        sph.sph_sync(ctx)
    assert e.value.status == 4


@pytest.mark.parametrize("prec,tol", PREC)
def test_lists_beyond_the_default_capacity(prec, tol):
    # ten particles with h raised 2.5x reach about 300 neighbours through
    # h_a + h_b: the default capacity of 256 reports it, a context with
    # max_neighbors = 600 holds the exact lists and rates
    st, eos = I.random_state(3000, seed=41, vel=0.2, stress=0.05)
    big = np.arange(0, 3000, 300)
    st["h"][big] *= 2.5
    o = oracle.rhs(st, eos, MAT, None, scales=True)
    assert o["ncount"].max() > 256
    dev = sph.device_state(st)
    ctx = sph.sph_init(dev, eos, MAT, None, prec)
    sph.sph_rhs(ctx, sph.alloc_rates(len(st["x"])))
    with pytest.raises(sph.SphError) as e:
        sph.sph_sync(ctx)
    assert e.value.status == 4
    sph.sph_free(ctx)
    _check(st, eos, prec=prec, tol=tol, options=dict(max_neighbors=600), label="cap 600")


def test_capacity_retry_grows_the_lists():
    # the host-side retry after SPH_ERR_CAPACITY: restore the checkpoint
    # taken before the failed steps, grow max_neighbors, step again; the
    # state equals a run with the larger capacity from the start
    st, eos = I.random_state(3000, seed=41, vel=0.2, stress=0.05)
    st["h"][np.arange(0, 3000, 300)] *= 2.5
    dt = 0.2 * I.cfl_dt(st, eos)
    dev = sph.device_state(st)
    ctx = sph.sph_init(dev, eos, MAT, None, sph.SPH_MIXED, dict(sort_every=3))
    blob = sph.sph_get_state(ctx)
    sph.sph_step(ctx, dt, 4)
    with pytest.raises(sph.SphError) as e:
        sph.sph_sync(ctx)
    assert e.value.status == 4
    sph.sph_set_state(ctx, blob)
    sph.sph_set_max_neighbors(ctx, 600)
    assert sph.sph_stats(ctx)[6] == 600
    sph.sph_step(ctx, dt, 4)
    sph.sph_sync(ctx)
    a = sph.to_numpy(dev)
    dev2 = sph.device_state(st)
    ref = sph.sph_init(dev2, eos, MAT, None, sph.SPH_MIXED, dict(sort_every=3, max_neighbors=600))
    sph.sph_step(ref, dt, 4)
    sph.sph_sync(ref)
    b = sph.to_numpy(dev2)
    for k in ("x", "y", "z", "vx", "vy", "vz", "u", "h", "S", "flags"):
        assert np.array_equal(a[k], b[k]), k
    with pytest.raises(sph.SphError):
        sph.sph_set_max_neighbors(ctx, 2000)


def test_nonfinite_input_is_reported():
    st, eos, _, _ = I.cube_state(n_side=6)
    st["x"][3] = np.nan
    dev = sph.device_state(st)
    ctx = sph.sph_init(dev, eos, MAT, None, sph.SPH_MIXED)
    sph.sph_rhs(ctx, sph.alloc_rates(len(st["x"])))
    with pytest.raises(sph.SphError) as e:
        sph.sph_sync(ctx)
    assert e.value.status == 6


def test_bad_arguments_rejected():
    st, eos, _, _ = I.cube_state(n_side=4)
    dev = sph.device_state(st)
    with pytest.raises(sph.SphError) as e:
        sph.sph_init(dev, dict(K=[1.0], Gamma=[1.0]), MAT, None, sph.SPH_MIXED)
    assert e.value.status == 1
    bad = dict(st)
    bad["star"] = np.full(len(st["x"]), 3, np.int32)
    with pytest.raises(sph.SphError):
        sph.sph_init(sph.device_state(bad), eos, MAT, None, sph.SPH_MIXED)


@pytest.mark.parametrize("prec,tol", PREC)
@pytest.mark.parametrize("kind", ["cubic", "fcc", "hcp"])
@pytest.mark.parametrize("h", [0.5, 0.5 * 2 ** 0.5])
def test_lattice_shell_boundaries(prec, tol, kind, h):
    # support 2h equal to the first (d = 1) or second (sqrt 2) shell distance:
    # whole shells sit on the strict r < h_a + h_b boundary, where only the
    # FP64 rounding of r^2 decides; lists must still equal the oracle's
    st, eos = I.lattice_state(kind, n=7, d=1.0, h=h)
    # h one ulp larger on a random half of the particles: pairs of two such
    # particles reach just past the shell, the others stop just at it
    pick = np.random.default_rng(3).random(len(st["h"])) < 0.5
    st["h"][pick] *= 1.0 + 2e-16
    if h > 0.6:
        _check(st, eos, prec=prec, tol=tol, label="lattice %s h=%g" % (kind, h))
        return
    # support 2h = d: every neighbour sits at q = r/h_ab ~ 2 where W and grad W
    # vanish like (2 - q)^2, so the pair forces are rounding noise (~1e-31) in
    # any precision; the lists and the density (self term) are what is defined
    o = oracle.rhs(st, eos, MAT, None, scales=True)
    g, ctx, _ = gpu_rhs(st, eos, MAT, None, prec)
    offs, idx = oracle.neighbors(st)
    assert_same_neighbors(ctx, offs, idx)
    assert offs[-1] > 0
    errs = field_errors(g, o)
    for k in ("D", "rho", "P", "cs"):
        assert errs[k] <= tol[k], (k, errs[k])
    assert np.array_equal(g["ncount"], o["ncount"])
