"""Particle relaxation in an external potential (Sec. II.A) through the C ABI.

The star is placed, jittered, given the relaxation EoS (Gamma = 1.01) and
confined by g_eff = -grad phi_eff of its own density profile, a wall and
velocity damping (see inputs.relax_external).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2107_07315_gb300 import inputs as I
from paper_2107_07315_gb300 import sph

from _parity import TOL_FP64, TOL_MIXED, assert_close, stream

pytestmark = pytest.mark.gpu
MAT = dict(I.DEFAULT_MATERIAL)


@pytest.fixture(scope="module")
def relax_case():
    st, eos_r, ext, eos, prof = I.relax_state(4000, seed=5)
    # some motion, so that the damping term is exercised
    rng = np.random.default_rng(9)
    cs = np.sqrt(eos_r["Gamma"][0] * eos_r["K"][0] * prof.rho_c ** (eos_r["Gamma"][0] - 1.0))
    for k in ("vx", "vy", "vz"):
        st[k] = 0.05 * cs * rng.normal(size=len(st["x"]))
    return st, eos_r, ext, eos, prof


def _ctx(st, eos, prec, ext=None, options=None):
    dev = sph.device_state(st)
    torch.cuda.synchronize()
    ctx = sph.sph_init(dev, eos, MAT, None, prec, options, stream=stream().cuda_stream)
    if ext is not None:
        sph.sph_set_external(ctx, ext)
    return ctx, dev


def _rhs(ctx, n):
    rates = sph.alloc_rates(n)
    torch.cuda.synchronize()
    sph.sph_rhs(ctx, rates)
    sph.sph_sync(ctx)
    torch.cuda.synchronize()
    return sph.to_numpy(rates)


@pytest.mark.parametrize("prec,tol", [(sph.SPH_FP64, TOL_FP64), (sph.SPH_MIXED, TOL_MIXED)])
def test_relax_rhs_parity(relax_case, prec, tol):
    st, eos_r, ext, _, _ = relax_case
    n = len(st["x"])
    o = oracle.rhs(st, eos_r, MAT, None, scales=True, external=ext)
    ctx, _ = _ctx(st, eos_r, prec, ext)
    assert_close(_rhs(ctx, n), o, tol, label="relax rhs")
    # switching the field off gives the plain right-hand side again
    sph.sph_set_external(ctx, None)
    o0 = oracle.rhs(st, eos_r, MAT, None, scales=True)
    assert_close(_rhs(ctx, n), o0, tol, label="field off")


def test_relax_steps_match_oracle(relax_case):
    st, eos_r, ext, _, _ = relax_case
    dt = I.cfl_dt(st, eos_r)
    o, _ = oracle.step(st, eos_r, MAT, None, dt, 5, external=ext)
    ctx, dev = _ctx(st, eos_r, sph.SPH_FP64, ext)
    sph.sph_step(ctx, dt, 5)
    sph.sph_sync(ctx)
    g = sph.to_numpy(dev)
    for k in ("x", "y", "z", "vx", "vy", "vz", "u"):
        scale = np.abs(o[k]).max() + 1e-300
        assert np.abs(g[k] - o[k]).max() <= 1e-11 * scale, k


def test_relax_mixed_run_settles():
    # 2e4 particles, mixed precision, graph-captured steps: the jitter's
    # kinetic energy is damped away and the residual force drops
    st, eos_r, ext, eos, prof = I.relax_state(20000, seed=6)
    n = len(st["x"])
    ctx, dev = _ctx(st, eos_r, sph.SPH_MIXED, ext, dict(use_graph=1))
    a0 = _rhs(ctx, n)
    res0 = np.sqrt(np.mean(a0["ax"] ** 2 + a0["ay"] ** 2 + a0["az"] ** 2))
    dt = I.cfl_dt(st, eos_r)
    ke = []
    for _ in range(8):
        sph.sph_step(ctx, dt, 25)
        sph.sph_sync(ctx)
        s = sph.to_numpy(dev)
        ke.append(0.5 * np.sum(s["m"] * (s["vx"] ** 2 + s["vy"] ** 2 + s["vz"] ** 2)))
    a1 = _rhs(ctx, n)
    res1 = np.sqrt(np.mean(a1["ax"] ** 2 + a1["ay"] ** 2 + a1["az"] ** 2))
    assert ke[-1] < 0.3 * max(ke), ke
    assert res1 < 0.5 * res0, (res0, res1)
    assert np.all(np.isfinite(s["x"]))


@pytest.mark.parametrize("prec", [sph.SPH_FP64, sph.SPH_MIXED])
def test_relax_finish_sets_u_from_star_eos(relax_case, prec):
    # modification step: the star's EoS replaces the relaxation EoS, u is the
    # polytrope's u(rho) at the current density, and the field is off
    st, eos_r, ext, eos, prof = relax_case
    n = len(st["x"])
    ctx, dev = _ctx(st, eos_r, prec, ext)
    sph.sph_step(ctx, I.cfl_dt(st, eos_r), 3)
    sph.sph_relax_finish(ctx, eos)
    sph.sph_sync(ctx)
    r = _rhs(ctx, n)
    u = sph.to_numpy(dev)["u"]
    K, G = float(eos["K"][0]), float(eos["Gamma"][0])
    want = K * r["rho"] ** (G - 1.0) / (G - 1.0)
    assert np.max(np.abs(u - want) / want) < 1e-12
    assert np.max(np.abs(r["P"] - K * r["rho"] ** G) / r["P"]) < (1e-12 if prec == sph.SPH_FP64
                                                                     else 3e-5)
    # no external field any more: the acceleration is the plain one
    o = oracle.rhs(sph.to_numpy(dev), eos, MAT, None, scales=True)
    tol = TOL_FP64 if prec == sph.SPH_FP64 else TOL_MIXED
    assert_close(r, o, tol, label="after finish")


def test_set_external_rejects_bad_tables(relax_case):
    st, eos_r, ext, _, _ = relax_case
    ctx, _ = _ctx(st, eos_r, sph.SPH_MIXED)
    bad = dict(ext, nr=1, g=ext["g"][:, :1])
    with pytest.raises(sph.SphError):
        sph.sph_set_external(ctx, bad)
    bad = dict(ext, damping=-1.0)
    with pytest.raises(sph.SphError):
        sph.sph_set_external(ctx, bad)
