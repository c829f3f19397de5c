"""Piecewise polytropic EoS (Sec. II.A, after Read et al. 2009) through the
C ABI: a three-piece TOV star against the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2107_07315_gb300 import inputs as I
from paper_2107_07315_gb300 import sph

from _parity import TOL_FP64, TOL_MIXED, assert_close, gpu_rhs, stream

pytestmark = pytest.mark.gpu
MAT = dict(I.DEFAULT_MATERIAL)
PP = dict(K=[100.0], Gamma=[2.0], rho_bound=[[0.0004, 0.001]], Gamma_above=[[2.5, 2.2]])


@pytest.fixture(scope="module")
def pp_star():
    prof = I.tov_solve_pieces(PP, 0.00128)
    st, eos, met, prof = I.star_state(4000, seed=11, prof=prof, crust_frac=0.1,
                                      amp_l0=1e-2, amp_l2=1e-2)
    return st, eos, met, prof


@pytest.mark.parametrize("prec,tol", [(sph.SPH_FP64, TOL_FP64), (sph.SPH_MIXED, TOL_MIXED)])
def test_pieces_rhs_parity(pp_star, prec, tol):
    st, eos, met, prof = pp_star
    assert eos["rho_bound"].shape == (1, 2)
    o = oracle.rhs(st, eos, MAT, met, scales=True)
    # the star spans all three pieces
    k = np.searchsorted(np.asarray(PP["rho_bound"][0]), o["rho"], side="right")
    assert set(np.unique(k)) == {0, 1, 2}
    g, ctx, _ = gpu_rhs(st, eos, MAT, met, prec)
    assert_close(g, o, tol, label="pieces")


def test_pieces_steps_match_oracle(pp_star):
    # FP64 steps: kicks, yield, damage (bulk modulus of the piece) and h update
    st, eos, met, prof = pp_star
    dt = I.cfl_dt(st, eos)
    o, _ = oracle.step(st, eos, MAT, met, dt, 4, h_nmin=55, h_nmax=65)
    dev = sph.device_state(st)
    torch.cuda.synchronize()
    ctx = sph.sph_init(dev, eos, MAT, met, sph.SPH_FP64, dict(h_nmin=55, h_nmax=65),
                       stream=stream().cuda_stream)
    sph.sph_step(ctx, dt, 4)
    sph.sph_sync(ctx)
    g = sph.to_numpy(dev)
    assert np.array_equal(g["h"], o["h"])
    assert np.array_equal(g["flags"], o["flags"])
    for key in ("x", "vx", "u"):
        scale = np.abs(o[key]).max() + 1e-300
        assert np.abs(g[key] - o[key]).max() <= 1e-11 * scale, key


def test_relax_finish_with_pieces(pp_star):
    # the modification step with a piecewise EoS: u(rho) of the piece holding rho
    st, eos, met, prof = pp_star
    dev = sph.device_state(st)
    torch.cuda.synchronize()
    one = dict(K=eos["K"], Gamma=eos["Gamma"])
    ctx = sph.sph_init(dev, one, MAT, met, sph.SPH_FP64, stream=stream().cuda_stream)
    sph.sph_relax_finish(ctx, eos)
    rates = sph.alloc_rates(len(st["x"]))
    torch.cuda.synchronize()
    sph.sph_rhs(ctx, rates)
    sph.sph_sync(ctx)
    r = sph.to_numpy(rates)
    u = sph.to_numpy(dev)["u"]
    want = np.array([oracle.eos_eval_star(eos, 0, x, True)[1] for x in r["rho"]])
    assert np.max(np.abs(u - want) / np.abs(want)) < 1e-12


def test_pieces_rejects_bad_bounds(pp_star):
    st, eos, met, prof = pp_star
    dev = sph.device_state(st)
    torch.cuda.synchronize()
    bad = dict(eos, rho_bound=np.array([[0.001, 0.0004]]))
    with pytest.raises(sph.SphError):
        sph.sph_init(dev, bad, MAT, met, sph.SPH_MIXED, stream=stream().cuda_stream)
