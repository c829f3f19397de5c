"""Run inside a process with SPH_CHECKED=1 (tests/test_gpu_checked.py): the
bounds-checked library on parity cases, then a planted out-of-range candidate
entry that its bounds check must report."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))

import numpy as np  # noqa: E402
import torch  # noqa: E402

import oracle  # noqa: E402
from _parity import TOL_FP64, TOL_MIXED, assert_close, assert_same_neighbors, gpu_rhs  # noqa: E402
from paper_2107_07315_gb300 import inputs as I  # noqa: E402
from paper_2107_07315_gb300 import sph  # noqa: E402

MAT = dict(I.DEFAULT_MATERIAL)


def main():
    assert sph.sph_build_checked(), sph.LIB_PATH
    # parity with every list and permutation entry checked
    st, eos = I.random_state(1500, seed=31, vel=0.2, stress=0.05)
    o = oracle.rhs(st, eos, MAT, None, scales=True)
    offs, idx = oracle.neighbors(st)
    for prec, tol, opts in ((sph.SPH_FP64, TOL_FP64, None), (sph.SPH_MIXED, TOL_MIXED, None),
                            (sph.SPH_MIXED, TOL_MIXED, dict(persistent=1, lanes_per_particle=4))):
        g, ctx, _ = gpu_rhs(st, eos, MAT, None, prec, opts)
        assert_same_neighbors(ctx, offs, idx)
        assert_close(g, o, tol, label="checked build")
        sph.sph_free(ctx)
    ens, eos6, met6, _ = I.ensemble_state(nstars=6, seed=2107, scale_n=0.02, nr=512)
    g, ctx, _ = gpu_rhs(ens, eos6, MAT, met6, sph.SPH_MIXED, dict(persistent=1))
    assert_close(g, oracle.rhs(ens, eos6, MAT, met6, scales=True), TOL_MIXED, label="ensemble")
    sph.sph_step(ctx, 0.5 * I.cfl_dt(ens, eos6), 4)
    sph.sph_sync(ctx)
    sph.sph_free(ctx)
    # a planted out-of-range candidate: the next right-hand side that reuses
    # the candidate lists (no sort, no rebuild) reads it
    st, eos = I.random_state(2000, seed=33, vel=0.0, stress=0.0, solid_frac=0.0)
    n = len(st["x"])
    dev = sph.device_state(st)
    torch.cuda.synchronize()
    ctx = sph.sph_init(dev, eos, MAT, None, sph.SPH_MIXED, dict(sort_every=1000))
    dt = 1e-3 * I.cfl_dt(st, eos)
    sph.sph_step(ctx, dt, 1)
    sph.sph_sync(ctx)
    builds = sph.sph_stats(ctx)[18]
    sph.sph_checked_set_candidate(ctx, 5, 0, n + 7)
    sph.sph_step(ctx, dt, 1)
    try:
        sph.sph_sync(ctx)
        raise AssertionError("the planted entry was not reported")
    except sph.SphError as e:
        assert e.status == 7, e
    assert sph.sph_stats(ctx)[18] == builds  # the lists were reused, not rebuilt
    sph.sph_free(ctx)
    print("checked ok")


if __name__ == "__main__":
    main()
