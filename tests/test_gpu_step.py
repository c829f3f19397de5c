"""Time stepping through the C ABI: integrator, yield, damage, h update,
totals, CUDA-graph replay and checkpoint/resume, against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2107_07315_gb300 import inputs as I
from paper_2107_07315_gb300 import sph

pytestmark = pytest.mark.gpu
MAT = dict(I.DEFAULT_MATERIAL)
KEYS = ("x", "y", "z", "vx", "vy", "vz", "u", "h", "S")


from _parity import stream


def _ctx(dev, eos, mat, metric, prec, options=None):
    torch.cuda.synchronize()
    return sph.sph_init(dev, eos, mat, metric, prec, options, stream=stream().cuda_stream)


def _run(st, eos, metric, mat, prec, dt, nsteps, options=None):
    dev = sph.device_state(st)
    ctx = _ctx(dev, eos, mat, metric, prec, options)
    sph.sph_step(ctx, dt, nsteps)
    sph.sph_sync(ctx)
    torch.cuda.synchronize()
    return sph.to_numpy(dev), ctx, dev


def _close(a, b, rel, keys=KEYS):
    for k in keys:
        x, y = np.asarray(a[k], np.float64), np.asarray(b[k], np.float64)
        scale = max(np.abs(y).max(), 1e-300)
        assert np.abs(x - y).max() <= rel * scale, (k, np.abs(x - y).max() / scale)


def test_cube_ten_steps_fp64():
    # config 0: 10 steps of dt = 1e-3 on the 16^3 elastic cube
    st, eos, _, _ = I.cube_state()
    g, ctx, _ = _run(st, eos, None, MAT, sph.SPH_FP64, 1e-3, 10)
    o, _ = oracle.step(st, eos, MAT, None, 1e-3, 10)
    _close(g, o, 1e-12)
    assert np.array_equal(g["flags"], o["flags"])


def test_cube_ten_steps_mixed_vs_fp64():
    st, eos, _, _ = I.cube_state()
    g64, _, _ = _run(st, eos, None, MAT, sph.SPH_FP64, 1e-3, 10)
    g32, _, _ = _run(st, eos, None, MAT, sph.SPH_MIXED, 1e-3, 10)
    _close(g32, g64, 1e-5, keys=("x", "y", "z", "vx", "vy", "vz", "u"))
    _close(g32, g64, 1e-4, keys=("S",))
    assert np.array_equal(g32["flags"], g64["flags"])


def _prestressed_cube(n_side, Y0, eps_b, seed, amp=0.01):
    # traceless initial stresses with von Mises stress between 0.8 and 1.5 Y0
    st, eos, _, _ = I.cube_state(n_side=n_side, amp=amp)
    rng = np.random.default_rng(seed)
    n = len(st["x"])
    S = rng.normal(size=(6, n))
    S[:3] -= S[:3].mean(axis=0)
    sv = np.sqrt(1.5 * (S[0] ** 2 + S[1] ** 2 + S[2] ** 2 + 2 * (S[3] ** 2 + S[4] ** 2 + S[5] ** 2)))
    st["S"] = S / sv * Y0 * rng.uniform(0.8, 1.5, size=n)
    st["Y0"][:] = Y0
    st["eps_break"][:] = eps_b
    return st, eos


@pytest.mark.parametrize("prec", [sph.SPH_FP64, sph.SPH_MIXED])
def test_yield_and_break_flags(prec):
    # deviatoric breaking criterion: yielded and broken sets must equal the
    # oracle's (decisions taken in FP64 on both sides)
    st, eos = _prestressed_cube(10, 0.05, 0.02, 3)
    mat = dict(MAT, break_stress=1)
    g, _, _ = _run(st, eos, None, mat, prec, 1e-3, 1)
    o, _ = oracle.step(st, eos, mat, None, 1e-3, 1)
    assert (o["flags"] & 2).sum() > 0 and (o["flags"] & 1).sum() > 0
    assert np.array_equal(g["flags"] & 2, o["flags"] & 2)
    assert np.array_equal(g["flags"] & 1, o["flags"] & 1)


def _marginal(state, Y0, band):
    # von Mises stress before the last return, relative to the yield stress:
    # a yielded particle was scaled by Y0^2/sv^2, which maps sv^2 to Y0^4/sv^2
    S = state["S"]
    sv2 = 1.5 * (S[0] ** 2 + S[1] ** 2 + S[2] ** 2 + 2 * (S[3] ** 2 + S[4] ** 2 + S[5] ** 2))
    y2 = np.where(Y0 > 0, Y0 ** 2, 1.0)
    pre = np.where((state["flags"] & 1) != 0, y2 ** 2 / np.where(sv2 > 0, sv2, 1.0), sv2)
    return np.abs(pre / y2 - 1.0) < band


def test_yield_and_break_flags_over_steps_fp64():
    # eight FP64 steps of the pre-stressed cube with the deviatoric breaking
    # criterion: the sticky broken flags equal the oracle's; yield flags equal
    # it except for particles within 1e-9 of the yield surface, where the two
    # runs' FP64 rounding orders decide (none is expected); the velocity
    # field (0.2 A x) keeps loading particles onto the yield surface
    st, eos = _prestressed_cube(10, 0.05, 0.02, 3, amp=0.2)
    mat = dict(MAT, break_stress=1)
    g, _, _ = _run(st, eos, None, mat, sph.SPH_FP64, 1e-3, 8)
    o, _ = oracle.step(st, eos, mat, None, 1e-3, 8)
    assert (o["flags"] & 2).sum() > 0 and (o["flags"] & 1).sum() >= 10
    assert np.array_equal(g["flags"] & 2, o["flags"] & 2)
    diff = ((g["flags"] ^ o["flags"]) & 1) != 0
    marg = _marginal(o, st["Y0"], 1e-9) | _marginal(g, st["Y0"], 1e-9)
    assert not np.any(diff & ~marg), np.where(diff & ~marg)[0][:10]
    assert diff.sum() <= 2
    _close(g, o, 1e-10, keys=("x", "y", "z", "vx", "vy", "vz", "u"))


def test_break_zero_stress_option():
    st, eos = _prestressed_cube(8, 0.05, 0.02, 4)
    mat = dict(MAT, break_stress=1, break_zero_S=1)
    g, _, _ = _run(st, eos, None, mat, sph.SPH_FP64, 2e-3, 6)
    o, _ = oracle.step(st, eos, mat, None, 2e-3, 6)
    assert np.array_equal(g["flags"], o["flags"])
    _close(g, o, 1e-11, keys=("S", "mu"))


def test_star_steps_with_metric_and_h_update():
    st, eos, met, _ = I.star_state(6000, seed=4, amp_l0=1e-2, amp_l2=1e-2)
    dt = I.cfl_dt(st, eos)
    opts = dict(h_nmin=55, h_nmax=65)
    g, _, _ = _run(st, eos, met, MAT, sph.SPH_FP64, dt, 4, opts)
    o, _ = oracle.step(st, eos, MAT, met, dt, 4, h_nmin=55, h_nmax=65)
    assert np.array_equal(g["h"], o["h"])
    _close(g, o, 1e-11)


@pytest.mark.parametrize("prec", [sph.SPH_FP64, sph.SPH_MIXED])
def test_graph_replay_matches_direct_launches(prec):
    st, eos = I.random_state(3000, seed=5, vel=0.1, stress=0.03)
    a, _, _ = _run(st, eos, None, MAT, prec, 1e-3, 5, dict(use_graph=1))
    b, _, _ = _run(st, eos, None, MAT, prec, 1e-3, 5, dict(use_graph=0))
    for k in KEYS + ("flags",):
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("prec", [sph.SPH_FP64, sph.SPH_MIXED])
@pytest.mark.parametrize("sort_every", [1, 3])
def test_checkpoint_resume_bit_exact(prec, sort_every):
    # with sort_every = 3 the resumed steps 2 and 4, 5 keep the order of the
    # sorts at steps 0 and 3: the checkpoint carries that order
    opts = dict(sort_every=sort_every)
    st, eos = I.random_state(2500, seed=6, vel=0.2, stress=0.05)
    full, _, _ = _run(st, eos, None, MAT, prec, 1e-3, 6, opts)
    dev = sph.device_state(st)
    ctx = _ctx(dev, eos, MAT, None, prec, opts)
    sph.sph_step(ctx, 1e-3, 2)
    blob = sph.sph_get_state(ctx)
    # resume in a fresh context bound to fresh buffers
    st2 = {k: (None if v is None else np.zeros_like(v)) for k, v in st.items()}
    st2["h"][:] = 1.0
    st2["m"] = st["m"].copy()
    st2["star"] = st["star"].copy()
    dev2 = sph.device_state(st2)
    ctx2 = _ctx(dev2, eos, MAT, None, prec, opts)
    sph.sph_set_state(ctx2, blob)
    sph.sph_step(ctx2, 1e-3, 4)
    sph.sph_sync(ctx2)
    res = sph.to_numpy(dev2)
    for k in KEYS + ("flags",):
        assert np.array_equal(res[k], full[k]), k


@pytest.mark.parametrize("prec", [sph.SPH_FP64, sph.SPH_MIXED])
def test_restore_into_the_same_context_after_a_sort(prec):
    # steps 0-1, checkpoint, steps 2-5 (a sort at step 3 gives a new order and
    # new candidate lists); restoring the checkpoint in the same context and
    # stepping 2-5 again repeats the first pass bit for bit: the candidate
    # lists of the later order are not reused for the restored one
    opts = dict(sort_every=3)
    st, eos = I.random_state(2500, seed=16, vel=0.2, stress=0.05)
    dev = sph.device_state(st)
    ctx = _ctx(dev, eos, MAT, None, prec, opts)
    sph.sph_step(ctx, 1e-3, 2)
    blob = sph.sph_get_state(ctx)
    sph.sph_step(ctx, 1e-3, 4)
    sph.sph_sync(ctx)
    first = sph.to_numpy(dev)
    builds = sph.sph_stats(ctx)[18]
    sph.sph_set_state(ctx, blob)
    sph.sph_step(ctx, 1e-3, 4)
    sph.sph_sync(ctx)
    again = sph.to_numpy(dev)
    for k in KEYS + ("flags",):
        assert np.array_equal(again[k], first[k]), k
    assert sph.sph_stats(ctx)[18] > builds  # the restore forced a build


@pytest.mark.parametrize("prec, rel", [(sph.SPH_FP64, 1e-12), (sph.SPH_MIXED, 2e-5)])
def test_sort_every_keeps_lists_exact(prec, rel):
    # steps 1-3 of sort_every = 4 keep the order of step 0's sort: the lists
    # of step 1 (same positions in both runs) are the same sets, and nine
    # steps differ from sorting every step by the rounding of the pair-sum
    # order only; h follows the neighbour counts, so it stays bit-identical
    st, eos, met, _ = I.star_state(8000, seed=3, amp_l0=0.02, amp_l2=0.02)
    dt = I.cfl_dt(st, eos)
    opts = lambda k: dict(h_nmin=55, h_nmax=65, sort_every=k)
    _, c1, _ = _run(st, eos, met, MAT, prec, dt, 2, opts(1))
    _, c4, _ = _run(st, eos, met, MAT, prec, dt, 2, opts(4))
    o1, i1 = sph.neighbors(c1)
    o4, i4 = sph.neighbors(c4)
    assert np.array_equal(o1, o4) and np.array_equal(i1, i4)
    assert sph.sph_stats(c4)[13] == 4
    a, ca, _ = _run(st, eos, met, MAT, prec, dt, 9, opts(1))
    b, cb, _ = _run(st, eos, met, MAT, prec, dt, 9, opts(4))
    assert np.array_equal(a["h"], b["h"]) and np.array_equal(a["flags"], b["flags"])
    _close(b, a, rel, keys=("x", "y", "z", "vx", "vy", "vz", "u"))
    # the steps that keep the order launch fewer kernels (no keys, no radix passes)
    la, lb = sph.sph_stats(ca)[12], sph.sph_stats(cb)[12]
    assert lb < la


def test_checkpoint_with_bad_order_is_rejected():
    # the order stored in a checkpoint must be a permutation of the particles
    st, eos = I.random_state(500, seed=8, vel=0.1)
    dev = sph.device_state(st)
    ctx = _ctx(dev, eos, MAT, None, sph.SPH_MIXED)
    sph.sph_step(ctx, 1e-3, 1)
    blob = sph.sph_get_state(ctx).copy()
    n = len(st["x"])
    perm = blob[-4 * n:].view(np.int32)
    perm[1] = perm[0]
    with pytest.raises(sph.SphError):
        sph.sph_set_state(ctx, blob)
    sph.sph_set_state(ctx, sph.sph_get_state(ctx))


def test_host_round_trip_steps_equal_device_steps():
    # the end-to-end loop (step fields copied in from pinned host memory and
    # back out around every step, one copy each way through the packed
    # layout) computes exactly what device-resident steps compute
    st, eos, met, _ = I.star_state(6000, seed=12, amp_l0=0.02)
    dt = I.cfl_dt(st, eos)
    opts = dict(h_nmin=55, h_nmax=65, sort_every=4)
    ref, _, _ = _run(st, eos, met, MAT, sph.SPH_MIXED, dt, 6, opts)
    fields, buf, step_bytes = sph.device_state_packed(st)
    ctx = _ctx(fields, eos, MAT, met, sph.SPH_MIXED, opts)
    host = buf[:step_bytes].cpu().pin_memory()
    dstep = buf[:step_bytes]
    s = stream()
    with torch.cuda.stream(s):
        for _ in range(6):
            dstep.copy_(host, non_blocking=True)
            sph.sph_step(ctx, dt, 1)
            host.copy_(dstep, non_blocking=True)
    sph.sph_sync(ctx)
    torch.cuda.synchronize()
    got = sph.to_numpy(fields)
    for k in KEYS + ("flags",):
        assert np.array_equal(got[k], ref[k]), k


def test_totals_match_oracle():
    st, eos, _, _ = I.cube_state(n_side=10)
    g, ctx, _ = _run(st, eos, None, MAT, sph.SPH_FP64, 1e-3, 3)
    o, ro = oracle.step(st, eos, MAT, None, 1e-3, 3)
    tg = sph.sph_totals(ctx)
    to = oracle.totals(o, ro["ncount"])
    assert np.allclose(tg, to, rtol=1e-11, atol=1e-12 * np.abs(to).max())


def test_energy_conservation_short_run():
    st, eos = I.random_state(3375, seed=7, box=7.0, lattice=True, vel=0.02, stress=0.0,
                             solid_frac=0.0)
    st["h"][:] = 1.3 * 7.0 / 15
    dev = sph.device_state(st)
    ctx = _ctx(dev, eos, MAT, None, sph.SPH_MIXED)
    e0 = sph.sph_totals(ctx)[6]
    sph.sph_step(ctx, 2e-3, 20)
    e1 = sph.sph_totals(ctx)[6]
    assert abs(e1 - e0) < 1e-4 * abs(e0)


def test_batch_equals_separate_stars():
    # three independent stars in one index space vs each star alone
    st, eos = I.random_state(2400, seed=8, nstars=3, vel=0.1, stress=0.03)
    o_all = oracle.rhs(st, eos, MAT, None)
    from _parity import gpu_rhs

    g_all, _, _ = gpu_rhs(st, eos, MAT, None, sph.SPH_FP64)
    for s in range(3):
        ids = np.where(st["star"] == s)[0]
        sub = {k: (v[..., ids] if v is not None else None) for k, v in st.items()}
        sub["star"] = np.zeros(len(ids), np.int32)
        e1 = dict(K=eos["K"][s:s + 1], Gamma=eos["Gamma"][s:s + 1])
        g1, _, _ = gpu_rhs(sub, e1, MAT, None, sph.SPH_FP64)
        for k in ("ax", "D", "dudt"):
            assert np.allclose(g1[k], g_all[k][ids], rtol=1e-12, atol=1e-13 * np.abs(o_all[k]).max())
        assert np.array_equal(g1["ncount"], g_all["ncount"][ids])
