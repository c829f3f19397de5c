#!/usr/bin/env python3
"""Benchmark: pair interactions/s of the full SPH-elastic right-hand side.

Workload (default): one TOV neutron star of 1e5 equal-mass particles
(M = 1.4 Msun, R = 12 km, Gamma = 2, outer 5 % of the radius solid crust with
mu = 0.01 P, Y0 = 0.1, eps_break = 0.05, isotropic background metric, l = 0
perturbation of 1e-3 c_s, h adapted to 60 +- 5 neighbours), mixed precision.
A step is one kick-drift-kick step: Hilbert-curve sort, neighbour lists, density,
equation of state, pair forces, stress rate, background force, integration,
yield scaling, damage test and h update.  Pairs = ordered neighbour pairs of
the step's right-hand side.

Multi-GPU (torchrun): every rank advances its own star (independent
problems, weak scaling, no data-path collective); rank 0 prints one JSON line.
`--impl reference` times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pair interactions/s of full SPH-elastic RHS, FP32 vs FP64 at stated error"
N_STAR = 100_000
FP32_LANES_PER_SM = 128
# Algorithmic FP32 flops per ordered pair (FMA = 2), counted from the formulas
# as the kernels evaluate them once per pair: force pass 74 for a fluid pair
# (+45 when either particle is solid), density pass 22.
FLOPS_FORCE_PAIR = 74.0
FLOPS_FORCE_SOLID_EXTRA = 45.0
FLOPS_DENSITY_PAIR = 22.0
# FP64 pair kernels run on the FP64 pipe: nominal dense FP64 rate of the GPU
# (context only; the roofline divides by the rate measured in the same run)
FP64_NOMINAL_TFLOPS = 1.25


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def select_stars(st, eos, met, stars):
    """Particles, EoS and metric tables of the listed stars, renumbered 0..k-1."""
    stars = list(stars)
    ids = np.where(np.isin(st["star"], stars))[0]
    sub = {k: (v[..., ids] if v is not None else None) for k, v in st.items()}
    remap = {s: i for i, s in enumerate(stars)}
    sub["star"] = np.array([remap[s] for s in sub["star"]], np.int32)
    e = {"K": np.asarray(eos["K"])[stars], "Gamma": np.asarray(eos["Gamma"])[stars]}
    g = dict(met)
    for k in ("r_max", "alpha", "dalpha", "psi4", "dpsi4", "M", "center"):
        g[k] = np.asarray(met[k])[stars]
    return sub, e, g


def make_star(seed: int, n: int = N_STAR):
    from paper_2107_07315_gb300 import inputs as I

    st, eos, met, prof = I.star_state(n, seed=seed)
    dt = I.cfl_dt(st, eos)
    return st, eos, met, dt


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


class _Nvml:
    """Minimal ctypes view of NVML (clock and clock-event-reason queries only)."""

    SM = 1  # NVML_CLOCK_SM
    REASONS = ((0x8, "hw_slowdown"), (0x40, "hw_thermal_slowdown"),
               (0x20, "sw_thermal_slowdown"), (0x4, "sw_power_cap"),
               (0x80, "hw_power_brake_slowdown"))

    def __init__(self, uuid: str | None, index: int):
        import ctypes as C

        self.C = C
        self.lib = C.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        self.h = C.c_void_p()
        ok = False
        if uuid:
            ok = self.lib.nvmlDeviceGetHandleByUUID(uuid.encode(), C.byref(self.h)) == 0
        if not ok and self.lib.nvmlDeviceGetHandleByIndex_v2(index, C.byref(self.h)) != 0:
            raise OSError("no NVML handle")
        try:
            self.reasons_fn = self.lib.nvmlDeviceGetCurrentClocksEventReasons
        except AttributeError:
            self.reasons_fn = self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
        v = C.c_uint()
        self.lib.nvmlDeviceGetMaxClockInfo(self.h, self.SM, C.byref(v))
        self.max_mhz = float(v.value)

    def sample(self):
        C = self.C
        mhz, bits = C.c_uint(), C.c_ulonglong()
        if self.lib.nvmlDeviceGetClockInfo(self.h, self.SM, C.byref(mhz)) != 0:
            return None
        self.reasons_fn(self.h, C.byref(bits))
        return float(mhz.value), int(bits.value)


class ClockSampler:
    """SM clock and clock-event reasons sampled during the timed region.

    NVML is polled every 0.5 ms from a thread (the timed region of a short run
    lasts only milliseconds); without NVML, nvidia-smi is polled every 200 ms.
    """

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, uuid: str | None = None):
        self.proc = None
        self.thread = None
        self.gpu = gpu_index
        self.uuid = uuid
        self.out = os.path.join("/tmp", "sph_clocks_%d_%d.csv" % (os.getpid(), gpu_index))
        try:
            self.nvml = _Nvml(uuid, gpu_index)
        except Exception:
            self.nvml = None

    def start(self):
        import threading

        self.samples = []
        if self.nvml is not None:
            self.stop_flag = threading.Event()

            def poll():
                while not self.stop_flag.is_set():
                    s = self.nvml.sample()
                    if s is not None:
                        self.samples.append(s)
                    time.sleep(0.0005)

            self.thread = threading.Thread(target=poll, daemon=True)
            self.thread.start()
            return
        try:
            self.f = open(self.out, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.thread is not None:
            self.stop_flag.set()
            self.thread.join()
            s = self.nvml.sample()
            if s is not None:
                self.samples.append(s)
            if not self.samples:
                return None
            reasons = set()
            for _, bits in self.samples:
                for b, nm in _Nvml.REASONS:
                    if bits & b:
                        reasons.add(nm)
            return {"sm_mhz": statistics.median(m for m, _ in self.samples),
                    "sm_max_mhz": self.nvml.max_mhz, "reasons": sorted(reasons),
                    "samples": len(self.samples), "source": "nvml, 0.5 ms period"}
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], 0.0, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in open(self.out):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = max(mx, float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm), "source": "nvidia-smi, 200 ms period"}


# the mixed force pass is two kernels (all-fluid blocks, blocks with a solid);
# each entry names the summaries and the sources their kernels are built from
PROFILE_FILES = {
    "force": (("force_mixed_fluid_star1e5.md", "force_mixed_solid_star1e5.md"),
              ("sph_pairs.cu", "sph_device.cuh")),
    "lists": (("tiles_star1e5.md", "screen_star1e5.md"),
              ("sph_tiles.cu", "sph_screen.cuh", "sph_device.cuh")),
}


def source_hash(srcs) -> str:
    """First 16 hex digits of the SHA-256 of the named kernel sources, in order."""
    hs = hashlib.sha256()
    for src in srcs:
        with open(os.path.join(ROOT, "paper_2107_07315_gb300", "csrc", src), "rb") as f:
            hs.update(f.read())
    return hs.hexdigest()[:16]


def traffic_from_profile(key: str):
    """DRAM bytes per pass from the committed ncu summaries of its kernels,
    or None when their sources changed since the counters were taken."""
    names, srcs = PROFILE_FILES[key]
    h = source_hash(srcs)
    total = 0.0
    for name in names:
        path = os.path.join(ROOT, "profiles", name)
        if not os.path.exists(path):
            return None
        src_ok, traffic = False, None
        for line in open(path):
            if line.startswith("kernel_source_sha256_16:") and line.split(":")[1].strip() == h:
                src_ok = True
            if line.startswith("dram_bytes_per_launch:"):
                try:
                    traffic = float(line.split(":")[1].strip())
                except ValueError:
                    traffic = None
        if not src_ok or traffic is None:
            return None
        total += traffic
    return total


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2107_07315_gb300 import inputs as I
    from paper_2107_07315_gb300 import sph

    ws, rank, local = dist_env()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    dev = torch.device("cuda", torch.cuda.current_device())
    if args.workload == "ensemble":
        from paper_2107_07315_gb300 import shard

        # the 64-star ensemble: this rank advances its LPT share of the stars
        full, eos_all, met_all, params = I.ensemble_state(nstars=args.nstars, seed=2107,
                                                          scale_n=args.scale, nr=1024)
        mine = shard.assign_stars(params["N"], ws)[rank]
        st, eos, met = select_stars(full, eos_all, met_all, mine)
        dt = 0.5 * I.cfl_dt(st, eos)
        nst = len(mine)
    elif args.workload == "relax":
        # relaxation of a jittered star in its external potential (Sec. II.A):
        # relaxation EoS (Gamma = 1.01), g_eff table, wall, damping; no metric
        st, eos, ext, _, _ = I.relax_state(args.n, seed=1 + rank)
        met = None
        dt = I.cfl_dt(st, eos)
        nst = 1
    else:
        st, eos, met, dt = make_star(1 + rank, args.n)
        nst = 1
    external = ext if args.workload == "relax" else None
    n = len(st["x"])
    prec = sph.SPH_MIXED if args.precision == "mixed" else sph.SPH_FP64
    stream = torch.cuda.Stream()
    # one device buffer; the fields a step changes lead it (one copy each way for e2e)
    dstate, dbuf, step_bytes = sph.device_state_packed(st, dev)
    torch.cuda.synchronize()
    # measured FP32 / FP64 FMA rates and SM count of this GPU (roofline peaks)
    rates = sph.sph_peak_rates()
    ctx = sph.sph_init(dstate, eos, I.DEFAULT_MATERIAL, met, prec,
                       dict(h_nmin=55, h_nmax=65, use_graph=1, sort_every=args.sort_every,
                            skin=args.skin, lanes_per_particle=-1 if args.tune else 0,
                            persistent=-1 if args.tune else args.persistent),
                       stream=stream.cuda_stream)
    if external is not None:
        sph.sph_set_external(ctx, external)
    shape = launch_shape(sph.sph_stats(ctx))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            sph.sph_step(ctx, dt, 1)
        sph.sph_sync(ctx)
    stats0 = sph.sph_stats(ctx)
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        pass
    clk = ClockSampler(torch.cuda.current_device(), uuid)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clk.start()
    t_ms, _ = time_steps(ctx, dt, args.steps, 0, flush, stream)
    if ws > 1:
        dist.barrier()
    clocks = clk.stop()
    sph.sph_sync(ctx)
    stats1 = sph.sph_stats(ctx)
    pairs = float(stats1[1] - stats0[1])
    # per-kernel times: a separate pass whose step graph carries event nodes
    # between the phases (the nodes cost time of their own, so the timed
    # steps above run without them); a whole number of sort cycles
    sph.sph_timing(ctx, True)
    with torch.cuda.stream(stream):
        sph.sph_step(ctx, dt, 1)  # captures the instrumented graph
    sph.sph_sync(ctx)
    sph.sph_timing_read(ctx)
    k_steps = max(1, args.sort_every) * max(1, 16 // max(1, args.sort_every))
    t_inst, _ = time_steps(ctx, dt, k_steps, 0, flush, stream)
    sph.sph_sync(ctx)
    tim = sph.sph_timing_read(ctx)
    sph.sph_timing(ctx, False)
    # solid-pair share for the flop count (pairs touching a crust particle)
    pairs_step = float(stats1[0])
    solid_pairs = 0.0
    if args.count_solid:
        offs, idx = sph.neighbors(ctx)
        ty = st["type"]
        cnt = np.diff(offs)
        owner = np.repeat(np.arange(n), cnt)
        solid_pairs = float(np.count_nonzero((ty[owner] == 1) | (ty[idx] == 1)))
    # re-capture the plain step graphs (both sort phases) outside the e2e timing
    with torch.cuda.stream(stream):
        for _ in range(max(1, args.sort_every)):
            sph.sph_step(ctx, dt, 1)
    sph.sph_sync(ctx)

    # end-to-end: the step's fields (positions, velocities, u, h, S, flags) live
    # in pinned host memory; every step copies them in, steps, copies them out
    host = dbuf[:step_bytes].cpu().pin_memory()
    dstep = dbuf[:step_bytes]
    h2d = step_bytes
    e2e_steps = max(3, min(args.steps, 20))
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    p_before = sph.sph_stats(ctx)[1]
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(e2e_steps):
            dstep.copy_(host, non_blocking=True)
            sph.sph_step(ctx, dt, 1)
            host.copy_(dstep, non_blocking=True)
        e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    e2e_pairs = float(sph.sph_stats(ctx)[1] - p_before)
    launches = int(stats1[12] - stats0[12])
    builds_per_step = float(stats1[18] - stats0[18]) / max(args.steps, 1)

    # the ensemble's only data collective: the per-star FP64 totals, gathered
    # from every rank (each star lives on one rank); every rank takes part
    star_totals = None
    if args.workload == "ensemble":
        from paper_2107_07315_gb300 import shard

        per = sph.sph_totals_per_star(ctx, nst)
        allt = shard.gather_star_totals(mine, per, args.nstars, dev)
        star_totals = {"stars": int(args.nstars), "mass": float(allt[:, 0].sum()),
                       "energy": float(allt[:, 6].sum()), "yielded": float(allt[:, 10].sum()),
                       "broken": float(allt[:, 11].sum())}
    # aggregate over ranks: total pairs, max time
    if ws > 1:
        from paper_2107_07315_gb300 import shard

        t_ms, pairs = shard.reduce_timing(t_ms, pairs, dev)
        e2e_ms, e2e_pairs = shard.reduce_timing(e2e_ms, e2e_pairs, dev)
    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return None

    value = pairs / (t_ms * 1e-3)
    rl = rooflines(tim, n, pairs_step, solid_pairs, prec == sph.SPH_MIXED, rates,
                   profiled=(args.workload == "star" and n == N_STAR and prec == sph.SPH_MIXED))
    out = {
        "metric": METRIC,
        "value": value,
        "unit": "pairs/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": t_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32" if prec == sph.SPH_MIXED else "f64",
        "data": "synthetic",
        "config": {
            "workload": ("TOV star, %d particles (M=1.4, R=12 km, Gamma=2, 5%% crust), "
                         "isotropic background, one KDK step per timed step incl. sort and "
                         "neighbour lists" % n) if args.workload == "star" else
                        ("relaxation of a jittered %d-particle star in its external potential "
                         "(Gamma 1.01, g_eff table, wall, damping), one KDK step per timed step"
                         % n) if args.workload == "relax" else
                        ("ensemble of %d stars (log-uniform N, Gamma 1.8-2.5, crust 3-10%%), "
                         "%d particles on this GPU, one launch per kernel for all stars"
                         % (args.nstars, n)),
            "precision": "mixed: FP32 pair sums (Kahan D, du), FP64 state/integration/totals"
                         if prec == sph.SPH_MIXED else "fp64",
            "n_particles": n,
            "pairs_per_step": pairs_step,
            "stars_per_gpu": nst,
            "sort_every": args.sort_every,
            "skin": args.skin if args.skin != 0 else 0.1,
            "library_defaults": {"sort_every": 1, "skin": 0.1},
            "candidate_builds_per_step": builds_per_step,
            "l2": "flushed between timed steps by a 256 MB write outside the events",
            "parallelism": "independent star per GPU" if ws > 1 else "single GPU",
        },
        "launch_shape": shape,
        "roofline": rl["dominant"],
        "kernels": rl["all"],
        "peaks": {"fp32_tflops_measured": rates["fp32_tflops"],
                  "fp64_tflops_measured": rates["fp64_tflops"], "sms": rates["sms"],
                  "fp32_tflops_nominal": rl["fp32_nominal"],
                  "how": "sph_peak_rates: 8 independent FMA chains per thread, "
                         "8 x 256-thread blocks per SM, CUDA events"},
        # the right-hand side alone (sort, tree, lists, density, force), from the
        # CUDA events inside the timed steps; the step adds both kicks
        "rhs_only": _rhs_only(tim, pairs_step),
        # the instrumented pass that gave the per-kernel times
        "instrumented_ms_per_step": t_inst / k_steps,
        "gpu_launches": launches,
        "e2e": {"value": e2e_pairs / (e2e_ms * 1e-3), "unit": "pairs/s",
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(h2d)},
        "clocks": clocks,
    }
    if ws == 1 and args.sort_every > 1:
        # the same protocol with a curve sort on every step, for comparison
        c1 = sph.sph_init(dstate, eos, I.DEFAULT_MATERIAL, met, prec,
                          dict(h_nmin=55, h_nmax=65, use_graph=1, sort_every=1,
                               lanes_per_particle=-1 if args.tune else 0,
                               persistent=-1 if args.tune else args.persistent),
                          stream=stream.cuda_stream)
        if external is not None:
            sph.sph_set_external(c1, external)
        with torch.cuda.stream(stream):
            for _ in range(max(3, args.warmup)):
                sph.sph_step(c1, dt, 1)
        sph.sph_sync(c1)
        l0 = int(sph.sph_stats(c1)[12])
        t1, p1 = time_steps(c1, dt, args.steps, 0, flush, stream)
        sph.sph_sync(c1)
        out["sort_every_1"] = {"value": p1 / (t1 * 1e-3), "unit": "pairs/s",
                               "ms_per_step": t1 / args.steps,
                               "gpu_launches": int(sph.sph_stats(c1)[12]) - l0}
        sph.sph_free(c1)
    if ws == 1 and args.fp64_steps > 0 and prec == sph.SPH_MIXED:
        # the plain FP64 GPU path on the same star, same step and flush protocol
        d64 = sph.device_state(st, dev)
        torch.cuda.synchronize()
        c64 = sph.sph_init(d64, eos, I.DEFAULT_MATERIAL, met, sph.SPH_FP64,
                           dict(h_nmin=55, h_nmax=65, use_graph=1, sort_every=args.sort_every),
                           stream=stream.cuda_stream)
        if external is not None:
            sph.sph_set_external(c64, external)
        t64, p64 = time_steps(c64, dt, args.fp64_steps, 3, flush, stream)
        sph.sph_free(c64)
        del d64
        v64 = p64 / (t64 * 1e-3)
        out["fp64"] = {"value": v64, "unit": "pairs/s", "ms_per_step": t64 / args.fp64_steps,
                       "steps": args.fp64_steps, "mixed_speedup": value / v64}
    if star_totals is not None:
        out["star_totals"] = star_totals
    if ws == 1 and args.mode_check and args.workload == "star":
        out["mode_accuracy"] = mode_accuracy(dev, stream)
    if not args.no_cpu_baseline and ws == 1:
        cb, ids, ro = cpu_baseline(st, eos, met, args.cpu_sample)
        out["cpu_baseline"] = cb
        if args.workload == "star":
            # per-field error of one right-hand side of the initial state against
            # the oracle on the sampled particles (normalised as in the tests)
            par = {"mixed": parity_errors(gpu_rates_at(st, eos, met, sph.SPH_MIXED, dev, stream),
                                          ro, ids)}
            if args.fp64_steps > 0:
                par["fp64"] = parity_errors(gpu_rates_at(st, eos, met, sph.SPH_FP64, dev, stream),
                                            ro, ids)
            par["tolerance"] = {"fp64": 1e-12, "mixed": {"D": 1e-5, "rho": 1e-5, "a": 1e-5,
                                                          "dudt": 1e-5, "drhodt": 1e-5,
                                                          "deps": 1e-4, "dS": 1e-4}}
            out["parity"] = par
    print(json.dumps(out), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return out


def rooflines(tim, n, pairs_step, solid_pairs, mixed, rates, profiled=True):
    """Roofline entries of the timed kernels; "dominant" is the pair pass.

    The pair pass is the neighbour-list stage (candidate-list build when
    stale, exact screening, in mixed precision the density summation and the
    equation of state) plus the force kernels.  Its algorithmic work counts
    true neighbour pairs only: 22 FP32 flops per ordered pair for the density
    and 74 for the force, plus 45 for pairs touching a solid particle (FMA =
    2).  Candidate tests that miss are not counted.  Peak: the FP32 (FP64)
    FMA rate measured in the same run; the nominal SMs x 128 lanes x 2 x
    sm_max_mhz is given beside it.
    """
    pk, src = peaks()
    sm_mhz = float(pk.get("sm_max_mhz", 2070.0))
    traffic_of = (lambda key: traffic_from_profile(key)) if profiled else (lambda key: None)
    fp32_nom = rates["sms"] * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
    alu_peak = rates["fp32_tflops"] if mixed else rates["fp64_tflops"]
    alu_src = ("%s FMA rate measured by sph_peak_rates in this run (%d SMs; nominal FP32 "
               "%.1f TFLOP/s at %.0f MHz)" % ("FP32" if mixed else "FP64", rates["sms"],
                                               fp32_nom, sm_mhz))
    ms = {
        "force": tim[0] / max(tim[1], 1),
        "lists": tim[8] / max(tim[9], 1),
        "sort_tree": tim[6] / max(tim[7], 1),
    }
    fl_force = FLOPS_FORCE_PAIR * pairs_step + FLOPS_FORCE_SOLID_EXTRA * solid_pairs
    fl_dens = FLOPS_DENSITY_PAIR * pairs_step
    t_pass = ms["lists"] + ms["force"]
    a = (fl_force + fl_dens) / (t_pass * 1e-3) / 1e12 if t_pass > 0 else 0.0
    tl, tf = traffic_of("lists"), traffic_of("force")
    dominant = {"bound": "alu", "kernel": "pair pass: k_tiles + k_screen (lists, density, EoS) "
                "+ k_force_%s (pair sums, finalize)" % ("mixed" if mixed else "fp64"),
                "achieved": a, "peak": alu_peak, "unit": "TFLOP/s", "frac": a / alu_peak,
                "kernel_ms": t_pass, "work_per_launch": fl_force + fl_dens,
                "peak_source": alu_src,
                "traffic": (tl + tf) if (tl is not None and tf is not None) else None}
    ent = {}
    a = fl_force / (ms["force"] * 1e-3) / 1e12 if ms["force"] > 0 else 0.0
    ent["force"] = {"kernel_ms": ms["force"], "achieved": a, "unit": "TFLOP/s",
                    "frac": a / alu_peak}
    a = fl_dens / (ms["lists"] * 1e-3) / 1e12 if ms["lists"] > 0 else 0.0
    ent["lists"] = {"kernel_ms": ms["lists"], "achieved": a, "unit": "TFLOP/s (density flops)",
                    "frac": a / alu_peak}
    ent["sort_tree"] = {"kernel_ms": ms["sort_tree"]}
    return {"dominant": dominant, "all": ent, "fp32_nominal": fp32_nom,
            "sort_tree_ms": ms["sort_tree"]}


def mode_accuracy(dev, stream, n=20000, nsteps=1200, every=10):
    """Mixed vs FP64 on the same star at equal radial-mode accuracy: the l = 0
    frequency fitted to each run's central-density series, their relative
    difference, and the ratio of their step times (Sec. III.B radial mode)."""
    import torch
    from scipy.optimize import curve_fit

    from paper_2107_07315_gb300 import inputs as I
    from paper_2107_07315_gb300 import sph

    st, eos, met, _ = I.star_state(n, seed=1, amp_l0=1e-2)
    dt = I.cfl_dt(st, eos)
    r0 = np.sqrt(st["x"] ** 2 + st["y"] ** 2 + st["z"] ** 2)
    core = torch.from_numpy(r0 < 0.2 * r0.max()).to(dev)
    res = {}
    for name, prec in (("mixed", sph.SPH_MIXED), ("fp64", sph.SPH_FP64)):
        d = sph.device_state(st, dev)
        torch.cuda.synchronize()
        ctx = sph.sph_init(d, eos, I.DEFAULT_MATERIAL, met, prec, dict(use_graph=1, sort_every=8),
                           stream=stream.cuda_stream)
        rates = sph.alloc_rates(n, dev)
        ms, series, t = 0.0, [], []
        for k in range(0, nsteps + 1, every):
            if k:
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                with torch.cuda.stream(stream):
                    e0.record(stream)
                    sph.sph_step(ctx, dt, every)
                    e1.record(stream)
                torch.cuda.synchronize()
                ms += e0.elapsed_time(e1)
            with torch.cuda.stream(stream):
                sph.sph_rhs(ctx, rates)
            sph.sph_sync(ctx)
            t.append(k * dt)
            series.append(float(rates["rho"][core].mean().item()))
        sph.sph_free(ctx)
        y = np.array(series) - np.mean(series)
        tt = np.array(t)
        f = np.fft.rfftfreq(len(tt), tt[1] - tt[0])
        amp = np.abs(np.fft.rfft(y * np.hanning(len(y))))
        w0 = 2 * math.pi * f[1 + np.argmax(amp[1:])]

        def model(x, a, w, ph, g, c0, c1):
            return a * np.exp(-g * x) * np.sin(w * x + ph) + c0 + c1 * x

        p, _ = curve_fit(model, tt, y, p0=[np.abs(y).max(), w0, 0.0, 0.0, 0.0, 0.0], maxfev=20000)
        res[name] = {"omega": abs(float(p[1])), "ms_per_step": ms / nsteps}
    return {"star_particles": n, "steps": nsteps, "sample_every": every,
            "omega_mixed": res["mixed"]["omega"], "omega_fp64": res["fp64"]["omega"],
            "rel_diff": abs(res["mixed"]["omega"] / res["fp64"]["omega"] - 1.0),
            "tolerance": 1e-3,
            "mixed_ms_per_step": res["mixed"]["ms_per_step"],
            "fp64_ms_per_step": res["fp64"]["ms_per_step"],
            "speedup": res["fp64"]["ms_per_step"] / res["mixed"]["ms_per_step"],
            "note": "l = 0 mode of a 2e4-particle TOV star (amplitude 1e-2 c_s), frequencies "
                    "fitted to the central-density series of each precision's own run"}


def _fit_omega(t, y):
    """Angular frequency of a damped sine fitted to a sampled series (the
    spectral peak starts the fit)."""
    from scipy.optimize import curve_fit

    y = np.asarray(y) - np.mean(y)
    t = np.asarray(t)
    f = np.fft.rfftfreq(len(t), t[1] - t[0])
    amp = np.abs(np.fft.rfft(y * np.hanning(len(y))))
    w0 = 2 * math.pi * f[1 + np.argmax(amp[1:])]

    def model(x, a, w, ph, g, c0, c1):
        return a * np.exp(-g * x) * np.sin(w * x + ph) + c0 + c1 * x

    p, _ = curve_fit(model, t, y, p0=[np.abs(y).max(), w0, 0.0, 0.0, 0.0, 0.0], maxfev=20000)
    return abs(float(p[1]))


def _cfl_dt_device(d, eos, C=0.3):
    """dt = C min h / (c + |v|) of a device state (c from u, polytrope)."""
    import torch

    G = torch.as_tensor(np.asarray(eos["Gamma"], np.float64), device=d["u"].device)
    g = G[d["star"].long()] if d.get("star") is not None else G[0]
    c = torch.sqrt(torch.clamp((g - 1.0) * g * d["u"], min=0.0))
    v = torch.sqrt(d["vx"] ** 2 + d["vy"] ** 2 + d["vz"] ** 2)
    return float(C * torch.min(d["h"] / (c + v)).item())


def _series_run(st, eos, met, prec, dt, nsteps, every, dev, stream, options):
    """Steps one star in graph-captured steps; every `every` steps records the
    core density (one RHS) and Q_zz = sum m (z^2 - r^2/3) about the centre of
    mass.  Returns times, the two series, device ms per step and the state."""
    import torch

    from paper_2107_07315_gb300 import inputs as I
    from paper_2107_07315_gb300 import sph

    n = len(st["x"])
    d = sph.device_state(st, dev)
    torch.cuda.synchronize()
    ctx = sph.sph_init(d, eos, I.DEFAULT_MATERIAL, met, prec, options, stream=stream.cuda_stream)
    rates = sph.alloc_rates(n, dev)
    r0 = np.sqrt(st["x"] ** 2 + st["y"] ** 2 + st["z"] ** 2)
    core = torch.from_numpy(r0 < 0.2 * r0.max()).to(dev)
    m = d["m"]
    ms, t, rho, qzz, eint = 0.0, [], [], [], []
    for k in range(0, nsteps + 1, every):
        if k:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                e0.record(stream)
                sph.sph_step(ctx, dt, every)
                e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
        with torch.cuda.stream(stream):
            sph.sph_rhs(ctx, rates)
        sph.sph_sync(ctx)
        torch.cuda.synchronize()
        t.append(k * dt)
        rho.append(float(rates["rho"][core].mean().item()))
        c = [float((m * d[a]).sum() / m.sum()) for a in ("x", "y", "z")]
        x, y, z = d["x"] - c[0], d["y"] - c[1], d["z"] - c[2]
        qzz.append(float((m * (z * z - (x * x + y * y + z * z) / 3.0)).sum()))
        eint.append(float(sph.sph_totals(ctx)[5]))  # sum m u, the paper's radial-mode signal
    out = sph.to_numpy(d)
    stats = sph.sph_stats(ctx)
    sph.sph_free(ctx)
    del d, rates
    torch.cuda.empty_cache()
    return np.array(t), np.array(rho), np.array(qzz), ms / nsteps, out, stats, np.array(eint)


def campaign(args):
    """Full-length runs of the paper-scale configurations, one JSON line each.

    star1e6 : 1e6-particle star, l = 0 and l = 2 perturbations of 1e-3 c_s,
              5000 steps in mixed precision and in FP64; radial frequency
              from the core density, quadrupole frequency from Q_zz.
    ensemble: the 64-star batch, 1000 mixed steps with the autotuned shape;
              throughput and per-star conservation.
    crust4e6: the 4e6-particle crust-failure star, 2000 steps mixed and FP64;
              yielded and broken counts of both; and the 2e4-particle star of
              the same configuration, FP64 GPU against the FP64 oracle over
              `--oracle-steps` steps (flags compared exactly)."""
    import torch

    from paper_2107_07315_gb300 import inputs as I
    from paper_2107_07315_gb300 import shard
    from paper_2107_07315_gb300 import sph

    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.Stream()
    opts = dict(h_nmin=55, h_nmax=65, use_graph=1, sort_every=8)
    out = {"campaign": args.campaign}
    if args.campaign == "star1e6":
        steps = args.campaign_steps or 5000
        st, eos, met, _ = I.star_state(1_000_000, seed=1, amp_l0=1e-3, amp_l2=1e-3)
        dt = I.cfl_dt(st, eos)
        every = max(1, steps // 250)
        res, ser = {}, {}
        for name, prec in (("mixed", sph.SPH_MIXED), ("fp64", sph.SPH_FP64)):
            t, rho, q, ms, _, stats, eu = _series_run(st, eos, met, prec, dt, steps, every, dev,
                                                      stream, opts)
            ser[name] = (rho, q, eu)
            res[name] = {"omega_radial": _fit_omega(t, rho),
                         "omega_radial_internal_energy": _fit_omega(t, eu),
                         "omega_quadrupole": _fit_omega(t, q),
                         "ms_per_step": ms, "pairs_per_step": int(stats[0])}
        if args.campaign_out:
            np.savez(args.campaign_out, t=t, rho_mixed=ser["mixed"][0], qzz_mixed=ser["mixed"][1],
                     eint_mixed=ser["mixed"][2], rho_fp64=ser["fp64"][0], qzz_fp64=ser["fp64"][1],
                     eint_fp64=ser["fp64"][2])
        # how closely the two runs' series agree, against each series' swing
        for j, key in ((0, "core_density"), (1, "qzz"), (2, "internal_energy")):
            a, b = ser["mixed"][j], ser["fp64"][j]
            out[key + "_max_diff_over_swing"] = float(np.max(np.abs(a - b)) / (np.ptp(b) or 1.0))
        out["radial_periods_covered"] = res["fp64"]["omega_radial"] * steps * dt / (2 * math.pi)
        out.update({"particles": len(st["x"]), "steps": steps, "sample_every": every, "dt": dt,
                    "mixed": res["mixed"], "fp64": res["fp64"],
                    "radial_rel_diff": abs(res["mixed"]["omega_radial"] /
                                           res["fp64"]["omega_radial"] - 1.0),
                    "radial_internal_energy_rel_diff": abs(
                        res["mixed"]["omega_radial_internal_energy"] /
                        res["fp64"]["omega_radial_internal_energy"] - 1.0),
                    "quadrupole_rel_diff": abs(res["mixed"]["omega_quadrupole"] /
                                               res["fp64"]["omega_quadrupole"] - 1.0),
                    "speedup": res["fp64"]["ms_per_step"] / res["mixed"]["ms_per_step"]})
    elif args.campaign == "ensemble":
        steps = args.campaign_steps or 1000
        full, eos_all, met_all, params = I.ensemble_state(nstars=64, seed=2107, scale_n=1.0,
                                                          nr=1024)
        mine = shard.assign_stars(params["N"], 1)[0]
        st, eos, met = select_stars(full, eos_all, met_all, mine)
        dt = 0.5 * I.cfl_dt(st, eos)
        d = sph.device_state(st, dev)
        torch.cuda.synchronize()
        ctx = sph.sph_init(d, eos, I.DEFAULT_MATERIAL, met, sph.SPH_MIXED,
                           dict(opts, lanes_per_particle=-1, persistent=-1),
                           stream=stream.cuda_stream)
        t0 = sph.sph_totals_per_star(ctx, len(mine))
        p0 = sph.sph_stats(ctx)[1]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            sph.sph_step(ctx, dt, steps)
            e1.record(stream)
        sph.sph_sync(ctx)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        stats = sph.sph_stats(ctx)
        t1 = sph.sph_totals_per_star(ctx, len(mine))
        mom0 = np.linalg.norm(t0[:, 1:4], axis=1)
        out.update({"stars": len(mine), "particles": len(st["x"]), "steps": steps,
                    "pairs_per_s": float(stats[1] - p0) / (ms * 1e-3), "ms_per_step": ms / steps,
                    "launch_shape": launch_shape(stats),
                    "max_rel_mass_change": float(np.max(np.abs(t1[:, 0] / t0[:, 0] - 1.0))),
                    "max_rel_energy_change": float(np.max(np.abs(t1[:, 6] / t0[:, 6] - 1.0))),
                    "max_momentum_change_over_mass": float(np.max(
                        np.linalg.norm(t1[:, 1:4] - t0[:, 1:4], axis=1) / t0[:, 0])),
                    "initial_momentum_over_mass_max": float(np.max(mom0 / t0[:, 0])),
                    "yielded": int(t1[:, 10].sum()), "broken": int(t1[:, 11].sum())})
        sph.sph_free(ctx)
    elif args.campaign == "crust4e6":
        import oracle

        steps = args.campaign_steps or 2000
        chunk = 20
        cfg = dict(crust_frac=0.08, mu_over_P=0.01, Y0_over_mu=1e-3, eps_break=0.01, amp_l0=0.0,
                   amp_l2=0.1)
        st, eos, met, _ = I.star_state(4_000_000, seed=7, **cfg)
        crust = st["type"] == 1
        flags, dts = {}, []
        # the strong forcing compresses the crust: dt = 0.3 min h / (c + |v|)
        # is taken again every `chunk` steps, from the FP64 run; the mixed run
        # replays the same sequence
        for name, prec in (("fp64", sph.SPH_FP64), ("mixed", sph.SPH_MIXED)):
            d = sph.device_state(st, dev)
            torch.cuda.synchronize()
            ctx = sph.sph_init(d, eos, I.DEFAULT_MATERIAL, met, prec, opts,
                               stream=stream.cuda_stream)
            # host-side retry: the state is saved every `every` steps; when
            # the lists overflow (ejecta of the strong forcing grow h, and
            # dense particles near them collect several hundred neighbours
            # through h_a + h_b) the run goes back to the last save, doubles
            # max_neighbors and steps again
            every, cap, grown = 10 * chunk, 256, []
            ms, done, err = 0.0, 0, None
            blob, blob_at = sph.sph_get_state(ctx), 0
            k = 0
            while k < steps:
                if k % every == 0 and k != blob_at:
                    blob, blob_at = sph.sph_get_state(ctx), k
                if len(dts) <= k // chunk:
                    dts.append(_cfl_dt_device(d, eos))
                dt = dts[k // chunk]
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                with torch.cuda.stream(stream):
                    e0.record(stream)
                    sph.sph_step(ctx, dt, min(chunk, steps - k))
                    e1.record(stream)
                try:
                    sph.sph_sync(ctx)
                except sph.SphError as e:
                    if e.status == 4 and cap < 1024:
                        cap *= 2
                        grown.append({"at_step": k, "max_neighbors": cap})
                        sph.sph_set_state(ctx, blob)
                        sph.sph_set_max_neighbors(ctx, cap)
                        k = blob_at
                        continue
                    err = str(e)
                    break
                torch.cuda.synchronize()
                ms += e0.elapsed_time(e1)
                k += min(chunk, steps - k)
                done = k
            f = d["flags"].cpu().numpy()
            flags[name] = f
            out[name] = {"steps_done": done, "error": err, "ms_per_step": ms / max(done, 1),
                         "capacity_retries": grown,
                         "yielded": int(((f & 1) != 0).sum()), "broken": int(((f & 2) != 0).sum())}
            sph.sph_free(ctx)
            del d
            torch.cuda.empty_cache()
            if name == "fp64":
                steps = done or steps
        diff = (flags["mixed"] ^ flags["fp64"]) & 3
        out.update({"particles": len(st["x"]), "crust_particles": int(crust.sum()), "steps": steps,
                    "dt_first_last_min": [dts[0], dts[-1], min(dts)],
                    "yield_flags_differ": int(((diff & 1) != 0).sum()),
                    "broken_flags_differ": int(((diff & 2) != 0).sum())})
        # the oracle-sized star of the same configuration: FP64 GPU vs oracle,
        # the same dt sequence (from the GPU state) on both
        k = args.oracle_steps
        s2, e2, m2, _ = I.star_state(20000, seed=7, **cfg)
        d = sph.device_state(s2, dev)
        torch.cuda.synchronize()
        ctx = sph.sph_init(d, e2, I.DEFAULT_MATERIAL, m2, sph.SPH_FP64, None,
                           stream=stream.cuda_stream)
        o = {kk: (None if v is None else np.array(v, copy=True)) for kk, v in s2.items()}
        r_or = None  # the oracle's rates carried across chunks, as the GPU's are
        t_or = 0.0
        for j in range(0, k, chunk):
            dt = _cfl_dt_device(d, e2)
            nst = min(chunk, k - j)
            with torch.cuda.stream(stream):
                sph.sph_step(ctx, dt, nst)
            sph.sph_sync(ctx)
            t0 = time.perf_counter()
            o, r_or = oracle.step(o, e2, I.DEFAULT_MATERIAL, m2, dt, nst, rates=r_or)
            t_or += time.perf_counter() - t0
        g = sph.to_numpy(d)
        sph.sph_free(ctx)
        out["oracle_2e4"] = {"steps": k, "oracle_s": t_or,
                             "yielded_gpu": int(((g["flags"] & 1) != 0).sum()),
                             "yielded_oracle": int(((o["flags"] & 1) != 0).sum()),
                             "broken_gpu": int(((g["flags"] & 2) != 0).sum()),
                             "broken_oracle": int(((o["flags"] & 2) != 0).sum()),
                             "flags_differ": int((g["flags"] != o["flags"]).sum()),
                             "max_rel_pos_diff": float(np.max(np.abs(g["x"] - o["x"])) /
                                                       np.max(np.abs(o["x"])))}
    print(json.dumps(out), flush=True)


def _rhs_only(tim, pairs_step):
    ms = (tim[10] / max(tim[11], 1) + tim[2] / max(tim[3], 1) + tim[0] / max(tim[1], 1))
    return {"ms": ms, "pairs_per_s": pairs_step / (ms * 1e-3) if ms > 0 else None,
            "sort_tree_ms": tim[6] / max(tim[7], 1), "lists_ms": tim[8] / max(tim[9], 1),
            "density_ms": tim[2] / max(tim[3], 1), "force_ms": tim[0] / max(tim[1], 1)}


def oracle_sample_rhs(st, eos, met, sample: int, seed: int):
    """Oracle rates of `sample` random particles (brute force over all)."""
    import oracle
    from paper_2107_07315_gb300 import inputs as I

    rng = np.random.default_rng(seed)
    ids = np.sort(rng.choice(len(st["x"]), size=sample, replace=False)).astype(np.int64)
    t0 = time.perf_counter()
    r = oracle.rhs(st, eos, I.DEFAULT_MATERIAL, met, subset=ids, scales=True)
    t1 = time.perf_counter()
    pairs = float(r["ncount"][ids].sum())
    return pairs, t1 - t0, ids, r


def oracle_full_rhs(st, eos, met):
    """Oracle right-hand side of every particle; returns (pairs, seconds, rates)."""
    import oracle
    from paper_2107_07315_gb300 import inputs as I

    t0 = time.perf_counter()
    r = oracle.rhs(st, eos, I.DEFAULT_MATERIAL, met, scales=True)
    t1 = time.perf_counter()
    return float(r["ncount"].sum()), t1 - t0, r


def cpu_baseline(st, eos, met, sample: int, min_seconds: float = 10.0):
    """The oracle timed on the host cores.

    sample <= 0: the full right-hand side of the star, repeated until at least
    min_seconds have passed (at most 4 times).  Its cost is nearly that of any
    sample, because the density of every neighbour of the sampled particles
    is needed.  sample > 0: one sampled right-hand side of that many particles.
    """
    import oracle

    if sample > 0:
        pairs, sec, ids, r = oracle_sample_rhs(st, eos, met, sample, 7)
        what = ("right-hand side of %d random particles of the %d-particle star "
                "(brute-force O(N^2) neighbour search over all particles, FP64), %.1f s"
                % (sample, len(st["x"]), sec))
    else:
        pairs, sec, reps = 0.0, 0.0, 0
        while reps < 4 and (reps == 0 or sec < min_seconds):
            p, t, r = oracle_full_rhs(st, eos, met)
            pairs, sec, reps = pairs + p, sec + t, reps + 1
        ids = np.arange(len(st["x"]), dtype=np.int64)
        what = ("full right-hand side of the %d-particle star, %d time(s) (brute-force O(N^2) "
                "neighbour search, FP64), %.1f s in total" % (len(st["x"]), reps, sec))
    return {"value": pairs / sec, "unit": "pairs/s", "cores": oracle.num_threads(),
            "kind": "oracle", "sample": what}, ids, r


def parity_errors(g, o, ids):
    """Max normalised error per field on the sampled particles:
    |q_gpu - q_oracle| / max(|q_oracle|, absolute-summand scale of q)."""
    sc = o["scale"]

    def err(qg, qo, s):
        d = np.abs(qg - qo)
        den = np.maximum(np.abs(qo), s)
        return float(np.max(np.where(den > 0, d / np.where(den > 0, den, 1.0),
                                     np.where(d == 0, 0.0, np.inf)))) if len(d) else 0.0

    e = {"D": err(g["D"][ids], o["D"][ids], sc["D"][ids]),
         "rho": err(g["rho"][ids], o["rho"][ids], 0.0),
         "a": max(err(g[k][ids], o[k][ids], sc["a"][ids]) for k in ("ax", "ay", "az")),
         "dudt": err(g["dudt"][ids], o["dudt"][ids], sc["du"][ids]),
         "drhodt": err(g["drhodt"][ids], o["drhodt"][ids], sc["drho"][ids])}
    sid = ids[sc["dS"][ids] > 0]
    if len(sid):
        e["deps"] = max(err(g["deps"][c][sid], o["deps"][c][sid], sc["eps"][sid]) for c in range(6))
        e["dS"] = max(err(g["dS"][c][sid], o["dS"][c][sid], sc["dS"][sid]) for c in range(6))
    e["neighbour_counts_equal"] = bool(np.array_equal(g["ncount"][ids], o["ncount"][ids]))
    e["particles"] = int(len(ids))
    e["solid_particles"] = int(len(sid))
    return e


def gpu_rates_at(st, eos, met, prec, dev, stream):
    """One right-hand side of the initial state through the C ABI (host copy)."""
    import torch

    from paper_2107_07315_gb300 import inputs as I
    from paper_2107_07315_gb300 import sph

    d = sph.device_state(st, dev)
    torch.cuda.synchronize()
    ctx = sph.sph_init(d, eos, I.DEFAULT_MATERIAL, met, prec, dict(h_nmin=55, h_nmax=65),
                       stream=stream.cuda_stream)
    rates = sph.alloc_rates(len(st["x"]), dev)
    torch.cuda.synchronize()
    sph.sph_rhs(ctx, rates)
    sph.sph_sync(ctx)
    out = sph.to_numpy(rates)
    sph.sph_free(ctx)
    return out


def time_steps(ctx, dt, steps, warmup, flush, stream):
    """Per-step CUDA-event time (ms) of `steps` KDK steps after `warmup`."""
    import torch

    from paper_2107_07315_gb300 import sph

    with torch.cuda.stream(stream):
        for _ in range(warmup):
            sph.sph_step(ctx, dt, 1)
    sph.sph_sync(ctx)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    p0 = sph.sph_stats(ctx)[1]
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for k in range(steps):
            flush.fill_(float(k))
            evs[k][0].record(stream)
            sph.sph_step(ctx, dt, 1)
            evs[k][1].record(stream)
    torch.cuda.synchronize()
    return float(sum(a.elapsed_time(b) for a, b in evs)), float(sph.sph_stats(ctx)[1] - p0)


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return None
    import oracle

    st, eos, met, _ = make_star(1, args.n)
    sample = args.cpu_sample
    n = len(st["x"])
    if sample <= 0:
        # one full right-hand side per step when the run fits in ~150 s; else a
        # particle sample (its cost is mostly the density of the sample's
        # neighbours, about 61 per particle, each summed over all particles)
        _, t_full, _ = oracle_full_rhs(st, eos, met)
        budget = 150.0 / max(args.steps, 1)
        if t_full > budget:
            sample = max(64, min(n, int(n / 61.0 * budget / t_full)))
    for k in range(max(args.warmup - 1, 0)):
        oracle_sample_rhs(st, eos, met, min(500, n), 100 + k)
    tot_p, tot_s = 0.0, 0.0
    for k in range(args.steps):
        # one step: the full right-hand side (or a sample of --cpu-sample particles)
        if sample > 0:
            p, s, _, _ = oracle_sample_rhs(st, eos, met, sample, 200 + k)
        else:
            p, s, _ = oracle_full_rhs(st, eos, met)
        tot_p += p
        tot_s += s
    v = tot_p / tot_s
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "pairs/s", "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": "TOV star, %d particles, FP64 CPU oracle right-hand side "
                                  "per step" % len(st["x"]),
                      "n_particles": len(st["x"])},
           "cpu_baseline": {"value": v, "unit": "pairs/s", "cores": oracle.num_threads(),
                            "kind": "oracle",
                            "sample": ("%d random particles per step" % sample if sample > 0
                                       else "full right-hand side per step")
                                      + ", brute-force O(N^2) neighbours, FP64"},
           "e2e": {"value": v, "unit": "pairs/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return out


def launch_shape(stats):
    """The launch shape sph_init chose (the search leaf of the candidate build,
    threads per particle of the exact screening and of the pair kernels, and
    whether screening and force run as one persistent launch) and the
    autotuner's per-launch times; the library's fixed default is a search
    leaf of one tree leaf (8 particles), 4 screening lanes, 8 pair lanes,
    separate launches."""
    src = {0: "fixed", 1: "autotuned", 2: "autotuned (process cache)"}[int(stats[20])]
    out = {"search_leaf_particles": 8 * int(stats[31]), "screen_lanes": int(stats[19]),
           "pair_lanes": int(stats[7]), "persistent_blocks": int(stats[25]), "source": src,
           "fixed_default": {"search_leaf_particles": 8, "screen_lanes": 4, "pair_lanes": 8,
                             "persistent": False}}
    if all(v > 0 for v in stats[28:31]):
        # one candidate-list build with search leaves of 8, 16 and 32 particles
        out["tuner_us_build"] = {"leaf_8": int(stats[28]) / 1e3, "leaf_16": int(stats[29]) / 1e3,
                                 "leaf_32": int(stats[30]) / 1e3}
    if stats[26] > 0 and stats[27] > 0:
        # screening + force of the chosen lanes: separate launches vs one persistent launch
        out["tuner_us_separate_vs_persistent"] = [int(stats[26]) / 1e3, int(stats[27]) / 1e3]
    t = [int(v) for v in stats[21:25]]
    if all(v > 0 for v in t):
        out["tuner_us_per_launch"] = {"screen_4": t[0] / 1e3, "screen_8": t[1] / 1e3,
                                      "pairs_4": t[2] / 1e3, "pairs_8": t[3] / 1e3}
        # screening + pair kernels of the chosen shape against the fixed one
        out["tuned_vs_fixed"] = (t[0] + t[3]) / (min(t[0], t[1]) + min(t[2], t[3]))
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--precision", choices=("mixed", "fp64"), default="mixed")
    ap.add_argument("--n", type=int, default=N_STAR)
    ap.add_argument("--workload", choices=("star", "ensemble", "relax"), default="star")
    ap.add_argument("--campaign", choices=("star1e6", "ensemble", "crust4e6"), default=None,
                    help="full-length paper-scale run instead of the benchmark line")
    ap.add_argument("--campaign-steps", type=int, default=0,
                    help="steps of the campaign (0: the configuration's own count)")
    ap.add_argument("--campaign-out", default="",
                    help="star1e6 campaign: also write the sampled series to this .npz file")
    ap.add_argument("--oracle-steps", type=int, default=200,
                    help="steps of the 2e4-particle oracle comparison in the crust4e6 campaign")
    ap.add_argument("--nstars", type=int, default=64)
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--cpu-sample", type=int, default=0,
                    help="oracle particle sample; 0 times the full right-hand side")
    ap.add_argument("--fp64-steps", type=int, default=5,
                    help="timed steps of the plain FP64 path on the same star (0: skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--count-solid", type=int, default=1)
    ap.add_argument("--skin", type=float, default=0.0,
                    help="candidate-list skin (0: library default 0.1; < 0: build every RHS)")
    ap.add_argument("--tune", type=int, default=1,
                    help="1: autotune the launch shape in sph_init (lane counts and the "
                         "persistent launch)")
    ap.add_argument("--persistent", type=int, default=0,
                    help="with --tune 0: 1 runs screening + force as one persistent launch")
    ap.add_argument("--mode-check", type=int, default=1,
                    help="also measure the mixed/FP64 speed-up at equal radial-mode accuracy")
    ap.add_argument("--sort-every", type=int, default=16,
                    help="curve sort every k steps (tree and exact lists every step; candidate "
                         "lists at the sorts and when stale)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.campaign:
        campaign(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
