"""Thin ctypes binding of libsph (include/sph.h).

Functions carry the C names and only marshal arguments: torch CUDA tensors
become device pointers, dicts become the ABI structs, non-OK statuses raise
SphError.  Every step of the computation runs in libsph's CUDA kernels; there
is no CPU path.  If libsph.so has not been built the import of the library
fails loudly.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# SPH_CHECKED=1 in the environment selects the bounds-checked build
LIB_PATH = os.path.join(_HERE, "libsph_checked.so" if os.environ.get("SPH_CHECKED") == "1"
                        else "libsph.so")

SPH_FP64 = 0
SPH_MIXED = 1

STATUS = {0: "SPH_OK", 1: "SPH_ERR_ARG", 2: "SPH_ERR_CUDA", 3: "SPH_ERR_OOM",
          4: "SPH_ERR_CAPACITY", 5: "SPH_ERR_TIMEOUT", 6: "SPH_ERR_NONFINITE",
          7: "SPH_ERR_BOUNDS", 8: "SPH_ERR_NODEVICE"}

# Every symbol include/sph.h declares.
EXPORTS = ("sph_init", "sph_rhs", "sph_step", "sph_sync", "sph_neighbors", "sph_totals",
           "sph_stats", "sph_timing", "sph_timing_read", "sph_state_size", "sph_get_state",
           "sph_set_state", "sph_free", "sph_last_error", "sph_neighbors_noalloc",
           "sph_set_external", "sph_relax_finish", "sph_set_wait_limit", "sph_peak_rates",
           "sph_totals_per_star", "sph_build_checked", "sph_checked_set_candidate",
           "sph_set_max_neighbors")


class SphError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__("%s: %s (%s)" % (where, STATUS.get(status, status), msg))
        self.status = status


_d = C.POINTER(C.c_double)
_u8 = C.POINTER(C.c_uint8)
_i32 = C.POINTER(C.c_int32)
_i64 = C.POINTER(C.c_int64)


class sph_particles(C.Structure):
    _fields_ = [("n", C.c_int64)] + [(k, C.c_void_p) for k in (
        "x", "y", "z", "vx", "vy", "vz", "u", "h", "m", "S", "type", "flags", "star", "mu", "Y0",
        "eps_break")]


class sph_eos(C.Structure):
    _fields_ = [("nstars", C.c_int32), ("K", _d), ("Gamma", _d), ("npieces", C.c_int32),
                ("rho_bound", _d), ("Gamma_above", _d)]


def _eos_struct(eos: dict, keep: list):
    """sph_eos from a dict (K, Gamma per star; optional piecewise rho_bound and
    Gamma_above of shape (nstars, npieces - 1))."""
    K, G = _f64(eos["K"]), _f64(eos["Gamma"])
    keep += [K, G]
    if eos.get("rho_bound") is None:
        return sph_eos(len(K), K.ctypes.data_as(_d), G.ctypes.data_as(_d), 0, None, None)
    rb = np.ascontiguousarray(np.asarray(eos["rho_bound"], np.float64).reshape(len(K), -1))
    ga = np.ascontiguousarray(np.asarray(eos["Gamma_above"], np.float64).reshape(len(K), -1))
    keep += [rb, ga]
    return sph_eos(len(K), K.ctypes.data_as(_d), G.ctypes.data_as(_d), rb.shape[1] + 1,
                   rb.ctypes.data_as(_d), ga.ctypes.data_as(_d))


class sph_material(C.Structure):
    _fields_ = [("alpha_av", C.c_double), ("beta_av", C.c_double), ("eta2", C.c_double),
                ("jaumann", C.c_int32), ("yield_mode", C.c_int32), ("break_stress", C.c_int32),
                ("break_zero_S", C.c_int32)]


class sph_metric(C.Structure):
    _fields_ = [("kind", C.c_int32), ("nstars", C.c_int32), ("nr", C.c_int32),
                ("pressure_form", C.c_int32)] + [(k, _d) for k in (
                    "r_max", "alpha", "dalpha", "psi4", "dpsi4", "M", "center")]


class sph_external(C.Structure):
    _fields_ = [("kind", C.c_int32), ("nstars", C.c_int32), ("nr", C.c_int32),
                ("reserved", C.c_int32)] + [(k, _d) for k in ("r_max", "g", "center", "r_wall")] + [
        ("k_wall", C.c_double), ("damping", C.c_double)]


class sph_rates(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in (
        "ax", "ay", "az", "dudt", "drhodt", "rho", "P", "D", "cs", "deps", "dR", "dS", "ncount")]


class sph_options(C.Structure):
    _fields_ = [("h_nmin", C.c_int32), ("h_nmax", C.c_int32), ("max_neighbors", C.c_int32),
                ("lanes_per_particle", C.c_int32), ("use_graph", C.c_int32),
                ("totals_every", C.c_int32), ("sort_every", C.c_int32), ("skin", C.c_double),
                ("screen_lanes", C.c_int32), ("persistent", C.c_int32),
                ("search_leaves", C.c_int32)]


_lib = None


def lib():
    """Load libsph.so (raises if it was not built; there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("%s is not built; run __graft_entry__.build()" % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        vp = C.c_void_p
        L.sph_init.argtypes = [C.POINTER(vp), C.POINTER(sph_particles), C.POINTER(sph_eos),
                               C.POINTER(sph_material), C.POINTER(sph_metric), C.c_int,
                               C.POINTER(sph_options), vp]
        L.sph_rhs.argtypes = [vp, C.POINTER(sph_rates)]
        L.sph_step.argtypes = [vp, C.c_double, C.c_int32]
        L.sph_sync.argtypes = [vp]
        L.sph_set_wait_limit.argtypes = [vp, C.c_int32]
        L.sph_peak_rates.argtypes = [_d]
        L.sph_totals_per_star.argtypes = [vp, _d, C.c_int32]
        L.sph_neighbors.argtypes = [vp, vp, vp, C.c_int64]
        L.sph_totals.argtypes = [vp, _d]
        L.sph_stats.argtypes = [vp, _i64]
        L.sph_timing.argtypes = [vp, C.c_int32]
        L.sph_timing_read.argtypes = [vp, _d]
        L.sph_state_size.argtypes = [vp, _i64]
        L.sph_get_state.argtypes = [vp, vp, C.c_int64]
        L.sph_set_state.argtypes = [vp, vp, C.c_int64]
        L.sph_free.argtypes = [vp]
        L.sph_free.restype = None
        L.sph_neighbors_noalloc.argtypes = [C.c_int64, vp, vp, vp, vp, vp, vp, C.c_int64, vp]
        L.sph_set_external.argtypes = [vp, C.POINTER(sph_external)]
        L.sph_relax_finish.argtypes = [vp, C.POINTER(sph_eos)]
        L.sph_last_error.restype = C.c_char_p
        L.sph_build_checked.argtypes = []
        L.sph_set_max_neighbors.argtypes = [vp, C.c_int32]
        L.sph_checked_set_candidate.argtypes = [vp, C.c_int64, C.c_int32, C.c_int32]
        for f in EXPORTS:
            if f not in ("sph_free", "sph_last_error"):
                getattr(L, f).restype = C.c_int
        _lib = L
    return _lib


def sph_last_error() -> str:
    return lib().sph_last_error().decode()


def _check(st: int, where: str):
    if st != 0:
        raise SphError(st, where, sph_last_error())


def _ptr(t):
    if t is None:
        return None
    return C.c_void_p(t.data_ptr())


class SphCtx:
    """Handle of an sph_ctx; keeps the bound tensors alive."""

    def __init__(self, handle, n, keep):
        self.handle = handle
        self.n = n
        self._keep = keep

    def __del__(self):
        try:
            if self.handle is not None:
                lib().sph_free(self.handle)
        except Exception:
            pass
        self.handle = None


PARTICLE_KEYS = ("x", "y", "z", "vx", "vy", "vz", "u", "h", "m", "S", "type", "flags", "star",
                 "mu", "Y0", "eps_break")


def device_state(state: dict, device="cuda"):
    """Copy a numpy particle state to contiguous device tensors."""
    import torch

    out = {}
    for k in PARTICLE_KEYS:
        v = state.get(k)
        if v is None:
            out[k] = None
            continue
        a = np.ascontiguousarray(v)
        if k in ("type", "flags"):
            a = a.astype(np.uint8)
        elif k == "star":
            a = a.astype(np.int32)
        else:
            a = a.astype(np.float64)
        out[k] = torch.from_numpy(a).to(device).contiguous()
    return out


# Fields a step changes, first in the packed layout so that one copy moves them.
# With the material option break_zero_S = 1 a step also zeroes mu of particles
# that break; such callers move mu as well.
STEP_KEYS = ("x", "y", "z", "vx", "vy", "vz", "u", "h", "S", "flags")


def device_state_packed(state: dict, device="cuda"):
    """Like device_state, but every field is a view into one device buffer.

    The fields a step changes (STEP_KEYS) come first, each at a 256-byte
    aligned offset, so a caller that keeps the state on the host can move a
    step's inputs and results with one copy each way.  Returns (fields,
    buffer, step_bytes): the field views (as device_state), the uint8 buffer
    and the length of its leading step part.
    """
    import torch

    arrays = {}
    for k in PARTICLE_KEYS:
        v = state.get(k)
        if v is None:
            continue
        a = np.ascontiguousarray(v)
        if k in ("type", "flags"):
            a = a.astype(np.uint8)
        elif k == "star":
            a = a.astype(np.int32)
        else:
            a = a.astype(np.float64)
        arrays[k] = a
    order = [k for k in STEP_KEYS if k in arrays] + [k for k in PARTICLE_KEYS
                                                      if k in arrays and k not in STEP_KEYS]
    offs, pos = {}, 0
    for k in order:
        offs[k] = pos
        pos = (pos + arrays[k].nbytes + 255) // 256 * 256
    last = [k for k in order if k in STEP_KEYS][-1]
    step_bytes = offs[last] + arrays[last].nbytes
    host = np.zeros(max(pos, 1), np.uint8)
    for k in order:
        host[offs[k]:offs[k] + arrays[k].nbytes] = arrays[k].reshape(-1).view(np.uint8)
    buf = torch.from_numpy(host).to(device)
    dtypes = {np.dtype(np.float64): torch.float64, np.dtype(np.uint8): torch.uint8,
              np.dtype(np.int32): torch.int32}
    fields = {k: None for k in PARTICLE_KEYS}
    for k in order:
        a = arrays[k]
        fields[k] = buf[offs[k]:offs[k] + a.nbytes].view(dtypes[a.dtype]).view(a.shape)
    return fields, buf, step_bytes


def alloc_rates(n: int, device="cuda"):
    import torch

    r = {k: torch.zeros(n, dtype=torch.float64, device=device)
         for k in ("ax", "ay", "az", "dudt", "drhodt", "rho", "P", "D", "cs")}
    r["deps"] = torch.zeros((6, n), dtype=torch.float64, device=device)
    r["dR"] = torch.zeros((3, n), dtype=torch.float64, device=device)
    r["dS"] = torch.zeros((6, n), dtype=torch.float64, device=device)
    r["ncount"] = torch.zeros(n, dtype=torch.int32, device=device)
    return r


def to_numpy(d: dict) -> dict:
    return {k: (None if v is None else v.detach().cpu().numpy()) for k, v in d.items()}


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).ravel())


def sph_init(particles: dict, eos: dict, material: dict, metric=None, precision=SPH_MIXED,
             options=None, stream=None) -> SphCtx:
    """Bind device particle tensors (see device_state) and create a context."""
    L = lib()
    n = int(particles["x"].numel())
    p = sph_particles(n, *[_ptr(particles.get(k)) for k in PARTICLE_KEYS])
    keep = [particles]
    e = _eos_struct(eos, keep)
    m = sph_material(float(material.get("alpha_av", 1.0)), float(material.get("beta_av", 2.0)),
                     float(material.get("eta2", 0.01)), int(material.get("jaumann", 0)),
                     int(material.get("yield_mode", 0)), int(material.get("break_stress", 0)),
                     int(material.get("break_zero_S", 0)))
    gp = None
    if metric is not None and int(metric.get("kind", 0)) == 1:
        arrs = {k: _f64(metric[k]) for k in ("r_max", "alpha", "dalpha", "psi4", "dpsi4", "M",
                                             "center")}
        keep.append(arrs)
        g = sph_metric(1, len(arrs["r_max"]), int(metric["nr"]), int(metric.get("pressure_form", 0)),
                       *[arrs[k].ctypes.data_as(_d) for k in ("r_max", "alpha", "dalpha", "psi4",
                                                               "dpsi4", "M", "center")])
        gp = C.byref(g)
    o = None
    if options is not None:
        o = sph_options(int(options.get("h_nmin", 0)), int(options.get("h_nmax", 0)),
                        int(options.get("max_neighbors", 0)),
                        int(options.get("lanes_per_particle", 0)), int(options.get("use_graph", 1)),
                        int(options.get("totals_every", 0)), int(options.get("sort_every", 0)),
                        float(options.get("skin", 0.0)), int(options.get("screen_lanes", 0)),
                        int(options.get("persistent", 0)), int(options.get("search_leaves", 0)))
    if stream is None:
        import torch

        stream = torch.cuda.current_stream().cuda_stream
    h = C.c_void_p()
    _check(L.sph_init(C.byref(h), C.byref(p), C.byref(e), C.byref(m), gp, int(precision),
                      C.byref(o) if o is not None else None, C.c_void_p(stream)), "sph_init")
    return SphCtx(h, n, keep)


def sph_rhs(ctx: SphCtx, rates: dict) -> None:
    r = sph_rates(*[_ptr(rates[k]) for k in ("ax", "ay", "az", "dudt", "drhodt", "rho", "P", "D",
                                             "cs", "deps", "dR", "dS", "ncount")])
    _check(lib().sph_rhs(ctx.handle, C.byref(r)), "sph_rhs")


def sph_step(ctx: SphCtx, dt: float, nsteps: int = 1) -> None:
    _check(lib().sph_step(ctx.handle, float(dt), int(nsteps)), "sph_step")


def sph_set_external(ctx: SphCtx, external) -> None:
    """External relaxation field (dict with nr, r_max, g, center, r_wall, k_wall,
    damping; see inputs.relax_external), or None to switch it off."""
    if external is None or int(external.get("kind", 1)) == 0:
        _check(lib().sph_set_external(ctx.handle, None), "sph_set_external")
        return
    arrs = {k: _f64(external[k]) for k in ("r_max", "g", "center", "r_wall")}
    x = sph_external(1, len(arrs["r_max"]), int(external["nr"]), 0,
                     *[arrs[k].ctypes.data_as(_d) for k in ("r_max", "g", "center", "r_wall")],
                     float(external["k_wall"]), float(external["damping"]))
    _check(lib().sph_set_external(ctx.handle, C.byref(x)), "sph_set_external")


def sph_relax_finish(ctx: SphCtx, eos: dict) -> None:
    """Modification step after a relaxation: new EoS, u from the density."""
    keep: list = []
    e = _eos_struct(eos, keep)
    _check(lib().sph_relax_finish(ctx.handle, C.byref(e)), "sph_relax_finish")


def sph_sync(ctx: SphCtx) -> None:
    _check(lib().sph_sync(ctx.handle), "sph_sync")


def sph_peak_rates() -> dict:
    """Measured FP32/FP64 FMA rates (TFLOP/s) and SM count of the current device."""
    out = np.zeros(4, np.float64)
    _check(lib().sph_peak_rates(out.ctypes.data_as(_d)), "sph_peak_rates")
    return {"fp32_tflops": float(out[0]), "fp64_tflops": float(out[1]), "sms": int(out[2])}


def sph_set_max_neighbors(ctx: SphCtx, max_neighbors: int) -> None:
    _check(lib().sph_set_max_neighbors(ctx.handle, int(max_neighbors)), "sph_set_max_neighbors")


def sph_build_checked() -> bool:
    return bool(lib().sph_build_checked())


def sph_checked_set_candidate(ctx: SphCtx, slot: int, k: int, value: int) -> None:
    _check(lib().sph_checked_set_candidate(ctx.handle, int(slot), int(k), int(value)),
           "sph_checked_set_candidate")


def sph_set_wait_limit(ctx: SphCtx, polls: int) -> None:
    _check(lib().sph_set_wait_limit(ctx.handle, int(polls)), "sph_set_wait_limit")


def sph_neighbors(ctx: SphCtx, offsets, idx, cap: int) -> None:
    _check(lib().sph_neighbors(ctx.handle, _ptr(offsets), _ptr(idx), int(cap)), "sph_neighbors")


def sph_totals(ctx: SphCtx) -> np.ndarray:
    out = np.zeros(16, np.float64)
    _check(lib().sph_totals(ctx.handle, out.ctypes.data_as(_d)), "sph_totals")
    return out


def sph_totals_per_star(ctx: SphCtx, nstars: int) -> np.ndarray:
    """FP64 totals of each star: array [nstars, 16] (columns as sph_totals)."""
    out = np.zeros((nstars, 16), np.float64)
    _check(lib().sph_totals_per_star(ctx.handle, out.ctypes.data_as(_d), int(nstars)),
           "sph_totals_per_star")
    return out


def sph_stats(ctx: SphCtx) -> np.ndarray:
    out = np.zeros(32, np.int64)
    _check(lib().sph_stats(ctx.handle, out.ctypes.data_as(_i64)), "sph_stats")
    return out


def sph_timing(ctx: SphCtx, enable: bool) -> None:
    _check(lib().sph_timing(ctx.handle, int(bool(enable))), "sph_timing")


def sph_timing_read(ctx: SphCtx) -> np.ndarray:
    out = np.zeros(12, np.float64)
    _check(lib().sph_timing_read(ctx.handle, out.ctypes.data_as(_d)), "sph_timing_read")
    return out


def sph_state_size(ctx: SphCtx) -> int:
    b = C.c_int64(0)
    _check(lib().sph_state_size(ctx.handle, C.byref(b)), "sph_state_size")
    return int(b.value)


def sph_get_state(ctx: SphCtx) -> np.ndarray:
    buf = np.zeros(sph_state_size(ctx), np.uint8)
    _check(lib().sph_get_state(ctx.handle, buf.ctypes.data_as(C.c_void_p), len(buf)),
           "sph_get_state")
    return buf


def sph_set_state(ctx: SphCtx, buf: np.ndarray) -> None:
    buf = np.ascontiguousarray(buf, dtype=np.uint8)
    _check(lib().sph_set_state(ctx.handle, buf.ctypes.data_as(C.c_void_p), len(buf)),
           "sph_set_state")


def sph_neighbors_noalloc(n: int, x, y, z, h, offsets, idx, cap: int, stream=None) -> None:
    """Neighbour CSR of one star with no context and no device allocation
    (for callers that cannot call cudaMalloc); n <= 16384."""
    _check(lib().sph_neighbors_noalloc(int(n), _ptr(x), _ptr(y), _ptr(z), _ptr(h),
                                       _ptr(offsets), _ptr(idx), int(cap),
                                       C.c_void_p(stream) if stream else None),
           "sph_neighbors_noalloc")


def sph_free(ctx: SphCtx) -> None:
    if ctx.handle is not None:
        lib().sph_free(ctx.handle)
        ctx.handle = None


def neighbors(ctx: SphCtx, device="cuda"):
    """Neighbour CSR of the last right-hand side as numpy (offsets, idx)."""
    import torch

    offs = torch.zeros(ctx.n + 1, dtype=torch.int64, device=device)
    cap = 1
    idx = torch.zeros(cap, dtype=torch.int32, device=device)
    torch.cuda.synchronize()
    try:
        sph_neighbors(ctx, offs, idx, 0)
    except SphError as e:
        if e.status != 4:
            raise
    total = int(offs[-1].item())
    idx = torch.zeros(max(total, 1), dtype=torch.int32, device=device)
    torch.cuda.synchronize()
    sph_neighbors(ctx, offs, idx, total)
    return offs.cpu().numpy(), idx[:total].cpu().numpy()
