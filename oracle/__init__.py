"""FP64 CPU oracle for the SPH right-hand side of arXiv 2107.07315 (Sec. I.B, I.C).

TEST INFRASTRUCTURE ONLY.  The test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product library
never imports, links or executes anything in this directory, and this module
imports nothing from the product package.

The arithmetic lives in ``sph_oracle.c`` (plain C, FP64, brute-force O(N^2)
neighbours, compiled with ``-ffp-contract=off``).  This module compiles it,
loads it with ctypes and marshals numpy arrays.  A particle state is a dict of
numpy arrays in caller order:

    x y z vx vy vz u h m mu Y0 eps_break : float64 [n]
    S : float64 [6, n]  (xx, yy, zz, xy, xz, yz)
    type, flags : uint8 [n]   star : int32 [n] or None

``eos`` is ``{"K": [nstars], "Gamma": [nstars]}``; ``material`` holds
``alpha_av beta_av eta2 jaumann yield_mode break_stress break_zero_S``;
``metric`` is None or ``{"kind": 1, "nr", "r_max", "alpha", "dalpha",
"psi4", "dpsi4", "M", "center"[, "pressure_form"]}`` with tables shaped
[nstars, nr].
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sph_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_d = C.POINTER(C.c_double)
_u8 = C.POINTER(C.c_uint8)
_i32 = C.POINTER(C.c_int32)
_i64 = C.POINTER(C.c_int64)


class _State(C.Structure):
    _fields_ = [("n", C.c_int64)] + [(k, _d) for k in
               ("x", "y", "z", "vx", "vy", "vz", "u", "h", "m", "S")] + [
        ("type", _u8), ("flags", _u8), ("star", _i32),
        ("mu", _d), ("Y0", _d), ("eps_break", _d)]


class _Eos(C.Structure):
    _fields_ = [("nstars", C.c_int32), ("K", _d), ("Gamma", _d), ("npieces", C.c_int32),
                ("rho_bound", _d), ("Gamma_above", _d)]


class _Material(C.Structure):
    _fields_ = [("alpha_av", C.c_double), ("beta_av", C.c_double), ("eta2", C.c_double),
                ("jaumann", C.c_int32), ("yield_mode", C.c_int32),
                ("break_stress", C.c_int32), ("break_zero_S", C.c_int32)]


class _Metric(C.Structure):
    _fields_ = [("kind", C.c_int32), ("nstars", C.c_int32), ("nr", C.c_int32),
                ("pressure_form", C.c_int32), ("r_max", _d), ("alpha", _d), ("dalpha", _d), ("psi4", _d),
                ("dpsi4", _d), ("M", _d), ("center", _d)]


class _External(C.Structure):
    _fields_ = [("kind", C.c_int32), ("nstars", C.c_int32), ("nr", C.c_int32),
                ("r_max", _d), ("g", _d), ("center", _d), ("r_wall", _d),
                ("k_wall", C.c_double), ("damping", C.c_double)]


class _Scales(C.Structure):
    _fields_ = [(k, _d) for k in ("a", "du", "drho", "D", "eps", "dS")]


class _Rates(C.Structure):
    _fields_ = [(k, _d) for k in ("ax", "ay", "az", "dudt", "drhodt", "rho", "P", "D", "cs",
                                  "deps", "dR", "dS")] + [("ncount", _i32)]


def build(force: bool = False) -> str:
    """Compile sph_oracle.c into liboracle.so next to it (gcc, OpenMP)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
           "-shared", "-std=c99", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _configure(L):
    """Declare argument and result types of the oracle's exported functions."""
    L.ora_kernel_W.restype = C.c_double
    L.ora_kernel_W.argtypes = [C.c_double, C.c_double]
    L.ora_kernel_dWdr.restype = C.c_double
    L.ora_kernel_dWdr.argtypes = [C.c_double, C.c_double]
    L.ora_yield_factor.restype = C.c_double
    L.ora_yield_factor.argtypes = [_d, C.c_double, C.c_int]
    L.ora_sym_eigvals.argtypes = [_d, _d]
    L.ora_breaks.restype = C.c_int
    L.ora_breaks.argtypes = [_d, C.c_double, C.c_double, C.c_double, C.c_double, C.c_int]
    L.ora_rhs.restype = C.c_int
    L.ora_step.restype = C.c_int
    L.ora_metric_eval.argtypes = [C.POINTER(_Metric), C.c_int, C.c_double, C.c_double,
                                  C.c_double, _d, _d, _d, _d]
    L.ora_tejeda_accel.argtypes = [C.c_double, _d, C.c_double, _d, _d, _d,
                                   C.c_double, _d]
    L.ora_eos_eval.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int,
                               _d, _d, _d, _d]
    L.ora_external_accel.argtypes = [C.POINTER(_External), C.c_int, C.c_double,
                                     C.c_double, C.c_double, _d, _d, _d]
    L.ora_eos_eval_star.argtypes = [C.POINTER(_Eos), C.c_int, C.c_double, C.c_int,
                                    _d, _d, _d, _d]
    L.ora_num_threads.restype = C.c_int
    L.ora_set_threads.argtypes = [C.c_int]
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _configure(C.CDLL(_LIB))
        return _lib


class mutant:
    """A copy of the oracle with planted mistakes, for tests that show a pin
    detects them.  ``edits`` is a list of (old, new) source snippets; each
    ``old`` must occur exactly once in sph_oracle.c.  Inside ``with
    mutant(edits, workdir):`` every function of this module runs the mutated
    copy; the real oracle is restored on exit.  The mutated library lives in
    ``workdir`` (a temporary directory of the caller)."""

    def __init__(self, edits, workdir: str):
        src = open(_SRC).read()
        for old, new in edits:
            if src.count(old) != 1:
                raise ValueError("mutation target must occur once: %r" % old)
            src = src.replace(old, new)
        tag = "%08x" % (abs(hash(tuple(edits))) & 0xffffffff)
        csrc = os.path.join(workdir, "oracle_mutant_%s.c" % tag)
        so = os.path.join(workdir, "liboracle_mutant_%s.so" % tag)
        with open(csrc, "w") as f:
            f.write(src)
        subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
                        "-shared", "-std=c99", "-o", so, csrc, "-lm"], check=True)
        self._lib = _configure(C.CDLL(so))
        self._saved = None

    def __enter__(self):
        global _lib
        lib()
        with _lock:
            self._saved, _lib = _lib, self._lib
        return self

    def __exit__(self, *exc):
        global _lib
        with _lock:
            _lib = self._saved
        return False


def _p(a, t=_d):
    return a.ctypes.data_as(t) if a is not None else None


_F64 = ("x", "y", "z", "vx", "vy", "vz", "u", "h", "m", "mu", "Y0", "eps_break")


def _prep_state(st: dict) -> dict:
    """Contiguous copies in the dtypes the C code expects."""
    n = len(st["x"])
    out = {k: np.ascontiguousarray(st[k], dtype=np.float64) for k in _F64}
    out["S"] = np.ascontiguousarray(np.asarray(st["S"], dtype=np.float64).reshape(6, n))
    out["type"] = np.ascontiguousarray(st["type"], dtype=np.uint8)
    out["flags"] = np.ascontiguousarray(st.get("flags", np.zeros(n, np.uint8)), dtype=np.uint8)
    star = st.get("star")
    out["star"] = None if star is None else np.ascontiguousarray(star, dtype=np.int32)
    return out


def _cstate(s: dict) -> _State:
    n = len(s["x"])
    return _State(n, *[_p(s[k]) for k in ("x", "y", "z", "vx", "vy", "vz", "u", "h", "m", "S")],
                  _p(s["type"], _u8), _p(s["flags"], _u8), _p(s["star"], _i32),
                  _p(s["mu"]), _p(s["Y0"]), _p(s["eps_break"]))


def _ceos(eos: dict, keep: list) -> _Eos:
    """ctypes view of an EoS dict: K, Gamma per star; optional piecewise
    rho_bound and Gamma_above of shape (nstars, npieces - 1)."""
    K = np.ascontiguousarray(eos["K"], dtype=np.float64).ravel()
    G = np.ascontiguousarray(eos["Gamma"], dtype=np.float64).ravel()
    keep += [K, G]
    if eos.get("rho_bound") is None:
        return _Eos(len(K), _p(K), _p(G), 0, None, None)
    rb = np.ascontiguousarray(eos["rho_bound"], dtype=np.float64).reshape(len(K), -1)
    ga = np.ascontiguousarray(eos["Gamma_above"], dtype=np.float64).reshape(len(K), -1)
    keep += [rb, ga]
    return _Eos(len(K), _p(K), _p(G), rb.shape[1] + 1, _p(rb), _p(ga))


def _cmat(mat: dict) -> _Material:
    return _Material(float(mat.get("alpha_av", 1.0)), float(mat.get("beta_av", 2.0)),
                     float(mat.get("eta2", 0.01)), int(mat.get("jaumann", 0)),
                     int(mat.get("yield_mode", 0)), int(mat.get("break_stress", 0)),
                     int(mat.get("break_zero_S", 0)))


def _cmetric(g, keep: list):
    if g is None or int(g.get("kind", 0)) == 0:
        return None
    arrs = {}
    for k in ("r_max", "alpha", "dalpha", "psi4", "dpsi4", "M", "center"):
        arrs[k] = np.ascontiguousarray(g[k], dtype=np.float64).ravel()
    keep.append(arrs)
    nstars = len(arrs["r_max"])
    return _Metric(1, nstars, int(g["nr"]), int(g.get("pressure_form", 0)), *[_p(arrs[k]) for k in
                   ("r_max", "alpha", "dalpha", "psi4", "dpsi4", "M", "center")])


def _cexternal(e, keep: list):
    """ctypes view of an external relaxation field dict (None: no field)."""
    if e is None or int(e.get("kind", 1)) == 0:
        return None
    arrs = {k: np.ascontiguousarray(e[k], dtype=np.float64).ravel()
            for k in ("r_max", "g", "center", "r_wall")}
    keep.append(arrs)
    return _External(1, len(arrs["r_max"]), int(e["nr"]), _p(arrs["r_max"]), _p(arrs["g"]),
                     _p(arrs["center"]), _p(arrs["r_wall"]), float(e["k_wall"]),
                     float(e["damping"]))


def external_accel(external: dict, star: int, x: float, y: float, z: float, v) -> tuple:
    """External relaxation acceleration (vector, magnitude) at one point."""
    keep: list = []
    ce = _cexternal(external, keep)
    vv = np.ascontiguousarray(v, dtype=np.float64)
    acc = np.zeros(3, np.float64)
    mag = np.zeros(1, np.float64)
    lib().ora_external_accel(C.byref(ce) if ce is not None else None, int(star), float(x),
                             float(y), float(z), _p(vv), _p(acc), _p(mag))
    return acc, float(mag[0])


_RATE_KEYS = ("ax", "ay", "az", "dudt", "drhodt", "rho", "P", "D", "cs")


def _alloc_rates(n: int) -> dict:
    r = {k: np.zeros(n, np.float64) for k in _RATE_KEYS}
    r["deps"] = np.zeros((6, n), np.float64)
    r["dR"] = np.zeros((3, n), np.float64)
    r["dS"] = np.zeros((6, n), np.float64)
    r["ncount"] = np.zeros(n, np.int32)
    return r


def _crates(r: dict) -> _Rates:
    return _Rates(*[_p(r[k]) for k in _RATE_KEYS + ("deps", "dR", "dS")],
                  _p(r["ncount"], _i32))


def set_threads(nt: int) -> None:
    lib().ora_set_threads(int(nt))


def num_threads() -> int:
    return int(lib().ora_num_threads())


def rhs(state: dict, eos: dict, material: dict, metric=None, subset=None,
        v=None, S=None, scales: bool = False, external=None) -> dict:
    """Rates of the full RHS (Eqs. solid1-solid6 + background force).

    ``subset``: optional int64 array of particle ids; only their rates are
    computed (other entries stay zero), using brute force over all particles.
    ``v`` (3 x n) and ``S`` (6 x n) override the state's velocity and stress.
    ``scales``: also return r["scale"], the absolute-summand magnitudes
    (keys a, du, drho, D, eps, dS) for cancellation-aware comparisons.
    """
    L = lib()
    s = _prep_state(state)
    n = len(s["x"])
    keep: list = []
    cs = _cstate(s)
    if v is not None:
        v = np.ascontiguousarray(v, dtype=np.float64).reshape(3, n)
        vx, vy, vz = v[0], v[1], v[2]
    else:
        vx, vy, vz = s["vx"], s["vy"], s["vz"]
    Sarr = s["S"] if S is None else np.ascontiguousarray(S, dtype=np.float64).reshape(6, n)
    ce = _ceos(eos, keep)
    cm = _cmat(material)
    cg = _cmetric(metric, keep)
    cx = _cexternal(external, keep)
    r = _alloc_rates(n)
    cr = _crates(r)
    if subset is not None:
        sub = np.ascontiguousarray(subset, dtype=np.int64)
        sp, ns = _p(sub, _i64), len(sub)
    else:
        sub, sp, ns = None, None, 0
    sc = None
    if scales:
        sc_arr = {k: np.zeros(n, np.float64) for k in ("a", "du", "drho", "D", "eps", "dS")}
        sc = _Scales(*[_p(sc_arr[k]) for k in ("a", "du", "drho", "D", "eps", "dS")])
    rc = L.ora_rhs(C.byref(cs), _p(vx), _p(vy), _p(vz), _p(Sarr), C.byref(ce), C.byref(cm),
                   C.byref(cg) if cg is not None else None,
                   C.byref(cx) if cx is not None else None, sp, C.c_int64(ns), C.byref(cr),
                   C.byref(sc) if sc is not None else None)
    if rc != 0:
        raise MemoryError("oracle rhs failed")
    if scales:
        r["scale"] = sc_arr
    return r


def neighbors(state: dict, subset=None):
    """Brute-force neighbour CSR (ascending ids): returns (offsets, idx)."""
    L = lib()
    s = _prep_state(state)
    cs = _cstate(s)
    if subset is not None:
        sub = np.ascontiguousarray(subset, dtype=np.int64)
        sp, ns = _p(sub, _i64), len(sub)
    else:
        sub, sp, ns = None, None, len(s["x"])
    cnt = np.zeros(ns, np.int64)
    L.ora_neighbor_counts(C.byref(cs), sp, C.c_int64(ns if sub is not None else 0), _p(cnt, _i64))
    offs = np.zeros(ns + 1, np.int64)
    np.cumsum(cnt, out=offs[1:])
    idx = np.zeros(max(int(offs[-1]), 1), np.int64)
    L.ora_neighbor_fill(C.byref(cs), sp, C.c_int64(ns if sub is not None else 0),
                        _p(offs, _i64), _p(idx, _i64))
    return offs, idx[: offs[-1]]


def step(state: dict, eos: dict, material: dict, metric, dt: float, nsteps: int,
         h_nmin: int = 0, h_nmax: int = 0, rates=None, external=None):
    """Advance ``nsteps`` leapfrog steps; returns (new_state, rates).

    ``rates`` from a previous call continue the scheme exactly; when None the
    rates are first evaluated at the given state.
    """
    L = lib()
    s = _prep_state(state)
    s = {k: (None if v is None else v.copy()) for k, v in s.items()}
    n = len(s["x"])
    keep: list = []
    cs = _cstate(s)
    ce = _ceos(eos, keep)
    cm = _cmat(material)
    cg = _cmetric(metric, keep)
    cx = _cexternal(external, keep)
    if rates is None:
        r, have = _alloc_rates(n), 0
    else:
        r = {k: np.array(v, copy=True) for k, v in rates.items()}
        have = 1
    cr = _crates(r)
    rc = L.ora_step(C.byref(cs), C.byref(ce), C.byref(cm),
                    C.byref(cg) if cg is not None else None,
                    C.byref(cx) if cx is not None else None, C.c_double(dt),
                    C.c_int32(nsteps), C.c_int32(h_nmin), C.c_int32(h_nmax), C.c_int32(have),
                    C.byref(cr))
    if rc != 0:
        raise MemoryError("oracle step failed")
    return s, r


def totals(state: dict, ncount=None) -> np.ndarray:
    L = lib()
    s = _prep_state(state)
    cs = _cstate(s)
    out = np.zeros(16, np.float64)
    nc = None if ncount is None else np.ascontiguousarray(ncount, dtype=np.int32)
    L.ora_totals(C.byref(cs), _p(nc, _i32), _p(out))
    return out


def kernel_W(r: float, h: float) -> float:
    return float(lib().ora_kernel_W(float(r), float(h)))


def kernel_dWdr(r: float, h: float) -> float:
    return float(lib().ora_kernel_dWdr(float(r), float(h)))


def yield_factor(s6, Y0: float, yield_mode: int = 0) -> float:
    a = np.ascontiguousarray(s6, dtype=np.float64)
    return float(lib().ora_yield_factor(_p(a), float(Y0), int(yield_mode)))


def sym_eigvals(s6) -> np.ndarray:
    a = np.ascontiguousarray(s6, dtype=np.float64)
    ev = np.zeros(3, np.float64)
    lib().ora_sym_eigvals(_p(a), _p(ev))
    return ev


def breaks(s6, P: float, Gamma: float, mu: float, eps_break: float, break_stress: int = 0) -> bool:
    a = np.ascontiguousarray(s6, dtype=np.float64)
    return bool(lib().ora_breaks(_p(a), float(P), float(Gamma), float(mu), float(eps_break),
                                 int(break_stress)))


def eos_eval(K: float, Gamma: float, rho: float, relativistic: bool):
    o = [np.zeros(1) for _ in range(4)]
    lib().ora_eos_eval(float(K), float(Gamma), float(rho), int(relativistic), *[_p(a) for a in o])
    return tuple(float(a[0]) for a in o)  # P, u, dP/drho, c_s


def eos_eval_star(eos: dict, star: int, rho: float, relativistic: bool):
    """(P, u, dP/drho, c_s) of star `star` at rho, with any number of pieces."""
    keep: list = []
    ce = _ceos(eos, keep)
    o = [np.zeros(1) for _ in range(4)]
    lib().ora_eos_eval_star(C.byref(ce), int(star), float(rho), int(relativistic),
                            *[_p(a) for a in o])
    return tuple(float(a[0]) for a in o)


def metric_eval(metric: dict, star: int, x: float, y: float, z: float):
    keep: list = []
    cg = _cmetric(metric, keep)
    ga, gq = np.zeros(3), np.zeros(3)
    al, q = np.zeros(1), np.zeros(1)
    lib().ora_metric_eval(C.byref(cg), int(star), float(x), float(y), float(z),
                          _p(al), _p(ga), _p(q), _p(gq))
    return float(al[0]), ga, float(q[0]), gq


def tejeda_accel(alpha, grad_alpha, psi4, grad_psi4, xdot, gradP_over, dtP_over) -> np.ndarray:
    ga = np.ascontiguousarray(grad_alpha, dtype=np.float64)
    gq = np.ascontiguousarray(grad_psi4, dtype=np.float64)
    xd = np.ascontiguousarray(xdot, dtype=np.float64)
    gp = np.ascontiguousarray(gradP_over, dtype=np.float64)
    acc = np.zeros(3)
    lib().ora_tejeda_accel(float(alpha), _p(ga), float(psi4), _p(gq), _p(xd), _p(gp),
                           float(dtP_over), _p(acc))
    return acc
