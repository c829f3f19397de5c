"""CPU checks of the C-ABI boundary: the library builds, loads and exports
every entry point include/sph.h declares; without a GPU it refuses cleanly;
the product package never imports the oracle."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sph.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sph_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2107_07315_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_lists_expected_entry_points():
    from paper_2107_07315_gb300 import sph

    assert _declared() == sorted(sph.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_no_device_is_reported_without_gpu(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import numpy as np

    from paper_2107_07315_gb300 import sph

    # host numpy pointers stand in for device buffers: sph_init must refuse
    # before touching them
    n = 4
    arrs = {k: np.zeros(n) for k in ("x", "y", "z", "vx", "vy", "vz", "u", "h", "m")}
    S = np.zeros(6 * n)
    ty = np.zeros(n, np.uint8)
    fl = np.zeros(n, np.uint8)
    vp = lambda a: ctypes.c_void_p(a.ctypes.data)  # noqa: E731
    p = sph.sph_particles(n, *[vp(arrs[k]) for k in ("x", "y", "z", "vx", "vy", "vz", "u", "h", "m")],
                          vp(S), vp(ty), vp(fl), None, None, None, None)
    K = np.array([1.0])
    G = np.array([2.0])
    e = sph.sph_eos(1, K.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                    G.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    m = sph.sph_material(1.0, 2.0, 0.01, 0, 0, 0, 0)
    h = ctypes.c_void_p()
    L = sph.lib()
    st = L.sph_init(ctypes.byref(h), ctypes.byref(p), ctypes.byref(e), ctypes.byref(m), None, 1,
                    None, None)
    assert st == 8, sph.sph_last_error()
    assert h.value is None
    assert "device" in sph.sph_last_error().lower()


def test_bad_arguments_rejected_before_device(lib):
    from paper_2107_07315_gb300 import sph

    L = sph.lib()
    h = ctypes.c_void_p()
    assert L.sph_init(ctypes.byref(h), None, None, None, None, 1, None, None) == 1
    assert L.sph_step(None, ctypes.c_double(1e-3), 1) == 1
    assert L.sph_sync(None) == 1


def test_product_package_does_not_use_oracle():
    pkg = os.path.join(ROOT, "paper_2107_07315_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle", txt, re.M), f
                assert "liboracle" not in txt and "sph_oracle" not in txt, f


def test_checked_build_exports_the_same_symbols_and_says_so(lib):
    # the bounds-checked variant (-DSPH_CHECKED) has the same boundary; each
    # build reports which one it is, and only the checked one accepts the
    # candidate-list write that exercises its bounds check
    from paper_2107_07315_gb300 import build

    chk = ctypes.CDLL(build.build(checked=True))
    for name in _declared():
        assert hasattr(chk, name), name
    chk.sph_build_checked.restype = ctypes.c_int32
    lib.sph_build_checked.restype = ctypes.c_int32
    assert chk.sph_build_checked() == 1 and lib.sph_build_checked() == 0
    lib.sph_checked_set_candidate.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                              ctypes.c_int32]
    assert lib.sph_checked_set_candidate(None, 0, 0, 0) == 1


def test_binding_wrappers_call_the_status_check_with_two_arguments():
    # every wrapper passes (status, name) to _check; a stray argument would
    # only surface on a GPU
    import ast

    src = open(os.path.join(ROOT, "paper_2107_07315_gb300", "sph.py")).read()
    calls = [n for n in ast.walk(ast.parse(src))
             if isinstance(n, ast.Call) and getattr(n.func, "id", None) == "_check"]
    assert calls
    for c in calls:
        assert len(c.args) == 2 and not c.keywords, ast.unparse(c)
