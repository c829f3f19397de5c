"""Roofline arithmetic of the benchmark (no GPU): achieved = algorithmic work
per launch / the launch's time, frac = achieved / peak, and the dominant
kernel is the slowest one."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_roofline_entries():
    b = _bench()
    # timing slots: 0/1 force, 2/3 density, 6/7 sort+tree, 8/9 lists, 10/11 search
    tim = [0.6, 10, 0.35, 10, 0, 0, 0.3, 10, 1.8, 10, 2.1, 10]
    n, pairs, solid = 100000, 6.0e6, 3.0e5
    r = b.rooflines(tim, n, pairs, solid, True, profiled=False)
    al = r["all"]
    assert al["lists"]["kernel_ms"] == pytest.approx(0.18)
    lists_bytes = 16.0 * n + 4.0 * pairs + 4.0 * n
    assert al["lists"]["achieved"] == pytest.approx(lists_bytes / 0.18e-3 / 1e9)
    force_flops = 74.0 * pairs + 45.0 * solid
    assert al["force"]["achieved"] == pytest.approx(force_flops / 0.06e-3 / 1e12)
    assert al["density"]["achieved"] == pytest.approx(22.0 * pairs / 0.035e-3 / 1e12)
    d = r["dominant"]
    assert d["kernel"].startswith("k_neighbors") and d["bound"] == "hbm"
    assert d["frac"] == pytest.approx(d["achieved"] / d["peak"])
    assert d["traffic"] is None
    # FP64 kernels are held to the FP64 rate, mixed ones to the FP32 rate
    r64 = b.rooflines(tim, n, pairs, solid, False, profiled=False)
    assert r64["all"]["force"]["frac"] > al["force"]["frac"] * 10
    rhs = b._rhs_only(tim, pairs)
    assert rhs["ms"] == pytest.approx(0.21 + 0.035 + 0.06)
