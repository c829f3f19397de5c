"""Roofline arithmetic of the benchmark (no GPU): the dominant entry is the
pair pass (neighbour-list stage + force) held to the measured FMA rate,
achieved = true-neighbour flops / the pass's time, frac = achieved / peak."""
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
    # timing slots: 0/1 force, 2/3 FP64 density, 6/7 sort+tree, 8/9 lists, 10/11 search
    tim = [0.6, 10, 0.0, 10, 0, 0, 0.3, 10, 1.2, 10, 1.5, 10]
    n, pairs, solid = 100000, 6.0e6, 3.0e5
    rates = {"fp32_tflops": 70.0, "fp64_tflops": 1.1, "sms": 152}
    r = b.rooflines(tim, n, pairs, solid, True, rates, profiled=False)
    al = r["all"]
    assert al["lists"]["kernel_ms"] == pytest.approx(0.12)
    force_flops = 74.0 * pairs + 45.0 * solid
    assert al["force"]["achieved"] == pytest.approx(force_flops / 0.06e-3 / 1e12)
    assert al["lists"]["achieved"] == pytest.approx(22.0 * pairs / 0.12e-3 / 1e12)
    d = r["dominant"]
    assert d["bound"] == "alu" and d["peak"] == 70.0
    assert d["kernel_ms"] == pytest.approx(0.18)
    assert d["achieved"] == pytest.approx((force_flops + 22.0 * pairs) / 0.18e-3 / 1e12)
    assert d["frac"] == pytest.approx(d["achieved"] / d["peak"])
    assert d["traffic"] is None
    assert r["fp32_nominal"] == pytest.approx(152 * 128 * 2 * 2070e6 / 1e12, rel=1e-3)
    # FP64 kernels are held to the measured FP64 rate
    r64 = b.rooflines(tim, n, pairs, solid, False, rates, profiled=False)
    assert r64["dominant"]["peak"] == 1.1
    assert r64["all"]["force"]["frac"] > al["force"]["frac"] * 10
    rhs = b._rhs_only(tim, pairs)
    assert rhs["ms"] == pytest.approx(0.15 + 0.0 + 0.06)
