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


def test_launch_shape_record():
    b = _bench()
    st = [0] * 32
    st[7], st[19], st[20], st[31] = 4, 8, 1, 2
    st[28:31] = [90000, 80000, 85000]
    st[21:25] = [50000, 40000, 30000, 45000]  # ns: screen 4/8, pairs 4/8
    sh = b.launch_shape(st)
    assert sh["screen_lanes"] == 8 and sh["pair_lanes"] == 4 and sh["source"] == "autotuned"
    assert sh["search_leaf_particles"] == 16 and sh["tuner_us_build"]["leaf_16"] == pytest.approx(80.0)
    assert sh["tuner_us_per_launch"]["screen_8"] == pytest.approx(40.0)
    # fixed default (screen 4, pairs 8) against the chosen (screen 8, pairs 4)
    assert sh["tuned_vs_fixed"] == pytest.approx((50000 + 45000) / (40000 + 30000))
    st[20], st[21:25], st[28:31] = 0, [0, 0, 0, 0], [0, 0, 0]
    sh = b.launch_shape(st)
    assert sh["source"] == "fixed" and "tuned_vs_fixed" not in sh


def test_profile_traffic_follows_source_hash(tmp_path, monkeypatch):
    # traffic is read from a summary only while its kernel sources are unchanged
    b = _bench()
    h = b.source_hash(("sph_tiles.cu", "sph_screen.cuh", "sph_device.cuh"))
    assert len(h) == 16
    prof = tmp_path / "profiles"
    prof.mkdir()
    for name, t in (("tiles_star1e5.md", 100), ("screen_star1e5.md", 50)):
        (prof / name).write_text("kernel_source_sha256_16: %s\ndram_bytes_per_launch: %d\n" % (h, t))
    csrc = os.path.join(ROOT, "paper_2107_07315_gb300", "csrc")
    (tmp_path / "paper_2107_07315_gb300").mkdir()
    os.symlink(csrc, tmp_path / "paper_2107_07315_gb300" / "csrc")
    monkeypatch.setattr(b, "ROOT", str(tmp_path))
    assert b.traffic_from_profile("lists") == 150.0
    (prof / "screen_star1e5.md").write_text("kernel_source_sha256_16: 0000000000000000\n"
                                            "dram_bytes_per_launch: 50\n")
    assert b.traffic_from_profile("lists") is None
