"""Mode-extraction helpers (Sec. III.B) against closed forms: spherical
components, the slab fit, spectral peaks, the unit conversion."""
import math

import numpy as np
import pytest

from paper_2107_07315_gb300 import inputs as I
from paper_2107_07315_gb300 import modes


def test_spherical_components():
    # a particle on the +x axis moving along -z has v_theta = +|v|; on the +z
    # side of the equator theta < pi/2; v_r of a radial velocity is its length
    pos = np.array([[2.0, 0.0, 0.0], [0.0, 1.0, 1.0], [1.0, 1.0, 0.0]])
    vel = np.array([[0.0, 0.0, -3.0], [0.0, 1.0, 1.0], [0.0, 0.0, 0.5]])
    r, th, vr, vth = modes.spherical(pos, vel)
    assert r == pytest.approx([2.0, math.sqrt(2), math.sqrt(2)])
    assert th == pytest.approx([math.pi / 2, math.pi / 4, math.pi / 2])
    assert vr[1] == pytest.approx(math.sqrt(2))
    assert vth[0] == pytest.approx(3.0) and vth[2] == pytest.approx(-0.5)
    assert vth[1] == pytest.approx(0.0, abs=1e-15)


def test_star_state_mode_velocity_matches_harmonic():
    # the generator's v_theta for (l, n, amp) equals amp c_s sin(n pi r/R) dY_l0/dtheta
    prof = I.tov_solve(100.0, 2.0, 0.00128)
    st, eos, met, _ = I.star_state(3000, seed=4, amp_l0=0.0, prof=prof, modes=[(3, 1, 0.02)])
    pos = np.stack([st["x"], st["y"], st["z"]], 1)
    vel = np.stack([st["vx"], st["vy"], st["vz"]], 1)
    r, th, vr, vth = modes.spherical(pos, vel)
    assert np.abs(vr).max() < 1e-12 * np.abs(vth).max()
    # Y_3^0 = sqrt(7/(4 pi)) (5 c^3 - 3 c)/2; dY/dtheta = -sqrt(7/(4 pi)) sin (15 c^2 - 3)/2
    c, s = np.cos(th), np.sin(th)
    shape = -math.sqrt(7.0 / (4.0 * math.pi)) * s * (15.0 * c * c - 3.0) / 2.0
    w = np.sin(math.pi * np.minimum(r, prof.rbar_s) / prof.rbar_s) * shape
    ratio = vth[np.abs(w) > 1e-3] / w[np.abs(w) > 1e-3]
    # the remaining factor is 0.02 c_s(r) > 0, the same sign everywhere
    assert ratio.min() > 0 and ratio.max() < 0.02


def test_slab_fit_recovers_linear_field():
    rng = np.random.default_rng(3)
    R0 = 10.0
    n = 20000
    r = R0 * rng.uniform(0.3, 0.7, n)
    th = rng.uniform(0.0, math.pi, n)
    ph = rng.uniform(-math.pi, math.pi, n)
    pos = np.stack([r * np.sin(th) * np.cos(ph), r * np.sin(th) * np.sin(ph), r * np.cos(th)], 1)
    vth = 0.3 + 2.0 * (r / R0 - 0.5) - 0.7 * (th - 2 * math.pi / 3)
    eth = np.stack([np.cos(th) * np.cos(ph), np.cos(th) * np.sin(ph), -np.sin(th)], 1)
    er = pos / r[:, None]
    vel = vth[:, None] * eth + 5.0 * er          # radial part must not leak in
    assert modes.slab_vtheta(pos, vel, R0) == pytest.approx(0.3, abs=1e-12)
    # the slab bounds: |r/R0 - 0.5| <= 0.04 and |theta - 2pi/3| <= 0.08 pi
    m = modes.slab_mask(r, th, R0)
    assert np.all(np.abs(r[m] / R0 - 0.5) <= 0.04)
    assert np.all(np.abs(th[m] - 2 * math.pi / 3) <= 0.08 * math.pi)
    with pytest.raises(ValueError):
        modes.slab_vtheta(pos[:2], vel[:2], R0)


def test_peak_frequencies_of_two_tones():
    t = np.arange(0.0, 400.0, 0.5)
    y = np.sin(2 * math.pi * 0.0213 * t) + 0.4 * np.cos(2 * math.pi * 0.0571 * t) + 0.01 * t
    pk = modes.peak_frequencies(t, y, k=2)
    assert pk[0][0] == pytest.approx(0.0213, rel=2e-3)
    assert pk[1][0] == pytest.approx(0.0571, rel=2e-3)
    assert pk[0][1] > pk[1][1]
    with pytest.raises(ValueError):
        modes.spectrum(np.array([0.0, 1.0, 3.0, 4.0]), np.zeros(4))


def test_geometric_time_unit():
    # G M_sun / c^3 = 4.9255 microseconds; a geometric frequency of 0.01 is ~2.03 kHz
    assert modes.T_SUN_S == pytest.approx(4.92549e-6, rel=1e-5)
    assert modes.to_hz(0.01) == pytest.approx(2030.25, rel=1e-4)
