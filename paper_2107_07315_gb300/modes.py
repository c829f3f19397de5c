"""Oscillation-mode extraction from particle snapshots (Sec. III.B).

The paper reads radial modes from the internal energy and non-radial modes
from v_theta of a slab of particles at r = (0.5 +- 0.04) R0, theta = 2 pi/3 +-
0.08 pi, whose velocities are described by a linear fit in r and theta; the
frequencies are the peaks of the spectrum of those series.  Host-side numpy,
applied to snapshots read back from the device.
"""
import math

import numpy as np

# G M_sun / c^3 in seconds: the time unit of geometric units with M_sun = 1
T_SUN_S = 1.32712440018e20 / 299792458.0 ** 3

SLAB_R = (0.5, 0.04)                       # r / R0: centre, half-width
SLAB_THETA = (2.0 * math.pi / 3.0, 0.08 * math.pi)


def spherical(pos, vel, center=(0.0, 0.0, 0.0)):
    """(r, theta, v_r, v_theta) of particles about `center`; theta from +z,
    theta_hat = (cos th cos ph, cos th sin ph, -sin th)."""
    p = np.asarray(pos, np.float64) - np.asarray(center, np.float64)[None, :]
    v = np.asarray(vel, np.float64)
    r = np.linalg.norm(p, axis=1)
    rs = np.where(r > 0, r, 1.0)
    rho_c = np.hypot(p[:, 0], p[:, 1])
    theta = np.arctan2(rho_c, p[:, 2])
    vr = (p * v).sum(1) / rs
    # theta_hat * rho_c * r = (x z, y z, -rho_c^2)
    num = p[:, 0] * p[:, 2] * v[:, 0] + p[:, 1] * p[:, 2] * v[:, 1] - rho_c * rho_c * v[:, 2]
    vth = num / np.where(rho_c > 0, rho_c * rs, 1.0)
    return r, theta, vr, np.where(rho_c > 0, vth, 0.0)


def slab_mask(r, theta, R0, slab_r=SLAB_R, slab_theta=SLAB_THETA):
    return ((np.abs(r / R0 - slab_r[0]) <= slab_r[1])
            & (np.abs(theta - slab_theta[0]) <= slab_theta[1]))


def slab_vtheta(pos, vel, R0, center=(0.0, 0.0, 0.0), slab_r=SLAB_R, slab_theta=SLAB_THETA):
    """v_theta at the slab centre: the constant term of the least-squares fit
    v_theta = c0 + c1 (r/R0 - r_mid) + c2 (theta - theta_mid) over the slab."""
    r, th, _, vth = spherical(pos, vel, center)
    m = slab_mask(r, th, R0, slab_r, slab_theta)
    if m.sum() < 3:
        raise ValueError("slab holds fewer than 3 particles")
    A = np.stack([np.ones(m.sum()), r[m] / R0 - slab_r[0], th[m] - slab_theta[0]], axis=1)
    coef, *_ = np.linalg.lstsq(A, vth[m], rcond=None)
    return float(coef[0])


def internal_energy(m, u):
    """Total internal energy sum_a m_a u_a (the radial-mode signal)."""
    return float(np.dot(np.asarray(m, np.float64), np.asarray(u, np.float64)))


def spectrum(t, y, pad: int = 16):
    """(f, |Y(f)|): cyclic frequencies and the amplitude spectrum of the series
    with its mean and linear trend removed, Hann-windowed and zero-padded to
    pad times its length.  t must be uniformly spaced."""
    t = np.asarray(t, np.float64)
    y = np.asarray(y, np.float64)
    if len(t) < 4:
        raise ValueError("need at least 4 samples")
    dt = t[1] - t[0]
    if not np.allclose(np.diff(t), dt, rtol=1e-9, atol=0.0):
        raise ValueError("samples must be uniformly spaced")
    y = y - np.polyval(np.polyfit(t - t[0], y, 1), t - t[0])
    n = len(y) * pad
    Y = np.abs(np.fft.rfft(y * np.hanning(len(y)), n))
    return np.fft.rfftfreq(n, dt), Y


def peak_frequencies(t, y, k: int = 3, pad: int = 16, f_min: float = 0.0):
    """The k strongest local maxima of the spectrum above f_min, strongest
    first, each refined by a parabola through its three bins."""
    f, Y = spectrum(t, y, pad)
    i = np.nonzero((Y[1:-1] > Y[:-2]) & (Y[1:-1] >= Y[2:]))[0] + 1
    i = i[f[i] > f_min]
    i = i[np.argsort(Y[i])[::-1]][:k]
    out = []
    for j in i:
        a, b, c = Y[j - 1], Y[j], Y[j + 1]
        den = a - 2.0 * b + c
        d = 0.5 * (a - c) / den if den != 0 else 0.0
        out.append((f[j] + d * (f[1] - f[0]), b))
    return out


def to_hz(f_geometric: float, mass_unit_msun: float = 1.0) -> float:
    """A cyclic frequency in 1/(G M/c^3) converted to Hz."""
    return f_geometric / (T_SUN_S * mass_unit_msun)
