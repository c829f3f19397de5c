"""Pins of the continuum toroidal-mode solver used by the crust-shell test,
against closed forms of the toroidal eigenproblem."""
import math

import numpy as np
import pytest

from _toroidal import toroidal_frequencies


def test_thin_uniform_shell_limit():
    # a thin shell of radius R: omega^2 = (l-1)(l+2) mu / (rho R^2)
    R, mu, rho0 = 1.0, 0.3, 2.0
    for l in (2, 3):
        w = toroidal_frequencies(lambda r: np.full_like(r, rho0), R - 1e-3, R + 1e-3, mu, l=l)[0]
        assert w == pytest.approx(math.sqrt((l - 1) * (l + 2) * mu / (rho0 * R * R)), rel=1e-5)


def test_inverse_square_density_has_rigid_profile_mode():
    # rho = rho0 / r^2 makes W = r an exact eigenfunction (the stress term
    # d(W/r)/dr vanishes and the angular term balances rho omega^2 W pointwise),
    # so omega^2 = (l-1)(l+2) mu / rho0 on any thick shell
    mu, rho0 = 0.5, 0.8
    for l in (2, 4):
        w = toroidal_frequencies(lambda r: rho0 / (r * r), 0.4, 1.0, mu, l=l)[0]
        assert w == pytest.approx(math.sqrt((l - 1) * (l + 2) * mu / rho0), rel=1e-6)


def test_uniform_thick_shell_overtone_spacing():
    # the overtones of a thick uniform shell approach the radial standing-wave
    # spacing omega_n ~ n pi c_t / (r_out - r_in), c_t^2 = mu / rho
    mu, rho0, r_in, r_out = 1.0, 1.0, 0.5, 1.0
    w = toroidal_frequencies(lambda r: np.full_like(r, rho0), r_in, r_out, mu, l=2, k=6)
    ct = math.sqrt(mu / rho0)
    assert w[5] - w[4] == pytest.approx(math.pi * ct / (r_out - r_in), rel=0.02)
    # the fundamental lies below the thin-shell value at the outer radius and
    # above that at the inner radius
    assert 2.0 * ct / r_out < w[0] < 2.0 * ct / r_in
