"""Continuum reference for toroidal oscillations of an elastic spherical shell.

A toroidal displacement xi = W(r) r_hat x grad Y_lm in a shell r_in <= r <= r_out
with constant shear modulus mu and density rho(r) has the energy balance

    omega^2 int rho W^2 r^2 dr = int mu [ (W' - W/r)^2 + (l-1)(l+2) W^2/r^2 ] r^2 dr,

and its eigenfrequencies are the stationary values of that Rayleigh quotient with
free (traction-free) ends: the natural boundary condition of the quotient is
sigma_r_phi = mu r d(W/r)/dr = 0.  This module solves the quotient with linear
finite elements.  It is test infrastructure: the toroidal crust experiment of
Sec. V compares the SPH run's frequency with it.
"""
import numpy as np
import scipy.linalg as sl


def toroidal_frequencies(rho, r_in: float, r_out: float, mu: float, l: int = 2,
                         n_el: int = 400, k: int = 3) -> np.ndarray:
    """The k lowest angular frequencies omega of the l toroidal modes.
    rho: callable giving the density at an array of radii."""
    x = np.linspace(r_in, r_out, n_el + 1)
    g, gw = np.polynomial.legendre.leggauss(6)
    a, b = x[:-1, None], x[1:, None]
    L = b - a
    r = a + (g[None, :] + 1.0) * L / 2.0          # [n_el, 6] quadrature points
    w = gw[None, :] * L / 2.0
    N0, N1 = (b - r) / L, (r - a) / L
    d0, d1 = -1.0 / L, 1.0 / L
    B0, B1 = d0 - N0 / r, d1 - N1 / r              # (W' - W/r) per shape function
    c = (l - 1) * (l + 2)
    wk = w * mu * r * r
    wm = w * rho(r) * r * r
    K = np.zeros((n_el + 1, n_el + 1))
    M = np.zeros((n_el + 1, n_el + 1))
    shapes = ((N0, B0), (N1, B1))
    for i, (Ni, Bi) in enumerate(shapes):
        for j, (Nj, Bj) in enumerate(shapes):
            kij = (wk * (Bi * Bj + c * Ni * Nj / (r * r))).sum(1)
            mij = (wm * Ni * Nj).sum(1)
            idx_i = np.arange(n_el) + i
            idx_j = np.arange(n_el) + j
            np.add.at(K, (idx_i, idx_j), kij)
            np.add.at(M, (idx_i, idx_j), mij)
    ev = sl.eigh(K, M, eigvals_only=True, subset_by_index=[0, k - 1])
    return np.sqrt(np.maximum(ev, 0.0))
