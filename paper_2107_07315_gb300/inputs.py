"""Seeded synthetic inputs: lattice cube, TOV neutron stars, star ensembles.

This module builds initial conditions only.  It holds none of the right-hand
side's arithmetic (no kernel, density summation, pair force, stress rate or
background force): both the CUDA path and the CPU oracle consume what it
returns.  Stars follow arXiv 2107.07315 Sec. II.A (TOV structure, particles
on concentric shells following the density profile, random perturbation of
the placement) and Sec. II.B (velocity perturbations exciting the l=0 and
l=2 modes); units are G = c = Msun = 1 (Sec. I.C).

A particle state is a dict of numpy arrays in caller order:
    x y z vx vy vz u h m mu Y0 eps_break : float64 [n]
    S : float64 [6, n] (xx, yy, zz, xy, xz, yz)
    type, flags : uint8 [n]   star : int32 [n]
together with ``eos`` {"K", "Gamma"} (per star), ``material`` (scalar
options) and ``metric`` (None or isotropic tables per star).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# Geometric units: 1 length unit = G Msun / c^2.
MSUN_G = 1.98847e33          # g
G_CGS = 6.67430e-8           # cm^3 g^-1 s^-2
C_CGS = 2.99792458e10        # cm/s
LEN_CM = G_CGS * MSUN_G / C_CGS ** 2          # 1.4766e5 cm
TIME_S = LEN_CM / C_CGS                       # 4.925e-6 s
RHO_CGS = MSUN_G / LEN_CM ** 3                # g/cm^3 per code density unit
KM = 1.0e5 / LEN_CM                           # code lengths per km


def k_code_to_cgs(K: float, Gamma: float) -> float:
    """Polytropic constant in cgs (P in dyn/cm^2, rho in g/cm^3)."""
    # P_cgs = rho_u c^2 P_code, rho_cgs = rho_u rho_code
    return K * (RHO_CGS * C_CGS ** 2) / RHO_CGS ** Gamma


DEFAULT_MATERIAL = dict(alpha_av=1.0, beta_av=2.0, eta2=0.01, jaumann=0, yield_mode=0,
                        break_stress=0, break_zero_S=0)


# ---------------------------------------------------------------------------
# TOV structure (Sec. II.A) in areal radius R, with lapse and isotropic radius
# ---------------------------------------------------------------------------
@dataclass
class TovProfile:
    K: float
    Gamma: float
    rho_c: float
    M: float            # gravitational mass
    R: float            # areal radius of the surface
    rbar_s: float       # isotropic radius of the surface
    M_baryon: float
    # arrays on an increasing isotropic radius grid (0 .. rbar_s)
    rbar: np.ndarray
    rho: np.ndarray
    P: np.ndarray
    u: np.ndarray
    alpha: np.ndarray
    dalpha: np.ndarray   # d alpha / d rbar
    psi4: np.ndarray
    dpsi4: np.ndarray    # d psi^4 / d rbar
    eos: dict | None = None  # the star's EoS (piecewise polytropes); K, Gamma: central piece


def _eos(K, Gamma, P):
    P = max(P, 0.0)
    rho = (P / K) ** (1.0 / Gamma)
    u = K * rho ** (Gamma - 1.0) / (Gamma - 1.0) if rho > 0 else 0.0
    return rho, u


def tov_solve(K: float, Gamma: float, rho_c: float, npts: int = 4000) -> TovProfile:
    """Integrate the TOV structure equations in the theta form of Sec. II.A.

    rho = rho_c theta^n, n = 1/(Gamma-1), s = R^2 (areal radius), from the
    centre (theta = 1) to the surface (theta = 0):
      ds/dtheta = -2 n s^(3/2)/(m theta) (dP/drho) (1 + u + P/rho)^-1
                  (1 + 4 pi R^3 P/m)^-1 (1 - 2m/R)
      dm/dtheta = 2 pi s^(1/2) rho (1 + u) ds/dtheta
    with P = K rho^Gamma, u = K rho^(Gamma-1)/(Gamma-1).  Alongside: the
    lapse alpha = e^Phi, dPhi/dR = (m + 4 pi R^3 P)/(R (R - 2m)), and the
    isotropic radius through w = ln(rbar/R), dw/dR = (1/sqrt(1-2m/R) - 1)/R.
    """
    from scipy.integrate import solve_ivp

    n = 1.0 / (Gamma - 1.0)
    Pc = K * rho_c ** Gamma
    uc = K * rho_c ** (Gamma - 1.0) / (Gamma - 1.0)
    ec = rho_c * (1.0 + uc)

    def f(th, y):
        s, m, _phi, _w = y
        th = max(th, 0.0)
        rho = rho_c * th ** n
        P = K * rho ** Gamma
        u = K * rho ** (Gamma - 1.0) / (Gamma - 1.0)
        dPdrho = Gamma * K * rho_c ** (Gamma - 1.0) * th  # rho^(Gamma-1) = rho_c^(Gamma-1) theta
        R = math.sqrt(s)
        # n/theta * dP/drho stays finite at theta -> 0 because dP/drho ~ theta
        ds = (-2.0 * n * s ** 1.5 / m * Gamma * K * rho_c ** (Gamma - 1.0)
              / (1.0 + u + (P / rho if rho > 0 else 0.0))
              / (1.0 + 4.0 * math.pi * R ** 3 * P / m) * (1.0 - 2.0 * m / R))
        dR = ds / (2.0 * R)
        dm = 2.0 * math.pi * R * rho * (1.0 + u) * ds
        g = (m + 4.0 * math.pi * R ** 3 * P) / (R * (R - 2.0 * m))
        dphi = g * dR
        dw = (1.0 / math.sqrt(1.0 - 2.0 * m / R) - 1.0) / R * dR
        return [ds, dm, dphi, dw]

    a = (2.0 * math.pi / 3.0) * (ec + Pc) * (ec + 3.0 * Pc) / ((n + 1.0) * Pc)
    th0 = 1.0 - 1e-8
    R0 = math.sqrt((1.0 - th0) / a)
    m0 = 4.0 / 3.0 * math.pi * ec * R0 ** 3
    y0 = [R0 * R0, m0, 0.0, 0.0]
    L = 1.0 / math.sqrt(ec)
    sol = solve_ivp(f, (th0, 0.0), y0, method="DOP853", rtol=1e-11,
                    atol=[1e-18 * L * L, 1e-18 * L, 1e-15, 1e-15], dense_output=True)
    if not sol.success:
        raise RuntimeError("TOV integration failed: " + sol.message)
    ys = sol.y[:, -1]
    Rs = math.sqrt(float(ys[0]))
    M = float(ys[1])
    phi_shift = 0.5 * math.log(1.0 - 2.0 * M / Rs) - float(ys[2])
    rbar_s = 0.5 * (Rs - M + math.sqrt(Rs * Rs - 2.0 * M * Rs))
    w_shift = math.log(rbar_s / Rs) - float(ys[3])

    # grid uniform in R between the centre and the surface
    Rgrid = np.linspace(0.0, Rs, npts)
    # invert R(theta) on a fine theta sampling (R is monotone in theta)
    th_f = np.concatenate([np.linspace(th0, 0.0, 20 * npts)])
    Yf = sol.sol(th_f)
    Rf = np.sqrt(Yf[0])
    order = np.argsort(Rf)
    Rf = Rf[order]
    th = np.interp(Rgrid, np.concatenate([[0.0], Rf]), np.concatenate([[1.0], th_f[order]]))
    Y = sol.sol(np.clip(th, 0.0, th0))
    m = np.where(Rgrid > R0, Y[1], 4.0 / 3.0 * math.pi * ec * Rgrid ** 3)
    rho = rho_c * np.maximum(th, 0.0) ** n
    P = K * rho ** Gamma
    u = K * rho ** (Gamma - 1.0) / (Gamma - 1.0)
    phi = np.where(Rgrid > R0, Y[2], 0.0) + phi_shift
    w = np.where(Rgrid > R0, Y[3], 0.0) + w_shift
    R = Rgrid
    rbar = R * np.exp(w)
    alpha = np.exp(phi)
    Rs_ = np.where(R > 0, R, 1.0)
    g = np.where(R > 0, (m + 4.0 * math.pi * R ** 3 * P) / (Rs_ * (Rs_ - 2.0 * m)), 0.0)
    dRdrb = np.sqrt(np.maximum(1.0 - 2.0 * m / Rs_, 0.0)) / np.exp(w)  # dR/drbar = R sqrt(1-2m/R)/rbar
    psi4 = np.exp(-2.0 * w)                                              # (R/rbar)^2
    rb_ = np.where(rbar > 0, rbar, 1.0)
    dpsi4 = np.where(rbar > 0, 2.0 * (R / rb_) * (dRdrb - R / rb_) / rb_, 0.0)
    dalpha = alpha * g * dRdrb
    integrand = rho * psi4 ** 1.5 * 4.0 * math.pi * rbar ** 2
    Mb = float(np.trapezoid(integrand, rbar))
    return TovProfile(K, Gamma, rho_c, M, Rs, rbar_s, Mb, rbar, rho, P, u, alpha, dalpha,
                      psi4, dpsi4)


def eos_pieces(eos: dict, star: int = 0):
    """(rho_b, K, Gamma, a) per piece of a (piecewise) polytrope: piece k holds
    rho >= rho_b[k-1]; K and a (u = a + K rho^(Gamma-1)/(Gamma-1)) follow from
    continuity of P and u at the dividing densities."""
    K = [float(np.ravel(eos["K"])[star])]
    G = [float(np.ravel(eos["Gamma"])[star])]
    a = [0.0]
    rb = []
    if eos.get("rho_bound") is not None:
        nb = np.asarray(eos["rho_bound"], np.float64).reshape(len(np.ravel(eos["K"])), -1)[star]
        ga = np.asarray(eos["Gamma_above"], np.float64).reshape(len(np.ravel(eos["K"])), -1)[star]
        for r, gn in zip(nb, ga):
            kn = K[-1] * r ** (G[-1] - gn)
            a.append(a[-1] + K[-1] * r ** (G[-1] - 1.0) / (G[-1] - 1.0)
                     - kn * r ** (gn - 1.0) / (gn - 1.0))
            K.append(kn)
            G.append(float(gn))
            rb.append(float(r))
    return np.array(rb), np.array(K), np.array(G), np.array(a)


def eos_eval_pieces(eos: dict, rho, star: int = 0):
    """P, u and dP/drho of a (piecewise) polytrope at densities rho (arrays)."""
    rb, K, G, a = eos_pieces(eos, star)
    rho = np.asarray(rho, np.float64)
    k = np.searchsorted(rb, rho, side="right")
    Kk, Gk, ak = K[k], G[k], a[k]
    r = np.maximum(rho, 0.0)
    P = Kk * r ** Gk
    u = ak + Kk * r ** (Gk - 1.0) / (Gk - 1.0)
    return P, u, Gk * Kk * r ** (Gk - 1.0)


def tov_solve_pieces(eos: dict, rho_c: float, npts: int = 4000) -> TovProfile:
    """TOV structure for a (piecewise) polytrope, integrated in the areal
    radius R with the pressure as variable:
      dP/dR = -(e + P)(m + 4 pi R^3 P)/(R (R - 2m)),  dm/dR = 4 pi R^2 e,
      e = rho (1 + u), with the lapse and isotropic radius as in tov_solve;
    ends where P falls to 1e-14 of the central pressure."""
    from scipy.integrate import solve_ivp

    rb, Kp, Gp, ap = eos_pieces(eos)
    Pb = Kp[1:] * rb ** Gp[1:] if len(rb) else np.array([])

    def rho_of_P(P):
        P = max(P, 0.0)
        k = int(np.searchsorted(Pb, P, side="right"))
        return (P / Kp[k]) ** (1.0 / Gp[k]), k

    Pc, uc, _ = (float(v) for v in eos_eval_pieces(eos, rho_c))
    ec = rho_c * (1.0 + uc)

    def f(R, y):
        P, m, _phi, _w = y
        rho, k = rho_of_P(P)
        u = ap[k] + Kp[k] * rho ** (Gp[k] - 1.0) / (Gp[k] - 1.0) if rho > 0 else 0.0
        e = rho * (1.0 + u)
        g = (m + 4.0 * math.pi * R ** 3 * P) / (R * (R - 2.0 * m))
        return [-(e + P) * g, 4.0 * math.pi * R * R * e, g,
                (1.0 / math.sqrt(1.0 - 2.0 * m / R) - 1.0) / R]

    L = 1.0 / math.sqrt(ec)
    R0 = 1e-6 * L
    y0 = [Pc - (2.0 * math.pi / 3.0) * (ec + Pc) * (ec + 3.0 * Pc) * R0 * R0,
          4.0 / 3.0 * math.pi * ec * R0 ** 3, 0.0, 0.0]
    surf = lambda R, y: y[0] - 1e-14 * Pc
    surf.terminal, surf.direction = True, -1
    sol = solve_ivp(f, (R0, 100.0 * L), y0, method="DOP853", rtol=1e-11,
                    atol=[1e-16 * Pc, 1e-18 * L, 1e-15, 1e-15], events=surf, dense_output=True)
    if not sol.success or not len(sol.t_events[0]):
        raise RuntimeError("TOV integration (pieces) failed: " + sol.message)
    Rs = float(sol.t_events[0][0])
    ys = sol.sol(Rs)
    M = float(ys[1])
    R = np.linspace(0.0, Rs, npts)
    Y = sol.sol(np.maximum(R, R0))
    P = np.where(R > R0, np.maximum(Y[0], 0.0), Pc)
    m = np.where(R > R0, Y[1], 4.0 / 3.0 * math.pi * ec * R ** 3)
    rho = np.array([rho_of_P(x)[0] for x in P])
    _, u, _ = eos_eval_pieces(eos, rho)
    phi = np.where(R > R0, Y[2], 0.0) + 0.5 * math.log(1.0 - 2.0 * M / Rs) - float(ys[2])
    rbar_s = 0.5 * (Rs - M + math.sqrt(Rs * Rs - 2.0 * M * Rs))
    w = np.where(R > R0, Y[3], 0.0) + math.log(rbar_s / Rs) - float(ys[3])
    kc = int(np.searchsorted(rb, rho_c, side="right"))
    return _isotropic_profile(float(Kp[kc]), float(Gp[kc]), rho_c, M, Rs, rbar_s, R, m, rho, P,
                              u, phi, w, eos)


def _isotropic_profile(K, Gamma, rho_c, M, Rs, rbar_s, R, m, rho, P, u, phi, w, eos=None):
    """TovProfile on the isotropic radius from areal-radius arrays: rbar = R e^w,
    alpha = e^phi, psi^4 = (R/rbar)^2 and their rbar-derivatives."""
    rbar = R * np.exp(w)
    alpha = np.exp(phi)
    Rs_ = np.where(R > 0, R, 1.0)
    g = np.where(R > 0, (m + 4.0 * math.pi * R ** 3 * P) / (Rs_ * (Rs_ - 2.0 * m)), 0.0)
    dRdrb = np.sqrt(np.maximum(1.0 - 2.0 * m / Rs_, 0.0)) / np.exp(w)
    psi4 = np.exp(-2.0 * w)
    rb_ = np.where(rbar > 0, rbar, 1.0)
    dpsi4 = np.where(rbar > 0, 2.0 * (R / rb_) * (dRdrb - R / rb_) / rb_, 0.0)
    dalpha = alpha * g * dRdrb
    Mb = float(np.trapezoid(rho * psi4 ** 1.5 * 4.0 * math.pi * rbar ** 2, rbar))
    return TovProfile(K, Gamma, rho_c, M, Rs, rbar_s, Mb, rbar, rho, P, u, alpha, dalpha, psi4,
                      dpsi4, eos)


def solve_star(Gamma: float, M_target: float = 1.4, R_target_km: float = 12.0):
    """(K, rho_c) with gravitational mass M_target and areal radius R_target.

    For a polytrope, K^(1/(2(Gamma-1))) is the only length scale: solve the
    dimensionless (K = 1) problem for the compactness M/R, then rescale.
    """
    from scipy.optimize import brentq

    Rt = R_target_km * KM
    Ct = M_target / Rt

    def comp(lrc):
        p = tov_solve(1.0, Gamma, math.exp(lrc), npts=50)
        return p.M / p.R - Ct

    # bracket on the stable branch: compactness grows with rho_c up to M_max
    lo, hi = math.log(1e-6), math.log(1e-6)
    while comp(hi) < 0:
        lo, hi = hi, hi + 0.5
        if hi > 10:
            raise ValueError("compactness %.4f not reachable for Gamma=%g" % (Ct, Gamma))
    lrc = brentq(comp, lo, hi, xtol=1e-13)
    p = tov_solve(1.0, Gamma, math.exp(lrc), npts=50)
    lam = M_target / p.M
    K = lam ** (2.0 * (Gamma - 1.0))
    rho_c = math.exp(lrc) / lam ** 2
    return K, rho_c


def metric_tables(profs, centers, nr: int = 4096) -> dict:
    """Isotropic metric tables on uniform nodes 0..rbar_s for each star."""
    ns = len(profs)
    out = dict(kind=1, nr=nr, r_max=np.zeros(ns), alpha=np.zeros((ns, nr)),
               dalpha=np.zeros((ns, nr)), psi4=np.zeros((ns, nr)), dpsi4=np.zeros((ns, nr)),
               M=np.zeros(ns), center=np.asarray(centers, dtype=np.float64).reshape(ns, 3))
    for s, p in enumerate(profs):
        grid = np.linspace(0.0, p.rbar_s, nr)
        out["r_max"][s] = p.rbar_s
        out["M"][s] = p.M
        for k in ("alpha", "dalpha", "psi4", "dpsi4"):
            out[k][s] = np.interp(grid, p.rbar, getattr(p, k))
        # make the last node exactly the exterior value at rbar_s
        kk = p.M / (2.0 * p.rbar_s)
        out["alpha"][s, -1] = (1 - kk) / (1 + kk)
        out["psi4"][s, -1] = (1 + kk) ** 4
    return out


# ---------------------------------------------------------------------------
# Particle placement
# ---------------------------------------------------------------------------
def _fibonacci_sphere(n: int) -> np.ndarray:
    if n == 1:
        return np.array([[0.0, 0.0, 1.0]])
    i = np.arange(n) + 0.5
    z = 1.0 - 2.0 * i / n
    r = np.sqrt(np.maximum(1.0 - z * z, 0.0))
    phi = i * math.pi * (3.0 - math.sqrt(5.0))
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def _random_rotation(rng) -> np.ndarray:
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([[a*a+b*b-c*c-d*d, 2*(b*c-a*d), 2*(b*d+a*c)],
                     [2*(b*c+a*d), a*a-b*b+c*c-d*d, 2*(c*d-a*b)],
                     [2*(b*d-a*c), 2*(c*d+a*b), a*a-b*b-c*c+d*d]])


def place_star(prof: TovProfile, N: int, rng, jitter: float = 0.05):
    """N equal-baryon-mass particles on concentric shells (Sec. II.A).

    Shell populations follow the cumulative baryon mass of rho psi^6; each
    shell is a Fibonacci sphere with a random rotation; radii carry a uniform
    relative jitter of +-``jitter`` of the local shell spacing.
    """
    return place_profile(prof.rbar, prof.rho * prof.psi4 ** 1.5, N, rng, jitter)


def place_profile(rb, dens, N: int, rng, jitter: float = 0.05):
    """N equal-mass particles on concentric Fibonacci shells following the
    radial density dens(rb) (zero where no matter is); returns (positions,
    particle mass).  Shells start where the density first becomes positive."""
    rb = np.asarray(rb, np.float64)
    dens = np.asarray(dens, np.float64)
    cum = np.concatenate([[0.0], np.cumsum(0.5 * (dens[1:] * rb[1:] ** 2 + dens[:-1] * rb[:-1] ** 2)
                                            * np.diff(rb))]) * 4.0 * math.pi
    Mb = cum[-1]
    mp = Mb / N
    # shell edges: spacing (mp/dens)^(1/3) evaluated at the shell's inner edge
    first = int(np.argmax(dens > 0))
    edges = [float(rb[max(first - 1, 0)])]
    while True:
        r0 = edges[-1]
        d = np.interp(r0, rb, dens)
        if d <= 0 and r0 <= rb[first]:
            # an inner edge where the matter only begins: size the first shell
            # by the mean density over one spacing at the peak density
            s0 = (mp / dens.max()) ** (1.0 / 3.0)
            d = float(np.mean(np.interp(np.linspace(r0, r0 + s0, 16), rb, dens)))
        if d <= 0:
            break
        s = (mp / d) ** (1.0 / 3.0)
        dm = np.interp(min(r0 + 0.5 * s, rb[-1]), rb, dens)
        s = (mp / max(dm, 1e-300)) ** (1.0 / 3.0)
        r1 = r0 + s
        if r1 >= rb[-1] or np.interp(r1, rb, cum) > Mb * (1 - 0.5 / N):
            edges.append(rb[-1])
            break
        edges.append(r1)
    edges = np.array(edges)
    cm = np.interp(edges, rb, cum)
    target = np.diff(cm) / mp
    counts = np.floor(target).astype(np.int64)
    rem = N - counts.sum()
    frac = target - counts
    order = np.argsort(-frac, kind="stable")
    counts[order[:rem]] += 1
    pos = []
    for k, nk in enumerate(counts):
        if nk <= 0:
            continue
        # radius where half of the shell's mass is inside
        mid_mass = cm[k] + 0.5 * (cm[k + 1] - cm[k])
        rk = float(np.interp(mid_mass, cum, rb))
        thick = edges[k + 1] - edges[k]
        pts = _fibonacci_sphere(int(nk)) @ _random_rotation(rng).T
        rr = rk + jitter * thick * rng.uniform(-1.0, 1.0, size=int(nk))
        if k == 0 and nk == 1:
            rr = np.abs(rr) * 0.0 + jitter * thick * rng.uniform(0, 1)
        pos.append(pts * rr[:, None])
    return np.concatenate(pos, axis=0)[:N], mp


def smoothing_lengths(pos: np.ndarray, n_target: int = 60) -> np.ndarray:
    """h_a = half the distance to the (n_target + 1/2)-th nearest particle.

    With support 2h this puts about n_target particles inside each particle's
    own support; the run-time h update keeps counts within the target band.
    """
    from scipy.spatial import cKDTree

    tree = cKDTree(pos)
    d, _ = tree.query(pos, k=n_target + 2)
    return 0.25 * (d[:, n_target] + d[:, n_target + 1])


def _sph_coords(pos):
    r = np.linalg.norm(pos, axis=1)
    rs = np.where(r > 0, r, 1.0)
    cth = np.clip(pos[:, 2] / rs, -1.0, 1.0)
    sth = np.sqrt(np.maximum(1.0 - cth ** 2, 0.0))
    phi = np.arctan2(pos[:, 1], pos[:, 0])
    return r, cth, sth, phi


def dYl0_dtheta(l: int, cth, sth):
    """d/dtheta of the orthonormal Y_l^0 = sqrt((2l+1)/(4 pi)) P_l(cos theta):
    -sin(theta) sqrt((2l+1)/(4 pi)) P_l'(cos theta)."""
    c = np.zeros(l + 1)
    c[l] = 1.0
    dP = np.polynomial.legendre.legval(cth, np.polynomial.legendre.legder(c))
    return -sth * math.sqrt((2 * l + 1) / (4.0 * math.pi)) * dP


def _empty_state(n: int) -> dict:
    z = np.zeros(n)
    return dict(x=z.copy(), y=z.copy(), z=z.copy(), vx=z.copy(), vy=z.copy(), vz=z.copy(),
                u=z.copy(), h=z.copy(), m=z.copy(), mu=z.copy(), Y0=z.copy(),
                eps_break=z.copy(), S=np.zeros((6, n)), type=np.zeros(n, np.uint8),
                flags=np.zeros(n, np.uint8), star=np.zeros(n, np.int32))


def star_state(N: int, Gamma: float = 2.0, seed: int = 1, crust_frac: float = 0.05,
               mu_over_P: float = 0.01, Y0: float = 0.1, eps_break: float = 0.05,
               amp_l0: float = 1e-3, amp_l2: float = 0.0, M: float = 1.4, R_km: float = 12.0,
               Y0_over_mu=None, nr: int = 4096, n_target: int = 60, center=(0.0, 0.0, 0.0),
               prof: TovProfile | None = None, modes=()):
    """One star: (state, eos, metric, profile).

    Crust = particles beyond (1 - crust_frac) of the isotropic surface radius,
    solid with mu = mu_over_P * P(r), Y0, eps_break per particle.  Velocity
    perturbations (Sec. II.B): v_r = amp_l0 c_s sin(pi r/R) and
    v_theta = amp_l2 c_s sin(pi r/R) d/dtheta Y_2^0, c_s relativistic.
    modes: further (l, n, amp) terms v_theta += amp c_s sin(n pi r/R) d/dtheta Y_l^0
    (the paper's (delta v_theta)_nl0 with the m = 0 harmonic).
    """
    rng = np.random.default_rng(seed)
    if prof is None:
        K, rho_c = solve_star(Gamma, M, R_km)
        prof = tov_solve(K, Gamma, rho_c)
    pos, mp = place_star(prof, N, rng)
    st = _empty_state(N)
    st["x"], st["y"], st["z"] = (pos[:, 0] + center[0], pos[:, 1] + center[1],
                                 pos[:, 2] + center[2])
    st["m"][:] = mp
    st["h"][:] = smoothing_lengths(pos, n_target)
    r, cth, sth, phi = _sph_coords(pos)
    Rs = prof.rbar_s
    rho = np.interp(r, prof.rbar, prof.rho)
    P = np.interp(r, prof.rbar, prof.P)
    u = np.interp(r, prof.rbar, prof.u)
    st["u"][:] = u
    if prof.eos is not None:
        dPdrho = eos_eval_pieces(prof.eos, rho)[2]
    else:
        dPdrho = prof.Gamma * prof.K * rho ** (prof.Gamma - 1.0)
    cs = np.sqrt(np.maximum(dPdrho, 0.0)
                 / (1.0 + u + np.where(rho > 0, P / np.where(rho > 0, rho, 1.0), 0.0)))
    sinr = np.sin(math.pi * np.minimum(r, Rs) / Rs)
    vr = amp_l0 * cs * sinr
    # d/dtheta Y_2^0 = sqrt(5/(16 pi)) * (-6 cos sin)
    vth = amp_l2 * cs * sinr * math.sqrt(5.0 / (16.0 * math.pi)) * (-6.0 * cth * sth)
    for l, nrad, amp in modes:
        vth = vth + amp * cs * np.sin(nrad * math.pi * np.minimum(r, Rs) / Rs) * dYl0_dtheta(l, cth, sth)
    er = pos / np.where(r > 0, r, 1.0)[:, None]
    eth = np.stack([cth * np.cos(phi), cth * np.sin(phi), -sth], axis=1)
    v = vr[:, None] * er + vth[:, None] * eth
    st["vx"], st["vy"], st["vz"] = v[:, 0].copy(), v[:, 1].copy(), v[:, 2].copy()
    crust = r > (1.0 - crust_frac) * Rs
    st["type"][crust] = 1
    st["mu"][crust] = mu_over_P * P[crust]
    if Y0_over_mu is not None:
        st["Y0"][crust] = Y0_over_mu * st["mu"][crust]
    else:
        st["Y0"][crust] = Y0
    st["eps_break"][crust] = eps_break
    if prof.eos is not None:
        eos = {k: np.asarray(v, np.float64) for k, v in prof.eos.items()}
    else:
        eos = dict(K=np.array([prof.K]), Gamma=np.array([prof.Gamma]))
    metric = metric_tables([prof], [center], nr=nr)
    return st, eos, metric, prof


# ---------------------------------------------------------------------------
# Relaxation in an external potential (Sec. II.A)
# ---------------------------------------------------------------------------
def relax_eos(prof: TovProfile, Gamma_r: float = 1.01) -> dict:
    """Relaxation EoS: Gamma ~ 1.01 (nearly uniform sound speed), K chosen to
    keep the star's central pressure, K_r = K rho_c^(Gamma - Gamma_r)."""
    K_r = prof.K * prof.rho_c ** (prof.Gamma - Gamma_r)
    return dict(K=np.array([K_r]), Gamma=np.array([Gamma_r]))


def relax_external(profs, centers, eos_r: dict, nr: int = 4096, wall_factor: float = 1.0,
                   k_wall=None, damping: float = 0.0, rho_floor: float = 0.01) -> dict:
    """External field of the relaxation for each star.

    Target profile: the coordinate (SPH) density of the star, rho_t = rho psi^6
    on the isotropic radius; phi_eff = -K Gamma rho_t^(Gamma-1)/(Gamma-1) with
    the relaxation EoS, tabulated on nr uniform nodes over [0, rbar_s] and
    differentiated by second-order differences: g = -d phi_eff/dr (negative =
    inward).  rho_t is floored at rho_floor * rho_t(0): with Gamma ~ 1 the
    equilibrium force K Gamma rho^(Gamma-2) grad rho diverges like 1/(R - r)
    at the surface, which no smoothed density resolves.  Wall at
    wall_factor * rbar_s with stiffness k_wall (default 10 max|g| / rbar_s);
    damping in 1/time.
    """
    ns = len(profs)
    K_r = np.asarray(eos_r["K"], np.float64)
    G_r = np.asarray(eos_r["Gamma"], np.float64)
    out = dict(kind=1, nr=nr, r_max=np.zeros(ns), g=np.zeros((ns, nr)),
               center=np.asarray(centers, dtype=np.float64).reshape(ns, 3),
               r_wall=np.zeros(ns), k_wall=0.0, damping=float(damping))
    kmax = 0.0
    for s, p in enumerate(profs):
        grid = np.linspace(0.0, p.rbar_s, nr)
        rho_t = np.interp(grid, p.rbar, p.rho * p.psi4 ** 1.5)
        rho_t = np.maximum(rho_t, rho_floor * rho_t[0])
        k, gm = K_r[min(s, len(K_r) - 1)], G_r[min(s, len(G_r) - 1)]
        phi = -k * gm * rho_t ** (gm - 1.0) / (gm - 1.0)
        out["g"][s] = -np.gradient(phi, grid, edge_order=2)
        out["r_max"][s] = p.rbar_s
        out["r_wall"][s] = wall_factor * p.rbar_s
        kmax = max(kmax, 10.0 * np.abs(out["g"][s]).max() / p.rbar_s)
    out["k_wall"] = float(kmax if k_wall is None else k_wall)
    return out


def relax_state(N: int, seed: int = 1, Gamma_r: float = 1.01, jitter: float = 0.15,
                damping_per_crossing: float = 2.0, M: float = 1.4, R_km: float = 12.0,
                nr: int = 4096, prof: TovProfile | None = None):
    """Start of a relaxation: the star of star_state (all fluid, at rest) with
    positions jittered by `jitter` times the local h, the relaxation EoS and
    its external field.  Returns (state, eos_r, external, eos_star, prof);
    damping = damping_per_crossing * c_s / R."""
    st, eos, _, prof = star_state(N, seed=seed, crust_frac=0.0, amp_l0=0.0, amp_l2=0.0, M=M,
                                  R_km=R_km, nr=nr, prof=prof)
    rng = np.random.default_rng(seed + 1000)
    d = rng.normal(size=(3, N)) * (jitter * st["h"] / math.sqrt(3.0))
    st["x"] = st["x"] + d[0]
    st["y"] = st["y"] + d[1]
    st["z"] = st["z"] + d[2]
    eos_r = relax_eos(prof, Gamma_r)
    K_r, G_r = float(eos_r["K"][0]), float(eos_r["Gamma"][0])
    rho_c = prof.rho_c
    st["u"][:] = K_r * rho_c ** (G_r - 1.0) / (G_r - 1.0)
    cs = math.sqrt(G_r * K_r * rho_c ** (G_r - 1.0))
    ext = relax_external([prof], [(0.0, 0.0, 0.0)], eos_r, nr=nr,
                         damping=damping_per_crossing * cs / prof.rbar_s)
    return st, eos_r, ext, eos, prof


# ---------------------------------------------------------------------------
# Elastic shell in an external potential (the crust-shell experiment, Sec. III)
# ---------------------------------------------------------------------------
def shell_state(N: int, r_in: float = 0.6, r_out: float = 1.0, rho0: float = 1.0,
                K: float = 0.5, Gamma: float = 2.0, shear: float = 0.1, seed: int = 1,
                nr: int = 2048, damping: float = 0.0):
    """A shell of matter between r_in and r_out with density
    rho_t = rho0 sin(pi (r - r_in)/(r_out - r_in)), held by the external
    potential of its own profile (as in the relaxation, Sec. II.A) and solid
    with shear modulus mu = shear * rho0 c_s0^2 (c_s0^2 = Gamma K rho0^(Gamma-1)),
    no yield and no breaking.  Returns (state, eos, external, info) with info
    holding the mean density and radius and the thin-shell estimate of the l=2
    toroidal frequency, omega^2 = (l-1)(l+2) mu / (rho R^2)."""
    rng = np.random.default_rng(seed)
    rb = np.linspace(0.0, r_out, 8 * nr)
    dens = np.where((rb > r_in) & (rb < r_out),
                    rho0 * np.sin(math.pi * (rb - r_in) / (r_out - r_in)), 0.0)
    pos, mp = place_profile(rb, dens, N, rng, jitter=0.05)
    n = len(pos)
    st = _empty_state(n)
    st["x"], st["y"], st["z"] = pos[:, 0].copy(), pos[:, 1].copy(), pos[:, 2].copy()
    st["m"][:] = mp
    st["h"][:] = smoothing_lengths(pos, 60)
    r = np.sqrt((pos ** 2).sum(1))
    rho = np.interp(r, rb, dens)
    st["u"][:] = K * np.maximum(rho, 1e-3 * rho0) ** (Gamma - 1.0) / (Gamma - 1.0)
    cs0 = math.sqrt(Gamma * K * rho0 ** (Gamma - 1.0))
    mu = shear * rho0 * cs0 * cs0
    st["type"][:] = 1
    st["mu"][:] = mu
    st["Y0"][:] = 1e30
    st["eps_break"][:] = 1e30
    eos = dict(K=np.array([K]), Gamma=np.array([Gamma]))
    # external field of the shell's own profile (floored at 1 % of rho0)
    grid = np.linspace(0.0, r_out, nr)
    rho_t = np.maximum(np.interp(grid, rb, dens), 0.01 * rho0)
    phi = -K * Gamma * rho_t ** (Gamma - 1.0) / (Gamma - 1.0)
    ext = dict(kind=1, nr=nr, r_max=np.array([r_out]), g=(-np.gradient(phi, grid, edge_order=2))[None, :],
               center=np.zeros((1, 3)), r_wall=np.array([r_out]),
               k_wall=10.0 * cs0 * cs0 / (r_out - r_in) ** 2, damping=float(damping))
    mass = 4.0 * math.pi * np.trapezoid(dens * rb ** 2, rb)
    rho_mean = mass / (4.0 / 3.0 * math.pi * (r_out ** 3 - r_in ** 3))
    R_mean = float(np.trapezoid(dens * rb ** 3, rb) / np.trapezoid(dens * rb ** 2, rb))
    omega = math.sqrt(4.0 * mu / (rho_mean * R_mean ** 2))
    info = dict(mu=mu, cs0=cs0, rho_mean=rho_mean, R_mean=R_mean, omega_thin=omega)
    return st, eos, ext, info


def toroidal_l2_velocity(st: dict, amp: float, R: float):
    """Axisymmetric l=2 toroidal velocity, v = amp (r/R) sin(theta) cos(theta) phi_hat
    (v proportional to r_hat x grad Y_2^0): in Cartesian form amp z (-y, x, 0)/(r R)."""
    x, y, z = st["x"], st["y"], st["z"]
    r = np.sqrt(x * x + y * y + z * z)
    f = amp * z / (np.where(r > 0, r, 1.0) * R)
    return -f * y, f * x, np.zeros_like(z)


def cfl_dt(state: dict, eos: dict, C: float = 0.3) -> float:
    """dt = C min_a h_a/(c_a + |v_a|) with the initial-profile sound speed."""
    # sound speed from u: c^2 = Gamma K rho^(Gamma-1) = (Gamma-1) Gamma u (polytrope)
    star = state.get("star")
    s = np.zeros(len(state["x"]), np.int64) if star is None else np.asarray(star, np.int64)
    G = np.asarray(eos["Gamma"])[s]
    c = np.sqrt(np.maximum((G - 1.0) * G * state["u"], 0.0))
    v = np.sqrt(state["vx"] ** 2 + state["vy"] ** 2 + state["vz"] ** 2)
    return float(C * np.min(state["h"] / (c + v)))


# ---------------------------------------------------------------------------
# Lattice cube (plain FP64 elastic cube)
# ---------------------------------------------------------------------------
def cube_state(n_side: int = 16, h: float = 1.3, seed: int = 0, K: float = 1.0,
               Gamma: float = 2.0, mu: float = 0.5, Y0: float = 0.1, eps_break: float = 0.05,
               amp: float = 0.01):
    """Unit-spacing lattice (i,j,k) in {0..n_side-1}^3, m = 1, all solid.

    v = amp * A (x - c) with A = (G + G^T)/2, G ~ N(0,1) from
    default_rng(seed) and c the cube centre; S = 0; u = K rho0^(Gamma-1)/(Gamma-1)
    with rho0 = 1.
    """
    rng = np.random.default_rng(seed)
    Gm = rng.normal(size=(3, 3))
    A = 0.5 * (Gm + Gm.T)
    g = np.arange(n_side, dtype=np.float64)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    pos = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    c = 0.5 * (n_side - 1)
    v = amp * (pos - c) @ A.T
    n = len(pos)
    st = _empty_state(n)
    st["x"], st["y"], st["z"] = pos[:, 0].copy(), pos[:, 1].copy(), pos[:, 2].copy()
    st["vx"], st["vy"], st["vz"] = v[:, 0].copy(), v[:, 1].copy(), v[:, 2].copy()
    st["m"][:] = 1.0
    st["h"][:] = h
    st["u"][:] = K / (Gamma - 1.0)
    st["type"][:] = 1
    st["mu"][:] = mu
    st["Y0"][:] = Y0
    st["eps_break"][:] = eps_break
    eos = dict(K=np.array([K]), Gamma=np.array([Gamma]))
    return st, eos, None, A


def lattice_positions(kind: str, n: int, d: float = 1.0) -> np.ndarray:
    """Points of a simple cubic ("cubic"), face-centred cubic ("fcc") or
    hexagonal close-packed ("hcp") lattice with nearest-neighbour distance d,
    n cells (cubic, fcc) or n x n x n sites (hcp) per direction."""
    if kind == "cubic":
        g = np.arange(n, dtype=np.float64) * d
        X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
        return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    if kind == "fcc":
        a = d * math.sqrt(2.0)                      # cubic cell edge
        basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]]) * a
        g = np.arange(n, dtype=np.float64) * a
        X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
        cells = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
        return (cells[:, None, :] + basis[None, :, :]).reshape(-1, 3)
    if kind == "hcp":
        # triangular layers (spacing d), A B A B stacking, layer distance d sqrt(2/3)
        pts = []
        for k in range(n):
            for j in range(n):
                for i in range(n):
                    x = d * (i + 0.5 * (j % 2) + (0.5 if k % 2 else 0.0))
                    y = d * math.sqrt(3.0) / 2.0 * j + (d / (2.0 * math.sqrt(3.0)) if k % 2 else 0.0)
                    pts.append((x, y, d * math.sqrt(2.0 / 3.0) * k))
        return np.array(pts, dtype=np.float64)
    raise ValueError("lattice kind must be cubic, fcc or hcp")


def lattice_state(kind: str = "fcc", n: int = 8, d: float = 1.0, h: float = 0.75,
                  seed: int = 0, K: float = 1.0, Gamma: float = 2.0, vel: float = 0.01,
                  solid: bool = True):
    """A block of particles on a lattice (Sec. II.A lists rectangular, hcp and
    fcc placing): equal masses (density 1 per unit volume of the lattice),
    smoothing length h, small random velocities, all solid or all fluid."""
    pos = lattice_positions(kind, n, d)
    npts = len(pos)
    vol_per = {"cubic": d ** 3, "fcc": d ** 3 / math.sqrt(2.0), "hcp": d ** 3 / math.sqrt(2.0)}[kind]
    rng = np.random.default_rng(seed)
    st = _empty_state(npts)
    st["x"], st["y"], st["z"] = pos[:, 0].copy(), pos[:, 1].copy(), pos[:, 2].copy()
    v = vel * rng.normal(size=(3, npts))
    st["vx"], st["vy"], st["vz"] = v[0].copy(), v[1].copy(), v[2].copy()
    st["m"][:] = vol_per
    st["h"][:] = h
    st["u"][:] = K / (Gamma - 1.0)
    if solid:
        st["type"][:] = 1
        st["mu"][:] = 0.5
        st["Y0"][:] = 0.1
        st["eps_break"][:] = 0.05
    eos = dict(K=np.array([K]), Gamma=np.array([Gamma]))
    return st, eos


def random_state(n: int, seed: int, box: float | None = None, h_lo: float = 0.5,
                 h_hi: float = 1.2, solid_frac: float = 0.5, vel: float = 0.05,
                 stress: float = 0.02, nstars: int = 1, lattice: bool = False,
                 n_target: float = 40.0):
    """Jittered particle sets with varied h, mixed fluid/solid and random S.

    Used for parity cases with ragged leaves and uneven neighbour counts.
    Stars (if nstars > 1) sit in disjoint, well separated boxes.  Without an
    explicit ``box`` the box edge is chosen so that a particle has about
    ``n_target`` neighbours within the mean support h_a + h_b.
    """
    rng = np.random.default_rng(seed)
    if box is None:
        hs = h_lo + h_hi
        per_star = max(n / max(nstars, 1), 1.0)
        box = (per_star * (4.0 / 3.0) * math.pi * hs ** 3 / n_target) ** (1.0 / 3.0)
    if lattice:
        side = int(round(n ** (1.0 / 3.0)))
        g = np.arange(side, dtype=np.float64) * (box / side)
        X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
        pos = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)[:n]
        pos = pos + rng.uniform(-0.2, 0.2, size=pos.shape) * (box / side)
        n = len(pos)
    else:
        pos = rng.uniform(0.0, box, size=(n, 3))
    st = _empty_state(n)
    star = rng.integers(0, nstars, size=n).astype(np.int32) if nstars > 1 else np.zeros(n, np.int32)
    pos = pos + (star[:, None] * (box * 3.0)) * np.array([1.0, 0.0, 0.0])
    st["x"], st["y"], st["z"] = pos[:, 0].copy(), pos[:, 1].copy(), pos[:, 2].copy()
    v = rng.normal(scale=vel, size=(n, 3))
    st["vx"], st["vy"], st["vz"] = v[:, 0].copy(), v[:, 1].copy(), v[:, 2].copy()
    st["h"][:] = rng.uniform(h_lo, h_hi, size=n)
    st["m"][:] = 1.0
    st["u"][:] = rng.uniform(0.5, 1.5, size=n)
    solid = rng.uniform(size=n) < solid_frac
    st["type"][solid] = 1
    S = rng.normal(scale=stress, size=(6, n))
    S[:3] -= S[:3].mean(axis=0)  # traceless
    st["S"] = np.where(solid[None, :], S, 0.0)
    st["mu"][solid] = rng.uniform(0.2, 0.8, size=int(solid.sum()))
    st["Y0"][solid] = rng.uniform(0.01, 0.1, size=int(solid.sum()))
    st["eps_break"][solid] = 0.05
    st["star"] = star
    eos = dict(K=rng.uniform(0.5, 1.5, size=nstars), Gamma=rng.uniform(1.8, 2.5, size=nstars))
    return st, eos


def ensemble_state(nstars: int = 64, seed: int = 2107, n_lo: float = 1e4, n_hi: float = 2e5,
                   scale_n: float = 1.0, nr: int = 1024):
    """Independent stars in disjoint boxes of one index space.

    N_i log-uniform in [n_lo, n_hi] (times ``scale_n``), Gamma ~ U[1.8, 2.5],
    crust 3-10 % of R, mu/P ~ U[0.005, 0.02], l=0 and l=2 amplitudes
    log-uniform in [1e-4, 1e-2].  Each star targets M = 1.4, R = 12 km.
    Returns (state, eos, metric, params) with per-star ``params``.
    """
    rng = np.random.default_rng(seed)
    Ns = np.round(np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=nstars)) * scale_n)
    Ns = np.maximum(Ns.astype(np.int64), 1)
    Gam = rng.uniform(1.8, 2.5, size=nstars)
    crust = rng.uniform(0.03, 0.10, size=nstars)
    muP = rng.uniform(0.005, 0.02, size=nstars)
    a0 = np.exp(rng.uniform(math.log(1e-4), math.log(1e-2), size=nstars))
    a2 = np.exp(rng.uniform(math.log(1e-4), math.log(1e-2), size=nstars))
    seeds = rng.integers(0, 2 ** 31, size=nstars)
    profs, states, centers = [], [], []
    side = int(math.ceil(nstars ** (1.0 / 3.0)))
    spacing = 12.0 * KM * 2.0 * 1.6
    prof_cache: dict = {}
    for s in range(nstars):
        key = round(float(Gam[s]), 12)
        if key not in prof_cache:
            K, rc = solve_star(float(Gam[s]))
            prof_cache[key] = tov_solve(K, float(Gam[s]), rc)
        prof = prof_cache[key]
        ix, iy, iz = s % side, (s // side) % side, s // (side * side)
        c = (ix * spacing, iy * spacing, iz * spacing)
        st, _, _, _ = star_state(int(Ns[s]), Gamma=float(Gam[s]), seed=int(seeds[s]),
                                 crust_frac=float(crust[s]), mu_over_P=float(muP[s]),
                                 amp_l0=float(a0[s]), amp_l2=float(a2[s]), center=c, prof=prof,
                                 nr=nr)
        st["star"][:] = s
        states.append(st)
        profs.append(prof)
        centers.append(c)
    state = {k: (np.concatenate([t[k] for t in states], axis=-1)) for k in states[0]}
    eos = dict(K=np.array([p.K for p in profs]), Gamma=np.array([p.Gamma for p in profs]))
    metric = metric_tables(profs, centers, nr=nr)
    params = dict(N=Ns, Gamma=Gam, crust=crust, mu_over_P=muP, amp_l0=a0, amp_l2=a2)
    return state, eos, metric, params
