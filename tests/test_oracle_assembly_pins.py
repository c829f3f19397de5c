"""Pins of the oracle's artificial viscosity, background-metric assembly and
smoothing-length update, each shown to fail on planted mistakes.

The expected values are computed here by hand from the paper's formulas
(Sec. I.B pair sums with Pi_ab; Sec. I.C computational density D = rho
sqrt(gamma) W, generalised Lorentz factor W~ and the trajectory equation) on
inputs small enough to write out, using only the kernel W(r, h) and dW/dr,
which are pinned by their own closed forms.  ``oracle.mutant`` compiles a copy
of the oracle with one planted mistake; every such copy must fail the pin.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2107_07315_gb300 import inputs as I

MAT = dict(I.DEFAULT_MATERIAL)


def _pair_state(xb, va, vb, ha=0.8, hb=1.0, m=1.3, solid=False):
    st = I._empty_state(2)
    st["x"][:] = [0.0, xb[0]]
    st["y"][:] = [0.0, xb[1]]
    st["z"][:] = [0.0, xb[2]]
    st["h"][:] = [ha, hb]
    st["m"][:] = m
    st["vx"][:] = [va[0], vb[0]]
    st["vy"][:] = [va[1], vb[1]]
    st["vz"][:] = [va[2], vb[2]]
    if solid:
        st["type"][:] = 1
        st["mu"][:] = 0.5
    return st


XB = np.array([0.9, 0.2, -0.1])
V_APPROACH = (np.array([0.3, 0.0, 0.1]), np.array([-0.2, 0.05, 0.0]))
K, GAM = 1.0, 2.0
EOS = dict(K=np.array([K]), Gamma=np.array([GAM]))


def _hand_newtonian(st, mat):
    """Two fluid particles, no metric: a, du/dt of both, written out."""
    m = st["m"][0]
    xa = np.array([st["x"][0], st["y"][0], st["z"][0]])
    xb = np.array([st["x"][1], st["y"][1], st["z"][1]])
    va = np.array([st["vx"][0], st["vy"][0], st["vz"][0]])
    vb = np.array([st["vx"][1], st["vy"][1], st["vz"][1]])
    ha, hb = st["h"]
    hab = 0.5 * (ha + hb)
    xab = xa - xb
    r = math.sqrt(xab @ xab)
    Da = m * oracle.kernel_W(0.0, ha) + m * oracle.kernel_W(r, hab)
    Db = m * oracle.kernel_W(0.0, hb) + m * oracle.kernel_W(r, hab)
    Pa, Pb = K * Da ** GAM, K * Db ** GAM
    ca = math.sqrt(GAM * K * Da ** (GAM - 1))
    cb = math.sqrt(GAM * K * Db ** (GAM - 1))
    gradW = oracle.kernel_dWdr(r, hab) * xab / r          # grad_a W_ab
    vab = va - vb
    vdx = vab @ xab
    if vdx < 0:
        mu = hab * vdx / (r * r + mat["eta2"] * hab * hab)
        Pi = (-mat["alpha_av"] * 0.5 * (ca + cb) * mu + mat["beta_av"] * mu * mu) / (0.5 * (Da + Db))
    else:
        Pi = 0.0
    aP = -m * (Pa / Da ** 2 + Pb / Db ** 2) * gradW
    aPi = -m * Pi * gradW
    vg = vab @ gradW
    du_a = m * (Pa / Da ** 2 + 0.5 * Pi) * vg
    du_b = m * (Pb / Db ** 2 + 0.5 * Pi) * vg  # grad_b W_ba = -grad_a W_ab, v_ba = -v_ab
    # particle b: grad_b W_ba = -grad_a W_ab with the same symmetric factors
    return dict(a=np.stack([aP + aPi, -(aP + aPi)]), du=np.array([du_a, du_b]), Pi=Pi,
                duP=np.array([m * Pa / Da ** 2 * vg, m * Pb / Db ** 2 * vg]))


def _check_visc(st, mat=MAT):
    r = oracle.rhs(st, EOS, mat, None)
    hand = _hand_newtonian(st, mat)
    a = np.stack([r["ax"], r["ay"], r["az"]], 1)
    np.testing.assert_allclose(a, hand["a"], rtol=1e-13, atol=1e-15 * np.abs(hand["a"]).max())
    np.testing.assert_allclose(r["dudt"], hand["du"], rtol=1e-13)
    return r, hand


def test_viscosity_approaching_pair_by_hand():
    # Pi_ab of an approaching pair enters the acceleration and du/dt exactly as
    # (-alpha cbar mu + beta mu^2)/Dbar with mu = h_ab v.x/(r^2 + eta^2 h_ab^2)
    st = _pair_state(XB, *V_APPROACH)
    r, hand = _check_visc(st)
    assert hand["Pi"] > 0
    # viscous heating: sum m du_Pi > 0 for an approaching pair
    heat = np.sum(st["m"] * (r["dudt"] - hand["duP"]))
    assert heat > 0


def test_viscosity_receding_pair_is_zero():
    va, vb = V_APPROACH
    st = _pair_state(XB, -va, -vb)  # v_ab . x_ab > 0: receding
    r, hand = _check_visc(st)
    assert hand["Pi"] == 0.0
    np.testing.assert_allclose(r["dudt"], hand["duP"], rtol=1e-13)


VISC_MUTANTS = [
    [("return (-mat->alpha_av * cbar * mu + mat->beta_av * mu * mu) / Dbar;",
      "return (mat->alpha_av * cbar * mu + mat->beta_av * mu * mu) / Dbar;")],
    [("double cbar = 0.5 * (ca + cb);", "double cbar = ca;")],
    [("double Dbar = 0.5 * (Da + Db);", "double Dbar = Da;")],
    [("double mu = hab * vdx / (r2 + mat->eta2 * hab * hab);",
      "double mu = hab * vdx / (r2 + mat->eta2 * hab);")],
    [("double Pi = art_visc(mat, hab, vdx, r2,", "double Pi = art_visc(mat, s->h[a], vdx, r2,")],
    [("if (!(vdx < 0.0)) return 0.0;", "if (!(vdx > 0.0)) return 0.0;")],
]


@pytest.mark.parametrize("edits", VISC_MUTANTS, ids=range(len(VISC_MUTANTS)))
def test_viscosity_pin_detects_planted_mistake(edits, tmp_path):
    with oracle.mutant(edits, str(tmp_path)):
        with pytest.raises(AssertionError):
            st = _pair_state(XB, *V_APPROACH)
            _check_visc(st)
            va, vb = V_APPROACH
            _check_visc(_pair_state(XB, -va, -vb))


# ------------------------------------------------- background metric --------
def _const_metric(alpha, psi4, form=0):
    nr = 2
    return dict(kind=1, nr=nr, r_max=np.array([100.0]),
                alpha=np.full((1, nr), alpha), dalpha=np.zeros((1, nr)),
                psi4=np.full((1, nr), psi4), dpsi4=np.zeros((1, nr)),
                M=np.array([0.1]), center=np.zeros((1, 3)), pressure_form=form)


def _hand_metric(st, alpha, psi4, form):
    """Trajectory equation of Sec. I.C for two fluid particles in a uniform
    (constant alpha, psi) background, receding (no viscosity), by hand."""
    m = st["m"][0]
    X = np.stack([st["x"], st["y"], st["z"]], 1)
    V = np.stack([st["vx"], st["vy"], st["vz"]], 1)
    h = st["h"]
    hab = 0.5 * (h[0] + h[1])
    xab = X[0] - X[1]
    r = math.sqrt(xab @ xab)
    D = np.array([m * oracle.kernel_W(0.0, h[k]) + m * oracle.kernel_W(r, hab) for k in (0, 1)])
    gW = [oracle.kernel_dWdr(r, hab) * xab / r, -oracle.kernel_dWdr(r, hab) * xab / r]
    out = {}
    rho, P, cP, hen, Wt = (np.zeros(2) for _ in range(5))
    for k in (0, 1):
        v2 = V[k] @ V[k]
        W = 1.0 / math.sqrt(1.0 - psi4 * v2 / alpha ** 2)           # v^i = xdot^i/alpha
        rho[k] = D[k] / (psi4 ** 1.5 * W)                            # D = rho sqrt(gamma) W
        P[k] = K * rho[k] ** GAM
        cP[k] = GAM * K * rho[k] ** (GAM - 1)
        hen[k] = 1.0 + K * rho[k] ** (GAM - 1) / (GAM - 1) + P[k] / rho[k]
        Wt[k] = 1.0 / math.sqrt(alpha ** 2 - psi4 * v2)              # W~ = (-g xdot xdot)^-1/2
    acc = np.zeros((2, 3))
    for k in (0, 1):
        o = 1 - k
        aP = -m * (P[k] / D[k] ** 2 + P[o] / D[o] ** 2) * gW[k]
        drho = D[k] * (m / D[o]) * ((V[k] - V[o]) @ gW[k])
        gradP = -D[k] * aP
        dtP = cP[k] * (rho[k] / D[k]) * drho - V[k] @ gradP
        C = 1.0 / (Wt[k] ** 2 * rho[k] * hen[k]) if form == 0 else 1.0 / (Wt[k] * rho[k] * hen[k])
        acc[k] = -(C * gradP) / psi4 - (V[k] / alpha ** 2) * (C * dtP)
    out.update(acc=acc, rho=rho, P=P)
    return out


METRIC_CASES = [(0.8, 1.3, 0), (0.6, 1.7, 1)]


def _check_metric(alpha, psi4, form):
    va = np.array([-0.05, 0.01, 0.0])
    vb = np.array([0.04, -0.02, 0.01])   # receding: v_ab . x_ab > 0 with x_b = XB
    st = _pair_state(XB, va, vb)
    r = oracle.rhs(st, EOS, MAT, _const_metric(alpha, psi4, form))
    hand = _hand_metric(st, alpha, psi4, form)
    np.testing.assert_allclose(r["rho"], hand["rho"], rtol=1e-13)
    np.testing.assert_allclose(r["P"], hand["P"], rtol=1e-13)
    a = np.stack([r["ax"], r["ay"], r["az"]], 1)
    np.testing.assert_allclose(a, hand["acc"], rtol=1e-12, atol=1e-14 * np.abs(hand["acc"]).max())


@pytest.mark.parametrize("alpha,psi4,form", METRIC_CASES)
def test_metric_assembly_uniform_background_by_hand(alpha, psi4, form):
    _check_metric(alpha, psi4, form)


METRIC_MUTANTS = [
    # psi^4 in place of psi^6 = sqrt(gamma)
    [("double sqrtg = p->psi4 * sqrt(p->psi4); /* psi^6 */", "double sqrtg = p->psi4; /* psi^6 */")],
    # sign of grad P = -D aP
    [("double gradP[3] = {-Da * aP[0], -Da * aP[1], -Da * aP[2]};",
      "double gradP[3] = {Da * aP[0], Da * aP[1], Da * aP[2]};")],
    # W~ without the spatial metric
    [("return 1.0 / sqrt(alpha * alpha - psi4 * v2);", "return 1.0 / sqrt(alpha * alpha - v2);")],
    # advective part of dP/dt with the wrong sign
    [("- (xdot[0] * gradP[0] + xdot[1] * gradP[1] + xdot[2] * gradP[2]);",
      "+ (xdot[0] * gradP[0] + xdot[1] * gradP[1] + xdot[2] * gradP[2]);")],
    # Lorentz factor of the density without 1/alpha in v^i
    [("double vv = p->psi4 * v2 / (p->alpha * p->alpha); /* v^i v_i */",
      "double vv = p->psi4 * v2; /* v^i v_i */")],
    # pressure coefficient of form 0 with one power of W~
    [("            double C = g->pressure_form == 1 ? 1.0 / (pa->Wt * pa->rho * pa->henth)\n"
      "                                             : 1.0 / (pa->Wt * pa->Wt * pa->rho * pa->henth);",
      "            double C = g->pressure_form == 1 ? 1.0 / (pa->Wt * pa->rho * pa->henth)\n"
      "                                             : 1.0 / (pa->Wt * pa->rho * pa->henth);")],
]


@pytest.mark.parametrize("edits", METRIC_MUTANTS, ids=range(len(METRIC_MUTANTS)))
def test_metric_pin_detects_planted_mistake(edits, tmp_path):
    with oracle.mutant(edits, str(tmp_path)):
        with pytest.raises(AssertionError):
            for case in METRIC_CASES:
                _check_metric(*case)


def test_minkowski_table_reduces_to_newtonian():
    # alpha = psi = 1: the trajectory equation is special-relativistic Euler,
    # equal to the Newtonian pair sums up to O(v^2, u, P/rho).
    st, eos = I.random_state(400, seed=5, box=5.0, solid_frac=0.0, vel=1e-3, stress=0.0)
    eos = dict(K=np.array([1e-6]), Gamma=np.array([2.0]))
    st["m"][:] *= 3.0                       # densities of order 3, so rho-scalings show
    st["u"][:] = 0.0
    g = _const_metric(1.0, 1.0, 0)
    r0 = oracle.rhs(st, eos, MAT, None)
    r1 = oracle.rhs(st, eos, MAT, g)
    small = (np.max(r1["P"] / r1["rho"]) + 1e-6 / (2.0 - 1.0) * np.max(r1["rho"]) +
             np.max(st["vx"] ** 2 + st["vy"] ** 2 + st["vz"] ** 2))
    a0 = np.stack([r0["ax"], r0["ay"], r0["az"]], 1)
    a1 = np.stack([r1["ax"], r1["ay"], r1["az"]], 1)
    scale = np.abs(a0).max()
    assert np.abs(a1 - a0).max() < 20 * small * scale
    np.testing.assert_allclose(r1["D"], r0["D"], rtol=1e-15)
    # and it is not trivially equal: the metric branch really ran
    assert np.abs(a1 - a0).max() > 0


def test_star_at_rest_residual_falls_with_resolution():
    # A placed TOV star at rest in its own background (Sec. I.C trajectory
    # equation with the SPH pressure gradient): the shell-averaged radial
    # residual mean(a.r_hat)/g is the systematic discretisation error and must
    # fall as N grows (h ~ N^-1/3).  The per-particle scatter is the SPH
    # zeroth-order error of the disordered placement, which does not converge
    # at a fixed neighbour number, so it is not what is compared.
    res = []
    for N in (2000, 16000):
        st, eos, met, prof = I.star_state(N, amp_l0=0.0, crust_frac=0.0, seed=3)
        r = oracle.rhs(st, eos, MAT, met)
        X = np.stack([st["x"], st["y"], st["z"]], 1)
        rr = np.linalg.norm(X, axis=1)
        ar = np.sum(np.stack([r["ax"], r["ay"], r["az"]], 1) * X / rr[:, None], 1)
        R = prof.rbar_s
        edges = np.linspace(0.2, 0.7, 6) * R
        shell = []
        for b0, b1 in zip(edges[:-1], edges[1:]):
            sel = np.where((rr >= b0) & (rr < b1))[0]
            g = [oracle.metric_eval(met, 0, *X[k]) for k in sel]
            gmag = np.mean([al * np.linalg.norm(ga) / q for al, ga, q, _ in g])
            shell.append(abs(ar[sel].mean()) / gmag)
        res.append(np.mean(shell))
    assert res[1] < 0.5 * res[0], res
    assert res[0] < 0.1, res


# ----------------------------------------------------- smoothing length -----
def _h_case():
    st, eos, _, _ = I.cube_state(n_side=8)
    st["vx"][:] *= 0.1
    st["vy"][:] *= 0.1
    st["vz"][:] *= 0.1
    r = oracle.rhs(st, eos, MAT, None)
    vals = np.unique(r["ncount"])
    nmin, nmax = int(vals[len(vals) // 3]), int(vals[2 * len(vals) // 3])
    return st, eos, nmin, nmax


def _check_h(st, eos, nmin, nmax):
    s1, r1 = oracle.step(st, eos, MAT, None, 1e-3, 1, h_nmin=nmin, h_nmax=nmax)
    cnt = r1["ncount"]
    f = np.where(cnt < nmin, 1.0625, np.where(cnt > nmax, 0.9375, 1.0))
    assert np.array_equal(s1["h"], st["h"] * f)
    # every branch and both band edges occur
    assert (cnt < nmin).any() and (cnt > nmax).any()
    assert (cnt == nmin).any() and (cnt == nmax).any()


def test_h_update_multipliers_on_known_counts():
    st, eos, nmin, nmax = _h_case()
    _check_h(st, eos, nmin, nmax)


H_MUTANTS = [
    [("if (r->ncount[a] < h_nmin) s->h[a] *= 1.0625;", "if (r->ncount[a] < h_nmin) s->h[a] *= 0.9375;")],
    [("if (r->ncount[a] < h_nmin) s->h[a] *= 1.0625;", "if (r->ncount[a] <= h_nmin) s->h[a] *= 1.0625;")],
    [("else if (r->ncount[a] > h_nmax) s->h[a] *= 0.9375;",
      "else if (r->ncount[a] >= h_nmax) s->h[a] *= 0.9375;")],
    [("else if (r->ncount[a] > h_nmax) s->h[a] *= 0.9375;",
      "else if (r->ncount[a] > h_nmax) s->h[a] *= 0.9;")],
]


@pytest.mark.parametrize("edits", H_MUTANTS, ids=range(len(H_MUTANTS)))
def test_h_update_pin_detects_planted_mistake(edits, tmp_path):
    st, eos, nmin, nmax = _h_case()
    with oracle.mutant(edits, str(tmp_path)):
        with pytest.raises(AssertionError):
            _check_h(st, eos, nmin, nmax)
