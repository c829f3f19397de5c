/*
 * sph_oracle.c -- plain, slow, FP64 CPU oracle for the SPH right-hand side of
 * elastic-perfectly-plastic matter in a fixed GR background
 * (arXiv 2107.07315, Sec. I.B "Solid SPH Equations" and Sec. I.C "Fixed metric
 * background").
 *
 * THIS FILE IS TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * header, table or constant with the CUDA library; neither includes the other.
 *
 * Design rules followed here:
 *   - every quantity is FP64; no blocking, fusion or reordering beyond what the
 *     equations state; neighbours are found by brute force over all pairs;
 *   - compiled with -ffp-contract=off so that a*b+c is two rounded operations;
 *   - each function names the equation or section it restates.
 *
 * Readings of passages the paper leaves open (kernel form, artificial
 * viscosity, Jaumann sign, metric coordinates, time integrator, h update) are
 * listed in the repository's design notes and repeated at the function that
 * implements each one.
 *
 * Parity status: every function here is pinned by a CPU test
 * (tests/test_oracle_pins.py) against closed forms, invariants, library
 * routines or values printed in the paper.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORA_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Data passed in from Python (numpy arrays, caller order, SoA).             */
/* S, dS, deps are component-major: comp c of particle a at [c*n + a],       */
/* component order xx, yy, zz, xy, xz, yz.  dR holds xy, xz, yz.             */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t n;
    double *x, *y, *z, *vx, *vy, *vz, *u, *h, *m, *S;
    uint8_t *type;   /* 0 fluid core, 1 solid crust (Sec. III) */
    uint8_t *flags;  /* bit0 yielded in the last step, bit1 broken (sticky) */
    int32_t *star;   /* NULL: every particle belongs to star 0 */
    double *mu, *Y0, *eps_break;
} ora_state;

typedef struct {
    int32_t nstars;
    const double *K, *Gamma; /* per star, P = K rho^Gamma (Eq. poly_eos); with pieces: piece 0 */
    /* Piecewise polytrope (Sec. II.A, "several polytropic models ... connected",
     * after Read et al. 2009): npieces 0 or 1 is the single polytrope.  With
     * npieces = p > 1, piece k+1 starts at rho_bound[s*(p-1)+k] (ascending)
     * with exponent Gamma_above[s*(p-1)+k]; its K follows from continuity of
     * P and the constant a of u = a + K rho^(Gamma-1)/(Gamma-1) from
     * continuity of u. */
    int32_t npieces;
    const double *rho_bound, *Gamma_above;
} ora_eos;

typedef struct {
    double alpha_av, beta_av, eta2;
    int32_t jaumann;      /* 0: objective R.S - S.R ; 1: as printed S.R - R.S */
    int32_t yield_mode;   /* 0: f = Y0^2/sv^2 as printed ; 1: f = Y0/sv */
    int32_t break_stress; /* 0: total stress -P I + S ; 1: deviatoric S only */
    int32_t break_zero_S; /* 1: a broken particle loses S and mu */
} ora_material;

typedef struct {
    int32_t kind; /* 0: no background metric ; 1: static isotropic table */
    int32_t nstars, nr;
    int32_t pressure_form; /* 0: 1/(W~^2 rho h) (from div T = 0) ; 1: 1/(W~ rho h) as printed */
    const double *r_max;  /* [nstars] table radius, uniform nodes 0..r_max */
    const double *alpha, *dalpha, *psi4, *dpsi4; /* [nstars*nr] */
    const double *M;      /* [nstars] exterior Schwarzschild mass */
    const double *center; /* [3*nstars] */
} ora_metric;

/* External field of the relaxation (Sec. II.A "particle relaxation"):     */
/* g_eff = -grad phi_eff with phi_eff = -K Gamma rho_t^(Gamma-1)/(Gamma-1)   */
/* for a target profile rho_t(r), tabulated as its radial component g on     */
/* uniform nodes 0..r_max (0 beyond).  Readings (the paper names walls and   */
/* leaves the relaxation's dissipation open): a wall a = -k_wall (r - r_wall) */
/* r_hat beyond r_wall, and velocity damping a = -damping v.                 */
typedef struct {
    int32_t kind; /* 0: none ; 1: radial table */
    int32_t nstars, nr;
    const double *r_max;  /* [nstars] */
    const double *g;      /* [nstars*nr] radial component (negative = inward) */
    const double *center; /* [3*nstars] */
    const double *r_wall; /* [nstars] */
    double k_wall, damping;
} ora_external;

typedef struct {
    double *ax, *ay, *az, *dudt, *drhodt, *rho, *P, *D, *cs;
    double *deps, *dR, *dS; /* 6n, 3n, 6n component-major */
    int32_t *ncount;
} ora_rates;

/* Magnitude scales for cancellation-aware error measures: for each output,
 * the same expression evaluated with every summand replaced by its absolute
 * value (one value per particle; vectors and tensors share one scale). */
typedef struct {
    double *a, *du, *drho, *D, *eps, *dS;
} ora_scales;

/* ------------------------------------------------------------------------ */
/* Smoothing kernel.  The paper uses W_ab = W(|r_a - r_b|, h_ab) with        */
/* h_ab = (h_a + h_b)/2 (Sec. I.B, below Eq. solid4) and leaves the form     */
/* open; the reading is the M4 cubic spline in 3-D with support 2h.          */
/* ------------------------------------------------------------------------ */
double ora_kernel_W(double r, double h)
{
    double sigma = 1.0 / (ORA_PI * h * h * h);
    double q = r / h;
    if (q < 1.0) return sigma * (1.0 - 1.5 * q * q + 0.75 * q * q * q);
    if (q < 2.0) {
        double t = 2.0 - q;
        return sigma * 0.25 * t * t * t;
    }
    return 0.0;
}

double ora_kernel_dWdr(double r, double h)
{
    double sigma = 1.0 / (ORA_PI * h * h * h);
    double q = r / h;
    if (q < 1.0) return (sigma / h) * (-3.0 * q + 2.25 * q * q);
    if (q < 2.0) {
        double t = 2.0 - q;
        return -(sigma / h) * 0.75 * t * t;
    }
    return 0.0;
}

/* ------------------------------------------------------------------------ */
/* Neighbour predicate: b is in N(a) iff b != a, same star, and              */
/* |r_a - r_b| < 2 h_ab = h_a + h_b ("summation is over particles b within   */
/* the support radius of particle a", Sec. I.B).  Written with the fixed     */
/* operation order r2 = (dx*dx + dy*dy) + dz*dz, hs = h_a + h_b, r2 < hs*hs. */
/* ------------------------------------------------------------------------ */
static int star_of(const ora_state *s, int64_t a) { return s->star ? s->star[a] : 0; }

static int is_neighbour(const ora_state *s, int64_t a, int64_t b)
{
    if (a == b) return 0;
    if (star_of(s, a) != star_of(s, b)) return 0;
    double dx = s->x[a] - s->x[b];
    double dy = s->y[a] - s->y[b];
    double dz = s->z[a] - s->z[b];
    double r2 = (dx * dx + dy * dy) + dz * dz;
    double hs = s->h[a] + s->h[b];
    return r2 < hs * hs;
}

/* Brute-force neighbour counts for the listed particles (all if list==NULL). */
void ora_neighbor_counts(const ora_state *s, const int64_t *list, int64_t nlist,
                         int64_t *counts)
{
    int64_t cnt = list ? nlist : s->n;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < cnt; ++k) {
        int64_t a = list ? list[k] : k;
        int64_t c = 0;
        for (int64_t b = 0; b < s->n; ++b) c += is_neighbour(s, a, b);
        counts[k] = c;
    }
}

/* Fill CSR lists (ascending b) given offsets[cnt+1] from the counts above. */
void ora_neighbor_fill(const ora_state *s, const int64_t *list, int64_t nlist,
                       const int64_t *offsets, int64_t *idx)
{
    int64_t cnt = list ? nlist : s->n;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < cnt; ++k) {
        int64_t a = list ? list[k] : k;
        int64_t o = offsets[k];
        for (int64_t b = 0; b < s->n; ++b)
            if (is_neighbour(s, a, b)) idx[o++] = b;
    }
}

/* ------------------------------------------------------------------------ */
/* Background metric (Sec. I.C).  Reading: static, spherically symmetric,    */
/* isotropic coordinates, zero shift:                                        */
/*   ds^2 = -alpha^2 dt^2 + psi^4 delta_ij dx^i dx^j.                        */
/* alpha, alpha', psi^4 and (psi^4)' are tabulated on nodes r_i = i dr,      */
/* dr = r_max/(nr-1), and interpolated linearly; beyond r_max the exterior   */
/* Schwarzschild solution in isotropic form is used:                         */
/*   alpha = (1 - M/2r)/(1 + M/2r),  psi = 1 + M/2r.                         */
/* ------------------------------------------------------------------------ */
typedef struct { double alpha, dalpha, psi4, dpsi4; } ora_metric_pt;

static ora_metric_pt metric_radial(const ora_metric *g, int s, double r)
{
    ora_metric_pt p;
    double rmax = g->r_max[s];
    if (r <= rmax) {
        double dr = rmax / (double)(g->nr - 1);
        double t = r / dr;
        int64_t i = (int64_t)floor(t);
        if (i > g->nr - 2) i = g->nr - 2;
        if (i < 0) i = 0;
        double f = t - (double)i;
        const double *A = g->alpha + (int64_t)s * g->nr;
        const double *dA = g->dalpha + (int64_t)s * g->nr;
        const double *Q = g->psi4 + (int64_t)s * g->nr;
        const double *dQ = g->dpsi4 + (int64_t)s * g->nr;
        p.alpha = A[i] + f * (A[i + 1] - A[i]);
        p.dalpha = dA[i] + f * (dA[i + 1] - dA[i]);
        p.psi4 = Q[i] + f * (Q[i + 1] - Q[i]);
        p.dpsi4 = dQ[i] + f * (dQ[i + 1] - dQ[i]);
    } else {
        double M = g->M[s];
        double k = M / (2.0 * r);
        double psi = 1.0 + k;
        /* d(k)/dr = -k/r */
        double dk = -k / r;
        p.alpha = (1.0 - k) / (1.0 + k);
        p.dalpha = (-dk * (1.0 + k) - (1.0 - k) * dk) / ((1.0 + k) * (1.0 + k));
        p.psi4 = psi * psi * psi * psi;
        p.dpsi4 = 4.0 * psi * psi * psi * dk;
    }
    return p;
}

/* Metric values and Cartesian gradients at a point of star s. */
void ora_metric_eval(const ora_metric *g, int s, double x, double y, double z,
                     double *alpha, double *grad_alpha, double *psi4, double *grad_psi4)
{
    double cx = x - g->center[3 * s + 0];
    double cy = y - g->center[3 * s + 1];
    double cz = z - g->center[3 * s + 2];
    double r = sqrt(cx * cx + cy * cy + cz * cz);
    ora_metric_pt p = metric_radial(g, s, r);
    double e[3] = {0.0, 0.0, 0.0};
    if (r > 0.0) { e[0] = cx / r; e[1] = cy / r; e[2] = cz / r; }
    *alpha = p.alpha;
    *psi4 = p.psi4;
    for (int k = 0; k < 3; ++k) {
        grad_alpha[k] = p.dalpha * e[k];
        grad_psi4[k] = p.dpsi4 * e[k];
    }
}

/*
 * Coordinate acceleration from the fixed-background equation of motion
 * (Sec. I.C, the Tejeda et al. trajectory equation, with W-tilde from the
 * generalised Lorentz factor) for the metric above with xdot^0 = 1:
 *
 *   d2x^i/dt2 = -(g^{i l} - xdot^i g^{0 l}) [ dP_l/(W~ rho h) + Gam_l ],
 *   Gam_l = (d_nu g_{mu l} - 1/2 d_l g_{mu nu}) xdot^mu xdot^nu.
 *
 * With g_00 = -alpha^2, g_ij = psi4 delta_ij, static:
 *   Gam_k = xdot^k (xdot . grad psi4) + alpha d_k alpha - 1/2 d_k psi4 |xdot|^2
 *   Gam_0 = -2 alpha (xdot . grad alpha)
 *   g^{ik} = delta_ik/psi4, g^{00} = -1/alpha^2, g^{0k} = 0.
 *
 * gradP_over: the spatial pressure gradient dP/dx^k already divided by the
 * pressure coefficient's denominator; dtP_over: the Eulerian dP/dt divided
 * by the same.
 *
 * Reading of the pressure coefficient: the equation as printed divides dP by
 * W~ rho h.  Conservation of the stated perfect-fluid T^{mu nu} with
 * u^mu = W~ xdot^mu gives (rho h) u^nu grad_nu u^mu = -(g^{mu nu} +
 * u^mu u^nu) d_nu P, whose coordinate-time form divides dP by W~^2 rho h; only
 * that form leaves a TOV star (Sec. II.A) static, since at rest W~ = 1/alpha
 * and the bracket becomes alpha^2 (dP/(rho h) + d ln alpha).  The default
 * (pressure_form 0) is W~^2 rho h; pressure_form 1 keeps the printed form.
 */
void ora_tejeda_accel(double alpha, const double *grad_alpha, double psi4,
                      const double *grad_psi4, const double *xdot,
                      const double *gradP_over, double dtP_over, double *acc)
{
    double v2 = xdot[0] * xdot[0] + xdot[1] * xdot[1] + xdot[2] * xdot[2];
    double vq = xdot[0] * grad_psi4[0] + xdot[1] * grad_psi4[1] + xdot[2] * grad_psi4[2];
    double va = xdot[0] * grad_alpha[0] + xdot[1] * grad_alpha[1] + xdot[2] * grad_alpha[2];
    double gam0 = -2.0 * alpha * va;
    for (int k = 0; k < 3; ++k) {
        double gamk = xdot[k] * vq + alpha * grad_alpha[k] - 0.5 * grad_psi4[k] * v2;
        acc[k] = -(1.0 / psi4) * (gradP_over[k] + gamk)
                 - (xdot[k] / (alpha * alpha)) * (dtP_over + gam0);
    }
}

/* Generalised Lorentz factor W~ = (-g_mu nu xdot^mu xdot^nu)^(-1/2). */
static double gen_lorentz(double alpha, double psi4, const double *xdot)
{
    double v2 = xdot[0] * xdot[0] + xdot[1] * xdot[1] + xdot[2] * xdot[2];
    return 1.0 / sqrt(alpha * alpha - psi4 * v2);
}

/* ------------------------------------------------------------------------ */
/* Equation of state (Eq. poly_eos and Sec. II.A): P = K rho^Gamma,          */
/* u = K rho^(Gamma-1)/(Gamma-1), dP/drho = Gamma K rho^(Gamma-1),           */
/* Newtonian c_s = sqrt(dP/drho), relativistic c_s = sqrt(dP/drho /          */
/* (1 + u + P/rho)), bulk modulus B = Gamma P (Eq. bulk_modulus).            */
/* ------------------------------------------------------------------------ */
/* The piece of star st's EoS that holds density rho: its K, Gamma and the
 * energy constant a (u = a + K rho^(Gamma-1)/(Gamma-1)). */
void ora_eos_piece(const ora_eos *e, int st, double rho, double *K, double *G, double *a)
{
    double Ki = e->K[st], Gi = e->Gamma[st], ai = 0.0;
    int np = e->npieces > 1 ? e->npieces : 1;
    for (int k = 0; k + 1 < np; ++k) {
        double rb = e->rho_bound[(int64_t)st * (np - 1) + k];
        if (!(rho >= rb)) break;
        double Gn = e->Gamma_above[(int64_t)st * (np - 1) + k];
        double Kn = Ki * pow(rb, Gi - Gn);                        /* P continuous at rb */
        ai += Ki * pow(rb, Gi - 1.0) / (Gi - 1.0) - Kn * pow(rb, Gn - 1.0) / (Gn - 1.0);
        Ki = Kn;
        Gi = Gn;
    }
    *K = Ki;
    *G = Gi;
    *a = ai;
}

/* P, u, dP/drho and c_s of star st at density rho (any number of pieces). */
void ora_eos_eval_star(const ora_eos *e, int st, double rho, int relativistic, double *P,
                       double *u, double *cP, double *cs)
{
    double K, G, a;
    ora_eos_piece(e, st, rho, &K, &G, &a);
    *P = K * pow(rho, G);
    *u = a + K * pow(rho, G - 1.0) / (G - 1.0);
    *cP = G * K * pow(rho, G - 1.0);
    if (relativistic) *cs = sqrt(*cP / (1.0 + *u + *P / rho));
    else *cs = sqrt(*cP);
}

void ora_eos_eval(double K, double Gamma, double rho, int relativistic,
                  double *P, double *u, double *cP, double *cs)
{
    *P = K * pow(rho, Gamma);
    *u = K * pow(rho, Gamma - 1.0) / (Gamma - 1.0);
    *cP = Gamma * K * pow(rho, Gamma - 1.0);
    if (relativistic) *cs = sqrt(*cP / (1.0 + *u + *P / rho));
    else *cs = sqrt(*cP);
}

/* ------------------------------------------------------------------------ */
/* Per-particle quantities derived from the density summation.               */
/* ------------------------------------------------------------------------ */
typedef struct {
    double D, rho, P, ue, cP, cs, PD2;
    double SD2[6];
    double alpha, psi4, grad_alpha[3], grad_psi4[3], Wt, henth;
} ora_prep;

/* Full symmetric 3x3 from the 6-component storage (xx,yy,zz,xy,xz,yz). */
static void sym_full(const double *s6, double M[3][3])
{
    M[0][0] = s6[0]; M[1][1] = s6[1]; M[2][2] = s6[2];
    M[0][1] = M[1][0] = s6[3];
    M[0][2] = M[2][0] = s6[4];
    M[1][2] = M[2][1] = s6[5];
}

static void get_S(const ora_state *s, const double *S, int64_t a, double *s6)
{
    for (int c = 0; c < 6; ++c) s6[c] = S[(int64_t)c * s->n + a];
}

/*
 * Density (Sec. I.C: "The computational density D is recovered from the
 * particle distribution using the standard formula"):
 *   D_a = m_a W(0, h_a) + sum_{b in N(a)} m_b W(r_ab, h_ab),
 * then rho = D/(sqrt(gamma) W) with sqrt(gamma) = psi^6 and W the usual
 * Lorentz factor of v^i = xdot^i/alpha (zero shift); rho = D with no metric.
 */
static void prep_particle(const ora_state *s, const double *vx, const double *vy,
                          const double *vz, const double *S, const ora_eos *eos,
                          const ora_metric *g, int64_t a, const int64_t *nb,
                          int64_t nnb, ora_prep *p)
{
    double D = s->m[a] * ora_kernel_W(0.0, s->h[a]);
    for (int64_t k = 0; k < nnb; ++k) {
        int64_t b = nb[k];
        double dx = s->x[a] - s->x[b];
        double dy = s->y[a] - s->y[b];
        double dz = s->z[a] - s->z[b];
        double r = sqrt(dx * dx + dy * dy + dz * dz);
        double hab = 0.5 * (s->h[a] + s->h[b]);
        D += s->m[b] * ora_kernel_W(r, hab);
    }
    p->D = D;
    int st = star_of(s, a);
    double xdot[3] = {vx[a], vy[a], vz[a]};
    if (g && g->kind == 1) {
        ora_metric_eval(g, st, s->x[a], s->y[a], s->z[a], &p->alpha, p->grad_alpha,
                        &p->psi4, p->grad_psi4);
        double v2 = xdot[0] * xdot[0] + xdot[1] * xdot[1] + xdot[2] * xdot[2];
        double vv = p->psi4 * v2 / (p->alpha * p->alpha); /* v^i v_i */
        double Wl = 1.0 / sqrt(1.0 - vv);
        double sqrtg = p->psi4 * sqrt(p->psi4); /* psi^6 */
        p->rho = D / (sqrtg * Wl);
        p->Wt = gen_lorentz(p->alpha, p->psi4, xdot);
    } else {
        p->alpha = 1.0; p->psi4 = 1.0; p->Wt = 1.0;
        for (int k = 0; k < 3; ++k) { p->grad_alpha[k] = 0.0; p->grad_psi4[k] = 0.0; }
        p->rho = D;
    }
    ora_eos_eval_star(eos, st, p->rho, g && g->kind == 1,
                 &p->P, &p->ue, &p->cP, &p->cs);
    p->henth = 1.0 + p->ue + p->P / p->rho;
    p->PD2 = p->P / (D * D);
    double s6[6];
    get_S(s, S, a, s6);
    for (int c = 0; c < 6; ++c) p->SD2[c] = s6[c] / (D * D);
}

/*
 * Artificial viscosity Pi_ab.  The paper names it (Sec. I.B) without a form;
 * the reading is Monaghan's standard form:
 *   mu_ab = h_ab (v_ab . x_ab)/(r_ab^2 + eta^2 h_ab^2) if v_ab . x_ab < 0,
 *   Pi_ab = (-alpha c_ab mu_ab + beta mu_ab^2)/Dbar_ab, else 0,
 * with c_ab, Dbar_ab the arithmetic means of the two particles' values.
 */
static double art_visc(const ora_material *mat, double hab, double vdx, double r2,
                       double ca, double cb, double Da, double Db)
{
    if (!(vdx < 0.0)) return 0.0;
    double mu = hab * vdx / (r2 + mat->eta2 * hab * hab);
    double cbar = 0.5 * (ca + cb);
    double Dbar = 0.5 * (Da + Db);
    return (-mat->alpha_av * cbar * mu + mat->beta_av * mu * mu) / Dbar;
}

/*
 * Right-hand side for the listed particles (all when list == NULL).
 *
 * Pair sums (Sec. I.B, Eqs. solid1, solid2, solid3, solid5, solid6), with the
 * coordinate density D in place of rho in the pair terms, for b in N(a):
 *   aP_a  = -sum m_b (P_a/D_a^2 + P_b/D_b^2) grad_a W_ab
 *   aV_a  = -sum m_b Pi_ab grad_a W_ab
 *   aS_a^i=  sum m_b (S_a/D_a^2 + S_b/D_b^2)^{ij} d_j W_ab
 *   du_a  =  sum m_b (P_a/D_a^2 + Pi_ab/2) v_ab . grad_a W_ab  (+ S:eps/D)
 *   dD_a  =  D_a sum (m_b/D_b) v_ab . grad_a W_ab
 *   eps^{ij} = 1/(2 D_a) sum m_b (v_ba^i d_j W + v_ba^j d_i W)
 *   R^{ij}   = 1/(2 D_a) sum m_b (v_ba^i d_j W - v_ba^j d_i W)
 * S_b is zero for fluid particles, so the stress sum only has terms when a
 * or b is solid; eps and R are formed for solid a only (fluid: zero).
 *
 * Stress rate (Eq. solid4), solid particles only:
 *   dS/dt = 2 mu (eps - delta tr(eps)/3) + J,
 *   J = R.S - S.R (objective reading, default) or S.R - R.S (as printed).
 *
 * Acceleration: without a metric a = aP + aV + aS.  With the background
 * metric the pressure part enters the trajectory equation of Sec. I.C through
 * dP/dx^i = -D_a aP^i and dP/dt = dP/drho (rho/D) dD/dt - xdot . grad P, and
 * the viscous and elastic parts are added in Newtonian form (Sec. III:
 * Newtonian elastodynamics combined with relativistic hydrodynamics).
 */
/* External acceleration of particle a with velocity v (added to the RHS    */
/* acceleration); *mag receives the sum of the magnitudes of its parts.      */
void ora_external_accel(const ora_external *e, int st, double x, double y, double z,
                        const double *v, double *acc, double *mag)
{
    acc[0] = acc[1] = acc[2] = 0.0;
    *mag = 0.0;
    if (!e || e->kind != 1) return;
    double c[3] = {x - e->center[3 * st + 0], y - e->center[3 * st + 1],
                   z - e->center[3 * st + 2]};
    double r = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    double gr = 0.0;
    double rmax = e->r_max[st];
    if (r <= rmax) {
        double dr = rmax / (double)(e->nr - 1);
        double t = r / dr;
        int i = (int)floor(t);
        if (i > e->nr - 2) i = e->nr - 2;
        if (i < 0) i = 0;
        double f = t - (double)i;
        const double *tab = e->g + (int64_t)st * e->nr;
        gr = tab[i] + f * (tab[i + 1] - tab[i]);
    }
    if (r > e->r_wall[st]) gr -= e->k_wall * (r - e->r_wall[st]);
    if (r > 0.0)
        for (int k = 0; k < 3; ++k) acc[k] = gr * c[k] / r;
    for (int k = 0; k < 3; ++k) acc[k] -= e->damping * v[k];
    *mag = fabs(gr) + e->damping * sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
}

int ora_rhs(const ora_state *s, const double *vx, const double *vy, const double *vz,
            const double *S, const ora_eos *eos, const ora_material *mat,
            const ora_metric *g, const ora_external *ext, const int64_t *list, int64_t nlist,
            ora_rates *out, ora_scales *scl)
{
    int64_t n = s->n;
    int64_t cnt = list ? nlist : n;
    /* The set of particles whose prep is needed: the listed ones and all
     * their neighbours. */
    uint8_t *need = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    int64_t *cnts = (int64_t *)malloc(sizeof(int64_t) * (size_t)(cnt + 1));
    int64_t *offs = (int64_t *)malloc(sizeof(int64_t) * (size_t)(cnt + 1));
    if (!need || !cnts || !offs) { free(need); free(cnts); free(offs); return 1; }
    ora_neighbor_counts(s, list, nlist, cnts);
    offs[0] = 0;
    for (int64_t k = 0; k < cnt; ++k) offs[k + 1] = offs[k] + cnts[k];
    int64_t *nb = (int64_t *)malloc(sizeof(int64_t) * (size_t)(offs[cnt] > 0 ? offs[cnt] : 1));
    if (!nb) { free(need); free(cnts); free(offs); return 1; }
    ora_neighbor_fill(s, list, nlist, offs, nb);
    for (int64_t k = 0; k < cnt; ++k) {
        need[list ? list[k] : k] = 1;
        for (int64_t j = offs[k]; j < offs[k + 1]; ++j) need[nb[j]] = 1;
    }
    int64_t nneed = 0;
    for (int64_t a = 0; a < n; ++a) nneed += need[a];
    int64_t *needlist = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nneed > 0 ? nneed : 1));
    int64_t *slot = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    ora_prep *prep = (ora_prep *)malloc(sizeof(ora_prep) * (size_t)(nneed > 0 ? nneed : 1));
    if (!needlist || !slot || !prep) {
        free(need); free(cnts); free(offs); free(nb); free(needlist); free(slot); free(prep);
        return 1;
    }
    nneed = 0;
    for (int64_t a = 0; a < n; ++a) {
        slot[a] = -1;
        if (need[a]) { slot[a] = nneed; needlist[nneed++] = a; }
    }
    /* Neighbour lists of every needed particle (for its density). */
    int64_t *ncnt = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nneed + 1));
    int64_t *noff = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nneed + 1));
    ora_neighbor_counts(s, needlist, nneed, ncnt);
    noff[0] = 0;
    for (int64_t k = 0; k < nneed; ++k) noff[k + 1] = noff[k] + ncnt[k];
    int64_t *nnb = (int64_t *)malloc(sizeof(int64_t) * (size_t)(noff[nneed] > 0 ? noff[nneed] : 1));
    ora_neighbor_fill(s, needlist, nneed, noff, nnb);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < nneed; ++k)
        prep_particle(s, vx, vy, vz, S, eos, g, needlist[k], nnb + noff[k],
                      noff[k + 1] - noff[k], &prep[k]);

    int metric = g && g->kind == 1;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < cnt; ++k) {
        int64_t a = list ? list[k] : k;
        const ora_prep *pa = &prep[slot[a]];
        int solid_a = s->type[a] == 1;
        double aP[3] = {0, 0, 0}, aV[3] = {0, 0, 0}, aS[3] = {0, 0, 0};
        double du = 0.0, dD = 0.0;
        double G[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}; /* sum m_b v_ba^i d_j W */
        double sP = 0.0, sV = 0.0, sS = 0.0, sdu = 0.0, sdD = 0.0, sG = 0.0; /* magnitudes */
        double va[3] = {vx[a], vy[a], vz[a]};
        for (int64_t j = offs[k]; j < offs[k + 1]; ++j) {
            int64_t b = nb[j];
            const ora_prep *pb = &prep[slot[b]];
            double dx[3] = {s->x[a] - s->x[b], s->y[a] - s->y[b], s->z[a] - s->z[b]};
            double r2 = dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2];
            double r = sqrt(r2);
            double hab = 0.5 * (s->h[a] + s->h[b]);
            double gradW[3] = {0, 0, 0};
            if (r > 0.0) {
                double dW = ora_kernel_dWdr(r, hab);
                for (int i = 0; i < 3; ++i) gradW[i] = dW * dx[i] / r;
            }
            double dv[3] = {va[0] - vx[b], va[1] - vy[b], va[2] - vz[b]}; /* v_ab */
            double vdx = dv[0] * dx[0] + dv[1] * dx[1] + dv[2] * dx[2];
            double vgW = dv[0] * gradW[0] + dv[1] * gradW[1] + dv[2] * gradW[2];
            double Pi = art_visc(mat, hab, vdx, r2, pa->cs, pb->cs, pa->D, pb->D);
            double mb = s->m[b];
            for (int i = 0; i < 3; ++i) {
                aP[i] -= mb * (pa->PD2 + pb->PD2) * gradW[i];
                aV[i] -= mb * Pi * gradW[i];
            }
            if (solid_a || s->type[b] == 1) {
                double T[3][3], Ta[3][3], Tb[3][3];
                sym_full(pa->SD2, Ta);
                sym_full(pb->SD2, Tb);
                for (int i = 0; i < 3; ++i)
                    for (int jj = 0; jj < 3; ++jj) T[i][jj] = Ta[i][jj] + Tb[i][jj];
                for (int i = 0; i < 3; ++i)
                    for (int jj = 0; jj < 3; ++jj) aS[i] += mb * T[i][jj] * gradW[jj];
            }
            du += mb * (pa->PD2 + 0.5 * Pi) * vgW;
            dD += (mb / pb->D) * vgW;
            {
                double gW = sqrt(gradW[0] * gradW[0] + gradW[1] * gradW[1] + gradW[2] * gradW[2]);
                double dvn = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
                double Tn = 0.0;
                for (int c = 0; c < 6; ++c) Tn += fabs(pa->SD2[c] + pb->SD2[c]) * (c < 3 ? 1.0 : 2.0);
                sP += mb * (fabs(pa->PD2) + fabs(pb->PD2)) * gW;
                sV += mb * fabs(Pi) * gW;
                sS += mb * Tn * gW;
                sdu += mb * (fabs(pa->PD2) + 0.5 * fabs(Pi)) * dvn * gW;
                sdD += (mb / pb->D) * dvn * gW;
                sG += mb * dvn * gW;
            }
            if (solid_a)
                for (int i = 0; i < 3; ++i)
                    for (int jj = 0; jj < 3; ++jj) G[i][jj] += mb * (-dv[i]) * gradW[jj];
        }
        double Da = pa->D;
        double drhodt = Da * dD;
        double eps[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, R[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        double dS[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        if (solid_a) {
            double Sa6[6], Sa[3][3];
            get_S(s, S, a, Sa6);
            sym_full(Sa6, Sa);
            for (int i = 0; i < 3; ++i)
                for (int jj = 0; jj < 3; ++jj) {
                    eps[i][jj] = (G[i][jj] + G[jj][i]) / (2.0 * Da);
                    R[i][jj] = (G[i][jj] - G[jj][i]) / (2.0 * Da);
                }
            double tr = eps[0][0] + eps[1][1] + eps[2][2];
            double mu = s->mu[a];
            for (int i = 0; i < 3; ++i)
                for (int jj = 0; jj < 3; ++jj) {
                    double RS = 0.0, SR = 0.0;
                    for (int l = 0; l < 3; ++l) {
                        RS += R[i][l] * Sa[l][jj];
                        SR += Sa[i][l] * R[l][jj];
                    }
                    double J = mat->jaumann == 1 ? (SR - RS) : (RS - SR);
                    dS[i][jj] = 2.0 * mu * (eps[i][jj] - (i == jj ? tr / 3.0 : 0.0)) + J;
                }
            double Seps = 0.0, Sn = 0.0;
            for (int i = 0; i < 3; ++i)
                for (int jj = 0; jj < 3; ++jj) {
                    Seps += Sa[i][jj] * eps[i][jj];
                    Sn += fabs(Sa[i][jj]);
                }
            du += Seps / Da;
            sdu += Sn * sG / (Da * Da);
        }
        double acc[3];
        double sa = sP + sV + sS;
        if (metric) {
            double xd2 = va[0] * va[0] + va[1] * va[1] + va[2] * va[2];
            double C0 = g->pressure_form == 1 ? 1.0 / (pa->Wt * pa->rho * pa->henth)
                                              : 1.0 / (pa->Wt * pa->Wt * pa->rho * pa->henth);
            double ga = sqrt(pa->grad_alpha[0] * pa->grad_alpha[0] + pa->grad_alpha[1] * pa->grad_alpha[1] +
                             pa->grad_alpha[2] * pa->grad_alpha[2]);
            double gq = sqrt(pa->grad_psi4[0] * pa->grad_psi4[0] + pa->grad_psi4[1] * pa->grad_psi4[1] +
                             pa->grad_psi4[2] * pa->grad_psi4[2]);
            double xn = sqrt(xd2);
            double sGam = xd2 * gq + pa->alpha * ga + 0.5 * gq * xd2;
            double sdt = pa->cP * (pa->rho / Da) * Da * sdD + xn * Da * sP;
            sa = (C0 * Da * sP + sGam) / pa->psi4 +
                 xn / (pa->alpha * pa->alpha) * (C0 * sdt + 2.0 * pa->alpha * xn * ga) + sV + sS;
        }
        if (scl) {
            scl->a[a] = sa;
            scl->du[a] = sdu;
            scl->drho[a] = Da * sdD;
            scl->D[a] = Da;
            scl->eps[a] = sG / Da;
            if (solid_a) {
                double Sn = 0.0;
                for (int c = 0; c < 6; ++c) Sn += fabs(S[(int64_t)c * n + a]) * (c < 3 ? 1.0 : 2.0);
                scl->dS[a] = 2.0 * fabs(s->mu[a]) * sG / Da + 2.0 * Sn * sG / Da;
            } else {
                scl->dS[a] = 0.0;
            }
        }
        if (metric) {
            double xdot[3] = {va[0], va[1], va[2]};
            double C = g->pressure_form == 1 ? 1.0 / (pa->Wt * pa->rho * pa->henth)
                                             : 1.0 / (pa->Wt * pa->Wt * pa->rho * pa->henth);
            double gradP[3] = {-Da * aP[0], -Da * aP[1], -Da * aP[2]};
            double dtP = pa->cP * (pa->rho / Da) * drhodt
                         - (xdot[0] * gradP[0] + xdot[1] * gradP[1] + xdot[2] * gradP[2]);
            double gpo[3] = {C * gradP[0], C * gradP[1], C * gradP[2]};
            ora_tejeda_accel(pa->alpha, pa->grad_alpha, pa->psi4, pa->grad_psi4, xdot, gpo,
                             C * dtP, acc);
            for (int i = 0; i < 3; ++i) acc[i] += aV[i] + aS[i];
        } else {
            for (int i = 0; i < 3; ++i) acc[i] = aP[i] + aV[i] + aS[i];
        }
        if (ext && ext->kind == 1) {
            double ea[3], em;
            ora_external_accel(ext, star_of(s, a), s->x[a], s->y[a], s->z[a], va, ea, &em);
            for (int i = 0; i < 3; ++i) acc[i] += ea[i];
            if (scl) scl->a[a] += em;
        }
        out->ax[a] = acc[0];
        out->ay[a] = acc[1];
        out->az[a] = acc[2];
        out->dudt[a] = du;
        out->drhodt[a] = drhodt;
        out->rho[a] = pa->rho;
        out->P[a] = pa->P;
        out->D[a] = Da;
        out->cs[a] = pa->cs;
        out->ncount[a] = (int32_t)(offs[k + 1] - offs[k]);
        static const int ci[6] = {0, 1, 2, 0, 0, 1}, cj[6] = {0, 1, 2, 1, 2, 2};
        for (int c = 0; c < 6; ++c) {
            out->deps[(int64_t)c * n + a] = eps[ci[c]][cj[c]];
            out->dS[(int64_t)c * n + a] = dS[ci[c]][cj[c]];
        }
        out->dR[0 * n + a] = R[0][1];
        out->dR[1 * n + a] = R[0][2];
        out->dR[2 * n + a] = R[1][2];
    }
    free(need); free(cnts); free(offs); free(nb); free(needlist); free(slot); free(prep);
    free(ncnt); free(noff); free(nnb);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* von Mises yield by stress scaling (Sec. I.B):                             */
/*   S -> f S, f = min(Y0^2/sv^2, 1), sv = sqrt(3/2 S:S).                    */
/* yield_mode 1 uses f = min(Y0/sv, 1).  f = 1 when sv == 0.                 */
/* ------------------------------------------------------------------------ */
double ora_yield_factor(const double *s6, double Y0, int yield_mode)
{
    double SS = s6[0] * s6[0] + s6[1] * s6[1] + s6[2] * s6[2]
                + 2.0 * (s6[3] * s6[3] + s6[4] * s6[4] + s6[5] * s6[5]);
    double sv2 = 1.5 * SS;
    if (!(sv2 > Y0 * Y0)) return 1.0;
    if (yield_mode == 1) return Y0 / sqrt(sv2);
    return (Y0 * Y0) / sv2;
}

/* ------------------------------------------------------------------------ */
/* Principal stresses of a symmetric 3x3 tensor by cyclic Jacobi rotations   */
/* (textbook method; the paper only needs the largest, Sec. I.B max-strain   */
/* damage model).  Eigenvalues returned in ascending order.                  */
/* ------------------------------------------------------------------------ */
void ora_sym_eigvals(const double *s6, double *ev)
{
    double A[3][3];
    sym_full(s6, A);
    for (int sweep = 0; sweep < 64; ++sweep) {
        double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
        if (off == 0.0) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                if (A[p][q] == 0.0) continue;
                double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
                double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
                for (int k = 0; k < 3; ++k) { /* A <- A J */
                    double akp = A[k][p], akq = A[k][q];
                    A[k][p] = c * akp - sn * akq;
                    A[k][q] = sn * akp + c * akq;
                }
                for (int k = 0; k < 3; ++k) { /* A <- J^T A */
                    double apk = A[p][k], aqk = A[q][k];
                    A[p][k] = c * apk - sn * aqk;
                    A[q][k] = sn * apk + c * aqk;
                }
                A[p][q] = A[q][p] = 0.0;
            }
    }
    double e[3] = {A[0][0], A[1][1], A[2][2]};
    for (int i = 0; i < 3; ++i)
        for (int j = i + 1; j < 3; ++j)
            if (e[j] < e[i]) { double t = e[i]; e[i] = e[j]; e[j] = t; }
    ev[0] = e[0]; ev[1] = e[1]; ev[2] = e[2];
}

/*
 * Maximum-strain damage test (Sec. I.B): eps = sigma_max/E,
 * E = 9 B mu/(3 B + mu), B = Gamma P (Eq. bulk_modulus for a polytrope).
 * sigma is the total stress -P I + S (tension positive) or S alone.
 * Returns 1 when eps >= eps_break.
 */
int ora_breaks(const double *s6, double P, double Gamma, double mu, double eps_break,
               int break_stress)
{
    double sig[6];
    for (int c = 0; c < 6; ++c) sig[c] = s6[c];
    if (break_stress == 0) { sig[0] -= P; sig[1] -= P; sig[2] -= P; }
    double ev[3];
    ora_sym_eigvals(sig, ev);
    double B = Gamma * P;
    double E = 9.0 * B * mu / (3.0 * B + mu);
    if (!(E > 0.0)) return 0;
    return ev[2] / E >= eps_break;
}

/* ------------------------------------------------------------------------ */
/* Totals: sum m, sum m v, kinetic, internal, total energy, sum m x cross v, */
/* yielded and broken counts, mean neighbour count, centre of mass.          */
/* out[16]: 0 M, 1-3 P, 4 Ekin, 5 Eint, 6 Etot, 7-9 L, 10 n_yielded,         */
/* 11 n_broken, 12 mean ncount, 13-15 centre of mass.                        */
/* ------------------------------------------------------------------------ */
void ora_totals(const ora_state *s, const int32_t *ncount, double *out)
{
    for (int k = 0; k < 16; ++k) out[k] = 0.0;
    double nsum = 0.0;
    for (int64_t a = 0; a < s->n; ++a) {
        double m = s->m[a];
        double v[3] = {s->vx[a], s->vy[a], s->vz[a]};
        double x[3] = {s->x[a], s->y[a], s->z[a]};
        out[0] += m;
        out[1] += m * v[0]; out[2] += m * v[1]; out[3] += m * v[2];
        out[4] += 0.5 * m * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        out[5] += m * s->u[a];
        out[7] += m * (x[1] * v[2] - x[2] * v[1]);
        out[8] += m * (x[2] * v[0] - x[0] * v[2]);
        out[9] += m * (x[0] * v[1] - x[1] * v[0]);
        out[10] += (s->flags[a] & 1) ? 1.0 : 0.0;
        out[11] += (s->flags[a] & 2) ? 1.0 : 0.0;
        if (ncount) nsum += (double)ncount[a];
        out[13] += m * x[0]; out[14] += m * x[1]; out[15] += m * x[2];
    }
    out[6] = out[4] + out[5];
    out[12] = s->n > 0 ? nsum / (double)s->n : 0.0;
    if (out[0] > 0.0) { out[13] /= out[0]; out[14] /= out[0]; out[15] /= out[0]; }
}

/* ------------------------------------------------------------------------ */
/* Time integration.  The paper does not state its integrator; the reading  */
/* is a kick-drift-kick leapfrog whose force evaluation uses the velocity    */
/* and stress predicted to the end of the step:                              */
/*   v' = v + dt/2 a0;  x += dt v';  vp = v' + dt/2 a0 (Sp likewise);        */
/*   (a1, du1, dS1) = RHS(x, vp, Sp);  v = v' + dt/2 a1 (u, S likewise);     */
/* then the yield scaling and the damage test on the updated stress, and    */
/* the smoothing-length update h *= 1.0625 if the neighbour count is below   */
/* nmin, h *= 0.9375 if above nmax (both factors exact in binary).           */
/* rates0 holds the previous rates on entry and the new ones on exit; when   */
/* have_rates == 0 they are first evaluated at the current state.            */
/* ------------------------------------------------------------------------ */
int ora_step(ora_state *s, const ora_eos *eos, const ora_material *mat, const ora_metric *g,
             const ora_external *ext, double dt, int32_t nsteps, int32_t h_nmin, int32_t h_nmax,
             int32_t have_rates, ora_rates *r)
{
    int64_t n = s->n;
    if (!have_rates) {
        if (ora_rhs(s, s->vx, s->vy, s->vz, s->S, eos, mat, g, ext, NULL, 0, r, NULL)) return 1;
    }
    double *vp = (double *)malloc(sizeof(double) * (size_t)(3 * n + 1));
    double *Sp = (double *)malloc(sizeof(double) * (size_t)(6 * n + 1));
    if (!vp || !Sp) { free(vp); free(Sp); return 1; }
    double hdt = 0.5 * dt;
    for (int32_t step = 0; step < nsteps; ++step) {
        for (int64_t a = 0; a < n; ++a) {
            s->vx[a] += hdt * r->ax[a];
            s->vy[a] += hdt * r->ay[a];
            s->vz[a] += hdt * r->az[a];
            s->u[a] += hdt * r->dudt[a];
            s->x[a] += dt * s->vx[a];
            s->y[a] += dt * s->vy[a];
            s->z[a] += dt * s->vz[a];
            vp[a] = s->vx[a] + hdt * r->ax[a];
            vp[n + a] = s->vy[a] + hdt * r->ay[a];
            vp[2 * n + a] = s->vz[a] + hdt * r->az[a];
            for (int c = 0; c < 6; ++c) {
                int64_t i = (int64_t)c * n + a;
                s->S[i] += hdt * r->dS[i];
                Sp[i] = s->S[i] + hdt * r->dS[i];
            }
        }
        if (ora_rhs(s, vp, vp + n, vp + 2 * n, Sp, eos, mat, g, ext, NULL, 0, r, NULL)) {
            free(vp); free(Sp); return 1;
        }
        for (int64_t a = 0; a < n; ++a) {
            s->vx[a] += hdt * r->ax[a];
            s->vy[a] += hdt * r->ay[a];
            s->vz[a] += hdt * r->az[a];
            s->u[a] += hdt * r->dudt[a];
            for (int c = 0; c < 6; ++c) {
                int64_t i = (int64_t)c * n + a;
                s->S[i] += hdt * r->dS[i];
            }
            s->flags[a] &= (uint8_t)~1u;
            if (s->type[a] == 1) {
                double s6[6];
                get_S(s, s->S, a, s6);
                double f = ora_yield_factor(s6, s->Y0[a], mat->yield_mode);
                if (f < 1.0) {
                    for (int c = 0; c < 6; ++c) s->S[(int64_t)c * n + a] = f * s6[c];
                    s->flags[a] |= 1u;
                }
                get_S(s, s->S, a, s6);
                int st = star_of(s, a);
                double Kp, Gp, ap;  /* B = rho dP/drho = Gamma_piece P */
                ora_eos_piece(eos, st, r->rho[a], &Kp, &Gp, &ap);
                if (ora_breaks(s6, r->P[a], Gp, s->mu[a], s->eps_break[a],
                               mat->break_stress)) {
                    s->flags[a] |= 2u;
                    if (mat->break_zero_S) {
                        for (int c = 0; c < 6; ++c) s->S[(int64_t)c * n + a] = 0.0;
                        s->mu[a] = 0.0;
                    }
                }
            }
            if (h_nmax > 0) {
                if (r->ncount[a] < h_nmin) s->h[a] *= 1.0625;
                else if (r->ncount[a] > h_nmax) s->h[a] *= 0.9375;
            }
        }
    }
    free(vp);
    free(Sp);
    return 0;
}

int ora_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void ora_set_threads(int nt)
{
#ifdef _OPENMP
    if (nt > 0) omp_set_num_threads(nt);
#else
    (void)nt;
#endif
}
