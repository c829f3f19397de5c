// Device helpers shared by the density/screening and force kernels: float
// <-> double conversions that stay off the FP64 pipe, the background metric
// (Sec. I.C) and external field (Sec. II.A) lookups, the equation of state
// and the per-particle finalize step of the force pass.
//
// Mixed precision keeps every per-particle term in FP32.  On this GPU the
// FP64 pipe is narrow, and conversions between float and double issue on it,
// so the mixed kernels convert with integer bit operations instead and take
// positions as the two-float split (Xhi on a power-of-two grid plus an FP32
// remainder) rather than as doubles.
#pragma once

#include "sph_internal.cuh"

namespace sph {

constexpr double kPi = 3.14159265358979323846;
constexpr float kInvPiF = 0.318309886183790671538f;
constexpr double kInvPi = 0.318309886183790671538;

// A float as a double by moving its exponent and mantissa bits: exact for
// zero and normal floats (subnormals, inf and NaN take the conversion
// instruction).
__device__ __forceinline__ double float_to_double_exact(float f)
{
    const uint32_t b = __float_as_uint(f);
    const uint32_t ex = (b >> 23) & 0xffu, man = b & 0x7fffffu;
    const unsigned long long sign = (unsigned long long)(b >> 31) << 63;
    if (ex == 0u) {
        if (man == 0u) return __longlong_as_double((long long)sign);
        return (double)f;
    }
    if (ex == 0xffu) return (double)f;
    const unsigned long long bits =
        sign | ((unsigned long long)(ex - 127u + 1023u) << 52) | ((unsigned long long)man << 29);
    return __longlong_as_double((long long)bits);
}

// A double rounded to the nearest float (ties to even) with integer
// operations.  Doubles whose float is normal are rounded here: the 52-bit
// mantissa loses its low 29 bits, rounding up when they exceed half an ulp
// or equal it with an odd result; a carry out of the 23-bit mantissa moves
// into the exponent (up to infinity).  Magnitudes below 2^-150 give a signed
// zero; float subnormals, infinities and NaN take the conversion instruction.
__device__ __forceinline__ float f64_to_f32_rn(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const uint32_t hi = (uint32_t)(b >> 32);
    const int ex = (int)((hi >> 20) & 0x7ffu);
    const uint32_t sign = hi & 0x80000000u;
    if (ex >= 897 && ex <= 1150) {  // 2^-126 <= |x| < 2^128
        const unsigned long long man = b & 0xfffffffffffffull;
        uint32_t m = (uint32_t)(man >> 29);
        const uint32_t rem = (uint32_t)(man & 0x1fffffffull);
        m += (rem > 0x10000000u || (rem == 0x10000000u && (m & 1u))) ? 1u : 0u;
        const uint32_t fe = (uint32_t)(ex - 1023 + 127);
        return __uint_as_float(sign | ((fe << 23) + m));
    }
    if (ex < 873) return __uint_as_float(sign);  // |x| < 2^-150
    return __double2float_rn(x);
}

template <typename T>
struct MetricPt {
    T alpha, dalpha, psi4, dpsi4;
};

// Static isotropic background (Sec. I.C): linear interpolation of the tables
// on uniform nodes 0..r_max, exterior Schwarzschild in isotropic form beyond.
template <typename T>
__device__ __forceinline__ MetricPt<T> metric_radial(const DevMetric &g, int s, T r)
{
    MetricPt<T> p;
    T rmax, M;
    if (sizeof(T) == 8) {
        rmax = (T)g.r_max[s];
        M = (T)g.M[s];
    } else {
        rmax = (T)g.fstar[s * kFStar + FS_RMAX];
        M = (T)g.fstar[s * kFStar + FS_M];
    }
    if (r <= rmax) {
        T dr = rmax / (T)(g.nr - 1);
        T t = r / dr;
        int i = (int)floor(t);
        i = max(0, min(i, g.nr - 2));
        T f = t - (T)i;
        int64_t o = ((int64_t)s * g.nr + i) * 4;
        T a0, a1, b0, b1, c0, c1, d0, d1;
        if (sizeof(T) == 8) {
            a0 = (T)g.tab[o + 0]; b0 = (T)g.tab[o + 1]; c0 = (T)g.tab[o + 2]; d0 = (T)g.tab[o + 3];
            a1 = (T)g.tab[o + 4]; b1 = (T)g.tab[o + 5]; c1 = (T)g.tab[o + 6]; d1 = (T)g.tab[o + 7];
        } else {
            a0 = (T)g.tabf[o + 0]; b0 = (T)g.tabf[o + 1]; c0 = (T)g.tabf[o + 2]; d0 = (T)g.tabf[o + 3];
            a1 = (T)g.tabf[o + 4]; b1 = (T)g.tabf[o + 5]; c1 = (T)g.tabf[o + 6]; d1 = (T)g.tabf[o + 7];
        }
        p.alpha = a0 + f * (a1 - a0);
        p.dalpha = b0 + f * (b1 - b0);
        p.psi4 = c0 + f * (c1 - c0);
        p.dpsi4 = d0 + f * (d1 - d0);
    } else {
        T k = M / ((T)2 * r);
        T psi = (T)1 + k;
        T dk = -k / r;
        p.alpha = ((T)1 - k) / ((T)1 + k);
        p.dalpha = -(T)2 * dk / (((T)1 + k) * ((T)1 + k));
        p.psi4 = psi * psi * psi * psi;
        p.dpsi4 = (T)4 * psi * psi * psi * dk;
    }
    return p;
}

// Particle position relative to a star centre: FP64 from the sorted FP64
// copies, or FP32 from the two-float split (hi - centre_hi) + (lo - centre_lo).
struct PosD {
    double x, y, z;
};
struct PosF {
    float hx, hy, hz, lx, ly, lz;
};

__device__ __forceinline__ void rel_pos(const double *center, const PosD &p, double c[3])
{
    c[0] = p.x - center[0];
    c[1] = p.y - center[1];
    c[2] = p.z - center[2];
}

__device__ __forceinline__ void rel_pos(const float *chi, const float *clo, const PosF &p, float c[3])
{
    c[0] = (p.hx - chi[0]) + (p.lx - clo[0]);
    c[1] = (p.hy - chi[1]) + (p.ly - clo[1]);
    c[2] = (p.hz - chi[2]) + (p.lz - clo[2]);
}

template <typename T>
__device__ __forceinline__ void metric_from_rel(const DevMetric &g, int s, const T c[3], T &alpha,
                                                T ga[3], T &psi4, T gq[3])
{
    T r = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    MetricPt<T> p = metric_radial<T>(g, s, r);
    T inv = r > (T)0 ? (T)1 / r : (T)0;
    alpha = p.alpha;
    psi4 = p.psi4;
    for (int k = 0; k < 3; ++k) {
        ga[k] = p.dalpha * c[k] * inv;
        gq[k] = p.dpsi4 * c[k] * inv;
    }
}

__device__ __forceinline__ void metric_at(const DevMetric &g, int s, const PosD &p, double &alpha,
                                          double ga[3], double &psi4, double gq[3])
{
    double c[3];
    rel_pos(g.center + 3 * s, p, c);
    metric_from_rel<double>(g, s, c, alpha, ga, psi4, gq);
}

__device__ __forceinline__ void metric_at(const DevMetric &g, int s, const PosF &p, float &alpha,
                                          float ga[3], float &psi4, float gq[3])
{
    float c[3];
    const float *f = g.fstar + s * kFStar;
    rel_pos(f + FS_CHI, f + FS_CLO, p, c);
    metric_from_rel<float>(g, s, c, alpha, ga, psi4, gq);
}

// External field of the relaxation (Sec. II.A) at a particle with velocity v:
// g_eff(r) r_hat from the table, the wall beyond r_wall, and -damping v.
template <typename T>
__device__ __forceinline__ void external_from_rel(const DevMetric &g, int s, const T c[3], T vx,
                                                  T vy, T vz, T acc[3])
{
    T r = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    T gr = (T)0;
    T rmax, rw, kw, d;
    if (sizeof(T) == 8) {
        rmax = (T)g.ext_rmax[s];
        rw = (T)g.ext_rwall[s];
        kw = (T)g.k_wall;
        d = (T)g.damping;
    } else {
        rmax = (T)g.fstar[s * kFStar + FS_EXT_RMAX];
        rw = (T)g.fstar[s * kFStar + FS_EXT_RWALL];
        kw = (T)g.k_wall_f;
        d = (T)g.damping_f;
    }
    if (r <= rmax) {
        T dr = rmax / (T)(g.ext_nr - 1);
        T t = r / dr;
        int i = (int)floor(t);
        i = max(0, min(i, g.ext_nr - 2));
        T f = t - (T)i;
        int64_t o = (int64_t)s * g.ext_nr + i;
        T g0, g1;
        if (sizeof(T) == 8) {
            g0 = (T)g.ext_g[o];
            g1 = (T)g.ext_g[o + 1];
        } else {
            g0 = (T)g.ext_gf[o];
            g1 = (T)g.ext_gf[o + 1];
        }
        gr = g0 + f * (g1 - g0);
    }
    if (r > rw) gr -= kw * (r - rw);
    T inv = r > (T)0 ? (T)1 / r : (T)0;
    acc[0] = gr * c[0] * inv - d * vx;
    acc[1] = gr * c[1] * inv - d * vy;
    acc[2] = gr * c[2] * inv - d * vz;
}

__device__ __forceinline__ void external_at(const DevMetric &g, int s, const PosD &p, double vx,
                                            double vy, double vz, double acc[3])
{
    double c[3];
    rel_pos(g.ext_center + 3 * s, p, c);
    external_from_rel<double>(g, s, c, vx, vy, vz, acc);
}

__device__ __forceinline__ void external_at(const DevMetric &g, int s, const PosF &p, float vx,
                                            float vy, float vz, float acc[3])
{
    float c[3];
    const float *f = g.fstar + s * kFStar;
    rel_pos(f + FS_EXT_CHI, f + FS_EXT_CLO, p, c);
    external_from_rel<float>(g, s, c, vx, vy, vz, acc);
}

// The piece of star s's EoS that holds density rho: K, Gamma and a (FP32
// copies of the tables in mixed precision).
__device__ __forceinline__ void eos_piece_t(const DevEos &e, int s, float rho, float &K, float &G,
                                            float &a)
{
    if (e.npieces <= 1) {
        K = e.Kf[s];
        G = e.Gf[s];
        a = 0.f;
        return;
    }
    int k = 0;
    for (int j = 0; j + 1 < e.npieces; ++j)
        if (rho >= e.rho_bf[s * (e.npieces - 1) + j]) k = j + 1;
    const int o = s * e.npieces + k;
    K = e.Kpf[o];
    G = e.Gpf[o];
    a = e.apf[o];
}

__device__ __forceinline__ void eos_piece_t(const DevEos &e, int s, double rho, double &K,
                                            double &G, double &a)
{
    eos_piece<double>(e, s, rho, K, G, a);
}

// Equation of state and the per-particle factors of the pair sums.
template <typename T>
struct Prep {
    T rho, P, cP, cs, henth, Wt;
};

template <typename T, typename Pos>
__device__ __forceinline__ Prep<T> eos_prep(const DevEos &eos, const DevMetric &g, int star, T D,
                                            T vx, T vy, T vz, const Pos &pos)
{
    Prep<T> p;
    const bool metric = g.kind == 1;
    if (metric) {
        T al, ga[3], q4, gq[3];
        metric_at(g, star, pos, al, ga, q4, gq);
        T v2 = vx * vx + vy * vy + vz * vz;
        T vv = q4 * v2 / (al * al);              // v^i v_i, v^i = xdot^i/alpha
        T Wl = (T)1 / sqrt((T)1 - vv);           // Lorentz factor
        T sqrtg = q4 * sqrt(q4);                 // psi^6
        p.rho = D / (sqrtg * Wl);
        p.Wt = (T)1 / sqrt(al * al - q4 * v2);   // generalised Lorentz factor
    } else {
        p.rho = D;
        p.Wt = (T)1;
    }
    T K, G, ea;
    eos_piece_t(eos, star, p.rho, K, G, ea);
    T rg1 = pow(p.rho, G - (T)1);
    p.P = K * p.rho * rg1;
    T ue = ea + K * rg1 / (G - (T)1);
    p.cP = G * K * rg1;
    p.henth = (T)1 + ue + p.P / p.rho;
    p.cs = metric ? sqrt(p.cP / p.henth) : sqrt(p.cP);
    return p;
}

// A value of the mixed path stored into an FP64 output array.
__device__ __forceinline__ double to_out(float v) { return float_to_double_exact(v); }
__device__ __forceinline__ double to_out(double v) { return v; }
__device__ __forceinline__ float from_state(double v, float) { return f64_to_f32_rn(v); }
__device__ __forceinline__ double from_state(double v, double) { return v; }

// -------------------------------------------------------------- finalize
// Strain rate, rotation rate, stress rate (Eq. solid4), elastic work
// (Eq. solid3) and acceleration, from the reduced pair sums of particle i.
//   G[p][q] = sum_b m_b v_ba^p d_q W_ab  (so eps = (G+G^T)/2D, R = (G-G^T)/2D)
template <typename T, typename Pos>
__device__ __forceinline__ void finalize(int c, int64_t N, const DevState &st,
                                         const DevMaterial &mat, const DevMetric &g, int star,
                                         bool solid, T D, const T aP[3], const T aX[3], T du,
                                         T dD, const T G[3][3], T rho, T cP, T henth, T Wt,
                                         T vx, T vy, T vz, const Pos &pos, const DevRates &out)
{
    T drhodt = D * dD;
    T eps[3][3], R[3][3], dS[3][3];
    for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 3; ++q) {
            eps[p][q] = (T)0;
            R[p][q] = (T)0;
            dS[p][q] = (T)0;
        }
    if (solid) {
        T inv2D = (T)1 / ((T)2 * D);
        for (int p = 0; p < 3; ++p)
            for (int q = 0; q < 3; ++q) {
                eps[p][q] = (G[p][q] + G[q][p]) * inv2D;
                R[p][q] = (G[p][q] - G[q][p]) * inv2D;
            }
        T tr3 = (eps[0][0] + eps[1][1] + eps[2][2]) / (T)3;
        T S6[6];
        for (int k = 0; k < 6; ++k) S6[k] = from_state(st.S[k * N + c], (T)0);
        T Sm[3][3] = {{S6[0], S6[3], S6[4]}, {S6[3], S6[1], S6[5]}, {S6[4], S6[5], S6[2]}};
        T mu = from_state(st.mu[c], (T)0);
        T Seps = (T)0;
        for (int p = 0; p < 3; ++p)
            for (int q = 0; q < 3; ++q) {
                T RS = R[p][0] * Sm[0][q] + R[p][1] * Sm[1][q] + R[p][2] * Sm[2][q];
                T SR = Sm[p][0] * R[0][q] + Sm[p][1] * R[1][q] + Sm[p][2] * R[2][q];
                T J = mat.jaumann == 1 ? SR - RS : RS - SR;
                dS[p][q] = (T)2 * mu * (eps[p][q] - (p == q ? tr3 : (T)0)) + J;
                Seps += Sm[p][q] * eps[p][q];
            }
        du += Seps / D;
    }
    T acc[3];
    if (g.kind == 1) {
        T al, ga[3], q4, gq[3];
        metric_at(g, star, pos, al, ga, q4, gq);
        T xd[3] = {vx, vy, vz};
        T C = g.pressure_form == 1 ? (T)1 / (Wt * rho * henth) : (T)1 / (Wt * Wt * rho * henth);
        T gradP[3] = {-D * aP[0], -D * aP[1], -D * aP[2]};
        T dtP = cP * (rho / D) * drhodt - (xd[0] * gradP[0] + xd[1] * gradP[1] + xd[2] * gradP[2]);
        T v2 = xd[0] * xd[0] + xd[1] * xd[1] + xd[2] * xd[2];
        T vq = xd[0] * gq[0] + xd[1] * gq[1] + xd[2] * gq[2];
        T va = xd[0] * ga[0] + xd[1] * ga[1] + xd[2] * ga[2];
        T gam0 = -(T)2 * al * va;
        for (int k = 0; k < 3; ++k) {
            T gamk = xd[k] * vq + al * ga[k] - (T)0.5 * gq[k] * v2;
            acc[k] = -(C * gradP[k] + gamk) / q4 - (xd[k] / (al * al)) * (C * dtP + gam0) + aX[k];
        }
    } else {
        for (int k = 0; k < 3; ++k) acc[k] = aP[k] + aX[k];
    }
    if (g.ext_kind == 1) {
        T e[3];
        external_at(g, star, pos, vx, vy, vz, e);
        for (int k = 0; k < 3; ++k) acc[k] += e[k];
    }
    out.ax[c] = to_out(acc[0]);
    out.ay[c] = to_out(acc[1]);
    out.az[c] = to_out(acc[2]);
    out.dudt[c] = to_out(du);
    out.drhodt[c] = to_out(drhodt);
    const int ci[6] = {0, 1, 2, 0, 0, 1}, cj[6] = {0, 1, 2, 1, 2, 2};
    for (int k = 0; k < 6; ++k) {
        out.deps[k * N + c] = to_out(eps[ci[k]][cj[k]]);
        out.dS[k * N + c] = to_out(dS[ci[k]][cj[k]]);
    }
    out.dR[c] = to_out(R[0][1]);
    out.dR[N + c] = to_out(R[0][2]);
    out.dR[2 * N + c] = to_out(R[1][2]);
}

// Kernels that consume the sorted order return at entry once a sort pass has
// timed out (ERR_TIMEOUT): the order of that right-hand side is not a
// permutation.  The error word does not change during these kernels.
__device__ __forceinline__ bool order_invalid(const DevScalars *sc)
{
    return (*(volatile const int *)&sc->err & ERR_TIMEOUT) != 0;
}

// A data-dependent index (a list entry or a permutation entry) about to be
// used for an access.  Bounds-checked builds (-DSPH_CHECKED) test
// 0 <= j < n and, outside, raise ERR_BOUNDS and return 0, an index in range,
// so the access stays in bounds and sph_sync reports SPH_ERR_BOUNDS.  Other
// builds return j unchanged.
#ifdef SPH_CHECKED
__device__ __forceinline__ int checked_index(int j, int64_t n, DevScalars *sc)
{
    if (j >= 0 && (int64_t)j < n) return j;
    atomicOr(&sc->err, ERR_BOUNDS);
    return 0;
}
#else
__device__ __forceinline__ int checked_index(int j, int64_t, DevScalars *) { return j; }
#endif

constexpr int kSpinLimit = 1 << 22;  // default polls of a device-side wait before giving up

// Polls a device-side wait may make (DevScalars::spin_limit: 0 the default,
// > 0 that many, < 0 none: the first poll gives up).
__device__ __forceinline__ int spin_limit_of(const DevScalars *sc)
{
    const int v = sc->spin_limit;
    return v == 0 ? kSpinLimit : (v < 0 ? 0 : v);
}

// Particle range [first, end) of leaf l: leaves of one star hold 8
// consecutive sorted particles; several stars read the leaf table.
template <bool MULTI_STAR>
__device__ __forceinline__ int2 leaf_range(const int32_t *leaf_start, int l, int64_t n)
{
    if (MULTI_STAR) return make_int2(leaf_start[l], leaf_start[l + 1]);
    const int lo = kLeaf * l;
    return make_int2(lo, (int)min((int64_t)lo + kLeaf, n));
}

// Spread the 8 nibbles of a 32-bit ballot (lane 4q + s -> bit 4q + s) to the
// low halves of the 8 bytes of a 64-bit word (bit 8q + s).
__device__ __forceinline__ unsigned long long spread_nibbles(uint32_t b)
{
    unsigned long long x = b;
    x = (x | (x << 16)) & 0x0000ffff0000ffffull;
    x = (x | (x << 8)) & 0x00ff00ff00ff00ffull;
    x = (x | (x << 4)) & 0x0f0f0f0f0f0f0f0full;
    return x;
}

}  // namespace sph
