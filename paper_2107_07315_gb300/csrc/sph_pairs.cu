// Pair kernels of the right-hand side.
//
// Each particle's exact neighbour list (built by the neighbour search) is
// shared by LPI consecutive threads of a warp; thread `sub` of the group
// takes entries sub, sub+LPI, ...  and the group's partial sums are combined
// with xor shuffles (fixed order, deterministic).
//
//   density : D_a = m_a W(0,h_a) + sum_b m_b W(r_ab, h_ab)    (Sec. I.C, D from
//             the "standard formula"), then the equation of state
//             (Eq. poly_eos, Sec. II.A) and rho = D/(sqrt(gamma) W).
//   force   : pair sums of Eqs. solid1, solid2, solid3, solid5, solid6 with
//             Monaghan viscosity, then per particle: strain and rotation
//             rates, the stress rate of Eq. solid4, the elastic work term of
//             Eq. solid3 and the background force of Sec. I.C.
//
// Mixed precision: pair arithmetic in FP32 on the two-float position split
// (exact Xhi differences plus FP32 remainders), compensated (Kahan) sums for
// D and du/dt, per-particle terms in FP32; FP64 stays with the state.
#include "sph_internal.cuh"

namespace sph {

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr float kInvPiF = 0.318309886183790671538f;
constexpr double kInvPi = 0.318309886183790671538;

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
    T rmax = (T)g.r_max[s];
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
        T M = (T)g.M[s];
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

// Metric value and Cartesian gradients at sorted particle i.
template <typename T>
__device__ __forceinline__ void metric_at(const DevMetric &g, int s, double x, double y, double z,
                                          T &alpha, T ga[3], T &psi4, T gq[3])
{
    T c[3] = {(T)(x - g.center[3 * s + 0]), (T)(y - g.center[3 * s + 1]),
              (T)(z - g.center[3 * s + 2])};
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

// Equation of state and the per-particle factors of the pair sums.
template <typename T>
struct Prep {
    T rho, P, cP, cs, henth, Wt;
};

template <typename T>
__device__ __forceinline__ Prep<T> eos_prep(const DevEos &eos, const DevMetric &g, int star,
                                            T D, T vx, T vy, T vz, double x, double y, double z)
{
    Prep<T> p;
    bool metric = g.kind == 1;
    if (metric) {
        T al, ga[3], q4, gq[3];
        metric_at<T>(g, star, x, y, z, al, ga, q4, gq);
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
    eos_piece<T>(eos, star, p.rho, K, G, ea);
    T rg1 = pow(p.rho, G - (T)1);
    p.P = K * p.rho * rg1;
    T ue = ea + K * rg1 / (G - (T)1);
    p.cP = G * K * rg1;
    p.henth = (T)1 + ue + p.P / p.rho;
    p.cs = metric ? sqrt(p.cP / p.henth) : sqrt(p.cP);
    return p;
}

// Block layout shared by the pair kernels: a block owns PB = (threads/LPI)*R
// consecutive sorted particles.  Phase 1 runs the pair sums: LPI threads
// share one particle's list, threads/LPI particles per round, R rounds; the
// group's sums are combined with xor shuffles (fixed order) and parked in
// shared memory.  Phase 2 gives each of the first PB threads one particle
// for the per-particle work (EoS, finalize).
constexpr int kTB = 128;    // threads per block, mixed precision
constexpr int kTB64 = 64;   // threads per block, FP64
constexpr int kRoundsD = 4;  // phase-1 rounds per block, density kernels
constexpr int kRoundsF = 2;  // phase-1 rounds per block, force kernels

// ------------------------------------------------------------------ density
// 12 blocks per SM (at most 40 registers): the 1e5-particle star's 1563
// blocks then fit in one wave; at 44 registers they took two.
template <int LPI, int R>
__global__ void __launch_bounds__(kTB, 12)
k_density_mixed(int64_t n, DevState st, Scratch s, DevEos eos, DevMetric g, DevRates out, int cap)
{
    constexpr int PB = kTB / LPI * R;  // particles per block
    __shared__ float s_D[PB];
    const int grp = threadIdx.x / LPI, sub = threadIdx.x % LPI;
    const int64_t base = (int64_t)blockIdx.x * PB;
#pragma unroll 1
    for (int r = 0; r < R; ++r) {
        const int slot = r * (kTB / LPI) + grp;
        const int64_t i = base + slot;
        const bool valid = i < n;
        const int cnt = valid ? s.ncnt[i] : 0;
        float4 a0 = make_float4(0.f, 0.f, 0.f, 1.f), a1 = make_float4(0.f, 0.f, 0.f, 0.f);
        if (valid) {
            a0 = s.rec[i];
            a1 = s.rec[n + i];
        }
        float sum = 0.f, comp = 0.f;
        const int32_t *list = s.nbr + i * (int64_t)cap;
        // the next list entry is loaded one iteration ahead, so the record
        // loads of a pair do not wait on their index load
        int jn = sub < cnt ? list[sub] : 0;
        for (int k = sub; k < cnt; k += LPI) {
            int j = jn;
            if (k + LPI < cnt) jn = list[k + LPI];
            float4 q0 = s.rec[j], q1 = s.rec[n + j];
            float dx = (a0.x - q0.x) + (a1.x - q1.x);
            float dy = (a0.y - q0.y) + (a1.y - q1.y);
            float dz = (a0.z - q0.z) + (a1.z - q1.z);
            float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            float hab = 0.5f * (a0.w + q0.w);
            float hinv = __frcp_rn(hab);
            float q = sqrtf(r2) * hinv;
            float sig = hinv * hinv * hinv * kInvPiF;
            float t = 2.f - q;
            float W = q < 1.f ? sig * fmaf(q * q, fmaf(0.75f, q, -1.5f), 1.f) : sig * 0.25f * t * t * t;
            float term = q1.w * W;
            float y = term - comp;
            float tt = sum + y;
            comp = (tt - sum) - y;
            sum = tt;
        }
        for (int o = LPI / 2; o > 0; o >>= 1) {
            sum += __shfl_xor_sync(0xffffffffu, sum, o);
            comp += __shfl_xor_sync(0xffffffffu, comp, o);
        }
        if (sub == 0) {
            float hi = a0.w;
            s_D[slot] = valid ? a1.w * kInvPiF / (hi * hi * hi) + (sum - comp) : 1.f;
        }
    }
    __syncthreads();
    const int64_t i = base + threadIdx.x;
    if (threadIdx.x >= PB || i >= n) return;
    const float D = s_D[threadIdx.x];
    const int c = s.perm[i];
    const int star = st.star ? st.star[c] : 0;
    const float vx = (float)st.vx[c], vy = (float)st.vy[c], vz = (float)st.vz[c];
    Prep<float> p = eos_prep<float>(eos, g, star, D, vx, vy, vz, s.xs[i], s.ys[i], s.zs[i]);
    const float invD = 1.f / D;
    const float PD2 = p.P * invD * invD;
    s.rec[2 * n + i] = make_float4(vx, vy, vz, D);
    s.rec[3 * n + i] = make_float4(PD2, p.cs, invD, s.tys[i] == 1 ? 1.f : 0.f);
    if (s.tys[i] == 1) {
        const int64_t N = st.n;
        const float f = invD * invD;
        s.sd2[i] = make_float4((float)st.S[c] * f, (float)st.S[N + c] * f,
                                       (float)st.S[2 * N + c] * f, (float)st.S[3 * N + c] * f);
        s.sd2[n + i] = make_float4((float)st.S[4 * N + c] * f, (float)st.S[5 * N + c] * f,
                                       0.f, 0.f);
    } else {
        s.sd2[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        s.sd2[n + i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    s.pp[i * 2 + 0] = make_float4(p.rho, p.P, p.cP, p.henth);
    s.pp[i * 2 + 1] = make_float4(p.Wt, p.cs, D, 0.f);
    out.D[c] = D;
    out.rho[c] = p.rho;
    out.P[c] = p.P;
    out.cs[c] = p.cs;
    out.ncount[c] = s.ncnt[i];
}

template <int LPI, int R>
__global__ void __launch_bounds__(kTB64)
k_density_fp64(int64_t n, DevState st, Scratch s, DevEos eos, DevMetric g, DevRates out, int cap)
{
    constexpr int PB = kTB64 / LPI * R;
    __shared__ double s_D[PB];
    const int grp = threadIdx.x / LPI, sub = threadIdx.x % LPI;
    const int64_t base = (int64_t)blockIdx.x * PB;
#pragma unroll 1
    for (int r = 0; r < R; ++r) {
        const int slot = r * (kTB64 / LPI) + grp;
        const int64_t i = base + slot;
        const bool valid = i < n;
        const int cnt = valid ? s.ncnt[i] : 0;
        double4_32a a0 = make_double4_32a(0, 0, 0, 1);
        double mi = 0.0;
        if (valid) {
            a0 = s.rec64[i * 3 + 0];
            mi = s.rec64[i * 3 + 1].x;
        }
        double sum = 0.0;
        const int32_t *list = s.nbr + i * (int64_t)cap;
        for (int k = sub; k < cnt; k += LPI) {
            int j = list[k];
            double4_32a q0 = s.rec64[(int64_t)j * 3 + 0];
            double mj = s.rec64[(int64_t)j * 3 + 1].x;
            double dx = a0.x - q0.x, dy = a0.y - q0.y, dz = a0.z - q0.z;
            double r2 = dx * dx + dy * dy + dz * dz;
            // r from the reciprocal square root (coincident particles: r = 0)
            double r = r2 > 0.0 ? r2 * rsqrt(r2) : 0.0;
            double hab = 0.5 * (a0.w + q0.w);
            // one division per pair: the FP64 pipe is narrow on this GPU
            double hinv = 1.0 / hab;
            double q = r * hinv;
            double sig = kInvPi * hinv * hinv * hinv;
            double W;
            if (q < 1.0) W = sig * (1.0 - 1.5 * q * q + 0.75 * q * q * q);
            else {
                double t = 2.0 - q;
                W = sig * 0.25 * t * t * t;
            }
            sum += mj * W;
        }
        for (int o = LPI / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (sub == 0) {
            double hi = a0.w;
            s_D[slot] = valid ? mi / (kPi * hi * hi * hi) + sum : 1.0;
        }
    }
    __syncthreads();
    const int64_t i = base + threadIdx.x;
    if (threadIdx.x >= PB || i >= n) return;
    const double D = s_D[threadIdx.x];
    const double4_32a a0 = s.rec64[i * 3 + 0];
    const double mi = s.rec64[i * 3 + 1].x;
    const int c = s.perm[i];
    const int star = st.star ? st.star[c] : 0;
    const double vx = st.vx[c], vy = st.vy[c], vz = st.vz[c];
    Prep<double> p = eos_prep<double>(eos, g, star, D, vx, vy, vz, a0.x, a0.y, a0.z);
    const double invD = 1.0 / D;
    const double PD2 = p.P / (D * D);
    s.rec64[i * 3 + 1] = make_double4_32a(mi, vx, vy, vz);
    s.rec64[i * 3 + 2] = make_double4_32a(D, invD, PD2, p.cs);
    double *sd = s.sd264 + i * 8;
    const int64_t N = st.n;
    const bool solid = s.tys[i] == 1;
    for (int k = 0; k < 6; ++k) sd[k] = solid ? st.S[k * N + c] / (D * D) : 0.0;
    double *q = s.pp64 + i * 8;
    q[0] = p.rho; q[1] = p.P; q[2] = p.cP; q[3] = p.henth; q[4] = p.Wt; q[5] = p.cs; q[6] = D;
    out.D[c] = D;
    out.rho[c] = p.rho;
    out.P[c] = p.P;
    out.cs[c] = p.cs;
    out.ncount[c] = s.ncnt[i];
}

// External field of the relaxation (Sec. II.A) at a particle with velocity v:
// g_eff(r) r_hat from the table, the wall beyond r_wall, and -damping v.
template <typename T>
__device__ __forceinline__ void external_at(const DevMetric &g, int s, double x, double y,
                                            double z, T vx, T vy, T vz, T acc[3])
{
    T c[3] = {(T)(x - g.ext_center[3 * s + 0]), (T)(y - g.ext_center[3 * s + 1]),
              (T)(z - g.ext_center[3 * s + 2])};
    T r = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    T gr = (T)0;
    T rmax = (T)g.ext_rmax[s];
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
    T rw = (T)g.ext_rwall[s];
    if (r > rw) gr -= (T)g.k_wall * (r - rw);
    T inv = r > (T)0 ? (T)1 / r : (T)0;
    T d = (T)g.damping;
    acc[0] = gr * c[0] * inv - d * vx;
    acc[1] = gr * c[1] * inv - d * vy;
    acc[2] = gr * c[2] * inv - d * vz;
}

// -------------------------------------------------------------- finalize
// Strain rate, rotation rate, stress rate (Eq. solid4), elastic work
// (Eq. solid3) and acceleration, from the reduced pair sums of particle i.
//   G[p][q] = sum_b m_b v_ba^p d_q W_ab  (so eps = (G+G^T)/2D, R = (G-G^T)/2D)
template <typename T>
__device__ __forceinline__ void finalize(int64_t i, int c, int64_t N, const DevState &st,
                                         const DevMaterial &mat, const DevMetric &g, int star,
                                         bool solid, T D, const T aP[3], const T aX[3], T du,
                                         T dD, const T G[3][3], T rho, T cP, T henth, T Wt,
                                         T vx, T vy, T vz, double x, double y, double z,
                                         const DevRates &out)
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
        for (int k = 0; k < 6; ++k) S6[k] = (T)st.S[k * N + c];
        T Sm[3][3] = {{S6[0], S6[3], S6[4]}, {S6[3], S6[1], S6[5]}, {S6[4], S6[5], S6[2]}};
        T mu = (T)st.mu[c];
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
        metric_at<T>(g, star, x, y, z, al, ga, q4, gq);
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
        external_at<T>(g, star, x, y, z, vx, vy, vz, e);
        for (int k = 0; k < 3; ++k) acc[k] += e[k];
    }
    out.ax[c] = (double)acc[0];
    out.ay[c] = (double)acc[1];
    out.az[c] = (double)acc[2];
    out.dudt[c] = (double)du;
    out.drhodt[c] = (double)drhodt;
    const int ci[6] = {0, 1, 2, 0, 0, 1}, cj[6] = {0, 1, 2, 1, 2, 2};
    for (int k = 0; k < 6; ++k) {
        out.deps[k * N + c] = (double)eps[ci[k]][cj[k]];
        out.dS[k * N + c] = (double)dS[ci[k]][cj[k]];
    }
    out.dR[c] = (double)R[0][1];
    out.dR[N + c] = (double)R[0][2];
    out.dR[2 * N + c] = (double)R[1][2];
}

// ------------------------------------------------------------------- force
// Reduced pair sums per particle, in the order stored in shared memory.
enum { A_P0, A_P1, A_P2, A_X0, A_X1, A_X2, A_DU, A_DUC, A_DD, A_G00, A_G01, A_G02, A_G10, A_G11,
       A_G12, A_G20, A_G21, A_G22, A_N };

// Two instantiations share the grid: SOLID = false takes the blocks whose
// particles are all fluid (no stress of its own, no velocity gradient: fewer
// live registers, 8 blocks of 128 threads per SM), SOLID = true the blocks
// holding a solid particle (6 blocks per SM: at most 85 registers, which
// keeps the allocation at 80).  Each returns at once on the other's blocks.
template <int LPI, int R, bool SOLID>
__global__ void __launch_bounds__(kTB, SOLID ? 6 : 8)
k_force_mixed(int64_t n, DevState st, Scratch s, DevEos eos, DevMaterial mat, DevMetric g,
              DevRates out, int cap)
{
    (void)eos;
    constexpr int PB = kTB / LPI * R;
    __shared__ float s_acc[A_N][PB];
    const int grp = threadIdx.x / LPI, sub = threadIdx.x % LPI;
    const int64_t base = (int64_t)blockIdx.x * PB;
    {
        const int64_t ib = base + threadIdx.x;
        const bool mine = threadIdx.x < PB && ib < n && s.tys[ib] == 1;
        if ((__syncthreads_or(mine) != 0) != SOLID) return;
    }
    const float alpha_av = (float)mat.alpha_av, beta_av = (float)mat.beta_av;
    const float eta2 = (float)mat.eta2;
#pragma unroll 1
    for (int r = 0; r < R; ++r) {
        const int slot = r * (kTB / LPI) + grp;
        const int64_t i = base + slot;
        const bool valid = i < n;
        const int cnt = valid ? s.ncnt[i] : 0;
        float4 a0 = make_float4(0.f, 0.f, 0.f, 1.f), a1 = a0, a2 = make_float4(0.f, 0.f, 0.f, 1.f),
               a3 = make_float4(0.f, 0.f, 1.f, 0.f), as0 = make_float4(0.f, 0.f, 0.f, 0.f),
               as1 = as0;
        bool solid_i = false;
        if (valid) {
            a0 = s.rec[i];
            a1 = s.rec[n + i];
            a2 = s.rec[2 * n + i];
            a3 = s.rec[3 * n + i];
            solid_i = SOLID && s.tys[i] == 1;
            if (solid_i) {
                as0 = s.sd2[i];
                as1 = s.sd2[n + i];
            }
        }
        float aP0 = 0.f, aP1 = 0.f, aP2 = 0.f, aX0 = 0.f, aX1 = 0.f, aX2 = 0.f;
        float du = 0.f, duc = 0.f, dD = 0.f;
        float G00 = 0.f, G01 = 0.f, G02 = 0.f, G10 = 0.f, G11 = 0.f, G12 = 0.f, G20 = 0.f,
              G21 = 0.f, G22 = 0.f;
        const int32_t *list = s.nbr + i * (int64_t)cap;
        int jn = sub < cnt ? list[sub] : 0;
        for (int k = sub; k < cnt; k += LPI) {
            const int j = jn;
            if (k + LPI < cnt) jn = list[k + LPI];
            const float4 q0 = s.rec[j], q1 = s.rec[n + j];
            const float4 q2 = s.rec[2 * n + j], q3 = s.rec[3 * n + j];
            const bool solid_j = q3.w != 0.f;  // type rides in the record: no extra load
            float dx = (a0.x - q0.x) + (a1.x - q1.x);
            float dy = (a0.y - q0.y) + (a1.y - q1.y);
            float dz = (a0.z - q0.z) + (a1.z - q1.z);
            float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            float r2c = fmaxf(r2, 1.17549435e-38f);
            float rinv = rsqrtf(r2c);
            float r = r2c * rinv;
            float hab = 0.5f * (a0.w + q0.w);
            float hinv = __frcp_rn(hab);
            float q = r * hinv;
            float hinv2 = hinv * hinv;
            float s5 = hinv2 * hinv2 * hinv * kInvPiF;
            float t = 2.f - q;
            float gW = q < 1.f ? s5 * fmaf(2.25f, q, -3.f) : -0.75f * s5 * t * t * hab * rinv;
            float w = q1.w * gW;
            float dvx = a2.x - q2.x, dvy = a2.y - q2.y, dvz = a2.z - q2.z;
            float vdx = fmaf(dvx, dx, fmaf(dvy, dy, dvz * dz));
            // Monaghan viscosity, zero for receding pairs (select, no branch)
            float muv = __fdividef(hab * vdx, fmaf(eta2 * hab, hab, r2));
            muv = vdx < 0.f ? muv : 0.f;
            float cbar = 0.5f * (a3.y + q3.y);
            float Pi = fmaf(-alpha_av * cbar, muv, beta_av * muv * muv) *
                       __fdividef(2.f, a2.w + q2.w);
            float fp = (a3.x + q3.x) * w;
            float fv = Pi * w;
            aP0 = fmaf(-fp, dx, aP0);
            aP1 = fmaf(-fp, dy, aP1);
            aP2 = fmaf(-fp, dz, aP2);
            aX0 = fmaf(-fv, dx, aX0);
            aX1 = fmaf(-fv, dy, aX1);
            aX2 = fmaf(-fv, dz, aX2);
            float vw = vdx * w;
            float term = fmaf(0.5f, Pi, a3.x) * vw;
            float yk = term - duc;
            float tk = du + yk;
            duc = (tk - du) - yk;
            du = tk;
            dD = fmaf(vw, q3.z, dD);
            if (solid_i || solid_j) {
                float wx = w * dx, wy = w * dy, wz = w * dz;
                float4 b0 = make_float4(0.f, 0.f, 0.f, 0.f), b1 = b0;
                if (solid_j) {
                    b0 = s.sd2[j];
                    b1 = s.sd2[n + j];
                }
                float Txx = as0.x + b0.x, Tyy = as0.y + b0.y, Tzz = as0.z + b0.z;
                float Txy = as0.w + b0.w, Txz = as1.x + b1.x, Tyz = as1.y + b1.y;
                aX0 = fmaf(Txx, wx, fmaf(Txy, wy, fmaf(Txz, wz, aX0)));
                aX1 = fmaf(Txy, wx, fmaf(Tyy, wy, fmaf(Tyz, wz, aX1)));
                aX2 = fmaf(Txz, wx, fmaf(Tyz, wy, fmaf(Tzz, wz, aX2)));
                if (solid_i) {
                    G00 = fmaf(-dvx, wx, G00); G01 = fmaf(-dvx, wy, G01); G02 = fmaf(-dvx, wz, G02);
                    G10 = fmaf(-dvy, wx, G10); G11 = fmaf(-dvy, wy, G11); G12 = fmaf(-dvy, wz, G12);
                    G20 = fmaf(-dvz, wx, G20); G21 = fmaf(-dvz, wy, G21); G22 = fmaf(-dvz, wz, G22);
                }
            }
        }
        float acc[A_N] = {aP0, aP1, aP2, aX0, aX1, aX2, du, duc, dD,
                          G00, G01, G02, G10, G11, G12, G20, G21, G22};
#pragma unroll
        for (int a = 0; a < A_N; ++a) {
            float v = acc[a];
            for (int o = LPI / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (sub == 0) s_acc[a][slot] = v;
        }
    }
    __syncthreads();
    const int64_t i = base + threadIdx.x;
    if (threadIdx.x >= PB || i >= n) return;
    const int t = threadIdx.x;
    const int c = s.perm[i];
    const int star = st.star ? st.star[c] : 0;
    const float4 a2 = s.rec[2 * n + i];
    const float4 p0 = s.pp[i * 2 + 0], p1 = s.pp[i * 2 + 1];
    const bool solid_i = SOLID && s.tys[i] == 1;
    float aP[3] = {s_acc[A_P0][t], s_acc[A_P1][t], s_acc[A_P2][t]};
    float aX[3] = {s_acc[A_X0][t], s_acc[A_X1][t], s_acc[A_X2][t]};
    float G[3][3] = {{s_acc[A_G00][t], s_acc[A_G01][t], s_acc[A_G02][t]},
                     {s_acc[A_G10][t], s_acc[A_G11][t], s_acc[A_G12][t]},
                     {s_acc[A_G20][t], s_acc[A_G21][t], s_acc[A_G22][t]}};
    finalize<float>(i, c, st.n, st, mat, g, star, solid_i, a2.w, aP, aX,
                    s_acc[A_DU][t] - s_acc[A_DUC][t], s_acc[A_DD][t], G, p0.x, p0.z, p0.w, p1.x,
                    a2.x, a2.y, a2.z, s.xs[i], s.ys[i], s.zs[i], out);
}

template <int LPI, int R>
__global__ void __launch_bounds__(kTB64)
k_force_fp64(int64_t n, DevState st, Scratch s, DevEos eos, DevMaterial mat, DevMetric g,
             DevRates out, int cap)
{
    (void)eos;
    constexpr int PB = kTB64 / LPI * R;
    __shared__ double s_acc[A_N][PB];
    const int grp = threadIdx.x / LPI, sub = threadIdx.x % LPI;
    const int64_t base = (int64_t)blockIdx.x * PB;
#pragma unroll 1
    for (int r = 0; r < R; ++r) {
        const int slot = r * (kTB64 / LPI) + grp;
        const int64_t i = base + slot;
        const bool valid = i < n;
        const int cnt = valid ? s.ncnt[i] : 0;
        double4_32a a0 = make_double4_32a(0, 0, 0, 1), a1 = make_double4_32a(0, 0, 0, 0),
                    a2 = make_double4_32a(1, 1, 0, 0);
        double sa[6] = {0, 0, 0, 0, 0, 0};
        bool solid_i = false;
        if (valid) {
            a0 = s.rec64[i * 3 + 0];
            a1 = s.rec64[i * 3 + 1];
            a2 = s.rec64[i * 3 + 2];
            solid_i = s.tys[i] == 1;
            if (solid_i)
                for (int k = 0; k < 6; ++k) sa[k] = s.sd264[i * 8 + k];
        }
        double aP[3] = {0, 0, 0}, aX[3] = {0, 0, 0}, du = 0.0, dD = 0.0;
        double G[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        const int32_t *list = s.nbr + i * (int64_t)cap;
        for (int k = sub; k < cnt; k += LPI) {
            const int j = list[k];
            const double4_32a q0 = s.rec64[(int64_t)j * 3 + 0], q1 = s.rec64[(int64_t)j * 3 + 1];
            const double4_32a q2 = s.rec64[(int64_t)j * 3 + 2];
            const bool solid_j = s.tys[j] == 1;
            double dx[3] = {a0.x - q0.x, a0.y - q0.y, a0.z - q0.z};
            double r2 = dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2];
            double hab = 0.5 * (a0.w + q0.w);
            // W'(r)/r with one division and one reciprocal square root per
            // pair (the FP64 pipe is narrow on this GPU):
            //   q < 1: h^-5/pi (2.25 q - 3);  q >= 1: -0.75 h^-4/pi (2 - q)^2 / r
            double hinv = 1.0 / hab;
            double gW = 0.0;
            if (r2 > 0.0) {
                double rinv = rsqrt(r2);
                double q = r2 * rinv * hinv;
                double h2 = hinv * hinv;
                double s4 = kInvPi * h2 * h2;
                if (q < 1.0) gW = s4 * hinv * (2.25 * q - 3.0);
                else {
                    double tq = 2.0 - q;
                    gW = -0.75 * s4 * tq * tq * rinv;
                }
            }
            double w = q1.x * gW;
            double dv[3] = {a1.y - q1.y, a1.z - q1.z, a1.w - q1.w};
            double vdx = dv[0] * dx[0] + dv[1] * dx[1] + dv[2] * dx[2];
            double Pi = 0.0;
            if (vdx < 0.0) {
                // mu = h vdx / den and Pi = (-alpha cbar mu + beta mu^2) / Dbar,
                // over one common denominator den^2 Dbar
                double den = r2 + mat.eta2 * hab * hab;
                double hv = hab * vdx;
                double cbar = 0.5 * (a2.w + q2.w);
                double Dbar = 0.5 * (a2.x + q2.x);
                Pi = (-mat.alpha_av * cbar * hv * den + mat.beta_av * hv * hv) / (den * den * Dbar);
            }
            double fp = (a2.z + q2.z) * w, fv = Pi * w;
            for (int d = 0; d < 3; ++d) {
                aP[d] -= fp * dx[d];
                aX[d] -= fv * dx[d];
            }
            double vw = vdx * w;
            du += (a2.z + 0.5 * Pi) * vw;
            dD += vw * q2.y;
            if (solid_i || solid_j) {
                double wd[3] = {w * dx[0], w * dx[1], w * dx[2]};
                double sb[6] = {0, 0, 0, 0, 0, 0};
                if (solid_j)
                    for (int kk = 0; kk < 6; ++kk) sb[kk] = s.sd264[(int64_t)j * 8 + kk];
                double T[3][3] = {{sa[0] + sb[0], sa[3] + sb[3], sa[4] + sb[4]},
                                  {sa[3] + sb[3], sa[1] + sb[1], sa[5] + sb[5]},
                                  {sa[4] + sb[4], sa[5] + sb[5], sa[2] + sb[2]}};
                for (int pp = 0; pp < 3; ++pp)
                    aX[pp] += T[pp][0] * wd[0] + T[pp][1] * wd[1] + T[pp][2] * wd[2];
                if (solid_i)
                    for (int pp = 0; pp < 3; ++pp)
                        for (int qq = 0; qq < 3; ++qq) G[pp][qq] -= dv[pp] * wd[qq];
            }
        }
        double acc[A_N] = {aP[0], aP[1], aP[2], aX[0], aX[1], aX[2], du, 0.0, dD,
                           G[0][0], G[0][1], G[0][2], G[1][0], G[1][1], G[1][2],
                           G[2][0], G[2][1], G[2][2]};
#pragma unroll
        for (int a = 0; a < A_N; ++a) {
            double v = acc[a];
            for (int o = LPI / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (sub == 0) s_acc[a][slot] = v;
        }
    }
    __syncthreads();
    const int64_t i = base + threadIdx.x;
    if (threadIdx.x >= PB || i >= n) return;
    const int t = threadIdx.x;
    const int c = s.perm[i];
    const int star = st.star ? st.star[c] : 0;
    const double4_32a a0 = s.rec64[i * 3 + 0], a1 = s.rec64[i * 3 + 1], a2 = s.rec64[i * 3 + 2];
    const double *pp = s.pp64 + i * 8;
    const bool solid_i = s.tys[i] == 1;
    double aP[3] = {s_acc[A_P0][t], s_acc[A_P1][t], s_acc[A_P2][t]};
    double aX[3] = {s_acc[A_X0][t], s_acc[A_X1][t], s_acc[A_X2][t]};
    double G[3][3] = {{s_acc[A_G00][t], s_acc[A_G01][t], s_acc[A_G02][t]},
                      {s_acc[A_G10][t], s_acc[A_G11][t], s_acc[A_G12][t]},
                      {s_acc[A_G20][t], s_acc[A_G21][t], s_acc[A_G22][t]}};
    finalize<double>(i, c, st.n, st, mat, g, star, solid_i, a2.x, aP, aX, s_acc[A_DU][t],
                     s_acc[A_DD][t], G, pp[0], pp[2], pp[3], pp[4], a1.y, a1.z, a1.w, a0.x,
                     a0.y, a0.z, out);
}

}  // namespace

// Particles per block of each kernel variant (threads / lanes * rounds).
template <int LPI>
constexpr int pb_mixed(int rounds) { return kTB / LPI * rounds; }
template <int LPI>
constexpr int pb_fp64(int rounds) { return kTB64 / LPI * rounds; }

void launch_density(const DevState &st, const Scratch &s, const DevEos &eos, const DevMetric &g,
                    const DevRates &out, int cap, int lanes, int fp64, cudaStream_t stream)
{
    int64_t n = st.n;
    if (fp64) {
        if (lanes == 4)
            k_density_fp64<4, kRoundsD><<<(int)((n + pb_fp64<4>(kRoundsD) - 1) / pb_fp64<4>(kRoundsD)), kTB64, 0,
                                         stream>>>(n, st, s, eos, g, out, cap);
        else
            k_density_fp64<8, kRoundsD><<<(int)((n + pb_fp64<8>(kRoundsD) - 1) / pb_fp64<8>(kRoundsD)), kTB64, 0,
                                         stream>>>(n, st, s, eos, g, out, cap);
    } else {
        if (lanes == 4)
            k_density_mixed<4, kRoundsD><<<(int)((n + pb_mixed<4>(kRoundsD) - 1) / pb_mixed<4>(kRoundsD)), kTB, 0,
                                          stream>>>(n, st, s, eos, g, out, cap);
        else
            k_density_mixed<8, kRoundsD><<<(int)((n + pb_mixed<8>(kRoundsD) - 1) / pb_mixed<8>(kRoundsD)), kTB, 0,
                                          stream>>>(n, st, s, eos, g, out, cap);
    }
}

void launch_force(const DevState &st, const Scratch &s, const DevEos &eos, const DevMaterial &mat,
                  const DevMetric &g, const DevRates &out, int cap, int lanes, int fp64,
                  cudaStream_t stream, cudaStream_t side, cudaEvent_t fork, cudaEvent_t join)
{
    int64_t n = st.n;
    if (fp64) {
        if (lanes == 4)
            k_force_fp64<4, kRoundsF><<<(int)((n + pb_fp64<4>(kRoundsF) - 1) / pb_fp64<4>(kRoundsF)), kTB64, 0,
                                       stream>>>(n, st, s, eos, mat, g, out, cap);
        else
            k_force_fp64<8, kRoundsF><<<(int)((n + pb_fp64<8>(kRoundsF) - 1) / pb_fp64<8>(kRoundsF)), kTB64, 0,
                                       stream>>>(n, st, s, eos, mat, g, out, cap);
        return;
    }
    // all-fluid blocks on stream; blocks holding a solid particle (same grid)
    // on side when given, so that the two kernels overlap
    const bool fan = side && fork && join;
    cudaStream_t s2 = stream;
    if (fan) {
        cudaEventRecord(fork, stream);
        cudaStreamWaitEvent(side, fork, 0);
        s2 = side;
    }
    if (lanes == 4) {
        const int nb = (int)((n + pb_mixed<4>(kRoundsF) - 1) / pb_mixed<4>(kRoundsF));
        k_force_mixed<4, kRoundsF, true><<<nb, kTB, 0, s2>>>(n, st, s, eos, mat, g, out, cap);
        k_force_mixed<4, kRoundsF, false><<<nb, kTB, 0, stream>>>(n, st, s, eos, mat, g, out, cap);
    } else {
        const int nb = (int)((n + pb_mixed<8>(kRoundsF) - 1) / pb_mixed<8>(kRoundsF));
        k_force_mixed<8, kRoundsF, true><<<nb, kTB, 0, s2>>>(n, st, s, eos, mat, g, out, cap);
        k_force_mixed<8, kRoundsF, false><<<nb, kTB, 0, stream>>>(n, st, s, eos, mat, g, out, cap);
    }
    if (fan) {
        cudaEventRecord(join, side);
        cudaStreamWaitEvent(stream, join, 0);
    }
}

}  // namespace sph
