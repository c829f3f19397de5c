// Pair kernels of the right-hand side over the neighbour lists written by the
// tile search (sph_tiles.cu).
//
// Each particle's exact neighbour list is shared by LPI consecutive threads
// of a warp; thread `sub` of the group takes entries sub, sub+LPI, ...  and the
// group's partial sums are combined with xor shuffles (fixed order,
// deterministic).
//
//   density (FP64 path; the mixed path sums the density in the tile kernel):
//             D_a = m_a W(0,h_a) + sum_b m_b W(r_ab, h_ab)   (Sec. I.C, D from
//             the "standard formula"), then the equation of state
//             (Eq. poly_eos, Sec. II.A) and rho = D/(sqrt(gamma) W).
//   force   : pair sums of Eqs. solid1, solid2, solid3, solid5, solid6 with
//             Monaghan viscosity, then per particle: strain and rotation
//             rates, the stress rate of Eq. solid4, the elastic work term of
//             Eq. solid3 and the background force of Sec. I.C.
//
// Mixed precision: pair arithmetic in FP32 on the two-float position split
// (exact Xhi differences plus FP32 remainders), a compensated (Kahan) sum for
// du/dt, per-particle terms in FP32 with integer-emulated conversions to and
// from the FP64 state (no FP64 instruction in the mixed force kernels).
#include <algorithm>

#include "sph_screen.cuh"

namespace sph {

namespace {

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

// ------------------------------------------------------------- density FP64
template <int LPI, int R>
__global__ void __launch_bounds__(kTB64)
k_density_fp64(int64_t n, DevState st, Scratch s, DevEos eos, DevMetric g, DevRates out, int cap)
{
    constexpr int PB = kTB64 / LPI * R;
    __shared__ double s_D[PB];
    if (order_invalid(s.sc)) return;  // uniform across the grid
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
            int j = checked_index(list[k], n, s.sc);
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
    const int c = checked_index(s.perm[i], n, s.sc);
    const int star = st.star ? st.star[c] : 0;
    const double vx = st.vx[c], vy = st.vy[c], vz = st.vz[c];
    const PosD pos{a0.x, a0.y, a0.z};
    Prep<double> p = eos_prep<double>(eos, g, star, D, vx, vy, vz, pos);
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

// ------------------------------------------------------------------- force
// Reduced pair sums per particle, in the order stored in shared memory.
enum { A_P0, A_P1, A_P2, A_X0, A_X1, A_X2, A_DU, A_DUC, A_DD, A_G00, A_G01, A_G02, A_G10, A_G11,
       A_G12, A_G20, A_G21, A_G22, A_N };

// Two instantiations share the grid: SOLID = false takes the blocks whose
// particles are all fluid (no stress of its own, no velocity gradient: fewer
// live registers, 8 blocks of 128 threads per SM), SOLID = true the blocks
// holding a solid particle (6 blocks per SM: at most 85 registers, which
// keeps the allocation at 80).  Each returns at once on the other's blocks.
//
// force_block runs block blk (PB = kTB / LPI * R consecutive sorted
// particles); every thread of the block calls it (one block barrier inside).
template <int LPI, int R>
__host__ __device__ constexpr int force_pb() { return kTB / LPI * R; }

// 1 when block blk of PB particles holds a solid particle (a block barrier).
template <int PB>
__device__ __forceinline__ bool block_has_solid(const Scratch &s, int64_t n, int64_t blk)
{
    const int64_t ib = blk * PB + threadIdx.x;
    const bool mine = threadIdx.x < PB && ib < n && s.tys[ib] == 1;
    return __syncthreads_or(mine) != 0;
}

template <int LPI, int R, bool SOLID>
__device__ __forceinline__ void force_block(int64_t n, const DevState &st, const Scratch &s,
                                            const DevMaterial &mat, const DevMetric &g,
                                            const DevRates &out, int cap, int64_t blk,
                                            float (*s_acc)[force_pb<LPI, R>()])
{
    constexpr int PB = force_pb<LPI, R>();
    const int grp = threadIdx.x / LPI, sub = threadIdx.x % LPI;
    const int64_t base = blk * PB;
    const float alpha_av = mat.alpha_f, beta_av = mat.beta_f, eta2 = mat.eta2_f;
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
        int jn = sub < cnt ? checked_index(list[sub], n, s.sc) : 0;
        for (int k = sub; k < cnt; k += LPI) {
            const int j = jn;
            if (k + LPI < cnt) jn = checked_index(list[k + LPI], n, s.sc);
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
    const int c = checked_index(s.perm[i], n, s.sc);
    const int star = st.star ? st.star[c] : 0;
    const float4 a0 = s.rec[i], a1 = s.rec[n + i];
    const float4 a2 = s.rec[2 * n + i];
    const float4 p0 = s.pp[i * 2 + 0], p1 = s.pp[i * 2 + 1];
    const bool solid_i = SOLID && s.tys[i] == 1;
    float aP[3] = {s_acc[A_P0][t], s_acc[A_P1][t], s_acc[A_P2][t]};
    float aX[3] = {s_acc[A_X0][t], s_acc[A_X1][t], s_acc[A_X2][t]};
    float G[3][3] = {{s_acc[A_G00][t], s_acc[A_G01][t], s_acc[A_G02][t]},
                     {s_acc[A_G10][t], s_acc[A_G11][t], s_acc[A_G12][t]},
                     {s_acc[A_G20][t], s_acc[A_G21][t], s_acc[A_G22][t]}};
    const PosF pos{a0.x, a0.y, a0.z, a1.x, a1.y, a1.z};
    finalize<float>(c, st.n, st, mat, g, star, solid_i, a2.w, aP, aX,
                    s_acc[A_DU][t] - s_acc[A_DUC][t], s_acc[A_DD][t], G, p0.x, p0.z, p0.w, p1.x,
                    a2.x, a2.y, a2.z, pos, out);
}

template <int LPI, int R, bool SOLID>
__global__ void __launch_bounds__(kTB, SOLID ? 6 : 8)
k_force_mixed(int64_t n, DevState st, Scratch s, DevEos eos, DevMaterial mat, DevMetric g,
              DevRates out, int cap)
{
    (void)eos;
    constexpr int PB = force_pb<LPI, R>();
    __shared__ float s_acc[A_N][PB];
    if (order_invalid(s.sc)) return;  // uniform across the grid
    if (block_has_solid<PB>(s, n, blockIdx.x) != SOLID) return;
    force_block<LPI, R, SOLID>(n, st, s, mat, g, out, cap, blockIdx.x, s_acc);
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
    if (order_invalid(s.sc)) return;  // uniform across the grid
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
            const int j = checked_index(list[k], n, s.sc);
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
    const int c = checked_index(s.perm[i], n, s.sc);
    const int star = st.star ? st.star[c] : 0;
    const double4_32a a0 = s.rec64[i * 3 + 0], a1 = s.rec64[i * 3 + 1], a2 = s.rec64[i * 3 + 2];
    const double *pp = s.pp64 + i * 8;
    const bool solid_i = s.tys[i] == 1;
    double aP[3] = {s_acc[A_P0][t], s_acc[A_P1][t], s_acc[A_P2][t]};
    double aX[3] = {s_acc[A_X0][t], s_acc[A_X1][t], s_acc[A_X2][t]};
    double G[3][3] = {{s_acc[A_G00][t], s_acc[A_G01][t], s_acc[A_G02][t]},
                      {s_acc[A_G10][t], s_acc[A_G11][t], s_acc[A_G12][t]},
                      {s_acc[A_G20][t], s_acc[A_G21][t], s_acc[A_G22][t]}};
    const PosD pos{a0.x, a0.y, a0.z};
    finalize<double>(c, st.n, st, mat, g, star, solid_i, a2.x, aP, aX, s_acc[A_DU][t],
                     s_acc[A_DD][t], G, pp[0], pp[2], pp[3], pp[4], a1.y, a1.z, a1.w, pos, out);
}

// ------------------------------------------------------- persistent RHS
// One launch for the exact screening (with the density and equation of
// state) and the force pass of all particles, of one star or of a batch of
// stars in one index space.  Every block loops: it takes the next item from
// the global counter sc->pq_head; items 0 .. nA-1 screen block `item` of
// 128 / LS particles, items nA .. nA+nB-1 run the force pass of block
// item - nA of force_pb<LF, kRoundsF>() particles (stars are contiguous in
// the sorted order, so one star's blocks are consecutive items).
//
// Dependency: a force item reads the density, pressure and stress of every
// neighbour, written by screening items.  A block finishing a screening item
// publishes it (block barrier, device fence, counter sc->pq_done); a force
// item first waits until pq_done == nA.  Every screening item precedes every
// force item in the queue, so when a force item is dequeued every screening
// item has been taken by a running block, and screening items never wait:
// the count always completes, whether or not all blocks are resident.  The
// wait still polls at most spin_limit_of(sc) times (ERR_TIMEOUT, after which
// every force item returns at once; the host reports SPH_ERR_TIMEOUT).
template <int LS, int LF>
__global__ void __launch_bounds__(kTB, 6)
k_rhs_persistent(int64_t n, DevState st, Scratch s, DevEos eos, DevMaterial mat, DevMetric g,
                 DevRates out, int cap, int n_screen, int n_force)
{
    constexpr int PB = force_pb<LF, kRoundsF>();
    __shared__ float s_acc[A_N][PB];
    __shared__ int s_item, s_ok;
    DevScalars *sc = s.sc;
    // one reading for the whole block: a force item of this launch may raise
    // the timeout while the block starts
    if (threadIdx.x == 0) s_ok = order_invalid(sc) ? 0 : 1;
    __syncthreads();
    if (!s_ok) return;
    const int total = n_screen + n_force;
    for (;;) {
        __syncthreads();  // the last item is done with s_acc and s_item
        if (threadIdx.x == 0) s_item = (int)atomicAdd(&sc->pq_head, 1u);
        __syncthreads();
        const int item = s_item;
        if (item >= total) return;
        if (item < n_screen) {
            screen_block<true, LS>(st, s, cap, eos, g, out, (int64_t)item);
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                atomicAdd(&sc->pq_done, 1u);
            }
            continue;
        }
        if (threadIdx.x == 0) {
            const int limit = spin_limit_of(sc);
            int polls = 0, ok = 1;
            while (*(volatile unsigned int *)&sc->pq_done < (unsigned int)n_screen) {
                if (order_invalid(sc) || polls >= limit) {
                    ok = 0;
                    break;
                }
                ++polls;
                __nanosleep(128);
            }
            if (!ok) atomicOr(&sc->err, ERR_TIMEOUT);
            __threadfence();
            s_ok = ok;
        }
        __syncthreads();
        if (!s_ok) return;  // uniform across the block
        const int64_t blk = item - n_screen;
        if (block_has_solid<PB>(s, n, blk))
            force_block<LF, kRoundsF, true>(n, st, s, mat, g, out, cap, blk, s_acc);
        else
            force_block<LF, kRoundsF, false>(n, st, s, mat, g, out, cap, blk, s_acc);
    }
}

}  // namespace

// Particles per block of each kernel variant (threads / lanes * rounds).
template <int LPI>
constexpr int pb_mixed(int rounds) { return kTB / LPI * rounds; }
template <int LPI>
constexpr int pb_fp64(int rounds) { return kTB64 / LPI * rounds; }

void launch_density_fp64(const DevState &st, const Scratch &s, const DevEos &eos,
                         const DevMetric &g, const DevRates &out, int cap, int lanes,
                         cudaStream_t stream)
{
    int64_t n = st.n;
    if (n == 0) return;
    if (lanes == 4)
        k_density_fp64<4, kRoundsD><<<(int)((n + pb_fp64<4>(kRoundsD) - 1) / pb_fp64<4>(kRoundsD)), kTB64, 0,
                                     stream>>>(n, st, s, eos, g, out, cap);
    else
        k_density_fp64<8, kRoundsD><<<(int)((n + pb_fp64<8>(kRoundsD) - 1) / pb_fp64<8>(kRoundsD)), kTB64, 0,
                                     stream>>>(n, st, s, eos, g, out, cap);
}

void launch_force(const DevState &st, const Scratch &s, const DevEos &eos, const DevMaterial &mat,
                  const DevMetric &g, const DevRates &out, int cap, int lanes, int fp64,
                  cudaStream_t stream, cudaStream_t side, cudaEvent_t fork, cudaEvent_t join)
{
    int64_t n = st.n;
    if (n == 0) return;
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

template <int LS, int LF>
static void *persistent_fn()
{
    return (void *)k_rhs_persistent<LS, LF>;
}

static void *persistent_kernel(int screen_lanes, int lanes)
{
    if (screen_lanes == 8) return lanes == 4 ? persistent_fn<8, 4>() : persistent_fn<8, 8>();
    return lanes == 4 ? persistent_fn<4, 4>() : persistent_fn<4, 8>();
}

PersistPlan plan_persistent(int64_t n, int screen_lanes, int lanes)
{
    PersistPlan p;
    const int ps = kScreenThreads / (screen_lanes == 8 ? 8 : 4);
    const int pf = lanes == 4 ? force_pb<4, kRoundsF>() : force_pb<8, kRoundsF>();
    p.n_screen = (int)((n + ps - 1) / ps);
    p.n_force = (int)((n + pf - 1) / pf);
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, persistent_kernel(screen_lanes, lanes),
                                                  kTB, 0);
    p.grid = std::max(1, sms * std::max(per, 1));
    return p;
}

void launch_persistent(const DevState &st, const Scratch &s, const DevEos &eos,
                       const DevMaterial &mat, const DevMetric &g, const DevRates &out, int cap,
                       int screen_lanes, int lanes, const PersistPlan &pp, cudaStream_t stream)
{
    const int64_t n = st.n;
    if (n == 0) return;
    const int grid = std::min(pp.grid, pp.n_screen + pp.n_force);
    if (screen_lanes == 8) {
        if (lanes == 4)
            k_rhs_persistent<8, 4><<<grid, kTB, 0, stream>>>(n, st, s, eos, mat, g, out, cap,
                                                             pp.n_screen, pp.n_force);
        else
            k_rhs_persistent<8, 8><<<grid, kTB, 0, stream>>>(n, st, s, eos, mat, g, out, cap,
                                                             pp.n_screen, pp.n_force);
    } else {
        if (lanes == 4)
            k_rhs_persistent<4, 4><<<grid, kTB, 0, stream>>>(n, st, s, eos, mat, g, out, cap,
                                                             pp.n_screen, pp.n_force);
        else
            k_rhs_persistent<4, 8><<<grid, kTB, 0, stream>>>(n, st, s, eos, mat, g, out, cap,
                                                             pp.n_screen, pp.n_force);
    }
}

}  // namespace sph
