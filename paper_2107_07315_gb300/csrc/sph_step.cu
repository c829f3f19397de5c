// Time-step kernels, totals and neighbour-list export.
//
// Integrator (the paper does not state one; kick-drift-kick leapfrog whose
// force evaluation sees the velocity and stress predicted to the end of the
// step), von Mises scaling and the maximum-strain test of Sec. I.B, and the
// smoothing-length update towards a neighbour-count band.  All FP64, in the
// caller's particle order.
#include "sph_internal.cuh"

namespace sph {

namespace {

// Modification step after a relaxation (Sec. II.A): the specific internal
// energy of the (piecewise) polytrope, u = a + K rho^(Gamma-1)/(Gamma-1), for
// the density of the last right-hand side.
__global__ void k_set_u(StepState s, DevRates r, DevEos eos)
{
    int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a >= s.n) return;
    const int star = s.star ? s.star[a] : 0;
    double K, G, ea;
    eos_piece<double>(eos, star, r.rho[a], K, G, ea);
    s.u[a] = ea + K * pow(r.rho[a], G - 1.0) / (G - 1.0);
}

// Half kick, drift, and the predicted velocity/stress used by the RHS.
__global__ void k_kick_drift(StepState s, DevRates r, double dt)
{
    int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a >= s.n) return;
    const int64_t n = s.n;
    double hdt = 0.5 * dt;
    double ax = r.ax[a], ay = r.ay[a], az = r.az[a];
    double vx = s.vx[a] + hdt * ax, vy = s.vy[a] + hdt * ay, vz = s.vz[a] + hdt * az;
    s.vx[a] = vx;
    s.vy[a] = vy;
    s.vz[a] = vz;
    s.u[a] += hdt * r.dudt[a];
    s.x[a] += dt * vx;
    s.y[a] += dt * vy;
    s.z[a] += dt * vz;
    s.vp[a] = vx + hdt * ax;
    s.vp[n + a] = vy + hdt * ay;
    s.vp[2 * n + a] = vz + hdt * az;
    // the predicted stress is read for solid particles only (the stress pair
    // term and the stress rate of fluid particles are zero), so fluid
    // particles skip it
    if (s.type[a] == 1) {
        for (int c = 0; c < 6; ++c) {
            int64_t i = c * n + a;
            double ds = r.dS[i];
            double Sv = s.S[i] + hdt * ds;
            s.S[i] = Sv;
            s.Sp[i] = Sv + hdt * ds;
        }
    }
}

// Largest eigenvalue of a symmetric 3x3 matrix: closed-form trigonometric
// solution of the characteristic cubic (the three roots of a real symmetric
// matrix are q + 2p cos(phi + 2 pi k/3)), polished by Newton steps on
// det(lambda I - A).
__device__ double max_eigen_sym(const double s[6])
{
    double a11 = s[0], a22 = s[1], a33 = s[2], a12 = s[3], a13 = s[4], a23 = s[5];
    double p1 = a12 * a12 + a13 * a13 + a23 * a23;
    if (p1 == 0.0) return fmax(a11, fmax(a22, a33));
    double q = (a11 + a22 + a33) / 3.0;
    double b11 = a11 - q, b22 = a22 - q, b33 = a33 - q;
    double p2 = b11 * b11 + b22 * b22 + b33 * b33 + 2.0 * p1;
    double p = sqrt(p2 / 6.0);
    double ip = 1.0 / p;
    double c11 = b11 * ip, c22 = b22 * ip, c33 = b33 * ip;
    double c12 = a12 * ip, c13 = a13 * ip, c23 = a23 * ip;
    double detB = c11 * (c22 * c33 - c23 * c23) - c12 * (c12 * c33 - c23 * c13) +
                  c13 * (c12 * c23 - c22 * c13);
    double r = fmin(fmax(0.5 * detB, -1.0), 1.0);
    double phi = acos(r) / 3.0;
    double lam = q + 2.0 * p * cos(phi);
    // characteristic polynomial f(l) = l^3 - t2 l^2 + t1 l - t0
    double t2 = a11 + a22 + a33;
    double t1 = a11 * a22 + a11 * a33 + a22 * a33 - a12 * a12 - a13 * a13 - a23 * a23;
    double t0 = a11 * (a22 * a33 - a23 * a23) - a12 * (a12 * a33 - a23 * a13) +
                a13 * (a12 * a23 - a22 * a13);
    for (int it = 0; it < 2; ++it) {
        double f = ((lam - t2) * lam + t1) * lam - t0;
        double fp = (3.0 * lam - 2.0 * t2) * lam + t1;
        if (!(fabs(fp) > 1e-300)) break;
        double nl = lam - f / fp;
        if (!isfinite(nl)) break;
        lam = nl;
    }
    return lam;
}

// Second half kick, yield scaling, damage test, smoothing-length update.
__global__ void k_kick_return(StepState s, DevRates r, DevEos eos, DevMaterial mat, double dt,
                              int h_nmin, int h_nmax)
{
    int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (a >= s.n) return;
    const int64_t n = s.n;
    double hdt = 0.5 * dt;
    s.vx[a] += hdt * r.ax[a];
    s.vy[a] += hdt * r.ay[a];
    s.vz[a] += hdt * r.az[a];
    s.u[a] += hdt * r.dudt[a];
    uint8_t fl = s.flags[a] & (uint8_t)~1u;
    if (s.type[a] == 1) {
        double S6[6];
        for (int c = 0; c < 6; ++c) S6[c] = s.S[c * n + a] + hdt * r.dS[c * n + a];
        // von Mises: S -> f S, f = min(Y0^2/sv^2, 1), sv^2 = 3/2 S:S
        double SS = S6[0] * S6[0] + S6[1] * S6[1] + S6[2] * S6[2] +
                    2.0 * (S6[3] * S6[3] + S6[4] * S6[4] + S6[5] * S6[5]);
        double sv2 = 1.5 * SS;
        double Y0 = s.Y0[a];
        if (sv2 > Y0 * Y0) {
            double f = mat.yield_mode == 1 ? Y0 / sqrt(sv2) : (Y0 * Y0) / sv2;
            for (int c = 0; c < 6; ++c) S6[c] *= f;
            fl |= 1u;
            SS *= f * f;
        }
        // maximum-strain test: eps = sigma_max/E, E = 9 B mu/(3B + mu), B = Gamma P
        int star = s.star ? s.star[a] : 0;
        double P = r.P[a];
        double Kp, Gp, ap;  // B = rho dP/drho = Gamma P of the piece holding rho
        eos_piece<double>(eos, star, r.rho[a], Kp, Gp, ap);
        double B = Gp * P;
        double mu = s.mu[a];
        double E = 9.0 * B * mu / (3.0 * B + mu);
        if (E > 0.0) {
            double shift = mat.break_stress == 0 ? -P : 0.0;
            // The largest eigenvalue of S is at most sqrt(2/3 S:S); test that
            // bound first and solve the cubic only when it can reach eps_b.
            double bound = shift + sqrt(SS * (2.0 / 3.0)) * (1.0 + 1e-12) + 1e-300;
            double thr = s.eps_break[a] * E;
            if (bound >= thr) {
                double sig[6] = {S6[0] + shift, S6[1] + shift, S6[2] + shift, S6[3], S6[4], S6[5]};
                if (max_eigen_sym(sig) / E >= s.eps_break[a]) {
                    fl |= 2u;
                    if (mat.break_zero_S) {
                        for (int c = 0; c < 6; ++c) S6[c] = 0.0;
                        s.mu[a] = 0.0;
                    }
                }
            }
        }
        for (int c = 0; c < 6; ++c) s.S[c * n + a] = S6[c];
    }
    s.flags[a] = fl;
    if (h_nmax > 0) {
        int cnt = r.ncount[a];
        if (cnt < h_nmin) s.h[a] *= 1.0625;
        else if (cnt > h_nmax) s.h[a] *= 0.9375;
    }
}

constexpr int kTotBlocks = 256;
constexpr int kTotThreads = 256;

// FP64 totals, fixed order: each block reduces a fixed grid-stride slice in
// a fixed tree order, then one block sums the block partials in order.
// Quantities: 0 m, 1-3 m v, 4 m v^2/2, 5 m u, 6 unused, 7-9 m x cross v,
// 10 yielded, 11 broken, 12 neighbour count, 13-15 m x.
__global__ void k_totals_partial(StepState s, const int32_t *ncount, double *partial)
{
    __shared__ double red[16][kTotThreads / 32];
    double acc[16];
    for (int k = 0; k < 16; ++k) acc[k] = 0.0;
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < s.n;
         a += (int64_t)gridDim.x * blockDim.x) {
        double m = s.m[a];
        double v[3] = {s.vx[a], s.vy[a], s.vz[a]};
        double x[3] = {s.x[a], s.y[a], s.z[a]};
        acc[0] += m;
        acc[1] += m * v[0];
        acc[2] += m * v[1];
        acc[3] += m * v[2];
        acc[4] += 0.5 * m * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        acc[5] += m * s.u[a];
        acc[7] += m * (x[1] * v[2] - x[2] * v[1]);
        acc[8] += m * (x[2] * v[0] - x[0] * v[2]);
        acc[9] += m * (x[0] * v[1] - x[1] * v[0]);
        uint8_t f = s.flags[a];
        acc[10] += (f & 1u) ? 1.0 : 0.0;
        acc[11] += (f & 2u) ? 1.0 : 0.0;
        acc[12] += ncount ? (double)ncount[a] : 0.0;
        acc[13] += m * x[0];
        acc[14] += m * x[1];
        acc[15] += m * x[2];
    }
    for (int k = 0; k < 16; ++k) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < 16) {
        double v = 0.0;
        for (int w = 0; w < kTotThreads / 32; ++w) v += red[threadIdx.x][w];
        partial[blockIdx.x * 16 + threadIdx.x] = v;
    }
}

__global__ void k_totals_sum(const double *partial, int nblocks, int64_t n, double *out)
{
    if (threadIdx.x != 0) return;
    double t[16];
    for (int k = 0; k < 16; ++k) t[k] = 0.0;
    for (int b = 0; b < nblocks; ++b)
        for (int k = 0; k < 16; ++k) t[k] += partial[b * 16 + k];
    t[6] = t[4] + t[5];
    t[12] = n > 0 ? t[12] / (double)n : 0.0;
    if (t[0] > 0.0) {
        t[13] /= t[0];
        t[14] /= t[0];
        t[15] /= t[0];
    }
    for (int k = 0; k < 16; ++k) out[k] = t[k];
}

// FP64 totals of each star (one block per star, over the star's caller
// indices in ascending order, fixed reduction order): the quantities of
// k_totals_partial/k_totals_sum for the star's particles alone.
__global__ void k_star_totals(StepState s, const int32_t *ncount, const int64_t *off,
                              const int32_t *idx, double *out)
{
    __shared__ double red[16][kTotThreads / 32];
    const int st = blockIdx.x;
    double acc[16];
    for (int k = 0; k < 16; ++k) acc[k] = 0.0;
    for (int64_t p = off[st] + threadIdx.x; p < off[st + 1]; p += blockDim.x) {
        const int64_t a = idx[p];
        double m = s.m[a];
        double v[3] = {s.vx[a], s.vy[a], s.vz[a]};
        double x[3] = {s.x[a], s.y[a], s.z[a]};
        acc[0] += m;
        acc[1] += m * v[0];
        acc[2] += m * v[1];
        acc[3] += m * v[2];
        acc[4] += 0.5 * m * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        acc[5] += m * s.u[a];
        acc[7] += m * (x[1] * v[2] - x[2] * v[1]);
        acc[8] += m * (x[2] * v[0] - x[0] * v[2]);
        acc[9] += m * (x[0] * v[1] - x[1] * v[0]);
        uint8_t f = s.flags[a];
        acc[10] += (f & 1u) ? 1.0 : 0.0;
        acc[11] += (f & 2u) ? 1.0 : 0.0;
        acc[12] += ncount ? (double)ncount[a] : 0.0;
        acc[13] += m * x[0];
        acc[14] += m * x[1];
        acc[15] += m * x[2];
    }
    for (int k = 0; k < 16; ++k) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    double t[16];
    for (int k = 0; k < 16; ++k) {
        double v = 0.0;
        for (int w = 0; w < kTotThreads / 32; ++w) v += red[k][w];
        t[k] = v;
    }
    const double cnt = (double)(off[st + 1] - off[st]);
    t[6] = t[4] + t[5];
    t[12] = cnt > 0.0 ? t[12] / cnt : 0.0;
    if (t[0] > 0.0) {
        t[13] /= t[0];
        t[14] /= t[0];
        t[15] /= t[0];
    }
    for (int k = 0; k < 16; ++k) out[st * 16 + k] = t[k];
}

__global__ void k_export_counts(const int32_t *perm, const int32_t *ncnt, int64_t n,
                                int64_t *counts_out)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    counts_out[perm[i]] = ncnt[i];
}

// Exclusive scan of n+1 int64 values in place (one block; export path only).
__global__ void k_scan_i64(int64_t *data, int64_t n)
{
    __shared__ int64_t part[1024];
    const int T = blockDim.x;
    int64_t chunk = (n + T - 1) / T;
    int64_t b0 = threadIdx.x * chunk, b1 = min(b0 + chunk, n);
    int64_t s = 0;
    for (int64_t i = b0; i < b1; ++i) s += data[i];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t run = 0;
        for (int t = 0; t < T; ++t) {
            int64_t v = part[t];
            part[t] = run;
            run += v;
        }
    }
    __syncthreads();
    int64_t run = part[threadIdx.x];
    for (int64_t i = b0; i < b1; ++i) {
        int64_t v = data[i];
        data[i] = run;
        run += v;
    }
}

// Row of sorted particle i in caller order: its list as caller indices in
// ascending order (insertion sort).
__global__ void k_export_fill(const int32_t *perm, const int32_t *nbr, const int32_t *ncnt,
                              int64_t n, int cap, const int64_t *offsets, int32_t *idx)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c = perm[i];
    int cnt = ncnt[i];
    int32_t *o = idx + offsets[c];
    const int32_t *l = nbr + i * (int64_t)cap;
    for (int k = 0; k < cnt; ++k) {
        int v = perm[l[k]];
        int p = k;
        while (p > 0 && o[p - 1] > v) {
            o[p] = o[p - 1];
            --p;
        }
        o[p] = v;
    }
}

}  // namespace

void launch_set_u_from_eos(const StepState &s, const DevRates &r, const DevEos &eos,
                           cudaStream_t stream)
{
    if (s.n == 0) return;
    k_set_u<<<(int)((s.n + 255) / 256), 256, 0, stream>>>(s, r, eos);
}

void launch_kick_drift(const StepState &s, const DevRates &r, double dt, cudaStream_t st)
{
    if (s.n == 0) return;
    k_kick_drift<<<(int)((s.n + 255) / 256), 256, 0, st>>>(s, r, dt);
}

void launch_kick_return(const StepState &s, const DevRates &r, const DevEos &eos,
                        const DevMaterial &mat, double dt, int h_nmin, int h_nmax,
                        cudaStream_t st)
{
    if (s.n == 0) return;
    k_kick_return<<<(int)((s.n + 255) / 256), 256, 0, st>>>(s, r, eos, mat, dt, h_nmin, h_nmax);
}

void launch_totals(const StepState &s, const int32_t *ncount, double *partial, double *out,
                   cudaStream_t st)
{
    k_totals_partial<<<kTotBlocks, kTotThreads, 0, st>>>(s, ncount, partial);
    k_totals_sum<<<1, 32, 0, st>>>(partial, kTotBlocks, s.n, out);
}

void launch_star_totals(const StepState &s, const int32_t *ncount, int nstars,
                        const int64_t *off, const int32_t *idx, double *out, cudaStream_t st)
{
    if (nstars < 1) return;
    k_star_totals<<<nstars, kTotThreads, 0, st>>>(s, ncount, off, idx, out);
}

void launch_export_counts(const Scratch &s, int64_t n, int64_t *counts_out, cudaStream_t st)
{
    if (n == 0) return;
    k_export_counts<<<(int)((n + 255) / 256), 256, 0, st>>>(s.perm, s.ncnt, n, counts_out);
}

void launch_scan_i64(int64_t *data, int64_t n, cudaStream_t st)
{
    k_scan_i64<<<1, 1024, 0, st>>>(data, n);
}

void launch_export_fill(const Scratch &s, int64_t n, int cap, const int64_t *offsets,
                        int32_t *idx, cudaStream_t st)
{
    if (n == 0) return;
    k_export_fill<<<(int)((n + 127) / 128), 128, 0, st>>>(s.perm, s.nbr, s.ncnt, n, cap, offsets,
                                                         idx);
}

}  // namespace sph
