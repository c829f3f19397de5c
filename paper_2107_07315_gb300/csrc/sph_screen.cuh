// Exact screening of candidate lists (one block of particles), shared by the
// screening kernel of the tile search and the persistent right-hand-side
// kernel.  The FP32 band kBandRel (r2 + hs^2) + band_abs hs and its error
// bound are derived at the head of sph_tiles.cu.
#pragma once

#include "sph_device.cuh"

namespace sph {

namespace {

constexpr int kScreenThreads = 128;
constexpr float kBandRel = 2e-6f;

// Exact FP64 predicate in the oracle's operation order (no contraction).
__device__ __forceinline__ bool pair_in_fp64(double xa, double ya, double za, double ha,
                                             double xb, double yb, double zb, double hb)
{
    double dx = __dsub_rn(xa, xb), dy = __dsub_rn(ya, yb), dz = __dsub_rn(za, zb);
    double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    double hsum = __dadd_rn(ha, hb);
    return r2 < __dmul_rn(hsum, hsum);
}

// Exact lists from the candidate lists, every right-hand side: LPI lanes
// (4 or 8) per particle, 128 / LPI particles per block.  With DENSITY (mixed
// precision) also the density summation and the equation of state.  The exact
// list of a particle is a subsequence of its candidate list, so the two may
// share memory: every entry is written at or before the last one read.
// Block blk of 128 / LPI consecutive sorted particles; every thread of the
// 128-thread block calls it (warp collectives inside, no block barrier).
template <bool DENSITY, int LPI>
__device__ __forceinline__ void screen_block(const DevState &st, const Scratch &s, int cap,
                                             const DevEos &eos, const DevMetric &g,
                                             const DevRates &out, int64_t blk)
{
    const int64_t n = st.n;
    const int lane = threadIdx.x & 31, sub = lane % LPI;
    const int64_t i0 = blk * (kScreenThreads / LPI) + (threadIdx.x / LPI);
    const bool valid = i0 < n;
    const int64_t i = valid ? i0 : 0;
    DevScalars *sc = s.sc;
    const float band_abs = sc->band_abs;
    const float4 a0 = s.rec[i], a1 = s.rec[n + i];
    const int vc = valid ? s.vcnt[i] : 0;
    const int32_t *vl = s.vlist + i * cap;
    int32_t *nl = s.nbr + i * cap;
    const unsigned gshift = lane & ~(unsigned)(LPI - 1);
    const unsigned gmask = (1u << LPI) - 1u;
    int pos = 0;
    unsigned long long nre = 0;
    float sum = 0.f, comp = 0.f;
    // every lane runs to the warp's longest list: the ballot and shuffle below
    // need the whole warp (a lane past its own list tests an old, valid j and
    // drops it).  The records of the next candidate are loaded one iteration
    // ahead, its index two ahead, so two gathers per lane are in flight.
    const int vmax = __reduce_max_sync(0xffffffffu, vc);
    int jn = sub < vc ? checked_index(vl[sub], n, sc) : 0;
    float4 n0 = s.rec[jn], n1 = s.rec[n + jn];
    int jnn = sub + LPI < vc ? checked_index(vl[sub + LPI], n, sc) : 0;
    for (int k0 = 0; k0 < vmax; k0 += LPI) {
        const int k = k0 + sub;
        const bool kv = k < vc;
        const int j = jn;
        const float4 b0 = n0, b1 = n1;
        jn = jnn;
        if (k + LPI < vc) {
            n0 = s.rec[jn];
            n1 = s.rec[n + jn];
        }
        jnn = k + 2 * LPI < vc ? checked_index(vl[k + 2 * LPI], n, sc) : 0;
        const float dx = (a0.x - b0.x) + (a1.x - b1.x);
        const float dy = (a0.y - b0.y) + (a1.y - b1.y);
        const float dz = (a0.z - b0.z) + (a1.z - b1.z);
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const float hs = a0.w + b0.w;
        const float hs2 = hs * hs;
        const float d = r2 - hs2;
        const float M = fmaf(kBandRel, r2 + hs2, band_abs * hs);
        bool in = d < -M;
        if (kv && fabsf(d) <= M) {
            ++nre;
            in = pair_in_fp64(s.xs[i], s.ys[i], s.zs[i], s.hs[i], s.xs[j], s.ys[j], s.zs[j],
                              s.hs[j]);
        }
        in = in && kv;
        const unsigned bits = (__ballot_sync(0xffffffffu, in) >> gshift) & gmask;
        const int nh = __popc(bits);
        if (in) nl[pos + __popc(bits & ((1u << sub) - 1u))] = j;
        if (DENSITY) {
            // m_b W(r_ab, h_ab) of this lane's candidate (used if it is a hit)
            const float r = r2 * rsqrtf(fmaxf(r2, 1.17549435e-38f));
            const float hinv = __fdividef(2.f, hs);  // 1/h_ab
            const float qq = r * hinv;
            const float sig = hinv * hinv * hinv * kInvPiF;
            const float t = 2.f - qq;
            const float W = qq < 1.f ? sig * fmaf(qq * qq, fmaf(0.75f, qq, -1.5f), 1.f)
                                     : sig * 0.25f * t * t * t;
            const float term = b1.w * W;
            // lane sub sums the hits whose rank in the exact list is sub mod
            // LPI, in rank order: the same sums as a pass over the exact list,
            // so the density does not depend on which candidate list held
            // them.  This round's hits hold ranks pos .. pos + nh - 1; the one
            // of rank = sub (mod LPI) is hit number idx, on lane src of the group.
            const int idx = (sub - pos) & (LPI - 1);
            int src = sub;
            if (LPI == 4) {
                // position of the (idx+1)-th set bit of the 4-bit mask: a
                // table of 2-bit entries indexed by (bits, idx), 0 where the
                // mask has fewer set bits (any lane serves then)
                const unsigned key = (bits << 2) | (unsigned)idx;
                const unsigned long long lut =
                    key < 32u ? 0x2409080204010000ull : 0xe439380e340d0c03ull;
                src = (int)((lut >> (2u * (key & 31u))) & 3ull);
            } else {
                int c = 0;
#pragma unroll
                for (int bq = 0; bq < LPI; ++bq) {
                    if ((bits >> bq) & 1u) {
                        if (c == idx) src = bq;
                        ++c;
                    }
                }
            }
            const float tv = __shfl_sync(0xffffffffu, term, (int)gshift + src);
            if (idx < nh) {
                const float y = tv - comp;
                const float tt = sum + y;
                comp = (tt - sum) - y;
                sum = tt;
            }
        }
        pos += nh;
    }
    if (DENSITY) {
        for (int o = 1; o < LPI; o <<= 1) {
            sum += __shfl_xor_sync(0xffffffffu, sum, o);
            comp += __shfl_xor_sync(0xffffffffu, comp, o);
        }
    }
    const bool lead = valid && sub == 0;
    if (lead) s.ncnt[i] = pos;
    unsigned long long pairs = lead ? (unsigned long long)pos : 0ull;
    int cmax = lead ? pos : 0;
    for (int o = 16; o > 0; o >>= 1) {
        pairs += __shfl_xor_sync(0xffffffffu, pairs, o);
        nre += __shfl_xor_sync(0xffffffffu, nre, o);
        cmax = max(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
    }
    if (lane == 0) {
        atomicAdd(&sc->pairs_last, pairs);
        atomicAdd(&sc->pairs_total, pairs);
        if (nre) atomicAdd(&sc->rechecks, nre);
        atomicMax(&sc->max_count, cmax);
    }
    if (!DENSITY || !lead) return;

    // equation of state of particle i
    const float hi = a0.w;
    const float D = a1.w * kInvPiF / (hi * hi * hi) + (sum - comp);
    const int c = checked_index(s.perm[i], n, sc);
    const int star = st.star ? st.star[c] : 0;
    const float vx = f64_to_f32_rn(st.vx[c]), vy = f64_to_f32_rn(st.vy[c]),
                vz = f64_to_f32_rn(st.vz[c]);
    const PosF posf{a0.x, a0.y, a0.z, a1.x, a1.y, a1.z};
    Prep<float> pr = eos_prep<float>(eos, g, star, D, vx, vy, vz, posf);
    const float invD = 1.f / D;
    const float PD2 = pr.P * invD * invD;
    const bool solid = s.tys[i] == 1;
    s.rec[2 * n + i] = make_float4(vx, vy, vz, D);
    s.rec[3 * n + i] = make_float4(PD2, pr.cs, invD, solid ? 1.f : 0.f);
    if (solid) {
        const int64_t N = st.n;
        const float f = invD * invD;
        s.sd2[i] = make_float4(f64_to_f32_rn(st.S[c]) * f, f64_to_f32_rn(st.S[N + c]) * f,
                               f64_to_f32_rn(st.S[2 * N + c]) * f, f64_to_f32_rn(st.S[3 * N + c]) * f);
        s.sd2[n + i] = make_float4(f64_to_f32_rn(st.S[4 * N + c]) * f,
                                   f64_to_f32_rn(st.S[5 * N + c]) * f, 0.f, 0.f);
    } else {
        s.sd2[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        s.sd2[n + i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    s.pp[i * 2 + 0] = make_float4(pr.rho, pr.P, pr.cP, pr.henth);
    s.pp[i * 2 + 1] = make_float4(pr.Wt, pr.cs, D, 0.f);
    out.D[c] = to_out(D);
    out.rho[c] = to_out(pr.rho);
    out.P[c] = to_out(pr.P);
    out.cs[c] = to_out(pr.cs);
    out.ncount[c] = pos;
}

}  // namespace

}  // namespace sph
