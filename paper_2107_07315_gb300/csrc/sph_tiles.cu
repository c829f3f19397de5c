// Neighbour search over pair tiles of leaves, with the density summation
// fused in (mixed precision).
//
// The neighbour predicate is the one of Sec. I.B: b is a neighbour of a iff
// b != a, both belong to the same star and |x_a - x_b| < 2 h_ab = h_a + h_b.
// It must equal an FP64 evaluation of
//     r2 = (dx*dx + dy*dy) + dz*dz < (h_a + h_b)^2
// bit for bit, in both precisions.
//
// One warp per leaf A (8 consecutive sorted particles of one star):
//   1. Walk: breadth first over the implicit 8-ary tree, level by level, one
//      child per lane, the next 32 children's boxes loaded while the current
//      ones are tested, so a level costs about one memory latency instead of
//      one per node.  Inner nodes are kept when their box lies within
//      h_max(A) + h_max(node) of A's box.  At the leaf level each candidate
//      leaf B gets the 8-bit mask of A's particles q that lie within
//      h_q + h_max(B) of B's box (its "reach"); B is kept when the mask is
//      not empty.  Testing particles rather than A's box keeps the list short
//      when A's 8 particles straddle a jump of the curve.
//   2. Tiles: the candidate leaves are staged in shared memory four at a time
//      (32 particles: FP32 position relative to A's first particle, h and m;
//      one coalesced load pair per lane), the next four loaded into registers
//      while the current ones are screened.  Lane 8r + b takes particle b of
//      B against particle r of A (first half) and r + 4 (second half); a half
//      whose particles cannot reach B is skipped.  The test is FP32 and,
//      inside its error band, the FP64 predicate.  The two ballots are the
//      tile's 64-bit neighbour mask (bit 8q + b); each hit is written to
//      particle q's list at its rank, so lists come out in ascending sorted
//      index.
//   3. Mixed precision: the warp then sums the density over the lists it has
//      just written (still in L1): four lanes per particle take every fourth
//      neighbour, add m_b W(r_ab, h_ab) to a compensated (Kahan) sum and
//      combine in a fixed order; the self term m_a W(0, h_a) is added and one
//      lane per particle runs the equation of state (Eq. poly_eos, Sec. II.A)
//      and rho = D/(sqrt(gamma) W) (Sec. I.C).  Summing over the lists touches
//      only true pairs, a seventh of the screened ones.
//
// FP32 screening band.  Positions are Xhi + Xlo with Xhi on a grid g (a power
// of two, |x|/g < 2^22), |x - Xhi| <= 3g/4 and |Xlo - fl32(x - Xhi)| <= 3gu/4
// (u = 2^-24).  Relative to A's first particle O the FP32 coordinate of p is
// X_p = (Xhi_p - Xhi_O) + (Xlo_p - Xlo_O): the first difference is exact, so X_p
// carries at most 3gu + u|x_p - x_O| of error.  For a in A (|x_a - x_O| <= e,
// the extent of A's box) and b at separation D = x_a - x_b, each computed
// component of X_a - X_b carries at most 6gu + 2ue + 2u|D_k|, and
// r2 - (h_a + h_b)^2 computed in FP32 differs from its exact value by at most
// 7u r2 + 5u hs^2 + 3.5 (6gu + 2ue) r + u|d| (hs = h_a + h_b; FP32 h carries u).
// The band M = 2e-6 (r2 + hs^2) + 48 u (g + e) hs is more than three times that
// bound for r <= 2 hs (and for r > 2 hs, d > 3 hs^2 >> M): outside the band the
// FP32 sign is the exact sign, inside it the FP64 predicate decides.
#include "sph_device.cuh"

namespace sph {

namespace {

constexpr int kTileWarps = 4;
constexpr int kTileThreads = 32 * kTileWarps;
constexpr int kChunk = 4;  // candidate leaves staged per chunk (32 particles)
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

template <bool MULTI_STAR, bool DENSITY>
__global__ void __launch_bounds__(kTileThreads, 8)
k_tiles(DevState st, Scratch s, TreeLevels tl, int nleaves, int cap, DevEos eos, DevMetric g,
        DevRates out)
{
    __shared__ int s_front[kTileWarps][2][kCandCap];
    __shared__ unsigned char s_reach[kTileWarps][2][kCandCap];
    __shared__ float4 s_p[kTileWarps][kLeaf];        // A's fl32 positions and h (walk)
    __shared__ float4 s_A[kTileWarps][kLeaf][2];     // A's records (Xhi, h), (Xlo, m)
    __shared__ float4 s_stage[kTileWarps][2][kChunk * kLeaf];  // (X, h) relative to A's first particle
    __shared__ int2 s_lr[kTileWarps][2][kChunk];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int A = blockIdx.x * kTileWarps + w;
    // whole warps only (no block-wide barrier below); nothing consumes an
    // order whose sort timed out
    if (A >= nleaves || order_invalid(s.sc)) return;
    const int64_t n = st.n;
    const unsigned lt = (1u << lane) - 1u;
    DevScalars *sc = s.sc;
    const float eps = sc->eps_abs_f;
    const float band_abs = sc->band_abs;

    const int2 ar = leaf_range<MULTI_STAR>(s.leaf_start, A, n);
    const int na = ar.y - ar.x;
    if (lane < kLeaf) {
        const bool v = lane < na;
        s_p[w][lane] = v ? s.pos4[ar.x + lane] : make_float4(3e38f, 3e38f, 3e38f, 0.f);
        s_A[w][lane][0] = v ? s.rec[ar.x + lane] : make_float4(3e38f, 3e38f, 3e38f, 0.f);
        s_A[w][lane][1] = v ? s.rec[n + ar.x + lane] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const int64_t a_node = 2 * (int64_t)tl.offset[0] + 2 * (int64_t)A;
    const float4 Alo = s.nodes[a_node], Ahi = s.nodes[a_node + 1];
    const int astar = MULTI_STAR ? s.leaf_star[A] : 0;
    __syncwarp();

    // ---------------------------------------------------------------- walk
    auto box_box = [&](const float4 &lo, const float4 &hi) -> bool {
        if (MULTI_STAR) {
            const int sr = __float_as_int(hi.w);
            if (astar < (sr & 0xffff) || astar > (int)((unsigned)sr >> 16)) return false;
        }
        const float gx = fmaxf(fmaxf(lo.x - Ahi.x, Alo.x - hi.x), 0.f);
        const float gy = fmaxf(fmaxf(lo.y - Ahi.y, Alo.y - hi.y), 0.f);
        const float gz = fmaxf(fmaxf(lo.z - Ahi.z, Alo.z - hi.z), 0.f);
        const float R = fmaf(Alo.w + lo.w, 1.0001f, eps);
        return fmaf(gx, gx, fmaf(gy, gy, gz * gz)) < R * R;
    };
    // particles of A within h_q + h_max of a leaf box (fl32 positions; leaf
    // boxes hold every FP64 position and h; the slack covers FP32 rounding)
    auto reach8 = [&](const float4 &lo, const float4 &hi) -> unsigned {
        unsigned r = 0u;
#pragma unroll
        for (int k = 0; k < kLeaf; ++k) {
            const float4 pk = s_p[w][k];
            const float gx = fmaxf(fmaxf(lo.x - pk.x, pk.x - hi.x), 0.f);
            const float gy = fmaxf(fmaxf(lo.y - pk.y, pk.y - hi.y), 0.f);
            const float gz = fmaxf(fmaxf(lo.z - pk.z, pk.z - hi.z), 0.f);
            const float R = fmaf(pk.w + lo.w, 1.0001f, eps);
            r |= (fmaf(gx, gx, fmaf(gy, gy, gz * gz)) < R * R) ? (1u << k) : 0u;
        }
        return r;
    };
    int *front = s_front[w][0], *next = s_front[w][1];
    unsigned char *rfront = s_reach[w][0], *rnext = s_reach[w][1];
    if (lane == 0) {
        front[0] = 0;  // the root (at level 0 when the tree is one leaf)
        rfront[0] = (unsigned char)((1u << na) - 1u);
    }
    int F = 1;
    bool over = false;
    __syncwarp();
    for (int lv = tl.nlevels - 1; lv >= 1; --lv) {
        const int nch = tl.count[lv - 1];
        const int64_t off = tl.offset[lv - 1];
        const int total = kBranch * F;
        const bool leaves = lv == 1;
        int nf = 0;
        int cn = 0;
        bool vn = false;
        float4 lon = make_float4(0.f, 0.f, 0.f, 0.f), hin = lon;
        auto fetch = [&](int t) {
            vn = false;
            if (t < total) {
                cn = front[t / kBranch] * kBranch + (t % kBranch);
                if (cn < nch) {
                    vn = true;
                    lon = s.nodes[2 * (off + cn)];
                    hin = s.nodes[2 * (off + cn) + 1];
                }
            }
        };
        fetch(lane);
        for (int t0 = 0; t0 < total; t0 += 32) {
            const int c = cn;
            const bool v = vn;
            const float4 lo = lon, hi = hin;
            if (t0 + 32 < total) fetch(t0 + 32 + lane);
            unsigned r = 0u;
            if (v && box_box(lo, hi)) r = leaves ? reach8(lo, hi) : 1u;
            const bool hit = r != 0u;
            const unsigned bal = __ballot_sync(0xffffffffu, hit);
            if (hit) {
                const int pos = nf + __popc(bal & lt);
                if (pos < kCandCap) {
                    next[pos] = c;
                    rnext[pos] = (unsigned char)r;
                }
            }
            nf += __popc(bal);
        }
        if (nf > kCandCap) {
            over = true;
            nf = kCandCap;
        }
        __syncwarp();
        int *tmp = front;
        front = next;
        next = tmp;
        unsigned char *rt = rfront;
        rfront = rnext;
        rnext = rt;
        F = nf;
    }
    const int nc = F;
    if (lane == 0) {
        atomicMax(&sc->max_cand, nc);
        atomicAdd(&sc->tiles_last, (unsigned long long)nc);
    }

    // --------------------------------------------------------------- tiles
    // FP32 coordinates relative to A's first particle O, and the band of this
    // leaf (48 u (g + e), e the largest extent of A's box)
    const float4 O0 = s_A[w][0][0], O1 = s_A[w][0][1];
    auto rel = [&](const float4 &r0, const float4 &r1) -> float4 {
        return make_float4((r0.x - O0.x) + (r1.x - O1.x), (r0.y - O0.y) + (r1.y - O1.y),
                           (r0.z - O0.z) + (r1.z - O1.z), r0.w);
    };
    const float ext = fmaxf(fmaxf(Ahi.x - Alo.x, Ahi.y - Alo.y), Ahi.z - Alo.z);
    const float band = fmaf(48.f * 5.9604645e-8f, ext, band_abs);
    // screening lanes: lane 8 hr + jj takes particle jj of B against rows hr
    // and hr + 4 of A
    const int hr = lane >> 3, jj = lane & 7;
    const bool v0 = hr < na, v1 = hr + 4 < na;
    const int i0 = ar.x + hr, i1 = ar.x + hr + 4;
    const float4 x0 = v0 ? rel(s_A[w][hr][0], s_A[w][hr][1]) : make_float4(3e18f, 3e18f, 3e18f, 0.f);
    const float4 x1 = v1 ? rel(s_A[w][hr + 4][0], s_A[w][hr + 4][1])
                         : make_float4(3e18f, 3e18f, 3e18f, 0.f);
    int pos0 = 0, pos1 = 0;  // list lengths of rows hr and hr + 4
    unsigned long long nre = 0;
    int32_t *list0 = s.nbr + (int64_t)(v0 ? i0 : ar.x) * cap;
    int32_t *list1 = s.nbr + (int64_t)(v1 ? i1 : ar.x) * cap;

    // pair test of row x (particle i) with staged particle b (j): FP32 screen,
    // and the FP64 predicate inside the band
    auto pair = [&](const float4 &x, const float4 &bq, bool valid, int i, int j) -> bool {
        const float dx = x.x - bq.x, dy = x.y - bq.y, dz = x.z - bq.z;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const float hs = x.w + bq.w;
        const float hs2 = hs * hs;
        const float d = r2 - hs2;
        const float M = fmaf(kBandRel, r2 + hs2, band * hs);
        bool in = d < -M;
        if (valid && fabsf(d) <= M) {
            ++nre;
            in = pair_in_fp64(s.xs[i], s.ys[i], s.zs[i], s.hs[i], s.xs[j], s.ys[j], s.zs[j],
                              s.hs[j]);
        }
        return in && valid;
    };

    float4 nb4 = make_float4(0.f, 0.f, 0.f, 0.f);
    int2 nlr = make_int2(0, 0);
    auto load_chunk = [&](int c0) {
        const int slot = c0 + (lane >> 3), b = lane & 7;
        nb4 = make_float4(0.f, 0.f, 0.f, 0.f);
        if (slot < nc) {
            const int2 lr = leaf_range<MULTI_STAR>(s.leaf_start, front[slot], n);
            if (b < lr.y - lr.x) nb4 = rel(s.rec[lr.x + b], s.rec[n + lr.x + b]);
        }
        nlr = make_int2(0, 0);
        if (lane < kChunk && c0 + lane < nc) nlr = leaf_range<MULTI_STAR>(s.leaf_start, front[c0 + lane], n);
    };
    load_chunk(0);
    for (int c0 = 0; c0 < nc; c0 += kChunk) {
        const int buf = (c0 / kChunk) & 1;
        s_stage[w][buf][lane] = nb4;
        if (lane < kChunk) s_lr[w][buf][lane] = nlr;
        __syncwarp();
        if (c0 + kChunk < nc) load_chunk(c0 + kChunk);
        const int kend = min(kChunk, nc - c0);
#pragma unroll
        for (int k = 0; k < kChunk; ++k) {
            if (k >= kend) break;  // warp-uniform
            const int2 lr = s_lr[w][buf][k];
            const unsigned reach = rfront[c0 + k];
            const float4 bq = s_stage[w][buf][k * kLeaf + jj];
            const int j = lr.x + jj;
            const bool vj = jj < lr.y - lr.x;
            if (reach & 0x0fu) {
                const bool in = pair(x0, bq, v0 && vj && j != i0, i0, j);
                const unsigned mine = (__ballot_sync(0xffffffffu, in) >> (8 * hr)) & 0xffu;
                if (in) {
                    const int p = pos0 + __popc(mine & ((1u << jj) - 1u));
                    if (p < cap) list0[p] = j;
                }
                pos0 += __popc(mine);
            }
            if (reach & 0xf0u) {
                const bool in = pair(x1, bq, v1 && vj && j != i1, i1, j);
                const unsigned mine = (__ballot_sync(0xffffffffu, in) >> (8 * hr)) & 0xffu;
                if (in) {
                    const int p = pos1 + __popc(mine & ((1u << jj) - 1u));
                    if (p < cap) list1[p] = j;
                }
                pos1 += __popc(mine);
            }
        }
    }

    // ------------------------------------------------- per-particle results
    // row totals: rows hr and hr + 4 sit on lanes 8 hr .. 8 hr + 7
    const int cnt0 = pos0, cnt1 = pos1;
    if ((v0 && cnt0 > cap) || (v1 && cnt1 > cap)) over = true;
    if (jj == 0) {
        if (v0) s.ncnt[i0] = min(cnt0, cap);
        if (v1) s.ncnt[i1] = min(cnt1, cap);
    }
    unsigned long long pairs = jj == 0 ? (unsigned long long)((v0 ? min(cnt0, cap) : 0) +
                                                              (v1 ? min(cnt1, cap) : 0)) : 0ull;
    int cmax = jj == 0 ? max(v0 ? cnt0 : 0, v1 ? cnt1 : 0) : 0;
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
    if (__any_sync(0xffffffffu, over) && lane == 0) atomicOr(&sc->err, ERR_CAPACITY);
    if (!DENSITY) return;
    // density over the lists just written (visible to the warp after the
    // barrier): lane 4q + s4 takes neighbours s4, s4 + 4, ... of row q
    __syncwarp();
    const int q = lane >> 2, s4 = lane & 3;
    const int src = 8 * (q & 3);
    const int c0r = __shfl_sync(0xffffffffu, cnt0, src);
    const int c1r = __shfl_sync(0xffffffffu, cnt1, src);
    const bool vq = q < na;
    const int cnt = vq ? min(q < 4 ? c0r : c1r, cap) : 0;
    const int64_t i = ar.x + (vq ? q : 0);
    const float4 pi0 = s_A[w][q][0], pi1 = s_A[w][q][1];
    const int32_t *lq = s.nbr + i * cap;
    float sum = 0.f, comp = 0.f;
    int jn = s4 < cnt ? lq[s4] : 0;
    for (int k = s4; k < cnt; k += 4) {
        const int j = jn;
        if (k + 4 < cnt) jn = lq[k + 4];
        const float4 b0 = s.rec[j], b1 = s.rec[n + j];
        const float dx = (pi0.x - b0.x) + (pi1.x - b1.x);
        const float dy = (pi0.y - b0.y) + (pi1.y - b1.y);
        const float dz = (pi0.z - b0.z) + (pi1.z - b1.z);
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const float r = r2 * rsqrtf(fmaxf(r2, 1.17549435e-38f));
        const float hinv = __fdividef(2.f, pi0.w + b0.w);  // 1/h_ab
        const float qq = r * hinv;
        const float sig = hinv * hinv * hinv * kInvPiF;
        const float t = 2.f - qq;
        const float W = qq < 1.f ? sig * fmaf(qq * qq, fmaf(0.75f, qq, -1.5f), 1.f)
                                 : sig * 0.25f * t * t * t;
        const float y = b1.w * W - comp;
        const float tt = sum + y;
        comp = (tt - sum) - y;
        sum = tt;
    }
    for (int o = 1; o < 4; o <<= 1) {
        sum += __shfl_xor_sync(0xffffffffu, sum, o);
        comp += __shfl_xor_sync(0xffffffffu, comp, o);
    }
    if (s4 != 0 || !vq) return;

    // equation of state of particle i (lane 4q)
    const float hi = pi0.w;
    const float D = pi1.w * kInvPiF / (hi * hi * hi) + (sum - comp);
    const int c = s.perm[i];
    const int star = MULTI_STAR ? astar : 0;
    const float vx = f64_to_f32_rn(st.vx[c]), vy = f64_to_f32_rn(st.vy[c]),
                vz = f64_to_f32_rn(st.vz[c]);
    const PosF pos{pi0.x, pi0.y, pi0.z, pi1.x, pi1.y, pi1.z};
    Prep<float> pr = eos_prep<float>(eos, g, star, D, vx, vy, vz, pos);
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
    out.ncount[c] = cnt;
}

}  // namespace

void launch_tiles(const DevState &st, const Scratch &s, const TreeLevels &tl, int nleaves,
                  int multi_star, int cap, int density, const DevEos &eos, const DevMetric &g,
                  const DevRates &out, cudaStream_t stream)
{
    if (nleaves <= 0) return;
    const int nb = (nleaves + kTileWarps - 1) / kTileWarps;
    if (multi_star) {
        if (density)
            k_tiles<true, true><<<nb, kTileThreads, 0, stream>>>(st, s, tl, nleaves, cap, eos, g, out);
        else
            k_tiles<true, false><<<nb, kTileThreads, 0, stream>>>(st, s, tl, nleaves, cap, eos, g, out);
    } else {
        if (density)
            k_tiles<false, true><<<nb, kTileThreads, 0, stream>>>(st, s, tl, nleaves, cap, eos, g, out);
        else
            k_tiles<false, false><<<nb, kTileThreads, 0, stream>>>(st, s, tl, nleaves, cap, eos, g, out);
    }
}

}  // namespace sph
