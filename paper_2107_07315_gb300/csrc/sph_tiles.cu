// Neighbour search: candidate lists from pair tiles of leaves, and the exact
// neighbour lists screened from them (with the density summation fused in,
// mixed precision).
//
// The neighbour predicate is the one of Sec. I.B: b is a neighbour of a iff
// b != a, both belong to the same star and |x_a - x_b| < 2 h_ab = h_a + h_b.
// It must equal an FP64 evaluation of
//     r2 = (dx*dx + dy*dy) + dz*dz < (h_a + h_b)^2
// bit for bit, in both precisions.
//
// Candidate lists (k_tiles), built when the tree kernel finds the last ones
// stale (a new curve order, or particles that may have moved or grown into a
// pair the lists miss), one warp per leaf A (8 consecutive sorted particles):
//   1. Walk: breadth first over the implicit 8-ary tree, level by level, one
//      child per lane, the next 32 children's boxes loaded while the current
//      ones are tested, so a level costs about one memory latency instead of
//      one per node.  Inner nodes are kept when their box lies within
//      s (h_max(A) + h_max(node)) of A's box, s = 1 + eps.  At the leaf level
//      each candidate leaf B gets the 8-bit mask of A's particles q that lie
//      within s (h_q + h_max(B)) of B's box (its "reach"); B is kept when the
//      mask is not empty.  Testing particles rather than A's box keeps the
//      list short when A's 8 particles straddle a jump of the curve.
//   2. Tiles: the candidate leaves are staged in shared memory four at a time
//      (32 particles: FP32 position relative to A's first particle and h; one
//      coalesced load pair per lane), the next four loaded into registers
//      while the current ones are screened.  Lane 8r + b takes particle b of
//      B against particle r of A (first half) and r + 4 (second half); a half
//      whose particles cannot reach B is skipped.  A pair is kept when its
//      FP32 distance is below s (h_a + h_b) or within the FP32 error band of
//      it (a superset is all a candidate list needs); missing particles sit
//      at +-3e18 and the self pair is cleared from the self tile.  The two
//      ballots are the tile's 64-bit mask (bit 8q + b), kept in shared
//      memory; a decode pass then writes each particle's list: four lanes per
//      particle take four tiles at a time, a 4-lane prefix of their counts
//      places the entries, so lists come out in ascending sorted index.
//
// Exact lists (k_screen), every right-hand side: four lanes per particle take
// every fourth candidate, test it in FP32 on the two-float positions and,
// inside the error band, with the FP64 predicate; hits are written at their
// rank (ascending) and counted.  In mixed precision each hit's m_b W(r_ab,
// h_ab) goes to the lane that owns its rank in the exact list modulo 4, which
// sums its hits in rank order in a compensated (Kahan) sum; the four lanes
// combine in a fixed order.  The density so depends on the exact list only,
// not on which candidate list held the pairs.  The self term is added and the
// equation of state (Eq. poly_eos, Sec. II.A) and rho = D/(sqrt(gamma) W)
// (Sec. I.C) evaluated.
//
// FP32 screening bands.  Positions are Xhi + Xlo with Xhi on a grid g (a power
// of two, |x|/g < 2^22), |x - Xhi| <= 3g/4 and |Xlo - fl32(x - Xhi)| <= 3gu/4
// (u = 2^-24).  On the two-float positions (k_screen) each computed component
// dx carries at most u|dx| + 3gu of error, and r2 - (h_a + h_b)^2 computed in
// FP32 differs from its exact value by at most 5u r2 + 5u hs^2 + 3.5 (3gu) r +
// u|d|; the band M = 2e-6 (r2 + hs^2) + 48 g u hs is more than three times
// that bound for r <= 2 hs (and for r > 2 hs, d > 3 hs^2 >> M).  In the tiles,
// relative to A's first particle O the FP32 coordinate of p is
// X_p = (Xhi_p - Xhi_O) + (Xlo_p - Xlo_O): the first difference is exact, so X_p
// carries at most 3gu + u|x_p - x_O| of error.  For a in A (|x_a - x_O| <= e,
// the extent of A's box) and b at separation D = x_a - x_b, each computed
// component of X_a - X_b carries at most 6gu + 2ue + 2u|D_k|, and
// r2 - (h_a + h_b)^2 computed in FP32 differs from its exact value by at most
// 7u r2 + 5u hs^2 + 3.5 (6gu + 2ue) r + u|d| (hs = h_a + h_b; FP32 h carries u),
// and the band takes 48 u (g + e) hs for its absolute part.  Outside a band
// the FP32 sign is the exact sign; inside it the FP64 predicate decides (exact
// lists) or the pair is kept (candidate lists).
#include "sph_screen.cuh"

namespace sph {

namespace {

constexpr int kChunk = 4;  // candidate leaves staged per chunk (32 particles)

// Shape of the tile search: G consecutive tree leaves (a search leaf of 8 G
// particles) share one walk, whose front holds at most kCap candidate
// leaves; kWarps warps per block (one walk per warp).  The candidate lists
// are the same for every G (see k_tiles); G sets only the cost of a build.
// BIG (list capacity above the default 256): one tree leaf per walk and a
// front of 1024 candidate leaves, one warp per block, for particles whose h
// is many times their neighbours' (the ejecta of a strongly driven star).
template <int G, bool BIG = false>
struct TileShape;
template <>
struct TileShape<1, true> {
    static constexpr int kWarps = 1, kCap = 4 * kCandCap, kMinBlocks = 8;
    using Reach = unsigned char;
};
template <>
struct TileShape<1> {
    static constexpr int kWarps = 4, kCap = kCandCap, kMinBlocks = 8;
    using Reach = unsigned char;
};
template <>
struct TileShape<2> {
    static constexpr int kWarps = 2, kCap = 2 * kCandCap, kMinBlocks = 12;
    using Reach = unsigned short;
};
template <>
struct TileShape<4> {
    static constexpr int kWarps = 2, kCap = 2 * kCandCap, kMinBlocks = 12;
    using Reach = unsigned int;
};

// One warp per search leaf of G tree leaves.  The walk uses the union of the
// G leaf boxes and their star range at inner levels and the reach mask of
// all 8 G particles at the leaf level.  Then, leaf by leaf, the candidate
// leaves that one of its own particles reaches (and, several stars, that
// belong to its star) are screened in tiles and decoded as for one leaf.  A
// leaf B reached by a particle q of leaf A is also kept by a walk of A alone
// (q lies in A's box, and every ancestor of B has a larger box and h_max),
// and both tests pass exactly the same pairs, so the candidate lists do not
// depend on G.
template <bool MULTI_STAR, int G, bool BIG>
__global__ void __launch_bounds__(32 * TileShape<G, BIG>::kWarps, TileShape<G, BIG>::kMinBlocks)
k_tiles(DevState st, Scratch s, TreeLevels tl, int nleaves, int cap)
{
    constexpr int W = TileShape<G, BIG>::kWarps, CAP = TileShape<G, BIG>::kCap, NP = kLeaf * G;
    using Reach = typename TileShape<G, BIG>::Reach;
    __shared__ int s_front[W][2][CAP];
    __shared__ Reach s_reach[W][2][CAP];
    __shared__ float4 s_p[W][NP];        // the group's fl32 positions and h (walk)
    __shared__ float4 s_A[W][NP][2];     // the group's records (Xhi, h), (Xlo, m)
    __shared__ float4 s_stage[W][2][kChunk * kLeaf];  // (X, h) relative to A's first particle
    __shared__ int2 s_lr[W][2][kChunk];
    __shared__ uint2 s_mask[W][CAP];     // tile masks of one leaf: rows 0-3, rows 4-7
    __shared__ short s_sel[W][G > 1 ? CAP : 1];  // front slots of one leaf (G > 1)
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int A0 = (blockIdx.x * W + w) * G;
    // whole warps only (no block-wide barrier below); nothing consumes an
    // order whose sort timed out; nothing to do while the lists are valid
    if (A0 >= nleaves || order_invalid(s.sc) || !s.sc->rebuild) return;
    const int ng = min(G, nleaves - A0);
    const int64_t n = st.n;
    const unsigned lt = (1u << lane) - 1u;
    DevScalars *sc = s.sc;
    const float eps = sc->eps_abs_f;
    const float band_abs = sc->band_abs;
    const float scale = 1.f + fmaxf(sc->skin, 0.f);  // s = 1 + eps of the candidate lists

    // the group's particles: lane 8 g + k holds particle k of leaf A0 + g
    bool pv = false;
    if (lane < NP) {
        const int g = lane / kLeaf, k = lane % kLeaf;
        int64_t ip = 0;
        if (g < ng) {
            const int2 r = leaf_range<MULTI_STAR>(s.leaf_start, A0 + g, n);
            pv = k < r.y - r.x;
            ip = r.x + k;
        }
        s_p[w][lane] = pv ? s.pos4[ip] : make_float4(3e38f, 3e38f, 3e38f, 0.f);
        s_A[w][lane][0] = pv ? s.rec[ip] : make_float4(3e38f, 3e38f, 3e38f, 0.f);
        s_A[w][lane][1] = pv ? s.rec[n + ip] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const unsigned pmask = __ballot_sync(0xffffffffu, pv);
    // the group's box (union of its leaf boxes, h_max in lo.w) and star range
    float4 Glo = make_float4(3e38f, 3e38f, 3e38f, 0.f), Ghi = make_float4(-3e38f, -3e38f, -3e38f, 0.f);
    int slo = 0x7fffffff, shi = -1;
    if (lane < ng) {
        const int64_t a_node = 2 * (int64_t)tl.offset[0] + 2 * (int64_t)(A0 + lane);
        Glo = s.nodes[a_node];
        Ghi = s.nodes[a_node + 1];
        slo = shi = MULTI_STAR ? s.leaf_star[A0 + lane] : 0;
    }
#pragma unroll
    for (int o = 1; o < G; o <<= 1) {
        Glo.x = fminf(Glo.x, __shfl_xor_sync(0xffffffffu, Glo.x, o));
        Glo.y = fminf(Glo.y, __shfl_xor_sync(0xffffffffu, Glo.y, o));
        Glo.z = fminf(Glo.z, __shfl_xor_sync(0xffffffffu, Glo.z, o));
        Glo.w = fmaxf(Glo.w, __shfl_xor_sync(0xffffffffu, Glo.w, o));
        Ghi.x = fmaxf(Ghi.x, __shfl_xor_sync(0xffffffffu, Ghi.x, o));
        Ghi.y = fmaxf(Ghi.y, __shfl_xor_sync(0xffffffffu, Ghi.y, o));
        Ghi.z = fmaxf(Ghi.z, __shfl_xor_sync(0xffffffffu, Ghi.z, o));
        slo = min(slo, __shfl_xor_sync(0xffffffffu, slo, o));
        shi = max(shi, __shfl_xor_sync(0xffffffffu, shi, o));
    }
    Glo.x = __shfl_sync(0xffffffffu, Glo.x, 0);
    Glo.y = __shfl_sync(0xffffffffu, Glo.y, 0);
    Glo.z = __shfl_sync(0xffffffffu, Glo.z, 0);
    Glo.w = __shfl_sync(0xffffffffu, Glo.w, 0);
    Ghi.x = __shfl_sync(0xffffffffu, Ghi.x, 0);
    Ghi.y = __shfl_sync(0xffffffffu, Ghi.y, 0);
    Ghi.z = __shfl_sync(0xffffffffu, Ghi.z, 0);
    slo = __shfl_sync(0xffffffffu, slo, 0);
    shi = __shfl_sync(0xffffffffu, shi, 0);
    __syncwarp();

    // ---------------------------------------------------------------- walk
    auto box_box = [&](const float4 &lo, const float4 &hi) -> bool {
        if (MULTI_STAR) {
            const int sr = __float_as_int(hi.w);
            if (shi < (sr & 0xffff) || slo > (int)((unsigned)sr >> 16)) return false;
        }
        const float gx = fmaxf(fmaxf(lo.x - Ghi.x, Glo.x - hi.x), 0.f);
        const float gy = fmaxf(fmaxf(lo.y - Ghi.y, Glo.y - hi.y), 0.f);
        const float gz = fmaxf(fmaxf(lo.z - Ghi.z, Glo.z - hi.z), 0.f);
        const float R = fmaf((Glo.w + lo.w) * scale, 1.0001f, eps);
        return fmaf(gx, gx, fmaf(gy, gy, gz * gz)) < R * R;
    };
    // particles of the group within h_q + h_max of a leaf box (fl32
    // positions; leaf boxes hold every FP64 position and h; the slack
    // covers FP32 rounding)
    auto reach_mask = [&](const float4 &lo, const float4 &hi) -> unsigned {
        unsigned r = 0u;
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            const float4 pk = s_p[w][k];
            const float gx = fmaxf(fmaxf(lo.x - pk.x, pk.x - hi.x), 0.f);
            const float gy = fmaxf(fmaxf(lo.y - pk.y, pk.y - hi.y), 0.f);
            const float gz = fmaxf(fmaxf(lo.z - pk.z, pk.z - hi.z), 0.f);
            const float R = fmaf((pk.w + lo.w) * scale, 1.0001f, eps);
            r |= (fmaf(gx, gx, fmaf(gy, gy, gz * gz)) < R * R) ? (1u << k) : 0u;
        }
        return r;
    };
    int *front = s_front[w][0], *next = s_front[w][1];
    Reach *rfront = s_reach[w][0], *rnext = s_reach[w][1];
    if (lane == 0) {
        front[0] = 0;  // the root (at level 0 when the tree is one leaf)
        rfront[0] = (Reach)pmask;
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
            if (v && box_box(lo, hi)) r = leaves ? reach_mask(lo, hi) : 1u;
            const bool hit = r != 0u;
            const unsigned bal = __ballot_sync(0xffffffffu, hit);
            if (hit) {
                const int pos = nf + __popc(bal & lt);
                if (pos < CAP) {
                    next[pos] = c;
                    rnext[pos] = (Reach)r;
                }
            }
            nf += __popc(bal);
        }
        if (nf > CAP) {
            over = true;
            nf = CAP;
        }
        __syncwarp();
        int *tmp = front;
        front = next;
        next = tmp;
        Reach *rt = rfront;
        rfront = rnext;
        rnext = rt;
        F = nf;
    }
    const int nc = F;
    if (lane == 0) atomicMax(&sc->max_cand, nc);

    // candidate test of row x with staged particle b: FP32 distance below
    // s (h_a + h_b), or within the FP32 error band of it
    auto pair = [&](const float4 &x, const float4 &bq, float band) -> bool {
        const float dx = x.x - bq.x, dy = x.y - bq.y, dz = x.z - bq.z;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const float hs = (x.w + bq.w) * scale;
        const float hs2 = hs * hs;
        const float M = fmaf(kBandRel, r2 + hs2, band * hs);
        return r2 - hs2 < M;
    };
    const int hr = lane >> 3, jj = lane & 7;
    const int q = lane >> 2, s4 = lane & 3;

    for (int g = 0; g < ng; ++g) {
        const int A = A0 + g;
        const int2 ar = leaf_range<MULTI_STAR>(s.leaf_start, A, n);
        const int na = ar.y - ar.x;
        // the front slots whose leaf one of A's particles reaches (and, several
        // stars, of A's star); every slot for a search leaf of one tree leaf
        int ncg = nc;
        if (G > 1) {
            const int astar = MULTI_STAR ? s.leaf_star[A] : 0;
            ncg = 0;
            for (int t0 = 0; t0 < nc; t0 += 32) {
                const int t = t0 + lane;
                bool keep = false;
                if (t < nc) {
                    keep = (((unsigned)rfront[t] >> (kLeaf * g)) & 0xffu) != 0u;
                    if (MULTI_STAR && keep) keep = s.leaf_star[front[t]] == astar;
                }
                const unsigned bal = __ballot_sync(0xffffffffu, keep);
                if (keep) s_sel[w][ncg + __popc(bal & lt)] = (short)t;
                ncg += __popc(bal);
            }
            __syncwarp();
        }
        auto slot_of = [&](int c) -> int { return G > 1 ? (int)s_sel[w][c] : c; };
        if (lane == 0) atomicAdd(&sc->tiles_last, (unsigned long long)ncg);

        // ----------------------------------------------------------- tiles
        // FP32 coordinates relative to A's first particle O, and the band of
        // this leaf (48 u (g + e), e the largest extent of A's box)
        const int64_t a_node = 2 * (int64_t)tl.offset[0] + 2 * (int64_t)A;
        const float4 Alo = s.nodes[a_node], Ahi = s.nodes[a_node + 1];
        const float4 O0 = s_A[w][kLeaf * g][0], O1 = s_A[w][kLeaf * g][1];
        auto rel = [&](const float4 &r0, const float4 &r1) -> float4 {
            return make_float4((r0.x - O0.x) + (r1.x - O1.x), (r0.y - O0.y) + (r1.y - O1.y),
                               (r0.z - O0.z) + (r1.z - O1.z), r0.w);
        };
        const float ext = fmaxf(fmaxf(Ahi.x - Alo.x, Ahi.y - Alo.y), Ahi.z - Alo.z);
        const float band = fmaf(48.f * 5.9604645e-8f, ext, band_abs);
        // screening lanes: lane 8 hr + jj takes particle jj of B against rows
        // hr and hr + 4 of A; missing rows and missing staged particles sit
        // far apart on opposite sides: such a pair is never a hit and never
        // inside the band
        const bool v0 = hr < na, v1 = hr + 4 < na;
        const float4 x0 = v0 ? rel(s_A[w][kLeaf * g + hr][0], s_A[w][kLeaf * g + hr][1])
                             : make_float4(3e18f, 3e18f, 3e18f, 0.f);
        const float4 x1 = v1 ? rel(s_A[w][kLeaf * g + hr + 4][0], s_A[w][kLeaf * g + hr + 4][1])
                             : make_float4(3e18f, 3e18f, 3e18f, 0.f);

        float4 nb4 = make_float4(0.f, 0.f, 0.f, 0.f);
        int2 nlr = make_int2(0, 0);
        auto load_chunk = [&](int c0) {
            const int slot = c0 + (lane >> 3), b = lane & 7;
            nb4 = make_float4(-3e18f, -3e18f, -3e18f, 0.f);
            if (slot < ncg) {
                const int2 lr = leaf_range<MULTI_STAR>(s.leaf_start, front[slot_of(slot)], n);
                if (b < lr.y - lr.x) nb4 = rel(s.rec[lr.x + b], s.rec[n + lr.x + b]);
            }
            nlr = make_int2(0, 0);
            if (lane < kChunk && c0 + lane < ncg)
                nlr = leaf_range<MULTI_STAR>(s.leaf_start, front[slot_of(c0 + lane)], n);
        };
        load_chunk(0);
        for (int c0 = 0; c0 < ncg; c0 += kChunk) {
            const int buf = (c0 / kChunk) & 1;
            s_stage[w][buf][lane] = nb4;
            if (lane < kChunk) s_lr[w][buf][lane] = nlr;
            __syncwarp();
            if (c0 + kChunk < ncg) load_chunk(c0 + kChunk);
            const int kend = min(kChunk, ncg - c0);
            uint2 mk = make_uint2(0u, 0u);  // lane k < kChunk: mask of slot c0 + k
#pragma unroll
            for (int k = 0; k < kChunk; ++k) {
                if (k >= kend) break;  // warp-uniform
                const int2 lr = s_lr[w][buf][k];
                const unsigned reach = ((unsigned)rfront[slot_of(c0 + k)] >> (kLeaf * g)) & 0xffu;
                const float4 bq = s_stage[w][buf][k * kLeaf + jj];
                unsigned b0 = 0u, b1 = 0u;
                if (reach & 0x0fu) b0 = __ballot_sync(0xffffffffu, pair(x0, bq, band));
                if (reach & 0xf0u) b1 = __ballot_sync(0xffffffffu, pair(x1, bq, band));
                if (lr.x == ar.x) {  // the self tile: particle q is not its own neighbour
                    b0 &= ~0x08040201u;
                    b1 &= ~0x80402010u;
                }
                if (lane == k) mk = make_uint2(b0, b1);
            }
            if (lane < kend) s_mask[w][c0 + lane] = mk;
        }
        __syncwarp();

        // decode: lane 4q + s4 takes tiles s4, s4 + 4, ... of row q; a 4-lane
        // prefix of the hit counts places each tile's entries, so the list of
        // row q is ascending
        const bool vq = q < na;
        const int64_t i = ar.x + (vq ? q : 0);
        int32_t *lq = s.vlist + i * cap;
        int cnt = 0;
        for (int k0 = 0; k0 < ncg; k0 += 4) {
            const int k = k0 + s4;
            unsigned byte = 0u;
            int start = 0;
            if (k < ncg) {
                const uint2 m = s_mask[w][k];
                byte = ((q < 4 ? m.x : m.y) >> (8 * (q & 3))) & 0xffu;
                start = leaf_range<MULTI_STAR>(s.leaf_start, front[slot_of(k)], n).x;
            }
            const int c = __popc(byte);
            int pre = c;
            for (int o = 1; o < 4; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, pre, o, 4);
                if (s4 >= o) pre += y;
            }
            int p = cnt + pre - c;
            cnt += __shfl_sync(0xffffffffu, pre, 3, 4);
            while (byte) {
                const int b = __ffs(byte) - 1;
                byte &= byte - 1u;
                if (p < cap) lq[p] = start + b;
                ++p;
            }
        }

        // --------------------------------------------- per-particle results
        if (vq && cnt > cap) over = true;
        if (vq && s4 == 0) {
            s.vcnt[i] = min(cnt, cap);
            const float4 p = s_p[w][kLeaf * g + q];
            s.pos_build[i] = p;  // the positions and h these lists hold for
        }
        __syncwarp();  // s_stage, s_lr, s_mask and s_sel are reused by the next leaf
    }
    if (__any_sync(0xffffffffu, over) && lane == 0) atomicOr(&sc->err, ERR_CAPACITY);
}

// Exact lists from the candidate lists, every right-hand side (with the
// density and equation of state when DENSITY): one block of particles per
// CUDA block.
template <bool DENSITY, int LPI>
__global__ void __launch_bounds__(kScreenThreads, 8)
k_screen(DevState st, Scratch s, int cap, DevEos eos, DevMetric g, DevRates out)
{
    if (order_invalid(s.sc)) return;  // uniform across the grid
    screen_block<DENSITY, LPI>(st, s, cap, eos, g, out, (int64_t)blockIdx.x);
}

}  // namespace

void launch_screen(const DevState &st, const Scratch &s, int cap, int density,
                   const DevEos &eos, const DevMetric &g, const DevRates &out,
                   cudaStream_t stream, int screen_lanes)
{
    if (st.n <= 0) return;
    if (screen_lanes == 8) {
        const int ns = (int)((st.n + kScreenThreads / 8 - 1) / (kScreenThreads / 8));
        if (density) k_screen<true, 8><<<ns, kScreenThreads, 0, stream>>>(st, s, cap, eos, g, out);
        else k_screen<false, 8><<<ns, kScreenThreads, 0, stream>>>(st, s, cap, eos, g, out);
    } else {
        const int ns = (int)((st.n + kScreenThreads / 4 - 1) / (kScreenThreads / 4));
        if (density) k_screen<true, 4><<<ns, kScreenThreads, 0, stream>>>(st, s, cap, eos, g, out);
        else k_screen<false, 4><<<ns, kScreenThreads, 0, stream>>>(st, s, cap, eos, g, out);
    }
}

template <int G, bool BIG = false>
static void launch_tiles_g(const DevState &st, const Scratch &s, const TreeLevels &tl,
                           int nleaves, int multi_star, int cap, cudaStream_t stream)
{
    constexpr int W = TileShape<G, BIG>::kWarps;
    const int nb = (nleaves + W * G - 1) / (W * G);
    if (multi_star) k_tiles<true, G, BIG><<<nb, 32 * W, 0, stream>>>(st, s, tl, nleaves, cap);
    else k_tiles<false, G, BIG><<<nb, 32 * W, 0, stream>>>(st, s, tl, nleaves, cap);
}

void launch_tiles_build(const DevState &st, const Scratch &s, const TreeLevels &tl, int nleaves,
                        int multi_star, int cap, cudaStream_t stream, int group)
{
    if (nleaves <= 0) return;
    if (cap > kRowCapDefault) launch_tiles_g<1, true>(st, s, tl, nleaves, multi_star, cap, stream);
    else if (group == 4) launch_tiles_g<4>(st, s, tl, nleaves, multi_star, cap, stream);
    else if (group == 2) launch_tiles_g<2>(st, s, tl, nleaves, multi_star, cap, stream);
    else launch_tiles_g<1>(st, s, tl, nleaves, multi_star, cap, stream);
}

void launch_tiles(const DevState &st, const Scratch &s, const TreeLevels &tl, int nleaves,
                  int multi_star, int cap, int density, const DevEos &eos, const DevMetric &g,
                  const DevRates &out, cudaStream_t stream, int *nlaunch, int screen_lanes,
                  int group)
{
    if (nleaves <= 0) return;
    launch_tiles_build(st, s, tl, nleaves, multi_star, cap, stream, group);
    launch_screen(st, s, cap, density, eos, g, out, stream, screen_lanes);
    if (nlaunch) *nlaunch += 2;
}

}  // namespace sph
