// Neighbour search, first half: bounding box, Hilbert keys, LSD radix sort,
// sorted gather and the leaf tree.  The pair tiles over the tree (candidate
// leaves and the exact neighbour masks) are built in sph_tiles.cu.
#include <cstdio>

#include "sph_device.cuh"

namespace sph {

namespace {

__device__ __forceinline__ double dec_double(unsigned long long e)
{
    unsigned long long u = (e & 0x8000000000000000ull) ? (e & ~0x8000000000000000ull) : ~e;
    return __longlong_as_double((long long)u);
}

constexpr int kBoxThreads = 256;

// Order-preserving integer image of a double's bits (dec_double inverts it).
__device__ __forceinline__ unsigned long long enc_bits(unsigned long long u)
{
    return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}

__device__ __forceinline__ bool finite_bits(unsigned long long u)
{
    return ((u >> 52) & 0x7ffull) != 0x7ffull;
}

// Order-preserving integer image of a float's bits, and its inverse.
__device__ __forceinline__ uint32_t enc_f32(float f)
{
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float dec_f32(uint32_t e)
{
    return __uint_as_float((e & 0x80000000u) ? (e & 0x7fffffffu) : ~e);
}

// Bounding box of all positions.  Each block writes a partial; the last
// block to finish reduces the partials, derives the position grid and
// resets the per-RHS counters.  Also flags non-finite positions and h.
// Minima and maxima are taken on order-preserving integer images of the
// doubles, which keeps the scan off the (narrow) FP64 pipe.
__global__ void k_bbox(DevState st, unsigned long long *partial, unsigned int *done,
                       DevScalars *sc, uint32_t *radix_tot, uint32_t *star_box, int nstars)
{
    unsigned long long lo[3] = {~0ull, ~0ull, ~0ull}, hi[3] = {0ull, 0ull, 0ull};
    bool bad = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < st.n;
         i += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long p[3] = {(unsigned long long)__double_as_longlong(st.x[i]),
                                   (unsigned long long)__double_as_longlong(st.y[i]),
                                   (unsigned long long)__double_as_longlong(st.z[i])};
        long long hb = __double_as_longlong(st.h[i]);
        // h must be finite and > 0: sign clear, not zero, exponent not all ones
        bad |= !(finite_bits(p[0]) && finite_bits(p[1]) && finite_bits(p[2]) &&
                 finite_bits((unsigned long long)hb) && hb > 0);
        for (int k = 0; k < 3; ++k) {
            unsigned long long e = enc_bits(p[k]);
            lo[k] = e < lo[k] ? e : lo[k];
            hi[k] = e > hi[k] ? e : hi[k];
        }
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&sc->err, ERR_NONFINITE);
    __shared__ unsigned long long s_lo[3][kBoxThreads / 32], s_hi[3][kBoxThreads / 32];
    for (int k = 0; k < 3; ++k) {
        unsigned long long a = lo[k], b = hi[k];
        for (int o = 16; o > 0; o >>= 1) {
            unsigned long long ao = __shfl_xor_sync(0xffffffffu, a, o);
            unsigned long long bo = __shfl_xor_sync(0xffffffffu, b, o);
            a = ao < a ? ao : a;
            b = bo > b ? bo : b;
        }
        if ((threadIdx.x & 31) == 0) {
            s_lo[k][threadIdx.x >> 5] = a;
            s_hi[k][threadIdx.x >> 5] = b;
        }
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        int k = threadIdx.x;
        unsigned long long a = s_lo[k][0], b = s_hi[k][0];
        for (int w = 1; w < kBoxThreads / 32; ++w) {
            a = s_lo[k][w] < a ? s_lo[k][w] : a;
            b = s_hi[k][w] > b ? s_hi[k][w] : b;
        }
        partial[blockIdx.x * 6 + k] = a;
        partial[blockIdx.x * 6 + 3 + k] = b;
    }
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    // the sort of this right-hand side starts from zero digit totals and tile
    // counters, and (several stars) from empty per-star boxes
    for (int k = threadIdx.x; k < 8 * 256; k += blockDim.x) radix_tot[k] = 0u;
    if (star_box)
        for (int k = threadIdx.x; k < 6 * nstars; k += blockDim.x)
            star_box[k] = k < 3 * nstars ? 0xffffffffu : 0u;
    if (threadIdx.x < 8) sc->tile_next[threadIdx.x] = 0u;
    // all threads of the last block reduce the block partials
    for (int k = 0; k < 3; ++k) {
        unsigned long long a = ~0ull, b = 0ull;
        for (int w = threadIdx.x; w < (int)gridDim.x; w += blockDim.x) {
            unsigned long long pa = __ldcg(&partial[w * 6 + k]), pb = __ldcg(&partial[w * 6 + 3 + k]);
            a = pa < a ? pa : a;
            b = pb > b ? pb : b;
        }
        for (int o = 16; o > 0; o >>= 1) {
            unsigned long long ao = __shfl_xor_sync(0xffffffffu, a, o);
            unsigned long long bo = __shfl_xor_sync(0xffffffffu, b, o);
            a = ao < a ? ao : a;
            b = bo > b ? bo : b;
        }
        if ((threadIdx.x & 31) == 0) {
            s_lo[k][threadIdx.x >> 5] = a;
            s_hi[k][threadIdx.x >> 5] = b;
        }
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        int k = threadIdx.x;
        unsigned long long a = s_lo[k][0], b = s_hi[k][0];
        for (int w = 1; w < kBoxThreads / 32; ++w) {
            a = s_lo[k][w] < a ? s_lo[k][w] : a;
            b = s_hi[k][w] > b ? s_hi[k][w] : b;
        }
        sc->bbox_lo[k] = a;
        sc->bbox_hi[k] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int k = 0; k < 3; ++k) {
            m = fmax(m, fabs(dec_double(sc->bbox_lo[k])));
            m = fmax(m, fabs(dec_double(sc->bbox_hi[k])));
        }
        // Grid for the two-float split: |x|/grid < 2^22 keeps Xhi exact in FP32.
        int e = 0;
        frexp(fmax(m, 1e-300), &e);  // m < 2^e
        sc->grid = ldexp(1.0, e - 22);
        sc->grid_inv = ldexp(1.0, 22 - e);
        sc->grid_f = (float)sc->grid;
        sc->grid_inv_f = (float)sc->grid_inv;
        for (int k = 0; k < 3; ++k) {
            double lo_k = dec_double(sc->bbox_lo[k]);
            double ext = dec_double(sc->bbox_hi[k]) - lo_k;
            sc->inv_ext[k] = ext > 0.0 ? 1.0 / ext : 0.0;
            sc->key_lo_f[k] = (float)lo_k;
            sc->key_scale_f[k] = (float)sc->inv_ext[k];
        }
        sc->eps_abs = 1e-6 * fmax(m, 1e-30);
        sc->eps_abs_f = (float)sc->eps_abs;
        // absolute part of the tile screening band: 48 g u with u = 2^-24
        sc->band_abs = (float)(48.0 * ldexp(sc->grid, -24));
        sc->pairs_last = 0ull;
        sc->tree_done = 0;
        sc->max_count = 0;
        sc->q_max = 0u;
        sc->resorted = 0;
        sc->xmax_f = (float)m * 1.000001f;
        sc->pq_head = 0u;
        sc->pq_done = 0u;
        sc->rhs_count += 1ull;
        *done = 0u;
    }
}

__device__ __forceinline__ uint32_t spread3(uint32_t v)
{
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

// Hilbert index of cell (x0, x1, x2), `bits` bits per axis.  Skilling's
// transform (J. Skilling, "Programming the Hilbert curve", AIP Conf. Proc. 707,
// 2004) turns the coordinates into the transposed index in place: per level,
// from the top, a set bit inverts the lower bits of the first axis, a clear
// bit exchanges them with those of its own axis; a Gray decode follows.  The
// transposed index read bit-plane by bit-plane is the position on the curve.
// Consecutive cells on the curve share a face, so runs of consecutive sorted
// particles (the tree leaves) are more compact than along a Morton curve.
__device__ __forceinline__ uint32_t hilbert3(uint32_t x0, uint32_t x1, uint32_t x2, int bits)
{
    uint32_t X[3] = {x0, x1, x2};
    const uint32_t top = 1u << (bits - 1);
    for (uint32_t Q = top; Q > 1; Q >>= 1) {
        const uint32_t P = Q - 1;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            if (X[i] & Q) {
                X[0] ^= P;
            } else {
                uint32_t t = (X[0] ^ X[i]) & P;
                X[0] ^= t;
                X[i] ^= t;
            }
        }
    }
    X[1] ^= X[0];
    X[2] ^= X[1];
    uint32_t t = 0;
    for (uint32_t Q = top; Q > 1; Q >>= 1)
        if (X[2] & Q) t ^= Q - 1;
    X[0] ^= t;
    X[1] ^= t;
    X[2] ^= t;
    return spread3(X[2]) | (spread3(X[1]) << 1) | (spread3(X[0]) << 2);
}

constexpr int kSortThreads = 256;
constexpr int kMaxPasses = 8;

// Bounding box of each star's fl32 positions (several stars, sort steps), so
// that each star's curve key is taken over its own box: a star's curve order,
// hence its leaves, then does not depend on where the other stars sit (over
// the common box the curve leaves and re-enters a star's region, and leaves
// of 8 consecutive particles at such jumps span much of the star).  Lanes of
// a warp holding the same star reduce together (match, then min / max over
// the group), one lane per star and warp updates the star's slots.
// star_box: [6][nstars] encodings, lo x, y, z then hi x, y, z (reset by
// k_bbox).
__global__ void k_star_box(DevState st, uint32_t *star_box, int nstars)
{
    const int64_t n = st.n;
    const int lane = threadIdx.x & 31;
    // the loop bound is block-uniform, so whole warps take part in every round
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < n; i0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = i0 + threadIdx.x;
        const bool v = i < n;
        const int s = v ? st.star[i] : -1;
        const unsigned grp = __match_any_sync(0xffffffffu, s);
        const bool lead = v && lane == __ffs(grp) - 1;
        const bool ok = v && s >= 0 && s < nstars;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const double *X = k == 0 ? st.x : (k == 1 ? st.y : st.z);
            const uint32_t e = v ? enc_f32(__double2float_rn(X[i])) : 0u;
            const uint32_t mn = __reduce_min_sync(grp, v ? e : 0xffffffffu);
            const uint32_t mx = __reduce_max_sync(grp, v ? e : 0u);
            if (lead && ok) {
                atomicMin(&star_box[k * nstars + s], mn);
                atomicMax(&star_box[(3 + k) * nstars + s], mx);
            }
        }
    }
}

// Space-filling-curve key of every particle (star id above the 3*bits bits of
// the cell's Hilbert index), its identity value, and the digit histograms of
// all radix passes at once (a digit count does not depend on the key order).
// Also clears the tile status words of all passes.
__global__ void k_keys_hist(DevState st, DevScalars *sc, int bits, int passes,
                            unsigned long long *keys, uint32_t *vals, uint32_t *radix_tot,
                            unsigned long long *status, int64_t status_words,
                            const uint32_t *star_box, int nstars)
{
    __shared__ uint32_t h[kMaxPasses][256];
    for (int p = 0; p < passes; ++p) h[p][threadIdx.x] = 0u;
    if (blockIdx.x == 0 && threadIdx.x == 0) sc->resorted = 1;  // the candidate lists are stale
    __syncthreads();
    // cell coordinates in FP32 (any fixed map of position to cell serves the
    // ordering; the clamp absorbs rounding at the box faces)
    const float cells = (float)(1u << bits);
    float lo[3], sc3[3];
    for (int k = 0; k < 3; ++k) {
        lo[k] = sc->key_lo_f[k];
        sc3[k] = sc->key_scale_f[k] * cells;
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < st.n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float p[3] = {__double2float_rn(st.x[i]), __double2float_rn(st.y[i]),
                            __double2float_rn(st.z[i])};
        uint32_t s = st.star ? (uint32_t)st.star[i] : 0u;
        uint32_t q[3];
        for (int k = 0; k < 3; ++k) {
            float a = lo[k], b = sc3[k];
            if (star_box && s < (uint32_t)nstars) {
                // the star's own box (several stars)
                a = dec_f32(star_box[k * nstars + s]);
                const float ext = dec_f32(star_box[(3 + k) * nstars + s]) - a;
                b = ext > 0.f ? cells / ext : 0.f;
            }
            float t = (p[k] - a) * b;
            t = fminf(fmaxf(t, 0.f), cells - 1.f);
            q[k] = (uint32_t)t;
        }
        unsigned long long key = (unsigned long long)hilbert3(q[0], q[1], q[2], bits);
        key |= (unsigned long long)s << (3 * bits);
        keys[i] = key;
        vals[i] = (uint32_t)i;
        for (int pp = 0; pp < passes; ++pp) atomicAdd(&h[pp][(key >> (8 * pp)) & 255u], 1u);
    }
    __syncthreads();
    for (int p = 0; p < passes; ++p) {
        uint32_t c = h[p][threadIdx.x];
        if (c) atomicAdd(&radix_tot[p * 256 + threadIdx.x], c);
    }
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < status_words;
         w += (int64_t)gridDim.x * blockDim.x)
        status[w] = 0ull;
}

// Tile status words hold a flag and a count in one aligned 64-bit word, so
// relaxed single-copy-atomic accesses suffice: no other data hangs on them.
__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

constexpr int kLookback = 8;  // predecessor words read together per look-back step

// One stable 8-bit digit pass in a single launch.  Blocks claim tiles in
// order from a counter, so every lower tile belongs to a block that is
// already running.  A tile counts its digits, publishes the counts (status
// word: 1 = tile count, 2 = inclusive prefix over tiles, value in the low 32
// bits), and thread d then walks back over lower tiles adding their counts
// until it meets a published prefix (decoupled look-back).  Keys are then
// scattered to base(d) + prefix + rank, the rank stable within the tile.
// Look-back reads kLookback lower tiles per step, so a tile whose
// predecessors have only published counts still finds its prefix in a few
// steps instead of waiting for a chain of prefixes.
// A tile that has made spin_limit_of(sc) rounds of look-back reads without
// finding its prefix, or that sees another tile's timeout, gives up and
// raises ERR_TIMEOUT (the sort is then invalid, the host reports it); scatter
// indices stay in bounds.  Passes after a timed-out one return at entry.
__global__ void k_onesweep(const unsigned long long *kin, const uint32_t *vin,
                           unsigned long long *kout, uint32_t *vout, int64_t n, int ipt,
                           int shift, const uint32_t *digit_total, unsigned long long *status,
                           unsigned int *tile_next, DevScalars *sc)
{
    __shared__ uint32_t cnt[256];
    __shared__ uint32_t run[256];
    __shared__ uint32_t wsum[kSortThreads / 32];
    __shared__ uint32_t wc[kSortThreads / 32][256];
    __shared__ int s_tile, s_abort;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    // set by an earlier pass, or by a tile of this pass that gave up: one
    // reading for the whole block, so that the block returns as one
    if (t == 0) s_abort = order_invalid(sc) ? 1 : 0;
    __syncthreads();
    if (s_abort) return;
    const int limit = spin_limit_of(sc);
    if (t == 0) s_tile = (int)atomicAdd(tile_next, 1u);
    cnt[t] = 0u;
    // base of digit t: keys of this pass with a smaller digit
    const uint32_t tot = digit_total[t];
    uint32_t x = tot;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    uint32_t base = x - tot;
    for (int w = 0; w < warp; ++w) base += wsum[w];
    const int tile = s_tile;
    const int64_t first = (int64_t)tile * kSortThreads * ipt;
    for (int r = 0; r < ipt; ++r) {
        int64_t i = first + (int64_t)r * kSortThreads + t;
        if (i < n) atomicAdd(&cnt[(kin[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    const uint32_t c = cnt[t];
    unsigned long long *mine = status + (int64_t)tile * 256 + t;
    uint32_t excl = 0u;
    if (tile == 0) {
        st_relaxed_u64(mine, (2ull << 32) | c);
    } else {
        st_relaxed_u64(mine, (1ull << 32) | c);
        int k = tile - 1;
        int polls = 0;
        while (k >= 0) {
            // a bounded wait: give up after `limit` rounds of reads, or at
            // once when another tile has already given up
            if (polls++ >= limit || order_invalid(sc)) {
                atomicOr(&sc->err, ERR_TIMEOUT);
                break;
            }
            // read up to kLookback lower tiles at once, then add them in order
            // until a prefix (done) or a word not yet written (poll again)
            unsigned long long w[kLookback];
#pragma unroll
            for (int u = 0; u < kLookback; ++u)
                w[u] = u <= k ? ld_relaxed_u64(status + (int64_t)(k - u) * 256 + t) : (2ull << 32);
            bool done = false, stall = false;
            int used = 0;
#pragma unroll
            for (int u = 0; u < kLookback; ++u) {
                if (done || stall) continue;
                uint32_t f = (uint32_t)(w[u] >> 32);
                if (f == 0u) {
                    stall = true;
                } else {
                    if (u <= k) excl += (uint32_t)w[u];
                    used = u + 1;
                    done = f == 2u;
                }
            }
            k -= used;
            if (done) break;
        }
        st_relaxed_u64(mine, (2ull << 32) | (excl + c));
    }
    run[t] = base + excl;
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    for (int r = 0; r < ipt; ++r) {
        int64_t i = first + (int64_t)r * kSortThreads + t;
        bool valid = i < n;
        unsigned long long k = valid ? kin[i] : 0ull;
        uint32_t v = valid ? vin[i] : 0u;
        uint32_t d = valid ? (uint32_t)((k >> shift) & 255u) : 256u;
        for (int w = 0; w < kSortThreads / 32; ++w) wc[w][t] = 0u;
        __syncthreads();
        unsigned peers = __match_any_sync(0xffffffffu, d);
        uint32_t rank = __popc(peers & lt);
        if (valid && (__ffs(peers) - 1) == lane) wc[warp][d] = __popc(peers);
        __syncthreads();
        uint32_t acc = 0;
        for (int w = 0; w < kSortThreads / 32; ++w) {
            uint32_t cw = wc[w][t];
            wc[w][t] = acc;
            acc += cw;
        }
        __syncthreads();
        if (valid) {
            uint32_t dst = run[d] + wc[warp][d] + rank;
            if ((int64_t)dst < n) {
                kout[dst] = k;
                vout[dst] = v;
            } else {  // only after a failed look-back (ERR_TIMEOUT is set too)
                atomicOr(&sc->err, ERR_BOUNDS);
            }
        }
        __syncthreads();
        run[t] += acc;
        __syncthreads();
    }
}

// Sorted copies and the FP32 j-record halves read by the list build.  order
// may be perm itself (keeping the last sort's order): each thread reads and
// rewrites only its own slot.
__global__ void k_gather(DevState st, const uint32_t *order, DevScalars *sc, int32_t *perm,
                         double *xs, double *ys, double *zs, double *hs, uint8_t *tys,
                         float4 *rec, float4 *pos4, double4_32a *rec64)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= st.n || order_invalid(sc)) return;
    uint32_t o = order[i];
    if ((int64_t)o >= st.n) {  // only after a failed sort (its error flag is set too)
        atomicOr(&sc->err, ERR_BOUNDS);
        o = 0u;
    }
    int32_t c = (int32_t)o;
    perm[i] = c;
    double p[3] = {st.x[c], st.y[c], st.z[c]};
    double h = st.h[c], m = st.m[c];
    xs[i] = p[0];
    ys[i] = p[1];
    zs[i] = p[2];
    hs[i] = h;
    tys[i] = st.type[c];
    // Two-float split: Xhi = g * rint(fl32(x)/g) on the power-of-two grid g
    // (exact in FP32 since |x|/g < 2^22), Xlo = fl32(x - Xhi) with the
    // difference taken exactly in FP64; |x - Xhi| <= 3g/4.
    const float gf = sc->grid_f, gi = sc->grid_inv_f;
    float xf[3], hi[3], lo[3];
    for (int k = 0; k < 3; ++k) {
        xf[k] = __double2float_rn(p[k]);
        hi[k] = rintf(xf[k] * gi) * gf;
        lo[k] = __double2float_rn(p[k] - float_to_double_exact(hi[k]));
    }
    const float hf = __double2float_rn(h);
    rec[i] = make_float4(hi[0], hi[1], hi[2], hf);
    rec[st.n + i] = make_float4(lo[0], lo[1], lo[2], __double2float_rn(m));
    pos4[i] = make_float4(xf[0], xf[1], xf[2], hf);
    if (rec64) {
        rec64[i * 3 + 0] = make_double4_32a(p[0], p[1], p[2], h);
        rec64[i * 3 + 1].x = m;
    }
}

__device__ __forceinline__ float4 node_merge_a(float4 a, float4 b)
{
    return make_float4(fminf(a.x, b.x), fminf(a.y, b.y), fminf(a.z, b.z), fmaxf(a.w, b.w));
}

__device__ __forceinline__ float4 node_merge_b(float4 a, float4 b)
{
    int sa = __float_as_int(a.w), sb = __float_as_int(b.w);
    int lo = min(sa & 0xffff, sb & 0xffff);
    int hi = max((int)((unsigned)sa >> 16), (int)((unsigned)sb >> 16));
    return make_float4(fmaxf(a.x, b.x), fmaxf(a.y, b.y), fmaxf(a.z, b.z),
                       __int_as_float((int)((unsigned)lo | ((unsigned)hi << 16))));
}

// Whether the candidate lists must be built again for this right-hand side
// (the last block of the tree kernel decides, once every block has reduced
// q_a = d_a / h_a0 + g_a, d_a the displacement of particle a since the lists
// were built, h_a0 its h then and g_a = h_a / h_a0 - 1).  A pair within
// h_a + h_b now was within h_a + h_b + d_a + d_b <= (1 + q_a) h_a0 +
// (1 + q_b) h_b0 <= (1 + max q)(h_a0 + h_b0) when the lists were built, so
// lists of every pair within (1 + eps)(h_a0 + h_b0) hold every neighbour while
// max q < eps.  q_a comes from fl32 positions and h with margins that make it
// an upper bound (k_tree).
__device__ void decide_rebuild(DevScalars *sc)
{
    const float eps = sc->skin;
    bool rebuild = !sc->built || sc->resorted || !(eps >= 0.f);
    if (!rebuild) {
        // NaN (lists never built for some slot) orders above every number
        const float q = __uint_as_float(*(volatile unsigned *)&sc->q_max);
        rebuild = !(q * 1.000001f < eps);
    }
    sc->rebuild = rebuild ? 1 : 0;
    if (rebuild) {
        sc->built = 1;
        sc->builds += 1ull;
        sc->tiles_last = 0ull;
        sc->max_cand = 0;
    }
}

// Leaf boxes and the implicit 8-ary tree above them.  Leaf boxes come from
// pos4 = fl32(x, y, z, h) widened by one FP32 ulp outward: a round-to-nearest
// value lies within half an ulp of the FP64 value, so the widened box holds
// every FP64 position (and h_max bounds every FP64 h) of the leaf.  Each
// thread also reduces its leaf's displacement and h growth since the
// candidate lists were built (pos_build), and the last block decides whether
// they are rebuilt.
__global__ void k_tree(const float4 *pos4, const float4 *pos_build, const int32_t *leaf_start,
                       const int32_t *leaf_star, TreeLevels tl, float4 *nodes, DevScalars *sc)
{
    __shared__ float4 sa[kTreeBlock], sb[kTreeBlock];
    if (order_invalid(sc)) return;  // uniform across the grid
    const int t = threadIdx.x;
    const int l = blockIdx.x * kTreeBlock + t;
    const int nleaves = tl.count[0];
    float4 a = make_float4(3e38f, 3e38f, 3e38f, 0.f), b = make_float4(-3e38f, -3e38f, -3e38f, 0.f);
    // q_a = d_a / h_a0 + g_a bounded from above: the fl32 displacement plus
    // 4 u |x|_max for the rounding of both fl32 positions, divided by the
    // fl32 h_a0 with a 1e-6 relative margin (the rounding of h_a0 and of the
    // division); g_a from the ratio of fl32 h rounded up plus 4e-7 (the
    // rounding of both h).  NaN (a slot never built) is kept.
    const float dabs = 4.f * 5.9604645e-8f * sc->xmax_f;
    float qm = 0.f;
    if (l < nleaves) {
        const int j0 = leaf_start[l], j1 = leaf_start[l + 1];
        float4 q[kLeaf];
#pragma unroll
        for (int k = 0; k < kLeaf; ++k) q[k] = pos4[j0 + k < j1 ? j0 + k : j0];
#pragma unroll
        for (int k = 0; k < kLeaf; ++k) {
            const float4 qb = pos_build[j0 + k < j1 ? j0 + k : j0];
            const float dx = q[k].x - qb.x, dy = q[k].y - qb.y, dz = q[k].z - qb.z;
            const float d = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz))) * 1.000001f + dabs;
            const float qa = __fdiv_ru(d, qb.w) * 1.000001f + (__fdiv_ru(q[k].w, qb.w) - 1.f) + 4e-7f;
            qm = (qa > qm || qa != qa) ? qa : qm;
        }
        float lo[3] = {q[0].x, q[0].y, q[0].z}, hi[3] = {q[0].x, q[0].y, q[0].z}, hm = q[0].w;
#pragma unroll
        for (int k = 1; k < kLeaf; ++k) {
            lo[0] = fminf(lo[0], q[k].x);
            lo[1] = fminf(lo[1], q[k].y);
            lo[2] = fminf(lo[2], q[k].z);
            hi[0] = fmaxf(hi[0], q[k].x);
            hi[1] = fmaxf(hi[1], q[k].y);
            hi[2] = fmaxf(hi[2], q[k].z);
            hm = fmaxf(hm, q[k].w);
        }
        const float ninf = -INFINITY, pinf = INFINITY;
        int s = leaf_star[l];
        a = make_float4(nextafterf(lo[0], ninf), nextafterf(lo[1], ninf), nextafterf(lo[2], ninf),
                        nextafterf(hm, pinf));
        b = make_float4(nextafterf(hi[0], pinf), nextafterf(hi[1], pinf), nextafterf(hi[2], pinf),
                        __int_as_float((int)((unsigned)s | ((unsigned)s << 16))));
        nodes[2 * ((int64_t)tl.offset[0] + l) + 0] = a;
        nodes[2 * ((int64_t)tl.offset[0] + l) + 1] = b;
    }
    sa[t] = a;
    sb[t] = b;
    __syncthreads();
    // In-block levels: node k of level v+1 is the union of nodes 8k..8k+7 of
    // level v.  A block of kTreeBlock = 8^kTreeBlockLevels leaves holds that many levels.
    int top_local = min(tl.nlevels - 1, kTreeBlockLevels);
    for (int v = 1; v <= top_local; ++v) {
        int width = kTreeBlock >> (3 * v);
        int node = blockIdx.x * width + t;
        float4 na, nb;
        bool act = t < width;
        if (act) {
            int child0 = blockIdx.x * (kTreeBlock >> (3 * (v - 1))) + 8 * t;
            na = sa[8 * t];
            nb = sb[8 * t];
            for (int c = 1; c < kBranch; ++c) {
                if (child0 + c < tl.count[v - 1]) {
                    na = node_merge_a(na, sa[8 * t + c]);
                    nb = node_merge_b(nb, sb[8 * t + c]);
                }
            }
        }
        __syncthreads();
        if (act) {
            sa[t] = na;
            sb[t] = nb;
            if (node < tl.count[v]) {
                nodes[2 * ((int64_t)tl.offset[v] + node) + 0] = na;
                nodes[2 * ((int64_t)tl.offset[v] + node) + 1] = nb;
            }
        }
        __syncthreads();
    }
    // largest q since the build: one atomic per warp on the bits of a
    // non-negative float (or NaN, whose bits order above every number)
    for (int o = 16; o > 0; o >>= 1) {
        const float qo = __shfl_xor_sync(0xffffffffu, qm, o);
        qm = (qo > qm || qo != qo) ? qo : qm;
    }
    if ((t & 31) == 0 && (qm > 0.f || qm != qm)) atomicMax(&sc->q_max, __float_as_uint(qm));
    __shared__ bool last;
    if (t == 0) {
        __threadfence();
        last = atomicAdd(&sc->tree_done, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (t == 0) decide_rebuild(sc);
    for (int v = kTreeBlockLevels + 1; v < tl.nlevels; ++v) {
        for (int node = t; node < tl.count[v]; node += kTreeBlock) {
            int64_t c = (int64_t)tl.offset[v - 1] + (int64_t)kBranch * node;
            float4 na = __ldcg(&nodes[2 * c]), nb = __ldcg(&nodes[2 * c + 1]);
            for (int k = 1; k < kBranch; ++k) {
                if ((int64_t)kBranch * node + k < tl.count[v - 1]) {
                    na = node_merge_a(na, __ldcg(&nodes[2 * (c + k)]));
                    nb = node_merge_b(nb, __ldcg(&nodes[2 * (c + k) + 1]));
                }
            }
            nodes[2 * ((int64_t)tl.offset[v] + node) + 0] = na;
            nodes[2 * ((int64_t)tl.offset[v] + node) + 1] = nb;
        }
        __threadfence_block();
        __syncthreads();
    }
    if (t == 0) sc->tree_done = 0;
}

}  // namespace

// Host-side launch sequence of the sort and the tree.
void launch_build(const DevState &st, const Scratch &s, const SortPlan &plan,
                  const TreeLevels &tl, int nleaves, int fp64_records, cudaStream_t stream,
                  int *nlaunch, bool resort)
{
    const int64_t n = st.n;
    int nl = 0;
    int64_t nb = (n + kBoxThreads - 1) / kBoxThreads;
    int bblocks = (int)(nb < kBoxBlocksMax ? nb : kBoxBlocksMax);
    if (bblocks < 1) bblocks = 1;
    const bool star_boxes = s.star_box && plan.nstars > 1 && st.star;
    k_bbox<<<bblocks, kBoxThreads, 0, stream>>>(
        st, reinterpret_cast<unsigned long long *>(s.bbox_partial), s.bbox_done, s.sc, s.radix_tot,
        star_boxes ? s.star_box : nullptr, plan.nstars);
    ++nl;
    // the order of the last sort (every entry of perm is a valid caller index)
    const uint32_t *order = reinterpret_cast<const uint32_t *>(s.perm);
    if (resort) {
        // keys, all digit histograms and cleared tile status words in one launch
        unsigned long long *status = reinterpret_cast<unsigned long long *>(s.hist);
        const int64_t status_words = (int64_t)plan.passes * plan.nblocks * 256;
        int kb = (int)((n + kSortThreads - 1) / kSortThreads);
        if (kb > 2 * kBoxBlocksMax) kb = 2 * kBoxBlocksMax;
        if (star_boxes) {
            k_star_box<<<kb, kSortThreads, 0, stream>>>(st, s.star_box, plan.nstars);
            ++nl;
        }
        k_keys_hist<<<kb, kSortThreads, 0, stream>>>(st, s.sc, plan.key_bits_axis, plan.passes,
                                                     s.keys[0], s.vals[0], s.radix_tot, status,
                                                     status_words, star_boxes ? s.star_box : nullptr,
                                                     plan.nstars);
        ++nl;
        for (int p = 0; p < plan.passes; ++p) {
            int src = p & 1, dst = src ^ 1;
            k_onesweep<<<plan.nblocks, kSortThreads, 0, stream>>>(
                s.keys[src], s.vals[src], s.keys[dst], s.vals[dst], n, plan.ipt, 8 * p,
                s.radix_tot + 256 * p, status + (int64_t)p * plan.nblocks * 256,
                &s.sc->tile_next[p], s.sc);
            ++nl;
        }
        order = s.vals[plan.passes & 1];
    }
    const int tb = 256;
    const int gb = (int)((n + tb - 1) / tb);
    k_gather<<<gb, tb, 0, stream>>>(st, order, s.sc, s.perm, s.xs, s.ys, s.zs, s.hs, s.tys, s.rec,
                                    s.pos4, fp64_records ? s.rec64 : nullptr);
    ++nl;
    k_tree<<<(nleaves + kTreeBlock - 1) / kTreeBlock, kTreeBlock, 0, stream>>>(
        s.pos4, s.pos_build, s.leaf_start, s.leaf_star, tl, s.nodes, s.sc);
    ++nl;
    if (nlaunch) *nlaunch += nl;
}

}  // namespace sph
