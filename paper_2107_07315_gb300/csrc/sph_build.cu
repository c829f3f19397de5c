// Neighbour search: bounding box, Morton keys, LSD radix sort, sorted
// gather, leaf tree and exact per-particle neighbour lists.
//
// The neighbour predicate is the one of Sec. I.B: b is a neighbour of a iff
// b != a, both belong to the same star and |x_a - x_b| < 2 h_ab = h_a + h_b.
// The lists must equal those of an FP64 evaluation of
//     r2 = (dx*dx + dy*dy) + dz*dz < (h_a + h_b)^2
// bit for bit, in both precisions.  Candidates are screened in FP32 from a
// two-float position split (Xhi on a power-of-two grid plus an FP32
// remainder) with an error bound; pairs inside the bound's band are decided
// again in FP64 with round-to-nearest operations in that exact order.
#include <cstdio>

#include "sph_internal.cuh"

namespace sph {

namespace {

__device__ __forceinline__ unsigned long long enc_double(double d)
{
    unsigned long long u = (unsigned long long)__double_as_longlong(d);
    return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}

__device__ __forceinline__ double dec_double(unsigned long long e)
{
    unsigned long long u = (e & 0x8000000000000000ull) ? (e & ~0x8000000000000000ull) : ~e;
    return __longlong_as_double((long long)u);
}

constexpr int kBoxThreads = 256;

// Bounding box of all positions.  Each block writes a partial; the last
// block to finish reduces the partials, derives the position grid and
// resets the per-RHS counters.  Also flags non-finite positions and h.
__global__ void k_bbox(DevState st, double *partial, unsigned int *done, DevScalars *sc)
{
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    bool bad = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < st.n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double p[3] = {st.x[i], st.y[i], st.z[i]};
        double hh = st.h[i];
        bad |= !(isfinite(p[0]) && isfinite(p[1]) && isfinite(p[2]) && isfinite(hh) && hh > 0.0);
        for (int k = 0; k < 3; ++k) {
            lo[k] = fmin(lo[k], p[k]);
            hi[k] = fmax(hi[k], p[k]);
        }
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&sc->err, ERR_NONFINITE);
    __shared__ double s_lo[3][kBoxThreads / 32], s_hi[3][kBoxThreads / 32];
    for (int k = 0; k < 3; ++k) {
        double a = lo[k], b = hi[k];
        for (int o = 16; o > 0; o >>= 1) {
            a = fmin(a, __shfl_xor_sync(0xffffffffu, a, o));
            b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
        }
        if ((threadIdx.x & 31) == 0) {
            s_lo[k][threadIdx.x >> 5] = a;
            s_hi[k][threadIdx.x >> 5] = b;
        }
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        int k = threadIdx.x;
        double a = s_lo[k][0], b = s_hi[k][0];
        for (int w = 1; w < kBoxThreads / 32; ++w) {
            a = fmin(a, s_lo[k][w]);
            b = fmax(b, s_hi[k][w]);
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
    if (threadIdx.x < 3) {
        int k = threadIdx.x;
        double a = 1e300, b = -1e300;
        for (int w = 0; w < (int)gridDim.x; ++w) {
            a = fmin(a, __ldcg(&partial[w * 6 + k]));
            b = fmax(b, __ldcg(&partial[w * 6 + 3 + k]));
        }
        sc->bbox_lo[k] = enc_double(a);
        sc->bbox_hi[k] = enc_double(b);
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
        sc->eps_abs = 1e-6 * fmax(m, 1e-30);
        sc->pairs_last = 0ull;
        sc->tree_done = 0;
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

// Morton key (star id above 3*bits interleaved cell bits) and identity value.
__global__ void k_keys(DevState st, const DevScalars *sc, int bits,
                       unsigned long long *keys, uint32_t *vals)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= st.n) return;
    double p[3] = {st.x[i], st.y[i], st.z[i]};
    uint32_t q[3];
    double cells = (double)(1u << bits);
    for (int k = 0; k < 3; ++k) {
        double lo = dec_double(sc->bbox_lo[k]), hi = dec_double(sc->bbox_hi[k]);
        double ext = hi - lo;
        double t = ext > 0.0 ? (p[k] - lo) / ext * cells : 0.0;
        t = fmin(fmax(t, 0.0), cells - 1.0);
        q[k] = (uint32_t)t;
    }
    unsigned long long key = (unsigned long long)(spread3(q[0]) | (spread3(q[1]) << 1) |
                                                  (spread3(q[2]) << 2));
    uint32_t s = st.star ? (uint32_t)st.star[i] : 0u;
    key |= (unsigned long long)s << (3 * bits);
    keys[i] = key;
    vals[i] = (uint32_t)i;
}

constexpr int kSortThreads = 256;

// Per-tile digit histogram of one pass over the keys in their current order
// (the tiles of pass p hold different keys than those of pass p-1, so each
// pass counts its own).  hist layout: [digit][block].
__global__ void k_radix_hist(const unsigned long long *keys, int64_t n, int ipt, int shift,
                             uint32_t *hist)
{
    __shared__ uint32_t cnt[256];
    cnt[threadIdx.x] = 0u;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kSortThreads * ipt;
    for (int r = 0; r < ipt; ++r) {
        int64_t i = base + (int64_t)r * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * gridDim.x + blockIdx.x] = cnt[threadIdx.x];
}

// Exclusive scan of each pass's histogram (one block per pass).
__global__ void k_radix_scan(uint32_t *hist, int nblocks)
{
    const int T = 1024;
    __shared__ uint32_t wsum[32];
    uint32_t *h = hist + (int64_t)blockIdx.x * 256 * nblocks;
    int64_t total = (int64_t)256 * nblocks;
    int64_t chunk = (total + T - 1) / T;
    int64_t b0 = threadIdx.x * chunk, b1 = min(b0 + chunk, total);
    uint32_t s = 0;
    for (int64_t i = b0; i < b1; ++i) s += h[i];
    // block exclusive scan of s
    uint32_t v = s;
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) wsum[w] = v;
    __syncthreads();
    if (w == 0) {
        uint32_t x = wsum[lane];
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += t;
        }
        wsum[lane] = x;
    }
    __syncthreads();
    uint32_t run = v - s + (w > 0 ? wsum[w - 1] : 0u);
    for (int64_t i = b0; i < b1; ++i) {
        uint32_t c = h[i];
        h[i] = run;
        run += c;
    }
}

// Stable scatter of one 8-bit digit pass.
__global__ void k_radix_scatter(const unsigned long long *kin, const uint32_t *vin,
                                unsigned long long *kout, uint32_t *vout, int64_t n, int ipt,
                                int shift, const uint32_t *hist_scanned)
{
    __shared__ uint32_t run[256];
    __shared__ uint32_t wc[kSortThreads / 32][256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    run[threadIdx.x] = hist_scanned[(int64_t)threadIdx.x * gridDim.x + blockIdx.x];
    const unsigned lt = (1u << lane) - 1u;
    int64_t base = (int64_t)blockIdx.x * kSortThreads * ipt;
    for (int r = 0; r < ipt; ++r) {
        int64_t i = base + (int64_t)r * kSortThreads + threadIdx.x;
        bool valid = i < n;
        unsigned long long k = valid ? kin[i] : 0ull;
        uint32_t v = valid ? vin[i] : 0u;
        uint32_t d = valid ? (uint32_t)((k >> shift) & 255u) : 256u;
        for (int w = 0; w < kSortThreads / 32; ++w) wc[w][threadIdx.x] = 0u;
        __syncthreads();
        unsigned peers = __match_any_sync(0xffffffffu, d);
        uint32_t rank = __popc(peers & lt);
        if (valid && (__ffs(peers) - 1) == lane) wc[warp][d] = __popc(peers);
        __syncthreads();
        uint32_t tot = 0;
        {
            int t = threadIdx.x;
            for (int w = 0; w < kSortThreads / 32; ++w) {
                uint32_t c = wc[w][t];
                wc[w][t] = tot;
                tot += c;
            }
        }
        __syncthreads();
        if (valid) {
            uint32_t dst = run[d] + wc[warp][d] + rank;
            kout[dst] = k;
            vout[dst] = v;
        }
        __syncthreads();
        run[threadIdx.x] += tot;
        __syncthreads();
    }
}

// Sorted copies and the FP32 j-record halves read by the list build.
__global__ void k_gather(DevState st, const uint32_t *order, const DevScalars *sc, int32_t *perm,
                         double *xs, double *ys, double *zs, double *hs, uint8_t *tys,
                         float4 *rec, double4_32a *rec64)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= st.n) return;
    int32_t c = (int32_t)order[i];
    perm[i] = c;
    double p[3] = {st.x[c], st.y[c], st.z[c]};
    double h = st.h[c], m = st.m[c];
    xs[i] = p[0];
    ys[i] = p[1];
    zs[i] = p[2];
    hs[i] = h;
    tys[i] = st.type[c];
    double g = sc->grid;
    float hi[3], lo[3];
    for (int k = 0; k < 3; ++k) {
        double H = g * rint(p[k] / g);
        hi[k] = (float)H;
        lo[k] = (float)(p[k] - H);
    }
    rec[i * 4 + 0] = make_float4(hi[0], hi[1], hi[2], (float)h);
    rec[i * 4 + 1] = make_float4(lo[0], lo[1], lo[2], (float)m);
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
    int lo = min(sa & 0xffff, sb & 0xffff), hi = max(sa >> 16, sb >> 16);
    return make_float4(fmaxf(a.x, b.x), fmaxf(a.y, b.y), fmaxf(a.z, b.z),
                       __int_as_float(lo | (hi << 16)));
}

// Leaf boxes and the implicit binary tree above them.  Boxes are rounded
// outward to FP32 so that they contain every FP64 position of the node.
__global__ void k_tree(const double *xs, const double *ys, const double *zs, const double *hs,
                       const int32_t *leaf_start, const int32_t *leaf_star, TreeLevels tl,
                       float4 *nodes, DevScalars *sc)
{
    __shared__ float4 sa[kTreeBlock], sb[kTreeBlock];
    const int t = threadIdx.x;
    const int l = blockIdx.x * kTreeBlock + t;
    const int nleaves = tl.count[0];
    float4 a = make_float4(3e38f, 3e38f, 3e38f, 0.f), b = make_float4(-3e38f, -3e38f, -3e38f, 0.f);
    if (l < nleaves) {
        double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300}, hm = 0.0;
        for (int i = leaf_start[l]; i < leaf_start[l + 1]; ++i) {
            double p[3] = {xs[i], ys[i], zs[i]};
            for (int k = 0; k < 3; ++k) {
                lo[k] = fmin(lo[k], p[k]);
                hi[k] = fmax(hi[k], p[k]);
            }
            hm = fmax(hm, hs[i]);
        }
        int s = leaf_star[l];
        a = make_float4(__double2float_rd(lo[0]), __double2float_rd(lo[1]),
                        __double2float_rd(lo[2]), __double2float_ru(hm));
        b = make_float4(__double2float_ru(hi[0]), __double2float_ru(hi[1]),
                        __double2float_ru(hi[2]), __int_as_float(s | (s << 16)));
        nodes[2 * ((int64_t)tl.offset[0] + l) + 0] = a;
        nodes[2 * ((int64_t)tl.offset[0] + l) + 1] = b;
    }
    sa[t] = a;
    sb[t] = b;
    __syncthreads();
    int top_local = min(tl.nlevels - 1, kTreeBlockLevels);
    for (int k = 1; k <= top_local; ++k) {
        int width = kTreeBlock >> k;
        int node = blockIdx.x * width + t;
        float4 na, nb;
        bool act = t < width;
        if (act) {
            int cl = 2 * t, cr = 2 * t + 1;
            int gl = blockIdx.x * (kTreeBlock >> (k - 1)) + cr;
            na = sa[cl];
            nb = sb[cl];
            if (gl < tl.count[k - 1]) {
                na = node_merge_a(na, sa[cr]);
                nb = node_merge_b(nb, sb[cr]);
            }
        }
        __syncthreads();
        if (act) {
            sa[t] = na;
            sb[t] = nb;
            if (node < tl.count[k]) {
                nodes[2 * ((int64_t)tl.offset[k] + node) + 0] = na;
                nodes[2 * ((int64_t)tl.offset[k] + node) + 1] = nb;
            }
        }
        __syncthreads();
    }
    if (tl.nlevels - 1 <= kTreeBlockLevels) return;
    __shared__ bool last;
    if (t == 0) {
        __threadfence();
        last = atomicAdd(&sc->tree_done, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int k = kTreeBlockLevels + 1; k < tl.nlevels; ++k) {
        for (int node = t; node < tl.count[k]; node += kTreeBlock) {
            int64_t c = (int64_t)tl.offset[k - 1] + 2 * node;
            float4 na = __ldcg(&nodes[2 * c]), nb = __ldcg(&nodes[2 * c + 1]);
            if (2 * node + 1 < tl.count[k - 1]) {
                na = node_merge_a(na, __ldcg(&nodes[2 * (c + 1)]));
                nb = node_merge_b(nb, __ldcg(&nodes[2 * (c + 1) + 1]));
            }
            nodes[2 * ((int64_t)tl.offset[k] + node) + 0] = na;
            nodes[2 * ((int64_t)tl.offset[k] + node) + 1] = nb;
        }
        __threadfence_block();
        __syncthreads();
    }
    if (t == 0) sc->tree_done = 0;
}

// Exact FP64 predicate in the oracle's operation order (no contraction).
__device__ __forceinline__ bool pair_in_fp64(double xa, double ya, double za, double ha,
                                             double xb, double yb, double zb, double hb)
{
    double dx = __dsub_rn(xa, xb), dy = __dsub_rn(ya, yb), dz = __dsub_rn(za, zb);
    double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    double hsum = __dadd_rn(ha, hb);
    return r2 < __dmul_rn(hsum, hsum);
}

constexpr int kListThreads = 128;

// One thread per sorted particle: depth-first walk of the tree (left child
// first, so neighbours come out in ascending sorted index), pruning nodes
// whose box lies farther than h_i + h_max(node) from the particle, then the
// screened predicate on the particles of each surviving leaf.
__global__ void __launch_bounds__(kListThreads)
k_neighbors(int64_t n, const float4 *rec, const double *xs, const double *ys, const double *zs,
            const double *hs, const int32_t *leaf_start, const int32_t *leaf_star,
            const int32_t *leaf_of, TreeLevels tl, const float4 *nodes, int cap, int32_t *nbr,
            int32_t *ncnt, DevScalars *sc)
// Stack entries pack (level << 26 | node index) in an unsigned int.
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    bool valid = i < n;
    int cnt = 0;
    unsigned long long nre = 0;
    bool over = false;
    if (valid) {
        float4 r0 = rec[i * 4 + 0], r1 = rec[i * 4 + 1];
        const float grid = (float)sc->grid;
        const float eps = (float)sc->eps_abs;
        const float xi = r0.x + r1.x, yi = r0.y + r1.y, zi = r0.z + r1.z;
        const float hi = r0.w;
        const int star = leaf_star[leaf_of[i]];
        unsigned stack[kMaxLevels + 2];
        int sp = 0;
        stack[sp++] = ((unsigned)(tl.nlevels - 1) << 26) | 0u;
        int32_t *out = nbr + i * (int64_t)cap;
        while (sp > 0) {
            unsigned e = stack[--sp];
            int lv = (int)(e >> 26), k = (int)(e & ((1u << 26) - 1u));
            int64_t gi = (int64_t)tl.offset[lv] + k;
            float4 a = nodes[2 * gi], b = nodes[2 * gi + 1];
            int sr = __float_as_int(b.w);
            if (star < (sr & 0xffff) || star > (sr >> 16)) continue;
            float gx = fmaxf(fmaxf(a.x - xi, xi - b.x), 0.f);
            float gy = fmaxf(fmaxf(a.y - yi, yi - b.y), 0.f);
            float gz = fmaxf(fmaxf(a.z - zi, zi - b.z), 0.f);
            float R = fmaf(hi + a.w, 1.0001f, eps);
            if (gx * gx + gy * gy + gz * gz >= R * R) continue;
            if (lv > 0) {
                int cr = 2 * k + 1;
                if (cr < tl.count[lv - 1]) stack[sp++] = ((unsigned)(lv - 1) << 26) | (unsigned)cr;
                stack[sp++] = ((unsigned)(lv - 1) << 26) | (unsigned)(2 * k);
                continue;
            }
            int j0 = leaf_start[k], j1 = leaf_start[k + 1];
            for (int j = j0; j < j1; ++j) {
                if (j == (int)i) continue;
                float4 q0 = rec[(int64_t)j * 4 + 0], q1 = rec[(int64_t)j * 4 + 1];
                float dx = (r0.x - q0.x) + (r1.x - q1.x);
                float dy = (r0.y - q0.y) + (r1.y - q1.y);
                float dz = (r0.z - q0.z) + (r1.z - q1.z);
                float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                float hsum = hi + q0.w;
                float hs2 = hsum * hsum;
                float d = r2 - hs2;
                float M = fmaf(4e-6f, hs2, 2e-6f * grid * hsum);
                bool in;
                if (d < -M) {
                    in = true;
                } else if (d > M) {
                    in = false;
                } else {
                    ++nre;
                    in = pair_in_fp64(xs[i], ys[i], zs[i], hs[i], xs[j], ys[j], zs[j], hs[j]);
                }
                if (in) {
                    if (cnt < cap) out[cnt] = j;
                    else over = true;
                    ++cnt;
                }
            }
        }
        ncnt[i] = cnt < cap ? cnt : cap;
    }
    // counters: one atomic per warp
    unsigned long long c = (unsigned long long)(cnt < cap ? cnt : cap);
    for (int o = 16; o > 0; o >>= 1) {
        c += __shfl_xor_sync(0xffffffffu, c, o);
        nre += __shfl_xor_sync(0xffffffffu, nre, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&sc->pairs_last, c);
        atomicAdd(&sc->pairs_total, c);
        if (nre) atomicAdd(&sc->rechecks, nre);
    }
    if (over) atomicOr(&sc->err, ERR_CAPACITY);
}

}  // namespace

// Host-side launch sequence of the neighbour search.
void launch_build(const DevState &st, const Scratch &s, const SortPlan &plan,
                  const TreeLevels &tl, int nleaves, int cap, int fp64_records,
                  cudaStream_t stream, int *nlaunch)
{
    const int64_t n = st.n;
    int nl = 0;
    int64_t nb = (n + kBoxThreads - 1) / kBoxThreads;
    int bblocks = (int)(nb < kBoxBlocksMax ? nb : kBoxBlocksMax);
    if (bblocks < 1) bblocks = 1;
    k_bbox<<<bblocks, kBoxThreads, 0, stream>>>(st, s.bbox_partial, s.bbox_done, s.sc);
    ++nl;
    int tb = 256;
    int gb = (int)((n + tb - 1) / tb);
    k_keys<<<gb, tb, 0, stream>>>(st, s.sc, plan.key_bits_axis, s.keys[0], s.vals[0]);
    ++nl;
    for (int p = 0; p < plan.passes; ++p) {
        int src = p & 1, dst = src ^ 1;
        uint32_t *hist = s.hist + (int64_t)p * 256 * plan.nblocks;
        k_radix_hist<<<plan.nblocks, kSortThreads, 0, stream>>>(s.keys[src], n, plan.ipt, 8 * p,
                                                                hist);
        k_radix_scan<<<1, 1024, 0, stream>>>(hist, plan.nblocks);
        k_radix_scatter<<<plan.nblocks, kSortThreads, 0, stream>>>(
            s.keys[src], s.vals[src], s.keys[dst], s.vals[dst], n, plan.ipt, 8 * p, hist);
        nl += 3;
    }
    const uint32_t *order = s.vals[plan.passes & 1];
    k_gather<<<gb, tb, 0, stream>>>(st, order, s.sc, s.perm, s.xs, s.ys, s.zs, s.hs, s.tys, s.rec,
                                    fp64_records ? s.rec64 : nullptr);
    ++nl;
    k_tree<<<(nleaves + kTreeBlock - 1) / kTreeBlock, kTreeBlock, 0, stream>>>(
        s.xs, s.ys, s.zs, s.hs, s.leaf_start, s.leaf_star, tl, s.nodes, s.sc);
    ++nl;
    k_neighbors<<<(int)((n + kListThreads - 1) / kListThreads), kListThreads, 0, stream>>>(
        n, s.rec, s.xs, s.ys, s.zs, s.hs, s.leaf_start, s.leaf_star, s.leaf_of, tl, s.nodes, cap,
        s.nbr, s.ncnt, s.sc);
    ++nl;
    if (nlaunch) *nlaunch += nl;
}

}  // namespace sph
