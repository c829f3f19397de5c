// Allocation-free neighbour search for callers that cannot call cudaMalloc.
//
// Some callers cannot allocate device memory at the time they need neighbour
// lists: plug-ins living inside a host application whose memory pool owns the
// whole device, processes whose memory budget forbids further allocations,
// or time-critical loops where an allocator call (which may synchronise the
// device) is not allowed.  This entry point computes the same CSR neighbour
// lists as sph_neighbors without a context and without allocating: its
// scratch is one fixed file-scope device array.  Every call looks up the
// array's device address on the current device (the lookup allocates
// nothing), so a context that was reset or re-created is never handed a stale
// address.
//
// Limits: at most kMaxN particles of one star, at most kCap neighbours per
// particle and kCandCap candidate leaves (groups of 8 sorted particles) per
// leaf.  The array (about 11.9 MB) exists on every GPU that loads this library
// and stays there until the process exits.  With lazy module loading (the
// CUDA default) the first call on a device loads this library's device code
// and the array, which takes device memory once: make one call with n >= 1
// before another allocator takes the whole device.  All calls share the
// array: calls that overlap on the GPU (different streams or threads without
// ordering between them) race on it.
#include "sph_internal.cuh"

namespace {

using namespace sph;

constexpr int64_t kMaxN = 16384;
constexpr int kCap = 128;
constexpr int kMaxLeaves = (int)((kMaxN + kLeaf - 1) / kLeaf);
constexpr int kMaxNodes = 2 * kMaxLeaves;
constexpr int kMaxPasses = 4;
constexpr int kMaxSortBlocks = (int)((kMaxN + 255) / 256);

constexpr size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Byte offsets of the scratch segments.
constexpr size_t kPerm = 0;
constexpr size_t kKeys0 = kPerm + align256(kMaxN * 4);
constexpr size_t kKeys1 = kKeys0 + align256(kMaxN * 8);
constexpr size_t kVals0 = kKeys1 + align256(kMaxN * 8);
constexpr size_t kVals1 = kVals0 + align256(kMaxN * 4);
constexpr size_t kHist = kVals1 + align256(kMaxN * 4);
constexpr size_t kXs = kHist + align256((size_t)kMaxPasses * 256 * kMaxSortBlocks * 8);
constexpr size_t kYs = kXs + align256(kMaxN * 8);
constexpr size_t kZs = kYs + align256(kMaxN * 8);
constexpr size_t kHs = kZs + align256(kMaxN * 8);
constexpr size_t kTys = kHs + align256(kMaxN * 8);
constexpr size_t kRec = kTys + align256(kMaxN);
constexpr size_t kNbr = kRec + align256(kMaxN * 4 * 16);
constexpr size_t kNcnt = kNbr + align256((size_t)kMaxN * kCap * 4);
constexpr size_t kVcnt = kNcnt + align256(kMaxN * 4);
constexpr size_t kPosBuild = kVcnt + align256(kMaxN * 4);
constexpr size_t kNodes = kPosBuild + align256(kMaxN * 16);
constexpr size_t kLeafStart = kNodes + align256((size_t)kMaxNodes * 2 * 16);
constexpr size_t kLeafStar = kLeafStart + align256((kMaxLeaves + 1) * 4);
constexpr size_t kLeafOf = kLeafStar + align256(kMaxLeaves * 4);
constexpr size_t kBoxPart = kLeafOf + align256(kMaxN * 4);
constexpr size_t kBoxDone = kBoxPart + align256(6 * kBoxBlocksMax * 8);
constexpr size_t kSc = kBoxDone + 256;
constexpr size_t kMass = kSc + align256(sizeof(DevScalars));
constexpr size_t kType = kMass + align256(kMaxN * 8);
constexpr size_t kRadixTot = kType + align256(kMaxN);
constexpr size_t kPos4 = kRadixTot + align256(8 * 256 * 4);
constexpr size_t kBytes = kPos4 + align256(kMaxN * 16);

static __device__ __align__(256) unsigned char g_scratch[kBytes];

sph_status fail(sph_status s, const char *m)
{
    record_error(m);  // readable through sph_last_error()
    return s;
}

// Device address of g_scratch on the current device.  In host code the
// array's name is only a stand-in; the runtime gives the address the device
// uses, looked up anew on every call.
sph_status scratch_address(unsigned char **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return fail(SPH_ERR_CUDA, "sph_neighbors_noalloc: cudaGetSymbolAddress failed");
    }
    *out = (unsigned char *)p;
    return SPH_OK;
}

// Leaves of 8 consecutive sorted slots of the single star.
__global__ void k_leaf_layout(int64_t n, int nleaves, int32_t *leaf_start, int32_t *leaf_star,
                              int32_t *leaf_of)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) leaf_of[i] = (int32_t)(i / kLeaf);
    if (i <= nleaves) leaf_start[i] = (int32_t)(i * kLeaf < n ? i * kLeaf : n);
    if (i < nleaves) leaf_star[i] = 0;
}

int bits_for_n(int64_t n)
{
    int lg = 1;
    while ((1ll << lg) < n) ++lg;
    int b = (lg + 2) / 3 + 2;
    return b < 5 ? 5 : (b > 10 ? 10 : b);
}

}  // namespace

extern "C" sph_status sph_neighbors_noalloc(int64_t n, const double *x, const double *y,
                                            const double *z, const double *h, int64_t *offsets,
                                            int32_t *idx, int64_t cap, void *cuda_stream)
{
    if (n < 0 || n > kMaxN)
        return fail(SPH_ERR_ARG, "sph_neighbors_noalloc: n must be in [0, 16384]");
    if (!offsets || cap < 0 || (cap > 0 && !idx) || (n > 0 && (!x || !y || !z || !h)))
        return fail(SPH_ERR_ARG, "sph_neighbors_noalloc: null pointer or negative cap");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
        cudaGetLastError();
        return fail(SPH_ERR_NODEVICE, "sph_neighbors_noalloc: no CUDA device");
    }
    // an error left pending by earlier, unrelated runtime calls is not ours
    cudaGetLastError();
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    unsigned char *base = nullptr;
    sph_status st0 = scratch_address(&base);
    if (st0 != SPH_OK) return st0;
    if (cudaMemsetAsync(offsets, 0, (size_t)(n + 1) * sizeof(int64_t), stream) != cudaSuccess) {
        cudaGetLastError();
        return fail(SPH_ERR_CUDA, "sph_neighbors_noalloc: memset of offsets failed");
    }
    if (n == 0) {
        if (cudaStreamSynchronize(stream) != cudaSuccess) {
            cudaGetLastError();
            return fail(SPH_ERR_CUDA, "sph_neighbors_noalloc: stream synchronisation failed");
        }
        return SPH_OK;
    }

    Scratch s{};
    s.perm = (int32_t *)(base + kPerm);
    s.keys[0] = (unsigned long long *)(base + kKeys0);
    s.keys[1] = (unsigned long long *)(base + kKeys1);
    s.vals[0] = (uint32_t *)(base + kVals0);
    s.vals[1] = (uint32_t *)(base + kVals1);
    s.hist = (uint32_t *)(base + kHist);
    s.radix_tot = (uint32_t *)(base + kRadixTot);
    s.xs = (double *)(base + kXs);
    s.ys = (double *)(base + kYs);
    s.zs = (double *)(base + kZs);
    s.hs = (double *)(base + kHs);
    s.tys = base + kTys;
    s.rec = (float4 *)(base + kRec);
    s.pos4 = (float4 *)(base + kPos4);
    s.nbr = (int32_t *)(base + kNbr);
    s.ncnt = (int32_t *)(base + kNcnt);
    // candidate lists are built on every call (skin 0 after the reset) and
    // screened in place into the exact lists
    s.vlist = s.nbr;
    s.vcnt = (int32_t *)(base + kVcnt);
    s.pos_build = (float4 *)(base + kPosBuild);
    s.nodes = (float4 *)(base + kNodes);
    s.leaf_start = (int32_t *)(base + kLeafStart);
    s.leaf_star = (int32_t *)(base + kLeafStar);
    s.leaf_of = (int32_t *)(base + kLeafOf);
    s.bbox_partial = (double *)(base + kBoxPart);
    s.bbox_done = (unsigned int *)(base + kBoxDone);
    s.sc = (DevScalars *)(base + kSc);
    double *mass = (double *)(base + kMass);
    uint8_t *type = base + kType;

    // Plans (host arithmetic only).
    SortPlan plan{};
    plan.key_bits_axis = bits_for_n(n);
    plan.star_bits = 0;
    plan.nstars = 1;
    plan.passes = (3 * plan.key_bits_axis + 7) / 8;
    plan.ipt = 1;
    plan.nblocks = (int)((n + 255) / 256);
    int nleaves = (int)((n + kLeaf - 1) / kLeaf);
    TreeLevels tl{};
    make_tree_levels(nleaves, tl, nullptr);

    // Scratch state that must start at zero on every call (the DevScalars
    // block holds the error word, the counters and the default wait limit).
    bool ok = cudaMemsetAsync(s.bbox_done, 0, sizeof(unsigned int), stream) == cudaSuccess &&
              cudaMemsetAsync(s.sc, 0, sizeof(DevScalars), stream) == cudaSuccess &&
              cudaMemsetAsync(mass, 0, (size_t)n * sizeof(double), stream) == cudaSuccess &&
              cudaMemsetAsync(type, 0, (size_t)n, stream) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        return fail(SPH_ERR_CUDA, "sph_neighbors_noalloc: scratch reset failed");
    }
    k_leaf_layout<<<(int)((n + 256) / 256), 256, 0, stream>>>(n, nleaves, s.leaf_start,
                                                               s.leaf_star, s.leaf_of);
    DevState st{};
    st.n = n;
    st.x = x;
    st.y = y;
    st.z = z;
    st.vx = st.vy = st.vz = nullptr;
    st.S = nullptr;
    st.h = h;
    st.m = mass;
    st.mu = nullptr;
    st.type = type;
    st.star = nullptr;
    launch_build(st, s, plan, tl, nleaves, 0, stream, nullptr);
    // the tile kernel without the density pass reads no rate or EoS field
    launch_tiles(st, s, tl, nleaves, 0, kCap, 0, DevEos{}, DevMetric{}, DevRates{}, stream);
    if (cudaGetLastError() != cudaSuccess)
        return fail(SPH_ERR_CUDA, "sph_neighbors_noalloc: a neighbour-search launch failed");
    launch_export_counts(s, n, offsets, stream);
    launch_scan_i64(offsets, n + 1, stream);
    if (cudaGetLastError() != cudaSuccess)
        return fail(SPH_ERR_CUDA, "sph_neighbors_noalloc: the count or scan launch failed");
    int64_t tot = 0;
    int err = 0;
    if (cudaMemcpyAsync(&tot, offsets + n, sizeof(int64_t), cudaMemcpyDeviceToHost, stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(&err, &s.sc->err, sizeof(int), cudaMemcpyDeviceToHost, stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess) {
        cudaGetLastError();
        return fail(SPH_ERR_CUDA, "sph_neighbors_noalloc: kernel or copy failed");
    }
    if (err & ERR_NONFINITE) return fail(SPH_ERR_NONFINITE, "sph_neighbors_noalloc: non-finite x or h");
    if (err & ERR_TIMEOUT) return fail(SPH_ERR_TIMEOUT, "sph_neighbors_noalloc: sort wait timed out");
    if (err & ERR_CAPACITY)
        return fail(SPH_ERR_CAPACITY,
                    "sph_neighbors_noalloc: a particle has more than 128 neighbours, or a leaf "
                    "more than 256 candidate leaves");
    if (err & ERR_BOUNDS) return fail(SPH_ERR_BOUNDS, "sph_neighbors_noalloc: index out of bounds");
    if (tot > cap) return fail(SPH_ERR_CAPACITY, "sph_neighbors_noalloc: lists exceed cap");
    launch_export_fill(s, n, kCap, offsets, idx, stream);
    if (cudaGetLastError() != cudaSuccess)
        return fail(SPH_ERR_CUDA, "sph_neighbors_noalloc: the export launch failed");
    if (cudaStreamSynchronize(stream) != cudaSuccess) {
        cudaGetLastError();
        return fail(SPH_ERR_CUDA, "sph_neighbors_noalloc: export failed");
    }
    return SPH_OK;
}
