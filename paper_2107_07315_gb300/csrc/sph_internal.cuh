// Internal declarations shared by the libsph translation units.
//
// Data layout in device memory (n particles, "sorted" = Hilbert-curve order):
//   caller order : the caller's state and rate buffers (borrowed).
//   perm[n]      : sorted slot -> caller index (int32).
//   xs,ys,zs,hs  : FP64 sorted positions and smoothing lengths.
//   rec[4][n]    : float4 j-record of each sorted particle, one array per
//                  field (structure of arrays: a warp gathering one field of
//                  nearby neighbours touches few cache lines):
//                  0 (Xhi.x, Xhi.y, Xhi.z, h)  1 (Xlo.x, Xlo.y, Xlo.z, m)
//                  2 (v.x, v.y, v.z, D)         3 (P/D^2, c_s, 1/D, solid)
//                  Xhi + Xlo is the FP64 position split into an FP32 value
//                  on a power-of-two grid and an FP32 remainder.
//   rec64[n][3]  : double4_32a j-record of the FP64 path: (x,y,z,h), (m,vx,vy,vz),
//                  (D, 1/D, P/D^2, c_s).
//   sd2 / sd264  : S/D^2 per sorted particle: sd2[2][n] float4 (xx,yy,zz,xy),
//                  (xz,yz,0,0); sd264[n][8] doubles.
//   pp / pp64    : per-particle EoS values for the finalize step:
//                  (rho, P, dP/drho, h_enth), (W~, c_s, D, 0).
//   pos4[n]      : float4 fl32(x, y, z, h) per sorted particle (leaf boxes).
//   tree nodes   : implicit 8-ary tree over leaves of 8 consecutive sorted
//                  particles of one star; node = float4 (lo.xyz, h_max) +
//                  float4 (hi.xyz, star range packed in the float bits).
//   vlist[n*cap] : candidate list of each sorted particle (ascending): every
//                  b with |x_a - x_b| < (1 + eps)(h_a + h_b) when it was built
//                  (pair-tile search), vcnt[n] its length; pos_build[n] the
//                  fl32 positions and h it was built from.  Reused while no
//                  particle can have moved or grown into a pair it misses.
//   nbr[n*cap]   : exact neighbour list of each sorted particle (ascending),
//                  ncnt[n] its length; screened from vlist every right-hand
//                  side.
//   star_box[6][nstars] : several stars only: each star's fl32 bounding box
//                  (order-preserving integer images, lo x y z then hi x y z);
//                  the curve keys of a star are taken over its own box.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/sph.h"

namespace sph {

constexpr int kLeaf = 8;          // particles per tree leaf
constexpr int kBranch = 8;        // children per tree node
constexpr int kMaxLevels = 16;
constexpr int kTreeBlock = 64;    // leaves per block in the tree kernel (8^2)
constexpr int kTreeBlockLevels = 2;
constexpr int kCandCap = 256;     // candidate leaves per leaf (pair tiles per leaf)
constexpr int kRowCap = 1024;     // largest max_neighbors (list capacity per particle)
constexpr int kRowCapDefault = 256;  // list capacity per particle when max_neighbors is 0

// Device error word bits.
enum : int {
    ERR_CAPACITY = 1,
    ERR_NONFINITE = 2,
    ERR_BOUNDS = 4,
    ERR_TIMEOUT = 8,
};

// Device scalars shared between kernels of one right-hand side.
struct DevScalars {
    unsigned long long bbox_lo[3];   // order-preserving encodings of doubles
    unsigned long long bbox_hi[3];
    double grid;                     // Xhi grid spacing (power of two)
    double grid_inv;                 // 1/grid (exact)
    double inv_ext[3];               // 1/(bbox extent) per axis, for the curve keys
    float key_lo_f[3], key_scale_f[3];  // FP32 copies of the box corner and 1/extent
    float grid_f, grid_inv_f;        // FP32 copies of grid and 1/grid (powers of two)
    double eps_abs;                  // absolute slack for tree pruning
    float eps_abs_f;                 // FP32 copy
    float band_abs;                  // absolute part of the FP32 screening band (48 grid 2^-24)
    int err;                         // ERR_* bits
    int tree_done;                   // block counter of the tree kernel
    int max_cand;                    // most candidate leaves of one leaf (last right-hand side)
    int max_count;                   // most neighbours of one particle (last right-hand side)
    unsigned int tile_next[8];       // next sort tile of each radix pass
    int spin_limit;                  // polls of a look-back wait before it gives up
    unsigned long long pairs_last;   // ordered pairs of the last RHS
    unsigned long long pairs_total;
    unsigned long long rechecks;     // marginal FP64 predicate evaluations
    unsigned long long rhs_count;
    unsigned long long tiles_last;   // candidate (leaf, leaf) tiles of the last build
    // candidate-list reuse (all FP32 as bit patterns of non-negative floats
    // where noted, so atomicMax orders them)
    float skin;                      // eps of the candidate lists (< 0: rebuild every RHS)
    unsigned int q_max;              // largest d_a / h_a0 + g_a since the build (float bits)
    int built;                       // candidate lists exist for the current order
    int resorted;                    // this RHS sorted along the curve again
    int rebuild;                     // this RHS rebuilds the candidate lists
    float xmax_f;                    // largest |coordinate| (for the displacement bound)
    unsigned long long builds;       // candidate-list builds so far
    // work queue of the persistent right-hand-side kernel (reset per RHS)
    unsigned int pq_head;            // next item to dequeue
    unsigned int pq_done;            // screening items completed
};
// the autotuner clears both queue counters with one 8-byte memset
static_assert(offsetof(DevScalars, pq_done) == offsetof(DevScalars, pq_head) + sizeof(unsigned int),
              "pq_head and pq_done must be adjacent");

struct DevState {
    int64_t n;
    const double *x, *y, *z;
    const double *vx, *vy, *vz;      // velocity used by the RHS (may be predicted)
    const double *S;                 // stress used by the RHS (may be predicted)
    const double *h, *m, *mu;
    const uint8_t *type;
    const int32_t *star;             // may be null
};

// Equation of state per star: P = K rho^Gamma (Eq. poly_eos), or a piecewise
// polytrope (npieces > 1): piece k of star s holds rho >= rho_b[s*(np-1)+k-1]
// with Kp, Gp and the energy constant ap (u = a + K rho^(Gamma-1)/(Gamma-1))
// at [s*np + k], K and a fixed by continuity of P and u.
struct DevEos {
    const double *K, *Gamma;
    int npieces;
    const double *rho_b, *Kp, *Gp, *ap;
    // FP32 copies for the mixed-precision kernels
    const float *Kf, *Gf, *rho_bf, *Kpf, *Gpf, *apf;
};

// The piece of star s's EoS that holds density rho: K, Gamma and a.
template <typename T>
__device__ __forceinline__ void eos_piece(const DevEos &e, int s, T rho, T &K, T &G, T &a)
{
    if (e.npieces <= 1) {
        K = (T)e.K[s];
        G = (T)e.Gamma[s];
        a = (T)0;
        return;
    }
    int k = 0;
    for (int j = 0; j + 1 < e.npieces; ++j)
        if (rho >= (T)e.rho_b[s * (e.npieces - 1) + j]) k = j + 1;
    const int o = s * e.npieces + k;
    K = (T)e.Kp[o];
    G = (T)e.Gp[o];
    a = (T)e.ap[o];
}

struct DevMaterial {
    double alpha_av, beta_av, eta2;
    int jaumann, yield_mode, break_stress, break_zero_S;
    float alpha_f, beta_f, eta2_f;  // FP32 copies
};

// FP32 per-star constants of the background and the external field
// (DevMetric::fstar, kFStar floats per star): table radius and mass, the
// centre split into hi + lo floats, the external table radius, wall radius
// and centre.
enum {
    FS_RMAX = 0, FS_M = 1, FS_CHI = 2, FS_CLO = 5, FS_EXT_RMAX = 8, FS_EXT_RWALL = 9,
    FS_EXT_CHI = 10, FS_EXT_CLO = 13, kFStar = 16
};

// Background fields of the right-hand side: the fixed metric (Sec. I.C) and
// the external field of the relaxation (Sec. II.A).
struct DevMetric {
    int kind, nstars, nr, pressure_form;
    const double *r_max, *M, *center;
    const double *tab;   // [nstars][nr][4]: alpha, dalpha, psi4, dpsi4
    const float *tabf;   // FP32 copy
    // external field: radial g_eff on nodes 0..ext_rmax (0 beyond), a wall
    // -k_wall (r - r_wall) beyond r_wall, damping -damping v; ext_kind 0: off
    int ext_kind, ext_nr;
    const double *ext_rmax, *ext_center, *ext_rwall;
    const double *ext_g;  // [nstars][ext_nr]
    const float *ext_gf;  // FP32 copy
    double k_wall, damping;
    float k_wall_f, damping_f;
    const float *fstar;   // [nstars][kFStar] FP32 per-star constants
};

struct DevRates {
    double *ax, *ay, *az, *dudt, *drhodt, *rho, *P, *D, *cs;
    double *deps, *dR, *dS;
    int32_t *ncount;
};

struct TreeLevels {
    int nlevels;
    int count[kMaxLevels];
    int offset[kMaxLevels];
};

// Level sizes of the implicit 8-ary tree over nleaves leaves (level 0 =
// leaves, last level = root).  Returns false if it needs too many levels.
inline bool make_tree_levels(int nleaves, TreeLevels &tl, int64_t *total_nodes)
{
    tl.nlevels = 0;
    int64_t total = 0;
    if (nleaves > 0) {
        int cnt = nleaves;
        while (true) {
            if (tl.nlevels >= kMaxLevels) return false;
            tl.count[tl.nlevels] = cnt;
            tl.offset[tl.nlevels] = (int)total;
            total += cnt;
            tl.nlevels++;
            if (cnt == 1) break;
            cnt = (cnt + kBranch - 1) / kBranch;
        }
    }
    if (total_nodes) *total_nodes = total;
    return true;
}

// Scratch of one context (device pointers).
struct Scratch {
    int32_t *perm;
    unsigned long long *keys[2];
    uint32_t *vals[2];
    uint32_t *hist;           // sort tile status: [passes][nblocks][256] 64-bit words
    uint32_t *radix_tot;      // [8][256] digit totals per pass
    double *xs, *ys, *zs, *hs;
    uint8_t *tys;             // sorted type
    float4 *rec;              // [4][n]
    float4 *pos4;             // [n] fl32(x, y, z, h) for neighbour screening
    double4_32a *rec64;           // [n][3]
    float4 *sd2;              // [2][n]
    double *sd264;            // [n][8]
    float4 *pp;               // [n][2]
    double *pp64;             // [n][8]
    int32_t *vlist;           // [n][cap] (may alias nbr: then rebuilt every RHS)
    int32_t *vcnt;            // [n]
    float4 *pos_build;        // [n]
    int32_t *nbr;             // [n][cap]
    int32_t *ncnt;            // [n]
    float4 *nodes;            // [total nodes][2]
    int32_t *leaf_start;      // [nleaves+1]
    int32_t *leaf_star;       // [nleaves]
    int32_t *leaf_of;         // [n] leaf of each sorted slot
    double *bbox_partial;     // [6 * 304]
    unsigned int *bbox_done;  // block counter of the bounding-box kernel
    uint32_t *star_box;       // [6][nstars] per-star fl32 box (several stars; else null)
    DevScalars *sc;
};

// Launch helpers implemented in sph_build.cu.
struct SortPlan {
    int key_bits_axis;  // cell bits per axis of the curve key
    int star_bits;
    int nstars;         // stars in the index space (per-star curve boxes when > 1)
    int passes;         // 8-bit digit passes
    int ipt;            // items per thread in sort kernels
    int nblocks;        // sort tiles
};

constexpr int kBoxBlocksMax = 304;

// Bounding box, curve keys and sort, sorted gather and leaf tree.  resort
// false keeps the particle order of s.perm (the last sort) instead of sorting
// along the curve again: the sorted copies and the tree are still rebuilt
// from the current positions and h.
void launch_build(const DevState &st, const Scratch &s, const SortPlan &plan,
                  const TreeLevels &tl, int nleaves, int fp64_records, cudaStream_t stream,
                  int *nlaunch, bool resort = true);

// Candidate lists from pair tiles (sph_tiles.cu), when the tree kernel found
// them stale (or always, with a negative skin): per leaf, the candidate leaves
// (tree walk) and, per particle, every b within (1 + eps)(h_a + h_b).  Then
// the exact lists and counts screened from the candidates, and with density
// true (mixed precision) the density summation and the equation of state.
// cap: list capacity per particle (SPH_ERR_CAPACITY above it).
void launch_tiles(const DevState &st, const Scratch &s, const TreeLevels &tl, int nleaves,
                  int multi_star, int cap, int density, const DevEos &eos, const DevMetric &g,
                  const DevRates &out, cudaStream_t stream, int *nlaunch = nullptr,
                  int screen_lanes = 4, int group = 1);

// Exact screening (with the density and equation of state when density is
// true) alone, from the candidate lists of the last build; the autotuner
// times it.
void launch_screen(const DevState &st, const Scratch &s, int cap, int density,
                   const DevEos &eos, const DevMetric &g, const DevRates &out,
                   cudaStream_t stream, int screen_lanes);

// Candidate-list build alone (the kernel returns at once unless the tree
// kernel asked for a rebuild).
// group: tree leaves per tile-search walk (1, 2 or 4: a search leaf of 8, 16
// or 32 particles; the candidate lists are the same for each).  With a list
// capacity above kRowCapDefault the walk takes one tree leaf and holds 1024
// candidate leaves (group is ignored).
void launch_tiles_build(const DevState &st, const Scratch &s, const TreeLevels &tl, int nleaves,
                        int multi_star, int cap, cudaStream_t stream, int group = 1);

// Persistent right-hand side, mixed precision (one launch): grid blocks
// dequeue items from a global counter; items 0 .. nA-1 screen a block of
// particles (exact lists, density, equation of state), the rest run the
// force pass of a block of particles once every screening item is done.
// screen_lanes / lanes: threads per particle of the two item kinds.
struct PersistPlan {
    int grid = 0;          // resident blocks (SMs x blocks per SM)
    int n_screen = 0;      // screening items
    int n_force = 0;       // force items
};
PersistPlan plan_persistent(int64_t n, int screen_lanes, int lanes);
void launch_persistent(const DevState &st, const Scratch &s, const DevEos &eos,
                       const DevMaterial &mat, const DevMetric &g, const DevRates &out, int cap,
                       int screen_lanes, int lanes, const PersistPlan &pp, cudaStream_t stream);

// FP64 density summation and equation of state over the neighbour lists.
void launch_density_fp64(const DevState &st, const Scratch &s, const DevEos &eos,
                         const DevMetric &g, const DevRates &out, int cap, int lanes,
                         cudaStream_t stream);

// Force pass over the neighbour lists.  Mixed precision runs an
// all-fluid-block kernel and a solid-block kernel over the same grid; with
// side, fork and join given, the solid-block kernel runs on side (after fork
// is recorded on stream) so the two overlap, and stream waits on join before
// it goes on.
void launch_force(const DevState &st, const Scratch &s, const DevEos &eos,
                  const DevMaterial &mat, const DevMetric &g, const DevRates &out, int cap,
                  int lanes, int fp64, cudaStream_t stream, cudaStream_t side = nullptr,
                  cudaEvent_t fork = nullptr, cudaEvent_t join = nullptr);

// Step kernels (sph_step.cu).
struct StepState {
    int64_t n;
    double *x, *y, *z, *vx, *vy, *vz, *u, *h, *S;
    const double *m;
    uint8_t *type, *flags;
    const int32_t *star;
    double *mu, *Y0, *eps_break;
    double *vp, *Sp;  // predicted velocity (3n) and stress (6n)
};

// Modification step after a relaxation (Sec. II.A): u = K rho^(Gamma-1)/(Gamma-1)
// from the density of the last right-hand side, per star's EoS.
void launch_set_u_from_eos(const StepState &s, const DevRates &r, const DevEos &eos,
                           cudaStream_t stream);

void launch_kick_drift(const StepState &s, const DevRates &r, double dt, cudaStream_t st);
void launch_kick_return(const StepState &s, const DevRates &r, const DevEos &eos,
                        const DevMaterial &mat, double dt, int h_nmin, int h_nmax,
                        cudaStream_t st);
constexpr int kTotalsBlocks = 256;
void launch_totals(const StepState &s, const int32_t *ncount, double *partial, double *out,
                   cudaStream_t st);
// FP64 totals of each star (out[nstars][16]) over the caller indices of each
// star, idx[off[s] .. off[s+1]) ascending.
void launch_star_totals(const StepState &s, const int32_t *ncount, int nstars,
                        const int64_t *off, const int32_t *idx, double *out, cudaStream_t st);
void launch_export_counts(const Scratch &s, int64_t n, int64_t *counts_out,
                          cudaStream_t st);
// Neighbour lists of the last right-hand side in caller order and ascending
// caller index (offsets from the counts by an exclusive scan).
void launch_export_fill(const Scratch &s, int64_t n, int cap, const int64_t *offsets,
                        int32_t *idx, cudaStream_t st);
void launch_scan_i64(int64_t *data, int64_t n, cudaStream_t st);

// Store a message for sph_last_error() on the calling thread (sph_api.cu).
void record_error(const char *msg);

}  // namespace sph
