/*
 * sph.h -- C ABI of libsph: the SPH right-hand side and time step for
 * elastic-perfectly-plastic matter in a fixed GR background
 * (arXiv 2107.07315, Sec. I.B "Solid SPH Equations", Sec. I.C "Fixed metric
 * background", Sec. II.A equation of state).
 *
 * Conventions for every entry point:
 *   - All particle and rate arrays are DEVICE memory owned by the caller,
 *     structure-of-arrays, in the caller's particle order, length n unless
 *     stated.  Symmetric tensors (S, dS, deps) are component-major:
 *     component c of particle a at [c*n + a], order xx, yy, zz, xy, xz, yz;
 *     the antisymmetric rotation rate dR holds xy, xz, yz the same way.
 *   - EoS, material and metric descriptions are HOST memory; sph_init copies
 *     them into memory the library owns.
 *   - Particle buffers passed to sph_init are borrowed: they must stay valid
 *     and in place until sph_free.  sph_step updates them in place.
 *   - Work is enqueued on the CUDA stream given to sph_init.  Calls marked
 *     "asynchronous" return after enqueueing; errors that only the device can
 *     see (list capacity, non-finite state) are reported by sph_sync.
 *   - Every call returns a status and never aborts.  There is no CPU path:
 *     without a usable CUDA device the call returns SPH_ERR_NODEVICE.
 *   - sph_last_error() returns a thread-local message for the last failure.
 */
#ifndef SPH_H
#define SPH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sph_ctx sph_ctx; /* opaque, owned by the library */

typedef enum {
    SPH_OK = 0,
    SPH_ERR_ARG = 1,        /* invalid argument (null pointer, bad size, ...) */
    SPH_ERR_CUDA = 2,       /* a CUDA runtime call failed */
    SPH_ERR_OOM = 3,        /* device allocation failed */
    SPH_ERR_CAPACITY = 4,   /* a neighbour list exceeded its capacity */
    SPH_ERR_TIMEOUT = 5,    /* a bounded device-side wait gave up */
    SPH_ERR_NONFINITE = 6,  /* non-finite position, velocity or smoothing length */
    SPH_ERR_BOUNDS = 7,     /* a checked index fell outside its buffer */
    SPH_ERR_NODEVICE = 8    /* no usable CUDA device */
} sph_status;

typedef enum {
    SPH_FP64 = 0,  /* pair sums and per-particle terms in FP64 (reference form) */
    SPH_MIXED = 1  /* pair sums in FP32 (compensated density and energy sums),
                      FP64 state, integration and totals */
} sph_precision;

/* Particle state (device, caller order).  Sec. I.B: positions x, velocity v
 * (the coordinate velocity dx/dt of Sec. I.C when a metric is given),
 * specific internal energy u, smoothing length h, baryonic mass m, deviatoric
 * stress S.  type: 0 fluid core, 1 solid crust (Sec. III).  flags: bit0 set
 * when the last step scaled S back to the yield surface, bit1 set (sticky)
 * once the maximum-strain test fired.  star: star index per particle, or
 * NULL for a single star; particles of different stars never interact.
 * mu, Y0, eps_break: shear modulus, yield stress and breaking strain per
 * particle (read for solid particles only; may be NULL if none is solid). */
typedef struct {
    int64_t n;
    double *x, *y, *z, *vx, *vy, *vz, *u, *h, *m;
    double *S;            /* 6*n */
    uint8_t *type, *flags;
    int32_t *star;        /* may be NULL */
    double *mu, *Y0, *eps_break;
} sph_particles;

/* Polytropic equation of state per star, P = K rho^Gamma (Eq. poly_eos), or a
 * piecewise polytrope ("several polytropic models ... connected", Sec. II.A,
 * after Read et al. 2009).  npieces 0 or 1: one polytrope (the other piece
 * fields are ignored and may be NULL).  npieces = p in 2..8: K[s], Gamma[s]
 * give piece 0; piece k+1 starts at rho_bound[s*(p-1)+k] (positive,
 * increasing) with exponent Gamma_above[s*(p-1)+k] > 1; its K follows from
 * continuity of P and u = a + K rho^(Gamma-1)/(Gamma-1) from continuity of u.
 * All host arrays; fields after Gamma may be zero-initialised by callers that
 * use one polytrope. */
typedef struct {
    int32_t nstars;
    const double *K, *Gamma; /* host arrays of nstars */
    int32_t npieces;
    const double *rho_bound, *Gamma_above;
} sph_eos;

/* Material and scheme options (host).  alpha_av, beta_av, eta2: Monaghan
 * artificial viscosity Pi_ab (named in Sec. I.B, form not given there).
 * jaumann: 0 objective rotation term R.S - S.R, 1 the printed S.R - R.S
 * (Eq. solid4).  yield_mode: 0 f = min(Y0^2/sv^2, 1) as printed, 1 with the
 * square root.  break_stress: 0 principal stresses of -P I + S, 1 of S.
 * break_zero_S: 1 zeroes S and mu of a particle once it breaks. */
typedef struct {
    double alpha_av, beta_av, eta2;
    int32_t jaumann, yield_mode, break_stress, break_zero_S;
} sph_material;

/* Fixed background metric (Sec. I.C), host tables.  kind 0: none.  kind 1:
 * static isotropic ds^2 = -alpha^2 dt^2 + psi^4 dx.dx per star, tabulated
 * on nr uniform nodes over [0, r_max[s]] around center[3*s..]: alpha,
 * d alpha/dr, psi^4, d psi^4/dr (arrays of nstars*nr, star-major); beyond
 * r_max the exterior Schwarzschild form with mass M[s].  pressure_form 0
 * divides dP by W~^2 rho h (from div T = 0), 1 by W~ rho h as printed. */
typedef struct {
    int32_t kind, nstars, nr, pressure_form;
    const double *r_max, *alpha, *dalpha, *psi4, *dpsi4, *M, *center;
} sph_metric;

/* External field of the particle relaxation (Sec. II.A), host tables.  The
 * relaxation confines the particles in phi_eff = -K Gamma rho_t^(Gamma-1) /
 * (Gamma-1) of a target density profile rho_t(r); g holds the radial
 * component of g_eff = -grad phi_eff (negative = inward) per star on nr
 * uniform nodes over [0, r_max[s]] around center[3*s..], zero beyond r_max.
 * Readings of passages the paper leaves open: beyond r_wall[s] a wall adds
 * -k_wall (r - r_wall) along r_hat ("potential walls"), and every particle
 * feels -damping v, which lets the particles settle into equilibrium.
 * kind 0 switches the field off. */
typedef struct {
    int32_t kind, nstars, nr, reserved;
    const double *r_max, *g, *center, *r_wall;
    double k_wall, damping;
} sph_external;

/* Rates and derived fields (device, caller order), all length n unless
 * noted: acceleration a (Eq. solid2 plus the background force of Sec. I.C),
 * du/dt (Eq. solid3), continuity rate (Eq. solid1 with the computational
 * density D of Sec. I.C), rest-mass density rho, pressure P, D, sound speed
 * cs, strain rate deps (6n, Eq. solid5), rotation rate dR (3n, Eq. solid6),
 * stress rate dS (6n, Eq. solid4), neighbour count ncount (int32). */
typedef struct {
    double *ax, *ay, *az, *dudt, *drhodt, *rho, *P, *D, *cs;
    double *deps, *dR, *dS;
    int32_t *ncount;
} sph_rates;

/* Run options (host); NULL in sph_init means the defaults in brackets.
 * h_nmin, h_nmax: after each step multiply h by 1.0625 when the neighbour
 * count is below h_nmin and by 0.9375 above h_nmax [0, 0: off].
 * max_neighbors: most neighbours a particle may have (1..1024; the
 * candidate list of a particle, every pair within (1 + skin)(h_a + h_b),
 * must fit too); more raise SPH_ERR_CAPACITY at sph_sync.  The context
 * holds two int32 lists of this length per particle [0: 256].
 * lanes_per_particle: 4 or 8 threads share one particle's list in the pair
 * kernels [0: 8]; -1 turns on the autotuner of the launch shape: sph_init
 * evaluates one right-hand side on the bound state (writing the rates),
 * then times the exact screening with 4 and 8 threads per particle, the
 * pair kernels with 4 and 8 and the candidate build with search_leaves 1, 2
 * and 4, keeps the fastest of each and restores the counters.  The
 * choice is cached for the process under (device, n, stars, precision,
 * max_neighbors, metric, any solid), so a later context of that
 * configuration reuses it without timing.  Lane counts set the order of the
 * density and pair sums: a tuned context agrees with a fixed one to
 * rounding.  sph_stats reports the shape and the times.
 * screen_lanes: threads per particle of the exact screening, 4 or 8 [0: 4];
 * ignored when lanes_per_particle is -1.
 * search_leaves: tree leaves (8 sorted particles each) that share one walk
 * of the candidate-list search, 1, 2 or 4; the candidate lists are the same
 * for each, only the cost of a build differs; a walk holds at most 256
 * candidate leaves for 1 and 512 for 2 or 4 (1024 with one tree leaf per
 * walk when max_neighbors is above 256) [0: 1; with lanes_per_particle
 * -1 the autotuner times all three and takes the fastest whose walk fills at
 * most half of its capacity on the bound state].
 * persistent: 1 runs the exact screening, density, equation of state and
 * force pass of every right-hand side as one persistent launch over a global
 * work queue of particle blocks (screening items first, then force items,
 * which wait with a bounded poll until every screening item is done; a wait
 * that runs out gives SPH_ERR_TIMEOUT at sph_sync); mixed precision only,
 * ignored in FP64; -1 lets sph_init time both forms (of the chosen lane
 * counts) and keep the faster, cached like the lane counts [0: separate
 * launches].  Same sums in the same order as the separate launches of the
 * same lane counts: the rates are identical either way.
 * use_graph: capture each step in a CUDA graph [1].
 * totals_every: compute totals every k steps inside sph_step [0: never].
 * sort_every: sph_step sorts the particles along the space-filling curve on
 * steps 0, k, 2k, ... (counted by the step counter) and keeps the last
 * sort's order on the others; every step still rebuilds the tree and
 * screens the exact neighbour lists from the current positions, so the
 * lists are the same sets (only the order of pair sums, hence rounding,
 * depends on k) [0 or 1: every step].  sph_rhs always sorts.
 * skin: the neighbour search builds candidate lists of every pair within
 * (1 + skin)(h_a + h_b) and screens them exactly on every right-hand side;
 * it builds them again after a curve sort, after sph_set_state or
 * sph_set_max_neighbors, or once a particle may have moved or grown into a
 * pair they miss (a device-side test: the largest displacement over own h
 * plus relative h growth of any particle since the build reaching skin),
 * so the exact lists are the same as with lists built every time [0: 0.1;
 * negative: build on every right-hand side; at most 1]. */
typedef struct {
    int32_t h_nmin, h_nmax;
    int32_t max_neighbors;
    int32_t lanes_per_particle;
    int32_t use_graph;
    int32_t totals_every;
    int32_t sort_every;
    double skin;
    int32_t screen_lanes;
    int32_t persistent;
    int32_t search_leaves;
} sph_options;

/* Create a context bound to the particle buffers.  Validates the inputs,
 * allocates scratch sized for n particles, copies EoS, material and metric
 * to the device.  metric may be NULL (no background).  cuda_stream is a
 * cudaStream_t (NULL: the legacy default stream).  Synchronous. */
sph_status sph_init(sph_ctx **out, const sph_particles *particles, const sph_eos *eos,
                    const sph_material *material, const sph_metric *metric,
                    sph_precision precision, const sph_options *options, void *cuda_stream);

/* Right-hand side at the bound state: Hilbert-curve sort, neighbour lists, density
 * summation (Sec. I.C "standard formula"), equation of state, pair sums of
 * Eqs. solid1-solid6, stress rate (Eq. solid4) and background force
 * (Sec. I.C), written to *out (device arrays of the caller).  Asynchronous. */
sph_status sph_rhs(sph_ctx *ctx, const sph_rates *out);

/* Advance nsteps kick-drift-kick steps of size dt: half kick, drift,
 * right-hand side at the predicted velocity and stress, half kick, von Mises
 * scaling (Sec. I.B), maximum-strain test (Sec. I.B), smoothing-length
 * update.  Updates the bound particle buffers in place.  Asynchronous. */
sph_status sph_step(sph_ctx *ctx, double dt, int32_t nsteps);

/* Wait for the context's stream and report device-side errors raised since
 * the last call (capacity, non-finite input, bounds, timeouts), then clear
 * them.  A timed-out sort is reported as SPH_ERR_TIMEOUT: every kernel of
 * that right-hand side that would read the sorted order returns without
 * work, and so do those of later ones until sph_sync clears the error. */
sph_status sph_sync(sph_ctx *ctx);

/* Bound on the context's device-side waits.  A sort tile that has made
 * `polls` rounds of reads of its predecessors' published counts without
 * finding its prefix (decoupled look-back), and a force item of the
 * persistent launch (options.persistent) that has polled the count of
 * finished screening items `polls` times, give up and raise the timeout
 * reported by sph_sync.  polls < 0 restores the default (2^22); 0 makes
 * every such wait give up at its first poll (a way to exercise the timeout
 * path: on inputs of more than one sort tile, n > 256, or on a persistent
 * step without a curve sort).  Library service, no counterpart in the
 * paper.  Synchronous.  Errors: SPH_ERR_ARG (NULL ctx), SPH_ERR_CUDA. */
sph_status sph_set_wait_limit(sph_ctx *ctx, int32_t polls);

/* Change the list capacity per particle (max_neighbors, 1..1024) of a live
 * context: the candidate and exact lists are allocated again at the new
 * length (the old ones freed), the step graphs are captured again and the
 * next right-hand side builds the candidate lists again.  With
 * sph_get_state / sph_set_state this is the host-side retry after
 * SPH_ERR_CAPACITY: restore the state saved before the failed steps, grow
 * the capacity, step again; the result equals a run with the larger capacity
 * from the start.  Library service, no counterpart in the paper.
 * Synchronous.  Errors: SPH_ERR_ARG, SPH_ERR_OOM (the old lists are kept),
 * SPH_ERR_CUDA. */
sph_status sph_set_max_neighbors(sph_ctx *ctx, int32_t max_neighbors);

/* Bounds-checked builds (libsph_checked.so, compiled with -DSPH_CHECKED):
 * every list entry and permutation entry is tested against the particle
 * range before it is used for an access; one outside raises a device error
 * flag, the access goes to an index in range, and sph_sync reports
 * SPH_ERR_BOUNDS.  sph_build_checked returns 1 in such a build, 0 otherwise.
 * Library service (stands in for a memory sanitizer), no counterpart in the
 * paper. */
int32_t sph_build_checked(void);

/* Checked builds only (SPH_ERR_ARG otherwise): overwrite entry k of the
 * candidate list of sorted slot `slot` with `value`, to exercise the bounds
 * check from the host.  The next right-hand side that reuses the candidate
 * lists (no curve sort and no rebuild) reads it.  Synchronous.  Errors:
 * SPH_ERR_ARG (NULL ctx, slot or k out of range, unchecked build),
 * SPH_ERR_CUDA. */
sph_status sph_checked_set_candidate(sph_ctx *ctx, int64_t slot, int32_t k, int32_t value);

/* Neighbour lists of the last right-hand side, CSR in caller order with
 * ascending caller indices (b in N(a) iff b != a, same star and
 * |x_a - x_b| < h_a + h_b, Sec. I.B).  offsets: device int64[n+1];
 * idx: device int32[cap].  Returns SPH_ERR_CAPACITY (offsets written, idx
 * not) when the lists hold more than cap entries.  Synchronous. */
sph_status sph_neighbors(sph_ctx *ctx, int64_t *offsets, int32_t *idx, int64_t cap);

/* Totals of the bound state, FP64, fixed reduction order (host out[16]):
 * 0 mass, 1-3 momentum, 4 kinetic, 5 internal, 6 total energy, 7-9 angular
 * momentum, 10 particles yielded in the last step, 11 broken particles,
 * 12 mean neighbour count of the last right-hand side, 13-15 centre of
 * mass.  Synchronous. */
sph_status sph_totals(sph_ctx *ctx, double out[16]);

/* Totals of each star separately, the quantities of sph_totals over the
 * particles of star s only (star index of sph_particles; all particles form
 * star 0 when it is NULL): host out[nstars * 16], row s holding star s.
 * Each star is reduced in FP64 over its particles in ascending caller
 * index, in a fixed order, so the result does not depend on the curve order.
 * These are what the batched ensemble gathers from several GPUs.
 * Synchronous.  Errors: SPH_ERR_ARG (NULL, nstars differs from the
 * context's), SPH_ERR_CUDA. */
sph_status sph_totals_per_star(sph_ctx *ctx, double *out, int32_t nstars);

/* Counters (host out[32]): 0 ordered neighbour pairs of the last right-hand
 * side, 1 pairs summed over all right-hand sides, 2 right-hand sides
 * evaluated, 3 kernel launches in the last step, 4 tree leaves, 5 marginal pairs
 * re-checked in FP64 (cumulative), 6 neighbour capacity per particle,
 * 7 lanes per particle, 8 1 if steps run as a CUDA graph, 9 steps taken,
 * 10 radix passes, 11 cell bits per axis of the curve key, 12 kernel
 * launches issued by sph_step (cumulative), 13 steps per curve sort,
 * 14 most candidate leaves of one tile-search walk and 16 candidate (leaf, leaf) tiles
 * in all (both of the last candidate-list build), 15 most neighbours of one
 * particle (last right-hand side), 17 1 for mixed precision, 18 candidate-list
 * builds so far, 19 lanes per particle of the exact screening, 20 launch
 * shape source (0 fixed by the options, 1 timed by sph_init, 2 taken from the
 * process cache), 21-24 the autotuner's times in ns per launch (screening
 * with 4 and 8 lanes, pair kernels with 4 and 8 lanes; zero when not tuned),
 * 25 blocks of the persistent right-hand-side launch (0: separate launches),
 * 26 and 27 the autotuner's times in ns of the screening and pair kernels in
 * series and of the persistent launch (zero unless persistent is -1),
 * 28-30 the autotuner's times in ns of a candidate build with search leaves
 * of 1, 2 and 4 tree leaves (zero when not tuned), 31 tree leaves per
 * search leaf in use.  Synchronous. */
sph_status sph_stats(sph_ctx *ctx, int64_t out[32]);

/* Device-time measurement with CUDA events on the context's stream.
 * enable 1 starts recording around the kernels of every step or right-hand
 * side; sph_timing_read returns (host out[12]) summed milliseconds and
 * sample counts: 0/1 force kernels, 2/3 FP64 density kernel (zero in mixed
 * precision, where the screening kernel sums the density), 4/5 whole steps
 * (or right-hand sides), 6/7 bounding box through tree (keys, sort, gather,
 * tree), 8/9 neighbour lists (the pair-tile candidate build when stale and
 * the exact screening; in mixed precision also the density and equation of
 * state), 10/11 both (6 plus 8).  With the persistent launch 8/9 hold the
 * candidate build only and 0/1 the persistent launch (screening, density,
 * equation of state and force).  Reading resets the sums.  Synchronous. */
sph_status sph_timing(sph_ctx *ctx, int32_t enable);
sph_status sph_timing_read(sph_ctx *ctx, double out[12]);

/* Checkpoint: the bound particle state plus the rates carried between steps,
 * flags, the step counter and the particle order of the last curve sort, as
 * an opaque host blob.  sph_state_size gives
 * its size; sph_get_state writes it; sph_set_state restores it so that
 * continuing reproduces an uninterrupted run bit for bit.  Synchronous. */
sph_status sph_state_size(sph_ctx *ctx, int64_t *bytes);
sph_status sph_get_state(sph_ctx *ctx, void *host_buf, int64_t bytes);
sph_status sph_set_state(sph_ctx *ctx, const void *host_buf, int64_t bytes);

/* Switch the external relaxation field on (kind 1) or off (NULL or kind 0)
 * for later right-hand sides and steps (Sec. II.A).  The tables are copied
 * into device memory owned by the context (each call allocates new copies,
 * freed by sph_free).  Errors: SPH_ERR_ARG (star count differs from the
 * context's, nr < 2, NULL table, non-finite or negative values). */
sph_status sph_set_external(sph_ctx *ctx, const sph_external *ext);

/* Modification step after a relaxation (Sec. II.A): replace the context's
 * equation of state by eos (the star's, per star), evaluate the density of
 * the current state (a right-hand side without the external field, which
 * this call switches off) and set u = K rho^(Gamma-1)/(Gamma-1) for every
 * particle.  Positions, velocities and h are kept.  Errors: SPH_ERR_ARG
 * (star count, K <= 0, Gamma <= 1), SPH_ERR_CUDA. */
sph_status sph_relax_finish(sph_ctx *ctx, const sph_eos *eos);

/* Release the context and its device memory (the caller's buffers stay).
 * Waits for the context's stream first.  NULL is ignored. */
void sph_free(sph_ctx *ctx);

/* Neighbour lists without a context and without any device allocation, for
 * callers that cannot call cudaMalloc: plug-ins whose host application owns
 * all device memory through its own pool, processes whose memory budget
 * forbids further allocations, and time-critical loops where an allocator
 * call (which may synchronise the device) is not allowed.  The paper has no
 * counterpart; this is a library service.  Same lists and CSR layout as
 * sph_neighbors for one star: x, y, z, h are device arrays of n particles
 * (caller order), offsets a device int64[n+1], idx a device int32[cap];
 * cuda_stream a cudaStream_t (NULL: legacy default stream).  Scratch is one
 * fixed device array of about 11.9 MB inside the library, present on every
 * GPU that loads it until the process exits.  Limits: n <= 16384 (larger n
 * returns SPH_ERR_ARG), at most 128 neighbours per particle and 256
 * candidate leaves (groups of 8 sorted particles) per leaf
 * (SPH_ERR_CAPACITY); more than cap entries in all returns SPH_ERR_CAPACITY
 * with offsets written and idx not.  Under lazy module loading (the CUDA
 * default) the first call on a device loads the library's device code and
 * the array, which takes device memory once: make one call with n >= 1
 * before another allocator takes the whole device.  Every call looks up the
 * array's address on the current device, shares the array with other calls
 * and resets what must start at zero; calls that overlap on the GPU race.
 * Synchronous. */
sph_status sph_neighbors_noalloc(int64_t n, const double *x, const double *y, const double *z,
                                 const double *h, int64_t *offsets, int32_t *idx, int64_t cap,
                                 void *cuda_stream);

/* Measured FP32 and FP64 fused multiply-add rates of the current device, the
 * peaks against which the pair kernels' throughput is reported (library
 * service, no counterpart in the paper).  out (host double[4]): 0 FP32 and
 * 1 FP64 TFLOP/s (eight independent FMA chains per thread over 8 blocks of
 * 256 threads per SM, timed with CUDA events after a warm-up), 2 the number
 * of SMs, 3 zero.  Allocates and frees a small device buffer.  Synchronous.
 * Errors: SPH_ERR_ARG (NULL out), SPH_ERR_NODEVICE, SPH_ERR_CUDA. */
sph_status sph_peak_rates(double out[4]);

/* Message for the last failing call on this thread ("" if none). */
const char *sph_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SPH_H */
