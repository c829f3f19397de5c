// C ABI of libsph (declared in include/sph.h): context set-up, the
// right-hand side and step sequences, CUDA-graph capture of steps,
// event timing, totals, neighbour export and checkpoints.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "sph_internal.cuh"

using namespace sph;

namespace {

thread_local char g_err[512] = "";

sph_status fail(sph_status st, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

// NVTX range around a host entry point (a profiler shows the library's calls
// on its timeline; without a tool attached the calls return at once).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

#define CUDA_TRY(call)                                                                   \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail(e_ == cudaErrorMemoryAllocation ? SPH_ERR_OOM : SPH_ERR_CUDA,     \
                        "%s: %s", #call, cudaGetErrorString(e_));                        \
    } while (0)

// Timing marks of one step (or one right-hand side): step start, sort+tree
// start, neighbour-list start, density start, force start, force end, step end.
enum { EV_STEP, EV_BUILD, EV_LISTS, EV_DENSITY, EV_FORCE, EV_FORCE_END, EV_STEP_END, EV_N };

struct TimingSlot {
    cudaEvent_t ev[EV_N];
};

}  // namespace

struct sph_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    // second stream of the mixed force pass (solid-block kernel) and the
    // events that fork it from and join it to stream
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int64_t n = 0;
    int nstars = 1;
    sph_precision prec = SPH_MIXED;
    sph_options opt{};
    sph_particles P{};
    bool any_solid = false;
    // owned device memory
    std::vector<void *> allocs;
    double *d_K = nullptr, *d_Gamma = nullptr;
    int npieces = 0;                                   // piecewise EoS (0: one polytrope)
    double *d_rho_b = nullptr, *d_Kp = nullptr, *d_Gp = nullptr, *d_ap = nullptr;
    float *f_K = nullptr, *f_Gamma = nullptr;          // FP32 copies (mixed precision)
    float *f_rho_b = nullptr, *f_Kp = nullptr, *f_Gp = nullptr, *f_ap = nullptr;
    std::vector<float> h_fstar;                        // per-star FP32 constants (host copy)
    float *d_fstar = nullptr;
    int multi = 0;                                     // several stars in one index space
    DevMaterial mat{};
    DevMetric met{};
    Scratch s{};
    SortPlan plan{};
    TreeLevels tl{};
    int nleaves = 0;
    int cap = 128;
    int lanes = 8;          // threads per particle of the pair kernels
    int screen_lanes = 4;   // threads per particle of the exact screening
    int tuned = 0;          // 0 fixed shape, 1 timed by sph_init, 2 from the process cache
    // autotuner times (ns per launch): screening 4 / 8 lanes, pair kernels
    // 4 / 8 lanes, screening + pair kernels in series, persistent launch
    // 4 / 8 lanes, screening + pair kernels in series, persistent launch,
    // candidate build with search leaves of 1, 2, 4 tree leaves
    int64_t tune_ns[9] = {};
    int tune_persist = 0;   // the autotuner chose the persistent launch
    int group = 1;          // tree leaves per tile-search walk
    PersistPlan pplan{};    // persistent right-hand side (grid 0: off)
    DevRates r{};
    double *vp = nullptr, *Sp = nullptr;
    double *tot_partial = nullptr, *tot_out = nullptr;
    int64_t *star_off = nullptr;                       // per-star caller indices (CSR)
    int32_t *star_idx = nullptr;
    double *star_tot = nullptr;                        // [nstars][16]
    double *zeros = nullptr;  // stand-in for absent per-particle material arrays
    int have_rates = 0;
    int64_t steps = 0;
    int launches_per_step = 0;
    int64_t launches_total = 0;        // kernel launches issued by sph_step
    // graphs of a step: [0] keeps the last sort's order, [1] sorts again
    cudaGraph_t graph[2] = {};         // kept alive: their nodes name the timing events
    cudaGraphExec_t gexec[2] = {};
    double gdt[2] = {};
    int gtiming[2] = {};
    int glaunches[2] = {};
    cudaGraphNode_t gev_nodes[2][EV_N] = {};
    // timing
    int timing = 0;
    std::vector<TimingSlot> slots;
    int slot_used = 0;
    int slot_kind_step = 0;

    template <typename T>
    sph_status alloc(T **p, size_t count)
    {
        *p = nullptr;
        if (count == 0) count = 1;
        cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
        if (e != cudaSuccess) {
            *p = nullptr;
            return fail(SPH_ERR_OOM, "cudaMalloc of %zu bytes failed: %s", count * sizeof(T),
                        cudaGetErrorString(e));
        }
        allocs.push_back((void *)*p);
        return SPH_OK;
    }
};

namespace {

#define STATUS_TRY(call)                 \
    do {                                 \
        sph_status s_ = (call);          \
        if (s_ != SPH_OK) return s_;     \
    } while (0)

DevState state_of(const sph_ctx *c, const double *vx, const double *vy, const double *vz,
                  const double *S)
{
    DevState st;
    st.n = c->n;
    st.x = c->P.x;
    st.y = c->P.y;
    st.z = c->P.z;
    st.vx = vx;
    st.vy = vy;
    st.vz = vz;
    st.S = S;
    st.h = c->P.h;
    st.m = c->P.m;
    st.mu = c->P.mu ? c->P.mu : c->zeros;
    st.type = c->P.type;
    st.star = c->P.star;
    return st;
}

StepState step_state_of(sph_ctx *c)
{
    StepState s;
    s.n = c->n;
    s.x = c->P.x;
    s.y = c->P.y;
    s.z = c->P.z;
    s.vx = c->P.vx;
    s.vy = c->P.vy;
    s.vz = c->P.vz;
    s.u = c->P.u;
    s.h = c->P.h;
    s.S = c->P.S;
    s.m = c->P.m;
    s.type = c->P.type;
    s.flags = c->P.flags;
    s.star = c->P.star;
    s.mu = c->P.mu ? c->P.mu : c->zeros;
    s.Y0 = c->P.Y0 ? c->P.Y0 : c->zeros;
    s.eps_break = c->P.eps_break ? c->P.eps_break : c->zeros;
    s.vp = c->vp;
    s.Sp = c->Sp;
    return s;
}

DevEos eos_of(const sph_ctx *c)
{
    DevEos e;
    e.K = c->d_K;
    e.Gamma = c->d_Gamma;
    e.npieces = c->npieces;
    e.rho_b = c->d_rho_b;
    e.Kp = c->d_Kp;
    e.Gp = c->d_Gp;
    e.ap = c->d_ap;
    e.Kf = c->f_K;
    e.Gf = c->f_Gamma;
    e.rho_bf = c->f_rho_b;
    e.Kpf = c->f_Kp;
    e.Gpf = c->f_Gp;
    e.apf = c->f_ap;
    return e;
}

constexpr int kMaxPieces = 8;

// Checks an EoS for nstars stars (one polytrope or a piecewise one).
sph_status check_eos(const sph_eos *eos, int nstars_expected)
{
    if (!eos || eos->nstars < 1 || eos->nstars > 65535 || !eos->K || !eos->Gamma)
        return fail(SPH_ERR_ARG, "eos must give 1..65535 stars with K and Gamma");
    if (nstars_expected > 0 && eos->nstars != nstars_expected)
        return fail(SPH_ERR_ARG, "eos must give K and Gamma for each of the %d stars",
                    nstars_expected);
    for (int s = 0; s < eos->nstars; ++s) {
        if (!(eos->Gamma[s] > 1.0) || !(eos->K[s] > 0.0) || !std::isfinite(eos->Gamma[s]) ||
            !std::isfinite(eos->K[s]))
            return fail(SPH_ERR_ARG, "star %d: need K > 0 and Gamma > 1", s);
    }
    const int np = eos->npieces;
    if (np < 0 || np > kMaxPieces) return fail(SPH_ERR_ARG, "npieces must be 0..%d", kMaxPieces);
    if (np > 1) {
        if (!eos->rho_bound || !eos->Gamma_above)
            return fail(SPH_ERR_ARG, "piecewise eos needs rho_bound and Gamma_above");
        for (int s = 0; s < eos->nstars; ++s)
            for (int k = 0; k + 1 < np; ++k) {
                const double rb = eos->rho_bound[(size_t)s * (np - 1) + k];
                const double ga = eos->Gamma_above[(size_t)s * (np - 1) + k];
                if (!(rb > 0.0) || !std::isfinite(rb) || !(ga > 1.0) || !std::isfinite(ga))
                    return fail(SPH_ERR_ARG, "star %d piece %d: need rho_bound > 0, Gamma > 1", s,
                                k + 1);
                if (k > 0 && !(rb > eos->rho_bound[(size_t)s * (np - 1) + k - 1]))
                    return fail(SPH_ERR_ARG, "star %d: rho_bound must increase", s);
            }
    }
    return SPH_OK;
}

// Copies a checked EoS into the context; for a piecewise one, K and the
// energy constant of each piece follow from continuity of P and u at the
// dividing densities.
sph_status upload_eos(sph_ctx *c, const sph_eos *eos)
{
    const int ns = eos->nstars;
    if (!c->d_K) {
        STATUS_TRY(c->alloc(&c->d_K, ns));
        STATUS_TRY(c->alloc(&c->d_Gamma, ns));
        STATUS_TRY(c->alloc(&c->f_K, ns));
        STATUS_TRY(c->alloc(&c->f_Gamma, ns));
    }
    CUDA_TRY(cudaMemcpy(c->d_K, eos->K, ns * sizeof(double), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(c->d_Gamma, eos->Gamma, ns * sizeof(double), cudaMemcpyHostToDevice));
    {
        std::vector<float> kf(ns), gf(ns);
        for (int k = 0; k < ns; ++k) {
            kf[k] = (float)eos->K[k];
            gf[k] = (float)eos->Gamma[k];
        }
        CUDA_TRY(cudaMemcpy(c->f_K, kf.data(), ns * sizeof(float), cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(c->f_Gamma, gf.data(), ns * sizeof(float), cudaMemcpyHostToDevice));
    }
    c->npieces = eos->npieces > 1 ? eos->npieces : 0;
    if (c->npieces > 1) {
        const int np = c->npieces;
        std::vector<double> rb((size_t)ns * (np - 1)), Kp((size_t)ns * np), Gp(Kp.size()),
            ap(Kp.size());
        for (int s = 0; s < ns; ++s) {
            double K = eos->K[s], G = eos->Gamma[s], a = 0.0;
            Kp[(size_t)s * np] = K;
            Gp[(size_t)s * np] = G;
            ap[(size_t)s * np] = 0.0;
            for (int k = 0; k + 1 < np; ++k) {
                const double r = eos->rho_bound[(size_t)s * (np - 1) + k];
                const double Gn = eos->Gamma_above[(size_t)s * (np - 1) + k];
                const double Kn = K * std::pow(r, G - Gn);
                a += K * std::pow(r, G - 1.0) / (G - 1.0) - Kn * std::pow(r, Gn - 1.0) / (Gn - 1.0);
                K = Kn;
                G = Gn;
                rb[(size_t)s * (np - 1) + k] = r;
                Kp[(size_t)s * np + k + 1] = K;
                Gp[(size_t)s * np + k + 1] = G;
                ap[(size_t)s * np + k + 1] = a;
            }
        }
        STATUS_TRY(c->alloc(&c->d_rho_b, rb.size()));
        STATUS_TRY(c->alloc(&c->d_Kp, Kp.size()));
        STATUS_TRY(c->alloc(&c->d_Gp, Gp.size()));
        STATUS_TRY(c->alloc(&c->d_ap, ap.size()));
        CUDA_TRY(cudaMemcpy(c->d_rho_b, rb.data(), rb.size() * sizeof(double), cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(c->d_Kp, Kp.data(), Kp.size() * sizeof(double), cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(c->d_Gp, Gp.data(), Gp.size() * sizeof(double), cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(c->d_ap, ap.data(), ap.size() * sizeof(double), cudaMemcpyHostToDevice));
        auto to_f = [&](const std::vector<double> &v, float **dst) -> sph_status {
            std::vector<float> f(v.size());
            for (size_t k = 0; k < v.size(); ++k) f[k] = (float)v[k];
            STATUS_TRY(c->alloc(dst, f.size()));
            CUDA_TRY(cudaMemcpy(*dst, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice));
            return SPH_OK;
        };
        STATUS_TRY(to_f(rb, &c->f_rho_b));
        STATUS_TRY(to_f(Kp, &c->f_Kp));
        STATUS_TRY(to_f(Gp, &c->f_Gp));
        STATUS_TRY(to_f(ap, &c->f_ap));
    }
    return SPH_OK;
}

DevRates rates_of(const sph_rates *o)
{
    DevRates r;
    r.ax = o->ax;
    r.ay = o->ay;
    r.az = o->az;
    r.dudt = o->dudt;
    r.drhodt = o->drhodt;
    r.rho = o->rho;
    r.P = o->P;
    r.D = o->D;
    r.cs = o->cs;
    r.deps = o->deps;
    r.dR = o->dR;
    r.dS = o->dS;
    r.ncount = o->ncount;
    return r;
}

sph_status ensure_slot(sph_ctx *c)
{
    if (c->slot_used < (int)c->slots.size()) return SPH_OK;
    size_t old = c->slots.size();
    c->slots.resize(old + 256);
    for (size_t k = old; k < c->slots.size(); ++k)
        for (int e = 0; e < EV_N; ++e) CUDA_TRY(cudaEventCreate(&c->slots[k].ev[e]));
    return SPH_OK;
}

// Events of the current timing slot (or null when timing is off).
cudaEvent_t slot_ev(sph_ctx *c, int e)
{
    if (!c->timing) return nullptr;
    return c->slots[c->slot_used].ev[e];
}

void rec(sph_ctx *c, cudaEvent_t ev, bool capturing)
{
    if (!ev) return;
    if (capturing) cudaEventRecordWithFlags(ev, c->stream, cudaEventRecordExternal);
    else cudaEventRecord(ev, c->stream);
}

// The right-hand side on the given velocity and stress, into `out`.
void enqueue_rhs(sph_ctx *c, const DevState &st, const DevRates &out, bool capturing,
                 int *nlaunch, bool resort = true)
{
    if (c->n == 0) return;
    const bool fp64 = c->prec == SPH_FP64;
    rec(c, slot_ev(c, EV_BUILD), capturing);
    launch_build(st, c->s, c->plan, c->tl, c->nleaves, fp64, c->stream, nlaunch, resort);
    rec(c, slot_ev(c, EV_LISTS), capturing);
    if (c->pplan.grid > 0 && !fp64) {
        // candidate lists (when stale), then screening, density, equation of
        // state and force in one persistent launch
        launch_tiles_build(st, c->s, c->tl, c->nleaves, c->multi, c->cap, c->stream, c->group);
        rec(c, slot_ev(c, EV_DENSITY), capturing);
        rec(c, slot_ev(c, EV_FORCE), capturing);
        launch_persistent(st, c->s, eos_of(c), c->mat, c->met, out, c->cap, c->screen_lanes,
                          c->lanes, c->pplan, c->stream);
        rec(c, slot_ev(c, EV_FORCE_END), capturing);
        if (nlaunch) *nlaunch += 2;
        return;
    }
    // candidate lists (when stale) and exact lists; in mixed precision the
    // density and equation of state too
    launch_tiles(st, c->s, c->tl, c->nleaves, c->multi, c->cap, fp64 ? 0 : 1, eos_of(c), c->met,
                 out, c->stream, nlaunch, c->screen_lanes, c->group);
    rec(c, slot_ev(c, EV_DENSITY), capturing);
    if (fp64) launch_density_fp64(st, c->s, eos_of(c), c->met, out, c->cap, c->lanes, c->stream);
    rec(c, slot_ev(c, EV_FORCE), capturing);
    launch_force(st, c->s, eos_of(c), c->mat, c->met, out, c->cap, c->lanes, fp64, c->stream,
                 c->side, c->ev_fork, c->ev_join);
    rec(c, slot_ev(c, EV_FORCE_END), capturing);
    // density and force (FP64) or the fluid-block and solid-block force
    // kernels (mixed precision)
    if (nlaunch) *nlaunch += 2;
}

void enqueue_step(sph_ctx *c, double dt, bool capturing, int *nlaunch, bool resort)
{
    StepState ss = step_state_of(c);
    rec(c, slot_ev(c, EV_STEP), capturing);
    launch_kick_drift(ss, c->r, dt, c->stream);
    DevState st = state_of(c, c->vp, c->vp + c->n, c->vp + 2 * c->n, c->Sp);
    enqueue_rhs(c, st, c->r, capturing, nlaunch, resort);
    launch_kick_return(ss, c->r, eos_of(c), c->mat, dt, c->opt.h_nmin, c->opt.h_nmax, c->stream);
    rec(c, slot_ev(c, EV_STEP_END), capturing);
    if (nlaunch) *nlaunch += 2;
}

// Autotuner over the launch shape: the search leaf of the candidate build
// (1, 2 or 4 tree leaves, 8 to 32 particles, per tile-search walk), threads
// per particle of the exact screening (4 or 8) and of the pair kernels (4 or
// 8), and in mixed precision whether the screening and force pass run as
// separate launches or as one persistent launch.  After one right-hand side
// on the bound state, sph_init times each variant of each stage (three
// launches after a warm-up one, CUDA events on the context's stream) and
// keeps the faster; the stages are separate kernels, so they are chosen
// independently, then the persistent launch of the chosen lanes is timed
// against the two stages in series.  A search leaf whose walk front fills
// more than half of its capacity on the bound state is not taken (the
// front grows as particles move).  The device counters are restored afterwards, so the tuning
// launches are not counted.  The choice is cached for the process under the
// configuration (device, n, stars, precision, capacity, metric, solids, what
// is tuned and the fixed lanes), so later contexts of the same configuration
// take the same shape without timing again.  Lane counts change the order of
// the density and pair sums (a tuned context agrees with a fixed one to
// rounding); the persistent launch does not change any result.
using TuneKey = std::tuple<int, int64_t, int, int, int, int, int, int, int, int>;
struct TuneVal {
    int screen_lanes, lanes, persist, group;
    int64_t ns[9];
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune_cache;

sph_status time_stage(sph_ctx *c, cudaEvent_t e0, cudaEvent_t e1, int64_t *ns,
                      const std::function<void()> &launch)
{
    launch();
    CUDA_TRY(cudaEventRecord(e0, c->stream));
    for (int rep = 0; rep < 3; ++rep) launch();
    CUDA_TRY(cudaEventRecord(e1, c->stream));
    CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    *ns = (int64_t)(ms * 1e6f / 3.f);
    return SPH_OK;
}

sph_status autotune_shape(sph_ctx *c, bool lanes, bool persist)
{
    NvtxRange nvtx_("sph_autotune");
    const bool fp64 = c->prec == SPH_FP64;
    persist = persist && !fp64;
    const int code = (lanes ? 1 : 0) | (persist ? 2 : 0) |
                     (lanes ? 0 : 4 * (c->screen_lanes == 8 ? 1 : 0) + 8 * (c->lanes == 8 ? 1 : 0));
    const TuneKey key{c->device, c->n, c->nstars, (int)c->prec, c->cap, c->met.kind,
                      c->any_solid ? 1 : 0, c->multi, code, 0};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            c->screen_lanes = it->second.screen_lanes;
            c->lanes = it->second.lanes;
            c->tune_persist = it->second.persist;
            if (lanes) c->group = it->second.group;
            for (int k = 0; k < 9; ++k) c->tune_ns[k] = it->second.ns[k];
            c->tuned = 2;
            return SPH_OK;
        }
    }
    DevScalars saved{};
    CUDA_TRY(cudaMemcpy(&saved, c->s.sc, sizeof(DevScalars), cudaMemcpyDeviceToHost));
    DevState st = state_of(c, c->P.vx, c->P.vy, c->P.vz, c->P.S);
    const int timing = c->timing;
    c->timing = 0;
    enqueue_rhs(c, st, c->r, false, nullptr);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    sph_status rc = SPH_OK;
    auto screen = [&](int sl) {
        launch_screen(st, c->s, c->cap, fp64 ? 0 : 1, eos_of(c), c->met, c->r, c->stream, sl);
    };
    auto force = [&](int fl) {
        if (fp64) launch_density_fp64(st, c->s, eos_of(c), c->met, c->r, c->cap, fl, c->stream);
        launch_force(st, c->s, eos_of(c), c->mat, c->met, c->r, c->cap, fl, fp64, c->stream,
                     c->side, c->ev_fork, c->ev_join);
    };
    const int shapes[2] = {4, 8};
    if (lanes) {
        for (int k = 0; k < 2 && rc == SPH_OK; ++k)
            rc = time_stage(c, e0, e1, &c->tune_ns[k], [&] { screen(shapes[k]); });
        for (int k = 0; k < 2 && rc == SPH_OK; ++k)
            rc = time_stage(c, e0, e1, &c->tune_ns[2 + k], [&] { force(shapes[k]); });
        if (rc == SPH_OK) {
            c->screen_lanes = c->tune_ns[1] < c->tune_ns[0] ? 8 : 4;
            c->lanes = c->tune_ns[3] < c->tune_ns[2] ? 8 : 4;
        }
        // candidate builds (the rebuild flag set before each launch); above
        // the default list capacity the walk has one shape only
        const int groups[3] = {1, 2, 4};
        const int caps[3] = {kCandCap, 2 * kCandCap, 2 * kCandCap};
        static const int one = 1;
        int best = 1;
        int64_t best_ns = 0;
        for (int k = 0; k < (c->cap > kRowCapDefault ? 1 : 3) && rc == SPH_OK; ++k) {
            const int gk = groups[k];
            rc = time_stage(c, e0, e1, &c->tune_ns[6 + k], [&] {
                cudaMemcpyAsync(&c->s.sc->rebuild, &one, sizeof(int), cudaMemcpyHostToDevice,
                                c->stream);
                launch_tiles_build(st, c->s, c->tl, c->nleaves, c->multi, c->cap, c->stream, gk);
            });
            if (rc != SPH_OK) break;
            DevScalars now{};
            if (cudaMemcpy(&now, c->s.sc, sizeof(DevScalars), cudaMemcpyDeviceToHost) != cudaSuccess) {
                rc = fail(SPH_ERR_CUDA, "autotune: reading the counters failed");
                break;
            }
            const bool fits = !(now.err & ERR_CAPACITY) && 2 * now.max_cand <= caps[k];
            if (fits && (k == 0 || c->tune_ns[6 + k] < best_ns)) {
                best = gk;
                best_ns = c->tune_ns[6 + k];
            }
            // the next variant starts from clean counters
            now.err &= ~ERR_CAPACITY;
            now.max_cand = 0;
            if (cudaMemcpy(c->s.sc, &now, sizeof(DevScalars), cudaMemcpyHostToDevice) != cudaSuccess) {
                rc = fail(SPH_ERR_CUDA, "autotune: resetting the counters failed");
                break;
            }
        }
        if (rc == SPH_OK) c->group = best;
    }
    if (persist && rc == SPH_OK) {
        const PersistPlan pp = plan_persistent(c->n, c->screen_lanes, c->lanes);
        rc = time_stage(c, e0, e1, &c->tune_ns[4], [&] {
            screen(c->screen_lanes);
            force(c->lanes);
        });
        // the queue counters are reset per right-hand side by the bounding-box
        // kernel; here before every timed launch
        if (rc == SPH_OK)
            rc = time_stage(c, e0, e1, &c->tune_ns[5], [&] {
                cudaMemsetAsync(&c->s.sc->pq_head, 0, 2 * sizeof(unsigned int), c->stream);
                launch_persistent(st, c->s, eos_of(c), c->mat, c->met, c->r, c->cap,
                                  c->screen_lanes, c->lanes, pp, c->stream);
            });
        if (rc == SPH_OK) c->tune_persist = c->tune_ns[5] < c->tune_ns[4] ? 1 : 0;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->timing = timing;
    if (rc != SPH_OK) return rc;
    // the counters go back to their state before tuning
    CUDA_TRY(cudaMemcpy(c->s.sc, &saved, sizeof(DevScalars), cudaMemcpyHostToDevice));
    c->tuned = 1;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    TuneVal v{c->screen_lanes, c->lanes, c->tune_persist, c->group, {}};
    for (int k = 0; k < 9; ++k) v.ns[k] = c->tune_ns[k];
    g_tune_cache.emplace(key, v);
    return SPH_OK;
}

// Candidate leaves one tile-search walk holds (sph_tiles.cu TileShape).
int walk_capacity(const sph_ctx *c)
{
    if (c->cap > kRowCapDefault) return 4 * kCandCap;
    return c->group > 1 ? 2 * kCandCap : kCandCap;
}

void drop_graph(sph_ctx *c, int k)
{
    if (c->gexec[k]) cudaGraphExecDestroy(c->gexec[k]);
    if (c->graph[k]) cudaGraphDestroy(c->graph[k]);
    c->gexec[k] = nullptr;
    c->graph[k] = nullptr;
}

void drop_graph(sph_ctx *c)
{
    drop_graph(c, 0);
    drop_graph(c, 1);
}

// Whether step number k (counted from the context's creation) sorts the
// particles along the curve again.
bool resort_at(const sph_ctx *c, int64_t k)
{
    return c->opt.sort_every <= 1 || k % c->opt.sort_every == 0;
}

sph_status capture_step(sph_ctx *c, double dt, bool resort)
{
    NvtxRange nvtx_("sph_capture_step");
    const int g = resort ? 1 : 0;
    drop_graph(c, g);
    cudaGraph_t graph = nullptr;
    // Timing slot 0's events mark the nodes; replays swap in the slot's events.
    int saved_used = c->slot_used;
    if (c->timing) {
        STATUS_TRY(ensure_slot(c));
    }
    CUDA_TRY(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    int nl = 0;
    enqueue_step(c, dt, true, &nl, resort);
    cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
    if (e != cudaSuccess) return fail(SPH_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&c->gexec[g], graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        c->gexec[g] = nullptr;
        return fail(SPH_ERR_CUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
    }
    for (int k = 0; k < EV_N; ++k) c->gev_nodes[g][k] = nullptr;
    if (c->timing) {
        size_t nn = 0;
        cudaGraphGetNodes(graph, nullptr, &nn);
        std::vector<cudaGraphNode_t> nodes(nn);
        cudaGraphGetNodes(graph, nodes.data(), &nn);
        for (auto nd : nodes) {
            cudaGraphNodeType ty;
            cudaGraphNodeGetType(nd, &ty);
            if (ty != cudaGraphNodeTypeEventRecord) continue;
            cudaEvent_t ev;
            cudaGraphEventRecordNodeGetEvent(nd, &ev);
            for (int k = 0; k < EV_N; ++k)
                if (ev == c->slots[saved_used].ev[k]) c->gev_nodes[g][k] = nd;
        }
    }
    c->graph[g] = graph;
    c->gdt[g] = dt;
    c->gtiming[g] = c->timing;
    c->glaunches[g] = nl;
    return SPH_OK;
}

// A point as hi + lo floats per coordinate: hi = fl32(x), lo = fl32(x - hi).
void split_float(const double *x, float *hi, float *lo)
{
    for (int k = 0; k < 3; ++k) {
        hi[k] = (float)x[k];
        lo[k] = (float)(x[k] - (double)hi[k]);
    }
}

int bits_for(int64_t n)
{
    int lg = 1;
    while ((1ll << lg) < n) ++lg;
    int b = (lg + 2) / 3 + 2;
    return b < 5 ? 5 : (b > 10 ? 10 : b);
}

sph_status validate(const sph_particles *p, const sph_eos *eos, const sph_material *mat,
                    const sph_metric *g, sph_precision prec, const sph_options *opt)
{
    if (!p) return fail(SPH_ERR_ARG, "particles is NULL");
    if (p->n < 0 || p->n > 0x7fffff00ll) return fail(SPH_ERR_ARG, "n = %lld out of range", (long long)p->n);
    if (p->n > 0) {
        if (!p->x || !p->y || !p->z || !p->vx || !p->vy || !p->vz || !p->u || !p->h || !p->m ||
            !p->S || !p->type || !p->flags)
            return fail(SPH_ERR_ARG, "a required particle array is NULL");
    }
    STATUS_TRY(check_eos(eos, 0));
    if (!mat) return fail(SPH_ERR_ARG, "material is NULL");
    if (mat->jaumann < 0 || mat->jaumann > 1 || mat->yield_mode < 0 || mat->yield_mode > 1 ||
        mat->break_stress < 0 || mat->break_stress > 1)
        return fail(SPH_ERR_ARG, "material option out of range");
    if (prec != SPH_FP64 && prec != SPH_MIXED) return fail(SPH_ERR_ARG, "unknown precision");
    if (g && g->kind != 0) {
        if (g->kind != 1) return fail(SPH_ERR_ARG, "metric kind must be 0 or 1");
        if (g->nstars != eos->nstars) return fail(SPH_ERR_ARG, "metric and eos star counts differ");
        if (g->nr < 2) return fail(SPH_ERR_ARG, "metric needs nr >= 2");
        if (!g->r_max || !g->alpha || !g->dalpha || !g->psi4 || !g->dpsi4 || !g->M || !g->center)
            return fail(SPH_ERR_ARG, "a metric table is NULL");
        if (g->pressure_form < 0 || g->pressure_form > 1)
            return fail(SPH_ERR_ARG, "metric pressure_form must be 0 or 1");
        for (int s = 0; s < g->nstars; ++s)
            if (!(g->r_max[s] > 0.0)) return fail(SPH_ERR_ARG, "metric r_max must be > 0");
    }
    if (opt) {
        if (opt->max_neighbors < 0 || opt->max_neighbors > kRowCap)
            return fail(SPH_ERR_ARG, "max_neighbors must be 0..%d", kRowCap);
        if (opt->lanes_per_particle != 0 && opt->lanes_per_particle != 4 &&
            opt->lanes_per_particle != 8 && opt->lanes_per_particle != -1)
            return fail(SPH_ERR_ARG, "lanes_per_particle must be -1, 0, 4 or 8");
        if (opt->screen_lanes != 0 && opt->screen_lanes != 4 && opt->screen_lanes != 8)
            return fail(SPH_ERR_ARG, "screen_lanes must be 0, 4 or 8");
        if (opt->persistent < -1 || opt->persistent > 1)
            return fail(SPH_ERR_ARG, "persistent must be -1, 0 or 1");
        if (opt->search_leaves != 0 && opt->search_leaves != 1 && opt->search_leaves != 2 &&
            opt->search_leaves != 4)
            return fail(SPH_ERR_ARG, "search_leaves must be 0, 1, 2 or 4");
        if (opt->h_nmax < 0 || opt->h_nmin < 0 || (opt->h_nmax > 0 && opt->h_nmin > opt->h_nmax))
            return fail(SPH_ERR_ARG, "h_nmin/h_nmax band invalid");
        if (opt->sort_every < 0) return fail(SPH_ERR_ARG, "sort_every must be >= 0");
        if (!std::isfinite(opt->skin) || opt->skin > 1.0)
            return fail(SPH_ERR_ARG, "skin must be finite and <= 1");
    }
    return SPH_OK;
}

sph_status init_impl(sph_ctx *c, const sph_particles *p, const sph_eos *eos,
                     const sph_material *mat, const sph_metric *g, sph_precision prec,
                     const sph_options *opt, void *stream)
{
    c->P = *p;
    c->n = p->n;
    c->nstars = eos->nstars;
    c->prec = prec;
    if (opt) c->opt = *opt;
    else {
        c->opt = sph_options{};
        c->opt.use_graph = 1;
    }
    c->cap = c->opt.max_neighbors > 0 ? c->opt.max_neighbors : kRowCapDefault;
    c->lanes = c->opt.lanes_per_particle > 0 ? c->opt.lanes_per_particle : 8;
    c->screen_lanes = c->opt.screen_lanes > 0 ? c->opt.screen_lanes : 4;
    c->group = c->opt.search_leaves > 0 ? c->opt.search_leaves : 1;
    c->stream = (cudaStream_t)stream;
    if (prec == SPH_MIXED) {
        CUDA_TRY(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
        CUDA_TRY(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
        CUDA_TRY(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
    }
    CUDA_TRY(cudaGetDevice(&c->device));
    const int64_t n = c->n;
    // Host copies of type and star: star layout, solid check.
    std::vector<int32_t> star(n > 0 ? n : 1, 0);
    std::vector<uint8_t> type(n > 0 ? n : 1, 0);
    if (n > 0) {
        if (p->star) CUDA_TRY(cudaMemcpy(star.data(), p->star, n * sizeof(int32_t), cudaMemcpyDeviceToHost));
        CUDA_TRY(cudaMemcpy(type.data(), p->type, n * sizeof(uint8_t), cudaMemcpyDeviceToHost));
    }
    std::vector<int64_t> per(c->nstars, 0);
    for (int64_t i = 0; i < n; ++i) {
        if (star[i] < 0 || star[i] >= c->nstars)
            return fail(SPH_ERR_ARG, "particle %lld has star %d outside [0, %d)", (long long)i,
                        star[i], c->nstars);
        if (type[i] > 1) return fail(SPH_ERR_ARG, "particle %lld has type %d", (long long)i, type[i]);
        per[star[i]]++;
        c->any_solid |= type[i] == 1;
    }
    if (c->any_solid && (!p->mu || !p->Y0 || !p->eps_break))
        return fail(SPH_ERR_ARG, "solid particles need mu, Y0 and eps_break arrays");
    // Leaves: 8 consecutive sorted particles of one star (stars are sorted by id).
    std::vector<int32_t> leaf_start(1, 0), leaf_star, leaf_of(n > 0 ? n : 1, 0);
    int64_t pos = 0;
    for (int s = 0; s < c->nstars; ++s) {
        for (int64_t k = 0; k < per[s]; k += kLeaf) {
            int64_t e = pos + (per[s] - k < kLeaf ? per[s] - k : kLeaf);
            for (int64_t i = pos; i < e; ++i) leaf_of[i] = (int32_t)leaf_star.size();
            leaf_star.push_back(s);
            leaf_start.push_back((int32_t)e);
            pos = e;
        }
    }
    c->nleaves = (int)leaf_star.size();
    // Tree levels.
    int64_t total_nodes = 0;
    if (!make_tree_levels(c->nleaves, c->tl, &total_nodes) || c->tl.nlevels > 10)
        return fail(SPH_ERR_ARG, "too many particles for the tree (more than 10 levels)");
    // Sort plan.
    int sb = 0;
    while ((1 << sb) < c->nstars) ++sb;
    c->plan.key_bits_axis = bits_for(n);
    c->plan.star_bits = sb;
    c->plan.nstars = c->nstars;
    c->multi = sb > 0 ? 1 : 0;
    int kb = 3 * c->plan.key_bits_axis + sb;
    c->plan.passes = (kb + 7) / 8;
    int64_t per_tile = 256ll * 304;
    int ipt = (int)((n + per_tile - 1) / per_tile);
    c->plan.ipt = ipt < 1 ? 1 : (ipt > 16 ? 16 : ipt);
    c->plan.nblocks = (int)((n + 256ll * c->plan.ipt - 1) / (256ll * c->plan.ipt));
    if (c->plan.nblocks < 1) c->plan.nblocks = 1;
    // Device memory.
    const int64_t nn = n > 0 ? n : 1;
    Scratch &s = c->s;
    STATUS_TRY(c->alloc(&s.perm, nn));
    if (n > 0) {
        // the identity until the first curve sort, so that a checkpoint taken
        // before any step restores
        std::vector<int32_t> ident((size_t)n);
        for (int64_t i = 0; i < n; ++i) ident[(size_t)i] = (int32_t)i;
        CUDA_TRY(cudaMemcpy(s.perm, ident.data(), (size_t)n * sizeof(int32_t),
                            cudaMemcpyHostToDevice));
    }
    STATUS_TRY(c->alloc(&s.keys[0], nn));
    STATUS_TRY(c->alloc(&s.keys[1], nn));
    STATUS_TRY(c->alloc(&s.vals[0], nn));
    STATUS_TRY(c->alloc(&s.vals[1], nn));
    STATUS_TRY(c->alloc(&s.hist, (size_t)c->plan.passes * 256 * c->plan.nblocks * 2));
    STATUS_TRY(c->alloc(&s.radix_tot, (size_t)8 * 256));
    STATUS_TRY(c->alloc(&s.xs, nn));
    STATUS_TRY(c->alloc(&s.ys, nn));
    STATUS_TRY(c->alloc(&s.zs, nn));
    STATUS_TRY(c->alloc(&s.hs, nn));
    STATUS_TRY(c->alloc(&s.tys, nn));
    STATUS_TRY(c->alloc(&s.rec, 4 * nn));
    STATUS_TRY(c->alloc(&s.pos4, nn));
    STATUS_TRY(c->alloc(&s.sd2, 2 * nn));
    STATUS_TRY(c->alloc(&s.pp, 2 * nn));
    if (prec == SPH_FP64) {
        STATUS_TRY(c->alloc(&s.rec64, 3 * nn));
        STATUS_TRY(c->alloc(&s.sd264, 8 * nn));
        STATUS_TRY(c->alloc(&s.pp64, 8 * nn));
    }
    STATUS_TRY(c->alloc(&s.vlist, (size_t)nn * c->cap));
    STATUS_TRY(c->alloc(&s.vcnt, nn));
    STATUS_TRY(c->alloc(&s.pos_build, nn));
    STATUS_TRY(c->alloc(&s.nbr, (size_t)nn * c->cap));
    STATUS_TRY(c->alloc(&s.ncnt, nn));
    STATUS_TRY(c->alloc(&s.nodes, 2 * (size_t)(total_nodes > 0 ? total_nodes : 1)));
    STATUS_TRY(c->alloc(&s.leaf_start, leaf_start.size()));
    STATUS_TRY(c->alloc(&s.leaf_star, leaf_star.size() > 0 ? leaf_star.size() : 1));
    STATUS_TRY(c->alloc(&s.leaf_of, nn));
    STATUS_TRY(c->alloc(&s.bbox_partial, 6 * kBoxBlocksMax));
    STATUS_TRY(c->alloc(&s.bbox_done, 1));
    s.star_box = nullptr;
    if (c->nstars > 1) {
        // per-star curve boxes: empty (lo at the top, hi at the bottom)
        STATUS_TRY(c->alloc(&s.star_box, (size_t)6 * c->nstars));
        CUDA_TRY(cudaMemset(s.star_box, 0xff, (size_t)3 * c->nstars * sizeof(uint32_t)));
        CUDA_TRY(cudaMemset(s.star_box + 3 * c->nstars, 0, (size_t)3 * c->nstars * sizeof(uint32_t)));
    }
    STATUS_TRY(c->alloc(&s.sc, 1));
    CUDA_TRY(cudaMemset(s.bbox_done, 0, sizeof(unsigned int)));
    CUDA_TRY(cudaMemset(s.sc, 0, sizeof(DevScalars)));
    CUDA_TRY(cudaMemset(s.ncnt, 0, nn * sizeof(int32_t)));
    CUDA_TRY(cudaMemset(s.vcnt, 0, nn * sizeof(int32_t)));
    CUDA_TRY(cudaMemset(s.pos_build, 0, nn * sizeof(float4)));
    {
        // eps of the candidate lists: option 0 the default 0.1, < 0 none
        // (built for every right-hand side)
        const double o = c->opt.skin;
        const float skin = o == 0.0 ? 0.1f : (o < 0.0 ? -1.f : (float)o);
        CUDA_TRY(cudaMemcpy(&s.sc->skin, &skin, sizeof(float), cudaMemcpyHostToDevice));
    }
    CUDA_TRY(cudaMemcpy(s.leaf_start, leaf_start.data(), leaf_start.size() * sizeof(int32_t),
                        cudaMemcpyHostToDevice));
    if (!leaf_star.empty())
        CUDA_TRY(cudaMemcpy(s.leaf_star, leaf_star.data(), leaf_star.size() * sizeof(int32_t),
                            cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(s.leaf_of, leaf_of.data(), nn * sizeof(int32_t), cudaMemcpyHostToDevice));
    // Rates carried between steps, predicted velocity and stress, totals.
    DevRates &r = c->r;
    for (double **f : {&r.ax, &r.ay, &r.az, &r.dudt, &r.drhodt, &r.rho, &r.P, &r.D, &r.cs})
        STATUS_TRY(c->alloc(f, nn));
    STATUS_TRY(c->alloc(&r.deps, 6 * nn));
    STATUS_TRY(c->alloc(&r.dR, 3 * nn));
    STATUS_TRY(c->alloc(&r.dS, 6 * nn));
    STATUS_TRY(c->alloc(&r.ncount, nn));
    CUDA_TRY(cudaMemset(r.ncount, 0, nn * sizeof(int32_t)));
    STATUS_TRY(c->alloc(&c->vp, 3 * nn));
    STATUS_TRY(c->alloc(&c->Sp, 6 * nn));
    STATUS_TRY(c->alloc(&c->tot_partial, 16 * kTotalsBlocks));
    STATUS_TRY(c->alloc(&c->tot_out, 16));
    STATUS_TRY(c->alloc(&c->zeros, nn));
    {
        // caller indices of each star, ascending (per-star totals)
        std::vector<int64_t> off(c->nstars + 1, 0);
        for (int s2 = 0; s2 < c->nstars; ++s2) off[s2 + 1] = off[s2] + per[s2];
        std::vector<int32_t> idx(nn, 0), fill(off.begin(), off.end() - 1);
        for (int64_t i = 0; i < n; ++i) idx[fill[star[i]]++] = (int32_t)i;
        STATUS_TRY(c->alloc(&c->star_off, off.size()));
        STATUS_TRY(c->alloc(&c->star_idx, nn));
        STATUS_TRY(c->alloc(&c->star_tot, (size_t)c->nstars * 16));
        CUDA_TRY(cudaMemcpy(c->star_off, off.data(), off.size() * sizeof(int64_t),
                            cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(c->star_idx, idx.data(), nn * sizeof(int32_t), cudaMemcpyHostToDevice));
    }
    CUDA_TRY(cudaMemset(c->zeros, 0, nn * sizeof(double)));
    // EoS, material, metric.
    STATUS_TRY(upload_eos(c, eos));
    c->mat.alpha_av = mat->alpha_av;
    c->mat.beta_av = mat->beta_av;
    c->mat.eta2 = mat->eta2;
    c->mat.jaumann = mat->jaumann;
    c->mat.yield_mode = mat->yield_mode;
    c->mat.break_stress = mat->break_stress;
    c->mat.break_zero_S = mat->break_zero_S;
    c->mat.alpha_f = (float)mat->alpha_av;
    c->mat.beta_f = (float)mat->beta_av;
    c->mat.eta2_f = (float)mat->eta2;
    c->met = DevMetric{};
    c->met.kind = 0;
    c->h_fstar.assign((size_t)c->nstars * kFStar, 0.f);
    STATUS_TRY(c->alloc(&c->d_fstar, c->h_fstar.size()));
    if (g && g->kind == 1) {
        int ns = g->nstars, nr = g->nr;
        c->met.kind = 1;
        c->met.nstars = ns;
        c->met.nr = nr;
        c->met.pressure_form = g->pressure_form;
        std::vector<double> tab((size_t)ns * nr * 4);
        std::vector<float> tabf(tab.size());
        for (size_t k = 0; k < (size_t)ns * nr; ++k) {
            tab[4 * k + 0] = g->alpha[k];
            tab[4 * k + 1] = g->dalpha[k];
            tab[4 * k + 2] = g->psi4[k];
            tab[4 * k + 3] = g->dpsi4[k];
        }
        for (size_t k = 0; k < tab.size(); ++k) tabf[k] = (float)tab[k];
        double *d_tab, *d_rmax, *d_M, *d_center;
        float *d_tabf;
        STATUS_TRY(c->alloc(&d_tab, tab.size()));
        STATUS_TRY(c->alloc(&d_tabf, tabf.size()));
        STATUS_TRY(c->alloc(&d_rmax, ns));
        STATUS_TRY(c->alloc(&d_M, ns));
        STATUS_TRY(c->alloc(&d_center, 3 * ns));
        CUDA_TRY(cudaMemcpy(d_tab, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(d_tabf, tabf.data(), tabf.size() * sizeof(float), cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(d_rmax, g->r_max, ns * sizeof(double), cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(d_M, g->M, ns * sizeof(double), cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(d_center, g->center, 3 * ns * sizeof(double), cudaMemcpyHostToDevice));
        c->met.tab = d_tab;
        c->met.tabf = d_tabf;
        c->met.r_max = d_rmax;
        c->met.M = d_M;
        c->met.center = d_center;
        for (int k = 0; k < ns; ++k) {
            float *f = &c->h_fstar[(size_t)k * kFStar];
            f[FS_RMAX] = (float)g->r_max[k];
            f[FS_M] = (float)g->M[k];
            split_float(g->center + 3 * k, f + FS_CHI, f + FS_CLO);
        }
    }
    CUDA_TRY(cudaMemcpy(c->d_fstar, c->h_fstar.data(), c->h_fstar.size() * sizeof(float),
                        cudaMemcpyHostToDevice));
    c->met.fstar = c->d_fstar;
    CUDA_TRY(cudaDeviceSynchronize());
    const bool tune_lanes = c->opt.lanes_per_particle == -1;
    const bool tune_persist = c->opt.persistent == -1 && prec == SPH_MIXED;
    if ((tune_lanes || tune_persist) && n > 0) STATUS_TRY(autotune_shape(c, tune_lanes, tune_persist));
    if ((c->opt.persistent == 1 || (tune_persist && c->tune_persist)) && prec == SPH_MIXED && n > 0) {
        c->pplan = plan_persistent(n, c->screen_lanes, c->lanes);
        CUDA_TRY(cudaGetLastError());
    }
    return SPH_OK;
}

int64_t state_blob_size(const sph_ctx *c)
{
    // header (8 int64) + doubles: x y z vx vy vz u h mu Y0 eps (11n) + S (6n)
    // + rates ax ay az dudt (4n) + dS (6n) + type, flags (2n bytes)
    // + the particle order of the last sort (4n bytes)
    return 64 + 8 * (27 * c->n) + 2 * c->n + 4 * c->n;
}

}  // namespace

extern "C" {

sph_status sph_init(sph_ctx **out, const sph_particles *particles, const sph_eos *eos,
                    const sph_material *material, const sph_metric *metric,
                    sph_precision precision, const sph_options *options, void *cuda_stream)
{
    NvtxRange nvtx_("sph_init");
    g_err[0] = 0;
    if (!out) return fail(SPH_ERR_ARG, "out is NULL");
    *out = nullptr;
    sph_status st = validate(particles, eos, material, metric, precision, options);
    if (st != SPH_OK) return st;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev < 1) {
        cudaGetLastError();
        return fail(SPH_ERR_NODEVICE, "no CUDA device: %s", cudaGetErrorString(e));
    }
    sph_ctx *c = new (std::nothrow) sph_ctx();
    if (!c) return fail(SPH_ERR_OOM, "host allocation failed");
    st = init_impl(c, particles, eos, material, metric, precision, options, cuda_stream);
    if (st != SPH_OK) {
        char keep[512];
        memcpy(keep, g_err, sizeof(keep));
        sph_free(c);
        memcpy(g_err, keep, sizeof(keep));
        return st;
    }
    *out = c;
    return SPH_OK;
}

sph_status sph_rhs(sph_ctx *c, const sph_rates *out)
{
    NvtxRange nvtx_("sph_rhs");
    if (!c || !out) return fail(SPH_ERR_ARG, "null argument");
    if (c->n > 0 && (!out->ax || !out->ay || !out->az || !out->dudt || !out->drhodt || !out->rho ||
                     !out->P || !out->D || !out->cs || !out->deps || !out->dR || !out->dS ||
                     !out->ncount))
        return fail(SPH_ERR_ARG, "a rate array is NULL");
    if (c->timing) {
        STATUS_TRY(ensure_slot(c));
        c->slot_kind_step = 0;
    }
    DevState st = state_of(c, c->P.vx, c->P.vy, c->P.vz, c->P.S);
    int nl = 0;
    enqueue_rhs(c, st, rates_of(out), false, &nl);
    if (c->timing) c->slot_used++;
    CUDA_TRY(cudaGetLastError());
    return SPH_OK;
}

sph_status sph_step(sph_ctx *c, double dt, int32_t nsteps)
{
    NvtxRange nvtx_("sph_step");
    if (!c) return fail(SPH_ERR_ARG, "ctx is NULL");
    if (!(dt > 0.0) || !std::isfinite(dt) || nsteps < 0) return fail(SPH_ERR_ARG, "bad dt or nsteps");
    if (c->n == 0) {
        c->steps += nsteps;
        return SPH_OK;
    }
    if (!c->have_rates) {
        // rates at the initial state (not a timed step: no events recorded)
        int timing = c->timing;
        c->timing = 0;
        DevState st = state_of(c, c->P.vx, c->P.vy, c->P.vz, c->P.S);
        enqueue_rhs(c, st, c->r, false, nullptr);
        c->timing = timing;
        c->have_rates = 1;
    }
    bool graph = c->opt.use_graph && c->stream != nullptr;
    for (int32_t k = 0; k < nsteps; ++k) {
        if (c->timing) {
            STATUS_TRY(ensure_slot(c));
            c->slot_kind_step = 1;
        }
        const bool resort = resort_at(c, c->steps);
        const int g = resort ? 1 : 0;
        if (graph) {
            if (!c->gexec[g] || c->gdt[g] != dt || c->gtiming[g] != c->timing)
                STATUS_TRY(capture_step(c, dt, resort));
            if (c->timing) {
                for (int e = 0; e < EV_N; ++e)
                    if (c->gev_nodes[g][e])
                        CUDA_TRY(cudaGraphExecEventRecordNodeSetEvent(
                            c->gexec[g], c->gev_nodes[g][e], c->slots[c->slot_used].ev[e]));
            }
            CUDA_TRY(cudaGraphLaunch(c->gexec[g], c->stream));
            c->launches_per_step = c->glaunches[g];
        } else {
            int nl = 0;
            enqueue_step(c, dt, false, &nl, resort);
            c->launches_per_step = nl;
        }
        c->launches_total += c->launches_per_step;
        if (c->timing) c->slot_used++;
        c->steps++;
        if (c->opt.totals_every > 0 && c->steps % c->opt.totals_every == 0) {
            StepState ss = step_state_of(c);
            launch_totals(ss, c->r.ncount, c->tot_partial, c->tot_out, c->stream);
        }
    }
    CUDA_TRY(cudaGetLastError());
    return SPH_OK;
}

sph_status sph_sync(sph_ctx *c)
{
    NvtxRange nvtx_("sph_sync");
    if (!c) return fail(SPH_ERR_ARG, "ctx is NULL");
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (c->n == 0) return SPH_OK;
    int err = 0;
    CUDA_TRY(cudaMemcpy(&err, &c->s.sc->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
        int zero = 0;
        CUDA_TRY(cudaMemcpy(&c->s.sc->err, &zero, sizeof(int), cudaMemcpyHostToDevice));
        if (err & ERR_NONFINITE) return fail(SPH_ERR_NONFINITE, "non-finite position, velocity or h");
        // a timed-out sort is the cause of any bounds flag raised with it
        if (err & ERR_TIMEOUT)
            return fail(SPH_ERR_TIMEOUT,
                        "a device-side wait gave up (a sort pass waiting for a predecessor "
                        "tile, or a force item of the persistent launch)");
        if (err & ERR_CAPACITY)
            return fail(SPH_ERR_CAPACITY,
                        "a particle has more than max_neighbors = %d neighbours, or a "
                        "tile-search walk more than %d candidate leaves",
                        c->cap, walk_capacity(c));
        if (err & ERR_BOUNDS) return fail(SPH_ERR_BOUNDS, "index out of bounds");
    }
    return SPH_OK;
}

sph_status sph_set_wait_limit(sph_ctx *c, int32_t polls)
{
    if (!c) return fail(SPH_ERR_ARG, "ctx is NULL");
    if (c->n == 0) return SPH_OK;
    // stored form: 0 the default, > 0 that many polls, < 0 none
    const int v = polls < 0 ? 0 : (polls == 0 ? -1 : polls);
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    CUDA_TRY(cudaMemcpy(&c->s.sc->spin_limit, &v, sizeof(int), cudaMemcpyHostToDevice));
    return SPH_OK;
}

sph_status sph_set_max_neighbors(sph_ctx *c, int32_t max_neighbors)
{
    if (!c) return fail(SPH_ERR_ARG, "ctx is NULL");
    if (max_neighbors < 1 || max_neighbors > kRowCap)
        return fail(SPH_ERR_ARG, "max_neighbors must be 1..%d", kRowCap);
    if (c->n == 0 || max_neighbors == c->cap) {
        c->cap = max_neighbors;
        c->opt.max_neighbors = max_neighbors;
        return SPH_OK;
    }
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (c->side) CUDA_TRY(cudaStreamSynchronize(c->side));
    const size_t count = (size_t)c->n * max_neighbors;
    int32_t *vl = nullptr, *nb = nullptr;
    cudaError_t e = cudaMalloc((void **)&vl, count * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc((void **)&nb, count * sizeof(int32_t));
    if (e != cudaSuccess) {
        if (vl) cudaFree(vl);
        cudaGetLastError();
        return fail(SPH_ERR_OOM, "lists of %d entries per particle: %s", max_neighbors,
                    cudaGetErrorString(e));
    }
    for (void *&p : c->allocs) {
        if (p == (void *)c->s.vlist) {
            cudaFree(p);
            p = vl;
        } else if (p == (void *)c->s.nbr) {
            cudaFree(p);
            p = nb;
        }
    }
    c->s.vlist = vl;
    c->s.nbr = nb;
    c->cap = max_neighbors;
    c->opt.max_neighbors = max_neighbors;
    // the step graphs hold the old lists and capacity; the next right-hand
    // side builds the candidate lists again
    drop_graph(c);
    const int zero = 0;
    CUDA_TRY(cudaMemcpy(&c->s.sc->built, &zero, sizeof(int), cudaMemcpyHostToDevice));
    return SPH_OK;
}

int32_t sph_build_checked(void)
{
#ifdef SPH_CHECKED
    return 1;
#else
    return 0;
#endif
}

sph_status sph_checked_set_candidate(sph_ctx *c, int64_t slot, int32_t k, int32_t value)
{
#ifdef SPH_CHECKED
    if (!c) return fail(SPH_ERR_ARG, "ctx is NULL");
    if (slot < 0 || slot >= c->n || k < 0 || k >= c->cap)
        return fail(SPH_ERR_ARG, "slot or entry out of range");
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    CUDA_TRY(cudaMemcpy(c->s.vlist + slot * (int64_t)c->cap + k, &value, sizeof(int32_t),
                        cudaMemcpyHostToDevice));
    return SPH_OK;
#else
    (void)c;
    (void)slot;
    (void)k;
    (void)value;
    return fail(SPH_ERR_ARG, "sph_checked_set_candidate exists only in bounds-checked builds");
#endif
}

sph_status sph_neighbors(sph_ctx *c, int64_t *offsets, int32_t *idx, int64_t cap)
{
    NvtxRange nvtx_("sph_neighbors");
    if (!c || !offsets || (cap > 0 && !idx) || cap < 0) return fail(SPH_ERR_ARG, "bad argument");
    const int64_t n = c->n;
    CUDA_TRY(cudaMemsetAsync(offsets, 0, (n + 1) * sizeof(int64_t), c->stream));
    // counts at [0, n), zero at n; the exclusive scan turns them into offsets
    launch_export_counts(c->s, n, offsets, c->stream);
    launch_scan_i64(offsets, n + 1, c->stream);
    int64_t total = 0;
    CUDA_TRY(cudaMemcpyAsync(&total, offsets + n, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (total > cap) return fail(SPH_ERR_CAPACITY, "neighbour lists hold %lld entries > cap %lld",
                                 (long long)total, (long long)cap);
    launch_export_fill(c->s, n, c->cap, offsets, idx, c->stream);
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    CUDA_TRY(cudaGetLastError());
    return SPH_OK;
}

sph_status sph_set_external(sph_ctx *c, const sph_external *e)
{
    if (!c) return fail(SPH_ERR_ARG, "ctx is NULL");
    if (!e || e->kind == 0) {
        c->met.ext_kind = 0;
        drop_graph(c);
        return SPH_OK;
    }
    if (e->kind != 1) return fail(SPH_ERR_ARG, "external kind must be 0 or 1");
    if (e->nstars != c->nstars) return fail(SPH_ERR_ARG, "external and eos star counts differ");
    if (e->nr < 2 || !e->r_max || !e->g || !e->center || !e->r_wall)
        return fail(SPH_ERR_ARG, "external table needs nr >= 2 and r_max, g, center, r_wall");
    if (!(e->k_wall >= 0.0) || !(e->damping >= 0.0) || !std::isfinite(e->k_wall) ||
        !std::isfinite(e->damping))
        return fail(SPH_ERR_ARG, "k_wall and damping must be finite and >= 0");
    const int ns = e->nstars, nr = e->nr;
    for (int s = 0; s < ns; ++s) {
        if (!(e->r_max[s] > 0.0) || !std::isfinite(e->r_max[s]) || !std::isfinite(e->r_wall[s]))
            return fail(SPH_ERR_ARG, "star %d: need finite r_max > 0 and r_wall", s);
        for (int k = 0; k < 3; ++k)
            if (!std::isfinite(e->center[3 * s + k])) return fail(SPH_ERR_ARG, "non-finite center");
    }
    std::vector<float> gf((size_t)ns * nr);
    for (size_t k = 0; k < gf.size(); ++k) {
        if (!std::isfinite(e->g[k])) return fail(SPH_ERR_ARG, "non-finite external table");
        gf[k] = (float)e->g[k];
    }
    double *d_g, *d_rmax, *d_center, *d_rwall;
    float *d_gf;
    STATUS_TRY(c->alloc(&d_g, gf.size()));
    STATUS_TRY(c->alloc(&d_gf, gf.size()));
    STATUS_TRY(c->alloc(&d_rmax, ns));
    STATUS_TRY(c->alloc(&d_center, 3 * ns));
    STATUS_TRY(c->alloc(&d_rwall, ns));
    CUDA_TRY(cudaMemcpy(d_g, e->g, gf.size() * sizeof(double), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(d_gf, gf.data(), gf.size() * sizeof(float), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(d_rmax, e->r_max, ns * sizeof(double), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(d_center, e->center, 3 * ns * sizeof(double), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(d_rwall, e->r_wall, ns * sizeof(double), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    c->met.ext_kind = 1;
    c->met.ext_nr = nr;
    c->met.ext_g = d_g;
    c->met.ext_gf = d_gf;
    c->met.ext_rmax = d_rmax;
    c->met.ext_center = d_center;
    c->met.ext_rwall = d_rwall;
    c->met.k_wall = e->k_wall;
    c->met.damping = e->damping;
    c->met.k_wall_f = (float)e->k_wall;
    c->met.damping_f = (float)e->damping;
    for (int k = 0; k < ns; ++k) {
        float *f = &c->h_fstar[(size_t)k * kFStar];
        f[FS_EXT_RMAX] = (float)e->r_max[k];
        f[FS_EXT_RWALL] = (float)e->r_wall[k];
        split_float(e->center + 3 * k, f + FS_EXT_CHI, f + FS_EXT_CLO);
    }
    CUDA_TRY(cudaMemcpy(c->d_fstar, c->h_fstar.data(), c->h_fstar.size() * sizeof(float),
                        cudaMemcpyHostToDevice));
    drop_graph(c);
    c->have_rates = 0;  // the field changes the accelerations
    return SPH_OK;
}

sph_status sph_relax_finish(sph_ctx *c, const sph_eos *eos)
{
    if (!c) return fail(SPH_ERR_ARG, "ctx is NULL");
    STATUS_TRY(check_eos(eos, c->nstars));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    STATUS_TRY(upload_eos(c, eos));
    c->met.ext_kind = 0;
    drop_graph(c);
    if (c->n > 0) {
        // density of the relaxed state, then u from the new equation of state
        int timing = c->timing;
        c->timing = 0;
        DevState st = state_of(c, c->P.vx, c->P.vy, c->P.vz, c->P.S);
        enqueue_rhs(c, st, c->r, false, nullptr);
        c->timing = timing;
        launch_set_u_from_eos(step_state_of(c), c->r, eos_of(c), c->stream);
        CUDA_TRY(cudaGetLastError());
    }
    c->have_rates = 0;  // the next step starts from rates of the modified state
    return SPH_OK;
}

sph_status sph_totals(sph_ctx *c, double out[16])
{
    NvtxRange nvtx_("sph_totals");
    if (!c || !out) return fail(SPH_ERR_ARG, "null argument");
    StepState ss = step_state_of(c);
    launch_totals(ss, c->have_rates ? c->r.ncount : nullptr, c->tot_partial, c->tot_out, c->stream);
    CUDA_TRY(cudaMemcpyAsync(out, c->tot_out, 16 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return SPH_OK;
}

sph_status sph_totals_per_star(sph_ctx *c, double *out, int32_t nstars)
{
    NvtxRange nvtx_("sph_totals_per_star");
    if (!c || !out) return fail(SPH_ERR_ARG, "null argument");
    if (nstars != c->nstars)
        return fail(SPH_ERR_ARG, "nstars = %d, the context holds %d stars", nstars, c->nstars);
    StepState ss = step_state_of(c);
    launch_star_totals(ss, c->have_rates ? c->r.ncount : nullptr, c->nstars, c->star_off,
                       c->star_idx, c->star_tot, c->stream);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaMemcpyAsync(out, c->star_tot, (size_t)nstars * 16 * sizeof(double),
                             cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return SPH_OK;
}

sph_status sph_stats(sph_ctx *c, int64_t out[32])
{
    if (!c || !out) return fail(SPH_ERR_ARG, "null argument");
    DevScalars sc{};
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    CUDA_TRY(cudaMemcpy(&sc, c->s.sc, sizeof(DevScalars), cudaMemcpyDeviceToHost));
    for (int k = 0; k < 32; ++k) out[k] = 0;
    out[0] = (int64_t)sc.pairs_last;
    out[1] = (int64_t)sc.pairs_total;
    out[2] = (int64_t)sc.rhs_count;
    out[3] = c->launches_per_step;
    out[4] = c->nleaves;
    out[5] = (int64_t)sc.rechecks;
    out[6] = c->cap;
    out[7] = c->lanes;
    out[8] = (c->opt.use_graph && c->stream != nullptr) ? 1 : 0;
    out[9] = c->steps;
    out[10] = c->plan.passes;
    out[11] = c->plan.key_bits_axis;
    out[12] = c->launches_total;
    out[13] = c->opt.sort_every > 1 ? c->opt.sort_every : 1;
    out[14] = sc.max_cand;
    out[15] = sc.max_count;
    out[16] = (int64_t)sc.tiles_last;
    out[17] = c->prec == SPH_FP64 ? 0 : 1;
    out[18] = (int64_t)sc.builds;
    out[19] = c->screen_lanes;
    out[20] = c->tuned;
    for (int k = 0; k < 4; ++k) out[21 + k] = c->tune_ns[k];
    out[25] = c->pplan.grid;
    out[26] = c->tune_ns[4];
    out[27] = c->tune_ns[5];
    for (int k = 0; k < 3; ++k) out[28 + k] = c->tune_ns[6 + k];
    out[31] = c->group;
    return SPH_OK;
}

sph_status sph_timing(sph_ctx *c, int32_t enable)
{
    if (!c) return fail(SPH_ERR_ARG, "ctx is NULL");
    c->timing = enable ? 1 : 0;
    c->slot_used = 0;
    return SPH_OK;
}

sph_status sph_timing_read(sph_ctx *c, double out[12])
{
    if (!c || !out) return fail(SPH_ERR_ARG, "null argument");
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    for (int k = 0; k < 12; ++k) out[k] = 0.0;
    auto add = [&](const TimingSlot &s, int a, int b, int k) -> bool {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, s.ev[a], s.ev[b]) != cudaSuccess) return false;
        out[k] += ms;
        out[k + 1] += 1;
        return true;
    };
    for (int k = 0; k < c->slot_used; ++k) {
        const TimingSlot &s = c->slots[k];
        add(s, EV_FORCE, EV_FORCE_END, 0);
        add(s, EV_DENSITY, EV_FORCE, 2);
        if (!add(s, EV_STEP, EV_STEP_END, 4)) add(s, EV_BUILD, EV_FORCE_END, 4);
        add(s, EV_BUILD, EV_LISTS, 6);
        add(s, EV_LISTS, EV_DENSITY, 8);
        add(s, EV_BUILD, EV_DENSITY, 10);
    }
    cudaGetLastError();
    c->slot_used = 0;
    return SPH_OK;
}

sph_status sph_state_size(sph_ctx *c, int64_t *bytes)
{
    if (!c || !bytes) return fail(SPH_ERR_ARG, "null argument");
    *bytes = state_blob_size(c);
    return SPH_OK;
}

sph_status sph_get_state(sph_ctx *c, void *host_buf, int64_t bytes)
{
    if (!c || !host_buf) return fail(SPH_ERR_ARG, "null argument");
    if (bytes < state_blob_size(c)) return fail(SPH_ERR_ARG, "buffer too small");
    const int64_t n = c->n;
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    int64_t *hdr = (int64_t *)host_buf;
    hdr[0] = 0x53504831;  // "SPH1"
    hdr[1] = n;
    hdr[2] = c->steps;
    hdr[3] = c->have_rates;
    hdr[4] = c->nstars;
    hdr[5] = hdr[6] = hdr[7] = 0;
    char *p = (char *)host_buf + 64;
    auto get = [&](const void *src, size_t sz) -> sph_status {
        if (src) CUDA_TRY(cudaMemcpy(p, src, sz, cudaMemcpyDeviceToHost));
        else memset(p, 0, sz);
        p += sz;
        return SPH_OK;
    };
    const size_t d = n * sizeof(double);
    const double *fields[11] = {c->P.x, c->P.y, c->P.z, c->P.vx, c->P.vy, c->P.vz,
                                c->P.u, c->P.h, c->P.mu, c->P.Y0, c->P.eps_break};
    for (const double *f : fields) STATUS_TRY(get(f, d));
    STATUS_TRY(get(c->P.S, 6 * d));
    for (const double *f : {c->r.ax, c->r.ay, c->r.az, c->r.dudt}) STATUS_TRY(get(f, d));
    STATUS_TRY(get(c->r.dS, 6 * d));
    STATUS_TRY(get(c->P.type, n));
    STATUS_TRY(get(c->P.flags, n));
    STATUS_TRY(get(c->s.perm, 4 * (size_t)n));
    return SPH_OK;
}

sph_status sph_set_state(sph_ctx *c, const void *host_buf, int64_t bytes)
{
    if (!c || !host_buf) return fail(SPH_ERR_ARG, "null argument");
    if (bytes < state_blob_size(c)) return fail(SPH_ERR_ARG, "buffer too small");
    const int64_t n = c->n;
    const int64_t *hdr = (const int64_t *)host_buf;
    if (hdr[0] != 0x53504831 || hdr[1] != n || hdr[4] != c->nstars)
        return fail(SPH_ERR_ARG, "checkpoint does not match this context");
    {
        // the stored particle order (the blob's last 4n bytes) must be a
        // permutation; checked before anything is copied
        const int32_t *perm =
            (const int32_t *)((const char *)host_buf + state_blob_size(c) - 4 * n);
        std::vector<unsigned char> seen((size_t)n, 0);
        for (int64_t i = 0; i < n; ++i) {
            if (perm[i] < 0 || perm[i] >= n)
                return fail(SPH_ERR_BOUNDS, "checkpoint order entry %lld = %d is outside [0, %lld)",
                            (long long)i, perm[i], (long long)n);
            if (seen[(size_t)perm[i]])
                return fail(SPH_ERR_ARG, "checkpoint order is not a permutation");
            seen[(size_t)perm[i]] = 1;
        }
    }
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    const char *p = (const char *)host_buf + 64;
    auto put = [&](void *dst, size_t sz) -> sph_status {
        if (dst) CUDA_TRY(cudaMemcpy(dst, p, sz, cudaMemcpyHostToDevice));
        p += sz;
        return SPH_OK;
    };
    const size_t d = n * sizeof(double);
    for (double *f : {c->P.x, c->P.y, c->P.z, c->P.vx, c->P.vy, c->P.vz, c->P.u, c->P.h, c->P.mu,
                      c->P.Y0, c->P.eps_break})
        STATUS_TRY(put(f, d));
    STATUS_TRY(put(c->P.S, 6 * d));
    for (double *f : {c->r.ax, c->r.ay, c->r.az, c->r.dudt}) STATUS_TRY(put(f, d));
    STATUS_TRY(put(c->r.dS, 6 * d));
    STATUS_TRY(put(c->P.type, n));
    STATUS_TRY(put(c->P.flags, n));
    // the order of the last sort (checked above): the steps that keep it sum
    // pairs in the same order as the run that wrote the checkpoint
    STATUS_TRY(put(c->s.perm, 4 * (size_t)n));
    c->steps = hdr[2];
    c->have_rates = (int)hdr[3];
    // the candidate lists belong to the order and positions of their own
    // build, not to the restored ones: the next right-hand side builds them
    const int zero = 0;
    CUDA_TRY(cudaMemcpy(&c->s.sc->built, &zero, sizeof(int), cudaMemcpyHostToDevice));
    return SPH_OK;
}

void sph_free(sph_ctx *c)
{
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    drop_graph(c);
    if (c->side) {
        cudaStreamSynchronize(c->side);
        cudaStreamDestroy(c->side);
    }
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    for (auto &s : c->slots)
        for (int e = 0; e < EV_N; ++e) cudaEventDestroy(s.ev[e]);
    for (void *p : c->allocs) cudaFree(p);
    cudaGetLastError();
    delete c;
}

const char *sph_last_error(void) { return g_err; }

}  // extern "C"

void sph::record_error(const char *msg) { snprintf(g_err, sizeof(g_err), "%s", msg); }
