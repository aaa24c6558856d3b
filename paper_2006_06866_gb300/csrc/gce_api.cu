// C ABI of the CE search library: argument checks, the handle's device
// workspace, the per-call kernel sequence (init -> scan -> trial constants ->
// per-curve prep -> persistent CE kernel -> top-k merge), its capture into
// CUDA graphs, and the launch-shape autotuner.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <numeric>
#include <string>
#include <tuple>
#include <vector>

#include "gce_internal.cuh"
#include "gce_topk.cuh"

using namespace gce;

namespace {

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

// mode, n_phase, n_mag, log2 bucket of N, Pdot axis (n_pdots > 1: period-major tiles)
typedef std::tuple<int, int, int, int, int> TuneKey;

enum JobKind { JOB_GRID = 0, JOB_TOPK = 1, JOB_SINGLE = 2, JOB_COUNTS = 3 };

struct GraphKey {
    int kind, mode, n_curves, n_periods, n_pdots, n_phase, n_mag, k, block, tpt, grid, chunk,
        table_smem, grab;
    long long n_points;
    bool operator<(const GraphKey &o) const {
        return std::tie(kind, mode, n_curves, n_periods, n_pdots, n_phase, n_mag, k, block, tpt,
                        grid, chunk, table_smem, grab, n_points) <
               std::tie(o.kind, o.mode, o.n_curves, o.n_periods, o.n_pdots, o.n_phase, o.n_mag,
                        o.k, o.block, o.tpt, o.grid, o.chunk, o.table_smem, o.grab, o.n_points);
    }
};

// Everything a captured call sequence bakes into its nodes besides the launch
// shape (which the GraphKey holds): the caller's arrays, the epoch, the flags,
// and the handle's own workspace and pinned staging buffers.  A call whose
// fingerprint equals the cached graph's replays that graph as it is.
struct Fingerprint {
    uintptr_t v[40];
    int n = 0;
    void add(const void *p) { v[n++] = (uintptr_t)p; }
    void add_u(unsigned long long x) { v[n++] = (uintptr_t)x; }
    bool operator==(const Fingerprint &o) const {
        return n == o.n && std::memcmp(v, o.v, sizeof(uintptr_t) * (size_t)n) == 0;
    }
};

// The inputs of a launch shape's fitting (mode, bins, longest curve, top-k,
// slot range, the tuning's block / tpt / chunk / CTA cap) and its result, so
// that repeated calls skip the driver queries of the fitting.
typedef std::tuple<int, int, int, int, int, int, int, int, int, int> ShapeKey;
struct LaunchShape {
    int block, tpt, chunk, table_smem, occ;
    size_t smem;
};

constexpr int kCheckedArrays = 14;

struct CachedGraph {
    cudaGraphExec_t exec = nullptr;
    Fingerprint fp;
    int launches = 0;  // kernels the sequence launches
};

}  // namespace

struct gce_handle_s {
    int device = 0;
    int n_sm = 0;
    int smem_optin = 0;
    std::string last_error;
    DevBuf payload, seg, trialc, order, offsets, cand, stats, table, state, in_times, in_mags,
        in_periods, in_pdots, out_H, out_idx, band_stats, cand2, stats2;
    int table_n = -1;                    // largest count the table covers
    int *h_order = nullptr;              // pinned staging
    long long *h_offsets = nullptr;
    size_t h_cap = 0;
    JobState *h_state = nullptr;         // pinned copy target for the check flags
    cudaEvent_t staged = nullptr;        // staging buffers free again after this
    bool staged_pending = false;
    cudaEvent_t k0 = nullptr, k1 = nullptr;  // around the CE kernel (GCE_FLAG_TIME_KERNEL)
    bool timed = false;
    int launches = 0;                    // kernels the last job launched (directly or in its graph)
    std::map<TuneKey, gce_tuning> tune;
    std::map<GraphKey, CachedGraph> graphs;
    std::map<ShapeKey, LaunchShape> shapes;  // launch shapes already fitted to the device
    const void *checked[kCheckedArrays] = {};  // arrays of the last call found on the device
};

static std::string g_create_error;

static gce_status fail(gce_handle h, gce_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (h) h->last_error = buf;
    else g_create_error = buf;
    return st;
}

#define CUDA_TRY(h, expr)                                                                   \
    do {                                                                                    \
        cudaError_t e_ = (expr);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return fail((h), GCE_ERR_CUDA, "%s failed: %s", #expr, cudaGetErrorString(e_)); \
    } while (0)

static gce_status ensure(gce_handle h, DevBuf &b, size_t bytes) {
    if (bytes <= b.bytes && b.p) return GCE_OK;
    size_t want = std::max(bytes, (size_t)256);
    want = std::max(want, b.bytes + b.bytes / 2);
    if (b.p) {
        // in-flight work may still read the old buffer
        CUDA_TRY(h, cudaDeviceSynchronize());
        CUDA_TRY(h, cudaFree(b.p));
        b.p = nullptr;
        b.bytes = 0;
    }
    if (cudaMalloc(&b.p, want) != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        if (cudaMalloc(&b.p, bytes) != cudaSuccess) {
            cudaGetLastError();
            b.p = nullptr;
            return fail(h, GCE_ERR_NOMEM, "device allocation of %zu bytes failed", bytes);
        }
        want = bytes;
    }
    b.bytes = want;
    return GCE_OK;
}

static int point_bytes(int mode) { return mode == GCE_PHASE_FP64 ? 8 : 16; }

static size_t trial_bytes(int mode) {
    switch (mode) {
        case GCE_PHASE_FP64: return sizeof(ModeTraits<GCE_PHASE_FP64>::trial_t);
        case GCE_PHASE_SPLIT32: return sizeof(ModeTraits<GCE_PHASE_SPLIT32>::trial_t);
        default: return sizeof(ModeTraits<GCE_PHASE_FIXED32>::trial_t);
    }
}

static int ilog2_ceil(long long v) {
    int e = 0;
    while ((1ll << e) < v) ++e;
    return e;
}

static gce_tuning default_tuning(int mode, int n_max) {
    gce_tuning t;
    t.block = 256;
    t.tpt = 2;
    t.ctas_per_sm = 0;
    t.chunk = mode == GCE_PHASE_FP64 ? 4096 : 2048;
    t.slot_range = 0;
    (void)n_max;
    return t;
}

static bool tuning_ok(const gce_tuning &t, int mode) {
    const bool block_ok = t.block == 64 || t.block == 128 || t.block == 256 || t.block == 512;
    const bool tpt_ok = t.tpt == 1 || t.tpt == 2 || (t.tpt == 4 && mode != GCE_PHASE_FP64);
    return block_ok && tpt_ok && t.ctas_per_sm >= 0 && t.ctas_per_sm <= 32 &&
           t.chunk >= 256 && t.chunk <= 8192 && t.chunk % 256 == 0 &&
           (t.slot_range == 0 || t.slot_range == 1);
}

static TuneKey tune_key(const gce_config *cfg, int n_obs, int pd_axis) {
    return TuneKey(cfg->phase_mode, cfg->n_phase_bins, cfg->n_mag_bins,
                   ilog2_ceil(std::max(n_obs, 1)), pd_axis);
}

// The cached shape for the key; a Pdot-axis job without its own entry uses the
// plain one.
static gce_tuning lookup_tuning(gce_handle h, const gce_config *cfg, int n_max, int pd_axis) {
    auto it = h->tune.find(tune_key(cfg, n_max, pd_axis));
    if (it != h->tune.end()) return it->second;
    if (pd_axis) return lookup_tuning(h, cfg, n_max, 0);
    return default_tuning(cfg->phase_mode, n_max);
}

extern "C" const char *gce_status_string(gce_status s) {
    switch (s) {
        case GCE_OK: return "ok";
        case GCE_ERR_INVALID: return "invalid argument or input value";
        case GCE_ERR_CUDA: return "CUDA error";
        case GCE_ERR_NOMEM: return "device memory exhausted";
        case GCE_ERR_UNSUPPORTED: return "input outside the range of the chosen phase fold";
        default: return "unknown status";
    }
}

extern "C" const char *gce_last_error(gce_handle h) {
    return h ? h->last_error.c_str() : g_create_error.c_str();
}

extern "C" gce_status gce_check_job(const int64_t *h_offsets, int32_t n_curves,
                                    int32_t n_periods, int32_t n_pdots, const gce_config *cfg,
                                    int32_t k) {
    if (!cfg) return GCE_ERR_INVALID;
    if (cfg->n_phase_bins < 1 || cfg->n_phase_bins > GCE_MAX_PHASE_BINS) return GCE_ERR_INVALID;
    if (cfg->n_mag_bins < 1 || cfg->n_mag_bins > GCE_MAX_MAG_BINS) return GCE_ERR_INVALID;
    if (cfg->phase_mode != GCE_PHASE_FP64 && cfg->phase_mode != GCE_PHASE_SPLIT32 &&
        cfg->phase_mode != GCE_PHASE_FIXED32)
        return GCE_ERR_INVALID;
    if (!std::isfinite(cfg->t0)) return GCE_ERR_INVALID;
    if ((cfg->flags & GCE_FLAG_OVERLAP) && cfg->n_phase_bins < 2) return GCE_ERR_INVALID;
    if (n_curves < 0 || n_periods < 1 || n_pdots < 1) return GCE_ERR_INVALID;
    const long long n_trials = (long long)n_periods * n_pdots;
    if (n_trials >= (1ll << 32)) return GCE_ERR_INVALID;
    if (k < 0 || k > GCE_MAX_TOPK || k > n_trials) return GCE_ERR_INVALID;
    if (n_curves > 0) {
        if (!h_offsets || h_offsets[0] != 0) return GCE_ERR_INVALID;
        for (int32_t c = 0; c < n_curves; ++c) {
            const long long n = h_offsets[c + 1] - h_offsets[c];
            if (n < 1 || n > GCE_MAX_CURVE_POINTS) return GCE_ERR_INVALID;
        }
    }
    return GCE_OK;
}

extern "C" gce_status gce_create(gce_handle *out, int32_t device) {
    if (!out) return fail(nullptr, GCE_ERR_INVALID, "gce_create: NULL output pointer");
    *out = nullptr;
    int n_dev = 0;
    cudaError_t e = cudaGetDeviceCount(&n_dev);
    if (e != cudaSuccess)
        return fail(nullptr, GCE_ERR_CUDA, "cudaGetDeviceCount: %s", cudaGetErrorString(e));
    if (device < 0 || device >= n_dev)
        return fail(nullptr, GCE_ERR_INVALID, "device %d out of range (%d devices)", device, n_dev);
    e = cudaSetDevice(device);
    if (e != cudaSuccess)
        return fail(nullptr, GCE_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    gce_handle h = new (std::nothrow) gce_handle_s();
    if (!h) return fail(nullptr, GCE_ERR_NOMEM, "host allocation failed");
    h->device = device;
    cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, device);
    cudaDeviceGetAttribute(&h->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    if (cudaEventCreateWithFlags(&h->staged, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreate(&h->k0) != cudaSuccess || cudaEventCreate(&h->k1) != cudaSuccess ||
        cudaMallocHost((void **)&h->h_state, sizeof(JobState)) != cudaSuccess) {
        e = cudaGetLastError();
        gce_destroy(h);
        return fail(nullptr, GCE_ERR_CUDA, "handle setup: %s", cudaGetErrorString(e));
    }
    if (ensure(h, h->state, sizeof(JobState)) != GCE_OK) {
        gce_destroy(h);
        return fail(nullptr, GCE_ERR_NOMEM, "workspace allocation failed");
    }
    *out = h;
    return GCE_OK;
}

extern "C" gce_status gce_destroy(gce_handle h) {
    if (!h) return GCE_ERR_INVALID;
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    for (auto &kv : h->graphs) cudaGraphExecDestroy(kv.second.exec);
    DevBuf *bufs[] = {&h->payload, &h->seg, &h->trialc, &h->order, &h->offsets, &h->cand, &h->stats,
                      &h->table, &h->state, &h->in_times, &h->in_mags, &h->in_periods,
                      &h->in_pdots, &h->out_H, &h->out_idx, &h->band_stats, &h->cand2,
                      &h->stats2};
    for (DevBuf *b : bufs)
        if (b->p) cudaFree(b->p);
    if (h->h_order) cudaFreeHost(h->h_order);
    if (h->h_offsets) cudaFreeHost(h->h_offsets);
    if (h->h_state) cudaFreeHost(h->h_state);
    if (h->staged) cudaEventDestroy(h->staged);
    if (h->k0) cudaEventDestroy(h->k0);
    if (h->k1) cudaEventDestroy(h->k1);
    delete h;
    return GCE_OK;
}

namespace {

struct Job {
    int kind;
    const double *times, *mags, *periods, *pdots;
    const int64_t *h_offsets;
    int n_curves, n_periods, n_pdots;
    const gce_config *cfg;
    int k;
    float *out;                  // grid (JOB_GRID, JOB_SINGLE)
    float *topk_H;               // JOB_TOPK
    int64_t *topk_idx;
    double *mean, *std_dev;      // JOB_TOPK with significance (rho != nullptr)
    float *rho;
    long long n_cells;           // JOB_COUNTS
    const int64_t *cell_curve, *cell_trial;
    uint32_t *counts;
    const gce_tuning *force;     // tuning override (autotuner)
    const unsigned char *bands;  // multi-filter input (nullptr: one filter, raw magnitudes)
    int n_bands;
};

struct Plan {
    long long n_points, n_trials, n_items, n_long_items;
    long long n_lists;    // top-k candidate lists (and moment records) per curve: tiles x warps
    int n_long, n_short;  // curves taken curve-major / tile-major (see MainArgs)
    int n_max, n_tiles, n_ptiles, pd_major, range, half, kv, block, tpt, grid, chunk, table_smem,
        grab;
    int n_groups, tiles_per_group;  // top-k: first merge level (0 groups: none)
    size_t smem;
};

// Curves of at most this many points are scheduled tile-major (Plan).
constexpr long long kShortCurve = 256;

gce_status make_plan(gce_handle h, const Job &j, Plan &pl) {
    const gce_config *cfg = j.cfg;
    pl.n_points = (long long)j.h_offsets[j.n_curves];
    pl.n_trials = (long long)j.n_periods * j.n_pdots;
    long long nmax = 1;
    for (int c = 0; c < j.n_curves; ++c) nmax = std::max<long long>(nmax, j.h_offsets[c + 1] - j.h_offsets[c]);
    pl.n_max = (int)nmax;
    const gce_tuning t = j.force ? *j.force : lookup_tuning(h, cfg, pl.n_max, j.n_pdots > 1 ? 1 : 0);
    const int kk = j.kind == JOB_TOPK ? j.k : 0;
    // SPLIT32's kept slot range: narrow with a Pdot axis (every fold re-reduced),
    // else the tuned one (mid: warps with many cycles re-reduce)
    pl.range = RANGE_WIDE;
    if (cfg->phase_mode == GCE_PHASE_SPLIT32)
        pl.range = j.n_pdots > 1 ? RANGE_NARROW : t.slot_range == 1 ? RANGE_MID : RANGE_WIDE;
    // one Pdot value: the SPLIT32 / FIXED32 staging holds 8-byte half points
    pl.half = (cfg->phase_mode != GCE_PHASE_FP64 && j.n_pdots == 1) ? 1 : 0;
    // the kernel instantiation: overlapping bins or not
    pl.kv = kernel_variant((cfg->flags & GCE_FLAG_OVERLAP) != 0);
    const int kv = pl.kv;
    const ShapeKey skey(cfg->phase_mode, cfg->n_phase_bins, cfg->n_mag_bins, pl.n_max, kk,
                        pl.range * 8 + pl.half * 4 + kv, t.block, t.tpt, t.chunk,
                        t.ctas_per_sm);
    int occ = 0;
    auto sit = h->shapes.find(skey);
    if (sit != h->shapes.end()) {
        const LaunchShape &ls = sit->second;
        pl.block = ls.block;
        pl.tpt = ls.tpt;
        pl.chunk = ls.chunk;
        pl.table_smem = ls.table_smem;
        pl.smem = ls.smem;
        occ = ls.occ;
    } else {
        pl.block = t.block;
        pl.tpt = t.tpt;
        pl.chunk = std::min(t.chunk, ((pl.n_max + 31) / 32) * 32);
        // the c ln c table in shared memory: the whole table when it has at most
        // 2048 entries (16 KB), so that lookups need no bounds test; longer curves
        // read counts above it from global memory
        pl.table_smem = std::min(pl.n_max + 1, 2048);
        // shrink the staged chunk, then the table, then trials per thread, then the
        // block, until the CTA fits in shared memory
        auto size = [&]() {
            return main_smem_bytes(cfg->phase_mode, pl.block, pl.tpt, pl.chunk, cfg->n_phase_bins,
                                   cfg->n_mag_bins, pl.table_smem, pl.range, pl.half);
        };
        auto limit = [&]() {
            return main_dynamic_smem_limit(cfg->phase_mode, pl.tpt, pl.block, kv, (size_t)h->smem_optin);
        };
        pl.smem = size();
        while (pl.smem > limit()) {
            if (pl.chunk > 512) pl.chunk /= 2;
            else if (pl.table_smem > 256) pl.table_smem /= 2;
            else if (pl.tpt > 1) pl.tpt /= 2;
            else if (pl.block > 64) pl.block /= 2;
            else if (pl.chunk > 64) pl.chunk /= 2;
            else break;
            pl.smem = size();
        }
        if (pl.smem > limit())
            return fail(h, GCE_ERR_UNSUPPORTED, "launch shape needs %zu bytes of shared memory", pl.smem);
        CUDA_TRY(h, main_kernel_attrs(cfg->phase_mode, pl.tpt, pl.block, kv, (size_t)h->smem_optin));
        const void *kern = main_kernel_ptr(cfg->phase_mode, pl.tpt, pl.block, kv);
        CUDA_TRY(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, pl.block, pl.smem));
        if (occ < 1) return fail(h, GCE_ERR_UNSUPPORTED, "launch shape does not fit on an SM");
        // A smaller staged chunk costs only more staging passes: take it whenever it
        // admits more CTAs per SM (the counters leave little room at many phase bins,
        // and the top-k buffer grows with k, so the tuned chunk can sit just past an
        // occupancy step for another k).
        // Every halving down to 256 points is tried; the largest chunk that reaches
        // the best occupancy is kept.
        {
            int best_chunk = pl.chunk;
            size_t best_smem = pl.smem;
            for (int c = pl.chunk; c > 256;) {
                c = std::max(256, (c / 2 + 31) / 32 * 32);
                pl.chunk = c;
                const size_t sm2 = size();
                int occ2 = 0;
                CUDA_TRY(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2, kern, pl.block, sm2));
                if (occ2 > occ) {
                    occ = occ2;
                    best_chunk = c;
                    best_smem = sm2;
                }
            }
            pl.chunk = best_chunk;
            pl.smem = best_smem;
        }
        h->shapes[skey] = LaunchShape{pl.block, pl.tpt, pl.chunk, pl.table_smem, occ, pl.smem};
    }
    const TileGrid tg = tile_grid(j.n_periods, j.n_pdots, pl.block, pl.tpt);
    pl.n_tiles = (int)tg.n_tiles;
    pl.n_ptiles = tg.n_ptiles;
    pl.pd_major = tg.pd_major;
    pl.n_items = (long long)j.n_curves * pl.n_tiles;
    // curves of at most kShortCurve points run tile-major: a CTA then takes one
    // tile for several curves and loads its trial constants once
    pl.n_short = 0;
    for (int c = 0; c < j.n_curves; ++c)
        if (j.h_offsets[c + 1] - j.h_offsets[c] <= kShortCurve) ++pl.n_short;
    pl.n_long = j.n_curves - pl.n_short;
    pl.n_long_items = (long long)pl.n_long * pl.n_tiles;
    // each warp of a tile writes its own candidate list and moments
    pl.n_lists = (long long)pl.n_tiles * (pl.block / 32);
    pl.n_groups = j.kind == JOB_TOPK ? topk_groups(pl.n_lists, j.k, &pl.tiles_per_group) : 0;
    if (j.kind != JOB_TOPK) pl.tiles_per_group = 0;
    if (t.ctas_per_sm > 0) occ = std::min(occ, t.ctas_per_sm);
    long long g = (long long)h->n_sm * occ;
    g = std::min(g, std::max(pl.n_items, 1ll));
    pl.grid = (int)g;
    // about 128 grabs per CTA: large enough to amortise the counter, small enough
    // that the last grabs leave little tail
    long long grab = pl.n_items / (g * 128);
    pl.grab = (int)std::max(1ll, std::min(grab, 64ll));
    return GCE_OK;
}

// Event around the CE kernel; under stream capture it becomes an event-record node.
gce_status mark(gce_handle h, cudaEvent_t e, cudaStream_t s, bool capturing) {
    if (capturing) CUDA_TRY(h, cudaEventRecordWithFlags(e, s, cudaEventRecordExternal));
    else CUDA_TRY(h, cudaEventRecord(e, s));
    return GCE_OK;
}

// Enqueue the whole sequence of one call on stream s (possibly under capture).
gce_status enqueue(gce_handle h, const Job &j, const Plan &pl, cudaStream_t s, bool capturing) {
    const gce_config *cfg = j.cfg;
    const int mode = cfg->phase_mode;
    JobState *st = (JobState *)h->state.p;
    CUDA_TRY(h, cudaMemcpyAsync(h->offsets.p, h->h_offsets, sizeof(long long) * (j.n_curves + 1),
                                cudaMemcpyHostToDevice, s));
    CUDA_TRY(h, cudaMemcpyAsync(h->order.p, h->h_order, sizeof(int) * j.n_curves,
                                cudaMemcpyHostToDevice, s));
    int n_launch = 0;  // kernels this sequence launches, for gce_last_launches
    CUDA_TRY(h, launch_init(st, s));
    CUDA_TRY(h, launch_scan(j.times, j.mags, pl.n_points, j.periods, j.n_periods, j.pdots,
                            j.n_pdots, cfg->t0, st, s));
    n_launch += 2;
    TrialArgs ta;
    ta.periods = j.periods;
    ta.pdots = j.pdots;
    ta.n_periods = j.n_periods;
    ta.n_pdots = j.n_pdots;
    ta.trialc = h->trialc.p;
    ta.state = st;
    CUDA_TRY(h, launch_trials(mode, ta, s));
    ++n_launch;
    PrepArgs pa;
    pa.times = j.times;
    pa.mags = j.mags;
    pa.offsets = (const long long *)h->offsets.p;
    pa.n_curves = j.n_curves;
    pa.n_mag = cfg->n_mag_bins;
    pa.t0 = cfg->t0;
    pa.payload = h->payload.p;
    pa.seg = (int *)h->seg.p;
    pa.state = st;
    pa.bands = j.bands;
    pa.band_stats = (const double2 *)h->band_stats.p;
    pa.n_bands = j.bands ? j.n_bands : 0;
    if (j.bands) {
        CUDA_TRY(h, launch_band_stats(j.mags, j.bands, pa.offsets, j.n_curves, j.n_bands,
                                      (double2 *)h->band_stats.p, st, s));
        ++n_launch;
    }
    CUDA_TRY(h, launch_prep(mode, pa, s));
    ++n_launch;
    MainArgs ma;
    ma.payload = h->payload.p;
    ma.offsets = (const long long *)h->offsets.p;
    ma.seg = (const int *)h->seg.p;
    ma.trialc = h->trialc.p;
    ma.order = (const int *)h->order.p;
    ma.table = (const unsigned long long *)h->table.p;
    ma.n_trials = pl.n_trials;
    ma.n_periods = j.n_periods;
    ma.n_pdots = j.n_pdots;
    ma.n_tiles = pl.n_tiles;
    ma.n_ptiles = pl.n_ptiles;
    ma.pd_major = pl.pd_major;
    ma.range = pl.range;
    ma.n_items = pl.n_items;
    ma.n_long_items = pl.n_long_items;
    ma.n_long = pl.n_long;
    ma.n_short = pl.n_short;
    ma.grab = pl.grab;
    ma.n_phase = cfg->n_phase_bins;
    ma.n_mag = cfg->n_mag_bins;
    ma.chunk = pl.chunk;
    ma.table_smem = pl.table_smem;
    ma.out = nullptr;
    ma.cand = nullptr;
    ma.k = 0;
    ma.stats = nullptr;
    ma.overlap = (cfg->flags & GCE_FLAG_OVERLAP) ? 1 : 0;
    ma.half = pl.half;
    ma.kv = pl.kv;
    ma.state = st;
    const bool timed = (cfg->flags & GCE_FLAG_TIME_KERNEL) != 0;
    gce_status ms;
    switch (j.kind) {
        case JOB_GRID:
            ma.out = j.out;
            if (timed && (ms = mark(h, h->k0, s, capturing)) != GCE_OK) return ms;
            CUDA_TRY(h, launch_main(mode, pl.tpt, pl.block, pl.grid, pl.smem, ma, s));
            ++n_launch;
            if (timed && (ms = mark(h, h->k1, s, capturing)) != GCE_OK) return ms;
            break;
        case JOB_TOPK:
            ma.cand = (unsigned long long *)h->cand.p;
            ma.k = j.k;
            if (j.rho) ma.stats = (TileStats *)h->stats.p;
            if (timed && (ms = mark(h, h->k0, s, capturing)) != GCE_OK) return ms;
            CUDA_TRY(h, launch_main(mode, pl.tpt, pl.block, pl.grid, pl.smem, ma, s));
            ++n_launch;
            if (timed && (ms = mark(h, h->k1, s, capturing)) != GCE_OK) return ms;
            if (pl.n_groups > 0) {
                // many tiles per curve: reduce groups of tiles first, then merge the groups
                TileStats *stats2 = j.rho ? (TileStats *)h->stats2.p : nullptr;
                CUDA_TRY(h, launch_topk_reduce((const unsigned long long *)h->cand.p, j.n_curves,
                                               (int)pl.n_lists, j.k, pl.tiles_per_group, pl.n_groups,
                                               ma.stats, (unsigned long long *)h->cand2.p, stats2,
                                               st, s));
                CUDA_TRY(h, launch_topk_merge((const unsigned long long *)h->cand2.p, j.n_curves,
                                              pl.n_groups, j.k, j.topk_H, (long long *)j.topk_idx,
                                              stats2, j.mean, j.std_dev, j.rho, st, s));
                n_launch += 2;
            } else {
                CUDA_TRY(h, launch_topk_merge((const unsigned long long *)h->cand.p, j.n_curves,
                                              (int)pl.n_lists, j.k, j.topk_H, (long long *)j.topk_idx,
                                              ma.stats, j.mean, j.std_dev, j.rho, st, s));
                ++n_launch;
            }
            break;
        case JOB_SINGLE:
            ma.out = j.out;
            if (timed && (ms = mark(h, h->k0, s, capturing)) != GCE_OK) return ms;
            for (int c = 0; c < j.n_curves; ++c) CUDA_TRY(h, launch_single(ma, c, 0, s));
            n_launch += j.n_curves;
            if (timed && (ms = mark(h, h->k1, s, capturing)) != GCE_OK) return ms;
            break;
        case JOB_COUNTS:
            CUDA_TRY(h, cudaMemsetAsync(j.counts, 0,
                                        sizeof(uint32_t) * (size_t)j.n_cells * cfg->n_mag_bins *
                                            cfg->n_phase_bins, s));
            CUDA_TRY(h, launch_counts(mode, ma, j.n_cells, (const long long *)j.cell_curve,
                                      (const long long *)j.cell_trial, (unsigned int *)j.counts, s));
            if (j.n_cells > 0) ++n_launch;
            break;
    }
    h->launches += n_launch;
    return GCE_OK;
}

// A device array must be on the handle's device: memory the runtime reports as
// another device's is rejected (managed and host-registered memory is left to
// the driver).
bool on_device(const void *ptr, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return a.type != cudaMemoryTypeDevice || a.device == dev;
}

gce_status run_job(gce_handle h, const Job &j, cudaStream_t s) {
    if (!h) return GCE_ERR_INVALID;
    h->launches = 0;
    const gce_status chk = gce_check_job(j.h_offsets, j.n_curves, j.n_periods, j.n_pdots, j.cfg,
                                         j.kind == JOB_TOPK ? j.k : 0);
    if (chk != GCE_OK) return fail(h, chk, "argument check failed");
    if (j.kind == JOB_TOPK && j.k < 1) return fail(h, GCE_ERR_INVALID, "k must be >= 1");
    if (j.kind == JOB_SINGLE && j.cfg->phase_mode != GCE_PHASE_FP64)
        return fail(h, GCE_ERR_INVALID, "the one-launch-per-curve baseline is FP64 only");
    if (j.n_curves == 0) return GCE_OK;
    if (!j.times || !j.mags || !j.periods || !j.pdots)
        return fail(h, GCE_ERR_INVALID, "NULL input array");
    if ((j.kind == JOB_GRID || j.kind == JOB_SINGLE) && !j.out)
        return fail(h, GCE_ERR_INVALID, "NULL output array");
    if (j.kind == JOB_TOPK && (!j.topk_H || !j.topk_idx))
        return fail(h, GCE_ERR_INVALID, "NULL output array");
    if (j.kind == JOB_TOPK && (j.rho || j.mean || j.std_dev) && !(j.rho && j.mean && j.std_dev))
        return fail(h, GCE_ERR_INVALID, "significance needs all of mean, std and rho");
    if (j.kind == JOB_COUNTS && j.n_cells > 0 && (!j.cell_curve || !j.cell_trial || !j.counts))
        return fail(h, GCE_ERR_INVALID, "NULL cell array");
    if (j.bands && (j.n_bands < 1 || j.n_bands > GCE_MAX_BANDS))
        return fail(h, GCE_ERR_INVALID, "n_bands must be 1 .. %d", GCE_MAX_BANDS);
    CUDA_TRY(h, cudaSetDevice(h->device));
    {
        // arrays already checked by the previous call (same argument, same
        // pointer) need no new query
        const void *arrays[kCheckedArrays] = {j.times, j.mags, j.periods, j.pdots, j.out,
                                              j.topk_H, j.topk_idx, j.mean, j.std_dev, j.rho,
                                              j.cell_curve, j.cell_trial, j.counts, j.bands};
        for (int i = 0; i < kCheckedArrays; ++i) {
            if (arrays[i] && arrays[i] != h->checked[i] && !on_device(arrays[i], h->device)) {
                std::fill(h->checked, h->checked + kCheckedArrays, nullptr);
                return fail(h, GCE_ERR_INVALID, "an array is on another device than the handle's");
            }
            h->checked[i] = arrays[i];
        }
    }

    Plan pl;
    gce_status st = make_plan(h, j, pl);
    if (st != GCE_OK) return st;
    const int mode = j.cfg->phase_mode;

    // workspace
    if ((st = ensure(h, h->payload, (size_t)point_bytes(mode) * pl.n_points)) != GCE_OK) return st;
    if ((st = ensure(h, h->seg, sizeof(int) * (size_t)j.n_curves * (j.cfg->n_mag_bins + 1))) != GCE_OK) return st;
    if ((st = ensure(h, h->trialc, trial_bytes(mode) * (size_t)pl.n_trials)) != GCE_OK) return st;
    if ((st = ensure(h, h->order, sizeof(int) * (size_t)j.n_curves)) != GCE_OK) return st;
    if ((st = ensure(h, h->offsets, sizeof(long long) * (size_t)(j.n_curves + 1))) != GCE_OK) return st;
    if (j.bands &&
        (st = ensure(h, h->band_stats, sizeof(double2) * (size_t)j.n_curves * j.n_bands)) != GCE_OK)
        return st;
    if (j.kind == JOB_TOPK &&
        (st = ensure(h, h->cand, 8 * (size_t)j.n_curves * pl.n_lists * j.k)) != GCE_OK)
        return st;
    if (j.kind == JOB_TOPK && j.rho &&
        (st = ensure(h, h->stats, sizeof(TileStats) * (size_t)j.n_curves * pl.n_lists)) != GCE_OK)
        return st;
    if (j.kind == JOB_TOPK && pl.n_groups > 0 &&
        (st = ensure(h, h->cand2, 8 * (size_t)j.n_curves * pl.n_groups * j.k)) != GCE_OK)
        return st;
    if (j.kind == JOB_TOPK && pl.n_groups > 0 && j.rho &&
        (st = ensure(h, h->stats2, sizeof(TileStats) * (size_t)j.n_curves * pl.n_groups)) != GCE_OK)
        return st;
    if (pl.n_max > h->table_n) {
        if ((st = ensure(h, h->table, 8 * (size_t)(pl.n_max + 1))) != GCE_OK) return st;
        CUDA_TRY(h, launch_table((unsigned long long *)h->table.p, pl.n_max, s));
        ++h->launches;
        h->table_n = pl.n_max;
    }

    // host staging (pinned): offsets and the longest-first curve order
    if (h->staged_pending) {
        CUDA_TRY(h, cudaEventSynchronize(h->staged));
        h->staged_pending = false;
    }
    if ((size_t)j.n_curves + 1 > h->h_cap) {
        if (h->h_order) cudaFreeHost(h->h_order);
        if (h->h_offsets) cudaFreeHost(h->h_offsets);
        h->h_order = nullptr;
        h->h_offsets = nullptr;
        h->h_cap = 0;
        size_t cap = (size_t)j.n_curves + 1;
        CUDA_TRY(h, cudaMallocHost((void **)&h->h_order, sizeof(int) * cap));
        CUDA_TRY(h, cudaMallocHost((void **)&h->h_offsets, sizeof(long long) * cap));
        h->h_cap = cap;
    }
    std::memcpy(h->h_offsets, j.h_offsets, sizeof(long long) * (j.n_curves + 1));
    std::iota(h->h_order, h->h_order + j.n_curves, 0);
    std::stable_sort(h->h_order, h->h_order + j.n_curves, [&](int a, int b) {
        return j.h_offsets[a + 1] - j.h_offsets[a] > j.h_offsets[b + 1] - j.h_offsets[b];
    });

    const bool use_graph = !(j.cfg->flags & GCE_FLAG_NO_GRAPH) && s != nullptr &&
                           j.kind != JOB_SINGLE;
    h->timed = (j.cfg->flags & GCE_FLAG_TIME_KERNEL) != 0 && j.kind != JOB_COUNTS;
    if (!use_graph) {
        st = enqueue(h, j, pl, s, false);
        if (st != GCE_OK) return st;
    } else {
        GraphKey key{j.kind * 8 + (j.bands ? 4 : 0) + (j.rho ? 2 : 0) +
                         ((j.cfg->flags & GCE_FLAG_OVERLAP) ? 1 : 0),
                     mode, j.n_curves, j.n_periods, j.n_pdots, j.cfg->n_phase_bins,
                     j.cfg->n_mag_bins, j.k, pl.block, pl.tpt, pl.grid, pl.chunk, pl.table_smem,
                     pl.grab, pl.n_points};
        Fingerprint fp;
        const void *ptrs[] = {j.times, j.mags, j.periods, j.pdots, j.out, j.topk_H, j.topk_idx,
                              j.mean, j.std_dev, j.rho, j.cell_curve, j.cell_trial, j.counts,
                              j.bands, h->payload.p, h->seg.p, h->trialc.p, h->order.p,
                              h->offsets.p, h->cand.p, h->stats.p, h->cand2.p, h->stats2.p,
                              h->table.p, h->state.p, h->band_stats.p, h->h_order, h->h_offsets};
        for (const void *p : ptrs) fp.add(p);
        unsigned long long t0_bits;
        std::memcpy(&t0_bits, &j.cfg->t0, sizeof(t0_bits));
        fp.add_u(t0_bits);
        fp.add_u(j.cfg->flags);
        fp.add_u((unsigned long long)j.n_bands);
        fp.add_u((unsigned long long)j.n_cells);
        fp.add_u((unsigned long long)pl.n_long);
        auto it = h->graphs.find(key);
        if (it != h->graphs.end() && it->second.fp == fp) {
            // same shape and the same arrays as the cached graph: replay it as it is
            h->launches += it->second.launches;
        } else {
            const int before = h->launches;
            cudaGraph_t graph = nullptr;
            CUDA_TRY(h, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
            st = enqueue(h, j, pl, s, true);
            cudaError_t e = cudaStreamEndCapture(s, &graph);
            if (st != GCE_OK) {
                if (graph) cudaGraphDestroy(graph);
                return st;
            }
            if (e != cudaSuccess) return fail(h, GCE_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
            bool ready = false;
            if (it != h->graphs.end()) {
                // same shape, other arrays: update the cached graph's parameters
                cudaGraphExecUpdateResultInfo info;
                if (cudaGraphExecUpdate(it->second.exec, graph, &info) == cudaSuccess) {
                    ready = true;
                } else {
                    cudaGetLastError();
                    cudaGraphExecDestroy(it->second.exec);
                    h->graphs.erase(it);
                }
            }
            if (!ready) {
                cudaGraphExec_t exec = nullptr;
                e = cudaGraphInstantiate(&exec, graph, 0);
                if (e != cudaSuccess) {
                    cudaGraphDestroy(graph);
                    return fail(h, GCE_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
                }
                if (h->graphs.size() > 64) {
                    for (auto &kv : h->graphs) cudaGraphExecDestroy(kv.second.exec);
                    h->graphs.clear();
                }
                h->graphs[key].exec = exec;
            }
            cudaGraphDestroy(graph);
            CachedGraph &cg = h->graphs[key];
            cg.fp = fp;
            cg.launches = h->launches - before;
        }
        CUDA_TRY(h, cudaGraphLaunch(h->graphs[key].exec, s));
    }
    CUDA_TRY(h, cudaEventRecord(h->staged, s));
    h->staged_pending = true;
    return GCE_OK;
}

gce_status state_status(gce_handle h) {
    const unsigned int e = h->h_state->err;
    if (e & (ERR_TIME | ERR_PERIOD | ERR_PDOT | ERR_BAND))
        return fail(h, GCE_ERR_INVALID, "device check: %s%s%s%s",
                    (e & ERR_TIME) ? "non-finite time or magnitude; " : "",
                    (e & ERR_PERIOD) ? "non-finite or non-positive period; " : "",
                    (e & ERR_PDOT) ? "non-finite period derivative; " : "",
                    (e & ERR_BAND) ? "filter index >= n_bands; " : "");
    if (e & ERR_RANGE)
        return fail(h, GCE_ERR_UNSUPPORTED, "device check: trial range beyond the phase fold's range");
    if (e & ERR_SLOT)
        return fail(h, GCE_ERR_CUDA, "checked build: a counter slot outside the kept range");
    return GCE_OK;
}

}  // namespace

extern "C" gce_status gce_ce_grid(gce_handle h, const double *times, const double *mags,
                                  const int64_t *h_offsets, int32_t n_curves,
                                  const double *periods, int32_t n_periods, const double *pdots,
                                  int32_t n_pdots, const gce_config *cfg, float *out,
                                  void *stream) {
    Job j{};
    j.kind = JOB_GRID;
    j.times = times; j.mags = mags; j.h_offsets = h_offsets; j.n_curves = n_curves;
    j.periods = periods; j.n_periods = n_periods; j.pdots = pdots; j.n_pdots = n_pdots;
    j.cfg = cfg; j.out = out;
    return run_job(h, j, (cudaStream_t)stream);
}

extern "C" gce_status gce_ce_topk(gce_handle h, const double *times, const double *mags,
                                  const int64_t *h_offsets, int32_t n_curves,
                                  const double *periods, int32_t n_periods, const double *pdots,
                                  int32_t n_pdots, const gce_config *cfg, int32_t k,
                                  float *topk_H, int64_t *topk_idx, void *stream) {
    Job j{};
    j.kind = JOB_TOPK;
    j.times = times; j.mags = mags; j.h_offsets = h_offsets; j.n_curves = n_curves;
    j.periods = periods; j.n_periods = n_periods; j.pdots = pdots; j.n_pdots = n_pdots;
    j.cfg = cfg; j.k = k; j.topk_H = topk_H; j.topk_idx = topk_idx;
    return run_job(h, j, (cudaStream_t)stream);
}

extern "C" gce_status gce_ce_detect(gce_handle h, const double *times, const double *mags,
                                    const int64_t *h_offsets, int32_t n_curves,
                                    const double *periods, int32_t n_periods,
                                    const double *pdots, int32_t n_pdots, const gce_config *cfg,
                                    int32_t k, float *topk_H, int64_t *topk_idx, double *mean,
                                    double *std_dev, float *rho, void *stream) {
    if (!mean || !std_dev || !rho) return h ? fail(h, GCE_ERR_INVALID, "NULL moment output") : GCE_ERR_INVALID;
    Job j{};
    j.kind = JOB_TOPK;
    j.times = times; j.mags = mags; j.h_offsets = h_offsets; j.n_curves = n_curves;
    j.periods = periods; j.n_periods = n_periods; j.pdots = pdots; j.n_pdots = n_pdots;
    j.cfg = cfg; j.k = k; j.topk_H = topk_H; j.topk_idx = topk_idx;
    j.mean = mean; j.std_dev = std_dev; j.rho = rho;
    return run_job(h, j, (cudaStream_t)stream);
}

extern "C" gce_status gce_ce_grid_bands(gce_handle h, const double *times, const double *mags,
                                        const uint8_t *bands, int32_t n_bands,
                                        const int64_t *h_offsets, int32_t n_curves,
                                        const double *periods, int32_t n_periods,
                                        const double *pdots, int32_t n_pdots,
                                        const gce_config *cfg, float *out, void *stream) {
    if (!bands) return h ? fail(h, GCE_ERR_INVALID, "NULL band array") : GCE_ERR_INVALID;
    Job j{};
    j.kind = JOB_GRID;
    j.times = times; j.mags = mags; j.h_offsets = h_offsets; j.n_curves = n_curves;
    j.periods = periods; j.n_periods = n_periods; j.pdots = pdots; j.n_pdots = n_pdots;
    j.cfg = cfg; j.out = out;
    j.bands = bands; j.n_bands = n_bands;
    return run_job(h, j, (cudaStream_t)stream);
}

extern "C" gce_status gce_ce_detect_bands(gce_handle h, const double *times, const double *mags,
                                          const uint8_t *bands, int32_t n_bands,
                                          const int64_t *h_offsets, int32_t n_curves,
                                          const double *periods, int32_t n_periods,
                                          const double *pdots, int32_t n_pdots,
                                          const gce_config *cfg, int32_t k, float *topk_H,
                                          int64_t *topk_idx, double *mean, double *std_dev,
                                          float *rho, void *stream) {
    if (!bands) return h ? fail(h, GCE_ERR_INVALID, "NULL band array") : GCE_ERR_INVALID;
    Job j{};
    j.kind = JOB_TOPK;
    j.times = times; j.mags = mags; j.h_offsets = h_offsets; j.n_curves = n_curves;
    j.periods = periods; j.n_periods = n_periods; j.pdots = pdots; j.n_pdots = n_pdots;
    j.cfg = cfg; j.k = k; j.topk_H = topk_H; j.topk_idx = topk_idx;
    j.mean = mean; j.std_dev = std_dev; j.rho = rho;
    j.bands = bands; j.n_bands = n_bands;
    return run_job(h, j, (cudaStream_t)stream);
}

extern "C" gce_status gce_ce_grid_single(gce_handle h, const double *times, const double *mags,
                                         const int64_t *h_offsets, int32_t n_curves,
                                         const double *periods, int32_t n_periods,
                                         const double *pdots, int32_t n_pdots,
                                         const gce_config *cfg, float *out, void *stream) {
    Job j{};
    j.kind = JOB_SINGLE;
    j.times = times; j.mags = mags; j.h_offsets = h_offsets; j.n_curves = n_curves;
    j.periods = periods; j.n_periods = n_periods; j.pdots = pdots; j.n_pdots = n_pdots;
    j.cfg = cfg; j.out = out;
    return run_job(h, j, (cudaStream_t)stream);
}

extern "C" gce_status gce_ce_counts(gce_handle h, const double *times, const double *mags,
                                    const int64_t *h_offsets, int32_t n_curves,
                                    const double *periods, int32_t n_periods,
                                    const double *pdots, int32_t n_pdots, const gce_config *cfg,
                                    int64_t n_cells, const int64_t *cell_curve,
                                    const int64_t *cell_trial, uint32_t *counts, void *stream) {
    if (n_cells < 0) return GCE_ERR_INVALID;
    Job j{};
    j.kind = JOB_COUNTS;
    j.times = times; j.mags = mags; j.h_offsets = h_offsets; j.n_curves = n_curves;
    j.periods = periods; j.n_periods = n_periods; j.pdots = pdots; j.n_pdots = n_pdots;
    j.cfg = cfg; j.n_cells = n_cells; j.cell_curve = cell_curve; j.cell_trial = cell_trial;
    j.counts = counts;
    return run_job(h, j, (cudaStream_t)stream);
}

extern "C" gce_status gce_stream_status(gce_handle h, void *stream) {
    if (!h) return GCE_ERR_INVALID;
    CUDA_TRY(h, cudaSetDevice(h->device));
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(h, cudaMemcpyAsync(h->h_state, h->state.p, sizeof(JobState), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(h, cudaStreamSynchronize(s));
    return state_status(h);
}

extern "C" gce_status gce_ce_topk_host(gce_handle h, const double *h_times, const double *h_mags,
                                       const int64_t *h_offsets, int32_t n_curves,
                                       const double *h_periods, int32_t n_periods,
                                       const double *h_pdots, int32_t n_pdots,
                                       const gce_config *cfg, int32_t k, float *h_topk_H,
                                       int64_t *h_topk_idx, void *stream) {
    if (!h) return GCE_ERR_INVALID;
    gce_status st = gce_check_job(h_offsets, n_curves, n_periods, n_pdots, cfg, k);
    if (st != GCE_OK) return fail(h, st, "argument check failed");
    if (k < 1) return fail(h, GCE_ERR_INVALID, "k must be >= 1");
    if (n_curves == 0) return GCE_OK;
    if (!h_times || !h_mags || !h_periods || !h_pdots || !h_topk_H || !h_topk_idx)
        return fail(h, GCE_ERR_INVALID, "NULL host array");
    CUDA_TRY(h, cudaSetDevice(h->device));
    cudaStream_t s = (cudaStream_t)stream;
    const size_t np = (size_t)h_offsets[n_curves];
    if ((st = ensure(h, h->in_times, 8 * np)) != GCE_OK) return st;
    if ((st = ensure(h, h->in_mags, 8 * np)) != GCE_OK) return st;
    if ((st = ensure(h, h->in_periods, 8 * (size_t)n_periods)) != GCE_OK) return st;
    if ((st = ensure(h, h->in_pdots, 8 * (size_t)n_pdots)) != GCE_OK) return st;
    if ((st = ensure(h, h->out_H, 4 * (size_t)n_curves * k)) != GCE_OK) return st;
    if ((st = ensure(h, h->out_idx, 8 * (size_t)n_curves * k)) != GCE_OK) return st;
    CUDA_TRY(h, cudaMemcpyAsync(h->in_times.p, h_times, 8 * np, cudaMemcpyHostToDevice, s));
    CUDA_TRY(h, cudaMemcpyAsync(h->in_mags.p, h_mags, 8 * np, cudaMemcpyHostToDevice, s));
    CUDA_TRY(h, cudaMemcpyAsync(h->in_periods.p, h_periods, 8 * (size_t)n_periods,
                                cudaMemcpyHostToDevice, s));
    CUDA_TRY(h, cudaMemcpyAsync(h->in_pdots.p, h_pdots, 8 * (size_t)n_pdots,
                                cudaMemcpyHostToDevice, s));
    st = gce_ce_topk(h, (const double *)h->in_times.p, (const double *)h->in_mags.p, h_offsets,
                     n_curves, (const double *)h->in_periods.p, n_periods,
                     (const double *)h->in_pdots.p, n_pdots, cfg, k, (float *)h->out_H.p,
                     (int64_t *)h->out_idx.p, stream);
    if (st != GCE_OK) return st;
    CUDA_TRY(h, cudaMemcpyAsync(h_topk_H, h->out_H.p, 4 * (size_t)n_curves * k,
                                cudaMemcpyDeviceToHost, s));
    CUDA_TRY(h, cudaMemcpyAsync(h_topk_idx, h->out_idx.p, 8 * (size_t)n_curves * k,
                                cudaMemcpyDeviceToHost, s));
    return gce_stream_status(h, stream);
}

extern "C" gce_status gce_kernel_time(gce_handle h, float *ms) {
    if (!h || !ms) return GCE_ERR_INVALID;
    if (!h->timed) return fail(h, GCE_ERR_INVALID, "the last call was not made with GCE_FLAG_TIME_KERNEL");
    CUDA_TRY(h, cudaEventSynchronize(h->k1));
    CUDA_TRY(h, cudaEventElapsedTime(ms, h->k0, h->k1));
    return GCE_OK;
}

extern "C" gce_status gce_last_launches(gce_handle h, int32_t *n) {
    if (!h || !n) return GCE_ERR_INVALID;
    *n = h->launches;
    return GCE_OK;
}

// ------------------------------------------------------------------ tuning

extern "C" gce_status gce_get_tuning(gce_handle h, const gce_config *cfg, int32_t n_obs_hint,
                                     int32_t n_pdots_hint, gce_tuning *t) {
    if (!h || !cfg || !t || n_pdots_hint < 1) return GCE_ERR_INVALID;
    *t = lookup_tuning(h, cfg, std::max(1, n_obs_hint), n_pdots_hint > 1 ? 1 : 0);
    return GCE_OK;
}

extern "C" gce_status gce_set_tuning(gce_handle h, const gce_config *cfg, int32_t n_obs_hint,
                                     const gce_tuning *t) {
    if (!h || !cfg || !t || !tuning_ok(*t, cfg->phase_mode)) return GCE_ERR_INVALID;
    h->tune[tune_key(cfg, std::max(1, n_obs_hint), 0)] = *t;
    h->tune[tune_key(cfg, std::max(1, n_obs_hint), 1)] = *t;
    return GCE_OK;
}

// Candidate launch shapes of the autotuners (slot_range: the kept SPLIT32 slot
// range of every candidate).
static std::vector<gce_tuning> tune_candidates(int mode, int n_obs, int slot_range = 0) {
    const int blocks[] = {128, 256, 512};
    const int tpts[] = {1, 2, 4};
    const int chunks[] = {256, 512, 1024, 2048};
    std::vector<gce_tuning> cands;
    for (int b : blocks)
        for (int tp : tpts)
            for (int ch : chunks) {
                if (ch > 512 && ch >= 2 * n_obs) continue;  // same plan as a smaller chunk
                if (tp == 4 && mode == GCE_PHASE_FP64) continue;  // not built
                gce_tuning c = default_tuning(mode, n_obs);
                c.block = b;
                c.tpt = tp;
                c.chunk = ch;
                c.slot_range = slot_range;
                cands.push_back(c);
            }
    return cands;
}

// Times every candidate on job j (one untimed run, then three timed ones), then
// times the three fastest again over six runs each and leaves the fastest of
// those in *best (a second look keeps close calls from being decided by one
// noisy measurement); shapes that do not fit are skipped.  also_wide: each of
// the three is timed with the wide slot range too (the candidates keep the mid
// one, whose re-reduced warps can make it the slower on long baselines).
static gce_status time_candidates(gce_handle h, Job j, const std::vector<gce_tuning> &cands,
                                  cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1,
                                  gce_tuning *best, bool also_wide = false) {
    auto timed = [&](const gce_tuning &cand, int reps, float *ms) -> gce_status {
        j.force = &cand;
        *ms = 1e30f;
        if (run_job(h, j, s) != GCE_OK) return GCE_OK;  // does not fit: stays 1e30
        cudaEventRecord(e0, s);
        for (int rep = 0; rep < reps; ++rep) run_job(h, j, s);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess)
            return fail(h, GCE_ERR_CUDA, "autotune: %s", cudaGetErrorString(cudaGetLastError()));
        cudaEventElapsedTime(ms, e0, e1);
        *ms /= (float)reps;
        return GCE_OK;
    };
    std::vector<std::pair<float, size_t>> first;
    for (size_t i = 0; i < cands.size(); ++i) {
        float ms;
        if (gce_status st = timed(cands[i], 3, &ms)) return st;
        if (ms < 1e30f) first.emplace_back(ms, i);
    }
    if (first.empty()) return GCE_OK;
    std::sort(first.begin(), first.end());
    float best_ms = 1e30f;
    for (size_t r = 0; r < std::min<size_t>(3, first.size()); ++r) {
        for (int w = 0; w < (also_wide ? 2 : 1); ++w) {
            gce_tuning c = cands[first[r].second];
            if (w) c.slot_range = 0;
            float ms;
            if (gce_status st = timed(c, 6, &ms)) return st;
            if (ms < best_ms) {
                best_ms = ms;
                *best = c;
            }
        }
    }
    return GCE_OK;
}

extern "C" gce_status gce_autotune_job(gce_handle h, const double *times, const double *mags,
                                       const int64_t *h_offsets, int32_t n_curves,
                                       const double *periods, int32_t n_periods,
                                       const double *pdots, int32_t n_pdots,
                                       const gce_config *cfg) {
    if (!h || !cfg) return GCE_ERR_INVALID;
    const gce_status chk = gce_check_job(h_offsets, n_curves, n_periods, n_pdots, cfg, 0);
    if (chk != GCE_OK) return fail(h, chk, "autotune: argument check failed");
    if (n_curves == 0) return GCE_OK;
    if (!times || !mags || !periods || !pdots) return fail(h, GCE_ERR_INVALID, "NULL input array");
    CUDA_TRY(h, cudaSetDevice(h->device));
    // the slice: up to 65536 periods and 8 Pdot values, each a strided subset that
    // spans the job's range, and a prefix of the curves with about 4e9 point-trials
    const int p_s = n_periods > 65536 ? (n_periods + 65535) / 65536 : 1;
    const int n_p2 = (n_periods + p_s - 1) / p_s;
    const int q_s = n_pdots > 8 ? (n_pdots + 7) / 8 : 1;
    const int n_q2 = (n_pdots + q_s - 1) / q_s;
    const long long trials = (long long)n_p2 * n_q2;
    int c2 = 0;
    long long pts = 0, nmax = 1;
    for (int c = 0; c < n_curves; ++c) nmax = std::max<long long>(nmax, h_offsets[c + 1] - h_offsets[c]);
    while (c2 < n_curves && pts * trials < 4000000000ll) {
        pts += h_offsets[c2 + 1] - h_offsets[c2];
        ++c2;
    }
    double *d_p = nullptr, *d_q = nullptr;
    float *d_H = nullptr;
    int64_t *d_I = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    gce_status result = GCE_OK;
    gce_tuning best = default_tuning(cfg->phase_mode, (int)nmax);
    gce_config c2cfg = *cfg;
    c2cfg.flags = (c2cfg.flags | GCE_FLAG_NO_GRAPH) & ~GCE_FLAG_TIME_KERNEL;
    do {
        if (cudaMalloc(&d_p, 8 * (size_t)n_p2) || cudaMalloc(&d_q, 8 * (size_t)n_q2) ||
            cudaMalloc(&d_H, 4 * (size_t)c2) || cudaMalloc(&d_I, 8 * (size_t)c2) ||
            cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) || cudaEventCreate(&e0) ||
            cudaEventCreate(&e1)) {
            result = fail(h, GCE_ERR_NOMEM, "autotune: allocation failed");
            break;
        }
        // strided copies: one element every p_s (q_s) of the caller's arrays
        if (cudaMemcpy2DAsync(d_p, 8, periods, 8 * (size_t)p_s, 8, n_p2, cudaMemcpyDeviceToDevice, s) ||
            cudaMemcpy2DAsync(d_q, 8, pdots, 8 * (size_t)q_s, 8, n_q2, cudaMemcpyDeviceToDevice, s)) {
            result = fail(h, GCE_ERR_CUDA, "autotune: %s", cudaGetErrorString(cudaGetLastError()));
            break;
        }
        Job j{};
        j.kind = JOB_TOPK;
        j.times = times; j.mags = mags; j.h_offsets = h_offsets; j.n_curves = c2;
        j.periods = d_p; j.n_periods = n_p2; j.pdots = d_q; j.n_pdots = n_q2;
        j.cfg = &c2cfg; j.k = 1; j.topk_H = d_H; j.topk_idx = d_I;
        // SPLIT32 without a Pdot axis: candidates with the mid slot range, the
        // finalists with the wide one as well
        const bool mid = cfg->phase_mode == GCE_PHASE_SPLIT32 && n_pdots == 1;
        result = time_candidates(h, j, tune_candidates(cfg->phase_mode, (int)nmax, mid ? 1 : 0), s,
                                 e0, e1, &best, mid);
    } while (0);
    if (s) cudaStreamSynchronize(s);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    cudaFree(d_p); cudaFree(d_q); cudaFree(d_H); cudaFree(d_I);
    if (result == GCE_OK) h->tune[tune_key(cfg, (int)nmax, n_pdots > 1 ? 1 : 0)] = best;
    return result;
}

extern "C" gce_status gce_autotune(gce_handle h, const gce_config *cfg, int32_t n_obs_hint,
                                   int64_t n_trials_hint) {
    if (!h || !cfg) return GCE_ERR_INVALID;
    const int n_obs = std::max(16, std::min<int>(n_obs_hint, GCE_MAX_CURVE_POINTS));
    const long long n_tr = std::max<long long>(4096, std::min<long long>(n_trials_hint, 1 << 22));
    // synthetic job of about 5e9 point-trials so that a candidate fills the GPU
    const int n_curves = (int)std::max<long long>(
        16, std::min<long long>(256, 5000000000ll / ((long long)n_obs * n_tr)));
    std::vector<int64_t> offs_v(n_curves + 1);
    for (int c = 0; c <= n_curves; ++c) offs_v[c] = (int64_t)c * n_obs;
    const int64_t *offs = offs_v.data();
    if (gce_check_job(offs, n_curves, (int32_t)n_tr, 1, cfg, 0) != GCE_OK)
        return fail(h, GCE_ERR_INVALID, "autotune: invalid config");
    CUDA_TRY(h, cudaSetDevice(h->device));
    // synthetic job: 3-year times, a square-ish signal, log-spaced periods
    const size_t np = (size_t)n_curves * n_obs;
    // the Pdot-axis pass: 8 Pdot values linear in [-1e-10, 0] over n_tr / 8 periods
    const int n_pd = 8;
    const long long n_trp = std::max<long long>(512, n_tr / n_pd);
    std::vector<double> t(np), m(np), per((size_t)n_tr), perp((size_t)n_trp), pd(n_pd);
    unsigned long long x = 0x9e3779b97f4a7c15ull;
    auto u01 = [&x]() {
        x ^= x << 13; x ^= x >> 7; x ^= x << 17;
        return (double)(x >> 11) * (1.0 / 9007199254740992.0);
    };
    for (size_t i = 0; i < np; ++i) {
        t[i] = u01() * 9.46e7;
        m[i] = 15.0 + (u01() < 0.1 ? 0.5 : 0.0) + 0.02 * u01();
    }
    for (long long p = 0; p < n_tr; ++p) per[p] = 300.0 * std::pow(288.0, (double)p / (double)(n_tr - 1));
    for (long long p = 0; p < n_trp; ++p)
        perp[p] = 300.0 * std::pow(288.0, (double)p / (double)(n_trp - 1));
    for (int q = 0; q < n_pd; ++q) pd[q] = -1e-10 * (double)q / (double)(n_pd - 1);
    double *d_t = nullptr, *d_m = nullptr, *d_p = nullptr, *d_pp = nullptr, *d_d = nullptr;
    float *d_out = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    gce_status result = GCE_OK;
    gce_tuning best[2] = {default_tuning(cfg->phase_mode, n_obs), default_tuning(cfg->phase_mode, n_obs)};
    gce_config c2 = *cfg;
    c2.flags |= GCE_FLAG_NO_GRAPH;
    do {
        if (cudaMalloc(&d_t, 8 * np) || cudaMalloc(&d_m, 8 * np) || cudaMalloc(&d_p, 8 * n_tr) ||
            cudaMalloc(&d_pp, 8 * n_trp) || cudaMalloc(&d_d, 8 * n_pd) ||
            cudaMalloc(&d_out, 4 * (size_t)n_curves * std::max(n_tr, n_trp * n_pd)) ||
            cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) || cudaEventCreate(&e0) ||
            cudaEventCreate(&e1)) {
            result = fail(h, GCE_ERR_NOMEM, "autotune: allocation failed");
            break;
        }
        cudaMemcpy(d_t, t.data(), 8 * np, cudaMemcpyHostToDevice);
        cudaMemcpy(d_m, m.data(), 8 * np, cudaMemcpyHostToDevice);
        cudaMemcpy(d_p, per.data(), 8 * n_tr, cudaMemcpyHostToDevice);
        cudaMemcpy(d_pp, perp.data(), 8 * n_trp, cudaMemcpyHostToDevice);
        cudaMemcpy(d_d, pd.data(), 8 * n_pd, cudaMemcpyHostToDevice);
        const std::vector<gce_tuning> cands = tune_candidates(cfg->phase_mode, n_obs);
        // pass 0: one Pdot value (pd[0] = 0); pass 1: the Pdot axis
        for (int pass = 0; pass < 2 && result == GCE_OK; ++pass) {
            Job j{};
            j.kind = JOB_GRID;
            j.times = d_t; j.mags = d_m; j.h_offsets = offs; j.n_curves = n_curves;
            if (pass == 0) {
                j.periods = d_p; j.n_periods = (int)n_tr; j.pdots = d_d; j.n_pdots = 1;
            } else {
                j.periods = d_pp; j.n_periods = (int)n_trp; j.pdots = d_d; j.n_pdots = n_pd;
            }
            j.cfg = &c2; j.out = d_out;
            result = time_candidates(h, j, cands, s, e0, e1, &best[pass]);
        }
    } while (0);
    if (s) cudaStreamSynchronize(s);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    cudaFree(d_t); cudaFree(d_m); cudaFree(d_p); cudaFree(d_pp); cudaFree(d_d); cudaFree(d_out);
    if (result == GCE_OK) {
        h->tune[tune_key(cfg, n_obs, 0)] = best[0];
        h->tune[tune_key(cfg, n_obs, 1)] = best[1];
    }
    return result;
}
