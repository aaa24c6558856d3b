// gce_ce_topk_static: the top-k search with every piece of device workspace
// taken from one fixed array compiled into the library, so the call itself
// allocates nothing.
//
// Who needs it: callers that must not call cudaMalloc, e.g. a process whose
// device memory is owned by another allocator (a framework's caching
// allocator or a pool that has reserved almost all of the GPU, where an outside
// cudaMalloc can fail or fragment that pool), or a latency-critical loop that
// cannot afford cudaMalloc's implicit device synchronisation.  They pass their
// own input and output buffers; the scratch comes from g_scratch.
//
// g_scratch is a file-scope __device__ array of kScratchBytes (32 MiB), so
// every GPU on which the library is loaded holds it until the process exits.
// The host never touches g_scratch by name: in host code that name is only a
// stand-in, not a device address.  Every call, with the caller's device current,
// asks the runtime for the array's device address (cudaGetSymbolAddress, a
// cheap lookup); the first call on a device, and any call that finds the
// address moved (after a device reset the module is loaded anew), fills the
// c ln c table held at the array's start (a few small synchronous CUDA calls),
// so the first call on a device should be made before any stream capture.
// Every call then passes that address to the kernels.
//
// Every call uses the same array, which keeps the previous call's contents.
// Each call rewrites all of it that it reads (the job state is cleared by
// k_init; trial constants, payload and candidates are fully written before
// they are read), so nothing depends on earlier contents.  Calls that overlap
// on the GPU (from two host threads, or two streams) race on the array: issue
// them one at a time.
//
// The call runs on the current device.  Every device array it is given must
// live on that device (checked with cudaPointerGetAttributes; memory of another
// device is GCE_ERR_INVALID).
#include <cstdint>
#include <cstring>
#include <mutex>

#include "gce_internal.cuh"

using namespace gce;

namespace {

constexpr size_t kScratchBytes = 32u << 20;  // 32 MiB
constexpr int kMaxDevices = 64;
constexpr size_t kTableEntries = GCE_MAX_CURVE_POINTS + 1;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct DeviceSetup {
    bool done = false;
    unsigned char *base = nullptr;  // device address of g_scratch
    int n_sm = 0;
    int smem_optin = 0;
};

std::mutex g_mutex;
DeviceSetup g_setup[kMaxDevices];

// Statuses only (this entry point has no handle to hold a message); the
// message documents each return.
inline gce_status fail(gce_status st, const char *) { return st; }

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Layout of one call inside g_scratch: the c ln c table first (filled once per
// device), then the per-call buffers.
struct Layout {
    size_t state, offsets, order, seg, trialc, payload, cand, end;
};

Layout layout(long long n_points, int n_curves, long long n_trials, int n_mag, int point_bytes,
              long long n_lists, int k) {
    Layout L;
    size_t o = align256(8 * kTableEntries);
    L.state = o;
    o = align256(o + sizeof(JobState));
    L.offsets = o;
    o = align256(o + 8 * (size_t)(n_curves + 1));
    L.order = o;
    o = align256(o + 4 * (size_t)n_curves);
    L.seg = o;
    o = align256(o + 4 * (size_t)n_curves * (n_mag + 1));
    L.trialc = o;
    o = align256(o + 32 * (size_t)n_trials);
    L.payload = o;
    o = align256(o + (size_t)point_bytes * (size_t)n_points);
    L.cand = o;
    o = align256(o + 8 * (size_t)n_curves * (size_t)n_lists * (size_t)k);
    L.end = o;
    return L;
}

__global__ void k_iota(int *order, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        order[i] = i;
}

gce_status setup(int dev, DeviceSetup *&out) {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (dev < 0 || dev >= kMaxDevices) return fail(GCE_ERR_UNSUPPORTED, "device index too large");
    DeviceSetup &d = g_setup[dev];
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return fail(GCE_ERR_CUDA, cudaGetErrorString(e));
    if (!d.done || d.base != static_cast<unsigned char *>(p)) {
        // first use on this device, or the module was loaded anew (the array moved
        // and its table is gone): fill the c ln c table again
        d.done = false;
        e = cudaDeviceGetAttribute(&d.n_sm, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return fail(GCE_ERR_CUDA, cudaGetErrorString(e));
        e = cudaDeviceGetAttribute(&d.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e != cudaSuccess) return fail(GCE_ERR_CUDA, cudaGetErrorString(e));
        e = launch_table(reinterpret_cast<unsigned long long *>(p), (int)kTableEntries - 1, 0);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return fail(GCE_ERR_CUDA, cudaGetErrorString(e));
        d.base = static_cast<unsigned char *>(p);
        d.done = true;
    }
    out = &d;
    return GCE_OK;
}

// A device array of the call must be on the current device: memory that the
// runtime reports as another device's is rejected (managed and host-registered
// memory is left to the driver).
bool on_device(const void *ptr, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return true;  // not a pointer the runtime knows: left to the kernels' own access
    }
    return a.type != cudaMemoryTypeDevice || a.device == dev;
}

}  // namespace

extern "C" gce_status gce_ce_topk_static(const double *times, const double *mags,
                                         const int64_t *h_offsets, int32_t n_curves,
                                         const double *periods, int32_t n_periods,
                                         const double *pdots, int32_t n_pdots,
                                         const gce_config *cfg, int32_t k, float *topk_H,
                                         int64_t *topk_idx, void *stream) {
    gce_status st = gce_check_job(h_offsets, n_curves, n_periods, n_pdots, cfg, k);
    if (st != GCE_OK) return fail(st, "argument check failed");
    if (k < 1) return fail(GCE_ERR_INVALID, "k must be >= 1");
    if (n_curves == 0) return GCE_OK;
    if (!times || !mags || !periods || !pdots || !topk_H || !topk_idx)
        return fail(GCE_ERR_INVALID, "NULL array");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(GCE_ERR_CUDA, cudaGetErrorString(e));
    DeviceSetup *d = nullptr;
    if ((st = setup(dev, d)) != GCE_OK) return st;
    const void *arrays[] = {times, mags, periods, pdots, topk_H, topk_idx};
    for (const void *a : arrays)
        if (!on_device(a, dev)) return fail(GCE_ERR_INVALID, "an array is on another device");
    cudaStream_t s = (cudaStream_t)stream;
    const int mode = cfg->phase_mode;

    // launch shape: block 256, 2 trials per thread, the curve staged in chunks
    long long n_max = 1;
    for (int c = 0; c < n_curves; ++c)
        n_max = h_offsets[c + 1] - h_offsets[c] > n_max ? h_offsets[c + 1] - h_offsets[c] : n_max;
    const long long n_points = h_offsets[n_curves];
    const long long n_trials = (long long)n_periods * n_pdots;
    const int block = 256, tpt = 2;
    int chunk = (int)((n_max + 31) / 32 * 32);
    if (chunk > 1024) chunk = 1024;
    int table_smem = (int)(n_max + 1 < 1024 ? n_max + 1 : 1024);
    const int range = (mode == GCE_PHASE_SPLIT32 && n_pdots > 1) ? RANGE_NARROW : RANGE_WIDE;
    const int half = (mode != GCE_PHASE_FP64 && n_pdots == 1) ? 1 : 0;
    const size_t smem = main_smem_bytes(mode, block, tpt, chunk, cfg->n_phase_bins,
                                        cfg->n_mag_bins, table_smem, range, half);
    const int kv = kernel_variant((cfg->flags & GCE_FLAG_OVERLAP) != 0);
    if (smem > main_dynamic_smem_limit(mode, tpt, block, kv, (size_t)d->smem_optin))
        return fail(GCE_ERR_UNSUPPORTED, "bin counts too large for this entry point");
    const TileGrid tg = tile_grid(n_periods, n_pdots, block, tpt);
    const long long n_tiles = tg.n_tiles;
    const int point_bytes = mode == GCE_PHASE_FP64 ? 8 : 16;
    const long long n_lists = n_tiles * (block / 32);  // one candidate list per warp and tile
    const Layout L = layout(n_points, n_curves, n_trials, cfg->n_mag_bins, point_bytes, n_lists, k);
    if (L.end > kScratchBytes)
        return fail(GCE_ERR_NOMEM, "job needs more than the 32 MiB of built-in scratch");

    e = main_kernel_attrs(mode, tpt, block, kv, (size_t)d->smem_optin);
    if (e != cudaSuccess) return fail(GCE_ERR_CUDA, cudaGetErrorString(e));
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, main_kernel_ptr(mode, tpt, block, kv), block, smem);
    if (e != cudaSuccess || occ < 1) return fail(GCE_ERR_CUDA, "occupancy query failed");
    const long long n_items = (long long)n_curves * n_tiles;
    long long grid = (long long)d->n_sm * occ;
    if (grid > n_items) grid = n_items;

    unsigned char *b = d->base;
    JobState *state = reinterpret_cast<JobState *>(b + L.state);
    long long *offsets = reinterpret_cast<long long *>(b + L.offsets);
    int *order = reinterpret_cast<int *>(b + L.order);
    // offsets from the caller's host array (pageable: the copy is staged by the driver)
    e = cudaMemcpyAsync(offsets, h_offsets, 8 * (size_t)(n_curves + 1), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return fail(GCE_ERR_CUDA, cudaGetErrorString(e));
    k_iota<<<(n_curves + 255) / 256 < 1024 ? (n_curves + 255) / 256 : 1024, 256, 0, s>>>(order, n_curves);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(GCE_ERR_CUDA, cudaGetErrorString(e));
    if ((e = launch_init(state, s)) != cudaSuccess) return fail(GCE_ERR_CUDA, cudaGetErrorString(e));
    e = launch_scan(times, mags, n_points, periods, n_periods, pdots, n_pdots, cfg->t0, state, s);
    if (e != cudaSuccess) return fail(GCE_ERR_CUDA, cudaGetErrorString(e));
    TrialArgs ta;
    ta.periods = periods;
    ta.pdots = pdots;
    ta.n_periods = n_periods;
    ta.n_pdots = n_pdots;
    ta.trialc = b + L.trialc;
    ta.state = state;
    if ((e = launch_trials(mode, ta, s)) != cudaSuccess) return fail(GCE_ERR_CUDA, cudaGetErrorString(e));
    PrepArgs pa;
    pa.times = times;
    pa.mags = mags;
    pa.offsets = offsets;
    pa.n_curves = n_curves;
    pa.n_mag = cfg->n_mag_bins;
    pa.t0 = cfg->t0;
    pa.payload = b + L.payload;
    pa.seg = reinterpret_cast<int *>(b + L.seg);
    pa.state = state;
    pa.bands = nullptr;
    pa.band_stats = nullptr;
    pa.n_bands = 0;
    if ((e = launch_prep(mode, pa, s)) != cudaSuccess) return fail(GCE_ERR_CUDA, cudaGetErrorString(e));
    MainArgs ma;
    ma.payload = b + L.payload;
    ma.offsets = offsets;
    ma.seg = reinterpret_cast<const int *>(b + L.seg);
    ma.trialc = b + L.trialc;
    ma.order = order;
    ma.table = reinterpret_cast<const unsigned long long *>(b);
    ma.n_trials = n_trials;
    ma.n_periods = n_periods;
    ma.n_pdots = n_pdots;
    ma.n_tiles = (int)n_tiles;
    ma.n_ptiles = tg.n_ptiles;
    ma.pd_major = tg.pd_major;
    ma.range = range;
    ma.n_items = n_items;
    ma.n_long_items = n_items;  // every curve curve-major
    ma.n_long = n_curves;
    ma.n_short = 0;
    ma.grab = 1;
    ma.n_phase = cfg->n_phase_bins;
    ma.n_mag = cfg->n_mag_bins;
    ma.chunk = chunk;
    ma.table_smem = table_smem;
    ma.out = nullptr;
    ma.cand = reinterpret_cast<unsigned long long *>(b + L.cand);
    ma.k = k;
    ma.stats = nullptr;
    ma.overlap = (cfg->flags & GCE_FLAG_OVERLAP) ? 1 : 0;
    ma.half = half;
    ma.kv = kv;
    ma.state = state;
    if ((e = launch_main(mode, tpt, block, (int)grid, smem, ma, s)) != cudaSuccess)
        return fail(GCE_ERR_CUDA, cudaGetErrorString(e));
    e = launch_topk_merge(ma.cand, n_curves, (int)n_lists, k, topk_H, (long long *)topk_idx,
                          nullptr, nullptr, nullptr, nullptr, state, s);
    if (e != cudaSuccess) return fail(GCE_ERR_CUDA, cudaGetErrorString(e));
    // device-side input checks: read the flags into host stack memory and wait
    unsigned int err = 0;
    e = cudaMemcpyAsync(&err, &state->err, sizeof(err), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(GCE_ERR_CUDA, cudaGetErrorString(e));
    if (err & (ERR_TIME | ERR_PERIOD | ERR_PDOT))
        return fail(GCE_ERR_INVALID, "device check: non-finite or non-positive input values");
    if (err & ERR_RANGE) return fail(GCE_ERR_UNSUPPORTED, "device check: trial range beyond the fold");
    if (err & ERR_SLOT) return fail(GCE_ERR_CUDA, "checked build: a counter slot outside the kept range");
    return GCE_OK;
}
