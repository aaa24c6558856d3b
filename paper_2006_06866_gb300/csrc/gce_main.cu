// The kernels around the CE kernel: per-curve top-k merge (and the Eq. 5
// moments), the plain one-launch-per-curve FP64 baseline, diagnostic counts,
// and the dispatch of the CE kernel's instantiations (one translation unit per
// fold mode and trials per thread: gce_main_<mode>_t<tpt>.cu).
#include "gce_kernel.cuh"

namespace gce {

namespace {

// Per-curve merge of the tiles' candidates: k rounds of "smallest key above the
// previous one" (keys are unique: H bits in the high word, trial index low).
__global__ void k_topk_merge(const unsigned long long *__restrict__ cand, int n_tiles, int k,
                             float *topk_H, long long *topk_idx, const TileStats *stats,
                             double *mean_out, double *std_out, float *rho_out, const JobState *st) {
    __shared__ unsigned long long sh[32];
    __shared__ double shs[3 * 32];
    if (st->err) return;
    const int c = blockIdx.x;
    const long long n = (long long)n_tiles * k;
    const unsigned long long *src = cand + (long long)c * n;
    unsigned long long last = 0ull;
    for (int r = 0; r < k; ++r) {
        unsigned long long mine = kNoKey;
        for (long long i = threadIdx.x; i < n; i += blockDim.x) {
            const unsigned long long v = src[i];
            if ((r == 0 || v > last) && v < mine) mine = v;
        }
        mine = warp_min_key(mine);
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = mine;
        __syncthreads();
        if (threadIdx.x < 32) {
            unsigned long long v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : kNoKey;
            v = warp_min_key(v);
            if (threadIdx.x == 0) sh[0] = v;
        }
        __syncthreads();
        last = sh[0];
        __syncthreads();
        if (threadIdx.x == 0) {
            topk_H[(long long)c * k + r] = __uint_as_float((unsigned int)(last >> 32));
            topk_idx[(long long)c * k + r] = (long long)(last & 0xffffffffull);
        }
    }
    if (!stats) return;
    // Eq. 5: rho = (mu - H_min) / sigma over the curve's whole grid, the tiles'
    // moments merged in a fixed order (each thread a strided run of tiles, then
    // a fixed tree), so the result is deterministic
    double nn = 0.0, mu = 0.0, m2 = 0.0;
    const TileStats *ts = stats + (long long)c * n_tiles;
    for (int i = threadIdx.x; i < n_tiles; i += blockDim.x) chan_merge(nn, mu, m2, ts[i].n, ts[i].mean, ts[i].m2);
    for (int o = 1; o < 32; o <<= 1) {
        const double nb = __shfl_down_sync(0xffffffffu, nn, o);
        const double mb = __shfl_down_sync(0xffffffffu, mu, o);
        const double qb = __shfl_down_sync(0xffffffffu, m2, o);
        if ((threadIdx.x & (2 * o - 1)) == 0) chan_merge(nn, mu, m2, nb, mb, qb);
    }
    if ((threadIdx.x & 31) == 0) {
        shs[3 * (threadIdx.x >> 5)] = nn;
        shs[3 * (threadIdx.x >> 5) + 1] = mu;
        shs[3 * (threadIdx.x >> 5) + 2] = m2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        nn = 0.0;
        mu = 0.0;
        m2 = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) chan_merge(nn, mu, m2, shs[3 * w], shs[3 * w + 1], shs[3 * w + 2]);
        const double sd = nn > 0.0 ? sqrt(m2 / nn) : 0.0;
        mean_out[c] = mu;
        std_out[c] = sd;
        // H_min is the first of the top-k this thread wrote above
        rho_out[c] = sd > 0.0 ? (float)((mu - (double)topk_H[(long long)c * k]) / sd) : 0.0f;
    }
}

// The plain baseline: one launch per curve, one thread per trial, the FP64
// fold, points read straight from global memory.
__global__ void __launch_bounds__(256) k_single(MainArgs a, int c) {
    extern __shared__ __align__(16) unsigned char smem[];
    if (a.state->err) return;
    const int B = blockDim.x, tid = threadIdx.x;
    const int n_phase = a.n_phase, n_mag = a.n_mag;
    unsigned int *cnt = reinterpret_cast<unsigned int *>(smem) + tid;
    const long long t = (long long)blockIdx.x * B + tid;
    const bool valid = t < a.n_trials;
    const double2 tr = valid ? reinterpret_cast<const double2 *>(a.trialc)[t] : double2{0.0, 0.0};
    const double *pts = reinterpret_cast<const double *>(a.payload) + a.offsets[c];
    const int *seg = a.seg + (long long)c * (n_mag + 1);
    const int n = (int)(a.offsets[c + 1] - a.offsets[c]);
    for (int j = 0; j < n_phase; ++j) cnt[j * B] = 0u;
    unsigned long long s_ij = 0ull;
    for (int i = 0; i < n_mag; ++i) {
        const int s0 = seg[i], s1 = seg[i + 1];
        if (s1 == s0) continue;
        for (int k = s0; k < s1; ++k) {
            const int j = fold_fp64<true>(__ldg(pts + k), tr.x, tr.y, (double)n_phase, n_phase);
            atomicAdd(cnt + j * B, 1u);
            if (a.overlap) atomicAdd(cnt + (j == 0 ? n_phase - 1 : j - 1) * B, 1u);
        }
        for (int j = 0; j < n_phase; ++j) s_ij += __ldg(a.table + take_segment(cnt + j * B));
    }
    unsigned long long sj = 0ull;
    for (int j = 0; j < n_phase; ++j) sj += __ldg(a.table + (cnt[j * B] & 0xffffu));
    long long d = (long long)(sj - s_ij);
    if (d < 0) d = 0;
    if (valid)
        a.out[(long long)c * a.n_trials + t] = __double2float_rn(
            __dmul_rn(__ll2double_rn(d), kTabInvScale / (double)(n * (a.overlap ? 2 : 1))));
}

// Diagnostic: full 2-D counts of selected cells through the same fold code.
template <int MODE>
__global__ void k_counts(MainArgs a, long long n_cells, const long long *cell_curve,
                         const long long *cell_trial, unsigned int *counts) {
    typedef typename ModeTraits<MODE>::point_t point_t;
    typedef typename ModeTraits<MODE>::trial_t trial_t;
    if (a.state->err) return;
    const long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= n_cells) return;
    const long long c = cell_curve[cell], t = cell_trial[cell];
    const trial_t tr0 = reinterpret_cast<const trial_t *>(a.trialc)[t];
    const typename Fold<MODE>::prep_t tr = Fold<MODE>::prepare(tr0);
    const point_t *pts = reinterpret_cast<const point_t *>(a.payload) + a.offsets[c];
    const int *seg = a.seg + c * (a.n_mag + 1);
    unsigned int *out = counts + cell * a.n_mag * a.n_phase;
    const bool pdot = Fold<MODE>::has_pdot(tr0);
    const FoldConst fk = fold_const(a.n_phase);
    for (int i = 0; i < a.n_mag; ++i) {
        for (int k = seg[i]; k < seg[i + 1]; ++k) {
            int j = (pdot ? Fold<MODE>::template raw_slot<true>(pts[k], tr, fk)
                          : Fold<MODE>::template raw_slot<false>(pts[k], tr, fk)) -
                    Fold<MODE>::kSlotBias;
            if (j >= a.n_phase) j -= a.n_phase;  // SPLIT32's second slot of a bin
            out[i * a.n_phase + j] += 1u;
            if (a.overlap) out[i * a.n_phase + (j == 0 ? a.n_phase - 1 : j - 1)] += 1u;
        }
    }
}

}  // namespace

size_t main_smem_bytes(int mode, int block, int tpt, int chunk, int n_phase, int n_mag,
                       int table_smem, int range, int half) {
    return main_smem_layout(mode, block, tpt, chunk, n_phase, n_mag, table_smem, range, half).total;
}

size_t single_smem_bytes(int n_phase, int block) { return 4 * (size_t)n_phase * block; }

const void *main_kernel_ptr(int mode, int tpt, int block, int kv) {
    switch (mode * 8 + tpt) {
        case GCE_PHASE_FP64 * 8 + 1: return main_kernel_ptr_fp64_t1(block, kv);
        case GCE_PHASE_FP64 * 8 + 2: return main_kernel_ptr_fp64_t2(block, kv);
        case GCE_PHASE_SPLIT32 * 8 + 1: return main_kernel_ptr_split32_t1(block, kv);
        case GCE_PHASE_SPLIT32 * 8 + 2: return main_kernel_ptr_split32_t2(block, kv);
        case GCE_PHASE_SPLIT32 * 8 + 4: return main_kernel_ptr_split32_t4(block, kv);
        case GCE_PHASE_FIXED32 * 8 + 1: return main_kernel_ptr_fixed32_t1(block, kv);
        case GCE_PHASE_FIXED32 * 8 + 2: return main_kernel_ptr_fixed32_t2(block, kv);
        case GCE_PHASE_FIXED32 * 8 + 4: return main_kernel_ptr_fixed32_t4(block, kv);
        default: return nullptr;
    }
}

// The dynamic shared memory a CTA of the kernel can have: the device's opt-in
// maximum less the kernel's static shared memory (0 if the kernel is unknown).
size_t main_dynamic_smem_limit(int mode, int tpt, int block, int kv, size_t smem_optin) {
    const void *f = main_kernel_ptr(mode, tpt, block, kv);
    cudaFuncAttributes fa;
    if (!f || cudaFuncGetAttributes(&fa, f) != cudaSuccess || fa.sharedSizeBytes > smem_optin) {
        cudaGetLastError();
        return 0;
    }
    return smem_optin - fa.sharedSizeBytes;
}

// The kernel's dynamic shared-memory limit is raised to that maximum, never set
// to one job's size, so that calls planned on other host threads (which all set
// the same value) cannot lower it between their planning and their launch.
cudaError_t main_kernel_attrs(int mode, int tpt, int block, int kv, size_t smem_optin) {
    const void *f = main_kernel_ptr(mode, tpt, block, kv);
    if (!f) return cudaErrorInvalidValue;
    const size_t lim = main_dynamic_smem_limit(mode, tpt, block, kv, smem_optin);
    if (lim == 0) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lim);
}

cudaError_t launch_main(int mode, int tpt, int block, int grid, size_t smem, const MainArgs &a,
                        cudaStream_t s) {
    switch (mode * 8 + tpt) {
        case GCE_PHASE_FP64 * 8 + 1: return launch_main_fp64_t1(block, grid, smem, a, s);
        case GCE_PHASE_FP64 * 8 + 2: return launch_main_fp64_t2(block, grid, smem, a, s);
        case GCE_PHASE_SPLIT32 * 8 + 1: return launch_main_split32_t1(block, grid, smem, a, s);
        case GCE_PHASE_SPLIT32 * 8 + 2: return launch_main_split32_t2(block, grid, smem, a, s);
        case GCE_PHASE_SPLIT32 * 8 + 4: return launch_main_split32_t4(block, grid, smem, a, s);
        case GCE_PHASE_FIXED32 * 8 + 1: return launch_main_fixed32_t1(block, grid, smem, a, s);
        case GCE_PHASE_FIXED32 * 8 + 2: return launch_main_fixed32_t2(block, grid, smem, a, s);
        case GCE_PHASE_FIXED32 * 8 + 4: return launch_main_fixed32_t4(block, grid, smem, a, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_topk_merge(const unsigned long long *cand, int n_curves, int n_tiles, int k,
                              float *topk_H, long long *topk_idx, const TileStats *stats,
                              double *mean, double *std_dev, float *rho, const JobState *st,
                              cudaStream_t s) {
    if (n_curves <= 0) return cudaSuccess;
    k_topk_merge<<<n_curves, 256, 0, s>>>(cand, n_tiles, k, topk_H, topk_idx, stats, mean,
                                          std_dev, rho, st);
    return cudaGetLastError();
}

cudaError_t launch_single(const MainArgs &a, int curve, long long, cudaStream_t s) {
    // the largest power-of-two block (<= 256) whose counters fit in 48 KB
    int B = 256;
    while (B > 32 && single_smem_bytes(a.n_phase, B) > 48 * 1024) B >>= 1;
    const long long g = (a.n_trials + B - 1) / B;
    const size_t smem = single_smem_bytes(a.n_phase, B);  // overlap needs no extra slot here
    k_single<<<(unsigned int)g, B, smem, s>>>(a, curve);
    return cudaGetLastError();
}

cudaError_t launch_counts(int mode, const MainArgs &a, long long n_cells,
                          const long long *cell_curve, const long long *cell_trial,
                          unsigned int *counts, cudaStream_t s) {
    if (n_cells <= 0) return cudaSuccess;
    const int B = 128;
    const unsigned int g = (unsigned int)((n_cells + B - 1) / B);
    switch (mode) {
        case GCE_PHASE_FP64: k_counts<GCE_PHASE_FP64><<<g, B, 0, s>>>(a, n_cells, cell_curve, cell_trial, counts); break;
        case GCE_PHASE_SPLIT32: k_counts<GCE_PHASE_SPLIT32><<<g, B, 0, s>>>(a, n_cells, cell_curve, cell_trial, counts); break;
        default: k_counts<GCE_PHASE_FIXED32><<<g, B, 0, s>>>(a, n_cells, cell_curve, cell_trial, counts); break;
    }
    return cudaGetLastError();
}

}  // namespace gce
