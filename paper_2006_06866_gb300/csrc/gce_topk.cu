// First level of the per-curve top-k merge.  The persistent CE kernel leaves k
// candidate keys per (curve, trial tile, warp) -- a "tile" below is one such
// list; a grid of 5e6 periods x 512 Pdot values has millions per curve, and one block per curve scanning them
// k times would leave the rest of the GPU idle.  Here many blocks per curve
// each stage one group of tiles' keys in shared memory once, keep its k
// smallest, and merge the group's tile moments (Eq. 5), so that the final
// per-curve merge reads a few thousand keys.
#include <cstdint>

#include "gce_topk.cuh"

namespace gce {

namespace {

constexpr unsigned long long kEmptyKey = ~0ull;
constexpr int kReduceBlock = 256;

// Smallest 64-bit key of the warp: the smallest high word, then the smallest
// low word among the lanes holding it.
__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v) {
    const unsigned int hi = __reduce_min_sync(0xffffffffu, (unsigned int)(v >> 32));
    const unsigned int lo =
        __reduce_min_sync(0xffffffffu, (unsigned int)(v >> 32) == hi ? (unsigned int)v : 0xffffffffu);
    return ((unsigned long long)hi << 32) | lo;
}

// (count, mean, M2) of two sets merged (Chan, Golub and LeVeque's pairwise
// update).
__device__ __forceinline__ void merge_moments(double &n, double &mean, double &m2, double nb,
                                              double meanb, double m2b) {
    if (nb <= 0.0) return;
    if (n <= 0.0) {
        n = nb;
        mean = meanb;
        m2 = m2b;
        return;
    }
    const double tot = n + nb;
    const double d = meanb - mean;
    mean += d * (nb / tot);
    m2 += m2b + d * d * (n * nb / tot);
    n = tot;
}

__global__ void __launch_bounds__(kReduceBlock)
    k_topk_reduce(const unsigned long long *__restrict__ cand, int n_tiles, int k,
                  int tiles_per_group, int n_groups, const TileStats *__restrict__ stats,
                  unsigned long long *__restrict__ cand2, TileStats *__restrict__ stats2,
                  const JobState *st) {
    __shared__ unsigned long long s_keys[kReduceKeys];
    __shared__ unsigned long long s_warp[kReduceBlock / 32];
    __shared__ double s_mom[3 * (kReduceBlock / 32)];
    if (st->err) return;
    const long long b = blockIdx.x;
    const int c = (int)(b / n_groups);
    const int g = (int)(b - (long long)c * n_groups);
    const int t0 = g * tiles_per_group;
    const int nt = min(tiles_per_group, n_tiles - t0);
    const int n = nt * k;  // <= kReduceKeys by the choice of tiles_per_group
    const unsigned long long *src = cand + ((long long)c * n_tiles + t0) * k;
    for (int i = threadIdx.x; i < n; i += kReduceBlock) s_keys[i] = src[i];
    __syncthreads();
    unsigned long long *dst = cand2 + (long long)b * k;
    // k rounds of "smallest key above the previous one"; keys are unique
    unsigned long long last = 0ull;
    for (int r = 0; r < k; ++r) {
        unsigned long long mine = kEmptyKey;
        for (int i = threadIdx.x; i < n; i += kReduceBlock) {
            const unsigned long long v = s_keys[i];
            if ((r == 0 || v > last) && v < mine) mine = v;
        }
        mine = warp_min_u64(mine);
        if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = mine;
        __syncthreads();
        unsigned long long m = s_warp[0];
#pragma unroll
        for (int w = 1; w < kReduceBlock / 32; ++w) m = s_warp[w] < m ? s_warp[w] : m;
        __syncthreads();
        last = m;
        if (threadIdx.x == 0) dst[r] = m;
    }
    if (!stats) return;
    // the group's tile moments, merged in a fixed order (a strided run of tiles
    // per thread, a fixed tree within each warp, then the warps in order)
    double nn = 0.0, mu = 0.0, m2 = 0.0;
    const TileStats *ts = stats + (long long)c * n_tiles + t0;
    for (int i = threadIdx.x; i < nt; i += kReduceBlock) merge_moments(nn, mu, m2, ts[i].n, ts[i].mean, ts[i].m2);
    for (int o = 1; o < 32; o <<= 1) {
        const double nb = __shfl_down_sync(0xffffffffu, nn, o);
        const double mb = __shfl_down_sync(0xffffffffu, mu, o);
        const double qb = __shfl_down_sync(0xffffffffu, m2, o);
        if ((threadIdx.x & (2 * o - 1)) == 0) merge_moments(nn, mu, m2, nb, mb, qb);
    }
    if ((threadIdx.x & 31) == 0) {
        s_mom[3 * (threadIdx.x >> 5)] = nn;
        s_mom[3 * (threadIdx.x >> 5) + 1] = mu;
        s_mom[3 * (threadIdx.x >> 5) + 2] = m2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        nn = 0.0;
        mu = 0.0;
        m2 = 0.0;
        for (int w = 0; w < kReduceBlock / 32; ++w) merge_moments(nn, mu, m2, s_mom[3 * w], s_mom[3 * w + 1], s_mom[3 * w + 2]);
        stats2[b] = TileStats{nn, mu, m2};
    }
}

}  // namespace

cudaError_t launch_topk_reduce(const unsigned long long *cand, int n_curves, int n_tiles, int k,
                               int tiles_per_group, int n_groups, const TileStats *stats,
                               unsigned long long *cand2, TileStats *stats2, const JobState *st,
                               cudaStream_t s) {
    if (n_curves <= 0 || n_groups <= 0) return cudaSuccess;
    if (k < 1 || (long long)tiles_per_group * k > kReduceKeys) return cudaErrorInvalidValue;
    const long long blocks = (long long)n_curves * n_groups;
    if (blocks > 0x7fffffffll) return cudaErrorInvalidValue;
    k_topk_reduce<<<(unsigned int)blocks, kReduceBlock, 0, s>>>(cand, n_tiles, k, tiles_per_group,
                                                               n_groups, stats, cand2, stats2, st);
    return cudaGetLastError();
}

}  // namespace gce
