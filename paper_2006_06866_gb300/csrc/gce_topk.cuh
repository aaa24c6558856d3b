// First level of the per-curve top-k merge (Sec. 2.3's grid minimum, batched
// minima merged as in Sec. 4) for grids with many trial tiles.
#pragma once

#include "gce_internal.cuh"

namespace gce {

// Candidate keys one reduction block holds in shared memory (32 KB).
constexpr int kReduceKeys = 4096;

// Groups of tiles per curve that a job with n_tiles tiles and top-k size k is
// reduced to before the final merge; 0 when the final merge reads the tiles'
// candidates directly (at most kReduceKeys of them per curve).
inline int topk_groups(long long n_tiles, int k, int *tiles_per_group) {
    if (k < 1 || n_tiles * k <= kReduceKeys) {
        *tiles_per_group = 0;
        return 0;
    }
    const int tpg = kReduceKeys / k > 1 ? kReduceKeys / k : 1;
    *tiles_per_group = tpg;
    return (int)((n_tiles + tpg - 1) / tpg);
}

// Block b of n_curves * n_groups: curve b / n_groups, group g = b % n_groups,
// tiles [g * tiles_per_group, min((g + 1) * tiles_per_group, n_tiles)).
//   cand:  u64 keys [n_curves][n_tiles][k] (H bits << 32 | flat trial index)
//   cand2: u64 keys [n_curves][n_groups][k], each group's k smallest,
//          ascending, padded with ~0 when the group holds fewer valid keys
//   stats (may be nullptr): tile moments [n_curves][n_tiles];
//   stats2: the group's tiles merged in tile order [n_curves][n_groups].
// Nothing is written when the job's device checks failed (st->err != 0).
cudaError_t launch_topk_reduce(const unsigned long long *cand, int n_curves, int n_tiles, int k,
                               int tiles_per_group, int n_groups, const TileStats *stats,
                               unsigned long long *cand2, TileStats *stats2, const JobState *st,
                               cudaStream_t s);

}  // namespace gce
