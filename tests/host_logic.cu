// Host-side planning logic of the CE library, checked on the CPU: the header
// functions that size the trial tiles, the first level of the top-k merge, the
// SPLIT32 counter slots and the CE kernel's shared-memory layout.  Built by tests/test_host_logic.py with nvcc and run
// without a GPU: no CUDA runtime call is made.  Prints "ok" and returns 0, or
// prints each failed check and returns 1.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <random>

#include "../paper_2006_06866_gb300/csrc/gce_internal.cuh"
#include "../paper_2006_06866_gb300/csrc/gce_topk.cuh"

using namespace gce;

static int g_fail = 0;

#define CHECK(cond, ...)                                 \
    do {                                                 \
        if (!(cond)) {                                   \
            if (g_fail < 20) {                           \
                std::printf("FAIL %s: ", #cond);         \
                std::printf(__VA_ARGS__);                \
                std::printf("\n");                       \
            }                                            \
            ++g_fail;                                    \
        }                                                \
    } while (0)

// Trial tiles of one curve: every (period, Pdot) trial falls in some tile, and
// no tile is wholly past the grid.
static void check_tile_grid(std::mt19937_64 &rng) {
    const int blocks[] = {64, 128, 256, 512};
    const int tpts[] = {1, 2, 4};
    for (int it = 0; it < 20000; ++it) {
        const long long n_p = 1 + (long long)(rng() % 200000);
        const long long n_q = (rng() % 4 == 0) ? 1 : 1 + (long long)(rng() % 600);
        const int B = blocks[rng() % 4], T = tpts[rng() % 3];
        const TileGrid g = tile_grid(n_p, n_q, B, T);
        if (g.pd_major) {
            CHECK(n_q > 1 && T > 1, "pd_major with n_q %lld tpt %d", n_q, T);
            CHECK((long long)g.n_ptiles * B >= n_p && (long long)(g.n_ptiles - 1) * B < n_p,
                  "period tiles %d x %d for %lld periods", g.n_ptiles, B, n_p);
            const long long q_tiles = g.n_tiles / g.n_ptiles;
            CHECK(g.n_tiles % g.n_ptiles == 0 && q_tiles * T >= n_q && (q_tiles - 1) * T < n_q,
                  "%lld tiles, %d per Pdot block, %lld Pdot x tpt %d", (long long)g.n_tiles,
                  g.n_ptiles, n_q, T);
        } else {
            const long long per = (long long)B * T, n = n_p * n_q;
            CHECK(g.n_tiles * per >= n && (g.n_tiles - 1) * per < n,
                  "%lld tiles of %lld for %lld trials", (long long)g.n_tiles, per, n);
        }
    }
}

// First merge level: groups cover every tile once, and one group's candidates
// fit the reduction block's shared array.
static void check_topk_groups(std::mt19937_64 &rng) {
    for (int it = 0; it < 50000; ++it) {
        const long long n_tiles = 1 + (long long)(rng() % (it % 2 ? 5000000 : 5000));
        const int k = 1 + (int)(rng() % GCE_MAX_TOPK);
        int tpg = -1;
        const int groups = topk_groups(n_tiles, k, &tpg);
        if (groups == 0) {
            CHECK(n_tiles * k <= kReduceKeys && tpg == 0, "no groups for %lld x %d", n_tiles, k);
        } else {
            CHECK(n_tiles * k > kReduceKeys, "groups for %lld x %d keys", n_tiles, k);
            CHECK(tpg >= 1 && (long long)tpg * k <= kReduceKeys, "tpg %d x k %d", tpg, k);
            CHECK((long long)groups * tpg >= n_tiles && (long long)(groups - 1) * tpg < n_tiles,
                  "%d groups of %d for %lld tiles", groups, tpg, n_tiles);
        }
    }
}

// SPLIT32 slots: the fold's residual x satisfies |x| <= 3/4 + 2^-20 under the
// job's range check (|x| <= 1/2 + 2^-20 where a fold re-reduces it; the mid
// range is used by folds whose warp's bound is within 9/16, the others
// re-reduce), and the slot of x is floor(n x + n); the kept range must hold
// every such slot and stay within the 2n slots of a trial, and the mid range
// must lie between the narrow and the wide one.  The other folds keep the n
// phase bins.
static void check_slot_range() {
    for (int n = 1; n <= GCE_MAX_PHASE_BINS; ++n) {
        for (int range : {RANGE_WIDE, RANGE_NARROW, RANGE_MID}) {
            const double xb = (range == RANGE_NARROW ? 0.5 : range == RANGE_MID ? 0.5625 : 0.75) +
                              std::ldexp(1.0, -20);
            const SlotRange r = slot_range(GCE_PHASE_SPLIT32, n, range);
            const int lo = (int)std::floor(-xb * n + n), hi = (int)std::floor(xb * n + n);
            CHECK(r.zmin <= std::max(lo, 0) && r.zmax >= std::min(hi, 2 * n - 1),
                  "n %d range %d: kept [%d, %d], reachable [%d, %d]", n, range, r.zmin, r.zmax,
                  lo, hi);
            CHECK(r.zmin >= 0 && r.zmax <= 2 * n - 1 && r.zmin <= r.zmax,
                  "n %d range %d: [%d, %d] outside [0, 2n)", n, range, r.zmin, r.zmax);
            CHECK(slots_per_trial(GCE_PHASE_SPLIT32, n, range) == r.zmax - r.zmin + 1,
                  "n %d: slots per trial", n);
            // every phase bin keeps at least one of its two slots (j and j + n)
            for (int j = 0; j < n; ++j)
                CHECK((j >= r.zmin && j <= r.zmax) || (j + n >= r.zmin && j + n <= r.zmax),
                      "n %d range %d: bin %d has no slot", n, range, j);
        }
        const SlotRange w = slot_range(GCE_PHASE_SPLIT32, n, RANGE_WIDE);
        const SlotRange m = slot_range(GCE_PHASE_SPLIT32, n, RANGE_MID);
        const SlotRange q = slot_range(GCE_PHASE_SPLIT32, n, RANGE_NARROW);
        CHECK(w.zmin <= m.zmin && m.zmin <= q.zmin && q.zmax <= m.zmax && m.zmax <= w.zmax,
              "n %d: mid range [%d, %d] not between narrow [%d, %d] and wide [%d, %d]", n,
              m.zmin, m.zmax, q.zmin, q.zmax, w.zmin, w.zmax);
        for (int mode : {GCE_PHASE_FP64, GCE_PHASE_FIXED32}) {
            for (int range : {RANGE_WIDE, RANGE_NARROW, RANGE_MID}) {
                const SlotRange r = slot_range(mode, n, range);
                CHECK(r.zmin == 0 && r.zmax == n - 1, "mode %d n %d: [%d, %d]", mode, n, r.zmin,
                      r.zmax);
            }
        }
    }
}

// The CE kernel's shared-memory layout (one function for the host's launch size
// and the kernel's carve-up): regions in order, each aligned for its type (16
// bytes for the staged points and the counters after them), the staged points
// sized 8 or 16 bytes each, and the total the sum of the parts.
static void check_smem_layout(std::mt19937_64 &rng) {
    const int blocks[] = {64, 128, 256, 512};
    const int tpts[] = {1, 2, 4};
    for (int it = 0; it < 20000; ++it) {
        const int mode = (int)(rng() % 3), B = blocks[rng() % 4], T = tpts[rng() % 3];
        const int chunk = 32 * (1 + (int)(rng() % 256));
        const int n_phase = 1 + (int)(rng() % GCE_MAX_PHASE_BINS);
        const int n_mag = 1 + (int)(rng() % GCE_MAX_MAG_BINS);
        const int table = 1 + (int)(rng() % 2048);
        const int range = (int)(rng() % 3), half = (int)(rng() % 2);
        const MainSmemLayout L =
            main_smem_layout(mode, B, T, chunk, n_phase, n_mag, table, range, half);
        const unsigned int pt = (mode == GCE_PHASE_FP64 || half) ? 8u : 16u;
        const unsigned int cnt = 4u * (unsigned int)(T * slots_per_trial(mode, n_phase, range) * B);
        CHECK(L.pts >= 8u * (unsigned int)table && L.pts % 16 == 0, "pts %u table %d", L.pts, table);
        CHECK(L.cnt == L.pts + pt * (unsigned int)chunk && L.cnt % 16 == 0, "cnt %u", L.cnt);
        CHECK(L.seg == L.cnt + cnt && L.seg % 4 == 0, "seg %u", L.seg);
        CHECK(L.total == L.seg + 4u * (unsigned int)(n_mag + 1), "total %u", L.total);
    }
}

int main() {
    std::mt19937_64 rng(20200611);
    check_tile_grid(rng);
    check_topk_groups(rng);
    check_slot_range();
    check_smem_layout(rng);
    if (g_fail) {
        std::printf("%d checks failed\n", g_fail);
        return 1;
    }
    std::printf("ok\n");
    return 0;
}
