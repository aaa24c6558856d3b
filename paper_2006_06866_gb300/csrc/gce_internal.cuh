// Internal definitions shared by the library's translation units: job state,
// per-point and per-trial payloads of the three fold modes, the folds
// themselves (Eq. 3 of arXiv:2006.06866) and the fixed-point entropy table
// (Eq. 4).  Nothing here is part of the C ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/gce.h"

namespace gce {

// ------------------------------------------------------------------ job state

// Device-side state of one call: reductions of the scan kernel, input-check
// flags and the persistent kernel's work counter.  Zeroed (pmin set to +inf)
// by k_init at the start of every call.
struct JobState {
    unsigned long long tau_max_bits;    // max |t - t0| as binary64 bits
    unsigned long long pmin_bits;       // min period as binary64 bits
    unsigned long long pdot_max_bits;   // max |Pdot| as binary64 bits
    unsigned long long work;            // next work item (persistent kernel)
    unsigned int err;                   // ERR_* bits
    unsigned int pad[3];
};

enum : unsigned int {
    ERR_TIME = 1u,      // non-finite time or magnitude
    ERR_PERIOD = 2u,    // non-finite or non-positive period
    ERR_PDOT = 4u,      // non-finite period derivative
    ERR_RANGE = 8u,     // trial range beyond what the chosen fold represents
    ERR_BAND = 16u,     // filter index outside [0, n_bands)
    ERR_SLOT = 32u,     // checked builds only: a counter slot outside the trial's kept range
};

// Fixed-point scaling of the FIXED32 fold, derived from the job's maxima.
// tau_max < 2^e_tau.  T = tau 2^s (|T| < 2^62), F = f 2^r with s + r = 96, so
// T F / 2^64 = tau f 2^32; U = tau^2 2^u (U < 2^62), A = a 2^v with
// u + v = 96, so U A / 2^64 = a tau^2 2^32.
struct FixedScale {
    int e_tau;
    int s, r, u, v;
};

__host__ __device__ inline FixedScale fixed_scale_from(double tau_max) {
    FixedScale fs;
    int e = 0;
    if (tau_max > 0.0) {
        int ex;
        frexp(tau_max, &ex);   // tau_max = m 2^ex, m in [0.5, 1)  =>  tau_max < 2^ex
        e = ex;
    }
    fs.e_tau = e;
    fs.s = 62 - e;
    fs.r = 96 - fs.s;
    fs.u = 62 - 2 * e;
    fs.v = 96 - fs.u;
    return fs;
}

// ------------------------------------------------------------------ payloads

// Per point, sorted by magnitude bin, in the layout of the fold mode.
//   FP64:    double tau                                        (8 bytes)
//   SPLIT32: float4 {tau_hi, tau_lo, tau2_hi, tau2_lo}          (16 bytes)
//   FIXED32: uint4  {T1 (int32), t0f, U1, u0f}                  (16 bytes)
//            T = tau 2^s = T1 2^32 + T0; U = tau^2 2^u = U1 2^32 + U0 (U0
//            balanced); t0f, u0f are the bit patterns of the floats
//            2^23 + (T0 >> 9) and 2^23 + ((U0 + 2^31) >> 9).
// Per flat trial:
//   FP64:    double2 {f, a}
//   SPLIT32: float4  {f_hi, f_lo, a_hi, a_lo}
//   FIXED32: FixedTrial, see fold_fixed.
struct FixedTrial {
    uint4 i;   // {F1, F0 (int32, balanced), A1 (int32), A0}: F = f 2^r, A = -a 2^v
    float4 f;  // {G0, G2, K, k as bits}: the FP32 cross terms' scales and offset
};
template <int MODE> struct ModeTraits;
// half_t: the first two words of a point, all a fold without a Pdot term reads
// (SPLIT32 {tau_hi, tau_lo}, FIXED32 {T1, t0f}); FP64 points are one word.
template <> struct ModeTraits<GCE_PHASE_FP64> {
    typedef double point_t;
    typedef double half_t;
    typedef double2 trial_t;
    __device__ static point_t widen(half_t h) { return h; }
};
template <> struct ModeTraits<GCE_PHASE_SPLIT32> {
    typedef float4 point_t;
    typedef float2 half_t;
    typedef float4 trial_t;
    __device__ static point_t widen(half_t h) { return make_float4(h.x, h.y, 0.0f, 0.0f); }
};
template <> struct ModeTraits<GCE_PHASE_FIXED32> {
    typedef uint4 point_t;
    typedef uint2 half_t;
    typedef FixedTrial trial_t;
    __device__ static point_t widen(half_t h) { return make_uint4(h.x, h.y, 0u, 0u); }
};

// Balanced split of a 64-bit value: x = hi 2^32 + lo with lo a signed 32-bit
// value in [-2^31, 2^31), so that signed multiply-high works on it.
__host__ __device__ inline void split_balanced(long long x, int *hi, int *lo) {
    long long h = x >> 32;  // arithmetic
    unsigned int l = (unsigned int)(x & 0xffffffffll);
    if (l >= 0x80000000u) h += 1;
    *hi = (int)h;
    *lo = (int)l;  // two's complement reinterpretation: l - 2^32 when l >= 2^31
}

// ------------------------------------------------------------------ folds

// Eq. 3 in binary64 with the pinned operation sequence (see gce.h); returns the
// phase bin.  With pdot == false, a is known to be +-0 and x = s exactly.  The
// period part s = tau f is split out so that trials sharing the period can
// share it (fold_fp64_from completes the fold from it).
__device__ __forceinline__ double fold_fp64_fpart(double tau, double f) { return __dmul_rn(tau, f); }

template <bool PDOT>
__device__ __forceinline__ int fold_fp64_from(double s, double tau, double a, double nphi,
                                              int n_phase) {
    double x = s;
    if (PDOT) {
        double b = __dmul_rn(a, tau);
        x = __fma_rn(-b, tau, s);
    }
    double phi = __dsub_rn(x, floor(x));
    int j = __double2int_rd(__dmul_rn(phi, nphi));
    return min(j, n_phase - 1);
}

template <bool PDOT>
__device__ __forceinline__ int fold_fp64(double tau, double f, double a, double nphi,
                                         int n_phase) {
    return fold_fp64_from<PDOT>(fold_fp64_fpart(tau, f), tau, a, nphi, n_phase);
}

// Eq. 3 in FP32 double-float.  tau = th + tl and f = fh + fl (float pairs),
// tau^2 = t2h + t2l and a = ah + al with the a pair stored negated.  The
// integer cycles of th fh are removed by an FMA against the rounding constant
// M = 1.5 2^23: t = fma(th, fh, M) holds rint(th fh) + M (|th fh| < 2^21 cycles,
// checked per job), and r = fma(th, fh, -(t - M)) is the exact product minus
// that integer, rounded once (|r| <= 1/2).  The cross terms tl fh and th fl
// (tl fl is below 2^-48 relative) are added by FMA.  The Pdot term -a tau^2 is
// reduced the same way and the sum reduced once more.  x then lies in
// (-1, 1), and one round-down FMA against the same constant gives
// n_phase + floor(x n_phase) in [0, 2 n_phase): the returned slot, where slots
// j and j + n_phase both stand for phase bin j (so no modulo is needed here).
// Phase error about 1e-7 cycles (a few 2^-25 roundings).
constexpr float kRound = 12582912.0f;  // 1.5 * 2^23

// The period part of the fold, shared by trials of the same period: th fh with
// its integer cycles removed, plus the cross terms (the whole residual x when
// Pdot = 0).
__device__ __forceinline__ float fold_split_fpart(float4 pt, float4 tr) {
    const float th = pt.x, tl = pt.y;
    const float fh = tr.x, fl = tr.y;
    const float t = __fmaf_rn(th, fh, kRound);
    const float r = __fmaf_rn(th, fh, __fsub_rn(kRound, t));
    return __fmaf_rn(th, fl, __fmaf_rn(tl, fh, r));
}

// The rest of the fold from the period part c: the Pdot term -a tau^2 reduced
// the same way, the sum reduced once more, then the slot.  REDUCE (without
// Pdot): the residual is reduced once more as well, to |x| <= 1/2, for folds that
// must stay in the narrow slot range (see slot_range).
template <bool PDOT, bool REDUCE = false>
__device__ __forceinline__ int fold_split_from(float c, float4 pt, float4 tr, float nphi,
                                               float zoff) {
    float x = c;
    if (!PDOT && REDUCE) x = __fsub_rn(c, __fsub_rn(__fadd_rn(c, kRound), kRound));
    if (PDOT) {
        const float t2h = pt.z, t2l = pt.w;
        const float nah = tr.z, nal = tr.w;  // -a split
        const float t2 = __fmaf_rn(nah, t2h, kRound);
        const float r2 = __fmaf_rn(nah, t2h, __fsub_rn(kRound, t2));
        c = __fmaf_rn(nah, t2l, c);
        c = __fmaf_rn(nal, t2h, c);
        const float y = __fadd_rn(c, r2);
        x = __fsub_rn(y, __fsub_rn(__fadd_rn(y, kRound), kRound));
    }
    const float z = __fmaf_rd(x, nphi, zoff);  // zoff = 1.5 2^23 + n_phase
    return __float_as_int(z) - __float_as_int(kRound);
}

template <bool PDOT>
__device__ __forceinline__ int fold_split(float4 pt, float4 tr, float nphi, float zoff) {
    return fold_split_from<PDOT>(fold_split_fpart(pt, tr), pt, tr, nphi, zoff);
}

// Eq. 3 in 32-bit-limb fixed point, the phase in units of 2^-32 cycles so that
// the integer cycles wrap out of a 32-bit word.  With T = T1 2^32 + T0 and
// F = F1 2^32 + F0, bits 64..95 of T F are
//   lo32(T1 F1) + hi32(T1 F0) + T0 F1 / 2^32            (+ dropped carries).
// The first two are exact integer products (IMAD, IMAD.HI).  The third is
// below g1 = F1 units and is computed on the FP32 pipe: t0f = 2^23 + (T0 >> 9)
// times G0 = F1 2^(-23-k), added to an offset K that removes the 2^23 G0
// term and carries the 1.5 2^23 rounding constant, so the FMA result's bit
// pattern holds the term rounded to 2^k units (k per trial, the smallest with
// F1 < 2^(22+k)); it joins the accumulator shifted left by k, and the integer
// offset C = -(bits(1.5 2^23) << k) cancels the constant's bits.  The Pdot term
// -a tau^2 is the same construction for U and A = -a 2^v: lo32(U1 A1) and
// hi32(A0 U1) exact, hi32(A1 U0) through u0f and G2 in the same FMA chain.
// Error: dropped carries (-1..+2 units), T0 >> 9 truncation (<= F1 2^-23),
// FP32 roundings (<= 3 2^(k-1)), so a few 2^-32 cycles for k <= 2.
// The phase bin is floor(phase n_phase / 2^32) = hi32(phase n_phase).
__device__ __forceinline__ unsigned int mad_lo_u32(unsigned int a, unsigned int b,
                                                   unsigned int c) {
    unsigned int d;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}
__device__ __forceinline__ unsigned int mad_hi_s32(int a, int b, unsigned int c) {
    int d;
    asm("mad.hi.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"((int)c));
    return (unsigned int)d;
}
__device__ __forceinline__ unsigned int mad_hi_u32(unsigned int a, unsigned int b,
                                                   unsigned int c) {
    unsigned int d;
    asm("mad.hi.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

// Per-trial values of the FIXED32 fold that stay in registers.
struct FixedPrep {
    unsigned int F1, A1, A0, C, k;
    int F0;
    float G0, G2, K;
};

__device__ __forceinline__ FixedPrep fixed_prep(const FixedTrial &t) {
    FixedPrep p;
    p.F1 = t.i.x;
    p.F0 = (int)t.i.y;
    p.A1 = t.i.z;
    p.A0 = t.i.w;
    p.G0 = t.f.x;
    p.G2 = t.f.y;
    p.K = t.f.z;
    p.k = __float_as_uint(t.f.w);
    p.C = 0u - (0x4B400000u << p.k);
    return p;
}

// The period part of the fixed-point fold, shared by trials of the same period:
// the exact integer products of T and F, with the offset C.
__device__ __forceinline__ unsigned int fold_fixed_fpart(uint4 pt, const FixedPrep &t) {
    const int T1 = (int)pt.x;
    const unsigned int acc = mad_lo_u32((unsigned int)T1, t.F1, t.C);
    return mad_hi_s32(T1, t.F0, acc);
}

// The rest of the fold from the period part acc: the Pdot products, the FP32
// cross terms and, for the bin, the multiply-high by n_phase.  K0: the shift
// by k is zero (every trial of the tile has F1 < 2^22).
template <bool PDOT, bool K0>
__device__ __forceinline__ unsigned int fold_fixed_phase_from(unsigned int acc, uint4 pt,
                                                              const FixedPrep &t) {
    float zin = t.K;
    if (PDOT) {
        const unsigned int U1 = pt.z;
        acc = mad_lo_u32(U1, t.A1, acc);
        acc = mad_hi_u32(t.A0, U1, acc);
        zin = __fmaf_rn(__uint_as_float(pt.w), t.G2, zin);
    }
    const unsigned int zb = __float_as_uint(__fmaf_rn(__uint_as_float(pt.y), t.G0, zin));
    return acc + (K0 ? zb : __funnelshift_l(0u, zb, t.k));
}

template <bool PDOT>
__device__ __forceinline__ int fold_fixed(uint4 pt, const FixedPrep &t, unsigned int n_phase) {
    return (int)__umulhi(fold_fixed_phase_from<PDOT, false>(fold_fixed_fpart(pt, t), pt, t),
                         n_phase);
}

template <bool PDOT, bool K0>
__device__ __forceinline__ unsigned int fold_fixed_bin_from(unsigned int acc, uint4 pt,
                                                            const FixedPrep &t,
                                                            unsigned int n_phase) {
    return __umulhi(fold_fixed_phase_from<PDOT, K0>(acc, pt, t), n_phase);
}

// ------------------------------------------------------------------ entropy

// The counter slots a trial keeps: logical slots [zmin, zmax] (fine phase
// bins; 50 %-overlapping bins are formed from them in the epilogue).  FP64 and
// FIXED32 count phase bins directly.  SPLIT32's slot is floor(x n + n) for the
// fold residual x, and the kept range is set by a bound on |x|:
//   RANGE_WIDE: a job that passes the range check (cycles < 2^21) has |x| <=
//     3/4 + 2^-20 (r within 1/2, each cross term within 2^-24 |th fh| < 1/8,
//     three roundings), so slots outside [floor(n (1/4 - 2^-16)),
//     floor(n (7/4 + 2^-16))] are never reached;
//   RANGE_NARROW: every fold of the job re-reduces its residual to |x| <= 1/2
//     (jobs with a Pdot axis, whose folds do that anyway), and only
//     [floor(n (1/2 - 2^-16)), floor(n (3/2 + 2^-16))] is kept;
//   RANGE_MID: |x| <= 9/16 + 2^-16 is kept; a warp whose trials could fold
//     outside it (the bound of split_slot_window) re-reduces its folds as in
//     RANGE_NARROW, the others fold as in RANGE_WIDE.
enum { RANGE_WIDE = 0, RANGE_NARROW = 1, RANGE_MID = 2 };
struct SlotRange {
    int zmin, zmax;
};
__host__ __device__ inline SlotRange slot_range(int mode, int n_phase, int range) {
    if (mode != GCE_PHASE_SPLIT32) return {0, n_phase - 1};
    const double xw =
        (range == RANGE_NARROW ? 0.5 : range == RANGE_MID ? 0.5625 : 0.75) + 1.0 / 65536.0;
    int zmin = (int)floor((double)n_phase * (1.0 - xw));
    int zmax = (int)floor((double)n_phase * (1.0 + xw));
    if (zmin < 0) zmin = 0;
    if (zmax > 2 * n_phase - 1) zmax = 2 * n_phase - 1;
    return {zmin, zmax};
}
__host__ __device__ inline int slots_per_trial(int mode, int n_phase, int range) {
    const SlotRange r = slot_range(mode, n_phase, range);
    return r.zmax - r.zmin + 1;
}

// Byte offsets of the CE kernel's dynamic shared-memory regions, in order: the
// c ln c table (an even number of 8-byte entries, so the points after it stay
// 16-byte aligned), the staged points (8 bytes each for FP64 and for half
// points, else 16; chunk is a multiple of 32), the counters and the segment
// starts.  The host sizes the launch with `total` and the kernel carves its
// memory with the same offsets.  (k and block do not enter: each warp writes its
// top-k keys and moments straight to global memory.)
struct MainSmemLayout {
    unsigned int pts, cnt, seg, total;
};
__host__ __device__ inline MainSmemLayout main_smem_layout(int mode, int block, int tpt, int chunk,
                                                           int n_phase, int n_mag,
                                                           int table_smem, int range, int half) {
    MainSmemLayout L;
    const unsigned int pt = (mode == GCE_PHASE_FP64 || half) ? 8u : 16u;
    L.pts = 8u * (unsigned int)((table_smem + 1) & ~1);
    L.cnt = L.pts + pt * (unsigned int)chunk;
    L.seg = L.cnt + 4u * (unsigned int)(tpt * slots_per_trial(mode, n_phase, range) * block);
    L.total = L.seg + 4u * (unsigned int)(n_mag + 1);
    return L;
}

// Fixed-point table of c ln c: tab[c] = round(c ln(c) 2^32), tab[0] = tab[1] = 0.
// Eq. 4 rewritten with integer counts is
//   N H = sum_j c_j ln c_j - sum_ij c_ij ln c_ij,
// and summing the table's integers makes both sums exact and independent of
// order; the only error is the table's rounding (at most 2^-33 per term).
constexpr double kTabScale = 4294967296.0;  // 2^32
constexpr double kTabInvScale = 1.0 / 4294967296.0;

// ------------------------------------------------------------------ launches

struct PrepArgs {
    const double *times;
    const double *mags;
    const long long *offsets;  // device copy, n_curves + 1
    int n_curves;
    int n_mag;
    double t0;
    void *payload;             // ModeTraits<MODE>::point_t[sum N], sorted by mag bin per curve
    int *seg;                  // [n_curves][n_mag + 1] segment starts (relative to the curve)
    const JobState *state;
    const unsigned char *bands;  // multi-filter input: filter of each point, or nullptr
    const double2 *band_stats;   // [n_curves][n_bands] {median, standard deviation}
    int n_bands;
};

struct TrialArgs {
    const double *periods;
    const double *pdots;
    int n_periods;
    int n_pdots;
    void *trialc;              // ModeTraits<MODE>::trial_t[n_periods * n_pdots]
    JobState *state;
};

// Moments of a tile's H values: count, mean, sum of squared deviations.
struct TileStats {
    double n, mean, m2;
};

// Trial tiles of one curve's grid for a launch of `block` threads x `tpt`
// trials.  With several Pdot values and tpt > 1 a tile is block periods x tpt
// consecutive Pdot values, so that a thread's trials share their period (and
// the fold's period part); otherwise a tile is a run of block x tpt flat trial
// indices q n_periods + p.
struct TileGrid {
    long long n_tiles;
    int n_ptiles, pd_major;
};
inline TileGrid tile_grid(long long n_periods, long long n_pdots, int block, int tpt) {
    TileGrid g;
    g.pd_major = (n_pdots > 1 && tpt > 1) ? 1 : 0;
    if (g.pd_major) {
        g.n_ptiles = (int)((n_periods + block - 1) / block);
        g.n_tiles = (long long)g.n_ptiles * ((n_pdots + tpt - 1) / tpt);
    } else {
        g.n_ptiles = 0;
        g.n_tiles = (n_periods * n_pdots + (long long)block * tpt - 1) / ((long long)block * tpt);
    }
    return g;
}

struct MainArgs {
    const void *payload;
    const long long *offsets;
    const int *seg;
    const void *trialc;
    const int *order;          // curves in processing order (longest first)
    const unsigned long long *table;
    long long n_trials;
    int n_periods, n_pdots;
    int n_tiles;               // trial tiles per curve
    int n_ptiles;              // period-major tiling: tiles along the periods
    int pd_major;              // tile = block periods x tpt Pdot values (else flat runs)
    int range;                 // SPLIT32: the kept slot range (RANGE_*)
    long long n_items;         // n_curves * n_tiles
    // items [0, n_long_items) are (curve, tile) pairs of the first n_long curves
    // of `order`, curve-major; the rest pair the n_short curves after them with
    // the tiles tile-major (curve index fastest)
    long long n_long_items;
    int n_long, n_short;
    int grab;                  // items taken per work-counter increment
    int n_phase;
    int n_mag;
    int chunk;                 // points staged per pass
    int table_smem;            // table entries staged in shared memory
    float *out;                // grid or nullptr
    unsigned long long *cand;  // top-k candidates [n_curves][n_tiles][k] or nullptr
    int k;
    TileStats *stats;          // per-tile moments [n_curves][n_tiles] or nullptr
    int overlap;               // 50 %-overlapping phase bins
    // SPLIT32 / FIXED32 with one Pdot value: the staging buffer holds `chunk`
    // half points (8 bytes); a job whose Pdot is 0 stages half points, one whose
    // single Pdot is not 0 stages chunk / 2 whole points in the same bytes
    int half;
    int kv;                    // CE kernel variant (KV_*): overlapping bins or not
    JobState *state;
};

// Instantiations of the CE kernel: without overlapping bins (snapshot counters),
// and with them (packed two-segment counters for curves of at most 1023 points,
// snapshot counters for longer ones).
enum { KV_SNAP = 0, KV_OVL = 1 };
inline int kernel_variant(bool overlap) { return overlap ? KV_OVL : KV_SNAP; }

// Kernel launchers (defined in the .cu files).
cudaError_t launch_init(JobState *st, cudaStream_t s);
cudaError_t launch_scan(const double *times, const double *mags, long long n_points,
                        const double *periods, int n_periods, const double *pdots, int n_pdots,
                        double t0, JobState *st, cudaStream_t s);
cudaError_t launch_trials(int mode, const TrialArgs &a, cudaStream_t s);
cudaError_t launch_prep(int mode, const PrepArgs &a, cudaStream_t s);
cudaError_t launch_band_stats(const double *mags, const unsigned char *bands,
                              const long long *offsets, int n_curves, int n_bands,
                              double2 *stats, JobState *st, cudaStream_t s);
cudaError_t launch_table(unsigned long long *table, int n_max, cudaStream_t s);
size_t main_smem_bytes(int mode, int block, int tpt, int chunk, int n_phase, int n_mag,
                       int table_smem, int range, int half);
size_t single_smem_bytes(int n_phase, int block);
size_t main_dynamic_smem_limit(int mode, int tpt, int block, int kv, size_t smem_optin);
cudaError_t main_kernel_attrs(int mode, int tpt, int block, int kv, size_t smem_optin);
const void *main_kernel_ptr(int mode, int tpt, int block, int kv);
// per fold mode and trials per thread (gce_main_<mode>_t<tpt>.cu)
#define GCE_MAIN_TU(name, t)                                                           \
    const void *main_kernel_ptr_##name##_t##t(int block, int kv);                       \
    cudaError_t launch_main_##name##_t##t(int block, int grid, size_t smem, const MainArgs &a, \
                                          cudaStream_t s);
GCE_MAIN_TU(fp64, 1)
GCE_MAIN_TU(fp64, 2)
GCE_MAIN_TU(split32, 1)
GCE_MAIN_TU(split32, 2)
GCE_MAIN_TU(split32, 4)
GCE_MAIN_TU(fixed32, 1)
GCE_MAIN_TU(fixed32, 2)
GCE_MAIN_TU(fixed32, 4)
#undef GCE_MAIN_TU
cudaError_t launch_main(int mode, int tpt, int block, int grid, size_t smem,
                        const MainArgs &a, cudaStream_t s);
cudaError_t launch_topk_merge(const unsigned long long *cand, int n_curves, int n_tiles,
                              int k, float *topk_H, long long *topk_idx, const TileStats *stats,
                              double *mean, double *std_dev, float *rho, const JobState *st,
                              cudaStream_t s);
cudaError_t launch_single(const MainArgs &a, int curve, long long n_points, cudaStream_t s);
cudaError_t launch_counts(int mode, const MainArgs &a, long long n_cells,
                          const long long *cell_curve, const long long *cell_trial,
                          unsigned int *counts, cudaStream_t s);

}  // namespace gce
