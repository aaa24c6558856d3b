// The CE kernel (included by one translation unit per fold mode and trials
// per thread, which instantiate it): fold (Eq. 3) -> phase x magnitude histogram (Sec. 2.3) ->
// entropy (Eq. 4) -> grid or per-curve top-k (Sec. 2.3, Sec. 4).
//
// Work decomposition.  One thread owns TPT trials (P, Pdot) of one light curve
// -- the paper's thread-per-grid-point design (Sec. 2.3.2) -- and a CTA owns a
// tile of block * TPT consecutive flat trial indices.  A work item is one
// (curve, tile) pair; CTAs are persistent and take items from one atomic
// counter, longest curves first.  The curve's points, regrouped by magnitude
// bin during preparation, are staged in shared memory and read by every thread
// as broadcasts.  Because the points arrive one magnitude bin at a time, each
// thread needs only a 1-D phase histogram per trial (the paper's
// 1/n_mag-memory observation).
//
// Counters.  One 32-bit shared-memory word per (trial, phase slot), private to
// its thread and laid out [trial][slot][thread] so a warp's accesses fall in
// distinct banks.  Without overlapping bins the low 16 bits count points
// (N <= 65535) and the high 16 bits hold a snapshot taken at the end of the
// previous magnitude segment, so the segment's c_ij is low - high; with them,
// short curves pack two segments' counts and the cumulative count into the word
// (FMT_PK2 below).  Points are counted with a shared-memory atomic add whose
// result is unused: it needs no read-modify-write round trip in the thread, and
// no other thread touches the word.
//
// Entropy.  N H = sum_j c_j ln c_j - sum_ij c_ij ln c_ij, accumulated as exact
// 64-bit integers from a fixed-point c ln c table (2^32 scale); H is converted
// to float32 once per trial.
#pragma once

#include <cmath>
#include <cstdint>

#include "gce_internal.cuh"

namespace gce {

namespace {

constexpr unsigned long long kNoKey = ~0ull;

// Warp minimum of (H bits, trial index) keys by two single-instruction warp
// reductions: the smallest high word, then the smallest low word among the
// lanes holding it (the same order as the 64-bit key).
__device__ __forceinline__ unsigned long long warp_min_key(unsigned long long v) {
    const unsigned int hi = (unsigned int)(v >> 32);
    const unsigned int mh = __reduce_min_sync(0xffffffffu, hi);
    const unsigned int ml = __reduce_min_sync(0xffffffffu, hi == mh ? (unsigned int)v : 0xffffffffu);
    return ((unsigned long long)mh << 32) | ml;
}


// Per-mode constants of the fold, computed once per kernel.
struct FoldConst {
    double nphi_d;
    float nphi_f;
    float zoff;          // SPLIT32: 1.5 2^23 + n_phase
    int n_phase;
#if defined(GCE_CHECK_SLOTS)
    // checked builds: the trial's kept logical slots and where to flag a miss
    int zmin, zmax;
    unsigned int *err;
#endif
};

__device__ __forceinline__ FoldConst fold_const(int n_phase) {
    FoldConst k;
    k.nphi_d = (double)n_phase;
    k.nphi_f = (float)n_phase;
    k.zoff = kRound + (float)n_phase;
    k.n_phase = n_phase;
    return k;
}

// Fold<MODE> turns a trial's stored constants into the registers its fold
// needs (prepare) and folds one point into a raw counter slot: the phase bin
// (FP64, FIXED32) or, for SPLIT32, the bit pattern of the rounding FMA, whose
// offset kSlotBias is removed once from the counter base address instead of
// per point.  raw - kSlotBias is the bin, or for SPLIT32 the bin or the bin
// plus n_phase (two slots per bin).
// fpart / offset_from split the fold at its period part (what trials of the same
// period share); offset is the two composed, so every path folds identically.
template <int MODE> struct Fold;
template <> struct Fold<GCE_PHASE_FP64> {
    typedef double2 prep_t;
    typedef double fpart_t;
    static constexpr int kSlotBias = 0;
    __device__ __forceinline__ static prep_t prepare(double2 t) { return t; }
    template <bool PDOT>
    __device__ __forceinline__ static int raw_slot(double p, const prep_t &t, const FoldConst &k) {
        return fold_fp64<PDOT>(p, t.x, t.y, k.nphi_d, k.n_phase);
    }
    __device__ __forceinline__ static fpart_t fpart(double p, const prep_t &t) {
        return fold_fp64_fpart(p, t.x);
    }
    template <bool PDOT, bool K0, int SH, bool RED>
    __device__ __forceinline__ static unsigned int offset_from(fpart_t f, double p,
                                                               const prep_t &t,
                                                               const FoldConst &k) {
        return (unsigned int)fold_fp64_from<PDOT>(f, p, t.y, k.nphi_d, k.n_phase) << SH;
    }
    template <bool PDOT, bool K0, int SH, bool RED>
    __device__ __forceinline__ static unsigned int offset(double p, const prep_t &t,
                                                          const FoldConst &k) {
        return offset_from<PDOT, K0, SH, RED>(fpart(p, t), p, t, k);
    }
    __device__ __forceinline__ static bool has_pdot(double2 t) { return t.y != 0.0; }
    __device__ __forceinline__ static bool k_zero(const prep_t &) { return true; }
};
template <> struct Fold<GCE_PHASE_SPLIT32> {
    typedef float4 prep_t;
    typedef float fpart_t;
    static constexpr int kSlotBias = 0x4B400000;  // bits of 1.5 2^23
    __device__ __forceinline__ static prep_t prepare(float4 t) { return t; }
    template <bool PDOT>
    __device__ __forceinline__ static int raw_slot(float4 p, const prep_t &t, const FoldConst &k) {
        return fold_split<PDOT>(p, t, k.nphi_f, k.zoff) + kSlotBias;
    }
    __device__ __forceinline__ static fpart_t fpart(float4 p, const prep_t &t) {
        return fold_split_fpart(p, t);
    }
    // RED: re-reduce the residual without Pdot as well (narrow slot window)
    template <bool PDOT, bool K0, int SH, bool RED>
    __device__ __forceinline__ static unsigned int offset_from(fpart_t f, float4 p,
                                                               const prep_t &t,
                                                               const FoldConst &k) {
        return (unsigned int)(fold_split_from<PDOT, RED>(f, p, t, k.nphi_f, k.zoff) + kSlotBias)
               << SH;
    }
    template <bool PDOT, bool K0, int SH, bool RED>
    __device__ __forceinline__ static unsigned int offset(float4 p, const prep_t &t,
                                                          const FoldConst &k) {
        return offset_from<PDOT, K0, SH, RED>(fpart(p, t), p, t, k);
    }
    __device__ __forceinline__ static bool has_pdot(float4 t) {
        return t.z != 0.0f || t.w != 0.0f;
    }
    __device__ __forceinline__ static bool k_zero(const prep_t &) { return true; }
};
template <> struct Fold<GCE_PHASE_FIXED32> {
    typedef FixedPrep prep_t;
    typedef unsigned int fpart_t;
    static constexpr int kSlotBias = 0;
    __device__ __forceinline__ static prep_t prepare(const FixedTrial &t) { return fixed_prep(t); }
    template <bool PDOT>
    __device__ __forceinline__ static int raw_slot(uint4 p, const prep_t &t, const FoldConst &k) {
        return fold_fixed<PDOT>(p, t, (unsigned int)k.n_phase);
    }
    __device__ __forceinline__ static fpart_t fpart(uint4 p, const prep_t &t) {
        return fold_fixed_fpart(p, t);
    }
    template <bool PDOT, bool K0, int SH, bool RED>
    __device__ __forceinline__ static unsigned int offset_from(fpart_t f, uint4 p, const prep_t &t,
                                                               const FoldConst &k) {
        return fold_fixed_bin_from<PDOT, K0>(f, p, t, (unsigned int)k.n_phase) << SH;
    }
    template <bool PDOT, bool K0, int SH, bool RED>
    __device__ __forceinline__ static unsigned int offset(uint4 p, const prep_t &t,
                                                          const FoldConst &k) {
        return offset_from<PDOT, K0, SH, RED>(fpart(p, t), p, t, k);
    }
    __device__ __forceinline__ static bool has_pdot(const FixedTrial &t) {
        return (t.i.z | t.i.w) != 0u;
    }
    __device__ __forceinline__ static bool k_zero(const prep_t &t) { return t.k == 0u; }
};

// The increment carries no memory clobber, so the compiler may schedule the
// next points' shared loads around it; compiler_fence() before and after each
// hot loop keeps the counters' plain loads and stores on their side of it.
__device__ __forceinline__ void red_shared_add(unsigned int addr, unsigned int inc) {
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(addr), "r"(inc));
}
__device__ __forceinline__ void compiler_fence() { asm volatile("" ::: "memory"); }

// One point folded for the thread's TPT trials and counted into their private
// counters.  base[s]: shared-memory address of trial s's logical slot 0 minus
// the mode's slot bias (mod 2^32); a slot's word is base + (raw << SH), SH =
// log2(4 block).  Each point counts once, in its fine phase bin, also with
// 50 %-overlapping bins (their counts are sums of adjacent fine bins, formed in
// the epilogue).  SHARED: the thread's trials share their period (period-major
// tiles), so the fold's period part is computed once for all of them.
template <int MODE, int TPT, int SH, bool PDOT, bool K0, bool RED, bool SHARED>
__device__ __forceinline__ void count_point(const typename ModeTraits<MODE>::point_t &p,
                                            const typename Fold<MODE>::prep_t (&tc)[TPT],
                                            const unsigned int (&base)[TPT], const FoldConst &fk,
                                            unsigned int inc) {
    typename Fold<MODE>::fpart_t fp{};
    if (SHARED) fp = Fold<MODE>::fpart(p, tc[0]);
#pragma unroll
    for (int s = 0; s < TPT; ++s) {
        const unsigned int addr =
            base[s] + (SHARED ? Fold<MODE>::template offset_from<PDOT, K0, SH, RED>(fp, p, tc[s], fk)
                              : Fold<MODE>::template offset<PDOT, K0, SH, RED>(p, tc[s], fk));
#if defined(GCE_CHECK_SLOTS)
        // checked builds: the logical slot of this increment must lie in the
        // kept range; a miss is flagged and the access skipped
        const int lslot =
            (int)(addr - (base[s] + ((unsigned int)Fold<MODE>::kSlotBias << SH))) >> SH;
        if (lslot < fk.zmin || lslot > fk.zmax) {
            atomicOr(fk.err, (unsigned int)ERR_SLOT);
            continue;
        }
#endif
        red_shared_add(addr, inc);
    }
}

// Two half points from one 16-byte word.
__device__ __forceinline__ void split_pair(const float4 &q, float2 &a, float2 &b) {
    a = make_float2(q.x, q.y);
    b = make_float2(q.z, q.w);
}
__device__ __forceinline__ void split_pair(const uint4 &q, uint2 &a, uint2 &b) {
    a = make_uint2(q.x, q.y);
    b = make_uint2(q.z, q.w);
}
template <class H> struct PairOf;
template <> struct PairOf<float2> { typedef float4 type; };
template <> struct PairOf<uint2> { typedef uint4 type; };

// The hot loop: every point of [ka, kb) (shared memory, broadcast) through
// count_point.  HALF: the staged points are half points (no Pdot term anywhere
// in the job); PAIRS below reads them two per 16-byte shared load (the chunk
// starts 16-byte aligned; a segment starting at an odd index takes its first
// point alone).
template <int MODE, int TPT, int SH, bool PDOT, bool K0, bool RED, bool SHARED, bool HALF>
__device__ __forceinline__ void count_points(
    const void *__restrict__ pts, int ka, int kb,
    const typename Fold<MODE>::prep_t (&tc)[TPT], const unsigned int (&base)[TPT],
    const FoldConst &fk, unsigned int inc) {
    typedef ModeTraits<MODE> MT;
    static_assert(!(HALF && PDOT), "half points carry no tau^2");
    // points unrolled by 16 (8 with the longer Pdot fold): measured faster than 8
    // and 4 on every workload without a Pdot axis, and than 16 with one
    constexpr int UNROLL = PDOT ? 8 : 16;
    // pairs measured faster with one trial per thread (+20 % at 50 overlapping
    // bins, where one point load serves one trial) and with FIXED32 (+5 % at
    // four trials), slower with SPLIT32 at two or four trials (-5 %, -1 %)
    constexpr bool PAIRS = HALF && (TPT == 1 || MODE == GCE_PHASE_FIXED32);
    if constexpr (PAIRS) {
        typedef typename MT::half_t half_t;
        typedef typename PairOf<half_t>::type pair_t;
        const half_t *hp = static_cast<const half_t *>(pts);
        int k = ka;
        if ((k & 1) && k < kb) {
            count_point<MODE, TPT, SH, PDOT, K0, RED, SHARED>(MT::widen(hp[k]), tc, base, fk, inc);
            ++k;
        }
        constexpr int UNROLL2 = UNROLL / 2;
#pragma unroll UNROLL2
        for (; k + 1 < kb; k += 2) {
            const pair_t q = *reinterpret_cast<const pair_t *>(hp + k);
            half_t h0, h1;
            split_pair(q, h0, h1);
            count_point<MODE, TPT, SH, PDOT, K0, RED, SHARED>(MT::widen(h0), tc, base, fk, inc);
            count_point<MODE, TPT, SH, PDOT, K0, RED, SHARED>(MT::widen(h1), tc, base, fk, inc);
        }
        if (k < kb)
            count_point<MODE, TPT, SH, PDOT, K0, RED, SHARED>(MT::widen(hp[k]), tc, base, fk, inc);
    } else {
#pragma unroll UNROLL
        for (int k = ka; k < kb; ++k) {
            const typename MT::point_t p =
                HALF ? MT::widen(static_cast<const typename MT::half_t *>(pts)[k])
                     : static_cast<const typename MT::point_t *>(pts)[k];
            count_point<MODE, TPT, SH, PDOT, K0, RED, SHARED>(p, tc, base, fk, inc);
        }
    }
}

template <int MODE, int TPT, int SH, bool PDOT, bool K0, bool RED = false, bool HALF = false>
__device__ __forceinline__ void count_points_any(
    bool shared, const void *__restrict__ pts, int ka, int kb,
    const typename Fold<MODE>::prep_t (&tc)[TPT], const unsigned int (&base)[TPT],
    const FoldConst &fk, unsigned int inc) {
    constexpr bool SH_OK = PDOT && TPT > 1;  // sharing pays only with a Pdot term
    if (SH_OK && shared) count_points<MODE, TPT, SH, PDOT, K0, RED, SH_OK, HALF>(pts, ka, kb, tc, base, fk, inc);
    else count_points<MODE, TPT, SH, PDOT, K0, RED, false, HALF>(pts, ka, kb, tc, base, fk, inc);
}

// c_ij of one phase bin at the end of a magnitude segment (low - snapshot), with
// the snapshot moved up to the current count: the new word is cur:cur (a byte
// permute), and new - old = (cur - prev) << 16.
__device__ __forceinline__ int take_segment(unsigned int *w) {
    const unsigned int v = *w;
    const unsigned int nv = __byte_perm(v, 0u, 0x1010);
    *w = nv;
    return (int)((nv - v) >> 16);
}

// Counter word formats.  Each (trial, slot) has one 32-bit shared word.
//   FMT_SNAP: (snapshot << 16) | count, for curves of up to 65535 points.  The
//     count is cumulative; the snapshot is the count at the end of the previous
//     magnitude segment, so the segment's count is count - snapshot.
//   FMT_PK2: (C << 20) | (B << 10) | A, for curves of at most kPk2MaxN points.
//     Consecutive non-empty magnitude segments alternate between the fields A
//     and B, and every point also counts in C, the cumulative count (the
//     increment is 1 + 2^20 or 2^10 + 2^20: still one shared atomic).  One sweep
//     then serves two segments: it reads A and B and clears them.
// No field can overflow: each is at most the curve's point count.  Nor can the
// field-wise sum of two words of different fine bins (the points are disjoint),
// so with FMT_PK2 an overlapping bin's counts are read from the sum of its two
// fine words (kPairWords).
enum { FMT_SNAP = 0, FMT_PK2 = 1 };
constexpr int kPk2MaxN = 1023;
constexpr unsigned int kPk2IncB = 1u << 10;
constexpr unsigned int kPk2IncC = 1u << 20;

// Per counter word: the byte offsets 8 c into the c ln c table of the counts a
// sweep reads, and the word it leaves behind.
// What a sweep reads from each counter word.
enum { SW_SEG = 0, SW_LAST = 1 };
//   SW_SEG:  the counts of the segments since the last sweep (subtracted: the
//            Sigma_ij T(c_ij) term), the word left with them moved to the
//            cumulative part;
//   SW_LAST: after the curve's last segment, those counts and the cumulative
//            count c_j (added: the Sigma_j T(c_j) term), the word cleared.
// Fields<FMT, KIND>::get returns the byte offsets 8 c into the c ln c table of
// the NF counts, and the word to store back; sign(f) says whether count f is
// added (+1) or subtracted (-1).  With kPairWords the offsets of a word (or of a
// field-wise sum of words) and the word to store back are also available apart
// (offsets, next).
template <int FMT, int KIND> struct Fields;
template <> struct Fields<FMT_SNAP, SW_SEG> {
    static constexpr int NF = 1;
    static constexpr bool kPairWords = false;
    __device__ __forceinline__ static int sign(int) { return -1; }
    __device__ __forceinline__ static unsigned int get(unsigned int v, unsigned int (&o)[1]) {
        const unsigned int nv = __byte_perm(v, 0u, 0x1010);  // snapshot moved up
        o[0] = (nv - v) >> 13;
        return nv;
    }
    // an extra slot's segment count joins its bin's first word
    __device__ __forceinline__ static unsigned int merge(unsigned int first, unsigned int extra) {
        return first + (extra & 0xffffu) - (extra >> 16);
    }
};
template <> struct Fields<FMT_SNAP, SW_LAST> {
    static constexpr int NF = 2;
    static constexpr bool kPairWords = false;
    __device__ __forceinline__ static int sign(int f) { return f == 0 ? -1 : 1; }
    __device__ __forceinline__ static unsigned int get(unsigned int v, unsigned int (&o)[2]) {
        o[0] = (__byte_perm(v, 0u, 0x1010) - v) >> 13;
        o[1] = (v & 0xffffu) << 3;
        return 0u;
    }
    __device__ __forceinline__ static unsigned int merge(unsigned int first, unsigned int extra) {
        return Fields<FMT_SNAP, SW_SEG>::merge(first, extra);
    }
};
template <> struct Fields<FMT_PK2, SW_SEG> {  // segments A and B; both cleared
    static constexpr int NF = 2;
    static constexpr bool kPairWords = true;
    __device__ __forceinline__ static int sign(int) { return -1; }
    __device__ __forceinline__ static void offsets(unsigned int w, unsigned int (&o)[2]) {
        o[0] = (w << 3) & 0x1ff8u;
        o[1] = (w >> 7) & 0x1ff8u;
    }
    __device__ __forceinline__ static unsigned int next(unsigned int v) { return v & 0xfff00000u; }
    __device__ __forceinline__ static unsigned int get(unsigned int v, unsigned int (&o)[2]) {
        offsets(v, o);
        return next(v);
    }
    __device__ __forceinline__ static unsigned int merge(unsigned int first, unsigned int extra) {
        return first + extra;
    }
};
template <> struct Fields<FMT_PK2, SW_LAST> {  // A, B and the cumulative C; word cleared
    static constexpr int NF = 3;
    static constexpr bool kPairWords = true;
    __device__ __forceinline__ static int sign(int f) { return f == 2 ? 1 : -1; }
    __device__ __forceinline__ static void offsets(unsigned int w, unsigned int (&o)[3]) {
        o[0] = (w << 3) & 0x1ff8u;
        o[1] = (w >> 7) & 0x1ff8u;
        o[2] = (w >> 17) & 0x7ff8u;
    }
    __device__ __forceinline__ static unsigned int next(unsigned int) { return 0u; }
    __device__ __forceinline__ static unsigned int get(unsigned int v, unsigned int (&o)[3]) {
        offsets(v, o);
        return next(v);
    }
    __device__ __forceinline__ static unsigned int merge(unsigned int first, unsigned int extra) {
        return first + extra;
    }
};

// The entropy sweep: for each of the thread's TPT trials, the c ln c terms,
// T(c) = c ln c from the fixed-point table, of every count the word format and
// the sweep kind hold, added to or subtracted from acc (N H 2^32, Eq. 4 as
// Sigma_j T(c_j) - Sigma_ij T(c_ij)).  The trial's counters for the window of
// logical slots [L, R] start at word w0[s] (slot L), STRIDE words apart; slot
// L + i counts bin (L + i) mod n, so the first n slots hold one bin each and
// the e = R - L + 1 - n extra slots L + n + i more points of the bin of slot
// L + (i mod n) (SPLIT32's two slots per bin).  Each extra word is first merged
// into its bin's first word and cleared, so the sweep proper reads one word per
// bin.  SW_LAST clears every word it reads, so the next work item starts from
// zero counters without a separate pass.
// OVL (50 %-overlapping bins, Sec. 2.3): overlapping bin j holds the fine bins j
// and j + 1 (mod n), so the sum is over T(c_j + c_(j+1)): the first bin is
// peeled off, each later bin pairs with the one before it, and the last pairs
// with the first (table offsets add like the counts).  G bins of every trial
// are loaded before any is stored, so the loads overlap.
template <int TPT, int FMT, int KIND, bool ALL_SMEM, bool OVL, int STRIDE>
struct Sweep {
    typedef Fields<FMT, KIND> F;
    static constexpr int NF = F::NF;
    unsigned int *const cnt;               // the thread's counter words
    const unsigned long long *const s_tab;  // the c ln c table in shared memory
    const int table_smem;
    const unsigned long long *const g_tab;
    // OVL: the first bin's and the previous bin's offsets, or with kPairWords
    // their words ([s][0])
    unsigned int first[TPT][NF] = {}, prev[TPT][NF] = {};

    // T(c) for the byte offset o = 8 c
    __device__ __forceinline__ unsigned long long look(unsigned int o) const {
        const unsigned long long *e = reinterpret_cast<const unsigned long long *>(
            reinterpret_cast<const char *>(s_tab) + o);
        if (ALL_SMEM) return *e;
        const int c = (int)(o >> 3);
        return c < table_smem ? *e : __ldg(g_tab + c);
    }
    __device__ __forceinline__ static void add(unsigned long long &t, int f, unsigned long long x) {
        if (F::sign(f) > 0) t += x;
        else t -= x;
    }

    // G bins of trial s at words cnt[w[s]], cnt[w[s] + STRIDE], ...; PEEL: the
    // first bin of an OVL sweep
    template <int G, bool PEEL>
    __device__ __forceinline__ void step(int (&w)[TPT], unsigned long long (&acc)[TPT]) {
        unsigned int v[TPT][G];
#pragma unroll
        for (int s = 0; s < TPT; ++s)
#pragma unroll
            for (int g = 0; g < G; ++g) v[s][g] = cnt[w[s] + g * STRIDE];
        unsigned long long t[TPT];
#pragma unroll
        for (int s = 0; s < TPT; ++s) {
            t[s] = 0ull;
#pragma unroll
            for (int g = 0; g < G; ++g) {
                unsigned int o[NF];
                if constexpr (OVL && F::kPairWords) {
                    // the overlapping bin's counts from the sum of its fine words
                    const unsigned int w0 = v[s][g];
                    if (PEEL && g == 0) {
                        first[s][0] = w0;
                    } else {
                        F::offsets(prev[s][0] + w0, o);
#pragma unroll
                        for (int f = 0; f < NF; ++f) add(t[s], f, look(o[f]));
                    }
                    prev[s][0] = w0;
                    v[s][g] = F::next(w0);
                } else {
                    v[s][g] = F::get(v[s][g], o);  // v now holds the word to store
#pragma unroll
                    for (int f = 0; f < NF; ++f) {
                        if (OVL) {
                            if (PEEL && g == 0) first[s][f] = o[f];
                            else add(t[s], f, look(prev[s][f] + o[f]));
                            prev[s][f] = o[f];
                        } else {
                            add(t[s], f, look(o[f]));
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int s = 0; s < TPT; ++s) {
#pragma unroll
            for (int g = 0; g < G; ++g) cnt[w[s] + g * STRIDE] = v[s][g];
            acc[s] += t[s];
            w[s] += G * STRIDE;
        }
    }

    // w0[s]: word offset (from cnt) of trial s's first window slot; e: extra
    // slots, merged first
    __device__ __forceinline__ void run(const int (&w0)[TPT], int n, int e,
                                        unsigned long long (&acc)[TPT]) {
        {
            for (int i = 0, b = 0; i < e; ++i, b = (b + 1 == n) ? 0 : b + 1) {
#pragma unroll
                for (int s = 0; s < TPT; ++s) {
                    unsigned int *q = cnt + w0[s] + (n + i) * STRIDE;
                    unsigned int *f = cnt + w0[s] + b * STRIDE;
                    const unsigned int x = *q;
                    *q = 0u;
                    *f = F::merge(*f, x);
                }
            }
        }
        int w[TPT];
#pragma unroll
        for (int s = 0; s < TPT; ++s) w[s] = w0[s];
        // bins per step: four to eight words in flight, eight bins with one trial
        // per thread (+1 % over four at 50 overlapping bins)
        constexpr int G = TPT * NF >= 4 ? 2 : (TPT == 1 ? 8 : 4);
        int j = 0;
        if (OVL) {
            step<1, true>(w, acc);
            j = 1;
        }
        for (; j + G <= n; j += G) step<G, false>(w, acc);
        if (G > 4 && (n - j) >= 4) {
            step<4, false>(w, acc);
            j += 4;
        }
        if (G > 2 && (n - j) >= 2) {
            step<2, false>(w, acc);
            j += 2;
        }
        if (j < n) step<1, false>(w, acc);
        if constexpr (OVL && F::kPairWords) {
#pragma unroll
            for (int s = 0; s < TPT; ++s) {
                unsigned int o[NF];
                F::offsets(prev[s][0] + first[s][0], o);
#pragma unroll
                for (int f = 0; f < NF; ++f) add(acc[s], f, look(o[f]));
            }
        } else if (OVL) {
#pragma unroll
            for (int s = 0; s < TPT; ++s)
#pragma unroll
                for (int f = 0; f < NF; ++f) add(acc[s], f, look(prev[s][f] + first[s][f]));
        }
    }

};

// Dispatch of one work item's sweeps over the run-time choice of where the c ln c
// table is read (whole in shared memory, or shared below table_smem and global
// above).
template <int TPT, int STRIDE, bool OVL>
struct Sweeper {
    unsigned int *cnt;
    const unsigned long long *s_tab;
    int table_smem;
    const unsigned long long *g_tab;
    int n;  // phase bins

    template <int FMT, int KIND>
    __device__ __forceinline__ void run(bool tab_all, const int (&w0)[TPT], int e,
                                        unsigned long long (&acc)[TPT]) const {
        if (tab_all) Sweep<TPT, FMT, KIND, true, OVL, STRIDE>{cnt, s_tab, table_smem, g_tab}.run(w0, n, e, acc);
        else Sweep<TPT, FMT, KIND, false, OVL, STRIDE>{cnt, s_tab, table_smem, g_tab}.run(w0, n, e, acc);
    }
};

// The half point of a whole point (FP64 points are already one word).
__device__ __forceinline__ float2 half_of(const float4 &q) { return make_float2(q.x, q.y); }
__device__ __forceinline__ uint2 half_of(const uint4 &q) { return make_uint2(q.x, q.y); }
__device__ __forceinline__ double half_of(double q) { return q; }

// fh of a SPLIT32 trial (other modes: unused)
__device__ __forceinline__ float split_fh(const float4 &t) { return t.x; }
template <class T>
__device__ __forceinline__ float split_fh(const T &) { return 0.0f; }


// The slots a SPLIT32 fold can reach.  The fold's residual x obeys |x| <=
// 1/2 + 2^-23 |th fh| (1 + 2^-22) + 2^-23 without the Pdot term (the two
// cross terms are each below 2^-24 |th fh|, and three roundings), and |x| <=
// 1/2 exactly with it (x is re-rounded); the slot is floor(x n + n), monotone
// in x.  The bound is taken in FP32 with margins (a factor 1.01 and 2^-16)
// far above its own rounding; cyc_max >= max |tau| f over the warp's trials.
__device__ __forceinline__ void split_slot_window(bool pdot, float cyc_max, int n_phase, int &zlo,
                                                  int &zhi) {
    const float nf = (float)n_phase;
    const float xm = 0.5f + (pdot ? 0.0f : cyc_max * 1.2040e-7f) + 1.5259e-5f;  // 1.01 2^-23, 2^-16
    zlo = max((int)floorf(nf - nf * xm), 0);
    zhi = min((int)floorf(nf + nf * xm), 2 * n_phase - 1);
}

// Chan et al.'s pairwise update of (count, mean, M2) moments.
__device__ __forceinline__ void chan_merge(double &n, double &mean, double &m2, double nb,
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

// CTAs per SM the register allocation is sized for.  With two trials per
// thread the counters (and FP64's wider staged points) already limit shared
// memory to about three 256-thread CTAs per SM at 15 phase bins, so those
// kernels take the registers that frees (80 at 256 threads) instead of 64.
// Four trials per thread need four times the counters of one: at most 512
// threads per SM fit, and those kernels take up to 128 registers.  One trial
// per thread is the shape for many phase bins (50 and up), where the counters
// again leave room for about 512 threads per SM: 128 registers as well, except
// the 128-thread kernel with overlapping bins, whose counters in the mid slot
// range fit five CTAs per SM: 96 registers there (measured 3.6 % faster at 50
// overlapping bins than four CTAs at 121 registers).
constexpr int main_min_blocks(int tpt, int log2b, int kv) {
    return (kv == KV_OVL && tpt == 1 && log2b == 7) ? 5 :
           tpt == 2 ? (log2b >= 9 ? 2 : (log2b == 8 ? 3 : (log2b == 7 ? 6 : 8)))
                    : (log2b >= 9 ? 1 : (log2b == 8 ? 2 : (log2b == 7 ? 4 : 8)));
}

template <int MODE, int TPT, int LOG2B, int KV>
__global__ void __launch_bounds__(1 << LOG2B, main_min_blocks(TPT, LOG2B, KV)) k_main(MainArgs a) {
    // the counter formats are fixed per instantiation (a kernel that carried
    // the overlapping-bin format with a run-time choice measured slower on the
    // path that never used it)
    constexpr bool OVL = KV == KV_OVL;
    constexpr int FMT = FMT_SNAP;  // without overlapping bins
    typedef typename ModeTraits<MODE>::point_t point_t;
    typedef typename ModeTraits<MODE>::trial_t trial_t;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long s_item;

    if (a.state->err) return;  // inputs failed the device checks: no work

    constexpr int B = 1 << LOG2B;
    constexpr int SH = LOG2B + 2;  // log2 of the byte stride between a thread's slots
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n_phase = a.n_phase, n_mag = a.n_mag;
    constexpr bool SPLIT = MODE == GCE_PHASE_SPLIT32;
    constexpr int ovl = OVL ? 1 : 0;  // 50 %-overlapping phase bins
    const int range = SPLIT ? a.range : (int)RANGE_WIDE;
    const SlotRange zr = slot_range(MODE, n_phase, range);
    const int n_slots = slots_per_trial(MODE, n_phase, range);
    const int slot_off = -zr.zmin;  // physical index of logical slot l: l + slot_off
    const int stride_j = B, stride_s = n_slots * B;

    // the regions at the offsets the host sized the launch with (the table first,
    // so that its address is a constant)
    const MainSmemLayout lay = main_smem_layout(MODE, B, TPT, a.chunk, n_phase, n_mag, a.table_smem,
                                                range, a.half);
    unsigned long long *s_tab = reinterpret_cast<unsigned long long *>(smem);
    point_t *s_pts = reinterpret_cast<point_t *>(smem + lay.pts);
    unsigned int *s_cnt = reinterpret_cast<unsigned int *>(smem + lay.cnt);
    int *s_seg = reinterpret_cast<int *>(smem + lay.seg);

    for (int i = tid; i < a.table_smem; i += B) s_tab[i] = a.table[i];

    const point_t *g_pts = reinterpret_cast<const point_t *>(a.payload);
    const trial_t *g_tr = reinterpret_cast<const trial_t *>(a.trialc);
    unsigned int *my_cnt = s_cnt + tid;
    // counters start at zero; every work item's final sweep clears the words it
    // used, so later items start from zero as well
    for (int i = 0; i < TPT * n_slots; ++i) my_cnt[i * B] = 0u;
#if defined(GCE_CHECK_SLOTS)
    FoldConst fk = fold_const(n_phase);
    fk.zmin = zr.zmin;
    fk.zmax = zr.zmax;
    fk.err = &a.state->err;
#else
    const FoldConst fk = fold_const(n_phase);
#endif
    unsigned int base[TPT];
    unsigned int *wbase[TPT];  // physical slot 0 of trial s
#pragma unroll
    for (int s = 0; s < TPT; ++s) {
        wbase[s] = my_cnt + s * stride_s;
        base[s] = (unsigned int)__cvta_generic_to_shared(wbase[s]) + ((unsigned int)slot_off << SH) -
                  ((unsigned int)Fold<MODE>::kSlotBias << SH);
    }
    // a job whose Pdot values are all 0 stages half points (a.half); one whose
    // single Pdot value is not 0 stages whole points, half as many per chunk
    const bool job_pdot = a.state->pdot_max_bits != 0ull;
    const bool half = a.half != 0 && !job_pdot;
    const int chunk_pts = (a.half != 0 && job_pdot) ? (a.chunk >> 1) : a.chunk;
    // max |tau| of the job (SPLIT32 slot windows), rounded up to FP32
    const float tau_max_f =
        SPLIT ? __double2float_ru(__longlong_as_double((long long)a.state->tau_max_bits)) : 0.0f;

    int staged_curve = -1, staged_lo = -1;
    // the tile whose trial constants, flags and counter window are loaded: work
    // items of the same tile reuse them
    int cur_tile = -1;
    typename Fold<MODE>::prep_t tc[TPT];
    long long tt[TPT];
    bool pdot = false, k0 = true;
    bool red = false;  // SPLIT32: this warp's folds re-reduce the residual (narrow window)
    const bool pdm = a.pd_major != 0;
    int wl[TPT];           // word offset (from my_cnt) of each trial's first window slot

    int n_extra = 0;       // window slots beyond n_phase
    long long item = 0, item_end = 0;
    for (;;) {
        if (item >= item_end) {
            __syncthreads();
            if (tid == 0) s_item = (long long)atomicAdd(&a.state->work, (unsigned long long)a.grab);
            __syncthreads();
            item = s_item;
            item_end = min(item + (long long)a.grab, a.n_items);
            if (item >= a.n_items) break;
        }
        // items [0, n_long_items) run curve-major over the long curves (consecutive
        // items share the staged curve); the rest tile-major over the short curves
        // at the end of the order (consecutive items share the tile's trials)
        int ci, tile;
        if (item < a.n_long_items) {
            ci = (int)(item / a.n_tiles);
            tile = (int)(item - (long long)ci * a.n_tiles);
        } else {
            const long long j = item - a.n_long_items;
            tile = (int)(j / a.n_short);
            ci = a.n_long + (int)(j - (long long)tile * a.n_short);
        }
        const int c = a.order[ci];
        const long long off = a.offsets[c];
        const int n = (int)(a.offsets[c + 1] - off);
        const bool tab_all = n < a.table_smem;  // every count of this curve is <= n
        if (c != staged_curve) {
            __syncthreads();
            for (int i = tid; i <= n_mag; i += B) s_seg[i] = a.seg[(long long)c * (n_mag + 1) + i];
            staged_curve = c;
            staged_lo = -1;
        }

        if (tile != cur_tile) {
            cur_tile = tile;
            bool any_pdot = false, all_k0 = true;
            // trial indices (n_trials marks a slot past the grid): a run of B x TPT
            // flat indices, or B periods x TPT Pdot values (period-major tiles)
            long long p_idx = 0;
            int q_base = 0;
            if (pdm) {
                p_idx = (long long)(tile % a.n_ptiles) * B + tid;
                q_base = (tile / a.n_ptiles) * TPT;
            }
#pragma unroll
            for (int s = 0; s < TPT; ++s) {
                if (pdm)
                    tt[s] = (p_idx < a.n_periods && q_base + s < a.n_pdots)
                                ? (long long)(q_base + s) * a.n_periods + p_idx
                                : a.n_trials;
                else
                    tt[s] = (long long)tile * (B * TPT) + (long long)s * B + tid;
                trial_t tr{};
                if (tt[s] < a.n_trials) {
                    tr = g_tr[tt[s]];
                    any_pdot |= Fold<MODE>::has_pdot(tr);
                }
                tc[s] = Fold<MODE>::prepare(tr);
                all_k0 &= Fold<MODE>::k_zero(tc[s]);
            }
            // the fold variant is chosen per warp (a warp vote, no CTA barrier)
            pdot = __any_sync(0xffffffffu, any_pdot);
            k0 = MODE != GCE_PHASE_FIXED32 || __all_sync(0xffffffffu, all_k0);
            // live logical slots [L, R] of this warp's counters (warp-uniform)
            int L = 0, R = n_phase - 1;
            if (SPLIT) {
                float fm = 0.0f;
#pragma unroll
                for (int s = 0; s < TPT; ++s)
                    if (tt[s] < a.n_trials) fm = fmaxf(fm, fabsf(split_fh(tc[s])));
                fm = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(fm)));
                // folds without a Pdot term re-reduce their residual with the
                // narrow range, and with the mid one where the warp's cycles
                // could fold outside it (a fold with a Pdot term always does)
                red = !pdot && range == RANGE_NARROW;
                int zlo, zhi;
                split_slot_window(pdot || red, tau_max_f * fm, n_phase, zlo, zhi);
                if (!pdot && range == RANGE_MID && (zlo < zr.zmin || zhi > zr.zmax)) {
                    red = true;
                    split_slot_window(true, tau_max_f * fm, n_phase, zlo, zhi);
                }
                L = max(zlo, zr.zmin);
                R = min(zhi, zr.zmax);
            }
#pragma unroll
            for (int s = 0; s < TPT; ++s) wl[s] = s * stride_s + (L + slot_off) * stride_j;
            n_extra = R - L + 1 - n_phase;

#if defined(GCE_CHECK_SLOTS)
            // checked builds: every increment must also lie in the warp's window
            fk.zmin = L;
            fk.zmax = R;
#endif
        }

        // N H 2^32 per trial (Eq. 4 as Sigma_j T(c_j) - Sigma_ij T(c_ij)), exact
        // modulo 2^64 while it is summed, non-negative at the end
        unsigned long long nh[TPT];
#pragma unroll
        for (int s = 0; s < TPT; ++s) nh[s] = 0ull;

        // FMT_PK2 (one sweep per two non-empty segments) with 50 %-overlapping
        // bins on curves of at most kPk2MaxN points, else the kernel's format (one
        // sweep per segment).  Each count costs the same table lookup and 64-bit add in both
        // formats; FMT_PK2 saves the loads, stores and the overlapping pairs' set-up
        // of every other sweep, which pays with overlapping bins and costs more
        // field arithmetic than it saves without them.
        const bool pk2 = ovl && n <= kPk2MaxN;
        const Sweeper<TPT, B, OVL> sw{my_cnt, s_tab, a.table_smem, a.table, n_phase};
        int ended = 0;  // non-empty segments ended so far (FMT_PK2: field = ended & 1)
        for (int lo = 0; lo < n; lo += chunk_pts) {
            const int hi = min(n, lo + chunk_pts);
            if (staged_lo != lo) {
                __syncthreads();
                const point_t *src = g_pts + off + lo;
                if (half) {
                    typedef typename ModeTraits<MODE>::half_t half_t;
                    half_t *s_half = reinterpret_cast<half_t *>(s_pts);
                    for (int k = tid; k < hi - lo; k += B) {
                        const point_t q = src[k];
                        s_half[k] = half_of(q);
                    }
                } else {
                    for (int k = tid; k < hi - lo; k += B) s_pts[k] = src[k];
                }
                __syncthreads();
                staged_lo = lo;
            }
            for (int i = 0; i < n_mag; ++i) {
                const int s0 = s_seg[i], s1 = s_seg[i + 1];
                const int ka = max(s0, lo), kb = min(s1, hi);
                if (ka < kb) {
                    const unsigned int inc = pk2 ? ((ended & 1) ? kPk2IncB : 1u) + kPk2IncC : 1u;
                    compiler_fence();
                    const void *pp = s_pts;
                    constexpr bool HP = MODE != GCE_PHASE_FP64;  // half points exist
                    if (k0) {
                        if (pdot) count_points_any<MODE, TPT, SH, true, true>(pdm, pp, ka - lo, kb - lo, tc, base, fk, inc);
                        // (red: the warp's slot window is the narrow one, so its folds
                        // must re-reduce, with half points as with whole ones)
                        else if (SPLIT && red && half) count_points_any<MODE, TPT, SH, false, true, SPLIT, HP>(pdm, pp, ka - lo, kb - lo, tc, base, fk, inc);
                        else if (SPLIT && red) count_points_any<MODE, TPT, SH, false, true, SPLIT>(pdm, pp, ka - lo, kb - lo, tc, base, fk, inc);
                        else if (HP && half) count_points_any<MODE, TPT, SH, false, true, false, HP>(pdm, pp, ka - lo, kb - lo, tc, base, fk, inc);
                        else count_points_any<MODE, TPT, SH, false, true>(pdm, pp, ka - lo, kb - lo, tc, base, fk, inc);
                    } else if (MODE == GCE_PHASE_FIXED32) {
                        if (pdot) count_points_any<MODE, TPT, SH, true, false>(pdm, pp, ka - lo, kb - lo, tc, base, fk, inc);
                        else if (half) count_points_any<MODE, TPT, SH, false, false, false, HP>(pdm, pp, ka - lo, kb - lo, tc, base, fk, inc);
                        else count_points_any<MODE, TPT, SH, false, false>(pdm, pp, ka - lo, kb - lo, tc, base, fk, inc);
                    }
                    compiler_fence();
                }
                if (s1 > s0 && s1 > lo && s1 <= hi) {
                    // end of non-empty magnitude segment i: sweep its counts (FMT_PK2:
                    // after every second one); after the curve's last segment one sweep
                    // takes its counts and the cumulative ones (the marginal term) and
                    // clears the counters for the next item
                    if (s1 == n) {
                        if (pk2) sw.run<FMT_PK2, SW_LAST>(tab_all, wl, n_extra, nh);
                        else sw.run<FMT, SW_LAST>(tab_all, wl, n_extra, nh);
                    } else if (!pk2) {
                        sw.run<FMT, SW_SEG>(tab_all, wl, n_extra, nh);
                    } else if (ended & 1) {
                        sw.run<FMT_PK2, SW_SEG>(tab_all, wl, n_extra, nh);
                    }
                    ++ended;
                }
            }
        }

        // H (the counts total 2N with overlapping bins, every point being in two)
        const double inv = kTabInvScale / (double)(n * (1 + ovl));
        unsigned long long key[TPT];
        float hv[TPT];
#pragma unroll
        for (int s = 0; s < TPT; ++s) {
            long long d = (long long)nh[s];
            if (d < 0) d = 0;
            const float h = __double2float_rn(__dmul_rn(__ll2double_rn(d), inv));
            hv[s] = h;
            key[s] = kNoKey;
            if (tt[s] < a.n_trials) {
                if (a.out) a.out[(long long)c * a.n_trials + tt[s]] = h;
                key[s] = ((unsigned long long)__float_as_uint(h) << 32) | (unsigned long long)tt[s];
            }
        }

        // each warp writes its own candidate list and moments (list index: curve,
        // tile, warp), so the tile needs no barrier; the merge kernels take B / 32
        // lists per tile
        const long long list = ((long long)c * a.n_tiles + tile) * (B >> 5) + warp;
        if (a.stats) {
            // moments of the warp's H for the significance of Eq. 5: sums of H - shift
            // in FP32 (shift = lane 0's first value, so the sums stay small), then
            // (count, mean, M2) in FP64
            const float shift = __shfl_sync(0xffffffffu, hv[0], 0);
            float s1 = 0.f, s2 = 0.f, cnt = 0.f;
#pragma unroll
            for (int s = 0; s < TPT; ++s)
                if (tt[s] < a.n_trials) {
                    const float dd = hv[s] - shift;
                    s1 += dd;
                    s2 = __fmaf_rn(dd, dd, s2);
                    cnt += 1.f;
                }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                s1 += __shfl_xor_sync(0xffffffffu, s1, o);
                s2 += __shfl_xor_sync(0xffffffffu, s2, o);
                cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
            }
            if (lane == 0) {
                const double nw = cnt;
                TileStats *t = a.stats + list;
                t->n = nw;
                t->mean = nw > 0 ? (double)shift + (double)s1 / nw : 0.0;
                t->m2 = nw > 0 ? fmax((double)s2 - (double)s1 * (double)s1 / nw, 0.0) : 0.0;
            }
        }

        if (a.cand) {
            // the warp's k smallest keys: k rounds of warp minima
            unsigned long long *dst = a.cand + list * a.k;
            for (int r = 0; r < a.k; ++r) {
                unsigned long long mine = key[0];
#pragma unroll
                for (int s = 1; s < TPT; ++s) mine = key[s] < mine ? key[s] : mine;
                const unsigned long long m = warp_min_key(mine);
                if (lane == 0) dst[r] = m;
#pragma unroll
                for (int s = 0; s < TPT; ++s)
                    if (key[s] == m) key[s] = kNoKey;
            }
        }
        ++item;
    }
}


template <int MODE, int TPT, int LOG2B>
cudaError_t launch_main_t(int grid, size_t smem, const MainArgs &a, cudaStream_t s) {
    switch (a.kv) {
        case KV_SNAP: k_main<MODE, TPT, LOG2B, KV_SNAP><<<grid, 1 << LOG2B, smem, s>>>(a); break;
        case KV_OVL: k_main<MODE, TPT, LOG2B, KV_OVL><<<grid, 1 << LOG2B, smem, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// The kernel instantiations: mode x trials per thread x block size.
template <int MODE, int TPT, int KV>
const void *kernel_for_block(int block) {
    switch (block) {
        case 64: return (const void *)k_main<MODE, TPT, 6, KV>;
        case 128: return (const void *)k_main<MODE, TPT, 7, KV>;
        case 256: return (const void *)k_main<MODE, TPT, 8, KV>;
        case 512: return (const void *)k_main<MODE, TPT, 9, KV>;
        default: return nullptr;
    }
}

template <int MODE, int TPT>
const void *kernel_for_variant(int block, int kv) {
    switch (kv) {
        case KV_SNAP: return kernel_for_block<MODE, TPT, KV_SNAP>(block);
        case KV_OVL: return kernel_for_block<MODE, TPT, KV_OVL>(block);
        default: return nullptr;
    }
}

template <int MODE, int TPT>
cudaError_t launch_for_block(int block, int grid, size_t smem, const MainArgs &a, cudaStream_t s) {
    switch (block) {
        case 64: return launch_main_t<MODE, TPT, 6>(grid, smem, a, s);
        case 128: return launch_main_t<MODE, TPT, 7>(grid, smem, a, s);
        case 256: return launch_main_t<MODE, TPT, 8>(grid, smem, a, s);
        case 512: return launch_main_t<MODE, TPT, 9>(grid, smem, a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

}  // namespace gce
