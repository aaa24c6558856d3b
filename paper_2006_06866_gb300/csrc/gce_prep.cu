// Trial-independent preparation (O(sum N + n_trials)): input checks and
// maxima, per-trial fold constants, per-curve magnitude binning with the
// points regrouped by magnitude bin, and the c ln c fixed-point table.
#include <cmath>
#include <cstdint>

#include "gce_internal.cuh"

namespace gce {

namespace {

constexpr unsigned long long kPosInfBits = 0x7ff0000000000000ull;

__global__ void k_init(JobState *st) {
    st->tau_max_bits = 0ull;
    st->pmin_bits = kPosInfBits;
    st->pdot_max_bits = 0ull;
    st->err = 0u;
    st->work = 0ull;
}

// Non-negative binary64 values order like their bit patterns, so maxima and
// minima reduce with 64-bit integer atomics.
__device__ inline void atomic_max_pos(unsigned long long *dst, double v) {
    atomicMax(dst, (unsigned long long)__double_as_longlong(v));
}
__device__ inline void atomic_min_pos(unsigned long long *dst, double v) {
    atomicMin(dst, (unsigned long long)__double_as_longlong(v));
}

__device__ inline double warp_max(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ inline double warp_min(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Checks every time, magnitude, period and period derivative; reduces
// max |t - t0|, min P and max |Pdot|.
__global__ void k_scan(const double *__restrict__ times, const double *__restrict__ mags,
                       long long n_points, const double *__restrict__ periods, int n_periods,
                       const double *__restrict__ pdots, int n_pdots, double t0, JobState *st) {
    unsigned int err = 0u;
    double tmax = 0.0, pmin = INFINITY, dmax = 0.0;
    long long stride = (long long)gridDim.x * blockDim.x;
    long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (long long i = i0; i < n_points; i += stride) {
        double t = times[i], m = mags[i];
        if (!isfinite(t) || !isfinite(m)) err |= ERR_TIME;
        double tau = fabs(t - t0);
        if (isfinite(tau)) tmax = fmax(tmax, tau);
        else err |= ERR_TIME;
    }
    for (long long i = i0; i < n_periods; i += stride) {
        double p = periods[i];
        if (!isfinite(p) || !(p > 0.0)) err |= ERR_PERIOD;
        else pmin = fmin(pmin, p);
    }
    for (long long i = i0; i < n_pdots; i += stride) {
        double d = pdots[i];
        if (!isfinite(d)) err |= ERR_PDOT;
        else dmax = fmax(dmax, fabs(d));
    }
    tmax = warp_max(tmax);
    dmax = warp_max(dmax);
    pmin = warp_min(pmin);
    err = __reduce_or_sync(0xffffffffu, err);
    if ((threadIdx.x & 31) == 0) {
        if (tmax > 0.0) atomic_max_pos(&st->tau_max_bits, tmax);
        if (dmax > 0.0) atomic_max_pos(&st->pdot_max_bits, dmax);
        if (pmin < INFINITY) atomic_min_pos(&st->pmin_bits, pmin);
        if (err) atomicOr(&st->err, err);
    }
}

// Per flat trial t = q n_periods + p: f = 1/P, a = (0.5 Pdot) f f (the oracle's
// sequence), stored in the fold mode's format.
template <int MODE>
__global__ void k_trials(TrialArgs a) {
    typedef typename ModeTraits<MODE>::trial_t trial_t;
    trial_t *out = reinterpret_cast<trial_t *>(a.trialc);
    const long long n = (long long)a.n_periods * a.n_pdots;
    const double tau_max = __longlong_as_double((long long)a.state->tau_max_bits);
    const FixedScale fs = fixed_scale_from(tau_max);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        // Range of the fold (checked once, from the maxima).
        const double pmin = __longlong_as_double((long long)a.state->pmin_bits);
        const double dmax = __longlong_as_double((long long)a.state->pdot_max_bits);
        if (pmin < INFINITY && pmin > 0.0) {
            const double fmax_ = 1.0 / pmin;
            const double amax = 0.5 * dmax * fmax_ * fmax_;
            bool bad = false;
            if (MODE == GCE_PHASE_SPLIT32) {
                // |x| < 1 needs |c| + |c2| < 1/2: cycles < 2^21 and Pdot cycles < 2^19
                bad = tau_max * fmax_ >= 2097152.0 || amax * tau_max * tau_max >= 524288.0;
            } else if (MODE == GCE_PHASE_FIXED32) {
                // F < 2^63, and the Pdot cross term small enough for its FP32 path
                bad = ldexp(fmax_, fs.e_tau) >= 536870912.0 ||
                      ldexp(amax, 2 * fs.e_tau) >= 262144.0;
            }
            if (bad) atomicOr(&a.state->err, ERR_RANGE);
        }
    }
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        const int p = (int)(t % a.n_periods);
        const int q = (int)(t / a.n_periods);
        const double f = 1.0 / a.periods[p];
        const double aa = (0.5 * a.pdots[q]) * f * f;
        trial_t v;
        if constexpr (MODE == GCE_PHASE_FP64) {
            v.x = f;
            v.y = aa;
        } else if constexpr (MODE == GCE_PHASE_SPLIT32) {
            // f split, and -a split (the fold adds -a tau^2)
            float fh = __double2float_rn(f);
            float nah = __double2float_rn(-aa);
            v.x = fh;
            v.y = __double2float_rn(f - (double)fh);
            v.z = nah;
            v.w = __double2float_rn(-aa - (double)nah);
        } else {
            // Out-of-range values are flagged above; clamp so the conversions stay defined.
            const double F = fmin(ldexp(f, fs.r), 9.2e18);
            const double A = fmax(fmin(ldexp(aa, fs.v), 9.2e18), -9.2e18);
            int f1, f0;
            split_balanced(__double2ll_rn(F), &f1, &f0);
            const long long an = -__double2ll_rn(A);
            const int a1 = (int)(an >> 32);
            const unsigned int a0 = (unsigned int)(an & 0xffffffffll);
            // k: the smallest shift with F1 < 2^(22+k)
            const unsigned int uf1 = (unsigned int)f1;
            const int bits = 32 - __clz(uf1);
            const int k = bits > 22 ? bits - 22 : 0;
            const float g0 = __double2float_rn(ldexp((double)uf1, -23 - k));
            const float g2 = __double2float_rn(ldexp((double)a1, -23 - k));
            const double kk = 12582912.0 - 8388608.0 * (double)g0 - 8388608.0 * (double)g2 -
                              ldexp((double)a1, -1 - k);
            v.i = make_uint4(uf1, (unsigned int)f0, (unsigned int)a1, a0);
            v.f = make_float4(g0, g2, __double2float_rn(kk), __uint_as_float((unsigned int)k));
        }
        out[t] = v;
    }
}

constexpr int kPrepBlock = 256;

__device__ inline double block_reduce(double v, bool is_max, double *sh) {
    v = is_max ? warp_max(v) : warp_min(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        v = l < (blockDim.x >> 5) ? sh[l] : (is_max ? -INFINITY : INFINITY);
        v = is_max ? warp_max(v) : warp_min(v);
        if (l == 0) sh[0] = v;
    }
    __syncthreads();
    v = sh[0];
    __syncthreads();
    return v;
}

// Magnitude bin of Sec. 2.3 with the oracle's operation sequence:
// i = floor(((m - mn) / (mx - mn)) * n_mag), clamped; mx == mn -> 0.
__device__ inline int mag_bin(double m, double mn, double mx, int n_mag) {
    if (mx == mn) return 0;
    double v = __ddiv_rn(__dsub_rn(m, mn), __dsub_rn(mx, mn));
    int i = __double2int_rd(__dmul_rn(v, (double)n_mag));
    return min(i, n_mag - 1);
}

// ------------------------------------------------------------------ filters

// Order-preserving map of binary64 to unsigned 64-bit keys (and back).
__device__ inline unsigned long long f64_key(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ inline double key_f64(unsigned long long k) {
    return __longlong_as_double((long long)((k >> 63) ? (k & 0x7fffffffffffffffull) : ~k));
}

// The kth smallest (0-based) magnitude of filter b among the curve's n points:
// an exact radix selection on the keys, 8 bits per pass from the top, with
// shared-memory digit histograms.  Every thread returns the value.
__device__ double band_select(const double *m, const unsigned char *bd, int n, int b, int kth,
                              unsigned int *hist, unsigned long long *s_pref, int *s_k) {
    unsigned long long prefix = 0ull;
    for (int shift = 56; shift >= 0; shift -= 8) {
        const unsigned long long high = shift == 56 ? 0ull : ~0ull << (shift + 8);
        for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0u;
        __syncthreads();
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            if (bd[k] != b) continue;
            const unsigned long long key = f64_key(m[k]);
            if ((key & high) == prefix) atomicAdd(&hist[(key >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned int cum = 0u;
            int d = 0;
            for (; d < 255; ++d) {
                if (cum + hist[d] > (unsigned int)kth) break;
                cum += hist[d];
            }
            *s_pref = prefix | ((unsigned long long)d << shift);
            *s_k = kth - (int)cum;
        }
        __syncthreads();
        prefix = *s_pref;
        kth = *s_k;
        __syncthreads();
    }
    return key_f64(prefix);
}

// One CTA per curve: for each filter b, the median and the population standard
// deviation of its magnitudes (the per-filter normalisation of Sec. 2.3), in the
// operation order stated in gce.h: the median exactly (radix selection), the
// mean and the sum of squared deviations in binary64 in point order (one
// thread), so that the normalised values match a plain sequential statement
// bit for bit.  A filter with no points gets {0, 0}.  Band indices >= n_bands
// set ERR_BAND.
__global__ void __launch_bounds__(256) k_band_stats(const double *__restrict__ mags,
                                                    const unsigned char *__restrict__ bands,
                                                    const long long *__restrict__ offsets,
                                                    int n_bands, double2 *stats, JobState *st) {
    __shared__ unsigned int hist[256];
    __shared__ unsigned long long s_pref;
    __shared__ int s_k, s_cnt[GCE_MAX_BANDS];
    const int c = blockIdx.x;
    const long long lo = offsets[c];
    const int n = (int)(offsets[c + 1] - lo);
    const double *m = mags + lo;
    const unsigned char *bd = bands + lo;
    if (threadIdx.x < GCE_MAX_BANDS) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    bool bad = false;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const int b = bd[k];
        if (b >= n_bands) bad = true;
        else atomicAdd(&s_cnt[b], 1);
    }
    if (__syncthreads_or(bad)) {
        if (threadIdx.x == 0) atomicOr(&st->err, ERR_BAND);
        return;
    }
    for (int b = 0; b < n_bands; ++b) {
        const int cnt = s_cnt[b];
        double2 r = make_double2(0.0, 0.0);
        if (cnt > 0) {
            double med = band_select(m, bd, n, b, (cnt - 1) / 2, hist, &s_pref, &s_k);
            if ((cnt & 1) == 0) {
                const double hi = band_select(m, bd, n, b, cnt / 2, hist, &s_pref, &s_k);
                med = __dmul_rn(__dadd_rn(med, hi), 0.5);
            }
            if (threadIdx.x == 0) {
                double sum = 0.0;
                for (int k = 0; k < n; ++k)
                    if (bd[k] == b) sum = __dadd_rn(sum, m[k]);
                const double mean = __ddiv_rn(sum, (double)cnt);
                double ss = 0.0;
                for (int k = 0; k < n; ++k)
                    if (bd[k] == b) {
                        const double d = __dsub_rn(m[k], mean);
                        ss = __dadd_rn(ss, __dmul_rn(d, d));
                    }
                r = make_double2(med, __dsqrt_rn(__ddiv_rn(ss, (double)cnt)));
            }
        }
        if (threadIdx.x == 0) stats[(long long)c * n_bands + b] = r;
    }
}

// The magnitude the bins of Sec. 2.3 see: the raw value, or with multi-filter
// input (m - median) / sd of the point's filter (0 when sd is 0).
struct MagView {
    const double *m;
    const unsigned char *bd;  // nullptr: raw magnitudes
    const double2 *bs;        // this curve's {median, sd} per filter
    int nb;
    __device__ double operator[](int k) const {
        if (!bd) return m[k];
        const int b = bd[k];
        if (b >= nb) return 0.0;  // flagged by k_band_stats; never read past the table
        const double2 s = bs[b];
        return s.y > 0.0 ? __ddiv_rn(__dsub_rn(m[k], s.x), s.y) : 0.0;
    }
};

// One CTA per curve: min/max of the magnitudes, magnitude bins, a counting sort
// of the points by magnitude bin (segment starts written to seg), and the
// points' fold payload written in the sorted order.  The order of points inside
// a segment is arbitrary; counts do not depend on it.
template <int MODE>
__global__ void __launch_bounds__(kPrepBlock) k_prep(PrepArgs a) {
    typedef typename ModeTraits<MODE>::point_t point_t;
    __shared__ double sh_red[32];
    __shared__ int hist[GCE_MAX_MAG_BINS + 1];
    const int c = blockIdx.x;
    const long long lo = a.offsets[c];
    const int n = (int)(a.offsets[c + 1] - lo);
    const MagView m{a.mags + lo, a.bands ? a.bands + lo : nullptr,
                    a.bands ? a.band_stats + (long long)c * a.n_bands : nullptr, a.n_bands};
    const double *t = a.times + lo;
    double mn = INFINITY, mx = -INFINITY;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        mn = fmin(mn, m[k]);
        mx = fmax(mx, m[k]);
    }
    mn = block_reduce(mn, false, sh_red);
    mx = block_reduce(mx, true, sh_red);
    for (int i = threadIdx.x; i <= a.n_mag; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    for (int k = threadIdx.x; k < n; k += blockDim.x) atomicAdd(&hist[mag_bin(m[k], mn, mx, a.n_mag)], 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        int *seg = a.seg + (long long)c * (a.n_mag + 1);
        for (int i = 0; i < a.n_mag; ++i) {
            int h = hist[i];
            hist[i] = run;
            seg[i] = run;
            run += h;
        }
        seg[a.n_mag] = run;
    }
    __syncthreads();
    const FixedScale fs = fixed_scale_from(__longlong_as_double((long long)a.state->tau_max_bits));
    point_t *out = reinterpret_cast<point_t *>(a.payload) + lo;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const int pos = atomicAdd(&hist[mag_bin(m[k], mn, mx, a.n_mag)], 1);
        const double tau = __dsub_rn(t[k], a.t0);
        point_t v;
        if constexpr (MODE == GCE_PHASE_FP64) {
            v = tau;
        } else if constexpr (MODE == GCE_PHASE_SPLIT32) {
            const double tau2 = __dmul_rn(tau, tau);
            float th = __double2float_rn(tau);
            float t2h = __double2float_rn(tau2);
            v.x = th;
            v.y = __double2float_rn(tau - (double)th);
            v.z = t2h;
            v.w = __double2float_rn(tau2 - (double)t2h);
        } else {
            // T = round(tau 2^s), |T| < 2^62; U = floor(T^2 / 2^62) = tau^2 2^u
            // computed exactly from T in 128-bit integer arithmetic.
            const long long T = __double2ll_rn(ldexp(tau, fs.s));
            const unsigned long long aT = (unsigned long long)(T < 0 ? -T : T);
            const unsigned long long hi = __umul64hi(aT, aT), lw = aT * aT;
            const long long U = (long long)((hi << 2) | (lw >> 62));
            int u1, u0;
            split_balanced(U, &u1, &u0);
            const unsigned int t0 = (unsigned int)(T & 0xffffffffll);
            v.x = (unsigned int)(int)(T >> 32);
            v.y = 0x4B000000u | (t0 >> 9);                               // 2^23 + (T0 >> 9)
            v.z = (unsigned int)u1;
            v.w = 0x4B000000u | (((unsigned int)u0 ^ 0x80000000u) >> 9);  // 2^23 + ((U0+2^31) >> 9)
        }
        out[pos] = v;
    }
}

__global__ void k_table(unsigned long long *table, int n_max) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c <= n_max; c += gridDim.x * blockDim.x) {
        double v = c > 1 ? (double)c * log((double)c) * kTabScale : 0.0;
        table[c] = (unsigned long long)__double2ll_rn(v);
    }
}

int grid_for(long long n, int block, int cap) {
    long long g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

}  // namespace

cudaError_t launch_init(JobState *st, cudaStream_t s) {
    k_init<<<1, 1, 0, s>>>(st);
    return cudaGetLastError();
}

cudaError_t launch_scan(const double *times, const double *mags, long long n_points,
                        const double *periods, int n_periods, const double *pdots, int n_pdots,
                        double t0, JobState *st, cudaStream_t s) {
    long long n = n_points;
    if (n_periods > n) n = n_periods;
    if (n_pdots > n) n = n_pdots;
    k_scan<<<grid_for(n, 256, 1216), 256, 0, s>>>(times, mags, n_points, periods, n_periods,
                                                     pdots, n_pdots, t0, st);
    return cudaGetLastError();
}

cudaError_t launch_trials(int mode, const TrialArgs &a, cudaStream_t s) {
    long long n = (long long)a.n_periods * a.n_pdots;
    int g = grid_for(n, 256, 4864);
    switch (mode) {
        case GCE_PHASE_FP64: k_trials<GCE_PHASE_FP64><<<g, 256, 0, s>>>(a); break;
        case GCE_PHASE_SPLIT32: k_trials<GCE_PHASE_SPLIT32><<<g, 256, 0, s>>>(a); break;
        default: k_trials<GCE_PHASE_FIXED32><<<g, 256, 0, s>>>(a); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_band_stats(const double *mags, const unsigned char *bands,
                              const long long *offsets, int n_curves, int n_bands,
                              double2 *stats, JobState *st, cudaStream_t s) {
    if (n_curves <= 0) return cudaSuccess;
    k_band_stats<<<n_curves, 256, 0, s>>>(mags, bands, offsets, n_bands, stats, st);
    return cudaGetLastError();
}

cudaError_t launch_prep(int mode, const PrepArgs &a, cudaStream_t s) {
    if (a.n_curves <= 0) return cudaSuccess;
    switch (mode) {
        case GCE_PHASE_FP64: k_prep<GCE_PHASE_FP64><<<a.n_curves, kPrepBlock, 0, s>>>(a); break;
        case GCE_PHASE_SPLIT32: k_prep<GCE_PHASE_SPLIT32><<<a.n_curves, kPrepBlock, 0, s>>>(a); break;
        default: k_prep<GCE_PHASE_FIXED32><<<a.n_curves, kPrepBlock, 0, s>>>(a); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_table(unsigned long long *table, int n_max, cudaStream_t s) {
    k_table<<<grid_for((long long)n_max + 1, 256, 1024), 256, 0, s>>>(table, n_max);
    return cudaGetLastError();
}

}  // namespace gce
