/*
 * Conditional-entropy (CE) period / period-derivative search: the CPU ORACLE.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the GPU path computes.  Only the test suite, the smoke
 * check and the benchmark's CPU-baseline / reference leg may load it.  It shares
 * no code, header, table or constant with the CUDA library, and the library
 * never loads it.
 *
 * Every step follows the paper (Katz et al., "GPU-Accelerated Periodic Source
 * Identification in Large-Scale Surveys: Measuring P and Pdot", arXiv:2006.06866):
 *
 *   - Sec. 2.3: magnitudes are normalised per light curve; the bin range used
 *     here is the curve's own min..max, under which the paper's median/std
 *     normalisation (an affine map) cancels.
 *   - Eq. 3 (Sec. 2.3): phase fold with a period derivative,
 *         P*phi(t) = (t - 1/2 (Pdot/P) t^2) mod P,
 *     i.e. phi = frac(tau/P - 1/2 Pdot tau^2 / P^2) with tau = t - t0.
 *   - Sec. 2.3: a 2-D histogram with n_mag magnitude bins and n_phase phase bins.
 *   - Eq. 4 (Sec. 2.3): H_c = sum_ij p(m_i,phi_j) ln( p(phi_j) / p(m_i,phi_j) ).
 *   - Sec. 2.3 / Sec. 4: the detection is the grid minimum of H_c; its
 *     significance (Eq. 5) is computed from the grid in oracle/__init__.py.
 *   - Sec. 2.3, options: half-overlapping neighbouring phase bins, and several
 *     filters per source, each normalised by its own median and standard
 *     deviation before the bins are taken.
 *
 * Every function is pinned by tests/oracle_pins.py to something other than
 * itself: exact rational arithmetic on dyadic inputs, closed forms, library
 * routines (scipy's Shannon entropy, numpy's median and standard deviation),
 * brute force on tiny inputs and the paper's worked example (Fig. 2).
 *
 * Floating point: IEEE binary64, round-to-nearest, each operation written out
 * in a fixed order (build with -ffp-contract=off, never -ffast-math; the one
 * fused multiply-add is the explicit fma() of the fold).  The GPU's FP64 fold
 * uses the same operation sequence, which is what makes histogram counts
 * bit-exact between the two.
 *
 * Readings of points where the paper is silent (all are listed in the design
 * notes): t0 is an explicit argument; bin edges use floor with the top edge
 * clamped into the last bin; a curve whose magnitudes are all equal puts every
 * point in magnitude bin 0; ln is the natural logarithm (H in nats); empty
 * cells contribute 0 (the x ln x -> 0 limit).
 *
 * Planted-mistake hooks: when compiled with -DORACLE_MUTANT=<k> one deliberate
 * error is switched on (see the MUTANT() sites).  Only the test that checks that
 * the oracle's pins catch such errors builds these variants; the normal build
 * defines no ORACLE_MUTANT.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif
#define MUTANT(k) (ORACLE_MUTANT == (k))

/* ---------------------------------------------------------------- magnitudes */

/* Magnitude bin of every point of one curve (Sec. 2.3, min..max range):
 *   mn = min m, mx = max m;  mx == mn -> bin 0;
 *   otherwise i = floor(((m - mn) / (mx - mn)) * n_mag), clamped to n_mag - 1
 *   (only m == mx reaches n_mag). */
void oracle_mag_bins(const double *mags, int64_t n, int32_t n_mag, int32_t *bins)
{
    if (n <= 0) return;
    double mn = mags[0], mx = mags[0];
    for (int64_t k = 1; k < n; ++k) {
        if (mags[k] < mn) mn = mags[k];
        if (mags[k] > mx) mx = mags[k];
    }
    for (int64_t k = 0; k < n; ++k) {
        if (mx == mn) { bins[k] = 0; continue; }
        double v = (mags[k] - mn) / (mx - mn);
        double y = v * (double)(MUTANT(6) ? n_mag - 1 : n_mag);
        int32_t i = (int32_t)floor(y);
        if (i > n_mag - 1) i = n_mag - 1;
        bins[k] = i;
    }
}

/* Multi-filter input (Sec. 2.3): the magnitudes of one curve come from several
 * filters, and each filter's points are normalised on their own -- the filter's
 * median subtracted, then divided by the filter's standard deviation -- so that
 * the filters combine into one light curve before the magnitude bins.
 * bands[k] < n_bands is the filter of point k; out[k] the normalised value.
 * Readings of what the paper leaves open: the median of an even count is the
 * mean of the two middle values, (a + b) * 0.5; the standard deviation is the
 * population one, sqrt(sum (m - mean)^2 / n) with the mean and the sum taken
 * in point order; a filter with zero spread normalises to 0.  Returns -1 (and
 * writes nothing) if a band index is out of range. */
static int cmp_double(const void *a, const void *b)
{
    const double x = *(const double *)a, y = *(const double *)b;
    return (x < y) ? -1 : (x > y);
}

int oracle_band_normalize(const double *mags, const uint8_t *bands, int64_t n, int32_t n_bands,
                          double *out)
{
    for (int64_t k = 0; k < n; ++k)
        if ((int32_t)bands[k] >= n_bands) return -1;
    double *tmp = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int32_t b = 0; b < n_bands; ++b) {
        int64_t cnt = 0;
        for (int64_t k = 0; k < n; ++k)
            if (MUTANT(11) || bands[k] == b) tmp[cnt++] = mags[k];  /* 11: one set of statistics for all filters */
        if (cnt == 0) continue;
        qsort(tmp, (size_t)cnt, sizeof(double), cmp_double);
        double med = (cnt % 2 == 1) ? tmp[cnt / 2] : (tmp[cnt / 2 - 1] + tmp[cnt / 2]) * 0.5;
        double sum = 0.0;
        for (int64_t k = 0; k < n; ++k)
            if (MUTANT(11) || bands[k] == b) sum += mags[k];
        const double mean = sum / (double)cnt;
        if (MUTANT(12)) med = mean;  /* 12: the mean subtracted instead of the median */
        double ss = 0.0;
        for (int64_t k = 0; k < n; ++k)
            if (MUTANT(11) || bands[k] == b) {
                const double d = mags[k] - mean;
                ss += d * d;
            }
        const double sd = sqrt(ss / (double)cnt);
        for (int64_t k = 0; k < n; ++k)
            if (bands[k] == b) out[k] = sd > 0.0 ? (mags[k] - med) / sd : 0.0;
    }
    free(tmp);
    return 0;
}

/* ---------------------------------------------------------------- trial grid */

/* Per-trial constants of Eq. 3: f = 1/P and a = (1/2 Pdot) f f, so that the
 * fold is x = tau f - a tau^2 = tau/P - 1/2 Pdot tau^2 / P^2. */
void oracle_trial_constants(double period, double pdot, double *f, double *a)
{
    double ff = 1.0 / period;
    double half_pdot = (MUTANT(1) ? 1.0 : 0.5) * pdot;
    double aa = MUTANT(10) ? half_pdot * ff : (half_pdot * ff) * ff;
    *f = ff;
    *a = aa;
}

/* Folded phase of one observation for one trial (Eq. 3), returned as
 * phi * n_phase (so that the phase bin is its floor), plus the bin itself.
 *   s = tau f;  b = a tau;  x = fma(-b, tau, s) = tau f - a tau^2;
 *   phi = x - floor(x) in [0, 1];  j = floor(phi * n_phase), clamped to n_phase-1
 * (for a tiny negative x, x - floor(x) = x + 1 rounds to exactly 1.0, so
 * phi * n_phase can equal n_phase). */
int32_t oracle_phase_bin(double tau, double f, double a, int32_t n_phase, double *phi_scaled)
{
    double s = tau * f;
    double b = a * tau;
    double x = MUTANT(2) ? fma(b, tau, s) : fma(-b, tau, s);
    double phi = x - floor(x);
    double y = phi * (double)n_phase;
    int32_t j = MUTANT(5) ? (int32_t)floor(y + 0.5) : (int32_t)floor(y);
    if (j > n_phase - 1) j = MUTANT(5) ? 0 : n_phase - 1;
    if (phi_scaled) *phi_scaled = y;
    return j;
}

/* ---------------------------------------------------------------- entropy */

/* Eq. 4 from integer counts c[i*n_phase + j] (i: magnitude bin, j: phase bin):
 *   N = sum c;  c_j = sum_i c_ij;
 *   H = sum_j sum_i [c_ij > 0] (c_ij / N) ln(c_j / c_ij),
 * summed j-major, then i, in binary64. */
double oracle_entropy(const int64_t *counts, int32_t n_mag, int32_t n_phase)
{
    int64_t n_total = 0;
    for (int64_t k = 0; k < (int64_t)n_mag * n_phase; ++k) n_total += counts[k];
    if (n_total <= 0) return 0.0;
    double h = 0.0;
    for (int32_t j = 0; j < n_phase; ++j) {
        int64_t cj = 0;
        for (int32_t i = 0; i < n_mag; ++i) cj += counts[(int64_t)i * n_phase + j];
        if (MUTANT(4)) { /* transposed marginal: the magnitude marginal c_i */
            cj = 0;
            int32_t ii = j < n_mag ? j : n_mag - 1;
            for (int32_t jj = 0; jj < n_phase; ++jj) cj += counts[(int64_t)ii * n_phase + jj];
        }
        for (int32_t i = 0; i < n_mag; ++i) {
            int64_t cij = counts[(int64_t)i * n_phase + j];
            if (cij <= 0) continue;
            double p = (double)cij / (double)(MUTANT(7) ? (int64_t)n_phase : n_total);
            double r = MUTANT(3) ? (double)cij / (double)cj : (double)cj / (double)cij;
            h += p * log(r);
        }
    }
    return h;
}

/* ---------------------------------------------------------------- one cell */

/* 2-D histogram of one curve for one (P, Pdot) trial, plus the smallest
 * distance (in cycles) of any folded phase from a phase-bin edge.
 * mag_bins: the curve's magnitude bins (oracle_mag_bins).  counts: n_mag*n_phase,
 * overwritten.  overlap != 0 takes Sec. 2.3's half-overlapping neighbouring
 * phase bins as phase bins of width 2/n_phase starting at j/n_phase
 * (modulo 1): a point in fine bin j then lies in bins j and j - 1 (mod
 * n_phase), and the probabilities of Eq. 4 are counts over their total 2N. */
static void cell_counts_from_bins(const double *t, const int32_t *mag_bins, int64_t n,
                                  double t0, double f, double a, int32_t n_phase,
                                  int32_t n_mag, int32_t overlap, int64_t *counts, double *dmin)
{
    memset(counts, 0, sizeof(int64_t) * (size_t)n_mag * (size_t)n_phase);
    double best = 1.0;
    for (int64_t k = 0; k < n; ++k) {
        double tau = MUTANT(9) ? t[k] + t0 : t[k] - t0;
        double y;
        int32_t j = oracle_phase_bin(tau, f, a, n_phase, &y);
        counts[(int64_t)mag_bins[k] * n_phase + j] += 1;
        /* 13: the second (overlapping) bin dropped; 14: no wrap from bin 0 to bin n_phase - 1 */
        if (overlap && !MUTANT(13) && !(MUTANT(14) && j == 0))
            counts[(int64_t)mag_bins[k] * n_phase + (j + n_phase - 1) % n_phase] += 1;
        double fr = y - floor(y);
        double d = fr < 1.0 - fr ? fr : 1.0 - fr;
        if (!MUTANT(15)) d /= (double)n_phase;  /* 15: edge distance left in bin units */
        if (d < best) best = d;
    }
    if (dmin) *dmin = best;
}

/* Counts, H and edge distance of one curve for one trial.  counts may be NULL. */
double oracle_cell(const double *t, const double *m, int64_t n, double t0,
                   double period, double pdot, int32_t n_phase, int32_t n_mag,
                   int32_t overlap, int64_t *counts_out, double *dmin)
{
    int32_t *bins = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int64_t *counts = (int64_t *)malloc(sizeof(int64_t) * (size_t)n_mag * (size_t)n_phase);
    double f, a;
    oracle_mag_bins(m, n, n_mag, bins);
    oracle_trial_constants(period, pdot, &f, &a);
    cell_counts_from_bins(t, bins, n, t0, f, a, n_phase, n_mag, overlap, counts, dmin);
    double h = oracle_entropy(counts, n_mag, n_phase);
    if (counts_out) memcpy(counts_out, counts, sizeof(int64_t) * (size_t)n_mag * (size_t)n_phase);
    free(counts);
    free(bins);
    return h;
}

/* ---------------------------------------------------------------- batches */

/* The full CE grid of a ragged batch.
 *   times, mags: concatenated curves; curve c owns [offsets[c], offsets[c+1]).
 *   out_H[(c * n_pdots + q) * n_periods + p] = H of curve c at (periods[p], pdots[q]).
 *   out_dmin: same layout, nullable.
 *   n_threads: OpenMP threads (<= 0: the runtime default).  The threads share
 *   out rows of (curve, pdot, run of ORACLE_PERIOD_RUN periods), so that a
 *   small batch still keeps every thread busy; each cell is computed exactly
 *   as by oracle_cell, whatever the split.
 * Returns the number of threads used. */
#define ORACLE_PERIOD_RUN 64
int oracle_ce_grid(const double *times, const double *mags, const int64_t *offsets,
                   int32_t n_curves, const double *periods, int32_t n_periods,
                   const double *pdots, int32_t n_pdots, int32_t n_phase, int32_t n_mag,
                   double t0, int32_t overlap, double *out_H, double *out_dmin,
                   int32_t n_threads)
{
    int used = 1;
    const int64_t runs = ((int64_t)n_periods + ORACLE_PERIOD_RUN - 1) / ORACLE_PERIOD_RUN;
    const int64_t rows = (int64_t)n_curves * n_pdots * runs;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel
    {
#pragma omp single
        used = omp_get_num_threads();
    }
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t r = 0; r < rows; ++r) {
        const int64_t cq = r / runs;  /* curve * n_pdots + pdot */
        int32_t c = (int32_t)(cq / n_pdots);
        int32_t q = (int32_t)(cq % n_pdots);
        int32_t p0 = (int32_t)((r % runs) * ORACLE_PERIOD_RUN);
        int32_t p1 = p0 + ORACLE_PERIOD_RUN < n_periods ? p0 + ORACLE_PERIOD_RUN : n_periods;
        int64_t lo = offsets[c], n = offsets[c + 1] - offsets[c];
        int32_t *bins = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
        int64_t *counts = (int64_t *)malloc(sizeof(int64_t) * (size_t)n_mag * (size_t)n_phase);
        oracle_mag_bins(mags + lo, n, n_mag, bins);
        for (int32_t p = p0; p < p1; ++p) {
            double f, a, dmin;
            oracle_trial_constants(periods[p], pdots[q], &f, &a);
            cell_counts_from_bins(times + lo, bins, n, t0, f, a, n_phase, n_mag, overlap, counts,
                                  &dmin);
            int64_t o = cq * n_periods + p;
            out_H[o] = oracle_entropy(counts, n_mag, n_phase);
            if (out_dmin) out_dmin[o] = dmin;
        }
        free(counts);
        free(bins);
    }
    return used;
}

/* Selected cells of a ragged batch: cell k is (cell_curve[k], cell_trial[k]) with
 * the flat trial index q * n_periods + p.  out_counts (nullable) receives
 * n_mag*n_phase counts per cell, magnitude-bin major. */
int oracle_ce_cells(const double *times, const double *mags, const int64_t *offsets,
                    const double *periods, int32_t n_periods, const double *pdots,
                    int32_t n_phase, int32_t n_mag, double t0, int32_t overlap, int64_t n_cells,
                    const int64_t *cell_curve, const int64_t *cell_trial,
                    double *out_H, double *out_dmin, int64_t *out_counts, int32_t n_threads)
{
    int used = 1;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel
    {
#pragma omp single
        used = omp_get_num_threads();
    }
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t k = 0; k < n_cells; ++k) {
        int64_t c = cell_curve[k];
        int64_t p = cell_trial[k] % n_periods, q = cell_trial[k] / n_periods;
        int64_t lo = offsets[c], n = offsets[c + 1] - offsets[c];
        if (MUTANT(16) && c > 0) lo = offsets[c - 1];  /* 16: the previous curve's start */
        int64_t *cnt = out_counts ? out_counts + k * (int64_t)n_mag * n_phase : NULL;
        double dmin;
        out_H[k] = oracle_cell(times + lo, mags + lo, n, t0, periods[p], pdots[q],
                               n_phase, n_mag, overlap, cnt, &dmin);
        if (out_dmin) out_dmin[k] = dmin;
    }
    return used;
}
