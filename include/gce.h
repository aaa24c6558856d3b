/*
 * gce.h -- C ABI of the GB300 conditional-entropy (P, Pdot) search library.
 *
 * The library computes, for every light curve of a ragged batch and every trial
 * (P, Pdot) of a grid, the conditional entropy of Katz et al. (arXiv:2006.06866):
 *
 *   fold (Eq. 3, Sec. 2.3):   phi = frac(tau/P - 1/2 Pdot tau^2 / P^2),  tau = t - t0
 *   bin  (Sec. 2.3):          magnitude bin i from the curve's min..max range,
 *                             phase bin j = floor(phi * n_phase)
 *   entropy (Eq. 4):          H = sum_ij p(m_i, phi_j) ln( p(phi_j) / p(m_i, phi_j) )
 *   selection (Sec. 2.3, 4):  the grid minimum, or the k smallest cells per curve
 *
 * Conventions shared by every call:
 *   - Array arguments are DEVICE pointers (cudaMalloc'd or managed) unless their
 *     name starts with h_, which marks HOST memory.  The caller owns every input
 *     and output buffer; the library never frees or keeps them past the call's
 *     stream work.  Device arrays must live on the handle's device: an array
 *     that the CUDA runtime reports as another device's memory is rejected with
 *     GCE_ERR_INVALID before anything is launched.
 *   - A ragged batch is (times, mags, h_offsets, n_curves): curve c owns elements
 *     [h_offsets[c], h_offsets[c+1]) of times and mags (float64); h_offsets is a
 *     HOST int64 array of n_curves + 1 entries starting at 0, non-decreasing.
 *   - The trial grid is periods[n_periods] (float64, > 0) x pdots[n_pdots]
 *     (float64, s/s, any sign -- Sec. 4 notes positive Pdot needs no other
 *     code).  The flat trial index is q * n_periods + p for pdots[q], periods[p].
 *   - Units only need to be consistent (e.g. seconds for times and periods).
 *   - Calls taking a stream are asynchronous on that stream (a cudaStream_t
 *     passed as void*; NULL is the legacy default stream).  Argument checks that
 *     need only host data run synchronously and return GCE_ERR_INVALID without
 *     launching anything.  Checks on device data (non-finite times or
 *     magnitudes, non-positive or non-finite periods, non-finite pdots, a trial
 *     range the chosen fold cannot represent) run on the GPU; they are reported
 *     by gce_stream_status(), and outputs of a flagged call are unspecified.
 *   - Nothing throws across the ABI.  A handle is not thread-safe: use one per
 *     host thread.  CUDA failures return GCE_ERR_CUDA with the text available
 *     from gce_last_error().
 */
#ifndef GCE_H
#define GCE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GCE_OK = 0,
    GCE_ERR_INVALID = 1,     /* bad argument (host check) or bad input values (device check) */
    GCE_ERR_CUDA = 2,        /* a CUDA call failed; see gce_last_error() */
    GCE_ERR_NOMEM = 3,       /* device workspace allocation failed */
    GCE_ERR_UNSUPPORTED = 4  /* valid input outside what the chosen fold supports */
} gce_status;

/* How the fold of Eq. 3 is evaluated.  Magnitude bins, counts and the entropy
 * are the same in every mode; only the phase-bin decision differs. */
typedef enum {
    /* binary64 with the operation sequence s = tau*f, b = a*tau,
     * x = fma(-b, tau, s), phi = x - floor(x), j = floor(phi*n_phase) (clamped),
     * f = 1/P, a = (0.5*Pdot)*f*f.  Counts are bit-identical to a CPU binary64
     * evaluation of that sequence. */
    GCE_PHASE_FP64 = 0,
    /* FP32 double-float: tau, tau^2, f and a split into (hi, lo) float pairs,
     * error-free products via fmaf, integer cycles removed with a rounding
     * constant.  Phase error about 1e-7 cycles; needs |tau|/P < 2^21 and
     * |Pdot| tau^2/(2 P^2) < 2^19 cycles. */
    GCE_PHASE_SPLIT32 = 1,
    /* fixed point: tau, tau^2, f and a as 64-bit integers split into 32-bit
     * limbs; the phase is the low 32 bits of their products (integer cycles wrap
     * away).  The large partial products are integer multiplies, the small
     * cross terms FP32 multiply-adds.  Phase error a few 2^-32 cycles up to
     * about 2^22 cycles, growing to ~6e-8 cycles at the limit; needs |tau|/P <
     * 2^28 and |Pdot| tau^2/P^2 < 2^16 cycles. */
    GCE_PHASE_FIXED32 = 2
} gce_phase_mode;

#define GCE_MAX_PHASE_BINS 256
#define GCE_MAX_MAG_BINS 255
#define GCE_MAX_CURVE_POINTS 65535
#define GCE_MAX_TOPK 64
#define GCE_MAX_BANDS 8

/* flags */
#define GCE_FLAG_NO_GRAPH 1u      /* launch kernels directly instead of through a CUDA graph */
#define GCE_FLAG_TIME_KERNEL 2u   /* record CUDA events around the CE kernel (gce_kernel_time) */
/* 50 %-overlapping phase bins (Sec. 2.3): phase bin j spans [j, j + 2) / n_phase
 * (modulo 1), so every point counts in its bin and the one below it, and the
 * probabilities of Eq. 4 are counts over 2N.  Needs n_phase_bins >= 2. */
#define GCE_FLAG_OVERLAP 4u

typedef struct {
    int32_t n_phase_bins;  /* 1 .. GCE_MAX_PHASE_BINS (the paper uses 15 and 50) */
    int32_t n_mag_bins;    /* 1 .. GCE_MAX_MAG_BINS (the paper uses 10) */
    int32_t phase_mode;    /* gce_phase_mode */
    uint32_t flags;        /* GCE_FLAG_* */
    double t0;             /* epoch of the fold, in the unit of times */
} gce_config;

/* Launch shape of the batched kernel.  block: threads per CTA (64, 128, 256
 * or 512); tpt: trials per thread (1, 2, or 4 except with GCE_PHASE_FP64);
 * ctas_per_sm: resident CTAs per SM
 * (0 = as many as fit); chunk: light-curve points staged in shared memory at
 * once (a multiple of 256, 256 .. 8192); slot_range (GCE_PHASE_SPLIT32 jobs
 * without a Pdot axis; ignored otherwise): 0 keeps a counter for every phase
 * slot a fold can reach within the job's cycle limit, 1 keeps about a quarter
 * fewer (fold residuals up to 9/16 cycle) and re-reduces the folds of every
 * warp of trials whose cycles, |t - t0| f, could exceed that (about 5e5
 * cycles): less shared memory per trial for the same counts, at three more
 * FP32 operations per point where the re-reduction runs. */
typedef struct {
    int32_t block;
    int32_t tpt;
    int32_t ctas_per_sm;
    int32_t chunk;
    int32_t slot_range;
} gce_tuning;

typedef struct gce_handle_s *gce_handle;

/* Create a handle on CUDA device `device` (it becomes current on the calling
 * thread).  The handle owns the device workspace, the autotune cache and the
 * captured CUDA graphs.  *h is NULL on failure.
 * The workspace grows to the largest job seen and is kept until gce_destroy:
 * 8 (FP64) or 16 bytes per point, 16 (FP64, SPLIT32) or 32 (FIXED32) bytes per
 * (P, Pdot) trial, 8 k bytes per (curve, warp of a trial tile) for top-k (24 more with
 * the significance), and 8 bytes per entry of the c ln c table (longest curve
 * + 1).  A grid of 5,183,995 periods x 512 Pdot values thus holds 42 GB of
 * trial constants in SPLIT32.  Growing a buffer waits for the device. */
gce_status gce_create(gce_handle *h, int32_t device);

/* Free everything the handle owns (waits for its outstanding work). */
gce_status gce_destroy(gce_handle h);

/* Static description of a status code; never NULL. */
const char *gce_status_string(gce_status s);

/* Text of the last failure on this handle ("" if none); valid until the next
 * call on the handle.  gce_last_error(NULL) describes the last gce_create(). */
const char *gce_last_error(gce_handle h);

/* Host-side argument checks of a job, without a device or handle.  Returns
 * GCE_ERR_INVALID if: n_curves < 0; h_offsets NULL (when n_curves > 0), not
 * starting at 0, decreasing, or any curve empty or longer than
 * GCE_MAX_CURVE_POINTS; n_periods < 1 or n_pdots < 1 or n_periods * n_pdots >=
 * 2^32; bins outside their ranges; an unknown phase_mode; k < 0, k >
 * GCE_MAX_TOPK or k > n_periods * n_pdots. */
gce_status gce_check_job(const int64_t *h_offsets, int32_t n_curves, int32_t n_periods,
                         int32_t n_pdots, const gce_config *cfg, int32_t k);

/* Full CE grid (Sec. 2.3, Eq. 3-4): out[(c * n_pdots + q) * n_periods + p] =
 * H of curve c at (periods[p], pdots[q]) as float32 nats, for every cell.
 * out must hold n_curves * n_pdots * n_periods floats.  n_curves == 0 is a
 * no-op. */
gce_status gce_ce_grid(gce_handle h, const double *times, const double *mags,
                       const int64_t *h_offsets, int32_t n_curves, const double *periods,
                       int32_t n_periods, const double *pdots, int32_t n_pdots,
                       const gce_config *cfg, float *out, void *stream);

/* Per-curve k smallest cells of the CE grid without materialising it (the
 * selection of Sec. 2.3; batched minima merged as in Sec. 4).  topk_H[c*k + r]
 * (float32, ascending) and topk_idx[c*k + r] (flat trial index q*n_periods + p)
 * are the r-th smallest cell; ties in H go to the smaller flat index. */
gce_status gce_ce_topk(gce_handle h, const double *times, const double *mags,
                       const int64_t *h_offsets, int32_t n_curves, const double *periods,
                       int32_t n_periods, const double *pdots, int32_t n_pdots,
                       const gce_config *cfg, int32_t k, float *topk_H, int64_t *topk_idx,
                       void *stream);

/* gce_ce_topk plus the significance of the minimum (Eq. 5, Sec. 2.3):
 * rho[c] = (mean[c] - topk_H[c*k]) / std[c], where mean and std (population,
 * ddof 0) are over all n_pdots * n_periods CE values of curve c.  The moments
 * are accumulated per trial tile and merged in a fixed order with Chan et al.'s
 * pairwise update (the batch-statistics merge of Sec. 4), so results are
 * deterministic.  mean, std: device double[n_curves]; rho: device
 * float[n_curves] (0 when std is 0). */
gce_status gce_ce_detect(gce_handle h, const double *times, const double *mags,
                         const int64_t *h_offsets, int32_t n_curves, const double *periods,
                         int32_t n_periods, const double *pdots, int32_t n_pdots,
                         const gce_config *cfg, int32_t k, float *topk_H, int64_t *topk_idx,
                         double *mean, double *std, float *rho, void *stream);

/* Multi-filter input (Sec. 2.3): the magnitudes of each light curve come from
 * up to GCE_MAX_BANDS filters, and each (curve, filter) is normalised on its
 * own -- its median subtracted, then divided by its standard deviation -- so
 * that the filters combine into one light curve; the magnitude bins of Sec. 2.3
 * then span the curve's normalised values.  bands: device uint8[sum N], the
 * filter index of each point, each < n_bands (1 .. GCE_MAX_BANDS).  Readings:
 * the median of an even count is the mean of the two middle values, taken as
 * (a + b) * 0.5; the standard deviation is the population one (ddof 0), with
 * the mean and the sum of squared deviations accumulated in binary64 in point
 * order; a filter whose points all share one value (or has one point)
 * normalises to 0.  A band index >= n_bands is a device-side input error
 * (GCE_ERR_INVALID from gce_stream_status).  With n_bands == 1 the bins are
 * those of the curve's own min..max as in gce_ce_grid, up to rounding at bin
 * edges.  Otherwise as gce_ce_grid. */
gce_status gce_ce_grid_bands(gce_handle h, const double *times, const double *mags,
                             const uint8_t *bands, int32_t n_bands, const int64_t *h_offsets,
                             int32_t n_curves, const double *periods, int32_t n_periods,
                             const double *pdots, int32_t n_pdots, const gce_config *cfg,
                             float *out, void *stream);

/* gce_ce_detect on multi-filter input (normalised as in gce_ce_grid_bands).
 * mean, std and rho may all be NULL: then only the top-k is computed. */
gce_status gce_ce_detect_bands(gce_handle h, const double *times, const double *mags,
                               const uint8_t *bands, int32_t n_bands,
                               const int64_t *h_offsets, int32_t n_curves,
                               const double *periods, int32_t n_periods, const double *pdots,
                               int32_t n_pdots, const gce_config *cfg, int32_t k,
                               float *topk_H, int64_t *topk_idx, double *mean, double *std,
                               float *rho, void *stream);

/* gce_ce_topk on HOST arrays (h_times, h_mags: sum N float64; h_periods,
 * h_pdots; outputs h_topk_H / h_topk_idx of n_curves * k).  Copies inputs to
 * the handle's device workspace, runs, copies the results back and waits; the
 * device-side input checks are folded into the returned status.  Pinned host
 * memory makes the copies asynchronous DMA; pageable memory works too. */
gce_status gce_ce_topk_host(gce_handle h, const double *h_times, const double *h_mags,
                            const int64_t *h_offsets, int32_t n_curves,
                            const double *h_periods, int32_t n_periods,
                            const double *h_pdots, int32_t n_pdots, const gce_config *cfg,
                            int32_t k, float *h_topk_H, int64_t *h_topk_idx, void *stream);

/* gce_ce_topk for callers that must not allocate device memory: the paper has
 * no counterpart.  Some callers cannot call cudaMalloc -- a process whose GPU
 * memory is owned by another allocator (a framework's caching allocator, or a
 * pool that has reserved nearly all of it, where an outside cudaMalloc can fail
 * or fragment that pool), or a latency-critical loop that cannot take
 * cudaMalloc's implicit synchronisation.  This call allocates nothing and needs
 * no handle: all its device workspace is a 32 MiB array built into the library
 * (held on every GPU where the library is loaded, until the process exits).
 * Arguments are those of gce_ce_topk, with the same meaning and layout; the
 * caller still owns the input and output buffers.  The call runs on the
 * calling thread's current device, and every device array must be there
 * (GCE_ERR_INVALID otherwise).  The call is synchronous on `stream` and folds
 * the device-side input checks into its status.
 * Returns GCE_ERR_NOMEM, launching nothing, when the job needs more than the
 * 32 MiB (about 16 B per point + 32 B per trial + 8 B per (curve, 64 trials,
 * k) + 0.5 MiB); use gce_ce_topk for larger jobs.  Returns
 * GCE_ERR_UNSUPPORTED when the bin counts need more shared memory than one CTA
 * of its fixed launch shape (256 threads, 2 trials each) can have.
 * Every call looks up the array's device address; the first call on a device
 * (and the first after a device reset, which moves the array) also fills a
 * table in it with a few synchronous CUDA calls: make the first call before
 * any stream capture.  Every call shares the array and keeps the last
 * call's contents; each call rewrites what it reads.  Calls that overlap on the
 * GPU (two host threads or two streams) race on the array: make them one at a
 * time. */
gce_status gce_ce_topk_static(const double *times, const double *mags,
                              const int64_t *h_offsets, int32_t n_curves, const double *periods,
                              int32_t n_periods, const double *pdots, int32_t n_pdots,
                              const gce_config *cfg, int32_t k, float *topk_H,
                              int64_t *topk_idx, void *stream);

/* Plain baseline: the FP64 fold with one kernel launch per light curve and one
 * thread per trial (the shape of the paper's own kernel, Sec. 2.3.2), same
 * output as gce_ce_grid.  cfg->phase_mode must be GCE_PHASE_FP64. */
gce_status gce_ce_grid_single(gce_handle h, const double *times, const double *mags,
                              const int64_t *h_offsets, int32_t n_curves,
                              const double *periods, int32_t n_periods, const double *pdots,
                              int32_t n_pdots, const gce_config *cfg, float *out,
                              void *stream);

/* Diagnostic: the full 2-D histogram of selected cells, computed with the same
 * fold and binning device code as the batched kernel for cfg->phase_mode.
 * cell_curve / cell_trial: device int64[n_cells] (curve index, flat trial
 * index).  counts: device uint32[n_cells][n_mag_bins][n_phase_bins]. */
gce_status gce_ce_counts(gce_handle h, const double *times, const double *mags,
                         const int64_t *h_offsets, int32_t n_curves, const double *periods,
                         int32_t n_periods, const double *pdots, int32_t n_pdots,
                         const gce_config *cfg, int64_t n_cells, const int64_t *cell_curve,
                         const int64_t *cell_trial, uint32_t *counts, void *stream);

/* Wait for `stream` and report the device-side input checks of the last call
 * made on this handle (GCE_OK, GCE_ERR_INVALID or GCE_ERR_UNSUPPORTED), or
 * GCE_ERR_CUDA if the stream failed. */
gce_status gce_stream_status(gce_handle h, void *stream);

/* Duration in milliseconds of the CE kernel (the persistent fold/histogram/
 * entropy kernel, without preparation or top-k merge) of the last call made
 * with GCE_FLAG_TIME_KERNEL, from CUDA events recorded on the call's stream
 * around that launch.  Waits for the events. */
gce_status gce_kernel_time(gce_handle h, float *ms);

/* Number of CUDA kernels the last search call on this handle launched, directly
 * or inside its CUDA graph: the checks, trial constants, preparation (plus the
 * per-filter statistics with multi-filter input), the CE kernel and the top-k
 * merge (two levels when a curve has more than 4096 tile candidates), one
 * launch per curve for gce_ce_grid_single, and the c ln c table when a call
 * extended it.  0 before any call and after a call on an empty batch.
 * Host-side only: no device work, no wait. */
gce_status gce_last_launches(gce_handle h, int32_t *n);

/* Time candidate launch shapes on a synthetic job of the given size and keep
 * the fastest for (phase mode, bins, curve-length bucket) in the handle's
 * cache; later calls with a matching key use it.  Jobs with a Pdot axis
 * (n_pdots > 1, whose tiles pair one period with several Pdot values) are
 * tuned separately on a synthetic job with 8 Pdot values and cached under
 * their own entry.  Synchronous. */
gce_status gce_autotune(gce_handle h, const gce_config *cfg, int32_t n_obs_hint,
                        int64_t n_trials_hint);

/* Tune on the caller's own job (arguments as gce_ce_grid, without the output):
 * the candidate shapes are timed on a bounded slice of it -- a prefix of the
 * curves holding about 4e9 point-trials of the slice, at most 65536 periods and
 * 8 Pdot values, each a strided subset spanning the job's range -- and the
 * fastest is cached under the job's key (phase mode, bins, length bucket of
 * its longest curve, Pdot axis or not), which later calls on that job use.
 * Synchronous; it allocates and frees a small scratch of its own. */
gce_status gce_autotune_job(gce_handle h, const double *times, const double *mags,
                            const int64_t *h_offsets, int32_t n_curves, const double *periods,
                            int32_t n_periods, const double *pdots, int32_t n_pdots,
                            const gce_config *cfg);

/* Read the launch shape the handle would use for a job with this config,
 * typical curve length and number of Pdot values (n_pdots_hint >= 1; > 1 means
 * a Pdot axis), or force one (gce_set_tuning replaces the cached choice for
 * that curve-length bucket, for jobs with and without a Pdot axis).
 * GCE_ERR_INVALID for n_pdots_hint < 1 or, from gce_set_tuning, for shapes
 * outside the documented ranges. */
gce_status gce_get_tuning(gce_handle h, const gce_config *cfg, int32_t n_obs_hint,
                          int32_t n_pdots_hint, gce_tuning *t);
gce_status gce_set_tuning(gce_handle h, const gce_config *cfg, int32_t n_obs_hint,
                          const gce_tuning *t);

#ifdef __cplusplus
}
#endif

#endif /* GCE_H */
