/*
 * gtls.h -- C ABI of the GB300 TLS period-grid search (libgtls.so).
 *
 * The library implements the data-parallel search of the GTLS paper
 * (arxiv 2607.00348, Sect. 2): for every trial period of an Ofir-sampled
 * grid (Sect. 2.2.1) it folds the light curve (Eq. phase), sorts it by
 * phase, slides a limb-darkened transit template of every trial duration
 * (Sect. 2.2.2) over the folded curve with T0 steps of max(1, floor(D dt0))
 * points (Eq. N_skip), fits the depth (Eqs. k, depth), evaluates chi2 of
 * the model (Eqs. edge, out, in) and reduces the per-period minimum chi2(P)
 * to the signal residue SR(P), SDE_raw(P) and the median-detrended SDE(P)
 * (Sect. 2.4).  All search arithmetic runs in CUDA kernels for sm_103a.
 *
 * Conventions for every entry point:
 *   - Returns a gtls_status; nothing is thrown across the ABI.  On failure
 *     gtls_last_error() returns a message for the calling thread.
 *   - Pointers documented as "device" must be CUDA device (or managed)
 *     memory on the plan's device; "host" pointers are ordinary memory.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *     that return results in host structs synchronise that stream.
 *   - A plan is not thread-safe: one search at a time per plan.
 *
 * Readings of the paper fixed by this ABI (the paper is silent on them):
 *   - SR(P) = chi2_min / chi2(P) in (0, 1] (Kovacs convention; the paper's
 *     printed ratio is inverted), 0/0 := 1.
 *   - durations come from one geometric grid of T14/P (ratio dur_ratio);
 *     a period searches the grid points inside its k_min/k_max/q_cap
 *     envelope; D = max(1, round(q n)) points.
 *   - the template is a central small-planet transit with quadratic limb
 *     darkening (u1, u2): s_k = 1 - u1(1-mu) - u2(1-mu)^2,
 *     mu = sqrt(1 - (2x-1)^2), x = (k + 1/2)/D.
 *   - depth = max(0, mean in-window flux deficit / mean template value).
 *   - phases are exact on a lattice of 2^-e days (e reported by
 *     gtls_plan_get_info); ties in phase keep the input order.
 *   - SDE(P) = SDE_raw(P) minus the running median of SDE_raw over an odd
 *     window (median_window; default 2 floor(N_P/200) + 1), truncated at
 *     the ends, lower median for even counts.
 */
#ifndef GTLS_H
#define GTLS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GTLS_OK = 0,
    GTLS_ERR_INVALID_ARG = 1, /* bad sizes/parameters, non-finite input, dy <= 0 */
    GTLS_ERR_CUDA = 2,        /* a CUDA runtime call failed */
    GTLS_ERR_OOM = 3,         /* device or host allocation failed */
    GTLS_ERR_TIMEOUT = 4,     /* a bounded device wait ran out */
    GTLS_ERR_INTERNAL = 5     /* an internal consistency check failed */
} gtls_status;

typedef struct gtls_plan gtls_plan;

/* Search configuration.  Fill with gtls_plan_params_default, then edit. */
typedef struct {
    double baseline_days;       /* S = t_max - t_min (days), > 0; sets A of Eq. (C, A) */
    int64_t n_points;           /* points per light curve, >= 2; D = round(q n) */
    double m_star, r_star;      /* stellar mass / radius in solar units (default 1, 1) */
    double oversampling;        /* OS of Eq. (C, A) (default 3) */
    double period_min_days;     /* 0 => Roche limit, Eq. (f_max) */
    double period_max_days;     /* 0 => S / 2, Eq. (f_min) */
    double k_min, k_max;        /* duration envelope, s^(2/3) (default 20.05, 620.84) */
    double q_cap;               /* maximum T14/P (default 0.15) */
    double dur_ratio;           /* geometric step of the T14/P grid (default 1.1) */
    double dt0;                 /* T0 step as a fraction of D (default 0.05) */
    double u1, u2;              /* quadratic limb darkening (default 0.4, 0.25) */
    int32_t median_window;      /* odd SDE median window; 0 => 2 floor(N_P/200) + 1 */
    int32_t periods_per_chunk;  /* periods folded per kernel wave; 0 => as many as fit 8 GiB of
                                   scratch (at most 4096), rounded down to a multiple of the SM
                                   count */
    const double* periods_days; /* optional explicit period grid (host, copied); NULL => Ofir */
    int64_t n_periods;          /* length of periods_days */
    int32_t refine_periods;     /* K > 0: re-search the K best periods by SDE(P) with T0 step 1
                                   (Sect. 2.5, two-stage T0 search), then recompute SR/SDE;
                                   0 => coarse pass only (default) */
    int32_t test_flags;         /* 0 for searches (default).  Bit 0: before its first work item
                                   the tensor-core window kernel waits about 1 ms on a barrier
                                   phase that nothing completes, records the timeout and stops,
                                   so that the search returns GTLS_ERR_TIMEOUT: a test of the
                                   bounded-wait path that faults nothing */
} gtls_plan_params;

/* Sizes of a plan (host struct filled by gtls_plan_get_info). */
typedef struct {
    int64_t n_periods;          /* trial periods, ascending */
    int64_t n_points;
    int32_t n_durations;        /* points of the global T14/P grid */
    int32_t time_exponent;      /* e: phases are exact on a 2^-e-day lattice */
    int64_t max_duration_points;/* largest D of any period */
    int64_t n_windows;          /* (period, duration, T0) triples per search */
    double wpe;                 /* window-point evaluations per search: sum of D over windows */
    int64_t device_bytes;       /* device memory the plan holds */
    int32_t median_window;
    int32_t periods_per_chunk;  /* periods folded and searched per kernel wave */
} gtls_plan_info;

/* Best candidate of one search (host struct). */
typedef struct {
    double period;        /* days, argmax of SDE(P) */
    double duration_days; /* q_j * period */
    double t0;            /* mid-transit time of the best window (days, input time system) */
    double depth;         /* fitted depth (fraction) */
    double sde;           /* SDE(P) at the best period */
    double chi2;          /* chi2(P) at the best period */
    double chi2_min;      /* global minimum of chi2(P) */
    double chi2_0;        /* chi2 of the constant model, sum(((y-1)/dy)^2) */
    int64_t period_idx;   /* index into the plan's period grid */
    int32_t dur_idx;      /* index into the global T14/P grid */
    int32_t dur_points;   /* D */
    int64_t t0_idx;       /* window start in folded order (multiple of the T0 step) */
    int32_t uniform_dy;   /* 1 if all dy were equal (uniform-weight kernel) */
    int32_t refined;      /* number of periods re-searched with T0 step 1 */
    double snr;           /* sqrt(max(0, chi2_0 - chi2)): the fit's improvement over the
                             constant model in units of the noise (the paper gives no SNR
                             formula; for white noise this is the matched-filter SNR) */
} gtls_result;

/* Optional per-period outputs (device pointers, each nullable, n_periods long). */
typedef struct {
    double* chi2;     /* chi2(P) */
    int32_t* dur_idx; /* argmin duration (global grid index) */
    int32_t* t0_idx;  /* argmin window start in folded order */
    double* depth;    /* depth at the argmin */
    double* t0;       /* mid-transit time at the argmin (days) */
    double* sr;       /* SR(P) */
    double* sde_raw;  /* SDE_raw(P) */
    double* sde;      /* SDE(P) */
    int32_t* refined; /* 1 where the period was re-searched with T0 step 1, else 0 */
} gtls_period_outputs;

/* Per-stage device time of the last search (host struct). */
typedef struct {
    double ms_prepare;        /* per-curve arrays, t_ref, chi2_0, input checks */
    double ms_fold_sort;      /* fold + sort + gather + prefix sums, all chunks */
    double ms_window_search;  /* depth fit + chi2 of every window, all chunks */
    double ms_finalize;       /* per-period chi2(P), depth, T0 */
    double ms_sr_sde;         /* SR, SDE_raw, running median, argmax */
    int64_t kernel_launches;  /* kernels the last search launched */
    int64_t window_search_launches;
    int32_t enabled;          /* 1 if the times above were measured */
    int32_t reserved0;
} gtls_profile;

/* Fill p with the defaults above (baseline_days and n_points set to 0). */
void gtls_plan_params_default(gtls_plan_params* p);

/*
 * Build the period grid (Eqs. f_min, f_max, f_i, C/A, N), the T14/P grid
 * and per-period ranges (Eqs. upper, lower), the template table and the
 * phase lattice on the host in FP64; upload them and allocate the scratch
 * the search needs on the current CUDA device.  The plan owns all of it.
 * Errors: INVALID_ARG (n_points < 2, baseline <= 0, P_min >= P_max, a period
 * with an empty duration range, a grid too large for the lattice), OOM, CUDA.
 */
gtls_status gtls_plan_create(const gtls_plan_params* p, gtls_plan** out);

gtls_status gtls_plan_get_info(const gtls_plan* plan, gtls_plan_info* out);

/* Copy the period grid (days, ascending; host array of n_periods). */
gtls_status gtls_plan_get_periods(const gtls_plan* plan, double* periods_days);

/* Copy the T14/P grid q_j and D_j (host arrays of n_durations). */
gtls_status gtls_plan_get_durations(const gtls_plan* plan, double* q, int32_t* points);

/* Copy each period's first / last T14/P grid index (host arrays of n_periods). */
gtls_status gtls_plan_get_ranges(const gtls_plan* plan, int32_t* jlo, int32_t* jhi);

/*
 * Search one light curve.  t, y, dy: device arrays of n doubles (n must
 * equal the plan's n_points); the caller owns them; they are read-only and
 * must stay valid until the stream work completes.  y is flux normalised to
 * 1, dy > 0.  Writes *out (host) after synchronising `stream`.  per_period
 * (nullable) receives per-period device outputs.
 * Errors: INVALID_ARG (n mismatch, NaN/inf in t/y/dy, dy <= 0), CUDA.
 */
gtls_status gtls_search(gtls_plan* plan, const double* t, const double* y,
                        const double* dy, int64_t n, void* stream,
                        gtls_result* out, const gtls_period_outputs* per_period);

/*
 * Same as gtls_search for host arrays: copies t, y, dy into plan-owned
 * device buffers on `stream` first (the end-to-end call).
 */
gtls_status gtls_search_host(gtls_plan* plan, const double* t, const double* y,
                             const double* dy, int64_t n, void* stream,
                             gtls_result* out);

/*
 * Batched search of many light curves (no counterpart in the paper, which
 * searches one light curve at a time; its periods of different curves are
 * as independent as those of one curve).  A batch references n_lc plans,
 * one per curve (plans[i] made for curve i's n and baseline; a plan may
 * appear once; the plans must outlive the batch and must not be searched on
 * their own while the batch runs, since the batch writes their per-curve and
 * per-period buffers).  The batch owns one chunk scratch shared by all
 * curves (sized for the largest curve; `wave_slots` periods in flight, 0 =
 * as many as fit 16 GiB, at most 4096, rounded down to a multiple of four
 * times the SM count) and runs the periods of all curves as
 * waves of (curve, period range) segments through the same kernels as
 * gtls_search.  Everything after the per-curve preparation is captured
 * once into a CUDA graph and replayed by later searches (recaptured when
 * the set of curves with uniform dy changes, or after gtls_batch_autotune).
 * The periods of all curves form a device work queue of (curve, first,
 * count) runs per kernel class; a while-loop node of the graph repeats
 * {cut the next wave from the queue's cursor on the device, fold, window
 * kernels, per-period results} until the queue is empty, so the graph's
 * size does not depend on the number of curves or waves, and no kernel
 * waits on another (stream order inside the loop body).
 * Results equal gtls_search on each curve alone.
 * Errors: INVALID_ARG (n_lc outside [1, 65535], null or repeated plans,
 * plans on another device), OOM, CUDA.
 */
typedef struct gtls_batch gtls_batch;

typedef struct gtls_batch_info {
    int64_t n_lc;
    int64_t n_points;          /* all curves */
    int64_t n_periods;         /* trial periods of all curves (coarse pass) */
    double wpe;                /* window-point evaluations of all curves */
    int32_t waves;             /* waves (coarse and refinement) one search runs (0 before the first) */
    int32_t wave_slots;        /* periods per wave */
    int32_t tile_floats;       /* folded-curve floats staged per window-tile item */
    int32_t graph_kernels;     /* kernels in the captured graph, a loop body counted once: the same
                                  for any number of curves of the same kernel classes */
    int64_t last_launches;     /* kernels launched by the last gtls_batch_search */
    int64_t device_bytes;      /* device memory owned by the batch */
    int32_t tuned;             /* 1 after gtls_batch_autotune */
    int32_t reserved0;
    double tuned_flops;        /* probe rate of the chosen configuration (2 x WPE / s) */
} gtls_batch_info;

gtls_status gtls_batch_create(gtls_plan* const* plans, int64_t n_lc, int32_t wave_slots,
                              gtls_batch** out);

/*
 * Search every curve of the batch: curve i is t[offsets[i] .. offsets[i+1])
 * and likewise y, dy (device arrays, caller-owned, read only);
 * offsets: host array of n_lc + 1 entries whose differences equal the
 * plans' n_points.  out: host array of n_lc results.  One stream
 * synchronisation after the preparation (input validation) and one at the
 * end.  Errors: INVALID_ARG (sizes, NaN/inf, dy <= 0; the message names the
 * curve), INTERNAL (a device index check), CUDA.
 */
gtls_status gtls_batch_search(gtls_batch* batch, const double* t, const double* y, const double* dy,
                              const int64_t* offsets, void* stream, gtls_result* out);

/*
 * Choose the wave size (the largest, a half, a quarter) by timing the
 * coarse pass of a probe (four runs of 256 periods spread over each of the
 * first four curves that take the tiled kernel) on these inputs; keeps the
 * fastest.  The staged tile stays the plans' own (the tile decomposition
 * fixes the order in which some window variants sum a window, so it must
 * match the single-curve search).  Results do not depend on the choice.
 * Same arguments as gtls_batch_search.
 */
gtls_status gtls_batch_autotune(gtls_batch* batch, const double* t, const double* y, const double* dy,
                                const int64_t* offsets, void* stream);

gtls_status gtls_batch_get_info(const gtls_batch* batch, gtls_batch_info* out);

/*
 * Per-period outputs of curve lc (0 <= lc < n_lc) from the last
 * gtls_batch_search: device arrays of that curve's n_periods, as in
 * gtls_search (null members are skipped).  Enqueued on `stream`.
 */
gtls_status gtls_batch_get_period_outputs(const gtls_batch* batch, int64_t lc,
                                          const gtls_period_outputs* per, void* stream);

/* Release the batch's device memory and graph (NULL is a no-op). */
void gtls_batch_destroy(gtls_batch* batch);

/*
 * One-call batched search: gtls_batch_create (default wave size),
 * gtls_batch_search, gtls_batch_destroy.  Same arguments and results as
 * gtls_batch_search with the plans given directly (each plan once).
 */
gtls_status gtls_search_batch(gtls_plan* const* plans, int64_t n_lc,
                              const double* t, const double* y, const double* dy,
                              const int64_t* offsets, void* stream,
                              gtls_result* out);

/*
 * The plan's chunk scratch (the folded curves, prefix sums and sort keys of
 * periods_per_chunk periods: plan info device_bytes counts it once it
 * exists) is allocated by the first gtls_search on the plan.
 * gtls_plan_reserve allocates it now (no-op when it exists);
 * gtls_plan_trim frees it (it waits for the device; no-op when absent) and
 * the next search allocates it again.  Many plans can then be kept for one
 * search each without holding one scratch per plan.  Neither changes a
 * result.  Errors: INVALID_ARG (null plan, another current device), OOM,
 * CUDA.
 */
gtls_status gtls_plan_reserve(gtls_plan* plan);
gtls_status gtls_plan_trim(gtls_plan* plan);

/*
 * Measure per-stage device time with CUDA events on the search stream
 * (on != 0) or stop measuring (on == 0; the default).  Measuring adds one
 * event record per stage and chunk; it changes no result.
 */
gtls_status gtls_plan_set_profiling(gtls_plan* plan, int32_t on);

/* Stage times and launch counts of the plan's last search (host struct). */
gtls_status gtls_plan_get_profile(const gtls_plan* plan, gtls_profile* out);

/*
 * SR, SDE_raw, SDE and the SDE argmax of a chi2(P) spectrum without any
 * device allocation.  (The paper has no counterpart: this exists for callers
 * that cannot call cudaMalloc, e.g. code confined to a pre-sized memory pool
 * or to buffers handed over by another framework.)  Its scratch lives in a
 * fixed device array compiled into the library: 2^19 trial periods at most
 * (8 MiB plus a small header, held by every GPU that loads the library until
 * the process exits); larger inputs return GTLS_ERR_INVALID_ARG.
 *   chi2       device, n_periods doubles (input, read only)
 *   sr_out, sde_raw_out   device, n_periods doubles each, nullable (then
 *              kept in the fixed array)
 *   sde_out    device, n_periods doubles (required)
 *   best_idx, best_sde    host, nullable: first index of the largest SDE
 *   median_window         0 => 2 floor(N_P/200) + 1, else odd
 * The computation is the one gtls_search applies to its own chi2(P).
 * Errors: GTLS_ERR_INVALID_ARG when a pointer is not device memory of the
 * current device (checked with cudaPointerGetAttributes, which allocates
 * nothing) or when some chi2 value is not finite and >= 0 (checked on the
 * device; the outputs are then unspecified); GTLS_ERR_INTERNAL when no SDE
 * value can be ranked.
 * The first call on a device looks up the array's device address (with
 * cudaGetSymbolAddress) and sets a kernel attribute; make that first call
 * before any stream capture.  All calls share the array and it keeps the
 * previous call's contents, so calls that overlap on the GPU (different
 * streams, or threads) race; serialise them.  Synchronises `stream`.
 */
gtls_status gtls_sr_sde_noalloc(const double* chi2, int64_t n_periods, int32_t median_window,
                                void* stream, double* sr_out, double* sde_raw_out, double* sde_out,
                                int64_t* best_idx, double* best_sde);

/*
 * Learned period proposal (no counterpart in the paper).  A 1D CNN reads a
 * light curve binned in time (4096 bins, not folded) and predicts, for each
 * of 128 regions that split [0.5, 1024) days evenly in log P, the largest
 * SR(P) that the search finds there; the full search then runs only on the
 * trial periods of the best regions (gtls_proposal_periods), falling back to
 * the whole grid when the prediction is not confident (caller's choice).
 *
 * Network: input x[B][4096]; six 'same' 1D convolutions (taps 7, 5, 5, 5,
 * 5, 5 spaced 1, 2, 2, 4, 4, 8 bins of the layer's input apart:
 * out[l] = b + sum_tap w[tap] x[l + (tap - (taps-1)/2) spacing]; 64 output
 * channels) each with bias, ReLU and max-pooling by 2
 * (pair (2j, 2j+1), the first wins ties); a linear head from the 64 x 64
 * features (feature = position * 64 + channel) to 128 logits; scores =
 * sigmoid(logits).  Loss: masked mean logistic loss with soft targets,
 *   L = sum mask (softplus(z) - target z) / max(1, sum mask).
 * Parameters: one FP32 vector of gtls_cnn_param_count() floats in the order
 * w0 b0 w1 b1 ... w5 b5 wh bh, with conv weights [64][taps][in channels],
 * head weights [128][4096].  The contractions run as BF16 tensor-core GEMMs
 * with FP32 accumulation (activations stored in BF16); master parameters,
 * gradients and Adam moments are FP32.
 * Device pointers below are arrays on the network's device; the network is
 * not thread-safe (one call at a time).
 */
typedef struct gtls_cnn gtls_cnn;

int64_t gtls_cnn_param_count(void);

/* max_batch in [1, 4096]; params: host FP32 vector (NULL = zeros). */
gtls_status gtls_cnn_create(int32_t max_batch, const float* params, gtls_cnn** out);
gtls_status gtls_cnn_get_params(const gtls_cnn* cnn, float* params);
/* Replace the parameters (host vector) and reset the Adam state. */
gtls_status gtls_cnn_set_params(gtls_cnn* cnn, const float* params);

/*
 * Network input of n_lc <= max_batch light curves packed as in
 * gtls_batch_search (t, y, dy device arrays; offsets host, n_lc + 1):
 * x[i][b] (device, n_lc x 4096 floats) = sum(w r) / sqrt(sum w) over the
 * points of curve i with floor((t - t_min) / (t_max - t_min) * 4096) = b
 * (the last point in bin 4095), r = 1 - y, w = 1/dy^2; 0 for empty bins.
 * mean, wsum (device, same shape, nullable): sum(w r) / sum w (0 when
 * empty) and sum w of every bin.  Synchronises `stream`.
 */
gtls_status gtls_cnn_bin(gtls_cnn* cnn, const double* t, const double* y, const double* dy,
                         const int64_t* offsets, int64_t n_lc, float* x, float* mean, float* wsum,
                         void* stream);

/* logits / scores: device [batch][128] floats, each nullable. */
gtls_status gtls_cnn_forward(gtls_cnn* cnn, const float* x, int32_t batch, float* logits,
                             float* scores, void* stream);

/*
 * Loss and gradient for targets / mask (device [batch][128]) without an
 * update: grad (host, gtls_cnn_param_count floats, nullable), loss (host,
 * nullable).  Synchronises `stream`.
 */
gtls_status gtls_cnn_gradient(gtls_cnn* cnn, const float* x, const float* target, const float* mask,
                              int32_t batch, float* grad, double* loss, void* stream);

/* Gradient and one Adam step (beta 0.9 / 0.999, eps 1e-8, learning rate lr). */
gtls_status gtls_cnn_train_step(gtls_cnn* cnn, const float* x, const float* target, const float* mask,
                                int32_t batch, float lr, double* loss, void* stream);

void gtls_cnn_destroy(gtls_cnn* cnn);

/*
 * Host helpers of the proposal.  Region of a period: floor(128 log(P/0.5) /
 * log(2048)); periods outside [0.5, 1024) belong to none.
 * gtls_region_targets: target[r] = largest sr[i] of region r's periods
 *   (sr: any per-period spectrum; training uses the clipped, scaled SDE),
 *   mask[r] = 1 where region r holds a period (host arrays of 128 floats).
 * gtls_proposal_periods: indices (ascending, into idx of n_periods capacity)
 *   of the periods inside the ceil(frac x regions holding a period) regions
 *   of largest score (ties: lower region first); *n_idx receives the count.
 */
gtls_status gtls_region_targets(const double* periods, const double* sr, int64_t n_periods,
                                float* target, float* mask);
gtls_status gtls_proposal_periods(const double* periods, int64_t n_periods, const float* scores,
                                  double frac, int64_t* idx, int64_t* n_idx);

/* Release the plan's device and host memory (NULL is a no-op). */
void gtls_plan_destroy(gtls_plan* plan);

/* Message of the last failure on the calling thread ("" if none). */
const char* gtls_last_error(void);

/* Name of a status code. */
const char* gtls_status_string(gtls_status s);

#ifdef __cplusplus
}
#endif

#endif /* GTLS_H */
