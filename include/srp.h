/*
 * srp.h -- C ABI of the GB300 steered response power (SRP) mapping library.
 *
 * Computes, per STFT frame, the SRP map of J candidate locations from the
 * PHAT-weighted cross spectra of all Q = M(M-1)/2 microphone pairs, either
 * conventionally (Sec. 2.3-2.4: the GCC of every pair evaluated at every
 * candidate's TDOA by a discrete inverse Fourier transform, Eq. GCC_IFT and
 * Eq. SRP_T_IFT) or by the Nyquist-Shannon approximation (Sec. 3: each GCC
 * sampled at the critical lags covering its bounded TDOA interval, then
 * interpolated with a truncated sinc series, Eq. SRPapprox, and summed over
 * pairs), followed by the per-frame maximiser (Sec. 2.2).
 *
 * Units and conventions (they fix the constant factors the paper leaves open):
 *  - K is the DFT length (even); inputs carry Kb = K/2 + 1 one-sided bins.
 *  - The critical sampling period is T = 1/fs (omega_0 = pi fs, Sec. 3.1);
 *    TDOAs and lags are measured in samples.
 *  - Pairs q <-> (m, m'), m > m', enumerated m' = 0..M-2 (outer),
 *    m = m'+1..M-1 (inner); psi_q(k) = y_m(k) y_m'(k)^* / |y_m(k) y_m'(k)^*|
 *    (Eq. corrmatrix with the PHAT weight), 0 where the denominator is 0.
 *  - The map value is sum_q xi_q(x_iq) with
 *    xi_q(x) = (1/K) sum_{k=0}^{K/2} a_k Re[psi_q(k) e^{j 2 pi k x / K}],
 *    a_0 = a_{K/2} = 1 and a_k = 2 otherwise (the two-sided frequency
 *    integral of Eq. SRP_T without its constant factor 2).
 *  - Nyquist mode samples xi_q at n = -(N_q+N_aux) .. N_q+N_aux with
 *    N_q = floor(d_q fs / c) (Eq. SRPapprox) and interpolates with
 *    sinc(u) = sin(pi u)/(pi u).
 *
 * Memory: the library copies the geometry, builds every plan table on the
 * device and owns it together with the scratch buffers a call needs; the
 * caller owns all input and output buffers.  Device pointers are plain CUDA
 * device addresses on the device that was current when the plan was built.
 *
 * Execution: srp_map and the other stage entry points only enqueue work on
 * the given stream and return; they never synchronise.  Calls on one handle
 * share its scratch buffers and must be ordered (one stream, or the caller
 * synchronises between streams).  Distinct handles are independent.
 *
 * Errors are returned as srp_status codes, never thrown or trapped; a
 * failing CUDA call maps to SRP_ERR_CUDA and srp_last_error_message() holds
 * the CUDA error text for the calling thread.
 */
#ifndef SRP_H
#define SRP_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SRP_API __attribute__((visibility("default")))
#else
#define SRP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st *srp_stream_t;

typedef enum {
    SRP_OK = 0,
    SRP_ERR_INVALID_ARG = 1, /* an argument is out of range or NULL */
    SRP_ERR_OOM = 2,         /* a device or host allocation failed */
    SRP_ERR_CUDA = 3,        /* a CUDA call failed (see srp_last_error_message) */
    SRP_ERR_UNSUPPORTED = 4, /* valid request the library does not implement */
    SRP_ERR_TIMEOUT = 5      /* a bounded device wait gave up */
} srp_status;

typedef enum {
    SRP_MODE_CONV = 1,   /* conventional SRP, Sec. 2.3-2.4 */
    SRP_MODE_NYQUIST = 2 /* Nyquist-Shannon approximation, Sec. 3.2 */
} srp_mode;

typedef enum {
    SRP_PREC_FP32 = 0, /* contractions in FP32 arithmetic */
    SRP_PREC_BF16 = 1, /* contraction operands in BF16, FP32 accumulation */
    SRP_PREC_FP16 = 2  /* contraction operands in FP16, FP32 accumulation */
} srp_precision;

typedef enum {
    SRP_GRID_POINTS = 0,    /* candidates are points q_i (near field, Eq. Deltat_i) */
    SRP_GRID_DIRECTIONS = 1 /* candidates are unit vectors r_i (far field, Eq. Deltat_i_spher) */
} srp_grid_kind;

typedef enum {
    SRP_IN_STFT = 0, /* input y[L][M][Kb] complex64 (interleaved re, im) STFT frames */
    SRP_IN_CROSS = 1 /* input psi[L][Q][Kb] complex64 cross spectra, already weighted */
} srp_input_kind;

typedef enum {
    SRP_WEIGHT_PHAT = 0, /* PHAT weighting: psi = y_m y_m'^* / |y_m y_m'^*| (Sec. 2.1) */
    SRP_WEIGHT_NONE = 1  /* no weighting: psi = y_m y_m'^* (plain cross power; the
                            method holds for any weighting, Sec. 2.1).  With
                            single-frame spectra the SCOT weighting equals PHAT */
} srp_weighting;

typedef enum {
    SRP_ENGINE_AUTO = 0,      /* tensor cores (tcgen05) where built, else CUDA cores */
    SRP_ENGINE_CUDA_CORES = 1 /* FP32 CUDA-core kernels only (FP32 precision) */
} srp_engine;

typedef enum {
    SRP_ARGMAX_RESCORE = 0, /* BF16/FP16 tensor-core plans: the maximiser is chosen in FP32
                               (see srp_map); FP32 plans: the map's own first maximiser */
    SRP_ARGMAX_MAP = 1      /* always the first maximiser of the computed map */
} srp_argmax_mode;

typedef struct {
    int32_t M;                /* microphones, 2 <= M <= 64 */
    const double *mic_xyz;    /* host [M][3] metres; copied by srp_plan */
    srp_grid_kind grid_kind;  /* points or far-field directions */
    int64_t J;                /* candidates, 1 <= J <= 2^31 - 2^20 */
    const double *grid_xyz;   /* host [J][3] metres or unit vectors; copied */
    double fs;                /* sampling rate in Hz (> 0); T = 1/fs */
    double c;                 /* speed of sound in m/s (> 0) */
    int32_t K;                /* DFT length, even, 4 <= K <= 8192 */
    srp_mode mode;            /* conventional or Nyquist */
    int32_t n_aux;            /* auxiliary samples N_aux >= 0 (Nyquist only) */
    srp_precision precision;  /* arithmetic of the map contraction */
    srp_input_kind input_kind;/* STFT frames or ready cross spectra */
    int32_t max_frames;       /* largest L a call may pass, >= 1 */
    int32_t host_io;          /* staging slots for the host entry points: 0 none,
                                 1 for srp_map_host, 2 also for srp_map_host_async */
    srp_engine engine;        /* which units run the map contraction */
    srp_weighting weighting;  /* GCC weighting of STFT input (ignored for cross spectra);
                                 SRP_WEIGHT_NONE is not available with SRP_PREC_FP16,
                                 whose range unnormalised spectra can exceed */
    float resident_fraction;  /* in [0, 1] (Nyquist, tensor cores): the part of the sinc
                                 interpolation matrix of Eq. SRPapprox (counted in 16-lag
                                 steps, whole pairs, interleaved with the others) that is
                                 computed once, at plan time, kept in device memory
                                 (J_pad x its lag slots x 2 bytes, twice for FP32) and
                                 streamed into every map; the rest is generated on chip
                                 while it streams.  0: all generated; 1: all streamed.
                                 The maps are the same either way */
    srp_argmax_mode argmax;   /* how the per-frame maximiser is decided (default 0) */
} srp_plan_desc;

/* Sizes of a plan, computed on the host (no device needed). */
typedef struct {
    int32_t M, Q, K, Kb;
    int64_t J;
    int32_t n_aux;
    int32_t S;           /* total critical samples sum_q (2 N_q + 2 N_aux + 1); 0 for conventional */
    int32_t max_nq;      /* max_q N_q */
    int32_t x_frac_bits; /* fractional bits of the fixed-point TDOA table */
    int32_t max_frames;
    int32_t tensor_cores; /* 1: the map runs on the tensor cores (tcgen05), 0: CUDA cores.
                             The tensor cores' FP32 accumulation carries a bias of about
                             1.5e-8 per 16-element step; an FP32 plan whose reduction is
                             long enough for it to reach half the 1e-4 tolerance
                             promotes its accumulators (accum_promotion), or, with more
                             than 64 frames per call (Nyquist maps, which never need it,
                             aside), runs on CUDA cores */
    size_t device_bytes;  /* bytes srp_plan allocates on the device */
    size_t weight_bytes;  /* of which the resident interpolation matrix (0 if generated) */
    int32_t argmax_rescored; /* 1: srp_map chooses the maximiser in FP32 (reduced-precision
                                tensor-core plan with SRP_ARGMAX_RESCORE) */
    int32_t accum_promotion; /* FP32 conventional maps on the tensor cores: every this many
                                64-slot chunks of the reduction, the accumulators are added
                                into FP32 sums and restarted (0: never) */
    int32_t gcc_tensor_cores; /* 1: the critical GCC samples (Eq. GCC_IFT at tau = nT) are
                                 the tensor cores' partial inverse DFT (Nyquist tensor-core
                                 plans with PHAT-weighted STFT input, K a multiple of 64,
                                 2 (max N_q + N_aux) + 1 <= 128); 0: CUDA cores */
} srp_plan_info;

typedef struct srp_plan_s *srp_handle;

/* Validate a descriptor and report its sizes and the lag count N_q of every
 * pair (Nq_out: host [Q] or NULL).  N_q = floor(d_q fs / c) follows
 * Eq. SRPapprox with T = 1/fs.  Host only: touches no device.            */
SRP_API srp_status srp_plan_describe(const srp_plan_desc *d, srp_plan_info *info, int32_t *Nq_out);

/* Operation counts of Sec. 3.3 (and of Sec. 2.3 for the conventional map)
 * for a descriptor, as the paper defines them, with P = Q pairs and K_b =
 * K / 2 one-sided bins (a 2048-point DFT gives K_b = 1024, the paper's K):
 *   N      = (2/P) sum_q N_q + 2 N_aux + 1   critical samples per pair
 *   C_samp = N P K_b   complex multiplications of the partial IDFT
 *   C_int  = N P J     real multiplications of the sinc interpolation
 *   C_conv = J P K_b   complex multiplications of the conventional map
 *   R_samp = N / J,  R_int = N / K_b,  R = R_samp + R_int.
 * N_aux of the descriptor is used in either mode.  The counts are per frame
 * and are not the operation counts of this library's kernels.  Host only:
 * touches no device.  Errors: those of srp_plan_describe; NULL out is
 * SRP_ERR_INVALID_ARG.                                                     */
typedef struct {
    double N;            /* average critical samples per pair */
    int32_t P;           /* microphone pairs */
    int32_t K_b;         /* one-sided frequency bins, K / 2 */
    int64_t J;           /* candidates */
    double C_samp, C_int, C_conv;
    double R_samp, R_int, R;
} srp_complexity;

SRP_API srp_status srp_plan_complexity(const srp_plan_desc *d, srp_complexity *out);

/* Device bytes srp_plan would allocate for d (host only).                */
SRP_API srp_status srp_plan_footprint(const srp_plan_desc *d, size_t *device_bytes);

/* Build a plan on the current device: pair table, TDOAs of every candidate
 * and pair (Eq. Deltat_i or Eq. Deltat_i_spher, computed in FP64 and stored
 * as fixed point of x = Delta t / T), lag tables (Eq. SRPapprox), twiddles
 * and scratch.  *out is set only on SRP_OK.  The only blocking call.     */
SRP_API srp_status srp_plan(const srp_plan_desc *d, srp_handle *out);

/* Sizes of a built plan.                                                  */
SRP_API srp_status srp_plan_get_info(srp_handle h, srp_plan_info *info);

/* Copy the plan's TDOA table back, decoded to samples: host x[J][Q]
 * (double).  Synchronous; for checking the plan against its definition.  */
SRP_API srp_status srp_plan_tdoa(srp_handle h, double *x_host);

/* The whole hot path for L frames (0 <= L <= max_frames), Sec. 3.2 order:
 *   d_in    device input, layout per input_kind (read only);
 *   d_maps  device [L][J] float maps, row-major by frame, or NULL to skip
 *           writing maps (argmax and peak are still produced);
 *   d_argmax device [L] int32: lowest-index maximiser of each frame's map;
 *   d_peak  device [L] float map value at d_argmax, or NULL.
 * Asynchronous on stream s.  The tensor-core engine runs three kernels
 * (GCC samples or conventional operands, formed from STFT input directly;
 * the map contraction; the per-frame argmax), the CUDA-core engine four
 * (cross spectra first).
 * Reduced precision (BF16/FP16 operands, argmax SRP_ARGMAX_RESCORE): the
 * maps are those of the reduced-precision contraction, but the maximiser is
 * decided in FP32.  Let m be the frame's largest map value.  Every
 * 128-candidate tile whose largest value is at least m - 0.02 |m| (twice the
 * 1e-2 x peak error bound of these maps below the maximum, so the tile of
 * the exact maximiser is among them whenever the bound holds and the
 * frame's peak is its maximum) is evaluated again candidate by candidate in
 * FP32 (Eq. SRPapprox from FP32 GCC samples, or Eq. GCC_IFT from the FP32
 * cross spectra), and d_argmax / d_peak are the lowest-index maximiser of
 * those FP32 values and its FP32 value.  If more than 64 tiles qualify
 * (a nearly flat map) the frame keeps the first maximiser of its
 * reduced-precision map.                                                  */
SRP_API srp_status srp_map(srp_handle h, const void *d_in, int32_t L, float *d_maps,
                   int32_t *d_argmax, float *d_peak, srp_stream_t s);

/* srp_map from and to host memory (pinned memory makes the copies
 * asynchronous): copies h_in to the plan's staging buffer, runs srp_map,
 * copies results back and synchronises s before returning.  Where the GPU
 * reaches host memory coherently (NVLink-C2C) and h_maps is pinned, the map
 * kernel stores the maps straight into h_maps instead of a staging buffer
 * and a copy.  Needs a plan built with host_io != 0.  h_maps and h_peak may
 * be NULL.                                                                */
SRP_API srp_status srp_map_host(srp_handle h, const void *h_in, int32_t L, float *h_maps,
                        int32_t *h_argmax, float *h_peak, srp_stream_t s);

/* Pipelined host entry point (plan built with host_io = 2): enqueues the
 * copy of h_in to one of two device staging slots on an internal copy
 * stream, the map on stream s, and the copies of the results back to h_maps
 * (may be NULL), h_argmax and h_peak (may be NULL) on a second internal copy
 * stream, ordered by events, and returns without waiting.  Consecutive calls
 * alternate the slots, so the copies of one call overlap the maps of its
 * neighbours; the maps themselves run in order on s.  h_in must stay
 * unchanged and the result buffers untouched until srp_map_host_wait
 * returns (pinned host memory keeps the copies asynchronous).  Do not mix
 * with srp_map_host on the same plan without a srp_map_host_wait between.  */
SRP_API srp_status srp_map_host_async(srp_handle h, const void *h_in, int32_t L, float *h_maps,
                                      int32_t *h_argmax, float *h_peak, srp_stream_t s);

/* Wait until every srp_map_host_async call on h has delivered its results,
 * then poll the device status as srp_poll_device_status does.            */
SRP_API srp_status srp_map_host_wait(srp_handle h);

/* First stage alone: cross spectra psi[L][Q][Kb] complex64 from STFT
 * frames y[L][M][Kb] (Eq. corrmatrix with the plan's GCC weighting, Sec. 2.1).
 * Plan must take SRP_IN_STFT.  Asynchronous on s.                         */
SRP_API srp_status srp_cross_spectra(srp_handle h, const void *d_y, int32_t L, void *d_psi,
                             srp_stream_t s);

/* Critical GCC samples of a Nyquist plan (Sec. 3.2, first step): for each
 * frame and pair q, xi_q(n) for n = -(N_q+N_aux)..N_q+N_aux, pairs
 * concatenated in pair order, written as float d_xi[L][S].  Input as for
 * srp_map.  Asynchronous on s.                                            */
SRP_API srp_status srp_gcc_samples(srp_handle h, const void *d_in, int32_t L, float *d_xi,
                           srp_stream_t s);

/* srp_gcc_samples without a plan and without any device allocation.  The
 * paper has no counterpart: this entry exists for callers that may not call
 * cudaMalloc, e.g. code inside a host application whose device allocator is
 * owned by someone else, or a real-time audio thread that must not block on
 * the allocator.  Everything a plan would allocate is replaced:
 *  - the cross spectra between the two kernels go to one file-scope device
 *    array of 8 MiB, which every GPU that loads this library holds until the
 *    process exits; L * Q * (K/2+1) * 8 bytes must fit in it, else the call
 *    returns SRP_ERR_INVALID_ARG and launches nothing;
 *  - the pair table travels as a kernel argument, so M <= 16;
 *  - twiddles are generated on the device.
 * Inputs: M and K as in srp_plan_desc, n_aux >= 0, Nq host [Q] lag counts
 * (for example from srp_plan_describe, which is host-only), d_y device
 * y[L][M][Kb] complex64, 0 <= L <= 65535.  Output: d_xi device float
 * [L][S], exactly as srp_gcc_samples writes it.  Asynchronous on s.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and sets the kernels' shared-memory limit, once,
 * with that device current; make that first call before any stream
 * capture.  All calls share the one array and every call
 * overwrites the part it reads, so nothing carries over between calls, but
 * calls whose work overlaps on the GPU (other streams, other threads) race
 * on it: order them.                                                     */
SRP_API srp_status srp_gcc_samples_static(int32_t M, int32_t K, int32_t n_aux,
                                          const int32_t *Nq, const void *d_y, int32_t L,
                                          float *d_xi, srp_stream_t s);

/* Device error flags raised since the previous poll, read on stream s
 * (which is synchronised) and cleared.  Returns SRP_ERR_TIMEOUT if a
 * bounded wait inside a tensor-core kernel gave up (the kernel then
 * returned early and its outputs are invalid), SRP_ERR_INVALID_ARG if
 * srp_refine met a centre index outside [0, J), else SRP_OK.
 * srp_map_host polls by itself.                                           */
SRP_API srp_status srp_poll_device_status(srp_handle h, srp_stream_t s);

/* Per-stage timing: when enabled, srp_map records CUDA events around each
 * stage on its stream; srp_stage_times waits for the last call's events and
 * returns milliseconds per stage in ms[0..n): 0 cross spectra, 1 GCC
 * samples, 2 map contraction, 3 argmax reduction (0 for a skipped stage;
 * on the tensor-core engine stage 1 includes forming the cross spectra, and
 * stage 0 is 0).                                                          */
SRP_API srp_status srp_set_timing(srp_handle h, int32_t enable);
SRP_API srp_status srp_stage_times(srp_handle h, float *ms, int32_t n);

/* Number of kernels the last srp_map call launched.                       */
SRP_API srp_status srp_last_launch_count(srp_handle h, int32_t *n);

/* Release every device and host resource of the plan.  NULL is a no-op.  */
SRP_API srp_status srp_destroy(srp_handle h);

/* ------------------------------------------------------------------------
 * Coarse-to-fine search on the interpolated map.  Sec. 3.3 notes that the
 * interpolation cost R_int = N/K falls far lower when, instead of every
 * candidate of a fine grid, only points near a coarse maximiser are
 * evaluated (a refinement the paper leaves outside its scope).  A refiner
 * evaluates the approximation of Eq. SRPapprox, summed over pairs as in
 * Eq. SRP_T_IFT, at arbitrary points, from the GCC samples of its plan's
 * last map:
 *   level 0 evaluates the points c + o_f (f < F) around the frame's centre c,
 *   level v evaluates c_v + shrink^v o_f around the best point c_v of level
 *   v - 1 (the first maximiser: the largest value, the lowest f),
 * and the best point of the last level is the result.  On a direction grid
 * (SRP_GRID_DIRECTIONS) every displaced point is normalised back onto the
 * unit sphere.  TDOAs are computed from the geometry (Eq. Deltat_i or
 * Eq. Deltat_i_spher) in FP32, relative to the microphones' centroid and
 * with the distance difference in a form without cancellation, not
 * quantised like the plan's table; the centres are kept in FP64; the
 * samples are read in the precision the map used.  Nyquist plans only.
 * ------------------------------------------------------------------------ */
typedef struct srp_refiner_s *srp_refiner;

typedef struct {
    int32_t n_offsets;      /* F in [1, 1024]: points per level */
    const double *offsets;  /* host [F][3] displacements o_f of level 0 (metres on a point
                               grid, unit-vector components on a direction grid); copied */
    int32_t levels;         /* in [1, 64] */
    double shrink;          /* in (0, 1]: level v scales the displacements by shrink^v */
    int32_t keep_grid;      /* 1: copy the plan's grid to the device so that srp_refine
                               can take centres as candidate indices (e.g. the argmax of
                               srp_map); 0: centres are given as coordinates */
} srp_refine_desc;

/* Build a refiner for plan h.  d must be the descriptor h was built from
 * (its geometry is read again: microphones, and the grid with keep_grid);
 * a descriptor that differs in M, J, K, N_aux, fs, c, grid kind or lag
 * counts is SRP_ERR_INVALID_ARG, a conventional plan SRP_ERR_UNSUPPORTED.
 * Allocates 24 (M + F) bytes on the plan's device, plus 24 J with
 * keep_grid.  h must outlive the refiner.  Blocking.                      */
SRP_API srp_status srp_refiner_create(srp_handle h, const srp_plan_desc *d,
                                      const srp_refine_desc *r, srp_refiner *out);

/* Refine frames 0 .. L-1 of the plan's last srp_map, srp_map_host or
 * srp_map_host_async call (not srp_map_batch, whose samples live in the
 * batch), enqueued on s after that call and before the plan's next map.
 * L in [0, frames of that call].  Centres: exactly one of d_argmax (device
 * [L] candidate indices; needs keep_grid) and d_centres (device [L][3]
 * coordinates).  Outputs (device): d_best_xyz [L][3] the best point of the
 * last level, d_best_val [L] its value, d_values [L][F] every value of the
 * last level, or NULL.  A centre index outside [0, J) makes that frame's
 * outputs NaN and is reported by srp_poll_device_status as
 * SRP_ERR_INVALID_ARG.  One kernel launch, asynchronous.                 */
SRP_API srp_status srp_refine(srp_refiner r, int32_t L, const int32_t *d_argmax,
                              const double *d_centres, double *d_best_xyz, float *d_best_val,
                              float *d_values, srp_stream_t s);

/* Release the refiner's device tables.  NULL is a no-op.                  */
SRP_API srp_status srp_refiner_destroy(srp_refiner r);

/* ------------------------------------------------------------------------
 * Batched uneven instances.  The paper maps one array at a time; a batch
 * maps several plans (arrays with their own M, J, K and geometry) in one
 * CUDA-graph launch of three kernels: the PHAT cross spectra and contraction
 * operands of every (plan, frame, pair) row; one persistent tensor-core
 * kernel running the map contraction of every plan (Eq. SRPapprox, or
 * Eq. GCC_IFT at every TDOA for the conventional map, summed over pairs) over
 * a work list of (plan, 128-candidate tile, frame tile) items, spread over
 * the SMs longest-first onto the least-loaded CTA; and the per-frame argmax
 * of every plan.  Each plan's maps, argmax and peak are exactly what srp_map
 * defines, up to floating-point rounding; BF16/FP16 Nyquist plans that re-score
 * their maximiser (srp_plan_info.argmax_rescored) re-score it in the batch
 * too, while conventional BF16/FP16 plans keep their map's own maximiser in a
 * batch.
 *
 * The batch reads the plans' device tables in place (the plans must outlive
 * the batch and must not be destroyed while it is in use) and owns its own
 * operand buffer, argmax partials, work list and graph, so the plans stay
 * usable by srp_map.  All plans must be on one device, share mode and
 * precision, and run on the tensor cores (srp_plan_info.tensor_cores == 1);
 * otherwise srp_batch_create returns SRP_ERR_UNSUPPORTED.  FP32 conventional
 * plans that promote their accumulators (srp_plan_info.accum_promotion > 0)
 * promote them in the batch too, every accum_promotion chunks; a batch that
 * holds such a plan keeps operand A in tensor memory and at most two CTAs per
 * SM.  Calls on one batch share its buffers and must be ordered, like calls on
 * one plan.
 * ------------------------------------------------------------------------ */
typedef struct srp_batch_s *srp_batch;

/* Tile shape of the persistent contraction kernel. */
typedef struct {
    int32_t frames_per_tile; /* frames per work item (the MMA N): a multiple of 16 in
                                [16, 128]; 0 = the largest max_frames rounded up to 16,
                                at most 64 */
    int32_t stages;          /* operand pipeline depth in [2, 4]; 0 = the most that fit */
    int32_t ctas_per_sm;     /* persistent CTAs per SM, 1, 2 or 4 (4: BF16/FP16 with A in
                                TMEM, 128 TMEM columns per CTA); 0 = the most that fit */
    int32_t operand_a;       /* where the generated operand A lives: 1 = tensor memory
                                (the MMAs read only B from shared memory), 2 = shared
                                memory; 0 = tensor memory where it fits */
    int32_t accumulators;    /* accumulators per work item: 2 = two MMA-issuing warps,
                                each summing every other 16-slot step into its own
                                accumulator (the epilogue adds the two); 1 = one warp and
                                one accumulator (half the TMEM columns), refused for an
                                FP32 batch whose longest reduction (per promotion epoch,
                                for a promoted plan) would accumulate a TMEM rounding
                                bias above 5e-5 in one accumulator; 0 = 2
                                where the tile fits, else 1 */
} srp_batch_tiles;

typedef struct {
    int32_t n;              /* plans in the batch */
    int32_t items;          /* work items (every plan at max_frames) */
    int32_t ctas;           /* persistent CTAs of the contraction kernel */
    srp_batch_tiles tiles;  /* tile shape in use */
    int32_t launches;       /* kernels per srp_map_batch call (all in one graph launch) */
    int32_t tuned;          /* 1 once srp_batch_tune has chosen the tiles */
    float tuned_ms;         /* one call with the chosen tiles, as timed by the tuner */
    size_t device_bytes;    /* device bytes the batch owns (the plans' own excluded) */
} srp_batch_info;

/* Build a batch over n >= 1 plans (host array of handles, copied).  tiles
 * may be NULL (defaults) and its zero fields take defaults.  Blocking.    */
SRP_API srp_status srp_batch_create(const srp_handle *plans, int32_t n,
                                    const srp_batch_tiles *tiles, srp_batch *out);

/* Map every plan of the batch, as srp_map would each one.  All arguments are
 * host arrays of n entries holding device pointers (or, for L, frame
 * counts): d_in[i] input of plan i in its input_kind layout; L[i] in
 * [0, max_frames of plan i] (a plan with L[i] = 0 is skipped and its
 * pointers are not read); d_maps[i] device [L][J] maps of plan i or NULL
 * (d_maps itself may be NULL: no maps); d_argmax[i] device [L] int32;
 * d_peak[i] device [L] float or NULL (d_peak may be NULL).  Enqueues one
 * host-to-device copy of the call table and one graph launch on s; waits
 * only for the previous call's table copy to finish.                      */
SRP_API srp_status srp_map_batch(srp_batch b, const void *const *d_in, const int32_t *L,
                                 float *const *d_maps, int32_t *const *d_argmax,
                                 float *const *d_peak, srp_stream_t s);

/* Autotuner: runs the call above with every tile shape that fits (frames per
 * item 16, 32, 64, 128 up to the largest L[i]; 2-4 stages; 1 or 2 CTAs per
 * SM; operand A in tensor or shared memory), times each by CUDA events on
 * s, keeps the fastest and leaves the outputs of a final run with it.
 * Blocking.                                                               */
SRP_API srp_status srp_batch_tune(srp_batch b, const void *const *d_in, const int32_t *L,
                                  float *const *d_maps, int32_t *const *d_argmax,
                                  float *const *d_peak, srp_stream_t s);

SRP_API srp_status srp_batch_get_info(srp_batch b, srp_batch_info *info);

/* Per-kernel timing: while enabled, srp_map_batch launches the same three
 * kernels directly instead of through the graph, with CUDA events around
 * each; srp_batch_stage_times waits for the last call and returns its
 * milliseconds in ms[0..n): 0 operands (cross spectra and GCC samples or
 * bin operands), 1 map contraction, 2 argmax.                              */
SRP_API srp_status srp_batch_set_timing(srp_batch b, int32_t enable);
SRP_API srp_status srp_batch_stage_times(srp_batch b, float *ms, int32_t n);

/* As srp_poll_device_status, for the batch's kernels.                      */
SRP_API srp_status srp_batch_poll_device_status(srp_batch b, srp_stream_t s);

/* Release the batch (not its plans).  NULL is a no-op.                    */
SRP_API srp_status srp_batch_destroy(srp_batch b);

/* ------------------------------------------------------------------------
 * Serving: many arrays (streams, one resident plan each) whose frame blocks
 * arrive over time, mapped by continuous batching.  The paper has no
 * counterpart; each result is the map, argmax and peak srp_map defines for
 * the request's frames alone.
 *
 * A worker thread forms iterations: each stream's queued requests, in
 * arrival order and up to the plan's max_frames, become one group of
 * consecutive frames; the groups of an iteration are mapped together (one
 * srp_map_batch launch over the tensor-core plans of one mode and precision,
 * srp_map for every other plan).  Up to max_inflight iterations are on the
 * GPU at once, each on its own CUDA stream, so requests that arrive while
 * others run join the next iteration as soon as a slot and memory free up,
 * and its copies and kernels overlap the running ones.  Admission is by
 * device memory: each group's inputs, maps, argmax and peak are carved from
 * one device arena of device_budget_bytes; a group that does not fit waits
 * for earlier ones to finish.  The plans must outlive the server.
 * ------------------------------------------------------------------------ */
typedef struct srp_server_s *srp_server;

typedef struct {
    size_t device_budget_bytes; /* device arena for the requests in flight (> 0) */
    size_t host_budget_bytes;   /* pinned host staging for queued and in-flight requests (> 0) */
    int32_t max_inflight;       /* iterations on the GPU at once, 1..8 */
    int32_t no_batching;        /* nonzero: every plan maps with its own srp_map call */
} srp_server_desc;

/* One finished request.  Times are milliseconds since srp_server_create on
 * the host's steady clock: submission, start of its iteration, and the
 * moment its results were in the caller's buffers.  The iteration fields
 * describe the iteration that mapped it: its sequence number (from 1), how
 * many streams' groups and frames it carried, and the GPU interval of its
 * work (CUDA events at the start of its first copy and after its last,
 * milliseconds since an event recorded at srp_server_create; 0 when the
 * request did not run).                                                  */
typedef struct {
    uint64_t request_id, tag;
    int32_t stream, L;
    int32_t status;             /* SRP_OK, SRP_ERR_TIMEOUT (deadline passed before it
                                   started) or the error of its iteration */
    int32_t iteration_streams, iteration_frames;
    int64_t iteration;
    double t_submit_ms, t_start_ms, t_done_ms;
    double t_gpu_start_ms, t_gpu_end_ms;
} srp_completion;

typedef struct {
    int64_t submitted, completed, frames_completed, rejected, timed_out, failed;
    int64_t iterations, kernel_launches, admission_waits, queued;
    size_t device_budget_bytes, device_bytes_in_use, device_bytes_peak;
    int32_t batched_streams;    /* streams mapped by the batched launch */
    int32_t max_iteration_streams;  /* most streams' groups in one iteration */
    /* iterations whose GPU interval intersected that of another iteration
     * (their copies and kernels were on the device at the same time)     */
    int64_t overlapped_iterations;
} srp_server_stats;

/* Start a server over n plans (stream i maps with plans[i]).  Allocates the
 * device arena, the pinned staging, max_inflight CUDA streams and (when two
 * or more plans share a tensor-core mode and precision) one batch per
 * in-flight slot, and starts the worker thread.                          */
SRP_API srp_status srp_server_create(const srp_handle *plans, int32_t n,
                                     const srp_server_desc *d, srp_server *out);

/* Queue L frames (1 <= L <= max_frames of the stream's plan) of host input
 * h_in in the plan's input_kind layout; it is copied before this returns.
 * Results go to host h_argmax [L] (required), h_peak [L] and h_maps [L][J]
 * (optional; pinned memory keeps the maps copy asynchronous), which must stay
 * valid until the request's completion is polled.  deadline_ms > 0: a
 * request not started within that many ms completes with SRP_ERR_TIMEOUT.
 * Returns SRP_ERR_OOM (and queues nothing) when the request alone exceeds
 * the device budget or the pinned staging is full.                      */
SRP_API srp_status srp_server_submit(srp_server s, int32_t stream, const void *h_in, int32_t L,
                                     int32_t *h_argmax, float *h_peak, float *h_maps,
                                     uint64_t tag, double deadline_ms, uint64_t *request_id);

/* Move up to max finished requests into out (oldest first); *n_out is the
 * count.  wait_ms > 0 waits up to that long for one to finish.            */
SRP_API srp_status srp_server_poll(srp_server s, srp_completion *out, int32_t max,
                                   int32_t *n_out, int32_t wait_ms);

/* hold != 0: keep queueing submitted requests but start no new iteration
 * (iterations already on the GPU finish and are delivered); hold = 0:
 * resume, and the next iterations take everything queued meanwhile (each
 * stream's group up to its plan's max_frames).  A batching window for a
 * caller that submits a burst, e.g. frames of many arrays that belong
 * together.  srp_server_destroy releases a hold.                          */
SRP_API srp_status srp_server_hold(srp_server s, int32_t hold);

SRP_API srp_status srp_server_get_stats(srp_server s, srp_server_stats *st);

/* Finish every queued request, stop the worker and release the server (not
 * its plans).  Completions not yet polled are dropped.  NULL is a no-op.  */
SRP_API srp_status srp_server_destroy(srp_server s);

/* Static description of a status code.                                    */
SRP_API const char *srp_status_string(srp_status s);

/* Detail of the calling thread's most recent error ("" if none).          */
SRP_API const char *srp_last_error_message(void);

#ifdef __cplusplus
}
#endif

#endif /* SRP_H */
