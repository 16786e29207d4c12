/*
 * sfft.h -- C ABI of libsfft, a GB300 (sm_103a) implementation of the aliasing-filter
 * sparse FFT with peeling decoding (FFAST for exactly sparse spectra, R-FFAST for noisy
 * ones), after Li, Jiang, Chen, "On Performance of Sparse Fast Fourier Transform
 * Algorithms Using the Aliasing Filter", arXiv 2011.05749, Sec. 2-4.
 *
 * Problem (Sec. 2.1): a length-N signal x whose spectrum xhat (Eq. 2, normalised by 1/N)
 * has K significant coefficients.  The library returns their positions and values.
 *
 * Method (Sec. 2.2, Sec. 3.2, Sec. 4.2):
 *   1. bucketization: for every stage d (subsampling factor L_d = f[d], B_d = N / L_d
 *      buckets, Eq. 5) and every delay tau_{d,r} (Eq. 3-4), the B_d-point DFT of the
 *      delayed subsample (Eq. 6, Eq. 19):
 *        Y_{d,r}[j] = sum_{m<B_d} x[(m L_d + tau_{d,r}) mod N] e^{-2 pi i j m / B_d}
 *                   = B_d * sum_{k = j mod B_d} xhat_k e^{+2 pi i k tau_{d,r} / N};
 *   2. classification of every bin as zero-ton, single-ton or multi-ton (Sec. 3.2,
 *      subproblem 1) with a location (subproblem 2) and a least-squares value;
 *   3. peeling in parallel rounds: every single-ton found in a round is subtracted from
 *      the bins it aliases into in every stage, and the changed bins are examined again
 *      (Sec. 3.2, subproblem 3, genie-assisted peeling, Eq. 20).
 *
 * Conventions:
 *   - delays are advances: the sample is x[(m L + tau) mod N], 0 <= tau < N (the paper
 *     writes delays, x'_i = x_{i - tau}; the paper's tau is minus this one).
 *   - output values are the paper-normalised xhat_f (Eq. 2), sorted by frequency f.
 *   - complex data are interleaved (re, im): SFFT_C64 = 2 x float, SFFT_C128 = 2 x double.
 *
 * Memory: every pointer argument may point to device memory or to host memory (pinned or
 * pageable), unless a call says otherwise; host buffers are copied through a staging area
 * the plan owns, and the call then waits for the stream before it returns.  With device
 * buffers every call is asynchronous on `stream` (a cudaStream_t, NULL = legacy default
 * stream) and returns as soon as the work is enqueued.
 *
 * Errors: calls return SFFT_OK (0) or a negative SFFT_E* code.  Per-signal outcomes are
 * written by the GPU into the caller's info array (see sfft_execute).
 */
#ifndef SFFT_H
#define SFFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sfft_plan_s* sfft_plan_t;
typedef struct sfft_server_s* sfft_server_t;

/* return and status codes */
#define SFFT_OK 0
#define SFFT_PENDING 1       /* sfft_poll: request not finished */
#define SFFT_INCOMPLETE 2    /* per-signal status: peeling ended with unresolved bins */
#define SFFT_EINVAL (-1)     /* invalid argument (see each call) */
#define SFFT_ENOMEM (-2)     /* device or host allocation failed */
#define SFFT_ECUDA (-3)      /* a CUDA call failed; sfft_last_cuda_error() names it */
#define SFFT_ETIMEDOUT (-4)  /* a bounded device-side wait ran out */
#define SFFT_EADMIT (-5)     /* server: request can never fit the memory budget */
#define SFFT_ENOTFOUND (-6)  /* server: unknown ticket */
#define SFFT_EBUSY (-7)      /* server: queue full */
#define SFFT_ETOOBIG (-8)    /* sfft_bucketize_static: problem exceeds its static scratch */

/* element type of x and of the returned values */
#define SFFT_C64 0
#define SFFT_C128 1

/* arithmetic of the bulk path */
#define SFFT_PREC_FP64 0     /* plain path: everything in FP64 */
#define SFFT_PREC_FP32 1     /* FP32 gather/DFT/peeling, FP64 location and fit */

/* singleton location rule (Sec. 3.2, subproblem 2) */
#define SFFT_LOCATE_ARG 0    /* phase of Y(tau=1) conj(Y(tau=0)), snapped to the bin's
                                candidates; needs delays 0 and 1 in every stage (FFAST) */
#define SFFT_LOCATE_ML 1     /* best delay-phasor correlation over the L_d candidates
                                {j, j + B_d, ...} of the bin (random delays, R-FFAST) */
#define SFFT_LOCATE_KAY 2    /* R-FFAST with structured delays (Sec. 3.2 subproblem 2,
                                Eq. 21-22): slot c m + t of every stage holds r_c + t 2^c
                                (mod N), C = n_delays / m iterations with 2^C >= L_d; each
                                iteration's Kay-weighted phase difference gives one bit of
                                f / N, and the bin's candidate nearest the resulting
                                interval is the location (m = opts->kay_m) */

/* decoder (Sec. 3) */
#define SFFT_DECODER_PEEL 0     /* FFAST / R-FFAST peeling across stages (Sec. 3.2) */
#define SFFT_DECODER_ONESHOT 1  /* sFFT-DT one-shot decoder on a single stage (Sec. 3.1):
                                   Hankel singular-value count, Prony enumeration of the
                                   positions, subspace-pursuit values */
#define SFFT_DECODER_DSFFT 2    /* DSFFT binary tree search (Sec. 3.3, Sec. 4.3): N a power of
                                   two; layer d holds the 2^d aliasing bins of subsampling
                                   factor N / 2^d with delays {0, 1}; the search starts at the
                                   layer of f[0] and goes down one layer at a time until every
                                   efficient (non-zero) node holds one frequency, which the
                                   phase encoding of Sec. 3.2 then recovers.  Host-driven: one
                                   device round trip per layer searched */

typedef struct {
    int32_t dtype;       /* SFFT_C64 or SFFT_C128 (default C64) */
    int32_t precision;   /* SFFT_PREC_FP32 or SFFT_PREC_FP64 (default FP32) */
    int32_t locate;      /* SFFT_LOCATE_ARG or SFFT_LOCATE_ML (default ML) */
    int32_t max_rounds;  /* peeling rounds at most (default 64) */
    int32_t max_batch;   /* signals per execute call at most; sizes the workspace (default 1) */
    int32_t max_tile;    /* B-tile: largest DFT tile in elements held by one CTA; 0 = whatever
                            shared memory allows (stages larger than it run as two passes, with
                            tiles of about max_tile elements, or 4096 (FP32) / 2048 (FP64) when
                            max_tile is 0) */
    double noise_var;    /* sigma^2 of the noise per time sample, 0 = exactly sparse */
    double a_min;        /* smallest significant |xhat| (default 1) */
    double eta;          /* relative numerical floor of the thresholds; 0 = default
                            (3e-3 for FP32, 1e-6 for FP64) */
    double c0, c1;       /* zero-ton / single-ton threshold multipliers (default 4, 2):
                            T0_d = R (c0 B_d sigma^2 + (eta B_d a_min)^2),
                            T1_d = R (c1 B_d sigma^2 + (eta B_d a_min)^2) */
    int32_t wait_limit_log2;  /* a device-side wait gives up after 2^this polls (about
                                 0.1-0.3 us each) and reports SFFT_ETIMEDOUT; 0 = 22 */
    int32_t fault_inject;     /* testing only: 0 none; 1 = one CTA of every multi-CTA decode
                                 group leaves before its first barrier, so the others' wait
                                 runs out (status SFFT_ETIMEDOUT); 2 = plan creation fails
                                 with SFFT_ENOMEM before allocating */
    int32_t decode_ctas;      /* CTAs per signal in the peeling rounds; 0 = automatic */
    int32_t decoder;          /* SFFT_DECODER_PEEL (default) or SFFT_DECODER_ONESHOT */
    int32_t oneshot_am;       /* one-shot decoder: a_m, the most frequencies one bucket may
                                 hold (1..3, default 3) */
    int32_t kay_m;            /* SFFT_LOCATE_KAY: delays per iteration m >= 2 (default 2) */
    int32_t noise_auto;       /* peeling decoder: 1 = estimate sigma^2 per signal from its bins
                                 (lower median over all bins of sum_r |Y_r|^2 / B_d, divided
                                 by the median of Gamma(R, 1)) and set T0, T1 from it;
                                 noise_var is then unused.  0 (default) = use noise_var */
    int32_t host_gather;      /* sfft_execute with a page-locked host signal (cudaHostAlloc,
                                 or cudaHostRegister with cudaHostRegisterMapped): 1 = the
                                 bucketization reads the samples it needs in place over the
                                 host link, so only the cache lines holding them cross it
                                 (about R sum_d 1/L_d x 64 / sizeof(sample) of the signal,
                                 capped at all of it) and signals larger than device memory
                                 can be decoded; pageable host signals are still copied.
                                 0 (default) = copy every host signal to device memory first */
    int32_t oneshot_method;   /* one-shot decoder, Step 2 (Sec. 3.1): 1 = roots of P(z)
                                 (polynomial method), 2 = enumeration of the L candidates
                                 (default; 0 means 2), 3 = matrix pencil on the SVD of Eq. 15's
                                 Toeplitz Y (as sFFT-DT3.0 in Sec. 4.1).  Methods 1 and 3 snap
                                 each root z to the candidate nearest arg(z) */
    int32_t dft_fma_only;     /* 1 = every DFT axis on the FMA pipes.  0 (default) = in FP32
                                 stages done in one pass, the odd axes with 17 <= P <= 127 (direct
                                 P-point DFTs: a cosine and a sine matrix applied to every
                                 sub-DFT) run on the tensor cores as 3-term split FP16 products
                                 with FP32 accumulation, FP32-level accuracy */
    int32_t peel_atomic;      /* peeling subtraction (Sec. 3.2 subproblem 3, Eq. 20).  0 (default):
                                 every accepted frequency's subtraction is queued on the bins it
                                 aliases into and applied in increasing order of frequency, each
                                 delay's sum compensated (TwoSum), so the results are the same
                                 bits on every run.  1 = subtract with unordered float atomics
                                 on the bins as frequencies are accepted (results may differ in
                                 the last bits from run to run) */
    int32_t overlap_gather;   /* 1: where a stage's whole FP32 tile fills more than half of a
                                 CTA's shared memory (one CTA per SM), the bucketization runs as
                                 one persistent CTA per SM that copies the next tile's samples
                                 into the other end of shared memory while it transforms the
                                 current one.  0 (default) = one CTA per tile: the scattered
                                 8-byte copies need L1 lines in flight, which the second tile
                                 region takes away (measured 2.4x slower on N = 127*128*129) */
    int32_t classify_lanes;   /* lanes of a warp that search one bin's L candidates on the FMA
                                 pipes in the first peeling round (ML locate): 1, 2, 4, 8, 16
                                 or 32.  0 (default) = the tensor-core search (ml_tc_tf32) in
                                 FP32 plans with n_delays <= 16 when a classify tile's bins lie
                                 in at most two stages; otherwise lanes chosen per tile from
                                 its non-zero bins, L and R */
    int32_t arg_mode;         /* SFFT_LOCATE_ARG precision experiment (Sec. 3.2 subproblem 2):
                                 0 (default) = the angle of Y(1) conj(Y(0)) in FP64, snapped to
                                 the bin's candidate set {j + q B_d}; bit 0 = the angle and its
                                 scaling by N / 2 pi in FP32; bit 1 = no snap, f = the integer
                                 nearest the estimate.  Modes 1-3 exist to measure what the FP64
                                 angle and the snap buy; they are not meant for use */
    int32_t ml_tc_tf32;       /* the first peeling round's ML search on the tensor cores (FP32
                                 plans, classify_lanes = 0, n_delays <= 16): the scores of a
                                 bin's L candidates as the product of the stage's candidate
                                 matrix with the bin's Z_r.  0 (default) = m16n8k16 FP16 MMAs, both
                                 operands split into high and low FP16 parts (three partial
                                 products, FP32 accumulation) after a power-of-two scale per
                                 bin; 1 = m16n8k8 TF32 MMAs with split operands, twice the
                                 MMAs.  Both give FP32-level scores */
} sfft_opts;

/* Fill *opts with the defaults above. */
void sfft_opts_default(sfft_opts* opts);

/* Create a plan for signals of length N (Sec. 3.2: N = product of co-prime factors).
 *   f[n_stages]          subsampling factor L_d of each stage; each divides N, the f are
 *                        pairwise co-prime, B_d = N / L_d (1 <= n_stages <= 4)
 *   delays[n_stages * n_delays]  tau_{d,r} at [d * n_delays + r], distinct within a stage,
 *                        0 <= tau < N (1 <= n_delays <= 16)
 *   K                    output size: the K largest recovered coefficients (Sec. 2.1)
 * With opts->decoder = SFFT_DECODER_ONESHOT (Sec. 3.1, Sec. 4.1): one stage, K <= B, and
 * the delays are the consecutive set -a_m .. 2 a_m - 1 (mod N) in slots 0 .. 3 a_m - 1
 * followed by P >= 2 a_m distinct random delays (a_m = opts->oneshot_am).
 * With opts->decoder = SFFT_DECODER_DSFFT: N a power of two, one stage whose f[0] (a power
 * of two) is the start layer's subsampling factor N / 2^p, delays {0, 1}; locate is ARG.
 * The plan holds the layers from p down to the deepest whose 2^d bins one CTA can
 * transform (2^14 in FP32, 2^13 in FP64); sfft_plan_num_bins returns that layer's 2^d.
 * The info row of a DSFFT execution holds the layer d the search stopped at in place of
 * the round count.
 * Host arrays; the plan copies them.  N < 2^30.  The plan owns device tables (twiddles,
 * index maps) and the workspace for opts->max_batch signals until sfft_plan_destroy.
 * Errors: SFFT_EINVAL (bad sizes, factors, delays, ARG without delays 0 and 1, KAY delays
 * without the structure of SFFT_LOCATE_KAY, a one-shot plan breaking the rules above),
 * SFFT_ENOMEM, SFFT_ECUDA.                                                                */
int sfft_plan_create(sfft_plan_t* out, int64_t N, int32_t K, int32_t n_stages, const int64_t* f,
                     int32_t n_delays, const int64_t* delays, const sfft_opts* opts);
void sfft_plan_destroy(sfft_plan_t plan);

/* Bins per signal: sum_d B_d (so the bucketization output has n_delays times as many). */
int64_t sfft_plan_num_bins(sfft_plan_t plan);

/* noise_auto plans: the sigma^2 estimated for workspace slot `slot` (0 <= slot < max_batch;
 * signal i of the last sfft_execute_batch group or execute call used slot i) by its last
 * execution, in *out (host).  The thresholds of Sec. 3.2 subproblem 1 assume sigma^2 known;
 * the estimate has no counterpart in the paper.  Waits for the device.
 * Errors: SFFT_EINVAL (plan without noise_auto, slot out of range, null out), SFFT_ECUDA. */
int sfft_plan_noise_var(sfft_plan_t plan, int32_t slot, double* out);

/* Recover one signal.
 *   x          N complex samples of the plan's dtype
 *   out_idx    int64[K]: recovered frequencies, ascending
 *   out_val    K complex values (plan dtype): xhat at out_idx
 *   out_info   int32[4]: {count, status (SFFT_OK or SFFT_INCOMPLETE, or SFFT_ETIMEDOUT),
 *              rounds, identifications (bins classified, over all rounds)}
 * Entries of out_idx/out_val past count are left untouched.  Calls that share a plan use
 * its single workspace: they must be ordered (one stream, or synchronised).              */
int sfft_execute(sfft_plan_t plan, const void* x, int64_t* out_idx, void* out_val,
                 int32_t* out_info, void* stream);

/* Recover n signals in one set of launches.  plans[i] (may repeat), xs[i], idx[i], val[i]
 * as in sfft_execute for signal i; infos: int32[4 * n], signal i at infos + 4 i.  The
 * host arrays of pointers are read during the call.  Signals that share a plan are
 * processed together wherever they sit in the batch, at most that plan's max_batch per
 * launch group; with device buffers, the groups of different plans run on streams of their
 * plans forked from `stream` and joined back into it, so they overlap on the device.  The buffers are
 * either all device memory (asynchronous) or all host memory (staged per launch group
 * through device memory the plan owns; the call returns when the outputs are written).
 * Mixing the two is SFFT_EINVAL.                                                          */
int sfft_execute_batch(int32_t n, const sfft_plan_t* plans, const void* const* xs,
                       int64_t* const* idx, void* const* val, int32_t* infos, void* stream);

/* Bucketization only (Eq. 6 / Eq. 19): writes the bins of one signal in natural order,
 * bins[off_d + r * B_d + j] with off_d = n_delays * sum_{d'<d} B_d', as complex of the
 * plan's arithmetic (FP32 -> C64, FP64 -> C128).  Device pointers only.  SFFT_EINVAL for
 * a DSFFT plan (its layers have different sizes).                                         */
int sfft_bucketize(sfft_plan_t plan, const void* x, void* bins, void* stream);

/* Bucketization without any device allocation (no counterpart in the paper: this is a
 * deployment variant of sfft_bucketize).  For callers that cannot call cudaMalloc -- an
 * application whose own allocator already holds the GPU's memory, or a latency-critical
 * loop where cudaMalloc/cudaFree would synchronise the device -- and so cannot create a
 * plan.  The problem is described directly (arguments as sfft_plan_create; precision
 * SFFT_PREC_*, dtype SFFT_C* of x); x (N samples) and bins (output, the layout and type of
 * sfft_bucketize) are device pointers the caller owns.  Tables, twiddles and the scratch
 * of two-pass stages live in one static 16 MiB device array inside the library, held by
 * every GPU that loads it until the process exits; a problem needing more than fits
 * (roughly sum_d B_d * (8 + 2 R * sizeof(complex)) bytes) returns SFFT_ETOOBIG before any
 * device work.  Every call resolves the array's device address on the current device; the
 * first call on a device also loads the library's device code there, so it should come
 * before any stream capture.  All calls share the array and leave their data
 * in it: calls that overlap on the GPU race, so the caller must order them.              */
int sfft_bucketize_static(int64_t N, int32_t n_stages, const int64_t* f, int32_t n_delays,
                          const int64_t* delays, int32_t precision, int32_t dtype,
                          const void* x, void* bins, void* stream);

/* Peeling decoder only, on caller-supplied bins in the layout of sfft_bucketize (read,
 * not modified).  Outputs as sfft_execute.  Device pointers only.  SFFT_EINVAL for a DSFFT
 * plan.                                                                                   */
int sfft_decode_bins(sfft_plan_t plan, const void* bins, int64_t* out_idx, void* out_val,
                     int32_t* out_info, void* stream);

/* Autotuning (no counterpart in the paper).  Times sfft_execute_batch on the caller's n
 * sample signals (device pointers, dtype of *base) for schedules chosen by coordinate
 * descent from the defaults, one axis at a time: the B-tile (max_tile: whole-stage DFT
 * tiles, or two passes of 16384, 8192 or 4096 elements), the gather schedule
 * (overlap_gather), the lanes per bin of the first round's ML search (classify_lanes, ML
 * plans) and the CTAs per signal of the peeling rounds (decode_ctas); a value is kept when
 * it is more than 1 % faster.  Writes the fastest into *best (a copy of *base with those
 * fields set, max_batch = n) and its rate in signals/s into *best_rate (may be NULL).
 * Creates and destroys its own plans; the stream is synchronised.  With a cache file set
 * (sfft_autotune_cache), a schedule found before for the same key -- N, f, R, K, n, dtype,
 * precision, locate, noise_auto, decoder, dft_fma_only and the GPU's name and SM count --
 * is returned without timing, and a new one is added to the file.                        */
int sfft_autotune(int64_t N, int32_t K, int32_t n_stages, const int64_t* f, int32_t n_delays,
                  const int64_t* delays, const sfft_opts* base, int32_t n, const void* const* xs,
                  void* stream, sfft_opts* best, double* best_rate);
/* The autotuner's cache file (a JSON object: key -> schedule fields and rate), or NULL to
 * use none (the default).  The file is rewritten whole (through a temporary file) when an
 * entry is added.  Host only.                                                              */
int sfft_autotune_cache(const char* path);

/* Phase timing.  While enabled, every execute call brackets its bucketization, decode and
 * compaction launches with CUDA events on the launch stream.  sfft_plan_profile waits for
 * the recorded events and returns the accumulated milliseconds, kernel launches and calls
 * per phase (ms[3], launches[3], calls[3]; any may be NULL), then clears them if reset.   */
int sfft_plan_set_profiling(sfft_plan_t plan, int enable);
int sfft_plan_profile(sfft_plan_t plan, double* ms, int64_t* launches, int64_t* calls, int reset);

/* Serving: continuous batching of requests of any plans on one GPU.  A host thread
 * admits queued requests onto idle workspaces of their plan while fewer than max_slots
 * groups are in flight, launches each admitted group (up to 32 requests of one plan) on
 * its workspace's stream (so groups overlap on the device), and a host function at the
 * end of each group's stream work retires it.  Workspaces fit in hbm_budget bytes.       */
int sfft_server_create(sfft_server_t* out, size_t hbm_budget, int32_t max_slots);
/* Create up to n_workspaces (at most max_slots) workspaces for requests of `plan` now,
 * within the memory budget: clones of the plan sized for a launch group of 32 requests,
 * each with its own stream.  The scheduler only reuses workspaces, so once they exist no
 * request waits for an allocation; a plan's first sfft_submit reserves max_slots
 * workspaces itself if none exist.  Idle workspaces of other plans with no queued
 * request are freed when the budget is full.  Synchronises the device (plan creation).
 * Errors: SFFT_EINVAL, SFFT_EADMIT (not even one workspace fits), SFFT_ENOMEM, SFFT_ECUDA. */
int sfft_server_reserve(sfft_server_t srv, sfft_plan_t plan, int32_t n_workspaces);
/* Queue one request (device pointers, as sfft_execute).  The buffers must stay valid until
 * sfft_poll reports a final status.  *ticket identifies it.  DSFFT plans (host-driven
 * layer search) are refused with SFFT_EINVAL.                                             */
int sfft_submit(sfft_server_t srv, sfft_plan_t plan, const void* x, int64_t* out_idx,
                void* out_val, int32_t* out_info, uint64_t* ticket);
/* *status = SFFT_PENDING while queued or running, else SFFT_OK once the outputs are
 * written (per-signal status in out_info).  Also reports the request's latency in
 * microseconds from submit to completion (latency_us may be NULL).                       */
int sfft_poll(sfft_server_t srv, uint64_t ticket, int32_t* status, double* latency_us);
/* Wait until every queued request has finished. */
int sfft_server_drain(sfft_server_t srv);
void sfft_server_destroy(sfft_server_t srv);

/* Text of a return code; name of the last CUDA error seen by the library. */
const char* sfft_error_string(int code);
const char* sfft_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SFFT_H */
