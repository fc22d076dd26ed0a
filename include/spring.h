/* spring.h -- C ABI of libspring, a GB300 (sm_103a) implementation of the data-parallel
 * hot path of Memetic Phase Retrieval (MPR), after Colombo et al., "SPRING: an effective
 * and reliable framework for image reconstruction in single-particle Coherent
 * Diffraction Imaging" (arXiv 2409.07413).  Citations name the paper's sections,
 * equations and algorithms.
 *
 * General conventions (every entry point):
 *  - Status: every call returns a spring_status; SPRING_OK = 0.  The library never
 *    aborts.  On failure a message is kept for the calling thread (spring_last_error).
 *  - Complex arrays are complex64: interleaved (re, im) float32 pairs, row-major N x N
 *    per image, images contiguous (batch x N x N).
 *  - Real-space arrays (densities, supports) are used in the caller's orientation.
 *    Fourier-space arrays given to the problem API (intensities, mask) are
 *    detector-centred (zero frequency at (N/2, N/2)); the operator API below takes them
 *    in DFT order (zero frequency at index 0).
 *  - The 2D Fourier transform is unitary (factor 1/N on an N x N transform, both
 *    directions), so that sum |rho|^2 = sum |FT rho|^2 (App. "Initialization of the
 *    starting densities").
 *  - Modulus encoding (operator API): M is N x N float32 in DFT order; an entry >= 0 is
 *    the measured modulus sqrt(I) (mask Xi = 1), an entry < 0 marks a pixel whose
 *    intensity is not measured (Xi = 0: beamstop/hole, detector gap, saturation).  A
 *    missing pixel whose modulus is bounded above (Eq. pm_bounds) carries M = -2 - U
 *    (M <= -2, bound U >= 0); entries in (-2, 0) (the library writes -1) are free.
 *  - Supports and masks are uint8, 0 or 1.
 *  - Sizes: square patterns, N in {64, 96, 128, 192, 256, 384, 512, 768, 1024} (every even
 *    N in [64, 1024] of the form 2^a 3^b with b <= 1).  Other sizes return
 *    SPRING_E_INVALID.
 *  - Streams: the operator API takes a cudaStream_t as void* (NULL = legacy default
 *    stream) and is asynchronous on it; device pointers must be valid on the current
 *    device.  Scratch memory is taken from the stream-ordered allocator of the current
 *    device and returned before the call's work completes (stream order).
 *  - Ownership: the library never takes ownership of caller buffers.  Handles
 *    (contexts, problems) are released by their destroy/shutdown call.
 */
#ifndef SPRING_H
#define SPRING_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SPRING_ABI_VERSION 2
/* columns of spring_result.gen_stats */
#define SPRING_GEN_STATS_COLS 9

typedef enum {
  SPRING_OK = 0,
  SPRING_E_INVALID = 1,   /* bad argument: size, pointer, parameter range */
  SPRING_E_NOMEM = 2,     /* device memory or HBM budget exhausted */
  SPRING_E_CUDA = 3,      /* a CUDA runtime error (message via spring_last_error) */
  SPRING_E_BUSY = 4,      /* not ready yet / still in use */
  SPRING_E_TIMEOUT = 5,   /* a bounded wait ran out */
  SPRING_E_NOT_FOUND = 6, /* unknown ticket */
  SPRING_E_NUMERIC = 7,   /* NaN/Inf met in a reduction */
  SPRING_E_CANCELLED = 8  /* the ticket was cancelled before it completed */
} spring_status;

typedef struct spring_ctx spring_ctx;         /* device, streams, HBM budget, scheduler */
typedef struct spring_problem spring_problem; /* one diffraction pattern resident on device */

/* Parameters of one MPR run (Table "params" of App. "Summary of the parameters and
 * further considerations").  spring_params_default() fills the defaults shown. */
typedef struct {
  int pop;                 /* P >= 4, population size (default 8) */
  int iters_per_gen;       /* iterations per individual per generation (100) */
  int generations;         /* G >= 1 (5) */
  int algorithm;           /* IA of the main sequence: 0 ER, 1 HIO, 2 RAAR (2) */
  float beta;              /* HIO/RAAR beta in (0, 1] (0.9) */
  float sw_sigma;          /* shrink-wrap Gaussian sigma, px (1.5) */
  float sw_threshold;      /* shrink-wrap threshold tau in (0, 1] (0.2) */
  float sw_sigma_end;      /* sigma at the last generation, linear in between (= sw_sigma) */
  float sw_threshold_end;  /* tau at the last generation (= sw_threshold) */
  int sw_period;           /* K: iterations between support updates (20) */
  int er_tail;             /* ER iterations of the evaluation sequence (10) */
  float chi;               /* phase range [-chi pi, chi pi]; 0.5 = positivity, >= 1 off (0.5) */
  float cw;                /* crossover differential weight C_w in [0, 2] (0.4) */
  float cp;                /* crossover tile probability C_p in [0, 1] (0.6) */
  int tile_min, tile_max;  /* crossover tile sides; tile_max 0 = N/8 (4, 0) */
  int init_n_spheres;      /* spheres per initial density N_init (5) */
  float init_gamma;        /* gamma applied to |rho| at initialisation (1) */
  float init_phi_max;      /* sphere phases uniform in [-phi_max, phi_max] (0) */
  int precision;           /* 0: complex64 state; 1: FP16 storage of the state and FFT
                              intermediate inside iteration blocks, FP32 math (0) */
  int use_graph;           /* 1: capture the run in a CUDA graph before launching (0) */
  int schedule;            /* 0: the blocks above (iters_per_gen, sw_period, er_tail);
                              1: the paper's Sequence (App. "The algorithms sequence"): R
                              repetitions of seq_ia IA + seq_er ER iterations, the IA count
                              linear to 0 and the ER count to seq_ia + seq_er over the
                              generations (halves rounded up), then seq_eval ER (0) */
  int mode;                /* 0: MPR (Alg. mpr); 1: P independent reconstructions
                              (Alg. randomsearch: Improve only, no crossover or selection;
                              the result is the best and the aligned average) (0) */
  int seq_ia;              /* schedule 1: starting IA iterations of a Sequence (40) */
  int seq_er;              /* schedule 1: starting ER iterations of a Sequence (40) */
  int seq_eval;            /* schedule 1: ER iterations of EvalSequence (40) */
  int repetitions;         /* schedule 1: R >= 2 (3) */
  float ca;                /* crossover averaging C_a in [0, 1] (App. "Crossover averaging",
                              Eq. crossavg) (0) */
  int monitor_avg;         /* 1: the average reconstruction and its error E(avg) every
                              generation (gen_stats column 3), not only at the end (0) */
  uint64_t seed;           /* key of the counter-based generator (0) */
} spring_params;

/* Result of one run.  Pointer members are caller-owned host buffers (may be NULL). */
typedef struct {
  float* rho_avg;          /* N*N complex64: average of the aligned population (Alg. mpr) */
  float* rho_best;         /* N*N complex64: lowest-error individual */
  uint8_t* support_avg;    /* N*N: union of the aligned supports (Eq. avgrec) */
  double* gen_stats;       /* G x SPRING_GEN_STATS_COLS (9) per generation: best E, mean E,
                              worst E, E(avg) (last generation only, else NaN), O_d (Eq.
                              oversampling), replacement factor, mean complexity Gamma (Eq.
                              complexity), mean |sum rho|, and the population standard
                              deviation of |sum rho| relative to that mean; may be NULL */
  double final_error_avg;  /* GetError (Eq. error_calc) of rho_avg on support_avg */
  double final_error_best; /* error of rho_best */
  double t_submit_s, t_admit_s, t_done_s; /* serving timestamps (monotonic seconds) */
} spring_result;

/* ---------------------------------------------------------------- context, errors */
int spring_abi_version(void);
const char* spring_status_string(spring_status s);
/* Message of the last failed call made by this thread ("" if none).  Owned by the
 * library; valid until the thread's next call. */
const char* spring_last_error(void);
void spring_params_default(spring_params* p);

/* Open a context on CUDA device `device`.  hbm_budget_bytes bounds what the context's
 * runs and admitted requests may hold on the device (0 = 90% of free memory at open).
 * Starts the serving scheduler thread.  Errors: INVALID (device), CUDA. */
spring_status spring_init(int device, size_t hbm_budget_bytes, spring_ctx** out);
/* Close a context: BUSY if tickets are still queued or running (cancel or poll them
 * first); otherwise stops the scheduler and frees the context. */
spring_status spring_shutdown(spring_ctx* ctx);

/* ---------------------------------------------------------------- problems
 * The problem statement of the paper (Sec. "The phase problem and conventional
 * approaches"; Eq. error_calc): measured intensities I = M^2, the mask Xi of measured
 * pixels and an initial support.  I and mask are detector-centred host arrays of
 * ny x nx (ny == nx == N); I >= 0 (negative values are treated as 0); support0 is in
 * real space.  The library copies them to the device (M = sqrt(I) in DFT order, with
 * the mask folded into M's sign); the caller keeps its arrays.
 * Errors: INVALID (sizes, NULL), NOMEM, CUDA. */
spring_status spring_problem_create(spring_ctx* ctx, int ny, int nx, const float* intensities,
                                    const uint8_t* mask, const uint8_t* support0,
                                    spring_problem** out);
/* Same, from device buffers (e.g. torch tensors) on `stream` (cudaStream_t as void*).
 * The call is asynchronous: the inputs must stay valid until `stream` reaches it. */
spring_status spring_problem_create_device(spring_ctx* ctx, int ny, int nx,
                                           const float* d_intensities, const uint8_t* d_mask,
                                           const uint8_t* d_support0, void* stream,
                                           spring_problem** out);
/* Upper bounds for missing intensities (App. "Constraining intensities at large
 * scattering angles", Eqs. avgint, stdint, upperbound, enforced by Eq. pm_bounds).
 * Pixels are grouped in rings by their distance from the detector centre (pixel
 * (N/2, N/2) of the centred arrays) rounded to the nearest integer.  Over the measured
 * pixels of a ring, mu = mean I and sigma^2 = mean (I - mu)^2; a missing, unsaturated
 * pixel of a ring with at most max_missing of its pixels missing and at most
 * max_saturated of them saturated gets the modulus bound U = sqrt(mu + eta sigma). */
typedef struct {
  float eta;            /* <= 0: no bounds (paper: 1.5) */
  float max_missing;    /* fraction of a ring that may be missing (paper: 0.2) */
  float max_saturated;  /* fraction of a ring that may be saturated (paper: 0.05) */
} spring_bounds;
void spring_bounds_default(spring_bounds* b);
/* spring_problem_create with upper bounds: `saturated` (host, detector-centred, 1 = the
 * pixel is saturated; such pixels should also be 0 in `mask`) may be NULL; bounds NULL
 * or eta <= 0 is spring_problem_create.  Every run of the problem uses the bounds.
 * Errors: as spring_problem_create. */
spring_status spring_problem_create_bounded(spring_ctx* ctx, int ny, int nx, const float* intensities,
                                            const uint8_t* mask, const uint8_t* support0,
                                            const uint8_t* saturated, const spring_bounds* bounds,
                                            spring_problem** out);
/* BUSY if an unfinished ticket still references the problem. */
spring_status spring_problem_destroy(spring_problem* prob);
/* Device bytes one run of an N x N problem with parameters p holds (admission). */
size_t spring_footprint_bytes(int n, const spring_params* p);

/* ---------------------------------------------------------------- runs
 * One blocking MPR reconstruction (Alg. mpr): Initialize; G x {Crossover (Alg.
 * crossover), Improve of both populations (Alg. improve), Select (Alg. select)};
 * Average.  Results go to the caller's buffers in *out.
 * Errors: INVALID (parameters), NOMEM (budget), CUDA, NUMERIC. */
spring_status spring_mpr_run(spring_problem* prob, const spring_params* p, spring_result* out);

/* K independent MPR reconstructions run together.  Problems of the same side share every
 * iteration, shrink-wrap and error launch, which covers all their populations (problem q's
 * moduli serve its own 2P images); the GA steps (Alg. crossover, Alg. select, the average)
 * run problem by problem.  Problems of different sides form one such group per side, and
 * the groups advance concurrently on their own streams — with p->use_graph, as parallel
 * branches of one CUDA graph, so that a single graph launch runs the whole batch.
 * probs[0..K) share one context; seeds[q] replaces p->seed for problem q; out[q] receives
 * problem q's result, equal bit for bit to spring_mpr_run(probs[q]) with p->seed = seeds[q].
 * p->precision and p->mode must be 0 when K > 1.  Blocking; the footprint is the sum of the
 * groups' (about K times a single run's).
 * Errors: INVALID (arguments, mixed contexts), then as spring_mpr_run; NUMERIC if any
 * problem's error is non-finite. */
spring_status spring_mpr_run_batch(spring_problem* const* probs, int K, const spring_params* p,
                                   const uint64_t* seeds, spring_result* out);

/* Checkpoint / resume.  The population state of a run after `generation` completed
 * generations: P images (caller-owned host buffers, P x N x N complex64, P x N x N uint8,
 * P doubles; errors are +inf before the first generation's evaluation). */
typedef struct {
  int generation;
  float* pop_x;
  uint8_t* pop_S;
  double* pop_err;
} spring_population;
/* Initialize and run generations 1..g_stop (1 <= g_stop <= p->generations) of the run that
 * spring_mpr_run would make with the same parameters, then copy its population to *save
 * (save->generation = g_stop).  Blocking.  Errors: as spring_mpr_run. */
spring_status spring_mpr_run_until(spring_problem* prob, const spring_params* p, int g_stop,
                                   spring_population* save);
/* Continue a run from a saved population: generations from->generation + 1 .. G, then the
 * average, into *out (gen_stats rows of the skipped generations are NaN).  With the same
 * problem and parameters the result equals spring_mpr_run's bit for bit (every random
 * draw is keyed by the generation).  INVALID if from->generation is not in [0, G). */
spring_status spring_mpr_resume(spring_problem* prob, const spring_params* p, const spring_population* from,
                                spring_result* out);

/* What one generation decided (spring_mpr_step).  Pointer members are caller-owned host
 * buffers and may be NULL; the rest is filled in.  For mode 1 (independent
 * reconstructions) only err_parents and gen_stats are meaningful. */
typedef struct {
  double* err_parents;  /* P: errors (Eq. error_calc) of the parents after their Improve, before
                           Select (Alg. mpr) */
  double* err_new;      /* P: errors of the new individuals after their Improve */
  uint8_t* replaced;    /* P: 1 where Select (Alg. select) took the new individual */
  int32_t* parents;     /* 3 x P: parents (a, b, c) of new individual p at 3p .. 3p + 2 (Alg.
                           crossover, RandomChoice) */
  int64_t areas[3];     /* alpha_best, alpha_all, alpha_eval (Alg. improve) */
  int32_t best;         /* the parent whose support area is alpha_best */
  double gen_stats[SPRING_GEN_STATS_COLS]; /* this generation's row of spring_result.gen_stats */
} spring_generation_trace;
/* One generation g = from->generation + 1 (g <= p->generations) of the run spring_mpr_run
 * would make, from the given parent population: Crossover, the areas, Improve of both
 * populations, Select (Alg. mpr), with the schedules of generation g of G.  The population
 * after it goes to *to (to->generation = g; may alias *from's buffers).  trace may be
 * NULL.  Chaining steps from g = 0 (a population of initial densities with errors +inf)
 * reproduces spring_mpr_run's population bit for bit.  Blocking.
 * Errors: INVALID (arguments, generation), then as spring_mpr_run. */
spring_status spring_mpr_step(spring_problem* prob, const spring_params* p, const spring_population* from,
                              spring_population* to, spring_generation_trace* trace);

/* Serving: queue a run; requests are admitted in arrival order while their footprint fits
 * the HBM budget.  An admitted request takes along the queued requests of the same side and
 * the same parameters (seeds aside; FP32 storage, mode 0) into a cohort: one set of launches
 * over all their populations, as spring_mpr_run_batch, up to SPRING_MAX_COHORT requests
 * (environment, default 32) and 2^26 pixels per launch.  Up to SPRING_MAX_ACTIVE cohorts
 * (environment, default 4) advance concurrently on the device, one generation per scheduler
 * turn, on streams whose priority is higher for smaller requests (continuous batching).  A
 * request's result is the same bit for bit alone or in a cohort.  *ticket identifies the
 * request.  The problem must stay alive until the ticket is polled or cancelled. */
spring_status spring_submit(spring_ctx* ctx, spring_problem* prob, const spring_params* p,
                            uint64_t* ticket);
/* Wait up to timeout_us (0 = do not wait, < 0 = wait forever) for a ticket.  SPRING_OK
 * fills *out (buffers as for spring_mpr_run) and retires the ticket; BUSY = not done yet;
 * NOT_FOUND = unknown or already retired; CANCELLED; or the run's own error. */
spring_status spring_poll(spring_ctx* ctx, uint64_t ticket, int timeout_us, spring_result* out);
/* Cancel a queued or running ticket.  A queued ticket is dropped at once; a running one stops
 * at its cohort's next generation boundary when every member of the cohort is cancelled, and
 * otherwise when the cohort completes (its result is discarded). */
spring_status spring_cancel(spring_ctx* ctx, uint64_t ticket);
/* Serving statistics of a context since spring_init: cohorts formed and requests admitted
 * (their ratio is the mean cohort size).  Either pointer may be NULL. */
spring_status spring_serving_stats(spring_ctx* ctx, uint64_t* cohorts, uint64_t* admitted);

/* ---------------------------------------------------------------- operators
 * The steps of the hot path on caller device buffers.  The run above is composed of
 * exactly these kernels.  All are asynchronous on `stream`. */

/* a1/a3: unitary 2D DFT of `batch` complex64 images in place (inverse != 0: F^-1). */
spring_status spring_fft2(void* data, int batch, int n, int inverse, void* stream);

/* The modulus array of the operator API from device arrays: I and mask (and saturated,
 * may be NULL) detector-centred N x N; M out in DFT order (sqrt(I) where mask = 1, the
 * bound encoding -2 - U where spring_problem_create_bounded would bound the pixel, -1
 * elsewhere).  bounds NULL or eta <= 0: no bounds.  Scratch: a few KB. */
spring_status spring_modulus_encode(const float* I, const uint8_t* mask, const uint8_t* saturated, int n,
                                    const spring_bounds* bounds, float* M, void* stream);

/* a1-a3: out = P_M x = F^-1[ M F x / |F x| where Xi = 1, F x elsewhere ]
 * (Eq. pm with the masked form Eq. pm_full; a zero modulus takes phase 0); with bound
 * entries in M (see the modulus encoding) the free values follow Eq. pm_bounds:
 * |F x| > U is brought down to U with its phase kept.
 * x and out: batch images (may alias).  M: one pattern shared by the batch. */
spring_status spring_project_modulus(const void* x, void* out, const float* M, int batch,
                                     int n, void* stream);

/* a1-a4: n_iter iterations x <- U(x, P_M x) in place, U = ER (algorithm 0), HIO (1) or
 * RAAR (2) (Sec. "The phase problem and conventional approaches"; ER = P_M P_S of
 * App. "The phase problem as an optimization problem").  Per pixel, with m = P_M x and
 * C = {S = 1 and |arg m| <= chi pi} (App. "Real-space constraints"):
 *   ER: x' = m on C, 0 elsewhere;  HIO: x' = m on C, x - beta m elsewhere;
 *   RAAR: x' = m on C, beta x + (1 - 2 beta) m elsewhere.
 * S: batch supports.  x must be 16-byte aligned (the row passes stream it into shared memory
 * in 16-byte copies; every device allocation is); INVALID otherwise.  Scratch: one
 * batch x N x N complex64 work buffer, the supports packed to bits and, where the side runs
 * the split passes (spring_set_iteration_path), M in their chunked layout. */
spring_status spring_iterate(void* x, const uint8_t* S, const float* M, int batch, int n,
                             int algorithm, float beta, float chi, int n_iter, void* stream);

/* a1-a4 on chip (N in {64, 128, 192, 256}): the same n_iter iterations as spring_iterate
 * with the image of each individual held in the shared memory of a thread-block cluster
 * of N/32 CTAs for the whole call (distributed shared memory between the row and the
 * column transforms); HBM is read once and written once per call.  Results equal
 * spring_iterate's with the default transform plan of side N (row variants 0-4, column
 * variants 0 and 2-7).  INVALID for other sides or where the device cannot hold such a
 * cluster.  No scratch. */
spring_status spring_iterate_fused(void* x, const uint8_t* S, const float* M, int batch, int n,
                                   int algorithm, float beta, float chi, int n_iter, void* stream);

/* a1-a4 with a choice of storage precision: precision 0 is spring_iterate; precision 1
 * keeps x and the FFT intermediate as FP16 (half2) between the passes while every
 * operation runs in FP32 (x is rounded to FP16 once on entry and returned as complex64).
 * Scratch: batch x N x N x 8 bytes. */
spring_status spring_iterate_ex(void* x, const uint8_t* S, const float* M, int batch, int n,
                                int algorithm, float beta, float chi, int n_iter, int precision,
                                void* stream);

/* a5 smoothing: out = periodic convolution of |x| with the separable normalised Gaussian
 * of width sigma (taps d = -r..r, r = ceil(4 sigma)); sigma = 0 copies |x|.
 * out: batch x N x N float32.  sigma <= 64. */
spring_status spring_smooth(const void* x, float* out, int batch, int n, float sigma,
                            void* stream);
/* a5 UpdateSupport (Eq. shrinkwrap): S = [rho_sigma >= tau max(rho_sigma)], per image.
 * Scratch: the smoothed map and per-image maxima. */
spring_status spring_update_support(const void* x, uint8_t* S, int batch, int n, float sigma,
                                    float tau, void* stream);
/* a5 UpdateSupportSize (App. "The modified Shrink-wrap"): S = the alpha[b] pixels of
 * largest rho_sigma (equal values taken in increasing linear index), so the area is
 * exactly alpha[b] (clamped to [0, N^2]).  alpha: DEVICE array of `batch` int64. */
spring_status spring_update_support_size(const void* x, uint8_t* S, int batch, int n,
                                         float sigma, const int64_t* alpha, void* stream);

/* a6 GetError (Eq. error_calc): err[b] = sqrt( sum_Xi (|F[S x]| - M)^2 / sum_Xi M^2 ),
 * accumulated in FP64 in a fixed order (deterministic).  err: DEVICE double[batch].
 * Scratch: one work image per batch entry and per-block partial sums. */
spring_status spring_fourier_error(const void* x, const uint8_t* S, const float* M, int batch,
                                   int n, double* err, void* stream);

/* GetError without allocation.  Some callers cannot call cudaMalloc or cudaMallocAsync
 * (a host framework whose allocator owns the device memory budget, code that must not
 * allocate while graphs are being captured, real-time loops that cannot take an
 * allocation's implicit synchronisation).  This entry point computes exactly what
 * spring_fourier_error computes, with its scratch (transformed images and partial sums)
 * in a fixed file-scope device array of SPRING_NOALLOC_SCRATCH_BYTES that every GPU
 * loading the library holds until exit; it calls no allocator.  The paper has no
 * counterpart: this is an interface convenience of this library.
 *  - Limit: batch * N * N * 8 bytes, rounded up to 256, plus batch * (N / 16) * 16 bytes
 *    must fit in SPRING_NOALLOC_SCRATCH_BYTES (16 MiB: e.g. batch <= 7 at 512 x 512,
 *    <= 1 at 1024 x 1024); larger requests return SPRING_E_INVALID with the sizes.
 *  - The first call on each device looks up the array's device address and uploads a
 *    twiddle table (no allocation); make that first call before any stream capture.
 *  - Every call shares the one array, which keeps the last call's contents (each call
 *    writes all it reads).  Calls that overlap on the GPU (different streams, or threads
 *    without ordering) race on it: serialise them.
 *  - err: DEVICE double[batch]. */
#define SPRING_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)
spring_status spring_fourier_error_noalloc(const void* x, const uint8_t* S, const float* M,
                                           int batch, int n, double* err, void* stream);

/* a7 area bookkeeping (Alg. improve, first three steps) on the parent population:
 * out[0] = alpha_best = area of the support of argmin err (ties: lowest index; err NULL:
 * individual 0), out[1] = alpha_all = area of the union of the P supports,
 * out[2] = alpha_eval = round_half_up((g alpha_best + (G - g) alpha_all) / G), exactly.
 * out: DEVICE int64[3]. */
spring_status spring_area_stats(const uint8_t* S, const double* err, int P, int n, int g,
                                int G, int64_t* out, void* stream);

/* a9 RandomChoice (App. "Crossover"): for each p < P three distinct parents a, b, c, all
 * != p, from Philox-4x32-10 keyed by seed at counter (g, p, 1 << 24, 0).  abc: DEVICE
 * int32[P x 3].  Integer draws are floor(u32 * m / 2^32) among the remaining candidates,
 * then the excluded indices are skipped in increasing order. */
spring_status spring_random_choice(uint64_t seed, int g, int P, int32_t* abc, void* stream);
/* a9 CrossoverMap (App. "Crossover", Fig. crossmap) of individual p at generation g:
 * map: DEVICE uint8[N x N] in DFT order.  tile_max 0 = N/8. */
spring_status spring_crossover_map(uint64_t seed, int g, int p, int n, int tile_min,
                                   int tile_max, float cp, uint8_t* map, void* stream);

/* a8 Reshift (App. "Aligning the reconstructions", Eq. crosscorr): align each x[b] (and
 * S[b]) onto ref[b]: c = F^-1[Xi conj(F x) F ref], c_t = F^-1[Xi F x F ref]; the larger
 * peak of |c|, |c_t| picks the twin (ties: not twin), its position s the shift (ties:
 * lowest linear index), its phase phi the global phase;
 *   x'(r) = e^{i phi} x(r - s)   or   e^{i phi} conj(x(s - r)).
 * x_out/S_out may be NULL; info: DEVICE int32[batch x 3] = (s_y, s_x, twin) or NULL;
 * phase: DEVICE float[batch] or NULL.  Scratch: spectra and correlations. */
spring_status spring_reshift(const void* x, const uint8_t* S, const void* ref, const float* M,
                             int batch, int n, void* x_out, uint8_t* S_out, int32_t* info,
                             float* phase, void* stream);

/* a8+a9 Crossover (Alg. crossover) of a population of P at generation g: new individual
 * p mixes its parents a, b, c aligned onto p, in Fourier space:
 *   F x_new = F a' + cw (F b' - F c')  on the crossover map,  F x_p elsewhere;
 *   S_new = S_a' OR (S_b' AND S_c' AND S_p).
 * parents: DEVICE int32[P x 3] (output) or NULL. */
/* a9 with crossover averaging (App. "Crossover averaging", Eq. crossavg): before the mix,
 * parent a's Fourier moduli become ca * mavg + (1 - ca) |F a| with its phases kept (a zero
 * modulus takes phase 0).  mavg: N x N float, DFT order, unitary scale (spring_average_moduli);
 * ca in [0, 1]; ca = 0 is spring_crossover (mavg may then be NULL).  Scratch and errors as
 * spring_crossover. */
spring_status spring_crossover_ca(const void* pop_x, const uint8_t* pop_S, const float* M, int P, int n,
                                  uint64_t seed, int g, float cw, float cp, int tile_min, int tile_max,
                                  float ca, const float* mavg, void* new_x, uint8_t* new_S,
                                  int32_t* parents, void* stream);
/* The average moduli of crossover averaging: mavg = (|F rho_avg| + mean_p |F rho_p|) / 2
 * (Eqs. avgint1, avgint2), rho_avg the population aligned onto its best individual
 * (argmin of err; err NULL: individual 0) and averaged as in spring_average.  mavg: N x N
 * float out, DFT order.  Scratch: (3P + 1) N^2 complex64. */
spring_status spring_average_moduli(const void* pop_x, const uint8_t* pop_S, const double* err, const float* M,
                                    int P, int n, float* mavg, void* stream);
spring_status spring_crossover(const void* pop_x, const uint8_t* pop_S, const float* M, int P,
                               int n, uint64_t seed, int g, float cw, float cp, int tile_min,
                               int tile_max, void* new_x, uint8_t* new_S, int32_t* parents,
                               void* stream);

/* a10 Select (Alg. select): for each p with new_err[p] < pop_err[p] (strict) copy the new
 * density, support and error over the parent's.  replaced: DEVICE uint8[P] or NULL. */
spring_status spring_select(void* pop_x, uint8_t* pop_S, double* pop_err, const void* new_x,
                            const uint8_t* new_S, const double* new_err, int P, int n,
                            uint8_t* replaced, void* stream);

/* a12 Average (Eq. avgrec): every individual aligned onto the best (argmin err, ties:
 * lowest index) and averaged; the support is the union of the aligned supports.
 * avg: DEVICE complex64 N x N; S_avg: DEVICE uint8 N x N. */
spring_status spring_average(const void* pop_x, const uint8_t* pop_S, const double* err,
                             const float* M, int P, int n, void* avg, uint8_t* S_avg,
                             void* stream);

/* a11 Initialize (App. "Initialization of the starting densities"): P densities, each a
 * sum of n_spheres projected spheres (thickness 2 sqrt(R^2 - d^2)) in the bounding square
 * of S0 with diameters in [0.2, 0.9] of its side and phases in [-phi_max, phi_max]
 * (Philox counter (0, p, 4 << 24 | sphere, 0)); then |rho|^gamma with the phase kept,
 * restriction to S0, and the scale sqrt(nu) of Eq. norm.  x: DEVICE complex64 P x N x N. */
spring_status spring_initialize(uint64_t seed, const uint8_t* S0, const float* M, int n, int P,
                                int n_spheres, float gamma, float phi_max, void* x,
                                void* stream);

/* ---------------------------------------------------------------- kernel variants
 * The two per-iteration passes (row pass: inverse row FFT, update, forward row FFT;
 * column pass: column FFT, P_M, inverse column FFT) have launch-shape variants per side N:
 *   row 0: state loads before the inverse transform, one block per SM of registers;
 *   row 1 / 2: state loads after it, register budget for two / three blocks per SM;
 *   row 3 / 4: x and S rows streamed into shared memory during the inverse transform;
 *   row 5 / 6: alternative radix plan, register budget for two / four blocks per SM;
 *   col 0: default radix plan, 16-column tiles; col 1: alternative radix plan;
 *   col 2: 32-column tiles (16 at N = 1024); col 3: 8-column tiles;
 *   col 4 / 5: persistent blocks fed by TMA (16 / 8-column tiles, next tile in flight);
 *   col 6 / 7: transposed tiles, one lane group per column (warp-level synchronisation);
 *   col 8 / 9: two adjacent columns per thread, 16-byte accesses throughout, the two
 *   columns' transforms on packed two-lane FP32 instructions (16 / 32-column tiles);
 *   col 10: column 1's plan in 512-thread blocks held to three per SM.
 * Variants sharing a radix plan and arithmetic give bit-identical results (row 0-4, row
 * 5-6; column 0 and 2-7, column 1 and 10 (10 is column 0 at N = 64, 96), column 8-9); the
 * others differ by rounding.  A run tunes each side once per process
 * (spring_autotune on the run's batch) unless the environment sets SPRING_AUTOTUNE=0 or
 * the variant was set explicitly. */
spring_status spring_set_kernel_variant(int n, int row_variant, int col_variant); /* -1 = keep */
spring_status spring_get_kernel_variant(int n, int* row_variant, int* col_variant);
/* Time every variant on `batch` scratch images of side n on `stream` and keep the
 * fastest.  Allocates scratch; blocks the host until done; do not call during capture. */
spring_status spring_autotune(int n, int batch, void* stream);
/* How runs iterate at side n: 0 = two passes through HBM per iteration (row pass, column
 * pass), 1 = the on-chip kernel of spring_iterate_fused (N <= 256; INVALID where the
 * device cannot hold its clusters), 2 = the split passes (N = 192, 384, 512, 768, 1024):
 * the column transform is decimated in frequency over the rows, n = n1 + (N/Q) n2, its
 * first radix-Q stage runs in the row pass on the Q rows n1 + (N/Q) n2 (Q = 3 at 192, 384
 * and 768, 2 at 512: all rows of a set in one lane group, the stage in registers; Q = 8 at
 * 1024: one block per set of 8 rows) and the column pass transforms N/Q-point chunks (the
 * same sums in another order).  The autotuner picks the fastest; an explicit choice is
 * kept; until either, the fastest measured on a GB300 (2 at 192 and 384-1024, 0 elsewhere). */
spring_status spring_set_iteration_path(int n, int path);
spring_status spring_get_iteration_path(int n, int* path);

/* ---------------------------------------------------------------- instrumentation
 * Per-kernel-class launch counts and (when enabled) CUDA-event durations recorded on the
 * launching stream.  Used by the benchmark for its roofline figures. */
typedef struct {
  uint64_t launches;       /* launches since the last reset */
  double total_ms;         /* summed event time (timing enabled only) */
  uint64_t timed;          /* launches that were timed */
  double bytes_per_launch; /* mean algorithmic bytes of the timed launches (of the last
                              launch if none was timed) */
} spring_kernel_stat;
#define SPRING_KC_ROW_ITER 0  /* iteration row pass (inverse row FFT, update, forward row FFT) */
#define SPRING_KC_COL_PM 1    /* iteration column pass (column FFT, P_M, inverse column FFT) */
#define SPRING_KC_OTHER 2     /* every other kernel of the library */
#define SPRING_KC_FUSED 3     /* on-chip whole iterations (spring_iterate_fused, N <= 256) */
#define SPRING_KC_COUNT 4
/* Failure detection.  Every device-side wait of the library is bounded: after its limit it
 * records the timed-out wait in a per-device status word and its kernel returns; blocking
 * runs read the word when their stream has completed and then return SPRING_E_TIMEOUT.
 * This call exercises that path: one block waits on a barrier that nothing completes, with
 * a limit of `cycles` clock cycles (1 .. 2^32), and the call returns SPRING_E_TIMEOUT when
 * the timeout was detected and reported (SPRING_OK would mean it was not).  Blocking; the
 * device stays usable.  INVALID for cycles outside the range. */
spring_status spring_check_wait_timeout(long long cycles);

void spring_stats_reset(void);
/* on = 0: no timing; on = k >= 1: every k-th launch of each timed class (ROW_ITER,
 * COL_PM, FUSED) is bracketed by two events (k = 1: every launch).  A stride that is
 * coprime to the run's block lengths samples every position of a block evenly. */
void spring_stats_enable_timing(int on);
void spring_stats_get(int kernel_class, spring_kernel_stat* out);
/* Total kernel launches of the library since the last reset. */
uint64_t spring_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* SPRING_H */
