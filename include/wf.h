/*
 * wf.h -- C ABI of the GB300 dual messenger Wiener-filter library.
 *
 * The library solves the Wiener-filter equation (S^-1 + N^-1) s_WF = N^-1 d
 * (Eq. 2 of Kodi Ramanah, Lavaux & Wandelt 2017) on the sphere with the
 * hybrid dual messenger iteration of the paper's Algorithm 2 (Eqs. 13-15):
 * a HEALPix-ring pixelisation with RING pixel order, a band-limited isotropic
 * signal covariance S = diag(C_l), a per-pixel noise variance N = diag(sigma^2_p)
 * and an arbitrary mask (N^-1 = 0 on masked pixels).
 *
 * Conventions used by every call:
 *  - Maps: double[Npix], Npix = 12 nside^2, HEALPix RING order.
 *  - Harmonic coefficients ("alm"): double[2 * Nalm], Nalm = (lmax+1)(lmax+2)/2,
 *    complex numbers stored (re, im) interleaved, m-major: the coefficient
 *    (l, m), 0 <= m <= l <= lmax, sits at complex index m*(2 lmax + 1 - m)/2 + l.
 *    Negative m follow from the reality of the field.  Y_lm are orthonormal
 *    with the Condon-Shortley phase.
 *  - Synthesis Y: s(p) = sum_l [a_l0 Y_l0(p) + 2 sum_{m>0} Re(a_lm Y_lm(p))].
 *    Analysis "map2alm" is Omega * Y^T with Omega = 4 pi / Npix (no ring
 *    weights): a_lm = Omega sum_p s(p) Y*_lm(p).
 *  - "_dev" pointers are CUDA device pointers; "_host" pointers are host memory.
 *    The caller owns every buffer it passes; the library owns its plan and
 *    the plan's workspaces.  Device arguments must stay valid until the call
 *    that uses them has completed on the plan's stream.
 *  - All work of a plan is ordered on the CUDA stream given at plan creation
 *    (NULL = the legacy default stream).  Calls return when their results are
 *    ready (they synchronise the plan's stream) unless documented otherwise.
 *  - No call throws; each returns a wf_status.  wf_last_error() gives a
 *    human-readable message for the last failing call of the calling thread.
 *  - A plan is not thread-safe: calls on one plan must not overlap.
 */
#ifndef WF_H
#define WF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wf_plan_s *wf_plan_t;

typedef enum {
  WF_OK = 0,
  WF_ERR_ARG = 1,            /* invalid argument (nothing was launched) */
  WF_ERR_CUDA = 2,           /* a CUDA call failed; see wf_last_error() */
  WF_ERR_NOT_CONVERGED = 3,  /* max_iter reached; outputs hold the last iterate */
  WF_ERR_NUMERIC = 4,        /* NaN/Inf met in the iteration */
  WF_ERR_TIMEOUT = 5,        /* a bounded device wait gave up */
  WF_ERR_UNIMPLEMENTED = 6,
  WF_ERR_STATE = 7           /* call not valid for this plan (e.g. no noise) */
} wf_status;

typedef enum { WF_PREC_FP64 = 0, WF_PREC_MIXED = 1 } wf_precision;

typedef enum {
  WF_METHOD_DUAL = 0,      /* the hybrid dual messenger (Algorithm 2) */
  WF_METHOD_MESSENGER = 1  /* the standard messenger (Algorithm 1, Sect. 2.1):
                              lambda cooling from lambda0 by beta (eta),
                              untruncated signal step C / (C + lambda alpha
                              Omega), tolerances in three steps (100 eps for
                              lambda >= 100, 10 eps for lambda >= 10, eps) */
} wf_method;

typedef enum {
  WF_STOP_CAUCHY = 0, /* last stage ends when ||x_i - x_{i-1}|| / ||x_i|| < eps_final */
  WF_STOP_ERROR = 1   /* last stage ends when the geometric error estimate
                         c_i r / (1 - r) is < eps_final, with r the larger of
                         c_i / c_{i-1} and (c_i / c_{i-16})^(1/16) */
} wf_stop_rule;

/* Solver options.  Start from wf_opts_default() and override fields. */
typedef struct {
  double beta;       /* cooling factor of xi, 0 < beta < 1 (Algorithm 2; default 0.75) */
  double eps_final;  /* tolerance of the last stage (default 1e-6) */
  double eps_cap;    /* relaxed tolerance of the early stages is
                        min(eps_cap, eps_final * mu / alpha) (default 1e-2) */
  double mu0;        /* initial mu in pixel-variance units; < 0 selects
                        mu0 * Omega = beta * max_l C_l (default -1) */
  int max_iter;      /* bound on the total number of iterations (default 200000) */
  int stop_rule;     /* wf_stop_rule (default WF_STOP_CAUCHY, the paper's
                        criterion of Sect. 3) */
  int precision;     /* wf_precision (default WF_PREC_FP64).  WF_PREC_MIXED
                        keeps FP32 copies of C_l, of the data and of
                        sigma^2 / alpha: C_l, |d| and the alm must lie in
                        FP32's normal range (~1e-38 to 3e38) for its FP32
                        stages to be accurate; the last stage's acceptance
                        test is FP64 either way. */
  int band_limit;    /* 1: restrict each stage's transforms to the band where
                        the truncated spectrum is nonzero (exact; default 1) */
  int graph_chunk;   /* iterations per captured CUDA graph launch; 0 = auto */
  int refine_max;    /* WF_PREC_MIXED: max FP64 refinement steps (default 8) */
  int timing;        /* 1: time the Legendre kernels of every iteration with
                        CUDA events recorded inside the captured graphs
                        (read with wf_kernel_stats; default 0) */
  int autotune;      /* 1: at plan creation, time the launch variants of the
                        Legendre kernels for this geometry and keep the
                        fastest (cached per nside, lmax; default 0) */
  int anchor;        /* WF_PREC_MIXED: arithmetic of the anchor steps
                        r = G(x_a) - x_a.  1 (default): the Legendre
                        transforms and ring FFTs in double-float (pairs of
                        FP32, ~48-bit significand) on the FP32 pipe;
                        0: plain FP64.  The last stage's acceptance test
                        and fp_residual always use plain FP64. */
  /* WF_PREC_MIXED anchoring.  The defaults reproduce the FP64 solve's
     result (same stage lengths; 1.9e-7 relative L2 at nside 1024, lmax
     2048; 5.7e-8 at nside 256): every stage anchored, re-anchoring bounds
     tied to the stage tolerance, the tail stages' decisions taken in the
     anchor arithmetic.  FP32 transforms err by ~1e-5 of their input's norm,
     while late-stage steps are ~1e-3 of the correction they act on; without
     these the late stages' Cauchy tests, whose thresholds the FP64 ratios
     cross within 1e-4, can end a stage one or two iterations off.
     anchor_eps = 3e-5, anchor_cap_tol = 0, tail_exact = 0 is ~1.3x faster
     with ~1e-5 distance from the FP64 result (both sit ~1e-2 from the
     fixed point under the paper's criterion). */
  double anchor_eps; /* stages whose tolerance is below anchor_eps run
                        anchored (correction form around an FP64 anchor);
                        the others run plain FP32 iterations.  >= eps_cap
                        anchors every stage (default 1). */
  double anchor_cap; /* an anchored stage takes a new anchor when
                        ||delta|| > anchor_cap ||x_a|| (default 1e-2). */
  double anchor_cap_tol; /* > 0 tightens anchor_cap to anchor_cap_tol times
                        the stage's tolerance (default 100). */
  int method;        /* wf_method (default WF_METHOD_DUAL) */
  double lambda0;    /* WF_METHOD_MESSENGER: initial lambda (default 1e4) */
  int tail_exact;    /* with WF_STOP_CAUCHY: 1 = the tail stages (those
                        whose tolerance is eps_final) take their stage
                        decisions in the anchor arithmetic, so that their
                        Cauchy tests see FP64-accurate steps (default 1). */
  double tail_window; /* with tail_exact: a tail stage runs FP32 correction
                        iterations until its FP32 Cauchy ratio is below
                        (1 + tail_window) eps_final, then anchor-arithmetic
                        iterations to its decision; <= 0: the whole tail in
                        the anchor arithmetic (default 0.08, above the FP32
                        ratio's measured error of 2.4 % there). */
  double tail_cap_tol; /* with tail_window > 0: the re-anchoring bound of the
                        tail stages' FP32 corrections, tail_cap_tol times
                        the stage tolerance (default 10): their trajectory
                        error moves the late steps the decisions read */
} wf_opts;

/* Per-solve statistics. */
typedef struct {
  int iterations;      /* inner iterations, all stages (mixed: all passes) */
  int stages;          /* cooling stages run (mixed: of the first pass) */
  int converged;       /* 1 if the last stage met its stop rule */
  int refinements;     /* WF_PREC_MIXED: FP64 correction steps taken */
  double alpha;        /* min noise variance over observed pixels */
  double final_cauchy; /* last Cauchy ratio */
  double err_estimate; /* last geometric error estimate (WF_STOP_ERROR) */
  double fp_residual;  /* WF_PREC_MIXED: final FP64 fixed-point residual */
  double elapsed_ms;   /* device time of the solve (CUDA events) */
  long kernel_launches; /* kernels of this library launched by the solve */
} wf_stats;

void wf_opts_default(wf_opts *opts);

/* Create a plan for one geometry and one problem.
 *  nside         HEALPix resolution, 1 <= nside <= 8192.
 *  lmax          band limit, 1 <= lmax <= 3 nside - 1.
 *  cl_host       host double[lmax+1]: C_l >= 0 (signal covariance, Eq. 2).
 *  noise_var_dev device double[Npix]: sigma^2_p > 0 on observed pixels; may be
 *                NULL for a transform-only plan (wf_alm2map / wf_map2alm).
 *  mask_dev      device uint8_t[Npix], nonzero = masked (N^-1 = 0); may be NULL.
 *  opts          NULL = defaults.   stream: cudaStream_t or NULL.
 * Errors: WF_ERR_ARG for out-of-range sizes, negative C_l, all pixels masked,
 * or a non-positive / non-finite variance on an observed pixel (checked on
 * the device during creation).  The noise and mask are copied; the caller
 * may free them after the call. */
wf_status wf_plan(wf_plan_t *out, int nside, int lmax, const double *cl_host,
                  const double *noise_var_dev, const uint8_t *mask_dev,
                  const wf_opts *opts, void *stream);

/* Replace the noise variance and mask of an existing plan (same geometry). */
wf_status wf_set_noise(wf_plan_t plan, const double *noise_var_dev,
                       const uint8_t *mask_dev);

/* Replace the spectrum C_l of an existing plan. */
wf_status wf_set_cl(wf_plan_t plan, const double *cl_host);

/* Solve (S^-1 + N^-1) s = N^-1 d with Algorithm 2 (Sect. 2.2).
 *  d_dev      device double[Npix] data map (values on masked pixels ignored).
 *  alm_dev    device double[2 Nalm] output: the harmonic coefficients of
 *             s_WF, or NULL.
 *  map_dev    device double[Npix] output: s_WF = Y alm, or NULL.
 *  init_alm_dev / init_map_dev  optional warm start (NULL = the paper's cold
 *             start s_0 = 0, t_0 = d): the initial signal coefficients and
 *             messenger field t_0; if only init_alm_dev is given, t_0 = d.
 *  stats      optional output.
 * Returns WF_OK, WF_ERR_NOT_CONVERGED (outputs hold the last iterate) or an
 * error. */
wf_status wf_solve(wf_plan_t plan, const double *d_dev, double *alm_dev,
                   double *map_dev, const double *init_alm_dev,
                   const double *init_map_dev, wf_stats *stats);

/* Solve n independent problems together (Sect. 2.2 per map).  plans[i] must
 * be distinct plans with noise; each may have its own nside, lmax, spectrum,
 * noise, mask and options.  d_dev[i] / alm_dev[i] / map_dev[i] as in
 * wf_solve (alm_dev, map_dev and their entries may be NULL).  The maps run
 * concurrently on private streams, each with its own captured iteration
 * graphs and device-side stage control, driven by a pool of host threads
 * (at most one per hardware thread) that take the maps largest first;
 * results equal wf_solve's map by map.  Concurrency is best when the
 * process sets CUDA_DEVICE_MAX_CONNECTIONS=32 before its CUDA context is
 * created (the default 8 hardware queues make streams share queues).
 * stats: NULL or n entries.  elapsed_ms: device
 * time from the start of the first map to the end of the last.  Returns the
 * first error, else WF_ERR_NOT_CONVERGED if a map hit max_iter, else WF_OK. */
wf_status wf_solve_batch(wf_plan_t *plans, int n, const double *const *d_dev,
                         double *const *alm_dev, double *const *map_dev, wf_stats *stats,
                         double *elapsed_ms);

/* Stop rules of wf_pcg. */
typedef enum {
  WF_PCG_STOP_CAUCHY = 0,   /* ||z_{i+1} - z_i|| / ||z_{i+1}|| < tol (App. C) */
  WF_PCG_STOP_RESIDUAL = 1  /* ||A z - y|| / ||y|| < tol (the residual of Fig. 5) */
} wf_pcg_stop;

/* The Wiener filter by preconditioned conjugate gradients, the paper's
 * comparison method (App. C): A z = y with A = 1 + C^1/2 Y^T N^-1 Y C^1/2,
 * y = C^1/2 Y^T N^-1 d, s_WF = C^1/2 z, preconditioned by the harmonic
 * diagonal 1 + C_l sum_p N^-1_p / (4 pi), restarted every `restart`
 * iterations (the paper: 200), FP64 transforms.  Unlike wf_solve, its fixed
 * point is Eq. (2) itself (no messenger, so no quadrature gap).
 *  d_dev      device double[Npix] data map (masked pixels ignored).
 *  alm_dev    device double[2 Nalm] output s_WF coefficients, or NULL.
 *  map_dev    device double[Npix] output s_WF = Y alm, or NULL.
 *  tol        tolerance of the stop rule; stop_rule: wf_pcg_stop.
 *  max_iter, restart  >= 1.
 *  stats      optional: iterations, converged, final_cauchy (the last
 *             step's Cauchy ratio), err_estimate = fp_residual (the last
 *             relative residual), elapsed_ms, kernel_launches.
 * Allocates its work vectors (8 alm-sized) for the call.  Returns WF_OK,
 * WF_ERR_NOT_CONVERGED (outputs hold the last iterate), WF_ERR_STATE for a
 * plan without noise, WF_ERR_NUMERIC, WF_ERR_ARG. */
wf_status wf_pcg(wf_plan_t plan, const double *d_dev, double *alm_dev, double *map_dev,
                 double tol, int stop_rule, int max_iter, int restart, wf_stats *stats);

/* Same as wf_solve with host buffers: copies d in, solves, copies the
 * requested outputs back (both copies are part of the call). */
wf_status wf_solve_host(wf_plan_t plan, const double *d_host, double *alm_host,
                        double *map_host, wf_stats *stats);

/* Diagnostics of a candidate solution alm_dev (Sect. 4, App. C), FP64:
 *  rel_res_wf  ||A x - y|| / ||y||, A = 1 + C^1/2 Y^T N^-1 Y C^1/2,
 *              x = C^-1/2 alm, y = C^1/2 Y^T N^-1 d (the residual of Fig. 5);
 *  rel_res_fp  ||G(alm) - alm|| / ||alm|| for one last-stage iteration G
 *              (xi = alpha, mu = 0): the messenger fixed-point residual;
 *  chi2        (d - Y alm)^T N^-1 (d - Y alm) + alm^T C^-1 alm.
 * Any output pointer may be NULL. */
wf_status wf_residual(wf_plan_t plan, const double *d_dev, const double *alm_dev,
                      double *rel_res_wf, double *rel_res_fp, double *chi2);

/* The same three diagnostics as wf_residual for callers that cannot
 * allocate device memory while they run: code bound to a fixed device-memory
 * budget, or running inside a framework whose pool allocator owns the device
 * memory (a cudaMalloc can fail there, or take memory the pool counts on),
 * and loops with a time budget per pass (cudaMalloc / cudaFree may
 * synchronise the device and stall them).  wf_residual takes its temporaries
 * from cudaMalloc on each call; this variant allocates nothing (no
 * cudaMalloc, no cudaFree, no host heap) and takes them from one static
 * device array of 4.8 MB that every GPU loading the library holds until
 * exit.  The paper has no counterpart; the results equal wf_residual's.
 *  - Size limit: 2 Npix + 6 Nalm + 3 (lmax + 1) + 256 doubles must fit in
 *    600,000 (e.g. nside <= 128 with lmax <= 256); larger plans get
 *    WF_ERR_ARG, and should use wf_residual.
 *  - Host-synchronous: the call waits for the plan's stream and returns the
 *    diagnostics as host scalars.
 *  - The current device must be the plan's (else WF_ERR_STATE).
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress); make that call before any stream capture.
 *  - All calls share the array: calls that overlap on the GPU race.  The
 *    call also uses the plan's own workspaces, so it must not overlap any
 *    other call on the same plan.
 * Arguments and outputs as for wf_residual. */
wf_status wf_residual_static(wf_plan_t plan, const double *d_dev, const double *alm_dev,
                             double *rel_res_wf, double *rel_res_fp, double *chi2);

/* FP64 spherical-harmonic transforms on the plan's geometry.
 * wf_alm2map: map = Y alm.  wf_map2alm: alm = Omega Y^T map. */
wf_status wf_alm2map(wf_plan_t plan, const double *alm_dev, double *map_dev);
wf_status wf_map2alm(wf_plan_t plan, const double *map_dev, double *alm_dev);

/* The same transforms computed with the FP32 kernels of WF_PREC_MIXED (FP64
 * recurrence seeds, FP32 recurrence, accumulation and ring FFTs); FP64 in
 * and out.  Their error against wf_alm2map / wf_map2alm is the transform
 * error the mixed-precision solve works with. */
wf_status wf_alm2map_f32(wf_plan_t plan, const double *alm_dev, double *map_dev);
wf_status wf_map2alm_f32(wf_plan_t plan, const double *map_dev, double *alm_dev);

/* The same transforms in double-float (each value an unevaluated sum of two
 * FP32 numbers, ~48-bit significand, run on the FP32 pipe), the Legendre
 * steps and the ring FFTs: the arithmetic of the mixed solver's anchor steps
 * (opts.anchor = 1).  FP64 in and out; errors as wf_alm2map_f32. */
wf_status wf_alm2map_df64(wf_plan_t plan, const double *alm_dev, double *map_dev);
wf_status wf_map2alm_df64(wf_plan_t plan, const double *map_dev, double *alm_dev);

/* Grouped transforms: the same two transforms (Sect. 2.2's Y and Omega Y^T)
 * of nmaps maps that share the plan's geometry, in one pass of the Legendre
 * step.  For each m, the Legendre step of all maps is one dense product of
 * a table lambda_lm(z_ring) with the maps' ring coefficients (2 columns per
 * map, real and imaginary parts).  It runs on the tensor cores (tcgen05,
 * TF32 operands split hi + lo, three products per term, FP32 accumulation),
 * so the accuracy is about that of wf_alm2map_f32 / wf_map2alm_f32.  The
 * ring FFTs are the FP32 ones of those two calls.
 *  maps_dev  nmaps x Npix doubles, map b at offset b * Npix.
 *  alm_dev   nmaps x Nalm complex (2 doubles each), map b at offset
 *            b * 2 * Nalm doubles, layout as for wf_solve.
 *  nmaps     >= 0; up to 128 maps go into one product, and more are done
 *            in groups of 128.  0 does nothing.
 * The first call builds the table on the device: two copies, one laid out
 * for each direction, each 8 bytes (TF32 hi and lo) per (l, m, ring pair),
 * about 16 bytes per term in all (~1.1 GB at Nside 256, lmax 512).  Its
 * operand buffers are sized for the largest
 * group seen.  Both stay until wf_destroy.  Host-synchronous.  Errors:
 * WF_ERR_ARG for nmaps < 0 or a NULL buffer with nmaps > 0; WF_ERR_CUDA
 * (e.g. out of device memory); WF_ERR_TIMEOUT if a device barrier wait gave
 * up. */
wf_status wf_map2alm_group(wf_plan_t plan, int nmaps, const double *maps_dev,
                           double *alm_dev);
wf_status wf_alm2map_group(wf_plan_t plan, int nmaps, const double *alm_dev,
                           double *maps_dev);

/* Device time and work of the grouped transforms' tensor-core
 * contractions since plan creation or the last reset.
 *  ms        summed CUDA-event time of the contraction launches.
 *  launches  number of contraction launches.
 *  gflop     algorithmic work: 2 flops per (l, m, ring pair, column) of
 *            the plain product.  This is before the 3x of the split
 *            products.
 *  gbyte     bytes the launches must move: both tables' hi and lo parts of
 *            the rows the tiles hold, the maps' operands once, the results
 *            once.
 * Any output pointer may be NULL; reset != 0 zeroes the counters after
 * reading. */
wf_status wf_group_stats(wf_plan_t plan, double *ms, long *launches, double *gflop,
                         double *gbyte, int reset);

/* Sizes of a plan. */
long wf_npix(int nside);
long wf_nalm(int lmax);

/* Copy the per-iteration trace of the last solve to host arrays of length
 * >= *count (in: capacity, out: entries written): stage index, xi, mu and
 * the Cauchy ratio of each iteration. */
wf_status wf_trace(wf_plan_t plan, int *count, int *stage, double *xi,
                   double *mu, double *cauchy);

/* Device time and work of the iteration's kernels in the solves run with
 * opts.timing = 1 since plan creation or the last reset.
 *  kernel    0 = Legendre analysis (Omega Y^T with the fused filter),
 *            1 = Legendre synthesis, 2 = ring step (fold, inverse ring
 *            FFTs, the t-update of Eq. 14, forward ring FFTs; both launches)
 *            of the captured FP32 / FP64 iterations; 3 = Legendre
 *            synthesis, 4 = Legendre analysis (with its tile combine),
 *            5 = ring step, all three in double-float, of the mixed solver's
 *            anchor-arithmetic steps (anchors, stage boundaries, tail).
 *  ms        summed CUDA-event time of the timed launches.
 *  launches  number of timed launches (iterations that did work).
 *  gflop     algorithmic work of those launches.  Kernels 0, 1, 3, 4: GFLOP, 7
 *            flops (recurrence 3, complex accumulate 4) per (l, m, ring pair)
 *            with l <= the band limit of the launch and |lambda_lm| >=
 *            2^-100 (the terms the method needs; the skipped ones are below
 *            that).  Kernels 2, 5: GB of DRAM traffic the step cannot avoid --
 *            ring coefficients read and written for m <= the band limit
 *            (8 bytes each in FP32 stages, 16 in FP64) and d, sigma^2 read
 *            (16 bytes per pixel).
 *  reset     nonzero: clear the counters after reading.
 * Any output pointer may be NULL. */
wf_status wf_kernel_stats(wf_plan_t plan, int kernel, double *ms, long *launches,
                          double *gflop, int reset);

/* Launch variants of the Legendre kernels in use by a plan, and the times
 * the autotuner measured for each candidate (opts.autotune = 1; a choice
 * cached for the geometry reports the timings it was made from; -1 where a
 * candidate was not timed, and everywhere with autotune = 0).
 * Index [0] = FP64 kernels, [1] = FP32 kernels.
 *  syn_np      ring pairs per thread of the synthesis.
 *  syn_packed  FP32 synthesis on packed f32x2 pairs of rings (1: syn_np 2, 4;
 *              2: syn_np 2 with duplicated shared-memory tables).
 *  ana_np      ring pairs per lane of the analysis.
 *  ana_queue   FP32 analysis scheduling: 0 = one CTA per m, 1 = warps take
 *              (m, tile) items from a queue, then a per-m combine kernel.
 *  ana_packed  FP32 per-m analysis on packed f32x2 pairs (ana_np 4, 6, 8).
 *  ana_global_acc  with ana_packed: the per-warp accumulators in global
 *              scratch instead of shared memory (more CTAs/SM); 1: ana_np 4,
 *              6 with 16-l chunks, 2: ana_np 4, 6, 8 with 8-l chunks, 3:
 *              ana_np 8 with 8-l chunks and the seeds in shared memory.
 *  syn_ms      candidates 1, 2, 4 pairs per thread, then (FP32) packed 2, 4
 *              and packed with duplicated tables 2: ms for two launches.
 *  ana_ms      candidates 2, 4, 8, 16 pairs per lane, then (FP32 only) queue
 *              4, 8, packed 4, 8, 6, packed with global accumulators 4, 6
 *              and the same with 8-l chunks 8, 6, 4 and with shared seeds 8:
 *              ms for two launches. */
typedef struct {
  int syn_np[2], syn_packed, ana_np[2], ana_queue, ana_packed, ana_global_acc;
  float syn_ms[2][6], ana_ms[2][15];
} wf_tuning;
wf_status wf_get_tuning(wf_plan_t plan, wf_tuning *out);
/* Set the launch variants (the int fields of *in; the ms fields are
 * ignored).  syn_np in {1, 2, 4}; ana_np in {2, 4, 8, 16} (FP64 {2, 4, 8});
 * ana_queue, ana_packed 0 or 1, syn_packed 0, 1 or 2; ana_queue and ana_packed not both;
 * syn_packed 1 needs syn_np[1] in {2, 4}, syn_packed 2 needs syn_np[1] = 2; ana_queue needs ana_np[1] in {4, 8},
 * ana_packed in {4, 6, 8}; ana_global_acc 1 needs ana_packed and ana_np[1]
 * in {4, 6}, ana_global_acc 2 ana_packed and ana_np[1] in {4, 6, 8}, ana_global_acc 3 ana_packed and ana_np[1] = 8.  The plan's captured iteration graphs are dropped and
 * re-captured on the next solve.  Errors: WF_ERR_ARG for NULL or a value
 * outside these sets (the plan is unchanged). */
wf_status wf_set_tuning(wf_plan_t plan, const wf_tuning *in);

/* Algorithmic work of one Legendre transform at band limit L (<= lmax): the
 * number of (l, m, ring pair) terms with l <= L and |lambda_lm| >= 2^-100. */
wf_status wf_legendre_terms(wf_plan_t plan, int L, double *terms);

/* Measured peak of the arithmetic pipe the Legendre kernels run on (the
 * denominator of their roofline; the paper has no counterpart): independent
 * FMA chains in every thread of a grid that fills every SM of the current
 * device, timed with CUDA events.
 *  kind     0 = FP64 FMA, 1 = FP32 FMA, 2 = packed FP32 (fma.rn.f32x2).
 *  reps     timed launches (1..100), each ~50 ms; the fastest is reported.
 *  tflops   out: 2 flops per FMA / the fastest launch's time, in TFLOP/s.
 *  best_ms, num_sms  out (may be NULL): that launch's time, the SM count.
 * Allocates one small output buffer and a stream of its own for the call.
 * Errors: WF_ERR_ARG for an unknown kind or reps out of range. */
wf_status wf_alu_peak(int kind, int reps, double *tflops, double *best_ms, int *num_sms);

/* ---- learned warm start (the paper has none; an extension of the method)
 * A small network maps (d, log sigma^2, mask) to an initial messenger field
 * t0 (Npix) and initial signal coefficients a0 (Nalm), for wf_solve's
 * init_map_dev / init_alm_dev.  Architecture: per-ring circular 1-D
 * convolutions (3 -> channels -> channels -> 1, odd kernel width) that
 * correct the masked data, t0 = (1-m) d + sigma_d r; a = Omega Y^T t0; a
 * per-l MLP (4 features -> hidden -> hidden -> 1, sigmoid) gives a gain q_l,
 * a0 = q_l a.  Weights are FP32 masters used rounded to BF16 (bf16 = 1) or
 * as FP32 (bf16 = 0); accumulation is FP32.  The net uses the plan's
 * geometry, spectrum, noise and mask (it reads them at each call) and the
 * plan's stream; it must not be used while the plan solves.
 * Parameters are one flat float vector (conv W1 [c][3][k], b1, W2 [c][c][k],
 * b2, W3 [1][c][k], b3, then MLP V1 [h][4], c1, V2 [h][h], c2, V3 [1][h], c3);
 * they start at zero -- set them with wf_net_set_params. */
typedef struct wf_net_s *wf_net_t;
wf_status wf_net_create(wf_net_t *out, wf_plan_t plan, int channels, int kernel,
                        int hidden, int bf16);
long wf_net_num_params(wf_net_t net);
wf_status wf_net_set_params(wf_net_t net, const float *params_host, long n);
wf_status wf_net_get_params(wf_net_t net, float *params_host, long n);
/* Forward pass on data d (device, Npix); t0_dev (Npix) and alm0_dev
 * (2 Nalm doubles) may be NULL. */
wf_status wf_net_forward(wf_net_t net, const double *d_dev, double *t0_dev,
                         double *alm0_dev);
/* Loss L = sum w |a0 - a*|^2 / sum w |a*|^2 against alm_target_dev (the
 * solver's solution) and its gradient w.r.t. every parameter (kept on the
 * device for wf_net_adam_step; copied to grad_host if not NULL). */
wf_status wf_net_loss_grad(wf_net_t net, const double *d_dev,
                           const double *alm_target_dev, double *loss, float *grad_host);
/* One Adam update with the last gradient. */
wf_status wf_net_adam_step(wf_net_t net, float lr, float beta1, float beta2, float eps);
void wf_net_destroy(wf_net_t net);

/* ---- the flat sky (the paper's own Sect. 3 set-up)
 * Algorithm 2 on an n x n periodic grid with 2-D FFTs, FP64: the basis
 * change is orthogonal, so the last stage's fixed point is the Wiener filter
 * of Eq. (2) itself.  With the DFT in numpy's convention one iteration is
 * s = ifft2(f_k fft2(t)), f_k = Sbar_k / (Sbar_k + xi Omega_pix),
 * Sbar_k = max(C_k - mu Omega_pix, 0), then t = s + xi / (sigma^2 + mu)
 * (d - s); cooling, start, tolerances and stop rules as wf_solve's.
 *  n              grid side, a power of two, 8 <= n <= 2048.
 *  pixel_area     Omega_pix = (L / n)^2 (sr): a pixel variance v has the
 *                 power v Omega_pix of the signal power C_k.
 *  ck_host        host double[n * n]: C at each DFT mode (row ky, column
 *                 kx, DFT frequency order), >= 0; copied.
 *  noise_var_dev  device double[n * n] sigma^2 > 0 per pixel (+inf masks a
 *                 pixel); copied.
 *  opts           NULL = defaults; beta, eps_final, eps_cap, mu0 (< 0:
 *                 mu0 Omega_pix = beta max C_k), max_iter, stop_rule,
 *                 graph_chunk are used.
 * Errors: WF_ERR_ARG for a bad size, spectrum, noise or option. */
typedef struct wf_flat_s *wf_flat_t;
wf_status wf_flat_plan(wf_flat_t *out, int n, double pixel_area, const double *ck_host,
                       const double *noise_var_dev, const wf_opts *opts, void *stream);
/* d_dev: device double[n * n] data; s_dev: device double[n * n] output s_WF.
 * Returns WF_OK, WF_ERR_NOT_CONVERGED (s_dev holds the last iterate) or an
 * error; stats as wf_solve's. */
wf_status wf_flat_solve(wf_flat_t plan, const double *d_dev, double *s_dev, wf_stats *stats);
/* Stage index and Cauchy ratio of each iteration of the last solve (host
 * arrays of length >= *count; *count in: capacity, out: entries). */
wf_status wf_flat_trace(wf_flat_t plan, int *count, int *stage, double *cauchy);
void wf_flat_destroy(wf_flat_t plan);

void wf_destroy(wf_plan_t plan);
const char *wf_status_str(wf_status s);
const char *wf_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* WF_H */
