// wf_internal.cuh -- shared declarations of the CUDA implementation behind
// include/wf.h.  Everything here is internal to libwf.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/wf.h"

namespace wf {

// ---------------------------------------------------------------- errors
void set_error(const std::string &msg);
// records a message with static storage (no allocation)
void set_error_static(const char *msg);

#define WF_CUDA(call)                                                        \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess) {                                                 \
      ::wf::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));   \
      return WF_ERR_CUDA;                                                    \
    }                                                                        \
  } while (0)

#define WF_TRY(expr)                    \
  do {                                  \
    wf_status s_ = (expr);              \
    if (s_ != WF_OK) return s_;         \
  } while (0)

// ---------------------------------------------------------------- geometry
// One iso-latitude ring pair: the north ring and its mirror image in the
// south (the equator ring is a "pair" with no south ring).  Both rings share
// nphi, |z| and phi0.
// the FP32 tables as one kernel argument
struct Tab32 {
  const float2 *seed_s;
  const float *zh, *zl;
  const float *rg;
  const float *cl;
};

struct RingPair {
  double z;        // z of the north ring
  double sth;      // sin(theta) of the north ring
  long ofsN;       // first pixel of the north ring
  long ofsS;       // first pixel of the south ring, -1 for the equator ring
  int ringN;       // 0-based ring index of the north ring
  int ringS;       // 0-based ring index of the south ring, -1 for the equator
  int nphi;        // pixels per ring
  int phi_num;     // phi0 = pi * phi_num / phi_den (exact rational)
  int phi_den;
  int fftM;        // FFT length used: nphi if a power of two, else the
                   // Bluestein length (power of two >= 2 nphi - 1)
  long chirp_ofs;  // offset into the chirp table (Bluestein rings), else -1
  long bhat_ofs;   // offset into the chirp-spectrum table, else -1
};

// Device-resident solver state; read by every kernel of an iteration and
// updated by the control kernel.  Stage control stays on the device.
struct SolverState {
  double xi, mu, alpha, beta, omega;
  double eps_final, eps_cap, eps_k;
  double prev_c, last_c, err_est;
  int stage, iter, done, converged, numeric_error;
  int lcur;    // largest l with a nonzero filter in the current stage
  int lnext;   // same for the next stage (the ring kernel fills G up to it)
  int max_iter, stop_rule, band_limit, trace_cap;
  int stage_iter;
  int flat;       // consecutive last-stage iterations without a Cauchy decrease
  int stagnated;  // the last stage stopped at the arithmetic noise floor
  int handoff;    // 1: stop (done, not converged) on entering the mu = 0 stage
  int boundary_stop;  // 1: stop (done) at every stage advance (anchored runs)
  int at_boundary;    // set when a run stopped at a stage advance
  double anchor_eps;  // > 0: stop at an advance into a stage whose tolerance
                      // is below it (FP32 data pass -> anchored stages)
  int noise_guard;  // 1 (FP32 passes): a stage whose Cauchy ratio stops
                    // falling below 1e-3 has reached the arithmetic noise
                    // floor and ends
  int at_final;   // set when the run stopped because of handoff
  int reanchor;   // set when the correction grew past delta_cap2
  double den_fixed;   // > 0: Cauchy denominator ||x||^2 of an anchored stage
  double rate_floor;  // lower bound of the contraction rate used by the
                      // error estimate (slow-mode rate of an earlier cycle)
  double delta_cap2;  // > 0: stop when ||delta||^2 exceeds it (re-anchor)
  double last_den;    // ||x_new||^2 of the last iteration
  double chist[16];   // Cauchy ratios of the last 16 iterations of the stage
  double cmin;        // smallest Cauchy ratio of the stage so far
  int since_min;      // iterations since cmin last fell by 1%
  // anchored stage: the anchor iterate x_a (the analysis then also sums
  // ||x_a + delta||^2, the Cauchy denominator ||x||^2 of the iterate the
  // correction stands for); NULL otherwise
  const double2 *xa;
  // the stage before the last advance (its xi, mu and band)
  double xi_prev, mu_prev;
  int lcur_prev;
  int messenger;  // 1: the standard messenger (Algorithm 1), xi = lambda alpha
  // anchored tail stage: stop (at_window) once the Cauchy ratio falls below
  // window_factor times the stage's threshold, without a stage decision
  // (the anchor arithmetic takes over for it); 0 = off
  double window_factor;
  int at_window;
};

// Tolerance of the stage at mu (pixel units): Algorithm 2 relaxes it as
// min(eps_cap, eps_final max(1, mu / alpha)); Algorithm 1 in three steps of
// lambda = xi / alpha = 1 + mu / alpha (100 eps from lambda 100, 10 eps from
// lambda 10, eps below).  Both end on eps_final.
__host__ __device__ inline double stage_tolerance(const SolverState &s, double mu) {
  if (s.messenger) {
    const double lam = 1.0 + mu / s.alpha;
    if (lam >= 100.0) return fmin(s.eps_cap, 100.0 * s.eps_final);
    if (lam >= 10.0) return fmin(s.eps_cap, 10.0 * s.eps_final);
    return s.eps_final;
  }
  return mu == 0.0 ? s.eps_final : fmin(s.eps_cap, s.eps_final * fmax(1.0, mu / s.alpha));
}

// mu of the signal step's truncation Sbar = max(C - mu Omega, 0): Algorithm 2
// truncates at the stage's mu; Algorithm 1 does not (Sbar = C)
__host__ __device__ inline double filter_mu(const SolverState &s, double mu) {
  return s.messenger ? 0.0 : mu;
}

struct TraceEntry {
  int stage, lcur;   // stage index and band limit of the iteration
  double xi, mu, cauchy;
};

// ---------------------------------------------------------------- plan
struct Plan {
  int nside = 0, lmax = 0, nring = 0, npairs = 0;
  int device = -1;  // the CUDA device current when the plan was created
  long npix = 0, nalm = 0;
  double omega = 0.0;
  cudaStream_t stream = nullptr;
  cudaStream_t capture_stream = nullptr;  // graphs are captured here
  // the ring step's two launches (polar, equatorial rings) run side by side:
  // forked from `stream` onto side_stream and joined back with two events
  cudaStream_t side_stream = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  wf_opts opts{};
  std::vector<double> cl;
  std::vector<RingPair> pairs_h;

  // geometry / Legendre tables
  RingPair *pairs = nullptr;     // [npairs]
  double *cl_d = nullptr;        // [lmax+1]
  double *rc = nullptr;          // [nalm] recurrence coefficient c_lm
  double *rg = nullptr;          // [nalm] scale g_lm (lambda = g u)
  float *rc32 = nullptr;         // [nalm] FP32 copy of rc
  float2 *rcdd = nullptr;        // [nalm] rc as double-float pairs (hi, lo)
  int *seed_l = nullptr;         // [lmax+1][npairs] first l with |lambda| >= 2^-100
  double2 *seed_u = nullptr;     // [lmax+1][npairs] (u_ls, u_ls+1)
  // FP32 kernels' tables (no FP64 arithmetic left in their tile loads and
  // epilogues): seeds in s-units (eps_ls u_ls, eps_ls+1 u_ls+1), z of each
  // pair split as zh + zl (two arrays: the packed kernels pair the zh of two
  // rings, so each value is loaded on its own), g_lm eps_l, C_l
  float2 *seed_s32 = nullptr;    // [lmax+1][npairs]
  float *zs32 = nullptr;         // [2][npairs]: zh, then zl
  float *rg32 = nullptr;         // [nalm]
  float *cl32 = nullptr;         // [lmax+1]

  // launch variants (ring pairs per thread), [0] = FP64, [1] = FP32; set by
  // the autotuner (opts.autotune) or the defaults below
  int syn_np[2] = {2, 2};
  int ana_np[2] = {4, 8};
  // FP32 analysis scheduling: 0 = one CTA per m, 1 = warps take (m, tile)
  // items from a queue and a combine kernel sums the tiles (ana_scratch)
  int ana_queue = 0;
  // FP32 kernels on packed f32x2 pairs of rings (NP even): 0 / 1 (synthesis:
  // 2 = packed with duplicated shared-memory tables)
  int syn_x2 = 0, ana_x2 = 0;
  // packed per-m FP32 analysis with its per-warp accumulators in global
  // scratch (ana_scratch rows [warp][alm]) instead of shared memory: 1 with
  // 16-l chunks, 2 with 8-l chunks
  int ana_gacc = 0;
  float *ana_scratch = nullptr;  // [tiles of 128 pairs][nalm] float2
  int *ana_lstart = nullptr;     // [lmax+1][tiles] first l written per item
  int *ana_counter = nullptr;    // the queue's next item (reset by the combine)
  int num_sms = 0;
  float tune_syn_ms[2][6] = {{-1, -1, -1, -1, -1, -1}, {-1, -1, -1, -1, -1, -1}};
  float tune_ana_ms[2][15] = {{-1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1},
                              {-1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1}};

  // FFT tables
  int fftMmax = 1;
  double2 *tw64 = nullptr;       // e^{-2 pi i k / Mmax}, k < Mmax/2
  float2 *tw32 = nullptr;
  double2 *chirp64 = nullptr;    // e^{i pi j^2 / n}, per Bluestein ring
  float2 *chirp32 = nullptr;
  double2 *bhat64 = nullptr;     // FFT_M of the chirp kernel, bit-reversed order
  float2 *bhat32 = nullptr;
  // the same three tables as double-float pairs (re hi, re lo, im hi, im lo)
  // for the double-float ring transforms of the anchor steps
  float4 *twdd = nullptr, *chirpdd = nullptr, *bhatdd = nullptr;
  // e^{i pi k / n} of every Bluestein ring (phi0 = pi / n), chirp layout
  float4 *phasedd = nullptr;
  long chirp_total = 0, bhat_total = 0;

  // noise
  bool has_noise = false;
  double alpha = 0.0;
  double *nvar = nullptr;        // [npix] sigma^2, +inf on masked pixels
  float *nvar32 = nullptr;       // [npix] sigma^2 / alpha in FP32 (FP32 ring step)
  float2 *nvardd = nullptr;      // [npix] sigma^2 as double-float (hi, lo); (+inf, 0) masked

  // work buffers
  double2 *F64 = nullptr, *G64 = nullptr;   // [nring][lmax+1]
  float2 *F32 = nullptr, *G32 = nullptr;
  double2 *x = nullptr;          // [nalm] current iterate
  double2 *xtmp = nullptr;       // [nalm]
  double2 *xacc = nullptr;       // [nalm] refined solution (mixed precision)
  double2 *xs64 = nullptr;       // [nalm] g_lm x_lm, synthesis input (FP64)
  float2 *xs32 = nullptr;        // [nalm] g_lm x_lm, synthesis input (FP32)
  double2 *src = nullptr;        // [nalm] harmonic source of a correction solve
  // mixed solver, stage boundaries between anchored stages: the unfiltered
  // FP64 analysis U = Omega Y^T t_a of the last two anchors and the next
  // source (allocated by the first mixed solve)
  double2 *uacc[2] = {nullptr, nullptr};
  std::vector<int> untimed;      // iterations run outside the timed graphs
  double *dmap = nullptr;        // [npix] data with masked pixels zeroed
  float *dmap32 = nullptr;       // [npix] FP32 copy of dmap (FP32 ring step)
  float2 *dmapdd = nullptr;      // [npix] dmap as double-float (double-float ring step)
  int data_iters = 0;            // iterations of the last solve that read d
  double *mtmp = nullptr;        // [npix]
  double *partials = nullptr;    // [lmax+1][2]
  double *red = nullptr;         // small reduction scratch
  SolverState *state = nullptr;  // device
  SolverState *state_h = nullptr;  // pinned host mirror
  TraceEntry *trace = nullptr;
  int trace_cap = 0;
  int trace_len = 0;

  // graphs (one per precision), captured lazily
  // 0: FP64 with data, 1: FP32 with data, 2: FP32 correction (harmonic source)
  cudaGraphExec_t graph[3] = {nullptr, nullptr, nullptr};
  int graph_chunk[3] = {0, 0, 0};
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;

  // kernel launches issued for this plan (graph launches count their kernel
  // nodes); mutable so that const launch helpers can count
  mutable long nlaunch = 0;
  long graph_kernels[3] = {0, 0, 0};

  // optional per-kernel timing inside the captured graphs (opts.timing):
  // events around the Legendre analysis (k = 0) and synthesis (k = 1) of
  // every iteration of a chunk; accumulated over active iterations only
  // timed kernels: 0 analysis, 1 synthesis, 2 ring step (both launches)
  std::vector<cudaEvent_t> tev;     // [3 kernels][2 (start, stop)][chunk]
  int tev_chunk = 0;
  // 3, 4: double-float Legendre synthesis / analysis and 5: FP64 ring step
  // of the anchor-arithmetic steps (anchors, boundary steps, tail stages),
  // timed with events around their launches
  double kern_ms[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  long kern_launches[6] = {0, 0, 0, 0, 0, 0};
  cudaEvent_t dd_ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  // algorithmic work of the timed launches: flops (0, 1), DRAM bytes (2)
  double kern_flop[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  std::vector<double> work_cache;    // reduced (l, m, ring-pair) count per band

  // grouped transforms (group.cu): tables and operands, built by the first
  // call; time, algorithmic flops and operand bytes of their contractions
  struct GroupState *group = nullptr;
  double group_ms = 0.0, group_flop = 0.0, group_bytes = 0.0;
  long group_launches = 0;
  std::vector<int> seed_l_h;         // host copy of seed_l
};

// ---------------------------------------------------------------- kernels
// Legendre transforms (legendre.cu).  Modes of the analysis:
enum AnalysisMode { ANA_PLAIN = 0, ANA_FILTER = 1 };

// The synthesis reads xs = g_lm a_lm in its own precision (written by the
// analysis of the previous iteration, or by launch_prescale).
template <typename T2>
wf_status launch_prescale(const Plan &P, const double2 *x, T2 *xs);
template <typename T2>
wf_status launch_legendre_synth(const Plan &P, const T2 *xs, T2 *F,
                                const SolverState *st, int lstatic);
// src (optional, FP64 alm): adds the harmonic source f_l xi Omega src_lm of an
// anchored stage to the filtered coefficients (ANA_FILTER only).
// xs_out (optional): also write g_lm a_lm in the transform precision.
template <typename T2>
wf_status launch_legendre_anal(const Plan &P, const T2 *G, double2 *x,
                               const SolverState *st, int mode, int lstatic,
                               const double2 *src = nullptr, T2 *xs_out = nullptr);

// Double-float (pairs of FP32) Legendre transforms with FP64 inputs and
// outputs, for the anchor steps of the mixed solver (legendre.cu): the same
// contracts as launch_legendre_synth<double2> / launch_legendre_anal<double2>.
// Their ring coefficients F, G and the synthesis input are double-float
// pairs (re hi, re lo, im hi, im lo), 16 bytes like an FP64 complex (the
// plan's F64 / G64 / xs64 buffers hold them in this form), the format of the
// double-float ring transforms.
wf_status launch_prescale_dd(const Plan &P, const double2 *x, float4 *xs);
wf_status launch_legendre_synth_dd(const Plan &P, const float4 *xs, float4 *F,
                                   const SolverState *st, int lstatic);
wf_status launch_legendre_anal_dd(const Plan &P, const float4 *G, double2 *x,
                                  const SolverState *st, int mode, int lstatic,
                                  const double2 *src = nullptr, double2 *xs_out = nullptr);

// Ring transforms (ringfft.cu).  Modes:
enum RingMode {
  RING_SYNTH = 0,     // F -> map (write s)
  RING_ANALYSIS = 1,  // map (masked pixels -> 0) -> G
  RING_FUSED = 2      // F -> s -> t = s + w (d - s) -> G  (in_map NULL: d = 0)
};
// The FP32 fused step (T2 = float2) reads d from in32 (FP32, NULL: d = 0)
// and sigma^2 / alpha from the plan's nvar32, and updates t in FP32; the
// FP64 one reads in_map and nvar.
template <typename T2>
wf_status launch_ring(const Plan &P, int mode, const T2 *F, T2 *G,
                      const double *in_map, double *out_map,
                      const SolverState *st, int lstatic,
                      const float *in32 = nullptr);
// The FP64 ring transforms (FP64 F, G, maps) computed in double-float
// arithmetic on the FP32 pipe (the anchor steps' arithmetic).
wf_status launch_ring_dd(const Plan &P, int mode, const float4 *F, float4 *G,
                         const double *in_map, double *out_map, const SolverState *st,
                         int lstatic, const float2 *in_dd = nullptr);
// The FP32 ring synthesis or analysis of nbatch maps in one launch pair
// (map b: F / G at b * fstride, maps at b * mstride; full band lmax).
wf_status launch_ring_batch32(const Plan &P, int mode, const float2 *F, float2 *G,
                              const double *in_map, double *out_map, int nbatch,
                              long fstride, long mstride);
// FP64 map -> double-float pairs (hi, lo); +inf -> (+inf, 0)
wf_status launch_to_dd(const Plan &P, const double *in, float2 *out, long n);

// once per plan (kernel attributes; allowed outside stream capture only)
wf_status init_legendre_attributes();
wf_status init_ring_attributes();

// autotune.cu: time the Legendre launch variants once per geometry
wf_status autotune(Plan &P);

// batch.cu
wf_status solve_batch(Plan **plans, int n, const double *const *d, double *const *alm,
                      double *const *map, wf_stats *stats, double *wall_ms);

// plan.cu
wf_status build_tables(Plan &P);
wf_status upload_noise(Plan &P, const double *nvar_dev, const uint8_t *mask_dev);

// solve.cu
wf_status solve(Plan &P, const double *d, double *alm, double *map,
                const double *init_alm, const double *init_map, wf_stats *st);
wf_status residual(Plan &P, const double *d, const double *alm, double *res_wf,
                   double *res_fp, double *chi2);
wf_status alm2map(Plan &P, const double *alm, double *map);
wf_status map2alm(Plan &P, const double *map, double *alm);
wf_status alm2map_f32(Plan &P, const double *alm, double *map);
wf_status map2alm_f32(Plan &P, const double *map, double *alm);
wf_status alm2map_df64(Plan &P, const double *alm, double *map);
wf_status map2alm_df64(Plan &P, const double *map, double *alm);
wf_status legendre_terms(Plan &P, int L, double *terms);
SolverState initial_state(const Plan &P);
wf_status residual_static(Plan &P, const double *d, const double *alm, double *res_wf,
                          double *res_fp, double *chi2);
// real-basis inner product of two alm (fixed-order reduction, host result)
wf_status alm_dot_host(Plan &P, const double2 *a, const double2 *b, double *res);

// group.cu: Legendre transforms of nmaps maps of this geometry at once
// (maps [nmaps][npix], alm [nmaps][nalm] complex), contracted on the
// tensor cores; free_group releases their tables
wf_status map2alm_group(Plan &P, int nmaps, const double *maps, double *alm);
wf_status alm2map_group(Plan &P, int nmaps, const double *alm, double *maps);
void free_group(Plan &P);

// pcg.cu
wf_status pcg(Plan &P, const double *d, double *alm, double *map, double tol, int stop_rule,
              int max_iter, int restart, wf_stats *stats);

// the stage-control kernel of solve.cu (launch with CONTROL_THREADS threads):
// Cauchy ratio from the per-slot partial sums partials[2 j], [2 j + 1],
// j <= nslots - 1 (passed as lmax), stage test, cooling, trace; cl may be
// NULL when the state's band_limit is 0
constexpr int CONTROL_THREADS = 256;
__global__ void __launch_bounds__(CONTROL_THREADS)
    k_control(SolverState *st, const double *__restrict__ partials, int lmax,
              const double *__restrict__ cl, TraceEntry *trace);

// helper kernels of solve.cu shared with noalloc.cu
__global__ void k_mask_data(const double *d, const double *nvar, long npix, double *out);
__global__ void k_alm_dot(const double2 *a, const double2 *b, const double *fl, int lmax,
                          double *out);
__global__ void k_alm_combine(const double2 *x, const double2 *u, const double *cm12,
                              const double *cp12, int lmax, double2 *r);
__global__ void k_pix_resid(const double *d, const double *s, const double *nvar,
                            long npix, double *r, double *y, double *out);

}  // namespace wf

// The opaque handle of the C ABI is the plan itself.
struct wf_plan_s : public wf::Plan {};
