// solve.cu -- the hybrid dual messenger iteration (Algorithm 2, Eqs. 13-15)
// driven from the device, plus the FP64 transforms and diagnostics.
//
// One iteration = four kernels on the plan's stream:
//   A  Legendre analysis of G (= FFT of the messenger field t) with the
//      truncated-spectrum filter fused: x <- f_l(xi, mu) Omega Y^T t, and the
//      per-m partial sums of ||x_new - x_old||^2 and ||x_new||^2;
//   S  Legendre synthesis x -> F (ring Fourier coefficients of s = Y x);
//   R  ring kernel: F -> s -> t = s + w (d - s) -> G, w = xi / (sigma^2 + mu);
//   C  control: Cauchy ratio, stage test, cooling xi <- max(alpha, beta xi),
//      mu = xi - alpha, the band limit of the next stage, trace, stop.
// The order follows Algorithm 2: s and t of iteration i use the xi of the
// stage that produced x_i; the cooling happens after the Cauchy test.
// Iterations are captured in a CUDA graph of `chunk` iterations; every kernel
// returns at once when the control kernel has set `done`, so the host only
// polls the state between graph launches.
#include <math.h>

#include <algorithm>
#include <vector>

#include "wf_internal.cuh"

namespace wf {

// ---------------------------------------------------------------- helpers
__global__ void k_mask_data(const double *d, const double *nvar, long npix,
                            double *out) {
  for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < npix;
       p += (long)gridDim.x * blockDim.x)
    out[p] = isinf(nvar[p]) ? 0.0 : d[p];
}

// the masked data in FP32 for the FP32 ring step
__global__ void k_data_f32(const double *d, long npix, float *out) {
  for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < npix;
       p += (long)gridDim.x * blockDim.x)
    out[p] = (float)d[p];
}

// largest l with C_l - mu Omega > 0 (the band where Sbar = Theta(S - U) is
// nonzero), -1 if none; block-wide, result valid in thread 0
__device__ int band_of(const double *cl, int lmax, double mu, double omega,
                       int *sh) {
  int best = -1;
  for (int l = threadIdx.x; l <= lmax; l += blockDim.x)
    if (cl[l] - mu * omega > 0.0) best = max(best, l);
  sh[threadIdx.x] = best;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] = max(sh[threadIdx.x], sh[threadIdx.x + s]);
    __syncthreads();
  }
  const int r = sh[0];
  __syncthreads();
  return r;
}

constexpr int CTRL_THREADS = CONTROL_THREADS;
constexpr int PLATEAU_ITERS = 256;

// mixed precision: bound on the re-anchorings of one solve
constexpr int MAX_REANCHORS = 4096;

__global__ void __launch_bounds__(CTRL_THREADS)
    k_control(SolverState *st, const double *__restrict__ partials, int lmax,
              const double *__restrict__ cl, TraceEntry *trace) {
  __shared__ double snum[CTRL_THREADS], sden[CTRL_THREADS];
  __shared__ int sh[CTRL_THREADS];
  __shared__ int advance;
  if (st->done) return;
  __shared__ double sdx[CTRL_THREADS];
  double num = 0.0, den = 0.0, dx = 0.0;
  const bool anchored = st->xa != nullptr;
  for (int m = threadIdx.x; m <= lmax; m += CTRL_THREADS) {
    num += partials[2 * m];
    den += partials[2 * m + 1];
    if (anchored) dx += partials[2 * (lmax + 1) + m];
  }
  snum[threadIdx.x] = num;
  sden[threadIdx.x] = den;
  sdx[threadIdx.x] = dx;
  __syncthreads();
  for (int s = CTRL_THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      snum[threadIdx.x] += snum[threadIdx.x + s];
      sden[threadIdx.x] += sden[threadIdx.x + s];
      sdx[threadIdx.x] += sdx[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    num = snum[0];
    den = sden[0];
    st->last_den = den;  // anchored: ||delta||^2 (the re-anchoring test)
    if (anchored) den = sdx[0];  // ||x_a + delta||^2 = ||x_i||^2
    else if (st->den_fixed > 0.0) den = st->den_fixed;
    const double c = den > 0.0 ? sqrt(num / den) : 0.0;
    const int it = ++st->iter;
    const int si = st->stage_iter;          // iterations of this stage before this one
    const double c16 = si >= 16 ? st->chist[si % 16] : -1.0;  // 16 iterations ago
    st->chist[si % 16] = c;
    st->stage_iter = si + 1;
    if (trace && it - 1 < st->trace_cap) {
      TraceEntry e;
      e.stage = st->stage;
      e.lcur = st->lcur;
      e.xi = st->xi;
      e.mu = st->mu;
      e.cauchy = c;
      trace[it - 1] = e;
    }
    int adv = 0;
    // progress tracker: an FP32 pass whose Cauchy ratio has not fallen by 1%
    // in PLATEAU_ITERS iterations sits at its arithmetic noise floor
    if (!(st->cmin > 0.0) || c < 0.99 * st->cmin) {
      st->cmin = c;
      st->since_min = 0;
    } else {
      st->since_min += 1;
    }
    const bool plateau = st->noise_guard && st->since_min >= PLATEAU_ITERS && c < 1e-3;
    const double thr = st->mu == 0.0 ? st->eps_final : st->eps_k;
    if (!isfinite(c) || !isfinite(num)) {
      st->numeric_error = 1;
      st->done = 1;
    } else if (anchored && st->window_factor > 0.0 && c < thr * st->window_factor) {
      st->done = 1;  // near the stage's decision: the anchor arithmetic decides
      st->at_window = 1;
    } else if (st->mu == 0.0) {
      // arithmetic noise floor: the Cauchy ratio has stopped falling
      st->flat = (st->prev_c > 0.0 && c >= st->prev_c) ? st->flat + 1 : 0;
      if ((st->flat >= 16 && c < 1e-4) || plateau) {
        st->done = 1;
        st->converged = 1;
        st->stagnated = 1;
      } else if (st->stop_rule == WF_STOP_ERROR) {
        if (c16 > 0.0 && st->prev_c > 0.0 && c > 0.0) {
          // contraction rate: the larger of the last ratio and the mean rate
          // over 16 iterations (a few fast modes can make a single ratio
          // small while slower modes still carry the error)
          const double r1 = c / st->prev_c;
          const double r16 = pow(c / c16, 1.0 / 16.0);
          const double r = fmin(fmax(fmax(r1, r16), st->rate_floor), 0.999999);
          const double err = c * r / (1.0 - r);
          st->err_est = err;
          if (err < st->eps_final) {
            st->done = 1;
            st->converged = 1;
          }
        } else if (c == 0.0) {
          st->err_est = 0.0;
          st->done = 1;
          st->converged = 1;
        }
      } else if (c < st->eps_final) {
        st->done = 1;
        st->converged = 1;
      }
    } else {
      if (c < st->eps_k) {
        adv = 1;
      } else if (plateau) {
        if (st->boundary_stop) {  // anchored: stalled progress -> new anchor
          st->done = 1;
          st->reanchor = 1;
        } else {
          adv = 1;  // plain FP32 pass: the stage sits at its noise floor
        }
      }
    }
    st->prev_c = c;
    st->last_c = c;
    if (adv) {
      st->xi_prev = st->xi;
      st->mu_prev = st->mu;
      st->lcur_prev = st->lcur;
      const double xi = fmax(st->alpha, st->beta * st->xi);
      st->xi = xi;
      st->mu = xi > st->alpha ? xi - st->alpha : 0.0;
      st->stage += 1;
      st->stage_iter = 0;
      st->prev_c = -1.0;
      st->flat = 0;
      st->cmin = -1.0;
      st->since_min = 0;
      st->eps_k = stage_tolerance(*st, st->mu);
      st->lcur = st->lnext;
    }
    if (adv && st->mu == 0.0 && st->handoff) {
      st->done = 1;
      st->at_final = 1;
    }
    if (adv && (st->boundary_stop || (st->anchor_eps > 0.0 && st->eps_k < st->anchor_eps))) {
      st->done = 1;
      st->at_boundary = 1;
    }
    if (!st->done && st->delta_cap2 > 0.0 && st->last_den > st->delta_cap2) {
      st->done = 1;
      st->reanchor = 1;
    }
    if (!st->done && st->iter >= st->max_iter) st->done = 1;
    advance = adv;
  }
  __syncthreads();
  if (advance) {
    // band of the stage after the new one
    const double xi2 = fmax(st->alpha, st->beta * st->xi);
    const double mu2 = xi2 > st->alpha ? xi2 - st->alpha : 0.0;
    const int b =
        st->band_limit ? band_of(cl, lmax, filter_mu(*st, mu2), st->omega, sh) : lmax;
    if (threadIdx.x == 0) st->lnext = b;
  }
}

// ---------------------------------------------------------------- reductions
// sum_lm w_m (a . b), optionally with a per-l factor fl (NULL = 1) applied to
// both; blocks stride over m, threads over l; deterministic two-level
// reduction (blocks -> out[0..gridDim), then host)
__global__ void k_alm_dot(const double2 *a, const double2 *b, const double *fl,
                          int lmax, double *out) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (int m = blockIdx.x; m <= lmax; m += gridDim.x) {
    const long base = (long)m * (2 * lmax + 1 - m) / 2;  // index of (l, m) = base + l
    const double w = m == 0 ? 1.0 : 2.0;
    for (int l = m + threadIdx.x; l <= lmax; l += blockDim.x) {
      const long i = base + l;
      const double f = fl ? fl[l] : 1.0;
      acc += w * f * f * (a[i].x * b[i].x + a[i].y * b[i].y);
    }
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = sh[0];
}

// r = cm12 * x - cp12 * u (per l), used by the App. C residual
__global__ void k_alm_combine(const double2 *x, const double2 *u, const double *cm12,
                              const double *cp12, int lmax, double2 *r) {
  const int m = blockIdx.x;
  const long base = (long)m * (2 * lmax + 1 - m) / 2;
  for (int l = m + threadIdx.x; l <= lmax; l += blockDim.x) {
    const long i = base + l;
    r[i] = make_double2(cm12[l] * x[i].x - cp12[l] * u[i].x,
                        cm12[l] * x[i].y - cp12[l] * u[i].y);
  }
}

// per-pixel: out = (d - s) / sigma^2 (0 masked); chi partial sums of
// (d - s)^2 / sigma^2; also y = d / sigma^2
__global__ void k_pix_resid(const double *d, const double *s, const double *nvar,
                            long npix, double *r, double *y, double *out) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < npix;
       p += (long)gridDim.x * blockDim.x) {
    const double v = nvar[p];
    if (isinf(v)) {
      r[p] = 0.0;
      y[p] = 0.0;
    } else {
      const double e = d[p] - s[p];
      r[p] = e / v;
      y[p] = d[p] / v;
      acc += e * e / v;
    }
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = sh[0];
}

static const int RED_BLOCKS = 256;

static wf_status host_sum(Plan &P, double *dev, int n, double *res) {
  std::vector<double> h(n);
  WF_CUDA(cudaMemcpyAsync(h.data(), dev, sizeof(double) * n, cudaMemcpyDeviceToHost,
                          P.stream));
  WF_CUDA(cudaStreamSynchronize(P.stream));
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += h[i];
  *res = s;
  return WF_OK;
}

static wf_status alm_dot(Plan &P, const double2 *a, const double2 *b,
                         const double *fl, double *res) {
  ++P.nlaunch;
  k_alm_dot<<<RED_BLOCKS, 256, 0, P.stream>>>(a, b, fl, P.lmax, P.red);
  WF_CUDA(cudaGetLastError());
  return host_sum(P, P.red, RED_BLOCKS, res);
}

wf_status alm_dot_host(Plan &P, const double2 *a, const double2 *b, double *res) {
  return alm_dot(P, a, b, nullptr, res);
}

// ---------------------------------------------------------------- transforms
wf_status alm2map(Plan &P, const double *alm, double *map) {
  const double2 *a = reinterpret_cast<const double2 *>(alm);
  WF_TRY(launch_prescale<double2>(P, a, P.xs64));
  WF_TRY(launch_legendre_synth<double2>(P, P.xs64, P.F64, nullptr, P.lmax));
  WF_TRY(launch_ring<double2>(P, RING_SYNTH, P.F64, nullptr, nullptr, map, nullptr,
                              P.lmax));
  return WF_OK;
}

wf_status map2alm(Plan &P, const double *map, double *alm) {
  WF_TRY(launch_ring<double2>(P, RING_ANALYSIS, nullptr, P.G64, map, nullptr,
                              nullptr, P.lmax));
  WF_TRY(launch_legendre_anal<double2>(P, P.G64, reinterpret_cast<double2 *>(alm),
                                       nullptr, ANA_PLAIN, P.lmax));
  return WF_OK;
}

wf_status alm2map_f32(Plan &P, const double *alm, double *map) {
  const double2 *a = reinterpret_cast<const double2 *>(alm);
  WF_TRY(launch_prescale<float2>(P, a, P.xs32));
  WF_TRY(launch_legendre_synth<float2>(P, P.xs32, P.F32, nullptr, P.lmax));
  WF_TRY(launch_ring<float2>(P, RING_SYNTH, P.F32, nullptr, nullptr, map, nullptr,
                             P.lmax));
  return WF_OK;
}

wf_status map2alm_f32(Plan &P, const double *map, double *alm) {
  WF_TRY(launch_ring<float2>(P, RING_ANALYSIS, nullptr, P.G32, map, nullptr, nullptr,
                             P.lmax));
  WF_TRY(launch_legendre_anal<float2>(P, P.G32, reinterpret_cast<double2 *>(alm),
                                      nullptr, ANA_PLAIN, P.lmax));
  return WF_OK;
}

// The double-float transforms keep their synthesis input and ring
// coefficients as double-float pairs in the plan's FP64 buffers (16 bytes
// per complex value either way).
static float4 *dd_view(double2 *p) { return reinterpret_cast<float4 *>(p); }

wf_status alm2map_df64(Plan &P, const double *alm, double *map) {
  const double2 *a = reinterpret_cast<const double2 *>(alm);
  WF_TRY(launch_prescale_dd(P, a, dd_view(P.xs64)));
  WF_TRY(launch_legendre_synth_dd(P, dd_view(P.xs64), dd_view(P.F64), nullptr, P.lmax));
  WF_TRY(launch_ring_dd(P, RING_SYNTH, dd_view(P.F64), nullptr, nullptr, map, nullptr,
                        P.lmax));
  return WF_OK;
}

wf_status map2alm_df64(Plan &P, const double *map, double *alm) {
  WF_TRY(launch_ring_dd(P, RING_ANALYSIS, nullptr, dd_view(P.G64), map, nullptr, nullptr,
                        P.lmax));
  WF_TRY(launch_legendre_anal_dd(P, dd_view(P.G64), reinterpret_cast<double2 *>(alm), nullptr,
                                 ANA_PLAIN, P.lmax));
  return WF_OK;
}

// ---------------------------------------------------------------- solve
static int band_host(const std::vector<double> &cl, double mu, double omega) {
  int b = -1;
  for (int l = 0; l < (int)cl.size(); ++l)
    if (cl[l] - mu * omega > 0.0) b = l;
  return b;
}

SolverState initial_state(const Plan &P) {
  SolverState s{};
  const wf_opts &o = P.opts;
  double cmax = 0.0;
  for (double c : P.cl) cmax = std::max(cmax, c);
  s.alpha = P.alpha;
  s.beta = o.beta;
  s.omega = P.omega;
  s.messenger = o.method == WF_METHOD_MESSENGER;
  // start: Algorithm 2, mu0 Omega = beta max C_l (or opts.mu0); Algorithm 1,
  // xi = lambda0 alpha
  const double mu0 = s.messenger ? (o.lambda0 - 1.0) * P.alpha
                     : o.mu0 < 0.0 ? o.beta * cmax / P.omega
                                   : o.mu0;
  s.mu = mu0;
  s.xi = P.alpha + mu0;
  s.eps_final = o.eps_final;
  s.eps_cap = o.eps_cap;
  s.eps_k = stage_tolerance(s, mu0);
  s.prev_c = -1.0;
  s.last_c = 0.0;
  s.err_est = 0.0;
  s.stage = 0;
  s.iter = 0;
  s.done = 0;
  s.converged = 0;
  s.numeric_error = 0;
  s.max_iter = o.max_iter;
  s.stop_rule = o.stop_rule;
  s.band_limit = o.band_limit;
  s.trace_cap = P.trace_cap;
  s.stage_iter = 0;
  s.flat = 0;
  s.stagnated = 0;
  s.handoff = 0;
  s.noise_guard = 0;
  s.boundary_stop = 0;
  s.at_boundary = 0;
  s.anchor_eps = 0.0;
  s.at_final = 0;
  s.reanchor = 0;
  s.den_fixed = 0.0;
  s.rate_floor = 0.0;
  s.cmin = -1.0;
  s.since_min = 0;
  s.delta_cap2 = 0.0;
  s.last_den = 0.0;
  if (o.band_limit) {
    s.lcur = band_host(P.cl, filter_mu(s, mu0), P.omega);
    const double xi2 = std::max(P.alpha, o.beta * s.xi);
    const double mu2 = xi2 > P.alpha ? xi2 - P.alpha : 0.0;
    s.lnext = band_host(P.cl, filter_mu(s, mu2), P.omega);
  } else {
    s.lcur = s.lnext = P.lmax;
  }
  return s;
}

template <typename T2> struct Scaled;
template <> struct Scaled<double2> {
  static double2 *get(Plan &P) { return P.xs64; }
};
template <> struct Scaled<float2> {
  static float2 *get(Plan &P) { return P.xs32; }
};

// one iteration; data = NULL runs a correction solve (d = 0) driven by the
// harmonic source `src`
template <typename T2>
static wf_status enqueue_iteration(Plan &P, T2 *F, T2 *G, const double *data,
                                   const double2 *src, int slot) {
  const bool timed = slot >= 0 && P.tev_chunk > 0;
  const int C = P.tev_chunk;
  if (timed) WF_CUDA(cudaEventRecordWithFlags(P.tev[0 * C + slot], P.stream, cudaEventRecordExternal));
  T2 *xs = Scaled<T2>::get(P);
  WF_TRY(launch_legendre_anal<T2>(P, G, P.x, P.state, ANA_FILTER, P.lmax, src, xs));
  if (timed) WF_CUDA(cudaEventRecordWithFlags(P.tev[1 * C + slot], P.stream, cudaEventRecordExternal));
  if (timed) WF_CUDA(cudaEventRecordWithFlags(P.tev[2 * C + slot], P.stream, cudaEventRecordExternal));
  WF_TRY(launch_legendre_synth<T2>(P, xs, F, P.state, P.lmax));
  if (timed) WF_CUDA(cudaEventRecordWithFlags(P.tev[3 * C + slot], P.stream, cudaEventRecordExternal));
  if (timed) WF_CUDA(cudaEventRecordWithFlags(P.tev[4 * C + slot], P.stream, cudaEventRecordExternal));
  // the FP32 loops run on the plan's masked data map, read from its FP32 copy
  const float *d32 = (sizeof(T2) == sizeof(float2) && data) ? P.dmap32 : nullptr;
  WF_TRY(launch_ring<T2>(P, RING_FUSED, F, G, data, nullptr, P.state, P.lmax, d32));
  if (timed) WF_CUDA(cudaEventRecordWithFlags(P.tev[5 * C + slot], P.stream, cudaEventRecordExternal));
  ++P.nlaunch;
  k_control<<<1, CTRL_THREADS, 0, P.stream>>>(P.state, P.partials, P.lmax, P.cl_d,
                                              P.trace);
  WF_CUDA(cudaGetLastError());
  return WF_OK;
}

// Iterations per graph launch: ~2^24 / Npix (fewer host polls for small
// maps), at least 8 (at Nside 1024 a poll every ~11 ms of work instead of
// every 2 iterations; iterations past `done` return at once).
static int auto_chunk(const Plan &P) {
  long k = (1L << 24) / std::max(1L, P.npix);
  return (int)std::max(8L, std::min(128L, k));
}

template <typename T2>
static wf_status capture_graph(Plan &P, int which, T2 *F, T2 *G, const double *data,
                               const double2 *src) {
  if (P.graph[which]) return WF_OK;
  const int chunk = P.opts.graph_chunk > 0 ? P.opts.graph_chunk : auto_chunk(P);
  cudaGraph_t g = nullptr;
  // capture on the plan's private stream (the caller's stream may be the
  // legacy default stream, which cannot be captured); launch on P.stream
  if (!P.capture_stream)
    WF_CUDA(cudaStreamCreateWithFlags(&P.capture_stream, cudaStreamNonBlocking));
  if (P.opts.timing && P.tev_chunk < chunk) {
    for (cudaEvent_t e : P.tev) cudaEventDestroy(e);
    P.tev.assign(6 * chunk, nullptr);
    for (auto &e : P.tev) WF_CUDA(cudaEventCreate(&e));
    P.tev_chunk = chunk;
  }
  if (P.opts.timing && P.tev_chunk != chunk) {
    set_error("graph capture: timing events sized for another chunk");
    return WF_ERR_STATE;
  }
  cudaStream_t user = P.stream;
  P.stream = P.capture_stream;
  cudaError_t eb = cudaStreamBeginCapture(P.stream, cudaStreamCaptureModeThreadLocal);
  if (eb != cudaSuccess) {
    P.stream = user;
    set_error(std::string("graph capture: ") + cudaGetErrorString(eb));
    return WF_ERR_CUDA;
  }
  wf_status s = WF_OK;
  const long n0 = P.nlaunch;
  for (int i = 0; i < chunk && s == WF_OK; ++i)
    s = enqueue_iteration<T2>(P, F, G, data, src, P.opts.timing ? i : -1);
  P.graph_kernels[which] = P.nlaunch - n0;  // nodes of the graph, not yet run
  P.nlaunch = n0;
  cudaError_t e = cudaStreamEndCapture(P.stream, &g);
  P.stream = user;
  if (s != WF_OK) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  if (e != cudaSuccess) {
    set_error(std::string("graph capture: ") + cudaGetErrorString(e));
    return WF_ERR_CUDA;
  }
  e = cudaGraphInstantiate(&P.graph[which], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    set_error(std::string("graph instantiate: ") + cudaGetErrorString(e));
    P.graph[which] = nullptr;
    return WF_ERR_CUDA;
  }
  P.graph_chunk[which] = chunk;
  return WF_OK;
}

// Run stages until the control kernel sets done.  tinit: initial messenger
// field (NULL = zero); data / src as in enqueue_iteration.  The state must
// have been uploaded.
template <typename T2>
static wf_status run_loop(Plan &P, int which, T2 *F, T2 *G, const double *tinit,
                          const double *data, const double2 *src, bool keep_G = false,
                          bool timed = true) {
  if (keep_G) {
    // G already holds the messenger's ring coefficients
  } else if (tinit) {
    WF_TRY(launch_ring<T2>(P, RING_ANALYSIS, nullptr, G, tinit, nullptr, nullptr,
                           P.lmax));
  } else {
    WF_CUDA(cudaMemsetAsync(G, 0, sizeof(T2) * (size_t)P.nring * (P.lmax + 1),
                            P.stream));
  }
  WF_TRY(capture_graph<T2>(P, which, F, G, data, src));
  int it0 = P.state_h->iter;
  for (;;) {
    WF_CUDA(cudaGraphLaunch(P.graph[which], P.stream));
    P.nlaunch += P.graph_kernels[which];
    WF_CUDA(cudaMemcpyAsync(P.state_h, P.state, sizeof(SolverState),
                            cudaMemcpyDeviceToHost, P.stream));
    WF_CUDA(cudaStreamSynchronize(P.stream));
    if (P.opts.timing && timed) {
      // iterations that did work in this launch: the first (iter - it0)
      const int active = std::min(P.state_h->iter - it0, P.graph_chunk[which]);
      const int C = P.tev_chunk;
      for (int i = 0; i < active; ++i) {
        for (int k = 0; k < 3; ++k) {
          float t = 0.f;
          WF_CUDA(cudaEventElapsedTime(&t, P.tev[2 * k * C + i], P.tev[(2 * k + 1) * C + i]));
          P.kern_ms[k] += t;
        }
      }
      for (int k = 0; k < 3; ++k) P.kern_launches[k] += active;
      it0 = P.state_h->iter;
    }
    if (P.state_h->done) break;
  }
  return WF_OK;
}

// r = G(x) - x (both FP64 alm) -> source of an anchored stage at (xi, mu):
// the analysis adds f_l xi Omega src, so src = r (Sbar + xi Omega) /
// (Sbar xi Omega), Sbar = max(C_l - mu Omega, 0); 0 where Sbar = 0 (there
// r = 0 as well)
__global__ void k_make_source(const double2 *gx, const double2 *x, const double *cl,
                              double xi, double mu, double omega, int lmax,
                              double2 *src) {
  const int m = blockIdx.x;
  const long base = (long)m * (2 * lmax + 1 - m) / 2;
  const double xo = xi * omega;
  for (int l = m + threadIdx.x; l <= lmax; l += blockDim.x) {
    const long i = base + l;
    const double sb = fmax(cl[l] - mu * omega, 0.0);
    const double s = sb > 0.0 ? (sb + xo) / (sb * xo) : 0.0;
    src[i] = make_double2(s * (gx[i].x - x[i].x), s * (gx[i].y - x[i].y));
  }
}

// gx = f U on l <= L (0 above), f = Sbar / (Sbar + xi Omega); partials of
// ||gx - x||^2 and ||gx||^2 per m (weights 1 for m = 0, 2 else)
__global__ void k_filter_from_u(const double2 *__restrict__ U, const double2 *__restrict__ x,
                                const double *__restrict__ cl, double xi, double mu,
                                double omega, int L, int lmax, double2 *__restrict__ gx,
                                double *__restrict__ partials) {
  __shared__ double sn[128], sd[128];
  const int m = blockIdx.x;
  const long base = (long)m * (2 * lmax + 1 - m) / 2;
  const double wm = m == 0 ? 1.0 : 2.0;
  double num = 0.0, den = 0.0;
  for (int l = m + threadIdx.x; l <= lmax; l += blockDim.x) {
    const long i = base + l;
    double2 g = make_double2(0.0, 0.0);
    if (l <= L) {
      const double sb = fmax(cl[l] - mu * omega, 0.0);
      const double f = sb / (sb + xi * omega);
      g = make_double2(f * U[i].x, f * U[i].y);
    }
    const double dr = g.x - x[i].x, di = g.y - x[i].y;
    num += wm * (dr * dr + di * di);
    den += wm * (g.x * g.x + g.y * g.y);
    gx[i] = g;
  }
  sn[threadIdx.x] = num;
  sd[threadIdx.x] = den;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sn[threadIdx.x] += sn[threadIdx.x + s];
      sd[threadIdx.x] += sd[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partials[2 * m] = sn[0];
    partials[2 * m + 1] = sd[0];
  }
}

__global__ void k_alm_add(double2 *x, const double2 *y, long n) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long)gridDim.x * blockDim.x)
    x[i] = make_double2(x[i].x + y[i].x, x[i].y + y[i].y);
}

// One FP64 iteration map of stage (xi, mu) with band L: gx = G(x); returns
// ||G(x) - x||^2 in *num.  (Defaults: the last stage, full band.)
// One iteration map of stage (xi, mu, band L) from x into gx, and the
// squared step norm.  dd: the Legendre transforms in double-float (the
// anchors of a mixed solve with opts.anchor = 1); else plain FP64.
// U (optional): also keep the unfiltered analysis Omega Y^T t up to band
// max(L, Lu) (the next stage's band) -- gx is then f U.
static wf_status fp64_step(Plan &P, const double2 *x, double2 *gx, double *num,
                           double xi, double mu, int L, bool dd = false,
                           double2 *U = nullptr, int Lu = -1, double *den = nullptr) {
  SolverState s = initial_state(P);
  s.xi = xi;
  s.mu = mu;
  s.lcur = L;
  s.lnext = U ? std::max(L, Lu) : L;
  s.done = 0;
  *P.state_h = s;
  WF_CUDA(cudaMemcpyAsync(P.state, P.state_h, sizeof(SolverState),
                          cudaMemcpyHostToDevice, P.stream));
  WF_CUDA(cudaMemcpyAsync(gx, x, sizeof(double2) * P.nalm, cudaMemcpyDeviceToDevice,
                          P.stream));
  if (dd)
    WF_TRY(launch_prescale_dd(P, x, dd_view(P.xs64)));
  else
    WF_TRY(launch_prescale<double2>(P, x, P.xs64));
  // opts.timing: events around the double-float synthesis, ring step and
  // analysis (kernels 3, 5, 4 of wf_kernel_stats)
  const bool timed = dd && P.opts.timing;
  if (timed && !P.dd_ev[0])
    for (auto &e : P.dd_ev) WF_CUDA(cudaEventCreate(&e));
  if (timed) WF_CUDA(cudaEventRecord(P.dd_ev[0], P.stream));
  if (dd)
    WF_TRY(launch_legendre_synth_dd(P, dd_view(P.xs64), dd_view(P.F64), nullptr,
                                    std::max(L, 0)));
  else
    WF_TRY(launch_legendre_synth<double2>(P, P.xs64, P.F64, nullptr, std::max(L, 0)));
  if (timed) WF_CUDA(cudaEventRecord(P.dd_ev[1], P.stream));
  if (dd)
    WF_TRY(launch_ring_dd(P, RING_FUSED, dd_view(P.F64), dd_view(P.G64), nullptr, nullptr,
                          P.state, P.lmax, P.dmapdd));
  else
    WF_TRY(launch_ring<double2>(P, RING_FUSED, P.F64, P.G64, P.dmap, nullptr, P.state,
                                P.lmax));
  if (timed) WF_CUDA(cudaEventRecord(P.dd_ev[2], P.stream));
  // band of the analysis launch: the state's lcur (= L) unless it also
  // computes the unfiltered analysis up to the next stage's band
  const int La = U ? std::max(L, Lu) : std::max(L, 0);
  if (U) {
    const int Lb = std::max(L, Lu);
    if (dd)
      WF_TRY(launch_legendre_anal_dd(P, dd_view(P.G64), U, nullptr, ANA_PLAIN, Lb));
    else
      WF_TRY(launch_legendre_anal<double2>(P, P.G64, U, nullptr, ANA_PLAIN, Lb));
    ++P.nlaunch;
    k_filter_from_u<<<P.lmax + 1, 128, 0, P.stream>>>(U, x, P.cl_d, xi, filter_mu(s, mu),
                                                      P.omega, L,
                                                      P.lmax, gx, P.partials);
    WF_CUDA(cudaGetLastError());
  } else if (dd) {
    WF_TRY(launch_legendre_anal_dd(P, dd_view(P.G64), gx, P.state, ANA_FILTER, P.lmax));
  } else {
    WF_TRY(launch_legendre_anal<double2>(P, P.G64, gx, P.state, ANA_FILTER, P.lmax));
  }
  if (timed) WF_CUDA(cudaEventRecord(P.dd_ev[3], P.stream));
  std::vector<double> part(2 * (P.lmax + 1));
  WF_CUDA(cudaMemcpyAsync(part.data(), P.partials, sizeof(double) * part.size(),
                          cudaMemcpyDeviceToHost, P.stream));
  WF_CUDA(cudaStreamSynchronize(P.stream));
  if (timed) {
    float t[3] = {0.f, 0.f, 0.f};
    for (int k = 0; k < 3; ++k)
      WF_CUDA(cudaEventElapsedTime(&t[k], P.dd_ev[k], P.dd_ev[k + 1]));
    double ts = 0.0, ta = 0.0;
    WF_TRY(legendre_terms(P, std::max(L, 0), &ts));
    WF_TRY(legendre_terms(P, La, &ta));
    P.kern_ms[3] += t[0];
    P.kern_ms[5] += t[1];
    P.kern_ms[4] += t[2];
    P.kern_flop[3] += 7.0 * ts;
    P.kern_flop[4] += 7.0 * ta;
    // ring step: F read and G written (FP64) for m <= its bands, d and sigma^2
    P.kern_flop[5] += 16.0 * P.nring * (std::max(L, 0) + La + 2.0) + 16.0 * P.npix;
    for (int k = 3; k < 6; ++k) P.kern_launches[k] += 1;
  }
  double acc = 0.0, acd = 0.0;
  for (int m = 0; m <= P.lmax; ++m) {
    acc += part[2 * m];
    acd += part[2 * m + 1];
  }
  *num = acc;
  if (den) *den = acd;
  return WF_OK;
}
static wf_status fp64_step(Plan &P, const double2 *x, double2 *gx, double *num) {
  return fp64_step(P, x, gx, num, P.alpha, 0.0, P.lmax);
}

// reduced term count of one Legendre transform at band L (cached per L)
wf_status legendre_terms(Plan &P, int L, double *terms) {
  if (P.seed_l_h.empty()) {
    P.seed_l_h.resize((size_t)P.npairs * (P.lmax + 1));
    WF_CUDA(cudaMemcpy(P.seed_l_h.data(), P.seed_l, sizeof(int) * P.seed_l_h.size(),
                       cudaMemcpyDeviceToHost));
    P.work_cache.assign(P.lmax + 1, -1.0);
  }
  if (P.work_cache[L] < 0.0) {
    double w = 0.0;
    for (int m = 0; m <= L; ++m)
      for (int k = 0; k < P.npairs; ++k) {
        const int ls = P.seed_l_h[(size_t)m * P.npairs + k];
        if (ls <= L) w += (double)(L - ls + 1);
      }
    P.work_cache[L] = w;
  }
  *terms = P.work_cache[L];
  return WF_OK;
}

// add the algorithmic work of the timed launches of iterations [i0, i1)
static wf_status account_work(Plan &P, int i0, int i1) {
  i1 = std::min(i1, P.trace_cap);
  if (i1 <= i0) return WF_OK;
  std::vector<TraceEntry> h(i1 - i0);
  WF_CUDA(cudaMemcpy(h.data(), P.trace + i0, sizeof(TraceEntry) * h.size(),
                     cudaMemcpyDeviceToHost));
  // ring step: F read and G written for m <= lcur on every ring (T2 each),
  // sigma^2 read once per pixel, and d in the iterations that read it
  // (FP64: 8 bytes each; FP32 step: 4)
  const bool f64 = P.opts.precision == WF_PREC_FP64;
  const double t2 = f64 ? 16.0 : 8.0, pb = f64 ? 8.0 : 4.0;
  for (int i = i0; i < i1; ++i) {
    const TraceEntry &e = h[i - i0];
    if (e.lcur < 0) continue;
    if (std::find(P.untimed.begin(), P.untimed.end(), i) != P.untimed.end()) continue;
    double t = 0.0;
    WF_TRY(legendre_terms(P, e.lcur, &t));
    P.kern_flop[0] += 7.0 * t;
    P.kern_flop[1] += 7.0 * t;
    P.kern_flop[2] += 2.0 * t2 * P.nring * (e.lcur + 1.0) +
                      (i < P.data_iters ? 2.0 : 1.0) * pb * P.npix;
  }
  return WF_OK;
}

// Contraction rate of the slow modes, fitted to the Cauchy ratios of the
// iterations [i0, i1) of the trace: the geometric decay rate over the last
// stretch where c is still far (30x) above its final value (the FP32 noise
// floor, where the ratio tends to 1 and says nothing about convergence).
static wf_status slow_rate(Plan &P, int i0, int i1, double *rate) {
  *rate = 0.0;
  i1 = std::min(i1, P.trace_cap);
  if (i1 - i0 < 8) return WF_OK;
  std::vector<TraceEntry> h(i1 - i0);
  WF_CUDA(cudaMemcpy(h.data(), P.trace + i0, sizeof(TraceEntry) * h.size(),
                     cudaMemcpyDeviceToHost));
  const int n = (int)h.size();
  const double cfin = h[n - 1].cauchy;
  int j = n - 1;
  while (j > 0 && !(h[j].cauchy > 30.0 * cfin)) --j;
  const int span = std::max(8, j / 5);
  const int i = std::max(0, j - span);
  if (j - i < 4 || !(h[i].cauchy > 0.0) || !(h[j].cauchy > 0.0)) return WF_OK;
  const double r = pow(h[j].cauchy / h[i].cauchy, 1.0 / (double)(j - i));
  if (r > 0.0 && r < 1.0) *rate = r;
  return WF_OK;
}

// First iterate of a new stage (h: the state just after the advance, with
// the old stage in xi_prev, mu_prev, lcur_prev), as Algorithm 2 takes it:
// t from the last iterate x = P.xacc with the old stage's weights, then
// x_first = f_new Omega Y^T t on the new band -- in the anchor arithmetic
// (the FP32 correction messenger, grown over the whole old stage, would
// bring an error of the size of a step).  Updates P.xacc, the iteration
// count and the trace; advances again (on the host, as k_control does) in
// the rare case that this step already passes the new stage's test.
static wf_status boundary_step(Plan &P, SolverState &hio, int *total_iter) {
  SolverState h = hio;  // hio may be the host mirror, which fp64_step overwrites
  for (;;) {
    double num = 0.0;
    WF_TRY(fp64_step(P, P.xacc, P.xtmp, &num, h.xi_prev, h.mu_prev, h.lcur_prev,
                     P.opts.anchor == 1, P.uacc[0], h.lcur));
    ++P.nlaunch;
    k_filter_from_u<<<P.lmax + 1, 128, 0, P.stream>>>(P.uacc[0], P.xacc, P.cl_d, h.xi,
                                                      filter_mu(h, h.mu),
                                                      P.omega, h.lcur, P.lmax, P.xtmp,
                                                      P.partials);
    WF_CUDA(cudaGetLastError());
    std::vector<double> part(2 * (P.lmax + 1));
    WF_CUDA(cudaMemcpyAsync(part.data(), P.partials, sizeof(double) * part.size(),
                            cudaMemcpyDeviceToHost, P.stream));
    WF_CUDA(cudaMemcpyAsync(P.xacc, P.xtmp, sizeof(double2) * P.nalm,
                            cudaMemcpyDeviceToDevice, P.stream));
    WF_CUDA(cudaStreamSynchronize(P.stream));
    double nu = 0.0, de = 0.0;
    for (int m = 0; m <= P.lmax; ++m) {
      nu += part[2 * m];
      de += part[2 * m + 1];
    }
    const double c = de > 0.0 ? sqrt(nu / de) : 0.0;
    const int it = (*total_iter)++;
    P.untimed.push_back(it);
    if (it < P.trace_cap) {
      TraceEntry e;
      e.stage = h.stage;
      e.lcur = h.lcur;
      e.xi = h.xi;
      e.mu = h.mu;
      e.cauchy = c;
      WF_CUDA(cudaMemcpy(P.trace + it, &e, sizeof(e), cudaMemcpyHostToDevice));
    }
    h.iter = *total_iter;
    h.last_c = c;
    if (!(h.mu > 0.0 && c < h.eps_k)) {
      hio = h;
      return WF_OK;
    }
    // the new stage's test passed at once: the next stage
    h.xi_prev = h.xi;
    h.mu_prev = h.mu;
    h.lcur_prev = h.lcur;
    h.xi = std::max(P.alpha, h.beta * h.xi);
    h.mu = h.xi > P.alpha ? h.xi - P.alpha : 0.0;
    h.stage += 1;
    h.eps_k = stage_tolerance(h, h.mu);
    h.lcur = h.lnext;
    const double xi2 = std::max(P.alpha, h.beta * h.xi);
    const double mu2 = xi2 > P.alpha ? xi2 - P.alpha : 0.0;
    h.lnext = P.opts.band_limit ? band_host(P.cl, filter_mu(h, mu2), P.omega) : P.lmax;
  }
}

// Iterations x <- G(x) of a tail stage (mu <= alpha) in the anchor
// arithmetic, from P.xacc, with the Cauchy test of k_control.  Returns with
// *last_done set when the last stage (mu = 0) passes its test, or with hio
// advanced to the next stage (not yet entered: its first iterate is the
// boundary step), or when max_iter is reached.
static wf_status tail_stage(Plan &P, SolverState &hio, int *total_iter, bool *last_done) {
  SolverState h = hio;  // hio may be the host mirror, which fp64_step overwrites
  const bool dd = P.opts.anchor == 1;
  *last_done = false;
  while (*total_iter < P.opts.max_iter) {
    double nu = 0.0, de = 0.0;
    WF_TRY(fp64_step(P, P.xacc, P.xtmp, &nu, h.xi, h.mu, h.lcur, dd, nullptr, -1, &de));
    WF_CUDA(cudaMemcpyAsync(P.xacc, P.xtmp, sizeof(double2) * P.nalm,
                            cudaMemcpyDeviceToDevice, P.stream));
    const double c = de > 0.0 ? sqrt(nu / de) : 0.0;
    const int it = (*total_iter)++;
    P.untimed.push_back(it);
    if (it < P.trace_cap) {
      TraceEntry e;
      e.stage = h.stage;
      e.lcur = h.lcur;
      e.xi = h.xi;
      e.mu = h.mu;
      e.cauchy = c;
      WF_CUDA(cudaMemcpy(P.trace + it, &e, sizeof(e), cudaMemcpyHostToDevice));
    }
    h.iter = *total_iter;
    h.last_c = c;
    if (!std::isfinite(c)) {
      set_error("wf_solve: NaN or Inf in a tail stage");
      return WF_ERR_NUMERIC;
    }
    if (h.mu == 0.0) {
      if (c < h.eps_final) {
        *last_done = true;
        break;
      }
    } else if (c < h.eps_k) {
      h.xi_prev = h.xi;
      h.mu_prev = h.mu;
      h.lcur_prev = h.lcur;
      h.xi = std::max(P.alpha, h.beta * h.xi);
      h.mu = h.xi > P.alpha ? h.xi - P.alpha : 0.0;
      h.stage += 1;
      h.eps_k = stage_tolerance(h, h.mu);
      h.lcur = h.lnext;
      const double xi2 = std::max(P.alpha, h.beta * h.xi);
      const double mu2 = xi2 > P.alpha ? xi2 - P.alpha : 0.0;
      h.lnext = P.opts.band_limit ? band_host(P.cl, filter_mu(h, mu2), P.omega) : P.lmax;
      break;
    }
  }
  hio = h;
  return WF_OK;
}

wf_status solve(Plan &P, const double *d, double *alm, double *map,
                const double *init_alm, const double *init_map, wf_stats *stats) {
  if (!P.has_noise) {
    set_error("wf_solve: plan has no noise variance");
    return WF_ERR_STATE;
  }
  WF_CUDA(cudaEventRecord(P.ev0, P.stream));
  P.untimed.clear();
  const long launches0 = P.nlaunch;
  ++P.nlaunch;
  k_mask_data<<<304, 256, 0, P.stream>>>(d, P.nvar, P.npix, P.dmap);
  WF_CUDA(cudaGetLastError());
  WF_TRY(launch_to_dd(P, P.dmap, P.dmapdd, P.npix));  // the double-float ring steps' d
  if (init_alm)
    WF_CUDA(cudaMemcpyAsync(P.x, init_alm, sizeof(double2) * P.nalm,
                            cudaMemcpyDeviceToDevice, P.stream));
  else
    WF_CUDA(cudaMemsetAsync(P.x, 0, sizeof(double2) * P.nalm, P.stream));
  const double *tinit = P.dmap;
  if (init_map) {
    ++P.nlaunch;
    k_mask_data<<<304, 256, 0, P.stream>>>(init_map, P.nvar, P.npix, P.mtmp);
    WF_CUDA(cudaGetLastError());
    tinit = P.mtmp;
  }
  int refinements = 0, total_iter = 0, first_stages = 0;
  double fp_res = -1.0;
  *P.state_h = initial_state(P);
  if (P.opts.precision == WF_PREC_MIXED) {
    // Mixed precision.  Stages with a loose tolerance (>= opts.anchor_eps) run
    // Algorithm 2 with FP32 transforms on x itself.  Every later stage runs
    // anchored: with x_a the iterate at the anchor and r = G64(x_a) - x_a
    // (one FP64 iteration map of the stage), iterate
    //   delta <- J32 delta + r,   x = x_a + delta,
    // which is the same iteration x <- G(x) written as a correction, so the
    // FP32 transform error scales with |delta| instead of |x|.  A new anchor
    // is taken at each stage change, when |delta| exceeds opts.anchor_cap |x_a|,
    // and when progress stalls.
    bool converged = false;
    SolverState &h = *P.state_h;
    ++P.nlaunch;
    k_data_f32<<<304, 256, 0, P.stream>>>(P.dmap, P.npix, P.dmap32);
    WF_CUDA(cudaGetLastError());
    h.noise_guard = 1;
    h.anchor_eps = P.opts.anchor_eps;
    // every stage anchored: one plain FP64 step from t0 = d gives the first
    // anchor (untimed: the kernel statistics cover the FP32 kernels)
    const bool first64 = h.eps_k < P.opts.anchor_eps;
    if (first64) h.max_iter = 1;
    WF_CUDA(cudaMemcpyAsync(P.state, P.state_h, sizeof(SolverState),
                            cudaMemcpyHostToDevice, P.stream));
    if (first64) {
      P.untimed.push_back(0);
      WF_TRY(run_loop<double2>(P, 0, P.F64, P.G64, tinit, P.dmap, nullptr, false, false));
    } else {
      WF_TRY(run_loop<float2>(P, 1, P.F32, P.G32, tinit, P.dmap, nullptr));
    }
    if (h.numeric_error) {
      set_error("wf_solve: NaN or Inf in the iteration");
      return WF_ERR_NUMERIC;
    }
    total_iter = h.iter;
    P.data_iters = total_iter;
    bool anchored = h.at_boundary || h.max_iter == 1;
    if (h.max_iter == 1 && !h.at_boundary) {
      // the single plain step did not advance: stay in the initial stage
      const SolverState keep = h;
      h = initial_state(P);
      h.iter = keep.iter;
    }
    WF_CUDA(cudaMemcpyAsync(P.xacc, P.x, sizeof(double2) * P.nalm,
                            cudaMemcpyDeviceToDevice, P.stream));
    double prev_rel = -1.0, rate_floor = 0.0;
    int cycles = 0, reanchors = 0, cycle_start = total_iter;
    if (!P.uacc[0]) WF_CUDA(cudaMalloc(&P.uacc[0], sizeof(double2) * P.nalm));
    // At a stage boundary Algorithm 2 carries the messenger t, not x, across
    // the cooling step: the new stage's first iterate is f_new Omega Y^T t
    // with t from the last iterate and the old stage's weights.  That step is
    // taken here in the anchor arithmetic (boundary_step), from the
    // accumulated iterate x_a + delta; the new stage then anchors at it.
    bool boundary = h.at_boundary != 0;
    bool tail_dd = false;  // the tail stage's decision is being taken in the anchor arithmetic
    while (anchored && reanchors <= MAX_REANCHORS && cycles <= P.opts.refine_max) {
      if (boundary) {
        WF_TRY(boundary_step(P, h, &total_iter));
        boundary = false;
        tail_dd = false;
      }
      const bool tail = P.opts.tail_exact && h.eps_k <= P.opts.eps_final &&
                        P.opts.stop_rule == WF_STOP_CAUCHY;
      if (tail && (tail_dd || !(P.opts.tail_window > 0.0))) {
        // the tail stages (each one's tolerance is eps_final)
        // iterate in the anchor arithmetic, so that their Cauchy tests see
        // the step to FP64 accuracy
        bool last_done = false;
        WF_TRY(tail_stage(P, h, &total_iter, &last_done));
        if (!last_done) {
          if (total_iter >= P.opts.max_iter) break;
          boundary = true;  // the next stage starts with its boundary step
          continue;
        }
        // accept when the plain FP64 step from the result passes the test
        const SolverState keep = h;
        double num = 0.0, xn2 = 0.0;
        WF_TRY(fp64_step(P, P.xacc, P.xtmp, &num, keep.xi, keep.mu, keep.lcur));
        WF_TRY(alm_dot(P, P.xacc, P.xacc, nullptr, &xn2));
        const double c64 = xn2 > 0.0 ? sqrt(num / xn2) : 0.0;
        h = keep;
        h.iter = total_iter;
        if (c64 < P.opts.eps_final) {
          converged = true;
          fp_res = c64;
          break;
        }
        ++reanchors;
        continue;
      }
      const SolverState stage = h;  // stage parameters of this anchor
      double num = 0.0, xn = 0.0;
      WF_TRY(fp64_step(P, P.xacc, P.xtmp, &num, stage.xi, stage.mu, stage.lcur,
                       P.opts.anchor == 1));
      WF_TRY(alm_dot(P, P.xacc, P.xacc, nullptr, &xn));
      ++P.nlaunch;
      k_make_source<<<P.lmax + 1, 128, 0, P.stream>>>(P.xtmp, P.xacc, P.cl_d, stage.xi,
                                                      filter_mu(stage, stage.mu), P.omega,
                                                      P.lmax, P.src);
      WF_CUDA(cudaGetLastError());
      WF_CUDA(cudaMemsetAsync(P.x, 0, sizeof(double2) * P.nalm, P.stream));
      SolverState s = initial_state(P);
      s.xi = stage.xi;
      s.mu = stage.mu;
      s.stage = stage.stage;
      s.eps_k = stage.eps_k;
      s.lcur = stage.lcur;
      s.lnext = stage.lnext;
      s.iter = total_iter;
      s.max_iter = P.opts.max_iter;
      s.xa = P.xacc;  // Cauchy ratios of the iterate x_a + delta
      // re-anchoring bound on ||delta|| / ||x_a||: anchor_cap, tightened to
      // anchor_cap_tol times the stage tolerance (the FP32 error of a step
      // scales with ||delta||, and late stages take steps of ~eps_k ||x||)
      double cap = P.opts.anchor_cap;
      if (P.opts.anchor_cap_tol > 0.0) cap = std::min(cap, P.opts.anchor_cap_tol * stage.eps_k);
      if (tail && P.opts.tail_cap_tol > 0.0)
        cap = std::min(cap, P.opts.tail_cap_tol * stage.eps_k);
      s.delta_cap2 = cap * cap * xn;
      s.rate_floor = stage.mu == 0.0 ? rate_floor : 0.0;
      s.noise_guard = 1;
      s.boundary_stop = 1;
      // a tail stage runs FP32 corrections until its Cauchy ratio is within
      // tail_window of the threshold; the anchor arithmetic takes the decision
      s.window_factor = tail ? 1.0 + P.opts.tail_window : 0.0;
      h = s;
      WF_CUDA(cudaMemcpyAsync(P.state, P.state_h, sizeof(SolverState),
                              cudaMemcpyHostToDevice, P.stream));
      WF_TRY(run_loop<float2>(P, 2, P.F32, P.G32, nullptr, nullptr, P.src));
      total_iter = h.iter;
      if (h.numeric_error) {
        set_error("wf_solve: NaN or Inf in an anchored stage");
        return WF_ERR_NUMERIC;
      }
      double dn = 0.0;
      WF_TRY(alm_dot(P, P.x, P.x, nullptr, &dn));
      ++P.nlaunch;
      k_alm_add<<<304, 256, 0, P.stream>>>(P.xacc, P.x, P.nalm);
      WF_CUDA(cudaGetLastError());
      ++refinements;
      if (h.at_window) {  // same stage: iterate it in the anchor arithmetic
        h.at_window = 0;
        tail_dd = true;
        continue;
      }
      boundary = h.at_boundary != 0;
      if (h.at_boundary) continue;  // next stage: h holds its parameters
      if (h.reanchor || (h.stagnated && h.mu == 0.0)) {
        ++reanchors;  // same stage, new anchor
        h.stagnated = 0;
        h.converged = 0;
        continue;
      }
      if (!h.converged) break;  // max_iter
      if (P.opts.stop_rule == WF_STOP_CAUCHY) {
        // accept when the FP64 step from the result passes the same test:
        // ||G64(x) - x|| / ||x|| < eps_final (else re-anchor and go on)
        double num = 0.0, xn2 = 0.0;
        WF_TRY(fp64_step(P, P.xacc, P.xtmp, &num, stage.xi, stage.mu, stage.lcur));
        WF_TRY(alm_dot(P, P.xacc, P.xacc, nullptr, &xn2));
        const double c64 = xn2 > 0.0 ? sqrt(num / xn2) : 0.0;
        h = stage;
        h.iter = total_iter;
        if (c64 < P.opts.eps_final) {
          converged = true;
          fp_res = c64;  // the accepted step is the reported residual
          break;
        }
        ++reanchors;
        continue;
      }
      // error-estimate rule: confirm with further cycles (see the header)
      ++cycles;
      {
        double r = 0.0;
        WF_TRY(slow_rate(P, cycle_start, total_iter, &r));
        rate_floor = std::max(rate_floor, r);
      }
      cycle_start = total_iter;
      const double rel = xn > 0.0 ? sqrt(dn / xn) : 0.0;
      if (rel < P.opts.eps_final ||
          (prev_rel > 0.0 && rel * (rel / prev_rel) < P.opts.eps_final / 3.0)) {
        converged = true;
        break;
      }
      prev_rel = rel;
      h.converged = 0;
    }
    if (!anchored) converged = h.converged;  // finished inside the data pass
    first_stages = h.stage + 1;
    if (!(converged && P.opts.stop_rule == WF_STOP_CAUCHY)) {
      const SolverState keep = h;
      double num = 0.0, xn = 0.0;
      WF_TRY(fp64_step(P, P.xacc, P.xtmp, &num));
      WF_TRY(alm_dot(P, P.xacc, P.xacc, nullptr, &xn));
      fp_res = xn > 0.0 ? sqrt(num / xn) : 0.0;
      h = keep;
    }
    WF_CUDA(cudaMemcpyAsync(P.x, P.xacc, sizeof(double2) * P.nalm,
                            cudaMemcpyDeviceToDevice, P.stream));
    h.converged = converged ? 1 : 0;
  } else {
    WF_CUDA(cudaMemcpyAsync(P.state, P.state_h, sizeof(SolverState),
                            cudaMemcpyHostToDevice, P.stream));
    WF_TRY(run_loop<double2>(P, 0, P.F64, P.G64, tinit, P.dmap, nullptr));
    total_iter = P.state_h->iter;
    P.data_iters = total_iter;
    first_stages = P.state_h->stage + 1;
  }
  if (map) WF_TRY(alm2map(P, reinterpret_cast<const double *>(P.x), map));
  if (alm)
    WF_CUDA(cudaMemcpyAsync(alm, P.x, sizeof(double2) * P.nalm,
                            cudaMemcpyDeviceToDevice, P.stream));
  WF_CUDA(cudaEventRecord(P.ev1, P.stream));
  WF_CUDA(cudaStreamSynchronize(P.stream));
  const SolverState &s = *P.state_h;
  P.trace_len = std::min(total_iter, P.trace_cap);
  if (P.opts.timing) WF_TRY(account_work(P, 0, total_iter));
  if (stats) {
    float ms = 0.f;
    WF_CUDA(cudaEventElapsedTime(&ms, P.ev0, P.ev1));
    stats->iterations = total_iter;
    stats->stages = first_stages;
    stats->converged = s.converged;
    stats->refinements = refinements;
    stats->alpha = P.alpha;
    stats->final_cauchy = s.last_c;
    stats->err_estimate = s.err_est;
    stats->fp_residual = fp_res;
    stats->elapsed_ms = ms;
    stats->kernel_launches = P.nlaunch - launches0;
  }
  if (s.numeric_error) {
    set_error("wf_solve: NaN or Inf in the iteration");
    return WF_ERR_NUMERIC;
  }
  if (!s.converged) {
    set_error("wf_solve: max_iter reached before the last stage converged");
    return WF_ERR_NOT_CONVERGED;
  }
  return WF_OK;
}

// ---------------------------------------------------------------- residual
wf_status residual(Plan &P, const double *d, const double *alm, double *res_wf,
                   double *res_fp, double *chi2) {
  if (!P.has_noise) {
    set_error("wf_residual: plan has no noise variance");
    return WF_ERR_STATE;
  }
  const double2 *x = reinterpret_cast<const double2 *>(alm);
  const long npix = P.npix;
  // buffers: s (mtmp), r = N^-1 (d - s) and y = N^-1 d (two pixel maps)
  double *pr = nullptr, *py = nullptr, *cm12 = nullptr, *cp12 = nullptr;
  double2 *u = nullptr, *v = nullptr, *rr = nullptr;
  WF_CUDA(cudaMalloc(&pr, sizeof(double) * npix));
  WF_CUDA(cudaMalloc(&py, sizeof(double) * npix));
  WF_CUDA(cudaMalloc(&u, sizeof(double2) * P.nalm));
  WF_CUDA(cudaMalloc(&v, sizeof(double2) * P.nalm));
  WF_CUDA(cudaMalloc(&rr, sizeof(double2) * P.nalm));
  WF_CUDA(cudaMalloc(&cm12, sizeof(double) * (P.lmax + 1)));
  WF_CUDA(cudaMalloc(&cp12, sizeof(double) * (P.lmax + 1)));
  wf_status status = WF_OK;
  do {
    ++P.nlaunch;
    k_mask_data<<<304, 256, 0, P.stream>>>(d, P.nvar, npix, P.dmap);
    if ((status = alm2map(P, alm, P.mtmp)) != WF_OK) break;
    ++P.nlaunch;
    k_pix_resid<<<RED_BLOCKS, 256, 0, P.stream>>>(P.dmap, P.mtmp, P.nvar, npix, pr,
                                                  py, P.red);
    double chi_pix = 0.0;
    if ((status = host_sum(P, P.red, RED_BLOCKS, &chi_pix)) != WF_OK) break;
    std::vector<double> hm(P.lmax + 1), hp(P.lmax + 1), hinv(P.lmax + 1);
    for (int l = 0; l <= P.lmax; ++l) {
      const double c = P.cl[l];
      hp[l] = sqrt(c);
      hm[l] = c > 0 ? 1.0 / sqrt(c) : 0.0;
      hinv[l] = c > 0 ? 1.0 / sqrt(c) : 0.0;  // for x^T C^-1 x via f^2
    }
    cudaMemcpyAsync(cm12, hm.data(), sizeof(double) * (P.lmax + 1),
                    cudaMemcpyHostToDevice, P.stream);
    cudaMemcpyAsync(cp12, hp.data(), sizeof(double) * (P.lmax + 1),
                    cudaMemcpyHostToDevice, P.stream);
    double prior = 0.0;
    if ((status = alm_dot(P, x, x, cm12, &prior)) != WF_OK) break;
    if (chi2) *chi2 = chi_pix + prior;
    // u = Y^T N^-1 (d - s), v = Y^T N^-1 d  (map2alm gives Omega Y^T)
    if ((status = map2alm(P, pr, reinterpret_cast<double *>(u))) != WF_OK) break;
    if ((status = map2alm(P, py, reinterpret_cast<double *>(v))) != WF_OK) break;
    // App. C: r = C^-1/2 x - C^1/2 Y^T N^-1 (d - s);  y = C^1/2 Y^T N^-1 d
    // with the Omega of map2alm divided out
    std::vector<double> hp_om(P.lmax + 1);
    for (int l = 0; l <= P.lmax; ++l) hp_om[l] = hp[l] / P.omega;
    cudaMemcpyAsync(cp12, hp_om.data(), sizeof(double) * (P.lmax + 1),
                    cudaMemcpyHostToDevice, P.stream);
    ++P.nlaunch;
    k_alm_combine<<<P.lmax + 1, 128, 0, P.stream>>>(x, u, cm12, cp12, P.lmax, rr);
    double rn = 0.0, yn = 0.0;
    if ((status = alm_dot(P, rr, rr, nullptr, &rn)) != WF_OK) break;
    if ((status = alm_dot(P, v, v, cp12, &yn)) != WF_OK) break;
    if (res_wf) *res_wf = yn > 0 ? sqrt(rn / yn) : 0.0;
    if (res_fp) {
      // one last-stage iteration G(x): xi = alpha, mu = 0, full band
      SolverState s = initial_state(P);
      s.xi = P.alpha;
      s.mu = 0.0;
      s.lcur = s.lnext = P.lmax;
      s.done = 0;
      *P.state_h = s;
      cudaMemcpyAsync(P.state, P.state_h, sizeof(SolverState), cudaMemcpyHostToDevice,
                      P.stream);
      cudaMemcpyAsync(P.xtmp, x, sizeof(double2) * P.nalm, cudaMemcpyDeviceToDevice,
                      P.stream);
      if ((status = launch_prescale<double2>(P, x, P.xs64)) != WF_OK) break;
      if ((status = launch_legendre_synth<double2>(P, P.xs64, P.F64, nullptr, P.lmax)) !=
          WF_OK)
        break;
      if ((status = launch_ring<double2>(P, RING_FUSED, P.F64, P.G64, P.dmap, nullptr,
                                         P.state, P.lmax)) != WF_OK)
        break;
      if ((status = launch_legendre_anal<double2>(P, P.G64, P.xtmp, P.state,
                                                  ANA_FILTER, P.lmax)) != WF_OK)
        break;
      std::vector<double> part(2 * (P.lmax + 1));
      cudaMemcpyAsync(part.data(), P.partials, sizeof(double) * part.size(),
                      cudaMemcpyDeviceToHost, P.stream);
      double xn = 0.0;
      if ((status = alm_dot(P, x, x, nullptr, &xn)) != WF_OK) break;
      double num = 0.0;
      for (int m = 0; m <= P.lmax; ++m) num += part[2 * m];
      *res_fp = xn > 0 ? sqrt(num / xn) : 0.0;
    }
  } while (0);
  cudaError_t e = cudaStreamSynchronize(P.stream);
  cudaFree(pr);
  cudaFree(py);
  cudaFree(u);
  cudaFree(v);
  cudaFree(rr);
  cudaFree(cm12);
  cudaFree(cp12);
  if (status == WF_OK && e != cudaSuccess) {
    set_error(std::string("wf_residual: ") + cudaGetErrorString(e));
    return WF_ERR_CUDA;
  }
  return status;
}

}  // namespace wf
