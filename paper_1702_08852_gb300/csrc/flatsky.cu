// flatsky.cu -- the dual messenger on the flat sky (Algorithm 2 on the
// paper's own Sect. 3 set-up: an n x n periodic grid, 2-D FFTs), FP64.
//
// The basis change is the 2-D DFT, which is orthogonal, so the last stage's
// fixed point is the Wiener filter of Eq. (2) itself.  With the DFT in numpy's
// convention (t_hat = fft2(t), s = ifft2(t_hat)) one iteration is
//   s     = ifft2(f_k fft2(t)),  f_k = Sbar_k / (Sbar_k + xi Omega_pix),
//           Sbar_k = max(C_k - mu Omega_pix, 0)            (signal step)
//   t     = s + xi / (sigma^2 + mu) (d - s)                (Eq. 14, Nbar)
// with the Cauchy ratio ||s_i - s_{i-1}|| / ||s_i|| taken on the spectra
// (Parseval) and the cooling of Algorithm 2 (k_control of solve.cu).
//
// Kernels, two per iteration (plus k_control), the spectrum kept row-
// transformed between them:
//   k_flat_cols  CB columns per CTA: forward column FFTs of the row-
//                transformed messenger, the filter, the Cauchy partial sums
//                against the last filtered spectrum, inverse column FFTs;
//   k_flat_rows  one row per CTA: inverse row FFT -> s, the pixel update ->
//                t, forward row FFT for the next iteration.
// Rows and columns are radix-2 FFTs in shared memory (n a power of two).
#include <math.h>

#include <algorithm>
#include <string>
#include <vector>

#include "wf_internal.cuh"

namespace wf {

constexpr int FLAT_THREADS = 256;
constexpr int FLAT_CB = 4;          // columns per CTA of the column kernel
constexpr int FLAT_NMAX = 2048;     // CB columns of FP64 complex in shared memory
enum FlatMode { FLAT_FWD = 0, FLAT_ITER = 1, FLAT_FINAL = 2 };

// In-place radix-2 FFTs of `cnt` sequences of length n = 2^logn stored one
// after the other in shared memory, by the whole CTA.  tw[k] = e^{-2 pi i k
// / n}, k < n / 2; inv: the conjugate twiddles (no scaling).
__device__ void flat_fft(double2 *buf, int n, int logn, int cnt,
                         const double2 *__restrict__ tw, bool inv) {
  const int tid = threadIdx.x, nt = blockDim.x;
  // bit-reversal permutation
  for (int e = tid; e < cnt * n; e += nt) {
    const int c = e >> logn, i = e & (n - 1);
    const int j = (int)(__brev((unsigned)i) >> (32 - logn));
    if (i < j) {
      const double2 a = buf[c * n + i];
      buf[c * n + i] = buf[c * n + j];
      buf[c * n + j] = a;
    }
  }
  __syncthreads();
  const int hn = n >> 1;
  for (int half = 1, ls = 0; half < n; half <<= 1, ++ls) {
    const int tstride = hn >> ls;  // n / (2 half)
    for (int b = tid; b < cnt * hn; b += nt) {
      const int c = b / hn, j = b - c * hn;
      const int grp = j >> ls, pos = j & (half - 1);
      const int i1 = c * n + grp * 2 * half + pos, i2 = i1 + half;
      double2 w = tw[pos * tstride];
      if (inv) w.y = -w.y;
      const double2 x = buf[i1], y = buf[i2];
      const double2 wy = make_double2(w.x * y.x - w.y * y.y, w.x * y.y + w.y * y.x);
      buf[i1] = make_double2(x.x + wy.x, x.y + wy.y);
      buf[i2] = make_double2(x.x - wy.x, x.y - wy.y);
    }
    __syncthreads();
  }
}

// Columns kx0 .. kx0 + FLAT_CB - 1 (a tile of n rows).  FLAT_ITER: forward
// FFT of T1's columns, filter (state's xi, mu), partial sums of
// |s_hat - S|^2 and |s_hat|^2 into partials[2 b], [2 b + 1], S <- s_hat,
// inverse FFT -> T2.  FLAT_FINAL: inverse FFT of S's columns -> T2.
__global__ void __launch_bounds__(FLAT_THREADS)
    k_flat_cols(int n, int logn, double omega, const double *__restrict__ ck,
                const double2 *__restrict__ T1, double2 *__restrict__ S,
                double2 *__restrict__ T2, const double2 *__restrict__ tw,
                const SolverState *__restrict__ st, double *__restrict__ partials, int mode) {
  extern __shared__ __align__(16) unsigned char flat_smem[];
  double2 *buf = reinterpret_cast<double2 *>(flat_smem);  // [FLAT_CB][n]
  __shared__ double red[2][FLAT_THREADS];
  if (mode == FLAT_ITER && st->done) return;
  const int kx0 = blockIdx.x * FLAT_CB, tid = threadIdx.x;
  const double2 *src = mode == FLAT_ITER ? T1 : S;
  for (int e = tid; e < FLAT_CB * n; e += FLAT_THREADS) {
    const int y = e / FLAT_CB, c = e - y * FLAT_CB;  // consecutive threads: one row
    buf[c * n + y] = src[(long)y * n + kx0 + c];
  }
  __syncthreads();
  double num = 0.0, den = 0.0;
  if (mode == FLAT_ITER) {
    flat_fft(buf, n, logn, FLAT_CB, tw, false);
    const double xi = st->xi, mu = st->mu;
    for (int e = tid; e < FLAT_CB * n; e += FLAT_THREADS) {
      const int ky = e / FLAT_CB, c = e - ky * FLAT_CB;
      const long k = (long)ky * n + kx0 + c;
      const double sbar = fmax(ck[k] - mu * omega, 0.0);
      const double f = sbar > 0.0 ? sbar / (sbar + xi * omega) : 0.0;
      const double2 v = buf[c * n + ky];
      const double2 sh = make_double2(f * v.x, f * v.y);
      const double2 old = S[k];
      const double dr = sh.x - old.x, di = sh.y - old.y;
      num += dr * dr + di * di;
      den += sh.x * sh.x + sh.y * sh.y;
      S[k] = sh;
      buf[c * n + ky] = sh;
    }
    __syncthreads();
  }
  flat_fft(buf, n, logn, FLAT_CB, tw, true);
  for (int e = tid; e < FLAT_CB * n; e += FLAT_THREADS) {
    const int y = e / FLAT_CB, c = e - y * FLAT_CB;
    T2[(long)y * n + kx0 + c] = buf[c * n + y];
  }
  if (mode == FLAT_ITER) {
    red[0][tid] = num;
    red[1][tid] = den;
    __syncthreads();
    for (int s = FLAT_THREADS / 2; s > 0; s >>= 1) {
      if (tid < s) {
        red[0][tid] += red[0][tid + s];
        red[1][tid] += red[1][tid + s];
      }
      __syncthreads();
    }
    if (tid == 0) {
      partials[2 * blockIdx.x] = red[0][0];
      partials[2 * blockIdx.x + 1] = red[1][0];
    }
  }
}

// Row y.  FLAT_FWD: forward FFT of the real map `in` (t_0 = d) -> T1.
// FLAT_ITER: inverse FFT of T2's row, s = Re / n^2, t = s + w (d - s),
// w = xi / (sigma^2 + mu) (0 where sigma^2 = +inf), forward FFT of t -> T1.
// FLAT_FINAL: inverse FFT of T2's row, s -> out.
__global__ void __launch_bounds__(FLAT_THREADS)
    k_flat_rows(int n, int logn, const double2 *__restrict__ T2, double2 *__restrict__ T1,
                const double *__restrict__ in, const double *__restrict__ d,
                const double *__restrict__ nvar, double *__restrict__ out,
                const double2 *__restrict__ tw, const SolverState *__restrict__ st, int mode) {
  extern __shared__ __align__(16) unsigned char flat_smem[];
  double2 *buf = reinterpret_cast<double2 *>(flat_smem);  // [n]
  if (mode == FLAT_ITER && st->done) return;
  const long row = (long)blockIdx.x * n;
  const int tid = threadIdx.x;
  if (mode == FLAT_FWD) {
    for (int x = tid; x < n; x += FLAT_THREADS) buf[x] = make_double2(in[row + x], 0.0);
    __syncthreads();
  } else {
    for (int x = tid; x < n; x += FLAT_THREADS) buf[x] = T2[row + x];
    __syncthreads();
    flat_fft(buf, n, logn, 1, tw, true);
    const double scale = 1.0 / ((double)n * (double)n);
    if (mode == FLAT_FINAL) {
      for (int x = tid; x < n; x += FLAT_THREADS) out[row + x] = buf[x].x * scale;
      return;
    }
    const double xi = st->xi, mu = st->mu;
    for (int x = tid; x < n; x += FLAT_THREADS) {
      const double s = buf[x].x * scale;
      const double v = nvar[row + x];
      const double w = isinf(v) ? 0.0 : xi / (v + mu);
      buf[x] = make_double2(s + w * (d[row + x] - s), 0.0);
    }
    __syncthreads();
  }
  flat_fft(buf, n, logn, 1, tw, false);
  for (int x = tid; x < n; x += FLAT_THREADS) T1[row + x] = buf[x];
}

// ------------------------------------------------------------------ plan
struct FlatPlan {
  int n = 0, logn = 0;
  double omega = 0.0, alpha = 0.0, ck_max = 0.0;
  wf_opts opts{};
  cudaStream_t stream = nullptr, capture_stream = nullptr;
  double *ck = nullptr, *nvar = nullptr, *d = nullptr, *partials = nullptr;
  double2 *T1 = nullptr, *T2 = nullptr, *S = nullptr, *tw = nullptr;
  SolverState *state = nullptr, *state_h = nullptr;
  TraceEntry *trace = nullptr;
  int trace_cap = 0, trace_len = 0;
  cudaGraphExec_t graph = nullptr;
  int chunk = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  long nlaunch = 0;
  size_t smem_cols = 0, smem_rows = 0;
};

static void flat_free(FlatPlan *F) {
  if (!F) return;
  if (F->graph) cudaGraphExecDestroy(F->graph);
  void *b[] = {F->ck, F->nvar, F->d, F->partials, F->T1, F->T2, F->S, F->tw, F->state,
               F->trace};
  for (void *x : b)
    if (x) cudaFree(x);
  if (F->state_h) cudaFreeHost(F->state_h);
  if (F->capture_stream) cudaStreamDestroy(F->capture_stream);
  if (F->ev0) cudaEventDestroy(F->ev0);
  if (F->ev1) cudaEventDestroy(F->ev1);
  delete F;
}

static SolverState flat_initial_state(const FlatPlan &F) {
  SolverState s{};
  const wf_opts &o = F.opts;
  s.alpha = F.alpha;
  s.beta = o.beta;
  s.omega = F.omega;
  // start: mu_0 Omega_pix = beta max_k C_k (or opts.mu0)
  const double mu0 = o.mu0 < 0.0 ? o.beta * F.ck_max / F.omega : o.mu0;
  s.mu = mu0;
  s.xi = F.alpha + mu0;
  s.eps_final = o.eps_final;
  s.eps_cap = o.eps_cap;
  s.eps_k = stage_tolerance(s, mu0);
  s.prev_c = -1.0;
  s.cmin = -1.0;
  s.max_iter = o.max_iter;
  s.stop_rule = o.stop_rule;
  s.band_limit = 0;  // every DFT mode is transformed
  s.trace_cap = F.trace_cap;
  s.lcur = s.lnext = 0;
  return s;
}

static int flat_ncols(const FlatPlan &F) { return F.n / FLAT_CB; }

static wf_status flat_enqueue_iteration(FlatPlan &F, cudaStream_t st) {
  F.nlaunch += 3;
  k_flat_cols<<<flat_ncols(F), FLAT_THREADS, F.smem_cols, st>>>(
      F.n, F.logn, F.omega, F.ck, F.T1, F.S, F.T2, F.tw, F.state, F.partials, FLAT_ITER);
  k_flat_rows<<<F.n, FLAT_THREADS, F.smem_rows, st>>>(F.n, F.logn, F.T2, F.T1, nullptr, F.d,
                                                      F.nvar, nullptr, F.tw, F.state,
                                                      FLAT_ITER);
  k_control<<<1, CONTROL_THREADS, 0, st>>>(F.state, F.partials, flat_ncols(F) - 1, nullptr,
                                           F.trace);
  WF_CUDA(cudaGetLastError());
  return WF_OK;
}

static wf_status flat_capture(FlatPlan &F) {
  if (F.graph) return WF_OK;
  F.chunk = F.opts.graph_chunk > 0 ? F.opts.graph_chunk
                                   : (int)std::max(8L, std::min(256L, (1L << 22) / ((long)F.n * F.n)));
  if (!F.capture_stream)
    WF_CUDA(cudaStreamCreateWithFlags(&F.capture_stream, cudaStreamNonBlocking));
  cudaError_t e = cudaStreamBeginCapture(F.capture_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    set_error(std::string("wf_flat: graph capture: ") + cudaGetErrorString(e));
    return WF_ERR_CUDA;
  }
  const long n0 = F.nlaunch;
  wf_status s = WF_OK;
  for (int i = 0; i < F.chunk && s == WF_OK; ++i) s = flat_enqueue_iteration(F, F.capture_stream);
  F.nlaunch = n0;
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(F.capture_stream, &g);
  if (s != WF_OK) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  if (e != cudaSuccess) {
    set_error(std::string("wf_flat: graph capture: ") + cudaGetErrorString(e));
    return WF_ERR_CUDA;
  }
  e = cudaGraphInstantiate(&F.graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    F.graph = nullptr;
    set_error(std::string("wf_flat: graph instantiate: ") + cudaGetErrorString(e));
    return WF_ERR_CUDA;
  }
  return WF_OK;
}

static wf_status flat_solve(FlatPlan &F, const double *d, double *s_out, wf_stats *stats) {
  const long n2 = (long)F.n * F.n;
  const long l0 = F.nlaunch;
  WF_CUDA(cudaEventRecord(F.ev0, F.stream));
  WF_CUDA(cudaMemcpyAsync(F.d, d, sizeof(double) * n2, cudaMemcpyDeviceToDevice, F.stream));
  WF_CUDA(cudaMemsetAsync(F.S, 0, sizeof(double2) * n2, F.stream));  // s_0 = 0
  *F.state_h = flat_initial_state(F);
  WF_CUDA(cudaMemcpyAsync(F.state, F.state_h, sizeof(SolverState), cudaMemcpyHostToDevice,
                          F.stream));
  // t_0 = d: its row transforms
  ++F.nlaunch;
  k_flat_rows<<<F.n, FLAT_THREADS, F.smem_rows, F.stream>>>(F.n, F.logn, nullptr, F.T1, F.d,
                                                            nullptr, nullptr, nullptr, F.tw,
                                                            nullptr, FLAT_FWD);
  WF_CUDA(cudaGetLastError());
  WF_TRY(flat_capture(F));
  long graph_nodes = 3L * F.chunk;
  for (;;) {
    WF_CUDA(cudaGraphLaunch(F.graph, F.stream));
    F.nlaunch += graph_nodes;
    WF_CUDA(cudaMemcpyAsync(F.state_h, F.state, sizeof(SolverState), cudaMemcpyDeviceToHost,
                            F.stream));
    WF_CUDA(cudaStreamSynchronize(F.stream));
    if (F.state_h->done) break;
  }
  // s of the last iteration: the inverse transforms of its filtered spectrum
  F.nlaunch += 2;
  k_flat_cols<<<flat_ncols(F), FLAT_THREADS, F.smem_cols, F.stream>>>(
      F.n, F.logn, F.omega, F.ck, F.T1, F.S, F.T2, F.tw, nullptr, nullptr, FLAT_FINAL);
  k_flat_rows<<<F.n, FLAT_THREADS, F.smem_rows, F.stream>>>(F.n, F.logn, F.T2, F.T1, nullptr,
                                                            nullptr, nullptr, s_out, F.tw,
                                                            nullptr, FLAT_FINAL);
  WF_CUDA(cudaGetLastError());
  WF_CUDA(cudaEventRecord(F.ev1, F.stream));
  WF_CUDA(cudaStreamSynchronize(F.stream));
  const SolverState &h = *F.state_h;
  F.trace_len = std::min(h.iter, F.trace_cap);
  if (stats) {
    float ms = 0.f;
    WF_CUDA(cudaEventElapsedTime(&ms, F.ev0, F.ev1));
    *stats = wf_stats{};
    stats->iterations = h.iter;
    stats->stages = h.stage + 1;
    stats->converged = h.converged;
    stats->alpha = F.alpha;
    stats->final_cauchy = h.last_c;
    stats->err_estimate = h.err_est;
    stats->elapsed_ms = ms;
    stats->kernel_launches = F.nlaunch - l0;
  }
  if (h.numeric_error) {
    set_error("wf_flat_solve: NaN or Inf in the iteration");
    return WF_ERR_NUMERIC;
  }
  if (!h.converged) {
    set_error("wf_flat_solve: max_iter reached before the last stage converged");
    return WF_ERR_NOT_CONVERGED;
  }
  return WF_OK;
}

}  // namespace wf

using namespace wf;

struct wf_flat_s : public FlatPlan {};

extern "C" {

wf_status wf_flat_plan(wf_flat_t *out, int n, double pixel_area, const double *ck_host,
                       const double *noise_var_dev, const wf_opts *opts, void *stream) {
  if (!out || !ck_host || !noise_var_dev) {
    set_error("wf_flat_plan: NULL argument");
    return WF_ERR_ARG;
  }
  *out = nullptr;
  int logn = 0;
  while ((1 << logn) < n) ++logn;
  if (n < 8 || n > FLAT_NMAX || (1 << logn) != n) {
    set_error("wf_flat_plan: n must be a power of two in [8, 2048]");
    return WF_ERR_ARG;
  }
  if (!(pixel_area > 0.0)) {
    set_error("wf_flat_plan: pixel_area must be > 0");
    return WF_ERR_ARG;
  }
  wf_opts o;
  wf_opts_default(&o);
  if (opts) o = *opts;
  if (!(o.beta > 0.0 && o.beta < 1.0) || !(o.eps_final > 0.0) || !(o.eps_cap > 0.0) ||
      o.max_iter < 1 || (o.stop_rule != WF_STOP_CAUCHY && o.stop_rule != WF_STOP_ERROR) ||
      o.graph_chunk < 0 || o.graph_chunk > 4096) {
    set_error("wf_flat_plan: invalid options (beta, eps, max_iter, stop_rule, graph_chunk)");
    return WF_ERR_ARG;
  }
  const long n2 = (long)n * n;
  std::vector<double> ck(ck_host, ck_host + n2);
  double cmax = 0.0;
  for (double c : ck) {
    if (!(c >= 0.0) || !std::isfinite(c)) {
      set_error("wf_flat_plan: C_k must be finite and >= 0");
      return WF_ERR_ARG;
    }
    cmax = std::max(cmax, c);
  }
  wf_flat_s *F = new (std::nothrow) wf_flat_s();
  if (!F) {
    set_error("wf_flat_plan: out of host memory");
    return WF_ERR_CUDA;
  }
  F->n = n;
  F->logn = logn;
  F->omega = pixel_area;
  F->opts = o;
  F->ck_max = cmax;
  F->stream = static_cast<cudaStream_t>(stream);
  F->trace_cap = 1 << 20;
  F->smem_cols = sizeof(double2) * FLAT_CB * n;
  F->smem_rows = sizeof(double2) * n;
  auto fail = [&](const char *what, cudaError_t e) {
    set_error(std::string("wf_flat_plan: ") + what + ": " + cudaGetErrorString(e));
    flat_free(F);
    return WF_ERR_CUDA;
  };
  cudaError_t e = cudaSuccess;
  for (double **b : {&F->ck, &F->nvar, &F->d})
    if ((e = cudaMalloc(b, sizeof(double) * n2)) != cudaSuccess) return fail("cudaMalloc", e);
  for (double2 **b : {&F->T1, &F->T2, &F->S})
    if ((e = cudaMalloc(b, sizeof(double2) * n2)) != cudaSuccess) return fail("cudaMalloc", e);
  if ((e = cudaMalloc(&F->tw, sizeof(double2) * (n / 2))) != cudaSuccess ||
      (e = cudaMalloc(&F->partials, sizeof(double) * 2 * (n / FLAT_CB))) != cudaSuccess ||
      (e = cudaMalloc(&F->state, sizeof(SolverState))) != cudaSuccess ||
      (e = cudaMallocHost(&F->state_h, sizeof(SolverState))) != cudaSuccess ||
      (e = cudaMalloc(&F->trace, sizeof(TraceEntry) * F->trace_cap)) != cudaSuccess ||
      (e = cudaEventCreate(&F->ev0)) != cudaSuccess ||
      (e = cudaEventCreate(&F->ev1)) != cudaSuccess)
    return fail("allocation", e);
  if (F->smem_cols > 48 * 1024 &&
      (e = cudaFuncSetAttribute(k_flat_cols, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)F->smem_cols)) != cudaSuccess)
    return fail("shared memory attribute", e);
  // twiddles e^{-2 pi i k / n}: sin and cos of pi (2k / n), exact argument
  std::vector<double2> tw(n / 2);
  for (int k = 0; k < n / 2; ++k) {
    double sn = 0.0, cs = 0.0;
    sincospi(2.0 * k / n, &sn, &cs);
    tw[k] = make_double2(cs, -sn);
  }
  // alpha = min sigma^2 over observed pixels (+inf: a masked pixel)
  std::vector<double> nv(n2);
  if ((e = cudaMemcpy(nv.data(), noise_var_dev, sizeof(double) * n2, cudaMemcpyDeviceToHost)) !=
      cudaSuccess)
    return fail("noise copy", e);
  double alpha = INFINITY;
  for (double v : nv) {
    if (!(v > 0.0) || std::isnan(v)) {
      set_error("wf_flat_plan: noise variances must be > 0 (+inf masks a pixel)");
      flat_free(F);
      return WF_ERR_ARG;
    }
    alpha = std::min(alpha, v);
  }
  if (!std::isfinite(alpha)) {
    set_error("wf_flat_plan: every pixel is masked");
    flat_free(F);
    return WF_ERR_ARG;
  }
  F->alpha = alpha;
  if ((e = cudaMemcpy(F->nvar, nv.data(), sizeof(double) * n2, cudaMemcpyHostToDevice)) !=
          cudaSuccess ||
      (e = cudaMemcpy(F->ck, ck.data(), sizeof(double) * n2, cudaMemcpyHostToDevice)) !=
          cudaSuccess ||
      (e = cudaMemcpy(F->tw, tw.data(), sizeof(double2) * tw.size(), cudaMemcpyHostToDevice)) !=
          cudaSuccess)
    return fail("upload", e);
  *out = F;
  return WF_OK;
}

wf_status wf_flat_solve(wf_flat_t plan, const double *d_dev, double *s_dev, wf_stats *stats) {
  if (!plan || !d_dev || !s_dev) {
    set_error("wf_flat_solve: NULL argument");
    return WF_ERR_ARG;
  }
  return flat_solve(*plan, d_dev, s_dev, stats);
}

wf_status wf_flat_trace(wf_flat_t plan, int *count, int *stage, double *cauchy) {
  if (!plan || !count || *count < 0) {
    set_error("wf_flat_trace: NULL argument");
    return WF_ERR_ARG;
  }
  const int k = std::min(*count, plan->trace_len);
  std::vector<TraceEntry> h(k);
  if (k > 0) {
    cudaError_t e = cudaMemcpy(h.data(), plan->trace, sizeof(TraceEntry) * k,
                               cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
      set_error(std::string("wf_flat_trace: ") + cudaGetErrorString(e));
      return WF_ERR_CUDA;
    }
  }
  for (int i = 0; i < k; ++i) {
    if (stage) stage[i] = h[i].stage;
    if (cauchy) cauchy[i] = h[i].cauchy;
  }
  *count = k;
  return WF_OK;
}

void wf_flat_destroy(wf_flat_t plan) { flat_free(plan); }

}  // extern "C"
