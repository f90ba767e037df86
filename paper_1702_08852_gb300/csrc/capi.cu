// capi.cu -- the extern "C" entry points declared in include/wf.h:
// argument checking, plan lifetime, error strings.
#include <algorithm>
#include <initializer_list>
#include <math.h>
#include <string.h>

#include <new>
#include <string>
#include <vector>

#include "wf_internal.cuh"

namespace wf {
static thread_local std::string g_last_error;
static thread_local const char *g_last_error_static = nullptr;
void set_error(const std::string &msg) {
  g_last_error = msg;
  g_last_error_static = nullptr;
}
void set_error_static(const char *msg) { g_last_error_static = msg; }

static wf_status arg_error(const char *msg) {
  set_error(msg);
  return WF_ERR_ARG;
}

static void free_plan(wf_plan_s *P) {
  if (!P) return;
  free_group(*P);
  for (int i = 0; i < 3; ++i)
    if (P->graph[i]) cudaGraphExecDestroy(P->graph[i]);
  void *bufs[] = {P->pairs, P->cl_d,   P->rc,      P->rg,     P->rc32,   P->seed_l,
                  P->seed_u, P->tw64,  P->tw32,    P->chirp64, P->chirp32, P->bhat64,
                  P->bhat32, P->nvar,  P->F64,     P->G64,    P->F32,    P->G32,
                  P->x,      P->xtmp,  P->dmap,    P->mtmp,   P->partials, P->red,
                  P->state,  P->trace, P->xacc,  P->src, P->xs64, P->xs32,
                  P->nvar32, P->dmap32, P->ana_scratch, P->ana_lstart,
                  P->ana_counter, P->uacc[0], P->uacc[1],
                  P->seed_s32, P->zs32, P->rg32, P->cl32, P->twdd, P->chirpdd, P->bhatdd,
                  P->phasedd, P->rcdd, P->nvardd, P->dmapdd};
  for (void *b : bufs)
    if (b) cudaFree(b);
  if (P->state_h) cudaFreeHost(P->state_h);
  if (P->capture_stream) cudaStreamDestroy(P->capture_stream);
  if (P->side_stream) cudaStreamDestroy(P->side_stream);
  if (P->fork_ev) cudaEventDestroy(P->fork_ev);
  if (P->join_ev) cudaEventDestroy(P->join_ev);
  for (cudaEvent_t e : P->tev) cudaEventDestroy(e);
  for (cudaEvent_t e : P->dd_ev)
    if (e) cudaEventDestroy(e);
  if (P->ev0) cudaEventDestroy(P->ev0);
  if (P->ev1) cudaEventDestroy(P->ev1);
  delete P;
}

static wf_status alloc_work(Plan &P) {
  WF_CUDA(cudaStreamCreateWithFlags(&P.side_stream, cudaStreamNonBlocking));
  WF_CUDA(cudaEventCreateWithFlags(&P.fork_ev, cudaEventDisableTiming));
  WF_CUDA(cudaEventCreateWithFlags(&P.join_ev, cudaEventDisableTiming));
  const size_t nF = (size_t)P.nring * (P.lmax + 1);
  WF_CUDA(cudaMalloc(&P.F64, sizeof(double2) * nF));
  WF_CUDA(cudaMalloc(&P.G64, sizeof(double2) * nF));
  WF_CUDA(cudaMalloc(&P.F32, sizeof(float2) * nF));
  WF_CUDA(cudaMalloc(&P.G32, sizeof(float2) * nF));
  WF_CUDA(cudaMalloc(&P.x, sizeof(double2) * P.nalm));
  WF_CUDA(cudaMalloc(&P.xtmp, sizeof(double2) * P.nalm));
  WF_CUDA(cudaMalloc(&P.xacc, sizeof(double2) * P.nalm));
  WF_CUDA(cudaMalloc(&P.xs64, sizeof(double2) * P.nalm));
  WF_CUDA(cudaMalloc(&P.xs32, sizeof(float2) * P.nalm));
  WF_CUDA(cudaMalloc(&P.src, sizeof(double2) * P.nalm));
  WF_CUDA(cudaMalloc(&P.dmap, sizeof(double) * P.npix));
  WF_CUDA(cudaMalloc(&P.dmap32, sizeof(float) * P.npix));
  WF_CUDA(cudaMalloc(&P.dmapdd, sizeof(float2) * P.npix));
  {
    // queue-scheduled FP32 analysis: partial sums of tiles of 128 ring pairs
    // (the smallest tile of its variants)
    const long tiles = (P.npairs + 127) / 128;
    int dev = 0;
    WF_CUDA(cudaGetDevice(&dev));
    P.device = dev;
    WF_CUDA(cudaDeviceGetAttribute(&P.num_sms, cudaDevAttrMultiProcessorCount, dev));
    // 16 bytes per entry: FP32 complex for the FP32 kernels, FP64 complex
    // for the double-float anchor analysis
    // (and the packed analysis' global accumulators: 4 warps x FP32 complex)
    WF_CUDA(cudaMalloc(&P.ana_scratch, sizeof(double2) * std::max(tiles, 2L) * P.nalm));
    WF_CUDA(cudaMalloc(&P.ana_lstart, sizeof(int) * tiles * (P.lmax + 1)));
    WF_CUDA(cudaMalloc(&P.ana_counter, sizeof(int)));
    WF_CUDA(cudaMemsetAsync(P.ana_counter, 0, sizeof(int), P.stream));
  }
  WF_CUDA(cudaMalloc(&P.mtmp, sizeof(double) * P.npix));
  // per m: ||x_new - x_old||^2, ||x_new||^2, then (anchored stages) ||x_a + delta||^2
  WF_CUDA(cudaMalloc(&P.partials, sizeof(double) * 3 * (P.lmax + 1)));
  WF_CUDA(cudaMalloc(&P.red, sizeof(double) * 1024));
  WF_CUDA(cudaMalloc(&P.state, sizeof(SolverState)));
  WF_CUDA(cudaMallocHost(&P.state_h, sizeof(SolverState)));
  P.trace_cap = 1 << 20;
  WF_CUDA(cudaMalloc(&P.trace, sizeof(TraceEntry) * P.trace_cap));
  WF_CUDA(cudaEventCreate(&P.ev0));
  WF_CUDA(cudaEventCreate(&P.ev1));
  WF_CUDA(cudaMemsetAsync(P.F64, 0, sizeof(double2) * nF, P.stream));
  WF_CUDA(cudaMemsetAsync(P.G64, 0, sizeof(double2) * nF, P.stream));
  WF_CUDA(cudaMemsetAsync(P.F32, 0, sizeof(float2) * nF, P.stream));
  WF_CUDA(cudaMemsetAsync(P.G32, 0, sizeof(float2) * nF, P.stream));
  return WF_OK;
}

static wf_status check_opts(const wf_opts &o) {
  if (!(o.beta > 0.0 && o.beta < 1.0)) return arg_error("wf: beta must be in (0, 1)");
  if (!(o.eps_final > 0.0) || !(o.eps_cap > 0.0))
    return arg_error("wf: eps_final and eps_cap must be > 0");
  if (o.max_iter < 1) return arg_error("wf: max_iter must be >= 1");
  if (o.stop_rule != WF_STOP_CAUCHY && o.stop_rule != WF_STOP_ERROR)
    return arg_error("wf: unknown stop_rule");
  if (o.precision != WF_PREC_FP64 && o.precision != WF_PREC_MIXED)
    return arg_error("wf: unknown precision");
  if (o.graph_chunk < 0 || o.graph_chunk > 4096)
    return arg_error("wf: graph_chunk out of range");
  if (o.anchor != 0 && o.anchor != 1) return arg_error("wf: anchor must be 0 or 1");
  if (!(o.anchor_eps >= 0.0) || !(o.anchor_cap > 0.0 && o.anchor_cap <= 1.0))
    return arg_error("wf: anchor_eps must be >= 0 and anchor_cap in (0, 1]");
  if (o.tail_exact != 0 && o.tail_exact != 1) return arg_error("wf: tail_exact must be 0 or 1");
  if (!(o.tail_window < 10.0)) return arg_error("wf: tail_window must be < 10");
  if (!(o.tail_cap_tol >= 0.0)) return arg_error("wf: tail_cap_tol must be >= 0");
  if (!(o.anchor_cap_tol >= 0.0)) return arg_error("wf: anchor_cap_tol must be >= 0");
  if (o.method != WF_METHOD_DUAL && o.method != WF_METHOD_MESSENGER)
    return arg_error("wf: unknown method");
  if (o.method == WF_METHOD_MESSENGER && !(o.lambda0 >= 1.0 && o.lambda0 < 1e300))
    return arg_error("wf: lambda0 must be >= 1");
  return WF_OK;
}

}  // namespace wf

using namespace wf;

extern "C" {

void wf_opts_default(wf_opts *o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->beta = 0.75;
  o->eps_final = 1e-6;
  o->eps_cap = 1e-2;
  o->mu0 = -1.0;
  o->max_iter = 200000;
  o->stop_rule = WF_STOP_CAUCHY;
  o->precision = WF_PREC_FP64;
  o->band_limit = 1;
  o->graph_chunk = 0;
  o->refine_max = 8;
  o->anchor = 1;
  o->anchor_eps = 1.0;
  o->anchor_cap = 1e-2;
  o->anchor_cap_tol = 100.0;
  o->tail_exact = 1;
  o->tail_window = 0.08;
  o->tail_cap_tol = 10.0;
  o->method = WF_METHOD_DUAL;
  o->lambda0 = 1e4;
}

long wf_npix(int nside) { return 12L * nside * nside; }
long wf_nalm(int lmax) { return (long)(lmax + 1) * (lmax + 2) / 2; }

const char *wf_status_str(wf_status s) {
  switch (s) {
    case WF_OK: return "ok";
    case WF_ERR_ARG: return "invalid argument";
    case WF_ERR_CUDA: return "CUDA error";
    case WF_ERR_NOT_CONVERGED: return "not converged";
    case WF_ERR_NUMERIC: return "NaN or Inf in the iteration";
    case WF_ERR_TIMEOUT: return "device wait timed out";
    case WF_ERR_UNIMPLEMENTED: return "not implemented";
    case WF_ERR_STATE: return "invalid call for this plan";
  }
  return "unknown status";
}

const char *wf_last_error(void) {
  return g_last_error_static ? g_last_error_static : g_last_error.c_str();
}

wf_status wf_plan(wf_plan_t *out, int nside, int lmax, const double *cl_host,
                  const double *noise_var_dev, const uint8_t *mask_dev,
                  const wf_opts *opts, void *stream) {
  if (!out) return arg_error("wf_plan: out is NULL");
  *out = nullptr;
  if (nside < 1 || nside > 8192) return arg_error("wf_plan: nside out of range [1, 8192]");
  if (lmax < 1 || lmax > 3 * nside - 1)
    return arg_error("wf_plan: lmax out of range [1, 3 nside - 1]");
  if (!cl_host) return arg_error("wf_plan: cl_host is NULL");
  for (int l = 0; l <= lmax; ++l)
    if (!(cl_host[l] >= 0.0) || isinf(cl_host[l]))
      return arg_error("wf_plan: C_l must be finite and >= 0");
  wf_opts o;
  wf_opts_default(&o);
  if (opts) o = *opts;
  WF_TRY(check_opts(o));
  wf_plan_s *P = new (std::nothrow) wf_plan_s();
  if (!P) return arg_error("wf_plan: out of host memory");
  P->nside = nside;
  P->lmax = lmax;
  P->nring = 4 * nside - 1;
  P->npairs = 2 * nside;
  P->npix = 12L * nside * nside;
  P->nalm = (long)(lmax + 1) * (lmax + 2) / 2;
  P->omega = 4.0 * M_PI / (double)P->npix;
  P->stream = (cudaStream_t)stream;
  P->opts = o;
  P->cl.assign(cl_host, cl_host + lmax + 1);
  wf_status s = WF_OK;
  try {
    s = build_tables(*P);
    if (s == WF_OK) s = alloc_work(*P);
    if (s == WF_OK && noise_var_dev) s = upload_noise(*P, noise_var_dev, mask_dev);
    if (s == WF_OK && o.autotune) s = autotune(*P);
    if (s == WF_OK) {
      cudaError_t e = cudaStreamSynchronize(P->stream);
      if (e != cudaSuccess) {
        set_error(std::string("wf_plan: ") + cudaGetErrorString(e));
        s = WF_ERR_CUDA;
      }
    }
  } catch (const std::bad_alloc &) {
    set_error("wf_plan: out of host memory");
    s = WF_ERR_ARG;
  }
  if (s != WF_OK) {
    free_plan(P);
    return s;
  }
  *out = P;
  return WF_OK;
}

wf_status wf_set_noise(wf_plan_t plan, const double *noise_var_dev,
                       const uint8_t *mask_dev) {
  if (!plan) return arg_error("wf_set_noise: plan is NULL");
  if (!noise_var_dev) return arg_error("wf_set_noise: noise_var_dev is NULL");
  return upload_noise(*plan, noise_var_dev, mask_dev);
}

wf_status wf_set_cl(wf_plan_t plan, const double *cl_host) {
  if (!plan) return arg_error("wf_set_cl: plan is NULL");
  if (!cl_host) return arg_error("wf_set_cl: cl_host is NULL");
  for (int l = 0; l <= plan->lmax; ++l)
    if (!(cl_host[l] >= 0.0) || isinf(cl_host[l]))
      return arg_error("wf_set_cl: C_l must be finite and >= 0");
  plan->cl.assign(cl_host, cl_host + plan->lmax + 1);
  const std::vector<float> cl32(plan->cl.begin(), plan->cl.end());
  WF_CUDA(cudaMemcpyAsync(plan->cl_d, plan->cl.data(), sizeof(double) * (plan->lmax + 1),
                          cudaMemcpyHostToDevice, plan->stream));
  WF_CUDA(cudaMemcpyAsync(plan->cl32, cl32.data(), sizeof(float) * (plan->lmax + 1),
                          cudaMemcpyHostToDevice, plan->stream));
  WF_CUDA(cudaStreamSynchronize(plan->stream));
  return WF_OK;
}

wf_status wf_solve(wf_plan_t plan, const double *d_dev, double *alm_dev,
                   double *map_dev, const double *init_alm_dev,
                   const double *init_map_dev, wf_stats *stats) {
  if (!plan) return arg_error("wf_solve: plan is NULL");
  if (!d_dev) return arg_error("wf_solve: d_dev is NULL");
  return solve(*plan, d_dev, alm_dev, map_dev, init_alm_dev, init_map_dev, stats);
}

wf_status wf_solve_host(wf_plan_t plan, const double *d_host, double *alm_host,
                        double *map_host, wf_stats *stats) {
  if (!plan) return arg_error("wf_solve_host: plan is NULL");
  if (!d_host) return arg_error("wf_solve_host: d_host is NULL");
  Plan &P = *plan;
  double *dd = nullptr, *mm = nullptr;
  double2 *aa = nullptr;
  WF_CUDA(cudaMalloc(&dd, sizeof(double) * P.npix));
  wf_status s = WF_OK;
  do {
    if (map_host && cudaMalloc(&mm, sizeof(double) * P.npix) != cudaSuccess) {
      s = WF_ERR_CUDA;
      break;
    }
    if (alm_host && cudaMalloc(&aa, sizeof(double2) * P.nalm) != cudaSuccess) {
      s = WF_ERR_CUDA;
      break;
    }
    if (cudaMemcpyAsync(dd, d_host, sizeof(double) * P.npix, cudaMemcpyHostToDevice,
                        P.stream) != cudaSuccess) {
      s = WF_ERR_CUDA;
      break;
    }
    s = solve(P, dd, reinterpret_cast<double *>(aa), mm, nullptr, nullptr, stats);
    if (s != WF_OK && s != WF_ERR_NOT_CONVERGED) break;
    if (alm_host &&
        cudaMemcpyAsync(alm_host, aa, sizeof(double2) * P.nalm, cudaMemcpyDeviceToHost,
                        P.stream) != cudaSuccess) {
      s = WF_ERR_CUDA;
      break;
    }
    if (map_host && cudaMemcpyAsync(map_host, mm, sizeof(double) * P.npix,
                                    cudaMemcpyDeviceToHost, P.stream) != cudaSuccess) {
      s = WF_ERR_CUDA;
      break;
    }
    if (cudaStreamSynchronize(P.stream) != cudaSuccess) s = WF_ERR_CUDA;
  } while (0);
  if (s == WF_ERR_CUDA) set_error("wf_solve_host: CUDA allocation or copy failed");
  cudaFree(dd);
  if (mm) cudaFree(mm);
  if (aa) cudaFree(aa);
  return s;
}

wf_status wf_residual(wf_plan_t plan, const double *d_dev, const double *alm_dev,
                      double *rel_res_wf, double *rel_res_fp, double *chi2) {
  if (!plan) return arg_error("wf_residual: plan is NULL");
  if (!d_dev || !alm_dev) return arg_error("wf_residual: NULL input");
  return residual(*plan, d_dev, alm_dev, rel_res_wf, rel_res_fp, chi2);
}

wf_status wf_pcg(wf_plan_t plan, const double *d_dev, double *alm_dev, double *map_dev,
                 double tol, int stop_rule, int max_iter, int restart, wf_stats *stats) {
  if (!plan) return arg_error("wf_pcg: plan is NULL");
  if (!d_dev) return arg_error("wf_pcg: d_dev is NULL");
  if (!(tol > 0.0)) return arg_error("wf_pcg: tol must be > 0");
  if (stop_rule != WF_PCG_STOP_CAUCHY && stop_rule != WF_PCG_STOP_RESIDUAL)
    return arg_error("wf_pcg: unknown stop_rule");
  if (max_iter < 1 || restart < 1) return arg_error("wf_pcg: max_iter and restart must be >= 1");
  return pcg(*plan, d_dev, alm_dev, map_dev, tol, stop_rule, max_iter, restart, stats);
}

wf_status wf_solve_batch(wf_plan_t *plans, int n, const double *const *d_dev,
                         double *const *alm_dev, double *const *map_dev, wf_stats *stats,
                         double *elapsed_ms) {
  if (!plans || n < 1 || !d_dev) return arg_error("wf_solve_batch: NULL or empty batch");
  if (n > 4096) return arg_error("wf_solve_batch: at most 4096 maps");
  std::vector<Plan *> ps(n);
  for (int i = 0; i < n; ++i) {
    if (!plans[i] || !d_dev[i]) return arg_error("wf_solve_batch: NULL plan or data");
    for (int j = 0; j < i; ++j)
      if (plans[j] == plans[i]) return arg_error("wf_solve_batch: a plan appears twice");
    if (!plans[i]->has_noise) return arg_error("wf_solve_batch: a plan has no noise");
    ps[i] = plans[i];
  }
  return solve_batch(ps.data(), n, d_dev, alm_dev, map_dev, stats, elapsed_ms);
}

wf_status wf_residual_static(wf_plan_t plan, const double *d_dev, const double *alm_dev,
                             double *rel_res_wf, double *rel_res_fp, double *chi2) {
  if (!plan) return arg_error("wf_residual_static: plan is NULL");
  if (!d_dev || !alm_dev) return arg_error("wf_residual_static: NULL input");
  return residual_static(*plan, d_dev, alm_dev, rel_res_wf, rel_res_fp, chi2);
}

wf_status wf_alm2map(wf_plan_t plan, const double *alm_dev, double *map_dev) {
  if (!plan) return arg_error("wf_alm2map: plan is NULL");
  if (!alm_dev || !map_dev) return arg_error("wf_alm2map: NULL buffer");
  WF_TRY(alm2map(*plan, alm_dev, map_dev));
  WF_CUDA(cudaStreamSynchronize(plan->stream));
  return WF_OK;
}

wf_status wf_map2alm(wf_plan_t plan, const double *map_dev, double *alm_dev) {
  if (!plan) return arg_error("wf_map2alm: plan is NULL");
  if (!alm_dev || !map_dev) return arg_error("wf_map2alm: NULL buffer");
  WF_TRY(map2alm(*plan, map_dev, alm_dev));
  WF_CUDA(cudaStreamSynchronize(plan->stream));
  return WF_OK;
}

wf_status wf_alm2map_f32(wf_plan_t plan, const double *alm_dev, double *map_dev) {
  if (!plan) return arg_error("wf_alm2map_f32: plan is NULL");
  if (!alm_dev || !map_dev) return arg_error("wf_alm2map_f32: NULL buffer");
  WF_TRY(alm2map_f32(*plan, alm_dev, map_dev));
  WF_CUDA(cudaStreamSynchronize(plan->stream));
  return WF_OK;
}

wf_status wf_map2alm_f32(wf_plan_t plan, const double *map_dev, double *alm_dev) {
  if (!plan) return arg_error("wf_map2alm_f32: plan is NULL");
  if (!alm_dev || !map_dev) return arg_error("wf_map2alm_f32: NULL buffer");
  WF_TRY(map2alm_f32(*plan, map_dev, alm_dev));
  WF_CUDA(cudaStreamSynchronize(plan->stream));
  return WF_OK;
}

wf_status wf_map2alm_group(wf_plan_t plan, int nmaps, const double *maps_dev,
                           double *alm_dev) {
  if (!plan) return arg_error("wf_map2alm_group: plan is NULL");
  if (nmaps < 0) return arg_error("wf_map2alm_group: nmaps must be >= 0");
  if (nmaps > 0 && (!maps_dev || !alm_dev)) return arg_error("wf_map2alm_group: NULL buffer");
  WF_TRY(map2alm_group(*plan, nmaps, maps_dev, alm_dev));
  WF_CUDA(cudaStreamSynchronize(plan->stream));
  return WF_OK;
}

wf_status wf_alm2map_group(wf_plan_t plan, int nmaps, const double *alm_dev,
                           double *maps_dev) {
  if (!plan) return arg_error("wf_alm2map_group: plan is NULL");
  if (nmaps < 0) return arg_error("wf_alm2map_group: nmaps must be >= 0");
  if (nmaps > 0 && (!maps_dev || !alm_dev)) return arg_error("wf_alm2map_group: NULL buffer");
  WF_TRY(alm2map_group(*plan, nmaps, alm_dev, maps_dev));
  WF_CUDA(cudaStreamSynchronize(plan->stream));
  return WF_OK;
}

wf_status wf_group_stats(wf_plan_t plan, double *ms, long *launches, double *gflop,
                         double *gbyte, int reset) {
  if (!plan) return arg_error("wf_group_stats: plan is NULL");
  if (ms) *ms = plan->group_ms;
  if (launches) *launches = plan->group_launches;
  if (gflop) *gflop = plan->group_flop * 1e-9;
  if (gbyte) *gbyte = plan->group_bytes * 1e-9;
  if (reset) {
    plan->group_ms = plan->group_flop = plan->group_bytes = 0.0;
    plan->group_launches = 0;
  }
  return WF_OK;
}

wf_status wf_alm2map_df64(wf_plan_t plan, const double *alm_dev, double *map_dev) {
  if (!plan) return arg_error("wf_alm2map_df64: plan is NULL");
  if (!alm_dev || !map_dev) return arg_error("wf_alm2map_df64: NULL buffer");
  WF_TRY(alm2map_df64(*plan, alm_dev, map_dev));
  WF_CUDA(cudaStreamSynchronize(plan->stream));
  return WF_OK;
}

wf_status wf_map2alm_df64(wf_plan_t plan, const double *map_dev, double *alm_dev) {
  if (!plan) return arg_error("wf_map2alm_df64: plan is NULL");
  if (!alm_dev || !map_dev) return arg_error("wf_map2alm_df64: NULL buffer");
  WF_TRY(map2alm_df64(*plan, map_dev, alm_dev));
  WF_CUDA(cudaStreamSynchronize(plan->stream));
  return WF_OK;
}

wf_status wf_trace(wf_plan_t plan, int *count, int *stage, double *xi, double *mu,
                   double *cauchy) {
  if (!plan || !count) return arg_error("wf_trace: NULL argument");
  const int n = std::min(*count, plan->trace_len);
  std::vector<TraceEntry> h(n > 0 ? n : 1);
  if (n > 0)
    WF_CUDA(cudaMemcpy(h.data(), plan->trace, sizeof(TraceEntry) * n,
                       cudaMemcpyDeviceToHost));
  for (int i = 0; i < n; ++i) {
    if (stage) stage[i] = h[i].stage;
    if (xi) xi[i] = h[i].xi;
    if (mu) mu[i] = h[i].mu;
    if (cauchy) cauchy[i] = h[i].cauchy;
  }
  *count = n;
  return WF_OK;
}

wf_status wf_kernel_stats(wf_plan_t plan, int kernel, double *ms, long *launches,
                          double *gflop, int reset) {
  if (!plan) return arg_error("wf_kernel_stats: plan is NULL");
  if (kernel < 0 || kernel > 5) return arg_error("wf_kernel_stats: kernel must be 0 .. 5");
  if (ms) *ms = plan->kern_ms[kernel];
  if (launches) *launches = plan->kern_launches[kernel];
  if (gflop) *gflop = plan->kern_flop[kernel] * 1e-9;
  if (reset) {
    plan->kern_ms[kernel] = 0.0;
    plan->kern_launches[kernel] = 0;
    plan->kern_flop[kernel] = 0.0;
  }
  return WF_OK;
}

wf_status wf_get_tuning(wf_plan_t plan, wf_tuning *out) {
  if (!plan || !out) return arg_error("wf_get_tuning: NULL argument");
  for (int k = 0; k < 2; ++k) {
    out->syn_np[k] = plan->syn_np[k];
    out->ana_np[k] = plan->ana_np[k];
    for (int c = 0; c < 6; ++c) out->syn_ms[k][c] = plan->tune_syn_ms[k][c];
    for (int c = 0; c < 15; ++c) out->ana_ms[k][c] = plan->tune_ana_ms[k][c];
  }
  out->syn_packed = plan->syn_x2;
  out->ana_queue = plan->ana_queue;
  out->ana_packed = plan->ana_x2;
  out->ana_global_acc = plan->ana_gacc;
  return WF_OK;
}

wf_status wf_set_tuning(wf_plan_t plan, const wf_tuning *in) {
  if (!plan || !in) return arg_error("wf_set_tuning: NULL argument");
  auto one_of = [](int v, std::initializer_list<int> set) {
    for (int s : set)
      if (v == s) return true;
    return false;
  };
  for (int k = 0; k < 2; ++k) {
    if (!one_of(in->syn_np[k], {1, 2, 4}))
      return arg_error("wf_set_tuning: syn_np must be 1, 2 or 4");
  }
  if (!one_of(in->ana_np[0], {2, 4, 8}))
    return arg_error("wf_set_tuning: FP64 ana_np must be 2, 4 or 8");
  if (!one_of(in->ana_queue, {0, 1}) || !one_of(in->ana_packed, {0, 1}) ||
      !one_of(in->syn_packed, {0, 1, 2}))
    return arg_error("wf_set_tuning: ana_queue, ana_packed must be 0 or 1, syn_packed 0, 1 or 2");
  if (in->ana_queue && in->ana_packed)
    return arg_error("wf_set_tuning: ana_queue and ana_packed exclude each other");
  if (!one_of(in->ana_global_acc, {0, 1, 2, 3}))
    return arg_error("wf_set_tuning: ana_global_acc must be 0, 1, 2 or 3");
  if (in->ana_global_acc == 1 && !(in->ana_packed && one_of(in->ana_np[1], {4, 6})))
    return arg_error("wf_set_tuning: ana_global_acc 1 needs ana_packed with ana_np 4 or 6");
  if (in->ana_global_acc == 2 && !(in->ana_packed && one_of(in->ana_np[1], {4, 6, 8})))
    return arg_error("wf_set_tuning: ana_global_acc 2 needs ana_packed with ana_np 4, 6 or 8");
  if (in->ana_global_acc == 3 && !(in->ana_packed && in->ana_np[1] == 8))
    return arg_error("wf_set_tuning: ana_global_acc 3 needs ana_packed with ana_np 8");
  if (in->ana_queue ? !one_of(in->ana_np[1], {4, 8})
                    : in->ana_packed ? !one_of(in->ana_np[1], {4, 6, 8})
                                     : !one_of(in->ana_np[1], {2, 4, 8, 16}))
    return arg_error("wf_set_tuning: FP32 ana_np must be 2, 4, 8 or 16 (queue: 4, 8; "
                     "packed: 4, 6, 8)");
  if (in->syn_packed == 1 && !one_of(in->syn_np[1], {2, 4}))
    return arg_error("wf_set_tuning: packed FP32 synthesis needs syn_np 2 or 4");
  if (in->syn_packed == 2 && in->syn_np[1] != 2)
    return arg_error("wf_set_tuning: packed FP32 synthesis with duplicated tables needs syn_np 2");
  for (int k = 0; k < 2; ++k) {
    plan->syn_np[k] = in->syn_np[k];
    plan->ana_np[k] = in->ana_np[k];
  }
  plan->syn_x2 = in->syn_packed;
  plan->ana_queue = in->ana_queue;
  plan->ana_x2 = in->ana_packed;
  plan->ana_gacc = in->ana_global_acc;
  for (int i = 0; i < 3; ++i) {
    if (plan->graph[i]) cudaGraphExecDestroy(plan->graph[i]);
    plan->graph[i] = nullptr;
  }
  return WF_OK;
}

wf_status wf_legendre_terms(wf_plan_t plan, int L, double *terms) {
  if (!plan || !terms) return arg_error("wf_legendre_terms: NULL argument");
  if (L < 0 || L > plan->lmax) return arg_error("wf_legendre_terms: L out of range");
  return legendre_terms(*plan, L, terms);
}

void wf_destroy(wf_plan_t plan) { free_plan(plan); }

}  // extern "C"
