// autotune.cu -- pick the launch variant (ring pairs per thread) of each
// Legendre kernel for a geometry by timing them once at full band.
//
// The best variant depends on the number of ring pairs and the band limit:
// more pairs per thread give more independent recurrences (latency hiding)
// and amortise the analysis' warp reduction, but cost registers and
// occupancy.  Results are cached per (nside, lmax) for the process.
#include <string.h>

#include <map>
#include <mutex>
#include <utility>

#include "wf_internal.cuh"

namespace wf {

namespace {
struct Choice {
  int syn[2], ana[2], ana_queue, syn_x2, ana_x2, ana_gacc;
  float syn_ms[2][6], ana_ms[2][15];  // the timings the choice was made from
};
std::mutex g_tune_mu;
std::map<std::pair<int, int>, Choice> g_tune_cache;
}  // namespace

template <typename T2>
static wf_status time_synth(Plan &P, T2 *xs, T2 *F, cudaEvent_t e0, cudaEvent_t e1,
                            float *ms) {
  WF_TRY(launch_legendre_synth<T2>(P, xs, F, nullptr, P.lmax));  // warm
  WF_CUDA(cudaEventRecord(e0, P.stream));
  for (int r = 0; r < 2; ++r) WF_TRY(launch_legendre_synth<T2>(P, xs, F, nullptr, P.lmax));
  WF_CUDA(cudaEventRecord(e1, P.stream));
  WF_CUDA(cudaEventSynchronize(e1));
  WF_CUDA(cudaEventElapsedTime(ms, e0, e1));
  return WF_OK;
}

template <typename T2>
static wf_status time_anal(Plan &P, T2 *G, cudaEvent_t e0, cudaEvent_t e1, float *ms) {
  WF_TRY(launch_legendre_anal<T2>(P, G, P.xtmp, nullptr, ANA_PLAIN, P.lmax));
  WF_CUDA(cudaEventRecord(e0, P.stream));
  for (int r = 0; r < 2; ++r)
    WF_TRY(launch_legendre_anal<T2>(P, G, P.xtmp, nullptr, ANA_PLAIN, P.lmax));
  WF_CUDA(cudaEventRecord(e1, P.stream));
  WF_CUDA(cudaEventSynchronize(e1));
  WF_CUDA(cudaEventElapsedTime(ms, e0, e1));
  return WF_OK;
}

wf_status autotune(Plan &P) {
  const std::pair<int, int> key(P.nside, P.lmax);
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      for (int k = 0; k < 2; ++k) {
        P.syn_np[k] = it->second.syn[k];
        P.ana_np[k] = it->second.ana[k];
      }
      P.ana_queue = it->second.ana_queue;
      P.syn_x2 = it->second.syn_x2;
      P.ana_x2 = it->second.ana_x2;
      P.ana_gacc = it->second.ana_gacc;
      memcpy(P.tune_syn_ms, it->second.syn_ms, sizeof(P.tune_syn_ms));
      memcpy(P.tune_ana_ms, it->second.ana_ms, sizeof(P.tune_ana_ms));
      return WF_OK;
    }
  }
  // inputs are zeros: the kernels' work does not depend on the values
  WF_CUDA(cudaMemsetAsync(P.xs32, 0, sizeof(float2) * P.nalm, P.stream));
  WF_CUDA(cudaMemsetAsync(P.xs64, 0, sizeof(double2) * P.nalm, P.stream));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  WF_CUDA(cudaEventCreate(&e0));
  WF_CUDA(cudaEventCreate(&e1));
  static const int syn_cand[3] = {1, 2, 4};
  static const int ana_cand32[4] = {2, 4, 8, 16};
  static const int ana_cand64[3] = {2, 4, 8};
  wf_status st = WF_OK;
  for (int k = 0; k < 2 && st == WF_OK; ++k) {  // 0 = FP64, 1 = FP32
    float best = 1e30f;
    int pick = P.syn_np[k];
    int pick_x2 = 0;
    // FP32 also tries the packed f32x2 synthesis with 2 and 4 pairs (slots
    // 3, 4) and with duplicated tables and 2 pairs (slot 5)
    const int nsyn = k ? 6 : 3;
    for (int ci = 0; ci < nsyn; ++ci) {
      const bool x2 = ci >= 3;
      const int c = x2 ? (ci == 4 ? 4 : 2) : syn_cand[ci];
      P.syn_np[k] = c;
      if (k) P.syn_x2 = ci == 5 ? 2 : (x2 ? 1 : 0);
      float ms = 0.f;
      st = k ? time_synth<float2>(P, P.xs32, P.F32, e0, e1, &ms)
             : time_synth<double2>(P, P.xs64, P.F64, e0, e1, &ms);
      if (st != WF_OK) break;
      P.tune_syn_ms[k][ci] = ms;
      if (ms < best) {
        best = ms;
        pick = c;
        pick_x2 = ci == 5 ? 2 : (x2 ? 1 : 0);
      }
    }
    if (k) P.syn_x2 = pick_x2;
    P.syn_np[k] = pick;
    best = 1e30f;
    pick = P.ana_np[k];
    int pick_q = 0, pick_ax2 = 0, pick_ga = 0;
    const int *cand = k ? ana_cand32 : ana_cand64;
    const int nc = k ? 4 : 3;
    // FP32 also tries the queue-scheduled analysis (slots 4, 5: 4 and 8
    // pairs per lane), the packed f32x2 one (slots 6, 7, 8: 4, 8, 6), the
    // packed one with global accumulators (slots 9, 10: 4, 6) and the same
    // with 8-l chunks (slots 11, 12, 13: 8, 6, 4), the last also with the
    // seeds in shared memory (slot 14: 8)
    const int ntot = k ? 15 : 3;
    static const int x2_np[9] = {4, 8, 6, 4, 6, 8, 6, 4, 8};
    for (int i = 0; i < ntot && st == WF_OK; ++i) {
      const bool q = k && i >= 4 && i < 6, x2 = k && i >= 6, ga = k && i >= 9;
      P.ana_queue = q ? 1 : 0;
      P.ana_x2 = x2 ? 1 : 0;
      P.ana_gacc = ga ? (i >= 14 ? 3 : i >= 11 ? 2 : 1) : 0;
      P.ana_np[k] = q ? ((i & 1) ? 8 : 4) : x2 ? x2_np[i - 6] : cand[i];
      float ms = 0.f;
      st = k ? time_anal<float2>(P, P.G32, e0, e1, &ms)
             : time_anal<double2>(P, P.G64, e0, e1, &ms);
      if (st == WF_OK) P.tune_ana_ms[k][i] = ms;
      if (st == WF_OK && ms < best) {
        best = ms;
        pick = P.ana_np[k];
        pick_q = P.ana_queue;
        pick_ax2 = P.ana_x2;
        pick_ga = P.ana_gacc;
      }
    }
    P.ana_np[k] = pick;
    P.ana_queue = k ? pick_q : P.ana_queue;
    P.ana_x2 = k ? pick_ax2 : P.ana_x2;
    P.ana_gacc = k ? pick_ga : P.ana_gacc;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != WF_OK) return st;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  Choice c;
  for (int k = 0; k < 2; ++k) {
    c.syn[k] = P.syn_np[k];
    c.ana[k] = P.ana_np[k];
  }
  c.ana_queue = P.ana_queue;
  c.syn_x2 = P.syn_x2;
  c.ana_x2 = P.ana_x2;
  c.ana_gacc = P.ana_gacc;
  memcpy(c.syn_ms, P.tune_syn_ms, sizeof(c.syn_ms));
  memcpy(c.ana_ms, P.tune_ana_ms, sizeof(c.ana_ms));
  g_tune_cache[key] = c;
  return WF_OK;
}

}  // namespace wf
