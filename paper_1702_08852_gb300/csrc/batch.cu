// batch.cu -- many independent Wiener-filter problems solved together.
//
// Each map keeps its own plan (geometry, noise, mask, spectrum, captured
// iteration graphs, device-side stage control).  A batch run gives every map
// a private non-blocking stream; a pool of host threads, one per hardware
// thread at most, takes maps from a queue (largest first) and drives each
// one's solve, so the small per-map kernels of maps with Nside 64-256
// execute concurrently and fill the GPU, while no more threads wait on the
// GPU than there are cores to run them; maps of different sizes and
// convergence speeds finish independently.  Results are identical to solving
// the maps one by one (each map's arithmetic does not depend on the
// others).
#include <algorithm>
#include <atomic>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "wf_internal.cuh"

namespace wf {

wf_status solve_batch(Plan **plans, int n, const double *const *d, double *const *alm,
                      double *const *map, wf_stats *stats, double *wall_ms) {
  std::vector<cudaStream_t> own(n, nullptr), keep(n, nullptr);
  for (int i = 0; i < n; ++i) {
    keep[i] = plans[i]->stream;
    cudaError_t e = cudaStreamCreateWithFlags(&own[i], cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      for (int j = 0; j < i; ++j) cudaStreamDestroy(own[j]);
      set_error(std::string("wf_solve_batch: cudaStreamCreate: ") + cudaGetErrorString(e));
      return WF_ERR_CUDA;
    }
  }
  // work already queued on the callers' streams comes first
  for (int i = 0; i < n; ++i) {
    cudaError_t e = cudaStreamSynchronize(keep[i]);
    if (e != cudaSuccess) {
      for (int j = 0; j < n; ++j) cudaStreamDestroy(own[j]);
      set_error(std::string("wf_solve_batch: ") + cudaGetErrorString(e));
      return WF_ERR_CUDA;
    }
    plans[i]->stream = own[i];
  }
  int dev = 0;
  cudaGetDevice(&dev);
  std::vector<wf_status> status(n, WF_OK);
  std::vector<std::string> msg(n);
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  const bool timed = cudaEventCreate(&t0) == cudaSuccess && cudaEventCreate(&t1) == cudaSuccess;
  if (timed) cudaEventRecord(t0, nullptr);
  for (int i = 0; i < n; ++i) cudaStreamWaitEvent(own[i], t0, 0);
  // largest maps first, so that the longest solves start at once
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return plans[a]->npix > plans[b]->npix; });
  const int hw = (int)std::thread::hardware_concurrency();
  const int nthreads = std::max(1, std::min(n, hw > 0 ? hw : n));
  std::atomic<int> next(0);
  std::vector<std::thread> threads;
  threads.reserve(nthreads);
  for (int w = 0; w < nthreads; ++w) {
    threads.emplace_back([&]() {
      cudaSetDevice(dev);
      for (int q = next.fetch_add(1); q < n; q = next.fetch_add(1)) {
        const int i = order[q];
        status[i] = solve(*plans[i], d[i], alm ? alm[i] : nullptr, map ? map[i] : nullptr,
                          nullptr, nullptr, stats ? &stats[i] : nullptr);
        if (status[i] != WF_OK) msg[i] = wf_last_error();
      }
    });
  }
  for (auto &t : threads) t.join();
  // the batch ends when the last map's stream is done
  for (int i = 0; i < n; ++i) {
    cudaEvent_t ev = nullptr;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess) {
      cudaEventRecord(ev, own[i]);
      cudaStreamWaitEvent(nullptr, ev, 0);
      cudaEventDestroy(ev);
    }
  }
  if (timed) {
    cudaEventRecord(t1, nullptr);
    cudaEventSynchronize(t1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, t0, t1);
    if (wall_ms) *wall_ms = ms;
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
  }
  for (int i = 0; i < n; ++i) {
    cudaStreamSynchronize(own[i]);
    plans[i]->stream = keep[i];
    cudaStreamDestroy(own[i]);
  }
  wf_status first = WF_OK;
  for (int i = 0; i < n; ++i)
    if (status[i] != WF_OK && status[i] != WF_ERR_NOT_CONVERGED) {
      set_error("wf_solve_batch: map " + std::to_string(i) + ": " + msg[i]);
      return status[i];
    }
  for (int i = 0; i < n; ++i)
    if (status[i] == WF_ERR_NOT_CONVERGED) {
      set_error("wf_solve_batch: map " + std::to_string(i) + ": " + msg[i]);
      first = WF_ERR_NOT_CONVERGED;
      break;
    }
  return first;
}

}  // namespace wf
