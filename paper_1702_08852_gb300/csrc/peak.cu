// peak.cu -- measured peak of the non-tensor arithmetic pipes, the
// denominators of the Legendre kernels' rooflines.
//
// The Legendre recurrence and contraction run on the FP32 (mixed solver) or
// FP64 (plain solver) FMA pipe, not on the tensor cores, so their roofline is
// the rate at which this GPU retires fused multiply-adds.  Each kernel below
// runs independent FMA chains in every thread of a grid that fills every SM
// (CHAINS chains per thread hide the pipe latency); the rate is 2 flops per
// FMA (4 per packed f32x2 instruction) over the CUDA-event time of the
// fastest of `reps` launches.
#include <algorithm>

#include "wf_internal.cuh"

namespace wf {

constexpr int PEAK_THREADS = 256;
constexpr int PEAK_CHAINS = 8;

template <typename T>
__global__ void __launch_bounds__(PEAK_THREADS)
    k_fma_chains(T *out, int iters, T a, T b) {
  T acc[PEAK_CHAINS];
#pragma unroll
  for (int c = 0; c < PEAK_CHAINS; ++c) acc[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < PEAK_CHAINS; ++c) acc[c] = fma(acc[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < PEAK_CHAINS; ++c) s += acc[c];
  out[(long)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// packed FP32 pairs: one fma.rn.f32x2 performs two FMAs
__global__ void __launch_bounds__(PEAK_THREADS)
    k_fma2_chains(float *out, int iters, float a, float b) {
  unsigned long long acc[PEAK_CHAINS];
  unsigned long long ra, rb;
  asm("mov.b64 %0, {%1, %1};" : "=l"(ra) : "f"(a));
  asm("mov.b64 %0, {%1, %1};" : "=l"(rb) : "f"(b));
#pragma unroll
  for (int c = 0; c < PEAK_CHAINS; ++c) {
    const float x = (float)(threadIdx.x + c) * 1e-3f, y = x + 0.5f;
    asm("mov.b64 %0, {%1, %2};" : "=l"(acc[c]) : "f"(x), "f"(y));
  }
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < PEAK_CHAINS; ++c)
      asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(acc[c]) : "l"(ra), "l"(rb));
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < PEAK_CHAINS; ++c) {
    float x, y;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(acc[c]));
    s += x + y;
  }
  out[(long)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace wf

using namespace wf;

extern "C" wf_status wf_alu_peak(int kind, int reps, double *tflops, double *best_ms,
                                 int *num_sms) {
  if (kind < 0 || kind > 2 || reps < 1 || reps > 100 || !tflops) {
    set_error("wf_alu_peak: kind must be 0, 1 or 2, reps 1..100, tflops not NULL");
    return WF_ERR_ARG;
  }
  int dev = 0, sms = 0, per_sm = 0;
  WF_CUDA(cudaGetDevice(&dev));
  WF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (kind == 0)
    WF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_chains<double>,
                                                          PEAK_THREADS, 0));
  else if (kind == 1)
    WF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_chains<float>,
                                                          PEAK_THREADS, 0));
  else
    WF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma2_chains,
                                                          PEAK_THREADS, 0));
  per_sm = std::max(1, per_sm);
  const int blocks = sms * per_sm;
  const long threads = (long)blocks * PEAK_THREADS;
  // ~0.05 s per launch at the nominal rates (FP64 ~1/64 of FP32)
  const int iters = kind == 0 ? 2048 : 65536;
  void *out = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  WF_CUDA(cudaMalloc(&out, sizeof(double) * threads));
  wf_status st = WF_OK;
  float best = 0.f;
  do {
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
      set_error("wf_alu_peak: stream or event creation failed");
      st = WF_ERR_CUDA;
      break;
    }
    auto launch = [&](int it) {
      if (kind == 0)
        k_fma_chains<double><<<blocks, PEAK_THREADS, 0, s>>>(static_cast<double *>(out), it,
                                                             0.999999, 1e-7);
      else if (kind == 1)
        k_fma_chains<float><<<blocks, PEAK_THREADS, 0, s>>>(static_cast<float *>(out), it,
                                                            0.999999f, 1e-7f);
      else
        k_fma2_chains<<<blocks, PEAK_THREADS, 0, s>>>(static_cast<float *>(out), it,
                                                      0.999999f, 1e-7f);
    };
    launch(iters / 16);  // warm-up
    for (int r = 0; r < reps && st == WF_OK; ++r) {
      cudaEventRecord(e0, s);
      launch(iters);
      cudaEventRecord(e1, s);
      cudaError_t e = cudaEventSynchronize(e1);
      if (e == cudaSuccess) e = cudaGetLastError();
      if (e != cudaSuccess) {
        set_error(std::string("wf_alu_peak: ") + cudaGetErrorString(e));
        st = WF_ERR_CUDA;
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (r == 0 || ms < best) best = ms;
    }
  } while (0);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  cudaFree(out);
  if (st != WF_OK) return st;
  const double fmas = (double)threads * iters * PEAK_CHAINS * (kind == 2 ? 2.0 : 1.0);
  *tflops = 2.0 * fmas / (best * 1e-3) / 1e12;
  if (best_ms) *best_ms = best;
  if (num_sms) *num_sms = sms;
  return WF_OK;
}
