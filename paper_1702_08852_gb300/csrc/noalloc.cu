// noalloc.cu -- wf_residual_static: the diagnostics of wf_residual computed
// without allocating any memory during the call.
//
// wf_residual takes its temporary maps and coefficient arrays from
// cudaMalloc on every call.  Some callers cannot do that: code that runs
// under a fixed device-memory budget, or inside a framework whose pool
// allocator owns the device memory, where a cudaMalloc can fail or take
// memory the pool counts on; and loops with a time budget per pass, where
// cudaMalloc / cudaFree may synchronise the device and stall.  For them this
// variant takes every temporary from one statically sized device array
// defined in this file.  The plan itself (created beforehand, when allocating
// is allowed) still provides its own workspaces.
//
// The call is host-synchronous: it waits for the plan's stream and returns
// its three diagnostics as host scalars.
//
// The array is a file-scope __device__ variable: each GPU that loads the
// library holds it (STATIC_SCRATCH_DOUBLES doubles, 4.8 MB) until the process
// exits.  Host code cannot use the variable's name as a device address, so the
// address is looked up with cudaGetSymbolAddress once per device, by the first
// call on that device; make that first call before any stream capture.  All
// calls share the array: calls that overlap on the GPU (other streams, other
// host threads) race on it.  The call also writes the plan's own workspaces
// (state, data map, ring coefficients, alm buffers, partial sums), so it must
// not overlap any other call on the same plan either.  Nothing in the array
// needs to start at zero: every slot is written before it is read within a
// call.
#include <math.h>

#include <mutex>

#include "wf_internal.cuh"

namespace wf {

// 2 Npix + 6 Nalm + 3 (lmax + 1) + 256 doubles must fit; e.g. Nside 128 with
// lmax 256 needs 592,905.
constexpr size_t STATIC_SCRATCH_DOUBLES = 600000;
static __device__ __align__(256) double g_residual_scratch[STATIC_SCRATCH_DOUBLES];

constexpr int STATIC_RED_BLOCKS = 256;
constexpr int STATIC_MAX_DEVICES = 64;
static std::mutex g_scratch_mu;
static double *g_scratch_ptr[STATIC_MAX_DEVICES] = {nullptr};

// device address of the array on the current device (looked up once)
static wf_status scratch_address(double **out) {
  int dev = -1;
  WF_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= STATIC_MAX_DEVICES) {
    set_error_static("wf_residual_static: device index out of range");
    return WF_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_residual_scratch);
    if (e != cudaSuccess || !p) {
      set_error_static("wf_residual_static: cudaGetSymbolAddress failed for the "
                       "static scratch array");
      return WF_ERR_CUDA;
    }
    g_scratch_ptr[dev] = static_cast<double *>(p);
  }
  *out = g_scratch_ptr[dev];
  return WF_OK;
}

// C^-1/2 (0 where C = 0), C^1/2 and C^1/2 / Omega, per l
__global__ void k_cl_factors(const double *cl, int lmax, double omega, double *cm12,
                             double *cp12, double *cpo) {
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l <= lmax;
       l += gridDim.x * blockDim.x) {
    const double c = cl[l];
    const double r = sqrt(c);
    cm12[l] = c > 0.0 ? 1.0 / r : 0.0;
    cp12[l] = r;
    cpo[l] = r / omega;
  }
}

// fixed-order host sum of n block partials copied into a stack buffer
static wf_status sum_partials(Plan &P, const double *dev, int n, double *res) {
  double h[STATIC_RED_BLOCKS];
  WF_CUDA(cudaMemcpyAsync(h, dev, sizeof(double) * n, cudaMemcpyDeviceToHost, P.stream));
  WF_CUDA(cudaStreamSynchronize(P.stream));
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += h[i];
  *res = s;
  return WF_OK;
}

static wf_status dot_static(Plan &P, const double2 *a, const double2 *b,
                            const double *fl, double *red, double *res) {
  ++P.nlaunch;
  k_alm_dot<<<STATIC_RED_BLOCKS, 256, 0, P.stream>>>(a, b, fl, P.lmax, red);
  WF_CUDA(cudaGetLastError());
  return sum_partials(P, red, STATIC_RED_BLOCKS, res);
}

wf_status residual_static(Plan &P, const double *d, const double *alm, double *res_wf,
                          double *res_fp, double *chi2) {
  if (!P.has_noise) {
    set_error_static("wf_residual_static: plan has no noise variance");
    return WF_ERR_STATE;
  }
  const size_t need = 2 * (size_t)P.npix + 6 * (size_t)P.nalm + 3 * (size_t)(P.lmax + 1) +
                      STATIC_RED_BLOCKS;
  if (need > STATIC_SCRATCH_DOUBLES) {
    set_error_static("wf_residual_static: plan too large for the static scratch array "
                     "(2 Npix + 6 Nalm + 3 (lmax+1) + 256 doubles must fit in 600000); "
                     "use wf_residual, which allocates");
    return WF_ERR_ARG;
  }
  int dev = -1;
  WF_CUDA(cudaGetDevice(&dev));
  if (dev != P.device) {
    set_error_static("wf_residual_static: the current device is not the plan's device");
    return WF_ERR_STATE;
  }
  double *base = nullptr;
  WF_TRY(scratch_address(&base));
  double *pr = base;                                        // N^-1 (d - s)
  double *py = pr + P.npix;                                 // N^-1 d
  double2 *u = reinterpret_cast<double2 *>(py + P.npix);    // Omega Y^T pr
  double2 *v = u + P.nalm;                                  // Omega Y^T py
  double2 *rr = v + P.nalm;                                 // App. C residual
  double *cm12 = reinterpret_cast<double *>(rr + P.nalm);
  double *cp12 = cm12 + (P.lmax + 1);
  double *cpo = cp12 + (P.lmax + 1);
  double *red = cpo + (P.lmax + 1);
  const double2 *x = reinterpret_cast<const double2 *>(alm);

  ++P.nlaunch;
  k_mask_data<<<304, 256, 0, P.stream>>>(d, P.nvar, P.npix, P.dmap);
  WF_CUDA(cudaGetLastError());
  WF_TRY(alm2map(P, alm, P.mtmp));
  ++P.nlaunch;
  k_pix_resid<<<STATIC_RED_BLOCKS, 256, 0, P.stream>>>(P.dmap, P.mtmp, P.nvar, P.npix, pr,
                                                       py, red);
  WF_CUDA(cudaGetLastError());
  double chi_pix = 0.0;
  WF_TRY(sum_partials(P, red, STATIC_RED_BLOCKS, &chi_pix));
  ++P.nlaunch;
  k_cl_factors<<<(P.lmax + 256) / 256, 256, 0, P.stream>>>(P.cl_d, P.lmax, P.omega, cm12,
                                                          cp12, cpo);
  WF_CUDA(cudaGetLastError());
  double prior = 0.0;
  WF_TRY(dot_static(P, x, x, cm12, red, &prior));
  if (chi2) *chi2 = chi_pix + prior;
  WF_TRY(map2alm(P, pr, reinterpret_cast<double *>(u)));
  WF_TRY(map2alm(P, py, reinterpret_cast<double *>(v)));
  ++P.nlaunch;
  k_alm_combine<<<P.lmax + 1, 128, 0, P.stream>>>(x, u, cm12, cpo, P.lmax, rr);
  WF_CUDA(cudaGetLastError());
  double rn = 0.0, yn = 0.0;
  WF_TRY(dot_static(P, rr, rr, nullptr, red, &rn));
  WF_TRY(dot_static(P, v, v, cpo, red, &yn));
  if (res_wf) *res_wf = yn > 0 ? sqrt(rn / yn) : 0.0;
  if (res_fp) {
    // one last-stage iteration G(x) (xi = alpha, mu = 0, full band) into the
    // plan's own workspaces; ||G(x) - x||^2 from the per-m partial sums
    SolverState s = initial_state(P);
    s.xi = P.alpha;
    s.mu = 0.0;
    s.lcur = s.lnext = P.lmax;
    s.done = 0;
    *P.state_h = s;
    WF_CUDA(cudaMemcpyAsync(P.state, P.state_h, sizeof(SolverState),
                            cudaMemcpyHostToDevice, P.stream));
    WF_CUDA(cudaMemcpyAsync(P.xtmp, x, sizeof(double2) * P.nalm, cudaMemcpyDeviceToDevice,
                            P.stream));
    WF_TRY(launch_prescale<double2>(P, x, P.xs64));
    WF_TRY(launch_legendre_synth<double2>(P, P.xs64, P.F64, nullptr, P.lmax));
    WF_TRY(launch_ring<double2>(P, RING_FUSED, P.F64, P.G64, P.dmap, nullptr, P.state,
                                P.lmax));
    WF_TRY(launch_legendre_anal<double2>(P, P.G64, P.xtmp, P.state, ANA_FILTER, P.lmax));
    // partials[2m] = ||G(x) - x||^2 over m: lmax + 1 <= 257 entries here
    double part[2 * 512];
    const int np = 2 * (P.lmax + 1);
    if (np > 2 * 512) {
      set_error_static("wf_residual_static: lmax too large for the static path");
      return WF_ERR_ARG;
    }
    WF_CUDA(cudaMemcpyAsync(part, P.partials, sizeof(double) * np, cudaMemcpyDeviceToHost,
                            P.stream));
    double xn = 0.0;
    WF_TRY(dot_static(P, x, x, nullptr, red, &xn));
    double num = 0.0;
    for (int m = 0; m <= P.lmax; ++m) num += part[2 * m];
    *res_fp = xn > 0 ? sqrt(num / xn) : 0.0;
  }
  WF_CUDA(cudaStreamSynchronize(P.stream));
  return WF_OK;
}

}  // namespace wf
