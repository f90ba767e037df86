// pcg.cu -- the Wiener filter by preconditioned conjugate gradients (App. C),
// the paper's comparison method, on the FP64 transforms of this library.
//
// System (App. C on the sphere): A z = y with
//   A = 1 + C^1/2 Y^T N^-1 Y C^1/2,   y = C^1/2 Y^T N^-1 d,   s_WF = C^1/2 z,
// Y^T = (Omega Y^T) / Omega from the analysis transform, N^-1 = 0 on masked
// pixels.  Preconditioner (App. C): diagonal in the harmonic basis, the
// diagonal of A, M^-1_ll = 1 + C_l sum_p N^-1_p / (4 pi) (|Y_lm|^2 averages
// 1 / (4 pi) over the sphere; the printed flat-sky form (sum_k n_k) C_l / L^4
// leaves out the identity's 1).  Restarted every `restart` iterations as the
// paper describes (r recomputed from z).  Stop rules: the paper's
// ||z_{i+1} - z_i|| / ||z_{i+1}|| < tol, or the relative residual
// ||A z - y|| / ||y|| < tol of Fig. 5.
//
// One iteration: alm2map of C^1/2 p, a pixel multiply by N^-1, map2alm, an
// alm combine (fused with the p.Ap partial sums), the z / r / q updates
// (fused with the r.r, r.q, p.p, z.z partial sums), the new direction.  The
// scalars are reduced on the host from fixed-order block partials.
#include <math.h>

#include <algorithm>
#include <vector>

#include "wf_internal.cuh"

namespace wf {

constexpr int CG_BLOCKS = 256;
constexpr int CG_THREADS = 256;

// real-basis weights of a complex m-major alm: 1 for m = 0, 2 for m > 0
__device__ __forceinline__ double alm_w(int m) { return m == 0 ? 1.0 : 2.0; }

// block partial sums of up to 4 values -> out[4 * block + j]
template <int K>
__device__ __forceinline__ void block_sums(double (&v)[K], double *out) {
  __shared__ double sh[K][CG_THREADS];
#pragma unroll
  for (int j = 0; j < K; ++j) sh[j][threadIdx.x] = v[j];
  __syncthreads();
  for (int s = CG_THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
#pragma unroll
      for (int j = 0; j < K; ++j) sh[j][threadIdx.x] += sh[j][threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < K; ++j) out[4 * blockIdx.x + j] = sh[j][0];
  }
}

// w = sq_l v (sq = C^1/2)
__global__ void k_cg_scale(const double2 *__restrict__ v, const double *__restrict__ sq,
                           int lmax, double2 *__restrict__ w) {
  for (int m = blockIdx.x; m <= lmax; m += gridDim.x) {
    const long base = (long)m * (2 * lmax + 1 - m) / 2;
    for (int l = m + threadIdx.x; l <= lmax; l += blockDim.x) {
      const double s = sq[l];
      const double2 a = v[base + l];
      w[base + l] = make_double2(s * a.x, s * a.y);
    }
  }
}

// map <- map / sigma^2 (sigma^2 = +inf on masked pixels gives 0); with
// d != NULL: map <- d / sigma^2 (the right-hand side)
__global__ void k_cg_ninv(double *__restrict__ map, const double *__restrict__ d,
                          const double *__restrict__ nvar, long npix) {
  for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < npix;
       p += (long)gridDim.x * blockDim.x) {
    const double v = nvar[p];
    const double x = d ? d[p] : map[p];
    map[p] = isinf(v) ? 0.0 : x / v;
  }
}

// out = v + (sq_l / Omega) u; partial sums of v . out
__global__ void __launch_bounds__(CG_THREADS)
    k_cg_apply(const double2 *__restrict__ v, const double2 *__restrict__ u,
               const double *__restrict__ sqo, int lmax, int add_v, double2 *__restrict__ out,
               double *__restrict__ part) {
  double acc[1] = {0.0};
  for (int m = blockIdx.x; m <= lmax; m += gridDim.x) {
    const long base = (long)m * (2 * lmax + 1 - m) / 2;
    const double wm = alm_w(m);
    for (int l = m + threadIdx.x; l <= lmax; l += blockDim.x) {
      const long i = base + l;
      const double s = sqo[l];
      const double2 a = add_v ? v[i] : make_double2(0.0, 0.0);
      const double2 o = make_double2(a.x + s * u[i].x, a.y + s * u[i].y);
      out[i] = o;
      if (add_v) acc[0] += wm * (a.x * o.x + a.y * o.y);
    }
  }
  block_sums<1>(acc, part);
}

// z += alpha p; r -= alpha Ap; q = r / pdiag_l; partials r.r, r.q, p.p, z.z
__global__ void __launch_bounds__(CG_THREADS)
    k_cg_update(double2 *__restrict__ z, double2 *__restrict__ r, double2 *__restrict__ q,
                const double2 *__restrict__ p, const double2 *__restrict__ ap,
                const double *__restrict__ pdiag, double alpha, int lmax,
                double *__restrict__ part) {
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int m = blockIdx.x; m <= lmax; m += gridDim.x) {
    const long base = (long)m * (2 * lmax + 1 - m) / 2;
    const double wm = alm_w(m);
    for (int l = m + threadIdx.x; l <= lmax; l += blockDim.x) {
      const long i = base + l;
      const double2 pv = p[i];
      const double2 zv = make_double2(z[i].x + alpha * pv.x, z[i].y + alpha * pv.y);
      const double2 rv = make_double2(r[i].x - alpha * ap[i].x, r[i].y - alpha * ap[i].y);
      const double ip = 1.0 / pdiag[l];
      const double2 qv = make_double2(rv.x * ip, rv.y * ip);
      z[i] = zv;
      r[i] = rv;
      q[i] = qv;
      acc[0] += wm * (rv.x * rv.x + rv.y * rv.y);
      acc[1] += wm * (rv.x * qv.x + rv.y * qv.y);
      acc[2] += wm * (pv.x * pv.x + pv.y * pv.y);
      acc[3] += wm * (zv.x * zv.x + zv.y * zv.y);
    }
  }
  block_sums<4>(acc, part);
}

// restart: r = y - Az (az NULL: z = 0), q = p = r / pdiag; partials r.r, r.q
__global__ void __launch_bounds__(CG_THREADS)
    k_cg_restart(const double2 *__restrict__ y, const double2 *__restrict__ az,
                 const double *__restrict__ pdiag, int lmax, double2 *__restrict__ r,
                 double2 *__restrict__ q, double2 *__restrict__ p, double *__restrict__ part) {
  double acc[2] = {0.0, 0.0};
  for (int m = blockIdx.x; m <= lmax; m += gridDim.x) {
    const long base = (long)m * (2 * lmax + 1 - m) / 2;
    const double wm = alm_w(m);
    for (int l = m + threadIdx.x; l <= lmax; l += blockDim.x) {
      const long i = base + l;
      const double2 a = az ? az[i] : make_double2(0.0, 0.0);
      const double2 rv = make_double2(y[i].x - a.x, y[i].y - a.y);
      const double ip = 1.0 / pdiag[l];
      const double2 qv = make_double2(rv.x * ip, rv.y * ip);
      r[i] = rv;
      q[i] = qv;
      p[i] = qv;
      acc[0] += wm * (rv.x * rv.x + rv.y * rv.y);
      acc[1] += wm * (rv.x * qv.x + rv.y * qv.y);
    }
  }
  block_sums<2>(acc, part);
}

// p = q + beta p
__global__ void k_cg_direction(double2 *__restrict__ p, const double2 *__restrict__ q,
                               double beta, long n) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long)gridDim.x * blockDim.x)
    p[i] = make_double2(q[i].x + beta * p[i].x, q[i].y + beta * p[i].y);
}

// sum of N^-1 over the pixels (block partials)
__global__ void __launch_bounds__(CG_THREADS)
    k_cg_ninv_sum(const double *__restrict__ nvar, long npix, double *__restrict__ part) {
  double acc[1] = {0.0};
  for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < npix;
       p += (long)gridDim.x * blockDim.x) {
    const double v = nvar[p];
    if (!isinf(v)) acc[0] += 1.0 / v;
  }
  block_sums<1>(acc, part);
}

namespace {

struct Cg {
  Plan &P;
  std::vector<double> hpart;
  double *part = nullptr;     // [4 * CG_BLOCKS]
  double *sq = nullptr, *sqo = nullptr, *pdiag = nullptr;  // [lmax + 1]
  double2 *y = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *ap = nullptr,
          *w = nullptr;       // [nalm]
  explicit Cg(Plan &P_) : P(P_), hpart(4 * CG_BLOCKS) {}
  ~Cg() {
    void *b[] = {part, sq, sqo, pdiag, y, r, p, q, ap, w};
    for (void *x : b)
      if (x) cudaFree(x);
  }
  wf_status alloc() {
    WF_CUDA(cudaMalloc(&part, sizeof(double) * 4 * CG_BLOCKS));
    for (double **a : {&sq, &sqo, &pdiag})
      WF_CUDA(cudaMalloc(a, sizeof(double) * (P.lmax + 1)));
    for (double2 **a : {&y, &r, &p, &q, &ap, &w})
      WF_CUDA(cudaMalloc(a, sizeof(double2) * P.nalm));
    return WF_OK;
  }
  // sums of the first k block partial values (fixed order)
  wf_status sums(int k, double *out) {
    WF_CUDA(cudaMemcpyAsync(hpart.data(), part, sizeof(double) * 4 * CG_BLOCKS,
                            cudaMemcpyDeviceToHost, P.stream));
    WF_CUDA(cudaStreamSynchronize(P.stream));
    for (int j = 0; j < k; ++j) out[j] = 0.0;
    for (int b = 0; b < CG_BLOCKS; ++b)
      for (int j = 0; j < k; ++j) out[j] += hpart[4 * b + j];
    return WF_OK;
  }
  // out = A v (add_v) or C^1/2 Y^T N^-1 Y C^1/2 v; partial v . out
  wf_status apply(const double2 *v, double2 *out, double *vav) {
    ++P.nlaunch;
    k_cg_scale<<<CG_BLOCKS, CG_THREADS, 0, P.stream>>>(v, sq, P.lmax, w);
    WF_CUDA(cudaGetLastError());
    WF_TRY(alm2map(P, reinterpret_cast<const double *>(w), P.mtmp));
    ++P.nlaunch;
    k_cg_ninv<<<304, 256, 0, P.stream>>>(P.mtmp, nullptr, P.nvar, P.npix);
    WF_CUDA(cudaGetLastError());
    WF_TRY(map2alm(P, P.mtmp, reinterpret_cast<double *>(w)));
    ++P.nlaunch;
    k_cg_apply<<<CG_BLOCKS, CG_THREADS, 0, P.stream>>>(v, w, sqo, P.lmax, 1, out, part);
    WF_CUDA(cudaGetLastError());
    if (vav) WF_TRY(sums(1, vav));
    return WF_OK;
  }
};

}  // namespace

wf_status pcg(Plan &P, const double *d, double *alm, double *map, double tol, int stop_rule,
              int max_iter, int restart, wf_stats *stats) {
  if (!P.has_noise) {
    set_error("wf_pcg: plan has no noise variance");
    return WF_ERR_STATE;
  }
  WF_CUDA(cudaEventRecord(P.ev0, P.stream));
  const long launches0 = P.nlaunch;
  Cg cg(P);
  WF_TRY(cg.alloc());
  // preconditioner and C^1/2 tables
  ++P.nlaunch;
  k_cg_ninv_sum<<<CG_BLOCKS, CG_THREADS, 0, P.stream>>>(P.nvar, P.npix, cg.part);
  WF_CUDA(cudaGetLastError());
  double ninv_sum = 0.0;
  WF_TRY(cg.sums(1, &ninv_sum));
  std::vector<double> hsq(P.lmax + 1), hsqo(P.lmax + 1), hpd(P.lmax + 1);
  for (int l = 0; l <= P.lmax; ++l) {
    hsq[l] = sqrt(P.cl[l]);
    hsqo[l] = hsq[l] / P.omega;  // C^1/2 Y^T = C^1/2 (Omega Y^T) / Omega
    hpd[l] = 1.0 + P.cl[l] * ninv_sum / (4.0 * M_PI);
  }
  WF_CUDA(cudaMemcpyAsync(cg.sq, hsq.data(), sizeof(double) * hsq.size(),
                          cudaMemcpyHostToDevice, P.stream));
  WF_CUDA(cudaMemcpyAsync(cg.sqo, hsqo.data(), sizeof(double) * hsqo.size(),
                          cudaMemcpyHostToDevice, P.stream));
  WF_CUDA(cudaMemcpyAsync(cg.pdiag, hpd.data(), sizeof(double) * hpd.size(),
                          cudaMemcpyHostToDevice, P.stream));
  // y = C^1/2 Y^T N^-1 d
  ++P.nlaunch;
  k_cg_ninv<<<304, 256, 0, P.stream>>>(P.mtmp, d, P.nvar, P.npix);
  WF_CUDA(cudaGetLastError());
  WF_TRY(map2alm(P, P.mtmp, reinterpret_cast<double *>(cg.w)));
  ++P.nlaunch;
  k_cg_apply<<<CG_BLOCKS, CG_THREADS, 0, P.stream>>>(nullptr, cg.w, cg.sqo, P.lmax, 0, cg.y,
                                                     cg.part);
  WF_CUDA(cudaGetLastError());
  double yy = 0.0;
  WF_TRY(alm_dot_host(P, cg.y, cg.y, &yy));
  const double ny = sqrt(yy);
  double2 *z = P.x;
  WF_CUDA(cudaMemsetAsync(z, 0, sizeof(double2) * P.nalm, P.stream));
  int it = 0;
  bool converged = false, first = true;
  double rel = 1.0, cauchy = 1.0;
  while (it < max_iter && ny > 0.0) {
    // restart: r = y - A z, p = q = r / pdiag
    if (!first) WF_TRY(cg.apply(z, cg.ap, nullptr));
    ++P.nlaunch;
    k_cg_restart<<<CG_BLOCKS, CG_THREADS, 0, P.stream>>>(cg.y, first ? nullptr : cg.ap,
                                                         cg.pdiag, P.lmax, cg.r, cg.q, cg.p,
                                                         cg.part);
    WF_CUDA(cudaGetLastError());
    first = false;
    double s2[2];
    WF_TRY(cg.sums(2, s2));
    double rz = s2[1];
    for (int k = 0; k < restart; ++k) {
      double pap = 0.0;
      WF_TRY(cg.apply(cg.p, cg.ap, &pap));
      if (!(pap > 0.0) || !isfinite(pap)) {
        set_error("wf_pcg: the system lost positive definiteness (p.Ap <= 0)");
        return WF_ERR_NUMERIC;
      }
      const double a = rz / pap;
      ++P.nlaunch;
      k_cg_update<<<CG_BLOCKS, CG_THREADS, 0, P.stream>>>(z, cg.r, cg.q, cg.p, cg.ap,
                                                          cg.pdiag, a, P.lmax, cg.part);
      WF_CUDA(cudaGetLastError());
      double s4[4];
      WF_TRY(cg.sums(4, s4));
      ++it;
      rel = sqrt(s4[0]) / ny;
      cauchy = s4[3] > 0.0 ? fabs(a) * sqrt(s4[2] / s4[3]) : 0.0;
      if (!isfinite(rel)) {
        set_error("wf_pcg: NaN or Inf in the iteration");
        return WF_ERR_NUMERIC;
      }
      if ((stop_rule == WF_PCG_STOP_CAUCHY ? cauchy : rel) < tol) {
        converged = true;
        break;
      }
      if (it >= max_iter) break;
      const double rz_new = s4[1];
      ++P.nlaunch;
      k_cg_direction<<<304, 256, 0, P.stream>>>(cg.p, cg.q, rz_new / rz, P.nalm);
      WF_CUDA(cudaGetLastError());
      rz = rz_new;
    }
    if (converged) break;
  }
  // s_WF = C^1/2 z
  ++P.nlaunch;
  k_cg_scale<<<CG_BLOCKS, CG_THREADS, 0, P.stream>>>(z, cg.sq, P.lmax, P.xtmp);
  WF_CUDA(cudaGetLastError());
  if (alm)
    WF_CUDA(cudaMemcpyAsync(alm, P.xtmp, sizeof(double2) * P.nalm, cudaMemcpyDeviceToDevice,
                            P.stream));
  if (map) WF_TRY(alm2map(P, reinterpret_cast<const double *>(P.xtmp), map));
  WF_CUDA(cudaEventRecord(P.ev1, P.stream));
  WF_CUDA(cudaStreamSynchronize(P.stream));
  if (stats) {
    float ms = 0.f;
    WF_CUDA(cudaEventElapsedTime(&ms, P.ev0, P.ev1));
    *stats = wf_stats{};
    stats->iterations = it;
    stats->stages = 1;
    stats->converged = converged ? 1 : 0;
    stats->alpha = P.alpha;
    stats->final_cauchy = cauchy;
    stats->err_estimate = rel;
    stats->fp_residual = rel;
    stats->elapsed_ms = ms;
    stats->kernel_launches = P.nlaunch - launches0;
  }
  if (!converged) {
    set_error("wf_pcg: max_iter reached before the stop rule was met");
    return WF_ERR_NOT_CONVERGED;
  }
  return WF_OK;
}

}  // namespace wf
