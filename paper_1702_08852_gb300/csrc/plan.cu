// plan.cu -- plan-time tables: HEALPix ring pairs, the Legendre recurrence
// coefficients, FP64 recurrence seeds, FFT twiddles and Bluestein chirps,
// and the noise variance upload/validation.
//
// Geometry: HEALPix RING scheme (Gorski et al. 2005): 4 nside - 1 rings;
// polar ring i < nside has 4i pixels at z = 1 - i^2/(3 nside^2) starting at
// phi = pi/(4i); equatorial ring nside <= i <= 2 nside has 4 nside pixels at
// z = 2 (2 nside - i)/(3 nside) starting at phi = 0 when i + nside is odd and
// at pi/(4 nside) when it is even; the south half mirrors the north.
//
// Legendre functions: lam_lm(z) (Y_lm = lam_lm(cos theta) e^{i m phi}) obey
// lam_l = a_l z lam_{l-1} - (a_l / a_{l-1}) lam_{l-2},
// a_l = sqrt((4 l^2 - 1) / (l^2 - m^2)).  The kernels run the rescaled
// variable u_l = lam_l / g_l with g_m = g_{m+1} = 1, g_l = (a_l/a_{l-1}) g_{l-2},
// which obeys u_l = c_l z u_{l-1} - u_{l-2}, c_l = a_l g_{l-1} / g_l: one
// multiply and one fused multiply-add per step.  The seed of each (m, ring)
// is the first l at which |lam_lm| reaches 2^-100, with the two values
// u_ls, u_ls+1 computed here in FP64 with an explicit power-of-two exponent
// (lam_mm = (-1)^m sqrt((2m+1)!!/(4 pi (2m)!!)) sin^m theta underflows any
// floating-point format at high m); terms below 2^-100 are dropped.
#include <math.h>

#include <algorithm>
#include <complex>
#include <vector>

#include "wf_internal.cuh"

namespace wf {

static long alm_idx(int lmax, int l, int m) {
  return (long)m * (2 * lmax + 1 - m) / 2 + l;
}
__device__ __forceinline__ long alm_idx_d(int lmax, int l, int m) {
  return (long)m * (2 * lmax + 1 - m) / 2 + l;
}

static bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }
static int next_pow2(int n) {
  int m = 1;
  while (m < n) m <<= 1;
  return m;
}

// ---------------------------------------------------------------- geometry
static void make_pairs(Plan &P) {
  const int N = P.nside;
  const long npix = P.npix;
  P.pairs_h.resize(P.npairs);
  for (int k = 0; k < P.npairs; ++k) {
    RingPair rp{};
    const int r = k + 1;  // 1-based north ring
    long ofs;
    if (r < N) {
      rp.nphi = 4 * r;
      double omz = (double)r * r / (3.0 * N * N);
      rp.z = 1.0 - omz;
      rp.sth = sqrt(omz * (2.0 - omz));
      rp.phi_num = 1;
      rp.phi_den = 4 * r;
      ofs = 2L * r * (r - 1);
    } else {
      rp.nphi = 4 * N;
      rp.z = 2.0 * (2.0 * N - r) / (3.0 * N);
      rp.sth = sqrt((1.0 - rp.z) * (1.0 + rp.z));
      if ((r + N) & 1) {
        rp.phi_num = 0;
        rp.phi_den = 1;
      } else {
        rp.phi_num = 1;
        rp.phi_den = 4 * N;
      }
      ofs = 2L * N * (N - 1) + (long)(r - N) * 4 * N;
    }
    rp.ofsN = ofs;
    rp.ringN = r - 1;
    if (r == 2 * N) {
      rp.ofsS = -1;
      rp.ringS = -1;
    } else {
      rp.ofsS = npix - ofs - rp.nphi;
      rp.ringS = 4 * N - 1 - r;  // 0-based index of ring 4N - r
    }
    rp.fftM = is_pow2(rp.nphi) ? rp.nphi : next_pow2(2 * rp.nphi - 1);
    rp.chirp_ofs = -1;
    rp.bhat_ofs = -1;
    P.pairs_h[k] = rp;
  }
}

// ---------------------------------------------------------------- FFT tables
// Host radix-2 FFT (sign -1), used once per Bluestein ring for the spectrum
// of the chirp kernel.
static void host_fft(std::vector<std::complex<double>> &a) {
  const int n = (int)a.size();
  for (int i = 1, j = 0; i < n; ++i) {
    int bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) std::swap(a[i], a[j]);
  }
  for (int len = 2; len <= n; len <<= 1) {
    for (int i = 0; i < n; i += len) {
      for (int j = 0; j < len / 2; ++j) {
        double ang = -2.0 * M_PI * (double)j / (double)len;
        std::complex<double> w(cos(ang), sin(ang));
        std::complex<double> u = a[i + j], v = a[i + j + len / 2] * w;
        a[i + j] = u + v;
        a[i + j + len / 2] = u - v;
      }
    }
  }
}

static int bitrev(int x, int bits) {
  int r = 0;
  for (int b = 0; b < bits; ++b) r |= ((x >> b) & 1) << (bits - 1 - b);
  return r;
}

// a complex FP64 table as double-float pairs (re hi, re lo, im hi, im lo)
// for the double-float ring transforms
static wf_status upload_dd(const std::vector<double2> &v, float4 **out) {
  std::vector<float4> h(v.size());
  for (size_t i = 0; i < v.size(); ++i) {
    const float rh = (float)v[i].x, ih = (float)v[i].y;
    h[i] = make_float4(rh, (float)(v[i].x - (double)rh), ih, (float)(v[i].y - (double)ih));
  }
  WF_CUDA(cudaMalloc(out, sizeof(float4) * h.size()));
  WF_CUDA(cudaMemcpy(*out, h.data(), sizeof(float4) * h.size(), cudaMemcpyHostToDevice));
  return WF_OK;
}

static wf_status make_fft_tables(Plan &P) {
  int Mmax = 2;
  long chirp_total = 0, bhat_total = 0;
  for (auto &rp : P.pairs_h) {
    Mmax = std::max(Mmax, rp.fftM);
    if (rp.fftM != rp.nphi) {
      rp.chirp_ofs = chirp_total;
      rp.bhat_ofs = bhat_total;
      chirp_total += rp.nphi;
      bhat_total += rp.fftM;
    }
  }
  P.fftMmax = Mmax;
  std::vector<double2> tw(Mmax / 2);
  std::vector<float2> tw32(Mmax / 2);
  for (int k = 0; k < Mmax / 2; ++k) {
    // angle = 2 pi k / Mmax; k / Mmax is exact in binary
    double t = (double)k / (double)Mmax;
    double c = cos(2.0 * M_PI * t), s = sin(2.0 * M_PI * t);
    tw[k] = make_double2(c, -s);
    tw32[k] = make_float2((float)c, (float)-s);
  }
  WF_CUDA(cudaMalloc(&P.tw64, sizeof(double2) * tw.size()));
  WF_CUDA(cudaMalloc(&P.tw32, sizeof(float2) * tw.size()));
  WF_CUDA(cudaMemcpy(P.tw64, tw.data(), sizeof(double2) * tw.size(),
                     cudaMemcpyHostToDevice));
  WF_CUDA(cudaMemcpy(P.tw32, tw32.data(), sizeof(float2) * tw.size(),
                     cudaMemcpyHostToDevice));
  WF_TRY(upload_dd(tw, &P.twdd));
  P.chirp_total = chirp_total;
  P.bhat_total = bhat_total;
  if (chirp_total > 0) {
    std::vector<double2> ch(chirp_total), bh(bhat_total);
    std::vector<float2> ch32(chirp_total), bh32(bhat_total);
    for (auto &rp : P.pairs_h) {
      if (rp.chirp_ofs < 0) continue;
      const int n = rp.nphi, M = rp.fftM;
      int bits = 0;
      while ((1 << bits) < M) ++bits;
      std::vector<std::complex<double>> w(n), b(M, 0.0);
      for (int j = 0; j < n; ++j) {
        long long q = ((long long)j * j) % (2LL * n);  // exact reduction
        double ang = M_PI * (double)q / (double)n;
        w[j] = std::complex<double>(cos(ang), sin(ang));
        ch[rp.chirp_ofs + j] = make_double2(w[j].real(), w[j].imag());
        ch32[rp.chirp_ofs + j] =
            make_float2((float)w[j].real(), (float)w[j].imag());
      }
      for (int j = 0; j < n; ++j) b[j] = w[j];
      for (int j = 1; j < n; ++j) b[M - j] = w[j];
      host_fft(b);
      for (int k = 0; k < M; ++k) {
        // stored in bit-reversed order and scaled by 1/M (the convolution
        // runs DIF -> pointwise -> inverse DIT, see ringfft.cu)
        std::complex<double> v = b[k] / (double)M;
        int q = bitrev(k, bits);
        bh[rp.bhat_ofs + q] = make_double2(v.real(), v.imag());
        bh32[rp.bhat_ofs + q] = make_float2((float)v.real(), (float)v.imag());
      }
    }
    WF_CUDA(cudaMalloc(&P.chirp64, sizeof(double2) * chirp_total));
    WF_CUDA(cudaMalloc(&P.chirp32, sizeof(float2) * chirp_total));
    WF_CUDA(cudaMalloc(&P.bhat64, sizeof(double2) * bhat_total));
    WF_CUDA(cudaMalloc(&P.bhat32, sizeof(float2) * bhat_total));
    WF_CUDA(cudaMemcpy(P.chirp64, ch.data(), sizeof(double2) * chirp_total,
                       cudaMemcpyHostToDevice));
    WF_CUDA(cudaMemcpy(P.chirp32, ch32.data(), sizeof(float2) * chirp_total,
                       cudaMemcpyHostToDevice));
    WF_CUDA(cudaMemcpy(P.bhat64, bh.data(), sizeof(double2) * bhat_total,
                       cudaMemcpyHostToDevice));
    WF_CUDA(cudaMemcpy(P.bhat32, bh32.data(), sizeof(float2) * bhat_total,
                       cudaMemcpyHostToDevice));
    WF_TRY(upload_dd(ch, &P.chirpdd));
    WF_TRY(upload_dd(bh, &P.bhatdd));
    // e^{i pi num k / den} (phi0 = pi num / den) of the Bluestein rings, for
    // the double-float ring transforms (FP64 sincospi costs more there)
    std::vector<double2> ph(chirp_total);
    for (auto &rp : P.pairs_h) {
      if (rp.chirp_ofs < 0) continue;
      for (int k = 0; k < rp.nphi; ++k) {
        if (rp.phi_num == 0) {
          ph[rp.chirp_ofs + k] = make_double2(1.0, 0.0);
        } else {
          const long long q = ((long long)k * rp.phi_num) % (2LL * rp.phi_den);
          const double ang = M_PI * (double)q / (double)rp.phi_den;
          ph[rp.chirp_ofs + k] = make_double2(cos(ang), sin(ang));
        }
      }
    }
    WF_TRY(upload_dd(ph, &P.phasedd));
  }
  return WF_OK;
}

// ---------------------------------------------------------------- Legendre
static wf_status make_recurrence_tables(Plan &P) {
  const int L = P.lmax;
  std::vector<double> c(P.nalm, 0.0), g(P.nalm, 1.0);
  std::vector<float> c32(P.nalm, 0.0f), g32(P.nalm, 1.0f);
  for (int m = 0; m <= L; ++m) {
    double a_prev = 0.0, g2 = 1.0, g1 = 1.0;  // g_{l-2}, g_{l-1}
    for (int l = m; l <= L; ++l) {
      long i = alm_idx(L, l, m);
      if (l == m) {
        g[i] = 1.0;
        c[i] = 0.0;
        g32[i] = ((l >> 1) & 1) ? -1.0f : 1.0f;
        continue;
      }
      double a = sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)m * m));
      double gl;
      if (l == m + 1) {
        gl = 1.0;
      } else {
        gl = (a / a_prev) * g2;
      }
      g[i] = gl;
      c[i] = a * g1 / gl;
      // FP32 kernels run s_l = eps_l u_l, eps_l = (-1)^floor(l/2): then
      // s_l = c'_l z s_{l-1} + s_{l-2} with c'_l = eps_{l-1} eps_l c_l =
      // -c_l for even l, +c_l for odd l (no negated operand, so two rings
      // fit one packed f32x2 FMA)
      c32[i] = (float)((l % 2 == 0) ? -c[i] : c[i]);
      g32[i] = (float)(((l >> 1) & 1) ? -gl : gl);  // g_l eps_l
      a_prev = a;
      g2 = g1;
      g1 = gl;
    }
  }
  WF_CUDA(cudaMalloc(&P.rc, sizeof(double) * P.nalm));
  WF_CUDA(cudaMalloc(&P.rg, sizeof(double) * P.nalm));
  WF_CUDA(cudaMalloc(&P.rc32, sizeof(float) * P.nalm));
  {
    // the double-float Legendre kernels' coefficient table (hi, lo)
    std::vector<float2> cdd(P.nalm);
    for (long i = 0; i < P.nalm; ++i) {
      const float h = (float)c[i];
      cdd[i] = make_float2(h, (float)(c[i] - (double)h));
    }
    WF_CUDA(cudaMalloc(&P.rcdd, sizeof(float2) * P.nalm));
    WF_CUDA(cudaMemcpy(P.rcdd, cdd.data(), sizeof(float2) * P.nalm, cudaMemcpyHostToDevice));
  }
  WF_CUDA(cudaMalloc(&P.rg32, sizeof(float) * P.nalm));
  WF_CUDA(cudaMemcpy(P.rg32, g32.data(), sizeof(float) * P.nalm, cudaMemcpyHostToDevice));
  WF_CUDA(cudaMemcpy(P.rc, c.data(), sizeof(double) * P.nalm,
                     cudaMemcpyHostToDevice));
  WF_CUDA(cudaMemcpy(P.rg, g.data(), sizeof(double) * P.nalm,
                     cudaMemcpyHostToDevice));
  WF_CUDA(cudaMemcpy(P.rc32, c32.data(), sizeof(float) * P.nalm,
                     cudaMemcpyHostToDevice));
  return WF_OK;
}

// lam_mm for every m of one ring pair, as mantissa * 2^exponent.
__global__ void k_seed_diag(const RingPair *pairs, int npairs, int lmax,
                            double *mant, int *expo) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= npairs) return;
  const double sth = pairs[k].sth;
  double v = 0.28209479177387814;  // 1/sqrt(4 pi)
  int e = 0;
  for (int m = 0; m <= lmax; ++m) {
    if (m > 0) {
      v *= -sth * sqrt((2.0 * m + 1.0) / (2.0 * m));
      if (fabs(v) < 0x1p-200) {
        v *= 0x1p+200;
        e -= 200;
      }
    }
    mant[(long)m * npairs + k] = v;
    expo[(long)m * npairs + k] = e;
  }
}

// For each (m, pair): walk the recurrence in scaled FP64 until |lam| >= 2^-100
// and store the start l and the two rescaled values there.
__global__ void k_seed_walk(const RingPair *pairs, int npairs, int lmax,
                            const double *mant, const int *expo,
                            const double *rg, int *seed_l, double2 *seed_u,
                            float2 *seed_s32) {
  long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long)npairs * (lmax + 1)) return;
  const int m = (int)(t / npairs);
  const int k = (int)(t % npairs);
  const double z = pairs[k].z;
  double v = mant[t], vp = 0.0;  // lam_l, lam_{l-1} scaled by 2^-e
  int e = expo[t];
  double a_prev = 0.0;
  int l = m;
  int found = lmax + 1;
  double lam0 = 0.0, lam1 = 0.0;
  for (;;) {
    // actual value v * 2^e; compare exponents against -100
    if (v != 0.0 && ilogb(v) + e >= -100) {
      found = l;
      lam0 = ldexp(v, e);
      if (l + 1 <= lmax) {
        double a = sqrt((4.0 * (l + 1) * (l + 1) - 1.0) /
                        ((double)(l + 1) * (l + 1) - (double)m * m));
        double vn = (l == m) ? a * z * v : a * z * v - (a / a_prev) * vp;
        lam1 = ldexp(vn, e);
      }
      break;
    }
    if (l == lmax) break;
    const int ln = l + 1;
    double a = sqrt((4.0 * ln * ln - 1.0) / ((double)ln * ln - (double)m * m));
    double vn = (l == m) ? a * z * v : a * z * v - (a / a_prev) * vp;
    vp = v;
    v = vn;
    a_prev = a;
    l = ln;
    if (e < 0 && fabs(v) > 0x1p+200) {
      v *= 0x1p-200;
      vp *= 0x1p-200;
      e += 200;
    }
  }
  seed_l[t] = found;
  double2 u = make_double2(0.0, 0.0);
  if (found <= lmax) {
    u.x = lam0 / rg[alm_idx_d(lmax, found, m)];
    if (found + 1 <= lmax) u.y = lam1 / rg[alm_idx_d(lmax, found + 1, m)];
  }
  seed_u[t] = u;
  // s-units of the FP32 kernels: s_l = eps_l u_l, eps_l = (-1)^floor(l/2)
  const double e0 = ((found >> 1) & 1) ? -1.0 : 1.0, e1 = (((found + 1) >> 1) & 1) ? -1.0 : 1.0;
  seed_s32[t] = make_float2((float)(e0 * u.x), (float)(e1 * u.y));
}

static wf_status make_seeds(Plan &P) {
  const long n = (long)P.npairs * (P.lmax + 1);
  double *mant = nullptr;
  int *expo = nullptr;
  WF_CUDA(cudaMalloc(&mant, sizeof(double) * n));
  WF_CUDA(cudaMalloc(&expo, sizeof(int) * n));
  WF_CUDA(cudaMalloc(&P.seed_l, sizeof(int) * n));
  WF_CUDA(cudaMalloc(&P.seed_u, sizeof(double2) * n));
  WF_CUDA(cudaMalloc(&P.seed_s32, sizeof(float2) * n));
  k_seed_diag<<<(P.npairs + 127) / 128, 128, 0, P.stream>>>(P.pairs, P.npairs,
                                                            P.lmax, mant, expo);
  WF_CUDA(cudaGetLastError());
  k_seed_walk<<<(unsigned)((n + 255) / 256), 256, 0, P.stream>>>(
      P.pairs, P.npairs, P.lmax, mant, expo, P.rg, P.seed_l, P.seed_u, P.seed_s32);
  WF_CUDA(cudaGetLastError());
  WF_CUDA(cudaStreamSynchronize(P.stream));
  WF_CUDA(cudaFree(mant));
  WF_CUDA(cudaFree(expo));
  return WF_OK;
}

wf_status build_tables(Plan &P) {
  WF_TRY(init_legendre_attributes());
  WF_TRY(init_ring_attributes());
  make_pairs(P);
  WF_TRY(make_fft_tables(P));
  WF_CUDA(cudaMalloc(&P.pairs, sizeof(RingPair) * P.npairs));
  WF_CUDA(cudaMemcpy(P.pairs, P.pairs_h.data(), sizeof(RingPair) * P.npairs,
                     cudaMemcpyHostToDevice));
  WF_CUDA(cudaMalloc(&P.cl_d, sizeof(double) * (P.lmax + 1)));
  WF_CUDA(cudaMemcpy(P.cl_d, P.cl.data(), sizeof(double) * (P.lmax + 1),
                     cudaMemcpyHostToDevice));
  {
    const std::vector<float> cl32(P.cl.begin(), P.cl.end());
    std::vector<float> zs(2 * (size_t)P.npairs);
    for (int k = 0; k < P.npairs; ++k) {  // z = zh + zl to ~2^-48
      const double z = P.pairs_h[k].z;
      zs[k] = (float)z;
      zs[P.npairs + k] = (float)(z - (double)zs[k]);
    }
    WF_CUDA(cudaMalloc(&P.cl32, sizeof(float) * (P.lmax + 1)));
    WF_CUDA(cudaMemcpy(P.cl32, cl32.data(), sizeof(float) * (P.lmax + 1),
                       cudaMemcpyHostToDevice));
    WF_CUDA(cudaMalloc(&P.zs32, sizeof(float) * zs.size()));
    WF_CUDA(cudaMemcpy(P.zs32, zs.data(), sizeof(float) * zs.size(), cudaMemcpyHostToDevice));
  }
  WF_TRY(make_recurrence_tables(P));
  WF_TRY(make_seeds(P));
  return WF_OK;
}

// ---------------------------------------------------------------- noise
// Copy sigma^2 (masked -> +inf) and reduce: number of observed pixels,
// number of invalid observed variances, min over observed pixels.
__global__ void k_noise_copy(const double *nv, const uint8_t *mask, long npix,
                             double *out, double *bmin, unsigned long long *bcnt,
                             unsigned long long *bbad) {
  __shared__ double smin[256];
  __shared__ unsigned long long scnt[256], sbad[256];
  double mn = INFINITY;
  unsigned long long cnt = 0, bad = 0;
  for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < npix;
       p += (long)gridDim.x * blockDim.x) {
    bool msk = mask != nullptr && mask[p] != 0;
    double v = nv[p];
    if (msk) {
      out[p] = INFINITY;
    } else {
      out[p] = v;
      ++cnt;
      if (!(v > 0.0) || isinf(v) || isnan(v))
        ++bad;
      else
        mn = fmin(mn, v);
    }
  }
  smin[threadIdx.x] = mn;
  scnt[threadIdx.x] = cnt;
  sbad[threadIdx.x] = bad;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + s]);
      scnt[threadIdx.x] += scnt[threadIdx.x + s];
      sbad[threadIdx.x] += sbad[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    bmin[blockIdx.x] = smin[0];
    bcnt[blockIdx.x] = scnt[0];
    bbad[blockIdx.x] = sbad[0];
  }
}

// sigma^2 / alpha in FP32 for the FP32 ring step (+inf stays +inf)
__global__ void k_noise_f32(const double *nv, long npix, double inv_alpha, float *out) {
  for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < npix;
       p += (long)gridDim.x * blockDim.x)
    out[p] = (float)(nv[p] * inv_alpha);
}

wf_status upload_noise(Plan &P, const double *nvar_dev, const uint8_t *mask_dev) {
  if (!P.nvar) WF_CUDA(cudaMalloc(&P.nvar, sizeof(double) * P.npix));
  const int nb = 304;
  double *bmin = nullptr;
  unsigned long long *bcnt = nullptr;
  WF_CUDA(cudaMalloc(&bmin, sizeof(double) * nb));
  WF_CUDA(cudaMalloc(&bcnt, sizeof(unsigned long long) * nb * 2));
  k_noise_copy<<<nb, 256, 0, P.stream>>>(nvar_dev, mask_dev, P.npix, P.nvar,
                                         bmin, bcnt, bcnt + nb);
  WF_CUDA(cudaGetLastError());
  std::vector<double> hmin(nb);
  std::vector<unsigned long long> hc(2 * nb);
  WF_CUDA(cudaMemcpyAsync(hmin.data(), bmin, sizeof(double) * nb,
                          cudaMemcpyDeviceToHost, P.stream));
  WF_CUDA(cudaMemcpyAsync(hc.data(), bcnt, sizeof(unsigned long long) * 2 * nb,
                          cudaMemcpyDeviceToHost, P.stream));
  WF_CUDA(cudaStreamSynchronize(P.stream));
  WF_CUDA(cudaFree(bmin));
  WF_CUDA(cudaFree(bcnt));
  double mn = INFINITY;
  unsigned long long cnt = 0, bad = 0;
  for (int b = 0; b < nb; ++b) {
    mn = std::min(mn, hmin[b]);
    cnt += hc[b];
    bad += hc[nb + b];
  }
  if (cnt == 0) {
    set_error("wf: every pixel is masked");
    return WF_ERR_ARG;
  }
  if (bad != 0) {
    set_error("wf: noise variance must be finite and > 0 on observed pixels");
    return WF_ERR_ARG;
  }
  P.alpha = mn;
  if (!P.nvar32) WF_CUDA(cudaMalloc(&P.nvar32, sizeof(float) * P.npix));
  k_noise_f32<<<nb, 256, 0, P.stream>>>(P.nvar, P.npix, 1.0 / mn, P.nvar32);
  WF_CUDA(cudaGetLastError());
  if (!P.nvardd) WF_CUDA(cudaMalloc(&P.nvardd, sizeof(float2) * P.npix));
  WF_TRY(launch_to_dd(P, P.nvar, P.nvardd, P.npix));
  P.has_noise = true;
  return WF_OK;
}

}  // namespace wf
