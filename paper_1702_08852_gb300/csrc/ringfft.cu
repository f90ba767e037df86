// ringfft.cu -- per-ring Fourier transforms between pixel values and ring
// Fourier coefficients, with the messenger (pixel-space) update fused in.
//
// For a ring with n pixels at phi_j = phi0 + 2 pi j / n:
//   synthesis  s_j  = sum_{|m| <= L} F[m] e^{i m phi_j},  F[-m] = conj F[m]
//            = sum_{k<n} c_k e^{2 pi i j k / n},  c_k = sum_{m = k mod n} F[m] e^{i m phi0}
//   analysis   G[m] = sum_j t_j e^{-i m phi_j} = e^{-i m phi0} X[m mod n],
//              X = DFT_n(t).
// The north and south ring of a pair have the same n and phi0 and both carry
// real data, so one complex DFT serves both: Z = c^N + i c^S on the way in,
// X^N_k = (X_k + conj X_{n-k}) / 2, X^S_k = (X_k - conj X_{n-k}) / (2i) on the
// way out.
//
// The fused step of one iteration (the t-update of Algorithm 2, Eq. 14):
//   s = Y a on the ring, t_p = s_p + w_p (d_p - s_p), w_p = xi / (sigma^2_p + mu)
// (w = 0 on masked pixels, where sigma^2 is stored as +inf), then G = FFT(t):
// the messenger field never leaves shared memory.
//
// DFTs: power-of-two n -- radix-2 in shared memory, decimation in frequency
// (natural -> bit-reversed order) for the inverse, decimation in time
// (bit-reversed -> natural) for the forward transform, so no permutation pass
// is needed.  Other n (the polar rings, n = 4i) -- Bluestein's chirp-z:
// X_k = conj(w_k) sum_j (x_j conj(w_j)) w_{k-j}, w_j = e^{i pi j^2 / n}, as a
// length-M circular convolution (M = 2^p >= 2n - 1) by DIF -> pointwise
// product with the kernel spectrum (stored bit-reversed) -> inverse DIT.
#include "wf_internal.cuh"

namespace wf {

template <typename T2> struct CT;
template <> struct CT<double2> {
  typedef double T;
  static __device__ __forceinline__ double2 mk(double a, double b) {
    return make_double2(a, b);
  }
  // sin, cos of pi r / den
  static __device__ __forceinline__ void sincospi_(int r, int den, double *s,
                                                   double *c) {
    sincospi((double)r / (double)den, s, c);
  }
};
template <> struct CT<float2> {
  typedef float T;
  static __device__ __forceinline__ float2 mk(float a, float b) {
    return make_float2(a, b);
  }
  static __device__ __forceinline__ void sincospi_(int r, int den, float *s,
                                                   float *c) {
    sincospif((float)r / (float)den, s, c);
  }
};

template <typename T2>
__device__ __forceinline__ T2 cmul(T2 a, T2 b) {
  return CT<T2>::mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T2>
__device__ __forceinline__ T2 cmulc(T2 a, T2 b) {  // a * conj(b)
  return CT<T2>::mk(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename T2>
__device__ __forceinline__ T2 cadd(T2 a, T2 b) {
  return CT<T2>::mk(a.x + b.x, a.y + b.y);
}
template <typename T2>
__device__ __forceinline__ T2 csub(T2 a, T2 b) {
  return CT<T2>::mk(a.x - b.x, a.y - b.y);
}
template <typename T2>
__device__ __forceinline__ T2 cconj(T2 a) {
  return CT<T2>::mk(a.x, -a.y);
}

// multiply by -i (forward) or +i (inverse)
template <typename T2, bool INV>
__device__ __forceinline__ T2 rot_q(T2 a) {
  return INV ? CT<T2>::mk(-a.y, a.x) : CT<T2>::mk(a.y, -a.x);
}

// natural -> bit-reversed; INV uses e^{+2 pi i jk/M}.  Two radix-2 stages
// (spans h and h/2) per pass over shared memory ("radix-2^2"): the output
// order stays bit-reversed, and the barriers and shared-memory round trips
// halve.  An odd number of stages ends with one radix-2 pass of span 1.
template <typename T2, bool INV>
__device__ void fft_dif(T2 *buf, int M, const T2 *__restrict__ tw, int Mmax) {
  int h = M >> 1;
  for (; h >= 2; h >>= 2) {
    const int q = h >> 1;
    const int ts = Mmax / (2 * h);
    for (int b = threadIdx.x; b < (M >> 2); b += blockDim.x) {
      const int j = b & (q - 1);
      const int i0 = ((b - j) << 2) + j, i1 = i0 + q, i2 = i0 + h, i3 = i2 + q;
      const T2 w1 = tw[j * ts], w2 = tw[2 * j * ts];  // W_2h^j, W_h^j
      const T2 x0 = buf[i0], x1 = buf[i1], x2 = buf[i2], x3 = buf[i3];
      const T2 a0 = cadd(x0, x2), a1 = cadd(x1, x3);
      const T2 a2 = INV ? cmulc(csub(x0, x2), w1) : cmul(csub(x0, x2), w1);
      const T2 a3 = rot_q<T2, INV>(INV ? cmulc(csub(x1, x3), w1) : cmul(csub(x1, x3), w1));
      buf[i0] = cadd(a0, a1);
      buf[i1] = INV ? cmulc(csub(a0, a1), w2) : cmul(csub(a0, a1), w2);
      buf[i2] = cadd(a2, a3);
      buf[i3] = INV ? cmulc(csub(a2, a3), w2) : cmul(csub(a2, a3), w2);
    }
    __syncthreads();
  }
  if (h == 1) {
    for (int b = threadIdx.x; b < (M >> 1); b += blockDim.x) {
      const T2 a = buf[2 * b], c = buf[2 * b + 1];
      buf[2 * b] = cadd(a, c);
      buf[2 * b + 1] = csub(a, c);
    }
    __syncthreads();
  }
}

// bit-reversed -> natural; an odd number of stages starts with one radix-2
// pass of span 1, then pairs of stages (spans h and 2h) per pass
template <typename T2, bool INV>
__device__ void fft_dit(T2 *buf, int M, const T2 *__restrict__ tw, int Mmax) {
  int h = 1;
  int bits = 0;
  while ((1 << bits) < M) ++bits;
  if (bits & 1) {
    for (int b = threadIdx.x; b < (M >> 1); b += blockDim.x) {
      const T2 a = buf[2 * b], c = buf[2 * b + 1];
      buf[2 * b] = cadd(a, c);
      buf[2 * b + 1] = csub(a, c);
    }
    __syncthreads();
    h = 2;
  }
  for (; h < M; h <<= 2) {
    const int ta = Mmax / (2 * h), tb = Mmax / (4 * h);
    for (int b = threadIdx.x; b < (M >> 2); b += blockDim.x) {
      const int j = b & (h - 1);
      const int i0 = ((b - j) << 2) + j, i1 = i0 + h, i2 = i0 + 2 * h, i3 = i2 + h;
      const T2 wa = tw[j * ta], wb = tw[j * tb];  // W_2h^j, W_4h^j
      const T2 x0 = buf[i0], x1 = buf[i1], x2 = buf[i2], x3 = buf[i3];
      const T2 c1 = INV ? cmulc(x1, wa) : cmul(x1, wa);
      const T2 c3 = INV ? cmulc(x3, wa) : cmul(x3, wa);
      const T2 a0 = cadd(x0, c1), a1 = csub(x0, c1);
      const T2 a2 = cadd(x2, c3), a3 = csub(x2, c3);
      const T2 d2 = INV ? cmulc(a2, wb) : cmul(a2, wb);
      const T2 d3 = rot_q<T2, INV>(INV ? cmulc(a3, wb) : cmul(a3, wb));
      buf[i0] = cadd(a0, d2);
      buf[i2] = csub(a0, d2);
      buf[i1] = cadd(a1, d3);
      buf[i3] = csub(a1, d3);
    }
    __syncthreads();
  }
}

// In place: buf[0..n) holds a_j = x_j conj(w_j) and buf[n..M) zeros on entry;
// on exit buf[0..n) holds X = DFT_n(x).
template <typename T2>
__device__ void bluestein(T2 *buf, int n, int M, const T2 *__restrict__ tw,
                          int Mmax, const T2 *__restrict__ chirp,
                          const T2 *__restrict__ bhat) {
  fft_dif<T2, false>(buf, M, tw, Mmax);
  for (int q = threadIdx.x; q < M; q += blockDim.x) buf[q] = cmul(buf[q], bhat[q]);
  __syncthreads();
  fft_dit<T2, true>(buf, M, tw, Mmax);
  for (int k = threadIdx.x; k < n; k += blockDim.x) buf[k] = cmulc(buf[k], chirp[k]);
  __syncthreads();
}

__device__ __forceinline__ int bitrev_n(int x, int bits) {
  return (int)(__brev((unsigned)x) >> (32 - bits));
}

// Ring offsets of HEALPix: phi0 = pi num / den with num = 0, or num = 1 and
// den = n (the ring's pixel count), so e^{i n phi0} = sgn = -1 or +1 and
// e^{i m phi0} = sgn^j e^{i k phi0} for m = k + j n: one phase per Fourier
// index k < n of the ring, not one per m.
//
// e^{i k phi0}, 0 <= k < den.  When 2 den divides the twiddle table's length
// (every equatorial ring) the value is a table entry: e^{i pi k / den} =
// conj(tw[k Mmax / (2 den)]), tw[i] = e^{-2 pi i i / Mmax}; otherwise
// sincospi with the exact rational argument k / den.
template <typename T2>
__device__ __forceinline__ T2 ring_phase(int k, int num, int den, int tstep,
                                         const T2 *__restrict__ tw) {
  typedef typename CT<T2>::T T;
  if (num == 0) return CT<T2>::mk((T)1, (T)0);
  if (tstep > 0) return cconj(tw[k * tstep]);
  T s, c;
  CT<T2>::sincospi_(k, den, &s, &c);
  return CT<T2>::mk(c, s);
}

// c_k = sum over m = +-k mod n, |m| <= L, of F[m] e^{i m phi0}
//     = e^{i k phi0} (sum_j sgn^j F[k + j n] + sum_{j >= 1} sgn^j conj F[j n - k])
template <typename T2>
__device__ __forceinline__ T2 fold(const T2 *__restrict__ Fr, int k, int n, int L,
                                   typename CT<T2>::T sgn, T2 ph) {
  typedef typename CT<T2>::T T;
  T2 acc = CT<T2>::mk((T)0, (T)0);
  T s = (T)1;
  for (int m = k; m <= L; m += n) {
    const T2 f = Fr[m];
    acc = CT<T2>::mk(acc.x + s * f.x, acc.y + s * f.y);
    s *= sgn;
  }
  s = sgn;
  for (int m = n - k; m <= L; m += n) {  // m >= 1 since k < n
    const T2 f = Fr[m];
    acc = CT<T2>::mk(acc.x + s * f.x, acc.y - s * f.y);
    s *= sgn;
  }
  return cmul(acc, ph);
}

constexpr int RING_THREADS = 256;

template <typename T2, int MODE>
__global__ void __launch_bounds__(RING_THREADS)
    k_ring(const RingPair *__restrict__ pairs, int pair_base, int lmax,
           const T2 *__restrict__ F, T2 *__restrict__ G,
           const double *__restrict__ in_map, double *__restrict__ out_map,
           const double *__restrict__ nvar, const T2 *__restrict__ tw, int Mmax,
           const T2 *__restrict__ chirp_all, const T2 *__restrict__ bhat_all,
           const SolverState *__restrict__ st, int lstatic) {
  typedef typename CT<T2>::T T;
  const RingPair rp = pairs[pair_base + blockIdx.x];
  int Lf = lstatic, Lg = lstatic;
  double xi = 0.0, mu = 0.0;
  if (st) {
    if (st->done) return;
    Lf = st->lcur;
    Lg = max(st->lcur, st->lnext);
    xi = st->xi;
    mu = st->mu;
  }
  extern __shared__ __align__(16) unsigned char smraw[];
  T2 *buf = reinterpret_cast<T2 *>(smraw);
  const int n = rp.nphi, M = rp.fftM;
  const bool blue = M != n;
  int bits = 0;
  while ((1 << bits) < M) ++bits;
  const T2 *chirp = blue ? chirp_all + rp.chirp_ofs : nullptr;
  const T2 *bhat = blue ? bhat_all + rp.bhat_ofs : nullptr;
  const long stride = lmax + 1;
  const bool south = rp.ringS >= 0;
  const T2 zero = CT<T2>::mk((T)0, (T)0);
  const T sgn = rp.phi_num ? (T)-1 : (T)1;  // e^{i n phi0}
  const int tstep = (rp.phi_num && Mmax % (2 * rp.phi_den) == 0) ? Mmax / (2 * rp.phi_den) : 0;

  if (MODE != RING_ANALYSIS) {
    const T2 *FN = F + rp.ringN * stride;
    const T2 *FS = south ? F + rp.ringS * stride : nullptr;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      T2 cN = zero, cS = zero;
      if (Lf >= 0 && (k <= Lf || n - k <= Lf)) {
        const T2 ph = ring_phase<T2>(k, rp.phi_num, rp.phi_den, tstep, tw);
        cN = fold(FN, k, n, Lf, sgn, ph);
        if (south) cS = fold(FS, k, n, Lf, sgn, ph);
      }
      const T2 Zk = CT<T2>::mk(cN.x - cS.y, cN.y + cS.x);  // cN + i cS
      buf[k] = blue ? cmulc(cconj(Zk), chirp[k]) : Zk;
    }
    if (blue)
      for (int k = n + threadIdx.x; k < M; k += blockDim.x) buf[k] = zero;
    __syncthreads();
    if (blue) {
      bluestein<T2>(buf, n, M, tw, Mmax, chirp, bhat);  // DFT(conj Z)
    } else {
      fft_dif<T2, true>(buf, M, tw, Mmax);  // bit-reversed output
    }
    // pixel step; position q holds pixel j
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
      const int j = blue ? q : bitrev_n(q, bits);
      T2 zz = buf[q];
      if (blue) zz = cconj(zz);
      const double sN = (double)zz.x, sS = (double)zz.y;
      const long pN = rp.ofsN + j, pS = south ? rp.ofsS + j : -1;
      if (MODE == RING_SYNTH) {
        out_map[pN] = sN;
        if (south) out_map[pS] = sS;
      } else {
        if (out_map) {
          out_map[pN] = sN;
          if (south) out_map[pS] = sS;
        }
        double tN = sN, tS = 0.0;
        {
          const double v = nvar[pN];
          const double w = xi / (v + mu);  // 0 on masked pixels (v = +inf)
          tN = sN + w * ((in_map ? in_map[pN] : 0.0) - sN);
        }
        if (south) {
          const double v = nvar[pS];
          const double w = xi / (v + mu);
          tS = sS + w * ((in_map ? in_map[pS] : 0.0) - sS);
        }
        const T2 tt = CT<T2>::mk((T)tN, (T)tS);
        buf[q] = blue ? cmulc(tt, chirp[q]) : tt;
      }
    }
    if (MODE == RING_SYNTH) return;
    if (blue)
      for (int k = n + threadIdx.x; k < M; k += blockDim.x) buf[k] = zero;
    __syncthreads();
  } else {
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      const double tN = in_map[rp.ofsN + j];
      const double tS = south ? in_map[rp.ofsS + j] : 0.0;
      const T2 tt = CT<T2>::mk((T)tN, (T)tS);
      if (blue)
        buf[j] = cmulc(tt, chirp[j]);
      else
        buf[bitrev_n(j, bits)] = tt;
    }
    if (blue)
      for (int k = n + threadIdx.x; k < M; k += blockDim.x) buf[k] = zero;
    __syncthreads();
  }
  // forward DFT of t (natural order output)
  if (blue)
    bluestein<T2>(buf, n, M, tw, Mmax, chirp, bhat);
  else
    fft_dit<T2, false>(buf, M, tw, Mmax);
  // split the two real rings and apply e^{-i m phi0}: for m = k + j n,
  // G[m] = sgn^j e^{-i k phi0} X_k (X^N or X^S)
  T2 *GN = G + rp.ringN * stride;
  T2 *GS = south ? G + rp.ringS * stride : nullptr;
  const T half = (T)0.5;
  const int kmax = min(n - 1, Lg);
  for (int k = threadIdx.x; k <= kmax; k += blockDim.x) {
    const int kk = k == 0 ? 0 : n - k;
    const T2 X = buf[k], Xc = cconj(buf[kk]);
    const T2 ph = cconj(ring_phase<T2>(k, rp.phi_num, rp.phi_den, tstep, tw));
    const T2 tN = cmul(CT<T2>::mk(half * (X.x + Xc.x), half * (X.y + Xc.y)), ph);
    // (X - Xc) / (2i)
    const T2 dlt = csub(X, Xc);
    const T2 tS = cmul(CT<T2>::mk(half * dlt.y, -half * dlt.x), ph);
    T s = (T)1;
    for (int m = k; m <= Lg; m += n) {
      GN[m] = CT<T2>::mk(s * tN.x, s * tN.y);
      if (south) GS[m] = CT<T2>::mk(s * tS.x, s * tS.y);
      s *= sgn;
    }
  }
}

template <typename T2> struct Tables;
template <> struct Tables<double2> {
  static const double2 *tw(const Plan &P) { return P.tw64; }
  static const double2 *ch(const Plan &P) { return P.chirp64; }
  static const double2 *bh(const Plan &P) { return P.bhat64; }
};
template <> struct Tables<float2> {
  static const float2 *tw(const Plan &P) { return P.tw32; }
  static const float2 *ch(const Plan &P) { return P.chirp32; }
  static const float2 *bh(const Plan &P) { return P.bhat32; }
};

template <typename T2, int MODE>
static wf_status launch_ring_mode(const Plan &P, const T2 *F, T2 *G,
                                  const double *in_map, double *out_map,
                                  const SolverState *st, int lstatic) {
  auto kern = k_ring<T2, MODE>;
  // two launches: the polar rings (pairs 0 .. nside-2, Bluestein unless n is
  // a power of two) and the equatorial belt (pairs nside-1 .. 2 nside-1)
  const int npolar = P.nside - 1;
  const int groups[2][2] = {{0, npolar}, {npolar, P.npairs}};
  for (int g = 0; g < 2; ++g) {
    const int b = groups[g][0], e = groups[g][1];
    if (e <= b) continue;
    int Mg = 1;
    for (int k = b; k < e; ++k) Mg = std::max(Mg, P.pairs_h[k].fftM);
    const size_t smem = sizeof(T2) * Mg;
    ++P.nlaunch;
    kern<<<e - b, RING_THREADS, smem, P.stream>>>(
        P.pairs, b, P.lmax, F, G, in_map, out_map, P.nvar, Tables<T2>::tw(P),
        P.fftMmax, Tables<T2>::ch(P), Tables<T2>::bh(P), st, lstatic);
    WF_CUDA(cudaGetLastError());
  }
  return WF_OK;
}

template <typename T2>
wf_status launch_ring(const Plan &P, int mode, const T2 *F, T2 *G,
                      const double *in_map, double *out_map,
                      const SolverState *st, int lstatic) {
  switch (mode) {
    case RING_SYNTH:
      return launch_ring_mode<T2, RING_SYNTH>(P, F, G, in_map, out_map, st, lstatic);
    case RING_ANALYSIS:
      return launch_ring_mode<T2, RING_ANALYSIS>(P, F, G, in_map, out_map, st,
                                                 lstatic);
    default:
      return launch_ring_mode<T2, RING_FUSED>(P, F, G, in_map, out_map, st, lstatic);
  }
}

wf_status init_ring_attributes() {
  const int big = 220 * 1024;
  WF_CUDA(cudaFuncSetAttribute(k_ring<double2, RING_SYNTH>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  WF_CUDA(cudaFuncSetAttribute(k_ring<double2, RING_ANALYSIS>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  WF_CUDA(cudaFuncSetAttribute(k_ring<double2, RING_FUSED>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  WF_CUDA(cudaFuncSetAttribute(k_ring<float2, RING_SYNTH>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  WF_CUDA(cudaFuncSetAttribute(k_ring<float2, RING_ANALYSIS>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  WF_CUDA(cudaFuncSetAttribute(k_ring<float2, RING_FUSED>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  return WF_OK;
}

template wf_status launch_ring<double2>(const Plan &, int, const double2 *,
                                        double2 *, const double *, double *,
                                        const SolverState *, int);
template wf_status launch_ring<float2>(const Plan &, int, const float2 *, float2 *,
                                       const double *, double *,
                                       const SolverState *, int);

}  // namespace wf
