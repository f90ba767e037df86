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
#include <limits.h>

#include <type_traits>

#include "wf_internal.cuh"

namespace wf {

template <typename T2> struct CT;
template <> struct CT<double2> {
  typedef double T;
  typedef double2 G;  // element type of the global data arrays (F, G)
  typedef double2 W;  // element type of the tables (twiddles, chirps)
  static __device__ __forceinline__ double2 ld(const G *p) { return *p; }
  static __device__ __forceinline__ double2 ldw(const W *p) { return *p; }
  static __device__ __forceinline__ void st(G *p, double2 v) { *p = v; }
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
  typedef float2 G;
  typedef float2 W;
  static __device__ __forceinline__ float2 ld(const G *p) { return *p; }
  static __device__ __forceinline__ float2 ldw(const W *p) { return *p; }
  static __device__ __forceinline__ void st(G *p, float2 v) { *p = v; }
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

// Shared-memory layout of the FFT buffer: element i is stored at
// sw(i) = i ^ (h(i >> 4) & 15), h(b) = b ^ (b << 2) -- an XOR inside each
// aligned block of 16 complex values.  Unit-stride sweeps stay conflict-free,
// and the radix-2^2 passes of short span (whose four operands sit 1..8
// elements apart, 16 lanes in the same few banks) spread over all banks:
// with it every pass of every power-of-two length needs the minimum number
// of shared-memory wavefronts.
__device__ __forceinline__ int sw(int i) {
  const int b = i >> 4;
  return i ^ ((b ^ (b << 2)) & 15);
}

// Twiddles of one pass: pair(j) gives W_2h^j = e^{-i pi j / h} and
// W_h^j = (W_2h^j)^2 (h a power of two, 0 <= j < h).  FP32 computes them:
// sincospi of the exact argument j / h (1/h is exact) and one complex square
// -- no memory access on the FFT's critical path.  FP64 reads the plan's
// table tw[i] = e^{-2 pi i i / Mmax} (FP64 sincospi would cost more than the
// butterfly on this part's FP64 pipe).
template <typename T2> struct TwPass;
template <> struct TwPass<float2> {
  float inv;
  __device__ __forceinline__ TwPass(int h, const float2 *, int) : inv(1.0f / (float)h) {}
  __device__ __forceinline__ void pair(int j, float2 &w2h, float2 &wh) const {
    float s, c;
    sincospif((float)j * inv, &s, &c);
    w2h = make_float2(c, -s);
    wh = make_float2(c * c - s * s, -2.0f * c * s);
  }
};
template <> struct TwPass<double2> {
  const double2 *tw;
  int ts;
  __device__ __forceinline__ TwPass(int h, const double2 *t, int Mmax)
      : tw(t), ts(Mmax / (2 * h)) {}
  __device__ __forceinline__ void pair(int j, double2 &w2h, double2 &wh) const {
    w2h = tw[j * ts];
    wh = tw[2 * j * ts];
  }
};

// ---------------------------------------------------------- double-float
// ddr: an unevaluated sum hi + lo of two floats (~48-bit significand) with
// the operations the ring transforms use -- sums by two-sum, products by
// the FMA two-product, one normalisation each (Dekker, Knuth); explicit _rn
// intrinsics, so nothing is contracted or reassociated.  The mixed solver's
// anchor steps run their ring FFTs in it on the FP32 pipe: this part's FP64
// pipe runs at ~1/64 of the FP32 rate, and those FFTs were FP64-bound.
// The ring coefficients F, G (written and read by the double-float Legendre
// kernels), the twiddle, chirp, kernel-spectrum and phase tables and the
// pixel step's d and sigma^2 are kept as (hi, lo) float pairs, so no FP64
// arithmetic is left but the maps of the API's own FP64 input and output.
struct ddr {
  float hi, lo;
  __device__ __forceinline__ ddr() : hi(0.f), lo(0.f) {}
  __device__ __forceinline__ ddr(float h, float l) : hi(h), lo(l) {}
  __device__ __forceinline__ ddr(int v) : hi((float)v), lo(0.f) {}
  __device__ __forceinline__ ddr(double v) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
  }
  __device__ __forceinline__ explicit operator double() const {
    return (double)hi + (double)lo;
  }
};
__device__ __forceinline__ ddr ddr_norm(float s, float e) {
  const float h = __fadd_rn(s, e);
  return ddr(h, __fsub_rn(e, __fsub_rn(h, s)));
}
__device__ __forceinline__ ddr operator+(ddr a, ddr b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  return ddr_norm(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ ddr operator-(ddr a) { return ddr(-a.hi, -a.lo); }
__device__ __forceinline__ ddr operator-(ddr a, ddr b) { return a + (-b); }
__device__ __forceinline__ ddr operator*(ddr a, ddr b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  return ddr_norm(p, e);
}
__device__ __forceinline__ ddr &operator*=(ddr &a, ddr b) {
  a = a * b;
  return a;
}
// a / b: the quotient of the hi parts, corrected by the remainder a - q b
// (finite b only)
__device__ __forceinline__ ddr operator/(ddr a, ddr b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const ddr r = a - ddr(q1, 0.f) * b;
  return ddr_norm(q1, __fdiv_rn(r.hi, b.hi));
}
__device__ __forceinline__ bool operator<(ddr a, ddr b) {
  return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}

struct ddc {
  ddr x, y;
};
template <> struct CT<ddc> {
  typedef ddr T;
  typedef float4 G;  // F, G as double-float pairs (re hi, re lo, im hi, im lo)
  typedef float4 W;  // tables in the same form
  static __device__ __forceinline__ ddc ld(const G *p) {
    const float4 v = *p;
    return {ddr(v.x, v.y), ddr(v.z, v.w)};
  }
  static __device__ __forceinline__ ddc ldw(const W *p) {
    const float4 v = *p;
    return {ddr(v.x, v.y), ddr(v.z, v.w)};
  }
  static __device__ __forceinline__ void st(G *p, ddc v) {
    *p = make_float4(v.x.hi, v.x.lo, v.y.hi, v.y.lo);
  }
  static __device__ __forceinline__ ddc mk(ddr a, ddr b) { return {a, b}; }
  // sin, cos of pi r / den, rounded from FP64
  static __device__ __forceinline__ void sincospi_(int r, int den, ddr *s, ddr *c) {
    double sd, cd;
    sincospi((double)r / (double)den, &sd, &cd);
    *s = ddr(sd);
    *c = ddr(cd);
  }
};
template <> struct TwPass<ddc> {
  const float4 *tw;
  int ts;
  __device__ __forceinline__ TwPass(int h, const float4 *t, int Mmax)
      : tw(t), ts(Mmax / (2 * h)) {}
  __device__ __forceinline__ void pair(int j, ddc &w2h, ddc &wh) const {
    w2h = CT<ddc>::ldw(tw + j * ts);
    wh = CT<ddc>::ldw(tw + 2 * j * ts);
  }
};

// natural -> bit-reversed; INV uses e^{+2 pi i jk/M}.  Two radix-2 stages
// (spans h and h/2) per pass over shared memory ("radix-2^2"): the output
// order stays bit-reversed, and the barriers and shared-memory round trips
// halve.  An odd number of stages ends with one radix-2 pass of span 1.
// Where the twiddle index j = b mod q is the same for all of a thread's
// butterflies (q <= blockDim), the twiddles are computed once per pass.
template <typename T2, bool INV>
__device__ void fft_dif(T2 *buf, int M, const typename CT<T2>::W *__restrict__ tw, int Mmax) {
  int h = M >> 1;
  for (; h >= 2; h >>= 2) {
    const int q = h >> 1;
    const TwPass<T2> tp(h, tw, Mmax);
    const bool fixed = q <= (int)blockDim.x;
    T2 w1f, w2f;
    if (fixed) tp.pair((int)threadIdx.x & (q - 1), w1f, w2f);
    #pragma unroll 4
    for (int b = threadIdx.x; b < (M >> 2); b += blockDim.x) {
      const int j = b & (q - 1);
      const int i0 = ((b - j) << 2) + j, i1 = i0 + q, i2 = i0 + h, i3 = i2 + q;
      T2 w1 = w1f, w2 = w2f;  // W_2h^j, W_h^j
      if (!fixed) tp.pair(j, w1, w2);
      const T2 x0 = buf[sw(i0)], x1 = buf[sw(i1)], x2 = buf[sw(i2)], x3 = buf[sw(i3)];
      const T2 a0 = cadd(x0, x2), a1 = cadd(x1, x3);
      const T2 a2 = INV ? cmulc(csub(x0, x2), w1) : cmul(csub(x0, x2), w1);
      const T2 a3 = rot_q<T2, INV>(INV ? cmulc(csub(x1, x3), w1) : cmul(csub(x1, x3), w1));
      buf[sw(i0)] = cadd(a0, a1);
      buf[sw(i1)] = INV ? cmulc(csub(a0, a1), w2) : cmul(csub(a0, a1), w2);
      buf[sw(i2)] = cadd(a2, a3);
      buf[sw(i3)] = INV ? cmulc(csub(a2, a3), w2) : cmul(csub(a2, a3), w2);
    }
    __syncthreads();
  }
  if (h == 1) {
    for (int b = threadIdx.x; b < (M >> 1); b += blockDim.x) {
      const T2 a = buf[sw(2 * b)], c = buf[sw(2 * b + 1)];
      buf[sw(2 * b)] = cadd(a, c);
      buf[sw(2 * b + 1)] = csub(a, c);
    }
    __syncthreads();
  }
}

// bit-reversed -> natural; an odd number of stages starts with one radix-2
// pass of span 1, then pairs of stages (spans h and 2h) per pass
template <typename T2, bool INV>
__device__ void fft_dit(T2 *buf, int M, const typename CT<T2>::W *__restrict__ tw, int Mmax) {
  int h = 1;
  int bits = 0;
  while ((1 << bits) < M) ++bits;
  if (bits & 1) {
    for (int b = threadIdx.x; b < (M >> 1); b += blockDim.x) {
      const T2 a = buf[sw(2 * b)], c = buf[sw(2 * b + 1)];
      buf[sw(2 * b)] = cadd(a, c);
      buf[sw(2 * b + 1)] = csub(a, c);
    }
    __syncthreads();
    h = 2;
  }
  for (; h < M; h <<= 2) {
    const TwPass<T2> tp(2 * h, tw, Mmax);  // pair(j) = (W_4h^j, W_2h^j)
    const bool fixed = h <= (int)blockDim.x;
    T2 waf, wbf;
    if (fixed) tp.pair((int)threadIdx.x & (h - 1), wbf, waf);
    #pragma unroll 4
    for (int b = threadIdx.x; b < (M >> 2); b += blockDim.x) {
      const int j = b & (h - 1);
      const int i0 = ((b - j) << 2) + j, i1 = i0 + h, i2 = i0 + 2 * h, i3 = i2 + h;
      T2 wa = waf, wb = wbf;  // W_2h^j, W_4h^j
      if (!fixed) tp.pair(j, wb, wa);
      const T2 x0 = buf[sw(i0)], x1 = buf[sw(i1)], x2 = buf[sw(i2)], x3 = buf[sw(i3)];
      const T2 c1 = INV ? cmulc(x1, wa) : cmul(x1, wa);
      const T2 c3 = INV ? cmulc(x3, wa) : cmul(x3, wa);
      const T2 a0 = cadd(x0, c1), a1 = csub(x0, c1);
      const T2 a2 = cadd(x2, c3), a3 = csub(x2, c3);
      const T2 d2 = INV ? cmulc(a2, wb) : cmul(a2, wb);
      const T2 d3 = rot_q<T2, INV>(INV ? cmulc(a3, wb) : cmul(a3, wb));
      buf[sw(i0)] = cadd(a0, d2);
      buf[sw(i2)] = csub(a0, d2);
      buf[sw(i1)] = cadd(a1, d3);
      buf[sw(i3)] = csub(a1, d3);
    }
    __syncthreads();
  }
}

// In place: buf[0..n) holds a_j = x_j conj(w_j) and buf[n..M) zeros on entry;
// on exit buf[0..n) holds X = DFT_n(x).
template <typename T2>
__device__ void bluestein(T2 *buf, int n, int M, const typename CT<T2>::W *__restrict__ tw,
                          int Mmax, const typename CT<T2>::W *__restrict__ chirp,
                          const typename CT<T2>::W *__restrict__ bhat) {
  fft_dif<T2, false>(buf, M, tw, Mmax);
  #pragma unroll 8
  for (int q = threadIdx.x; q < M; q += blockDim.x)
    buf[sw(q)] = cmul(buf[sw(q)], CT<T2>::ldw(bhat + q));
  __syncthreads();
  fft_dit<T2, true>(buf, M, tw, Mmax);
  #pragma unroll 8
  for (int k = threadIdx.x; k < n; k += blockDim.x)
    buf[sw(k)] = cmulc(buf[sw(k)], CT<T2>::ldw(chirp + k));
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
                                         const typename CT<T2>::W *__restrict__ tw,
                                         const typename CT<T2>::W *__restrict__ ph) {
  typedef typename CT<T2>::T T;
  if (num == 0) return CT<T2>::mk((T)1, (T)0);
  if (tstep > 0) return cconj(CT<T2>::ldw(tw + k * tstep));
  if (ph) return CT<T2>::ldw(ph + k);  // the ring's own phase table
  T s, c;
  CT<T2>::sincospi_(k, den, &s, &c);
  return CT<T2>::mk(c, s);
}

// c_k = sum over m = +-k mod n, |m| <= L, of F[m] e^{i m phi0}
//     = e^{i k phi0} (sum_j sgn^j F[k + j n] + sum_{j >= 1} sgn^j conj F[j n - k])
// When n > L each sum has at most one term (every equatorial ring, the outer
// polar rings): the two loads are issued together, not in dependent loops.
template <typename T2>
__device__ __forceinline__ T2 fold(const typename CT<T2>::G *__restrict__ Fr, int k, int n,
                                   int L, typename CT<T2>::T sgn, T2 ph) {
  typedef typename CT<T2>::T T;
  T2 acc = CT<T2>::mk((T)0, (T)0);
  if (n > L) {
    const T2 zero = CT<T2>::mk((T)0, (T)0);
    const T2 a = k <= L ? CT<T2>::ld(Fr + k) : zero;
    const T2 b = n - k <= L ? CT<T2>::ld(Fr + (n - k)) : zero;
    acc = CT<T2>::mk(a.x + sgn * b.x, a.y - sgn * b.y);
    return cmul(acc, ph);
  }
  T s = (T)1;
#pragma unroll 4
  for (int m = k; m <= L; m += n) {
    const T2 f = CT<T2>::ld(Fr + m);
    acc = CT<T2>::mk(acc.x + s * f.x, acc.y + s * f.y);
    s *= sgn;
  }
  s = sgn;
#pragma unroll 4
  for (int m = n - k; m <= L; m += n) {  // m >= 1 since k < n
    const T2 f = CT<T2>::ld(Fr + m);
    acc = CT<T2>::mk(acc.x + s * f.x, acc.y - s * f.y);
    s *= sgn;
  }
  return cmul(acc, ph);
}

// threads per ring pair: 512 for launches whose largest FFT has 8192 or more
// points (the polar Bluestein rings at Nside >= 1024: more warps to hide the
// latency of the table and twiddle loads at 3 CTAs per SM), else 256
constexpr int RING_THREADS = 256;
constexpr int RING_THREADS_BIG = 512;

template <typename T2, int MODE>
__global__ void __launch_bounds__(RING_THREADS_BIG)
    k_ring(const RingPair *__restrict__ pairs, int pair_base, int lmax,
           const typename CT<T2>::G *__restrict__ F, typename CT<T2>::G *__restrict__ G,
           const double *__restrict__ in_map, double *__restrict__ out_map,
           const double *__restrict__ nvar, const typename CT<T2>::W *__restrict__ tw,
           int Mmax, const typename CT<T2>::W *__restrict__ chirp_all,
           const typename CT<T2>::W *__restrict__ bhat_all,
           const SolverState *__restrict__ st, int lstatic, int reverse,
           const float *__restrict__ in32, const float *__restrict__ nv32, int red_ofs,
           const typename CT<T2>::W *__restrict__ phase_all,
           const float2 *__restrict__ in_dd, const float2 *__restrict__ nv_dd,
           long bstride_f, long bstride_m) {
  typedef typename CT<T2>::T T;
  typedef typename CT<T2>::G GT;
  typedef typename CT<T2>::W WT;
  // reverse: the polar rings grow with the pair index; taking the largest
  // first keeps the small ones for the tail of the launch
  const int blk = reverse ? (int)(gridDim.x - 1 - blockIdx.x) : (int)blockIdx.x;
  // batched launches (plain transforms of several maps): map blockIdx.y
  if (gridDim.y > 1) {
    const long bm = blockIdx.y;
    if (F) F += bm * bstride_f;
    if (G) G += bm * bstride_f;
    if (in_map) in_map += bm * bstride_m;
    if (out_map) out_map += bm * bstride_m;
  }
  const RingPair rp = pairs[pair_base + blk];
  int Lf = lstatic, Lg = lstatic;
  double xi = 0.0, mu = 0.0, alpha = 1.0;
  if (st) {
    if (st->done) return;
    Lf = st->lcur;
    Lg = max(st->lcur, st->lnext);
    xi = st->xi;
    mu = st->mu;
    alpha = st->alpha;
  }
  // FP32 step: w = (xi / alpha) / (sigma^2 / alpha + mu / alpha) -- the same
  // weight with every operand scaled to O(1) for the FP32 range.  The two
  // quotients are uniform: lane 0 of each warp divides (FP64 division is
  // slow on this part) and broadcasts.
  constexpr bool F32STEP = MODE == RING_FUSED && sizeof(T) == 4;
  float xia = 0.f, mua = 0.f;
  if constexpr (F32STEP) {
    if ((threadIdx.x & 31) == 0) {
      xia = (float)(xi / alpha);
      mua = (float)(mu / alpha);
    }
    xia = __shfl_sync(0xffffffffu, xia, 0);
    mua = __shfl_sync(0xffffffffu, mua, 0);
  }
  // the double-float step's xi and mu (converted once)
  ddr xd(0), md(0);
  if constexpr (std::is_same<T2, ddc>::value && MODE == RING_FUSED) {
    xd = ddr(xi);
    md = ddr(mu);
  }
  extern __shared__ __align__(16) unsigned char smraw[];
  T2 *buf = reinterpret_cast<T2 *>(smraw);
  const int n = rp.nphi, M = rp.fftM;
  const bool blue = M != n;
  int bits = 0;
  while ((1 << bits) < M) ++bits;
  const WT *chirp = blue ? chirp_all + rp.chirp_ofs : nullptr;
  const WT *bhat = blue ? bhat_all + rp.bhat_ofs : nullptr;
  const WT *phs = (blue && phase_all) ? phase_all + rp.chirp_ofs : nullptr;
  const long stride = lmax + 1;
  const bool south = rp.ringS >= 0;
  const T2 zero = CT<T2>::mk((T)0, (T)0);
  const T sgn = rp.phi_num ? (T)-1 : (T)1;  // e^{i n phi0}
  const int tstep = (rp.phi_num && Mmax % (2 * rp.phi_den) == 0) ? Mmax / (2 * rp.phi_den) : 0;

  if (MODE != RING_ANALYSIS) {
    const GT *FN = F + rp.ringN * stride;
    const GT *FS = south ? F + rp.ringS * stride : nullptr;
    if (n < (int)blockDim.x) {
      // small rings (n < threads): each k's sums over j are split across
      // P = threads / n threads (j = part mod P), whose partials are added
      // in part order -- all threads load, none walks (L+1)/n terms alone
      T2 *red = buf + red_ofs;  // [2][blockDim]: north, south partials
      const int P = blockDim.x / n, k = threadIdx.x % n, part = threadIdx.x / n;
      if (part < P) {
        T2 pN = zero, pS = zero;
        if (Lf >= 0) {
          for (int j = part; k + j * n <= Lf; j += P) {  // m = k + j n
            const T s = (sgn < (T)0 && (j & 1)) ? (T)-1 : (T)1;
            const T2 f = CT<T2>::ld(FN + (k + j * n));
            pN = CT<T2>::mk(pN.x + s * f.x, pN.y + s * f.y);
            if (south) {
              const T2 g = CT<T2>::ld(FS + (k + j * n));
              pS = CT<T2>::mk(pS.x + s * g.x, pS.y + s * g.y);
            }
          }
          for (int j = 1 + part; j * n - k <= Lf; j += P) {  // m = j n - k, conj
            const T s = (sgn < (T)0 && (j & 1)) ? (T)-1 : (T)1;
            const T2 f = CT<T2>::ld(FN + (j * n - k));
            pN = CT<T2>::mk(pN.x + s * f.x, pN.y - s * f.y);
            if (south) {
              const T2 g = CT<T2>::ld(FS + (j * n - k));
              pS = CT<T2>::mk(pS.x + s * g.x, pS.y - s * g.y);
            }
          }
        }
        red[threadIdx.x] = pN;
        red[blockDim.x + threadIdx.x] = pS;
      }
      __syncthreads();
      if ((int)threadIdx.x < n) {
        T2 cN = zero, cS = zero;
        for (int q = 0; q < P; ++q) {
          cN = cadd(cN, red[q * n + k]);
          cS = cadd(cS, red[blockDim.x + q * n + k]);
        }
        const T2 ph = ring_phase<T2>(k, rp.phi_num, rp.phi_den, tstep, tw, phs);
        cN = cmul(cN, ph);
        cS = cmul(cS, ph);
        const T2 Zk = CT<T2>::mk(cN.x - cS.y, cN.y + cS.x);  // cN + i cS
        buf[sw(k)] = blue ? cmulc(cconj(Zk), CT<T2>::ldw(chirp + k)) : Zk;
      }
    } else {
      #pragma unroll 4
      for (int k = threadIdx.x; k < n; k += blockDim.x) {
        T2 cN = zero, cS = zero;
        if (Lf >= 0 && (k <= Lf || n - k <= Lf)) {
          const T2 ph = ring_phase<T2>(k, rp.phi_num, rp.phi_den, tstep, tw, phs);
          cN = fold(FN, k, n, Lf, sgn, ph);
          if (south) cS = fold(FS, k, n, Lf, sgn, ph);
        }
        const T2 Zk = CT<T2>::mk(cN.x - cS.y, cN.y + cS.x);  // cN + i cS
        buf[sw(k)] = blue ? cmulc(cconj(Zk), CT<T2>::ldw(chirp + k)) : Zk;
      }
    }
    if (blue)
      for (int k = n + threadIdx.x; k < M; k += blockDim.x) buf[sw(k)] = zero;
    __syncthreads();
    if (blue) {
      bluestein<T2>(buf, n, M, tw, Mmax, chirp, bhat);  // DFT(conj Z)
    } else {
      fft_dif<T2, true>(buf, M, tw, Mmax);  // bit-reversed output
    }
    // pixel step; position q holds pixel j
    #pragma unroll 4
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
      const int j = blue ? q : bitrev_n(q, bits);
      T2 zz = buf[sw(q)];
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
        T2 tt;
        if constexpr (std::is_same<T2, ddc>::value) {
          // double-float step on double-float copies of d and sigma^2
          const float2 vN = nv_dd[pN];
          const ddr wN = isinf(vN.x) ? ddr(0) : xd / (ddr(vN.x, vN.y) + md);
          const ddr dN = in_dd ? ddr(in_dd[pN].x, in_dd[pN].y) : ddr(0);
          const ddr tN = zz.x + wN * (dN - zz.x);
          ddr tS(0);
          if (south) {
            const float2 vS = nv_dd[pS];
            const ddr wS = isinf(vS.x) ? ddr(0) : xd / (ddr(vS.x, vS.y) + md);
            const ddr dS = in_dd ? ddr(in_dd[pS].x, in_dd[pS].y) : ddr(0);
            tS = zz.y + wS * (dS - zz.y);
          }
          tt = CT<T2>::mk(tN, tS);
        } else if constexpr (F32STEP) {
          // 0 on masked pixels (sigma^2 / alpha = +inf)
          const float sNf = zz.x, sSf = zz.y;
          float tN = sNf + xia / (nv32[pN] + mua) * ((in32 ? in32[pN] : 0.f) - sNf);
          float tS = 0.f;
          if (south) tS = sSf + xia / (nv32[pS] + mua) * ((in32 ? in32[pS] : 0.f) - sSf);
          tt = CT<T2>::mk((T)tN, (T)tS);
        } else {
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
          tt = CT<T2>::mk((T)tN, (T)tS);
        }
        buf[sw(q)] = blue ? cmulc(tt, CT<T2>::ldw(chirp + q)) : tt;
      }
    }
    if (MODE == RING_SYNTH) return;
    if (blue)
      for (int k = n + threadIdx.x; k < M; k += blockDim.x) buf[sw(k)] = zero;
    __syncthreads();
  } else {
    #pragma unroll 4
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      const double tN = in_map[rp.ofsN + j];
      const double tS = south ? in_map[rp.ofsS + j] : 0.0;
      const T2 tt = CT<T2>::mk((T)tN, (T)tS);
      if (blue)
        buf[sw(j)] = cmulc(tt, CT<T2>::ldw(chirp + j));
      else
        buf[sw(bitrev_n(j, bits))] = tt;
    }
    if (blue)
      for (int k = n + threadIdx.x; k < M; k += blockDim.x) buf[sw(k)] = zero;
    __syncthreads();
  }
  // forward DFT of t (natural order output)
  if (blue)
    bluestein<T2>(buf, n, M, tw, Mmax, chirp, bhat);
  else
    fft_dit<T2, false>(buf, M, tw, Mmax);
  // split the two real rings and apply e^{-i m phi0}: for m = k + j n,
  // G[m] = sgn^j e^{-i k phi0} X_k (X^N or X^S)
  GT *GN = G + rp.ringN * stride;
  GT *GS = south ? G + rp.ringS * stride : nullptr;
  const T half = (T)0.5;
  const int kmax = min(n - 1, Lg);
  // small rings: the copies m = k + j n of each k are split across
  // P = threads / n threads, as in the fold
  const int P = n < (int)blockDim.x ? (int)blockDim.x / n : 1;
  const int kstep = n < (int)blockDim.x ? n : (int)blockDim.x;
  const int part = n < (int)blockDim.x ? (int)threadIdx.x / n : 0;
  if (part < P) {
    #pragma unroll 4
    for (int k = (n < (int)blockDim.x ? (int)threadIdx.x % n : (int)threadIdx.x);
         k <= kmax; k += kstep) {
      const int kk = k == 0 ? 0 : n - k;
      const T2 X = buf[sw(k)], Xc = cconj(buf[sw(kk)]);
      const T2 ph = cconj(ring_phase<T2>(k, rp.phi_num, rp.phi_den, tstep, tw, phs));
      const T2 tN = cmul(CT<T2>::mk(half * (X.x + Xc.x), half * (X.y + Xc.y)), ph);
      // (X - Xc) / (2i)
      const T2 dlt = csub(X, Xc);
      const T2 tS = cmul(CT<T2>::mk(half * dlt.y, -half * dlt.x), ph);
      for (int j = part; k + j * n <= Lg; j += P) {
        const int m = k + j * n;
        const T s = (sgn < (T)0 && (j & 1)) ? (T)-1 : (T)1;
        CT<T2>::st(GN + m, CT<T2>::mk(s * tN.x, s * tN.y));
        if (south) CT<T2>::st(GS + m, CT<T2>::mk(s * tS.x, s * tS.y));
      }
    }
  }
}

template <typename T2> struct Tables;
template <> struct Tables<double2> {
  static const double2 *ph(const Plan &) { return nullptr; }
  static const double2 *tw(const Plan &P) { return P.tw64; }
  static const double2 *ch(const Plan &P) { return P.chirp64; }
  static const double2 *bh(const Plan &P) { return P.bhat64; }
};
template <> struct Tables<float2> {
  static const float2 *ph(const Plan &) { return nullptr; }
  static const float2 *tw(const Plan &P) { return P.tw32; }
  static const float2 *ch(const Plan &P) { return P.chirp32; }
  static const float2 *bh(const Plan &P) { return P.bhat32; }
};
template <> struct Tables<ddc> {
  static const float4 *ph(const Plan &P) { return P.phasedd; }
  static const float4 *tw(const Plan &P) { return P.twdd; }
  static const float4 *ch(const Plan &P) { return P.chirpdd; }
  static const float4 *bh(const Plan &P) { return P.bhatdd; }
};

template <typename T2, int MODE>
static wf_status launch_ring_mode(const Plan &P, const typename CT<T2>::G *F,
                                  typename CT<T2>::G *G, const double *in_map,
                                  double *out_map, const SolverState *st, int lstatic,
                                  const float *in32, const float2 *in_dd = nullptr,
                                  int nbatch = 1, long bstride_f = 0, long bstride_m = 0) {
  auto kern = k_ring<T2, MODE>;
  // two launches: the polar rings (pairs 0 .. nside-2, Bluestein unless n is
  // a power of two) and the equatorial belt (pairs nside-1 .. 2 nside-1);
  // they touch disjoint rings and run concurrently on two streams
  const int npolar = P.nside - 1;
  const int groups[2][2] = {{0, npolar}, {npolar, P.npairs}};
  const bool fork = npolar > 0 && P.side_stream;
  if (fork) {
    WF_CUDA(cudaEventRecord(P.fork_ev, P.stream));
    WF_CUDA(cudaStreamWaitEvent(P.side_stream, P.fork_ev, 0));
  }
  for (int g = 0; g < 2; ++g) {
    const int b = groups[g][0], e = groups[g][1];
    if (e <= b) continue;
    int Mg = 1, nmin = INT_MAX;
    for (int k = b; k < e; ++k) {
      Mg = std::max(Mg, P.pairs_h[k].fftM);
      nmin = std::min(nmin, P.pairs_h[k].nphi);
    }
    const int threads = Mg >= 8192 ? RING_THREADS_BIG : RING_THREADS;
    // rings with fewer pixels than threads fold through a partial-sum area
    // of 2 x threads entries placed after the FFT buffer
    const int red_ofs = nmin < threads ? Mg : 0;
    const size_t smem = sizeof(T2) * (Mg + (nmin < threads ? 2 * threads : 0));
    cudaStream_t s = (fork && g == 1) ? P.side_stream : P.stream;
    ++P.nlaunch;
    kern<<<dim3(e - b, nbatch), threads, smem, s>>>(
        P.pairs, b, P.lmax, F, G, in_map, out_map, P.nvar, Tables<T2>::tw(P),
        P.fftMmax, Tables<T2>::ch(P), Tables<T2>::bh(P), st, lstatic, g == 0, in32,
        P.nvar32, red_ofs, Tables<T2>::ph(P), in_dd, P.nvardd, bstride_f, bstride_m);
    WF_CUDA(cudaGetLastError());
  }
  if (fork) {
    WF_CUDA(cudaEventRecord(P.join_ev, P.side_stream));
    WF_CUDA(cudaStreamWaitEvent(P.stream, P.join_ev, 0));
  }
  return WF_OK;
}

template <typename T2>
wf_status launch_ring(const Plan &P, int mode, const T2 *F, T2 *G,
                      const double *in_map, double *out_map,
                      const SolverState *st, int lstatic, const float *in32) {
  switch (mode) {
    case RING_SYNTH:
      return launch_ring_mode<T2, RING_SYNTH>(P, F, G, in_map, out_map, st, lstatic, in32);
    case RING_ANALYSIS:
      return launch_ring_mode<T2, RING_ANALYSIS>(P, F, G, in_map, out_map, st, lstatic,
                                                 in32);
    default:
      if (sizeof(T2) == sizeof(float2) && !P.nvar32) {
        set_error("ring step: the plan has no noise variance");
        return WF_ERR_STATE;
      }
      return launch_ring_mode<T2, RING_FUSED>(P, F, G, in_map, out_map, st, lstatic, in32);
  }
}

wf_status launch_ring_batch32(const Plan &P, int mode, const float2 *F, float2 *G,
                             const double *in_map, double *out_map, int nbatch,
                             long fstride, long mstride) {
  if (mode == RING_SYNTH)
    return launch_ring_mode<float2, RING_SYNTH>(P, F, G, in_map, out_map, nullptr, P.lmax,
                                                nullptr, nullptr, nbatch, fstride, mstride);
  if (mode == RING_ANALYSIS)
    return launch_ring_mode<float2, RING_ANALYSIS>(P, F, G, in_map, out_map, nullptr,
                                                   P.lmax, nullptr, nullptr, nbatch, fstride,
                                                   mstride);
  set_error("batched ring transform: synthesis or analysis only");
  return WF_ERR_ARG;
}

wf_status launch_ring_dd(const Plan &P, int mode, const float4 *F, float4 *G,
                         const double *in_map, double *out_map, const SolverState *st,
                         int lstatic, const float2 *in_dd) {
  switch (mode) {
    case RING_SYNTH:
      return launch_ring_mode<ddc, RING_SYNTH>(P, F, G, in_map, out_map, st, lstatic,
                                               nullptr);
    case RING_ANALYSIS:
      return launch_ring_mode<ddc, RING_ANALYSIS>(P, F, G, in_map, out_map, st, lstatic,
                                                  nullptr);
    default:
      if (!P.nvardd) {
        set_error("ring step: the plan has no noise variance");
        return WF_ERR_STATE;
      }
      return launch_ring_mode<ddc, RING_FUSED>(P, F, G, in_map, out_map, st, lstatic,
                                               nullptr, in_dd);
  }
}

__global__ void k_to_dd(const double *__restrict__ in, float2 *__restrict__ out, long n) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long)gridDim.x * blockDim.x) {
    const double v = in[i];
    const float h = (float)v;
    out[i] = make_float2(h, isinf(v) ? 0.f : (float)(v - (double)h));
  }
}

wf_status launch_to_dd(const Plan &P, const double *in, float2 *out, long n) {
  ++P.nlaunch;
  k_to_dd<<<304, 256, 0, P.stream>>>(in, out, n);
  WF_CUDA(cudaGetLastError());
  return WF_OK;
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
  WF_CUDA(cudaFuncSetAttribute(k_ring<ddc, RING_SYNTH>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  WF_CUDA(cudaFuncSetAttribute(k_ring<ddc, RING_ANALYSIS>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  WF_CUDA(cudaFuncSetAttribute(k_ring<ddc, RING_FUSED>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  return WF_OK;
}

template wf_status launch_ring<double2>(const Plan &, int, const double2 *,
                                        double2 *, const double *, double *,
                                        const SolverState *, int, const float *);
template wf_status launch_ring<float2>(const Plan &, int, const float2 *, float2 *,
                                       const double *, double *,
                                       const SolverState *, int, const float *);

}  // namespace wf
