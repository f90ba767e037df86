// legendre.cu -- associated-Legendre synthesis and analysis between ring
// Fourier coefficients F_r[m] and harmonic coefficients a_lm.
//
// Synthesis (the Y step of the paper's Algorithm 2 moved to the sphere):
//   F_r[m] = sum_{l >= m} lam_lm(z_r) a_lm,
// computed for the north and south ring of a pair at once from the parity
// lam_lm(-z) = (-1)^(l+m) lam_lm(z): E = sum over even l-m, O = over odd,
// F_north = E + O, F_south = E - O.
// Analysis (Omega Y^T):
//   a_lm = Omega sum_r lam_lm(z_r) G_r[m]
//        = Omega g_l sum_pairs u_l(z) (G_N + (-1)^(l+m) G_S).
// Both run the rescaled recurrence u_l = c_l z u_{l-1} - u_{l-2}
// (lam = g u, tables from plan.cu) from FP64 seeds at the first l where
// |lam| >= 2^-100, so no value ever leaves the normal range of FP32 or FP64.
//
// Work split: synthesis -- one CTA row per m, one thread per 2 ring pairs,
// a warp-uniform loop over l (pairs with a later seed stay at u = 0 until
// their seed is injected).  Analysis -- one CTA per m, warps own ring pairs,
// each warp accumulates 16 l values x (re, im) per lane and reduces them
// across the warp with a 31-shuffle transpose-reduction; per-warp partial
// sums live in shared memory and are combined in a fixed order at the end
// (deterministic).  The analysis of the solver fuses the truncated-spectrum
// filter f_l = Sbar_l / (Sbar_l + xi Omega), Sbar_l = max(C_l - mu Omega, 0)
// (Eq. 15, App. B) and the partial sums of the Cauchy norms.
#include <limits.h>

#include "wf_internal.cuh"

namespace wf {

template <typename T> struct Vec2;
template <> struct Vec2<double> {
  typedef double2 type;
  static __device__ __forceinline__ double2 make(double a, double b) {
    return make_double2(a, b);
  }
};
template <> struct Vec2<float> {
  typedef float2 type;
  static __device__ __forceinline__ float2 make(float a, float b) {
    return make_float2(a, b);
  }
};
template <typename T2> struct Scalar;
template <> struct Scalar<double2> { typedef double type; };
template <> struct Scalar<float2> { typedef float type; };

__device__ __forceinline__ long lm_index(int lmax, int l, int m) {
  return (long)m * (2 * lmax + 1 - m) / 2 + l;
}

template <typename T>
__device__ __forceinline__ T coef(const double *rc, const float *rc32, long i);
template <>
__device__ __forceinline__ double coef<double>(const double *rc, const float *,
                                               long i) {
  return rc[i];
}
template <>
__device__ __forceinline__ float coef<float>(const double *, const float *rc32,
                                             long i) {
  return rc32[i];
}

__device__ __forceinline__ int warp_min(int v) {
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ int warp_max(int v) {
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// One step of u_l = c_l z u_{l-1} - u_{l-2}.  In FP32, z = cos(theta) is
// carried as zh + zl (two floats): rounding z alone to FP32 displaces a ring
// near the pole by ~6e-8 / sin(theta) rad, a phase error of l times that.
__device__ __forceinline__ double rec_step(double c, double zh, double, double u1,
                                           double u2) {
  return fma(c * zh, u1, -u2);
}
__device__ __forceinline__ float rec_step(float c, float zh, float zl, float u1,
                                          float u2) {
  const float a = c * u1;
  return fmaf(a, zh, fmaf(a, zl, -u2));
}
template <typename T>
__device__ __forceinline__ void split_z(double z, T &zh, T &zl) {
  zh = (T)z;
  zl = (T)(z - (double)zh);
}

static inline size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }
__device__ __forceinline__ size_t align16d(size_t b) { return (b + 15) & ~(size_t)15; }

// ------------------------------------------------------------------ synthesis
constexpr int SYN_THREADS = 128;

template <typename T, int NP>
__global__ void __launch_bounds__(SYN_THREADS)
    k_legendre_synth(const RingPair *__restrict__ pairs, int npairs, int lmax,
                     const double *__restrict__ rc, const float *__restrict__ rc32,
                     const double *__restrict__ rg, const int *__restrict__ seed_l,
                     const double2 *__restrict__ seed_u,
                     const typename Vec2<T>::type *__restrict__ xs,
                     typename Vec2<T>::type *__restrict__ F,
                     const SolverState *__restrict__ st, int lstatic) {
  typedef typename Vec2<T>::type T2;
  const int m = blockIdx.y;
  int L = lstatic;
  if (st) {
    if (st->done) return;
    L = st->lcur;
  }
  if (m > L) return;  // the ring step ignores m above the band
  extern __shared__ __align__(16) unsigned char smraw[];
  const int nl = L - m + 1;
  T2 *sx = reinterpret_cast<T2 *>(smraw);
  T *sc = reinterpret_cast<T *>(smraw + align16d(sizeof(T2) * nl));
  const long base = lm_index(lmax, m, m);
  for (int j = threadIdx.x; j < nl; j += blockDim.x) {
    const long i = base + j;
    sc[j] = coef<T>(rc, rc32, i);
    sx[j] = xs[i];
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int pair0 = (blockIdx.x * (SYN_THREADS / 32) + warp) * 32 * NP;
  if (pair0 >= npairs) return;

  T zh[NP], zl[NP], u1[NP], u2[NP], s0[NP], s1[NP];
  T er[NP], ei[NP], orr[NP], oi[NP];
  int ls[NP];
  int lmin = INT_MAX, linj = -1;
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    const int k = pair0 + lane + 32 * j;
    u1[j] = u2[j] = er[j] = ei[j] = orr[j] = oi[j] = (T)0;
    if (k < npairs) {
      split_z<T>(pairs[k].z, zh[j], zl[j]);
      ls[j] = seed_l[(long)m * npairs + k];
      const double2 su = seed_u[(long)m * npairs + k];
      s0[j] = (T)su.x;
      s1[j] = (T)su.y;
    } else {
      zh[j] = zl[j] = (T)0;
      ls[j] = INT_MAX - 2;
      s0[j] = s1[j] = (T)0;
    }
    if (ls[j] <= L) {
      lmin = min(lmin, ls[j]);
      linj = max(linj, ls[j] + 1);
    }
  }
  lmin = warp_min(lmin);
  linj = warp_max(linj);

  if (lmin <= L) {
    int l = lmin;
    if ((l - m) & 1) --l;
    // phase A: seeds may still be injected
    for (; l <= L && l <= linj; l += 2) {
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        const int ll = l + p;
        const int li = min(ll, L) - m;  // ll > L only on the last odd step
        const T c = sc[li];
        T2 xv = sx[li];
        if (ll > L) xv = Vec2<T>::make((T)0, (T)0);
#pragma unroll
        for (int j = 0; j < NP; ++j) {
          T u = rec_step(c, zh[j], zl[j], u1[j], u2[j]);
          u = (ll == ls[j]) ? s0[j] : u;
          u = (ll == ls[j] + 1) ? s1[j] : u;
          u2[j] = u1[j];
          u1[j] = u;
          if (p == 0) {
            er[j] = fma(u, xv.x, er[j]);
            ei[j] = fma(u, xv.y, ei[j]);
          } else {
            orr[j] = fma(u, xv.x, orr[j]);
            oi[j] = fma(u, xv.y, oi[j]);
          }
        }
      }
    }
    // phase B: plain recurrence
    // l - m is even here: (c_l, c_l+1) is one aligned pair of T and, in
    // FP32, (x_l, x_l+1) one aligned 16-byte load
    for (; l + 1 <= L; l += 2) {
      const T2 cp = *reinterpret_cast<const T2 *>(sc + (l - m));
      const T c0 = cp.x, c1 = cp.y;
      T2 x0, x1;
      if constexpr (sizeof(T) == 4) {
        const float4 xp = *reinterpret_cast<const float4 *>(sx + (l - m));
        x0 = Vec2<T>::make(xp.x, xp.y);
        x1 = Vec2<T>::make(xp.z, xp.w);
      } else {
        x0 = sx[l - m];
        x1 = sx[l + 1 - m];
      }
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        T u = rec_step(c0, zh[j], zl[j], u1[j], u2[j]);
        er[j] = fma(u, x0.x, er[j]);
        ei[j] = fma(u, x0.y, ei[j]);
        T v = rec_step(c1, zh[j], zl[j], u, u1[j]);
        orr[j] = fma(v, x1.x, orr[j]);
        oi[j] = fma(v, x1.y, oi[j]);
        u2[j] = u;
        u1[j] = v;
      }
    }
    if (l <= L) {
      const T c0 = sc[l - m];
      const T2 x0 = sx[l - m];
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        T u = rec_step(c0, zh[j], zl[j], u1[j], u2[j]);
        er[j] = fma(u, x0.x, er[j]);
        ei[j] = fma(u, x0.y, ei[j]);
      }
    }
  }
  const long stride = lmax + 1;
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    const int k = pair0 + lane + 32 * j;
    if (k >= npairs) continue;
    const RingPair &rp = pairs[k];
    F[rp.ringN * stride + m] = Vec2<T>::make(er[j] + orr[j], ei[j] + oi[j]);
    if (rp.ringS >= 0)
      F[rp.ringS * stride + m] = Vec2<T>::make(er[j] - orr[j], ei[j] - oi[j]);
  }
}

// ------------------------------------------------------------------ analysis
constexpr int ANA_THREADS = 128;
constexpr int ANA_WARPS = ANA_THREADS / 32;
constexpr int LCHUNK = 16;


// v[0..31] per lane -> lane i returns sum over lanes of v[i]
template <typename T>
__device__ __forceinline__ T transpose_reduce32(T (&v)[32], int lane) {
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    const bool upper = (lane & s) != 0;
#pragma unroll
    for (int j = 0; j < s; ++j) {
      const T send = upper ? v[j] : v[j + s];
      const T keep = upper ? v[j + s] : v[j];
      v[j] = keep + __shfl_xor_sync(0xffffffffu, send, s);
    }
  }
  return v[0];
}

// One chunk of LCHUNK consecutive l for NP ring pairs per lane: v[2 jj] and
// v[2 jj + 1] receive this lane's contribution (re, im) to a_{lc+jj, m}.
// INJ: some lane of the warp still has its seed (ls, ls + 1) in or after this
// chunk.  TAIL: the chunk runs past L (l > L contributes 0).  In FP32 full
// chunks the coefficients c_l come from shared memory in 16-byte loads
// (lc - m is a multiple of LCHUNK and the table starts 16-byte aligned).
template <typename T, int NP, bool INJ, bool TAIL>
__device__ __forceinline__ void anal_chunk(T (&v)[32], int lc, int L, int m,
                                           const T *__restrict__ sc, const T (&zh)[NP],
                                           const T (&zl)[NP], T (&u1)[NP], T (&u2)[NP],
                                           const T (&s0)[NP], const T (&s1)[NP],
                                           const int (&ls)[NP], const T (&pr)[NP],
                                           const T (&pim)[NP], const T (&qr)[NP],
                                           const T (&qim)[NP]) {
  // FP32 full chunks: the 16 coefficients in four 16-byte loads
  constexpr bool VEC = sizeof(T) == 4 && !TAIL;
  T cc[VEC ? LCHUNK : 1];
  if constexpr (VEC) {
    const uint4 *s4 = reinterpret_cast<const uint4 *>(sc + (lc - m));
#pragma unroll
    for (int q = 0; q < LCHUNK / 4; ++q) {
      const uint4 w = s4[q];
      memcpy(&cc[4 * q], &w, 16);
    }
  }
#pragma unroll
  for (int jj = 0; jj < LCHUNK; ++jj) {
    const int l = lc + jj;
    // two partial sums (even, odd j) halve the dependent FMA chain
    T a_re = (T)0, a_im = (T)0, b_re = (T)0, b_im = (T)0;
    if (!TAIL || l <= L) {
      T c;
      if constexpr (VEC)
        c = cc[jj];
      else
        c = sc[l - m];
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        T u = rec_step(c, zh[j], zl[j], u1[j], u2[j]);
        if (INJ) {
          u = (l == ls[j]) ? s0[j] : u;
          u = (l == ls[j] + 1) ? s1[j] : u;
        }
        u2[j] = u1[j];
        u1[j] = u;
        const T pre = (jj & 1) == 0 ? pr[j] : qr[j];
        const T pim_ = (jj & 1) == 0 ? pim[j] : qim[j];
        if ((j & 1) == 0) {
          a_re = fma(u, pre, a_re);
          a_im = fma(u, pim_, a_im);
        } else {
          b_re = fma(u, pre, b_re);
          b_im = fma(u, pim_, b_im);
        }
      }
    }
    v[2 * jj] = a_re + b_re;
    v[2 * jj + 1] = a_im + b_im;
  }
}

template <typename T, int NP>
__global__ void __launch_bounds__(ANA_THREADS)
    k_legendre_anal(const RingPair *__restrict__ pairs, int npairs, int lmax,
                    const double *__restrict__ rc, const float *__restrict__ rc32,
                    const double *__restrict__ rg, const int *__restrict__ seed_l,
                    const double2 *__restrict__ seed_u,
                    const double *__restrict__ cl, double omega,
                    const typename Vec2<T>::type *__restrict__ G,
                    double2 *__restrict__ x, double *__restrict__ partials,
                    const double2 *__restrict__ src,
                    typename Vec2<T>::type *__restrict__ xs_out,
                    const SolverState *__restrict__ st, int mode, int lstatic) {
  typedef typename Vec2<T>::type T2;
  const int m = blockIdx.x;
  int L = lstatic;
  double xi = 0.0, mu = 0.0;
  if (st) {
    if (st->done) return;
    L = st->lcur;
    xi = st->xi;
    mu = st->mu;
  }
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long base = lm_index(lmax, m, m);
  const double wm = (m == 0) ? 1.0 : 2.0;
  __shared__ double red_num[ANA_THREADS], red_den[ANA_THREADS];
  double num = 0.0, den = 0.0;

  if (m <= L) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int nl = L - m + 1;
    T2 *acc = reinterpret_cast<T2 *>(smraw);  // [ANA_WARPS][nl]
    T *sc = reinterpret_cast<T *>(smraw + align16d(sizeof(T2) * nl * ANA_WARPS));
    for (int j = tid; j < nl; j += ANA_THREADS) sc[j] = coef<T>(rc, rc32, base + j);
    for (int j = tid; j < nl * ANA_WARPS; j += ANA_THREADS)
      acc[j] = Vec2<T>::make((T)0, (T)0);
    __syncthreads();
    T2 *myacc = acc + (long)warp * nl;
    const long stride = lmax + 1;

    for (int tile = 0; tile < npairs; tile += ANA_THREADS * NP) {
      const int pair0 = tile + warp * 32 * NP;
      if (pair0 >= npairs) continue;  // warp-uniform
      T zh[NP], zl[NP], u1[NP], u2[NP], s0[NP], s1[NP];
      T pr[NP], pim[NP], qr[NP], qim[NP];
      int ls[NP];
      int lmin = INT_MAX, linj = -1;
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        const int k = pair0 + lane + 32 * j;
        u1[j] = u2[j] = (T)0;
        if (k < npairs) {
          const RingPair &rp = pairs[k];
          split_z<T>(rp.z, zh[j], zl[j]);
          ls[j] = seed_l[(long)m * npairs + k];
          const double2 su = seed_u[(long)m * npairs + k];
          s0[j] = (T)su.x;
          s1[j] = (T)su.y;
          const T2 gn = G[rp.ringN * stride + m];
          T2 gs = Vec2<T>::make((T)0, (T)0);
          if (rp.ringS >= 0) gs = G[rp.ringS * stride + m];
          pr[j] = gn.x + gs.x;
          pim[j] = gn.y + gs.y;
          qr[j] = gn.x - gs.x;
          qim[j] = gn.y - gs.y;
        } else {
          zh[j] = zl[j] = s0[j] = s1[j] = pr[j] = pim[j] = qr[j] = qim[j] = (T)0;
          ls[j] = INT_MAX - 2;
        }
        if (ls[j] <= L) {
          lmin = min(lmin, ls[j]);
          linj = max(linj, ls[j] + 1);
        }
      }
      lmin = warp_min(lmin);
      linj = warp_max(linj);
      if (lmin > L) continue;
      const int lc0 = m + ((lmin - m) / LCHUNK) * LCHUNK;
      for (int lc = lc0; lc <= L; lc += LCHUNK) {
        T v[32];
        // three specialisations of the chunk body: seeds still to come in
        // this warp (selects on every step), a full chunk with every seed of
        // the warp already in (the plain recurrence: 5 FP instructions per
        // term), and the last, partial chunk
        if (lc + LCHUNK - 1 > L)
          anal_chunk<T, NP, true, true>(v, lc, L, m, sc, zh, zl, u1, u2, s0, s1, ls,
                                        pr, pim, qr, qim);
        else if (lc <= linj)
          anal_chunk<T, NP, true, false>(v, lc, L, m, sc, zh, zl, u1, u2, s0, s1, ls,
                                         pr, pim, qr, qim);
        else
          anal_chunk<T, NP, false, false>(v, lc, L, m, sc, zh, zl, u1, u2, s0, s1, ls,
                                          pr, pim, qr, qim);
        const T tot = transpose_reduce32<T>(v, lane);
        const int l = lc + (lane >> 1);
        if (l <= L) {
          T2 &dst = myacc[l - m];
          if (lane & 1)
            dst.y += tot;
          else
            dst.x += tot;
        }
      }
    }
    __syncthreads();
    for (int j = tid; j < nl; j += ANA_THREADS) {
      double sr = 0.0, si = 0.0;
#pragma unroll
      for (int w = 0; w < ANA_WARPS; ++w) {
        sr += (double)acc[w * nl + j].x;
        si += (double)acc[w * nl + j].y;
      }
      const long i = base + j;
      const double s = omega * rg[i];
      double ar = s * sr, ai = s * si;
      if (mode == ANA_FILTER) {
        const int l = m + j;
        const double sbar = fmax(cl[l] - mu * omega, 0.0);
        const double f = sbar / (sbar + xi * omega);
        if (src) {  // harmonic source term of a correction solve
          ar += xi * omega * src[i].x;
          ai += xi * omega * src[i].y;
        }
        ar *= f;
        ai *= f;
        const double2 old = x[i];
        const double dr = ar - old.x, di = ai - old.y;
        num += wm * (dr * dr + di * di);
        den += wm * (ar * ar + ai * ai);
      }
      x[i] = make_double2(ar, ai);
      if (xs_out) xs_out[i] = Vec2<T>::make((T)(rg[i] * ar), (T)(rg[i] * ai));
    }
  }
  // coefficients of this m above the band are zero
  const int lz = max(m, L + 1);
  for (int l = lz + tid; l <= lmax; l += ANA_THREADS) {
    const long i = base + (l - m);
    if (mode == ANA_FILTER) {
      const double2 old = x[i];
      num += wm * (old.x * old.x + old.y * old.y);
    }
    x[i] = make_double2(0.0, 0.0);
    if (xs_out) xs_out[i] = Vec2<T>::make((T)0, (T)0);
  }
  if (mode == ANA_FILTER) {
    red_num[tid] = num;
    red_den[tid] = den;
    __syncthreads();
    for (int s = ANA_THREADS / 2; s > 0; s >>= 1) {
      if (tid < s) {
        red_num[tid] += red_num[tid + s];
        red_den[tid] += red_den[tid + s];
      }
      __syncthreads();
    }
    if (tid == 0) {
      partials[2 * m] = red_num[0];
      partials[2 * m + 1] = red_den[0];
    }
  }
}

// ------------------------------------------------------------------ launch
template <typename T2>
struct Kernels;

template <>
struct Kernels<double2> {
  typedef double T;
};
template <>
struct Kernels<float2> {
  typedef float T;
};

template <typename T, int NP>
static void synth_variant(const Plan &P, const typename Vec2<T>::type *xs,
                          typename Vec2<T>::type *F, const SolverState *st, int lstatic) {
  typedef typename Vec2<T>::type T2;
  const size_t smem = align16(sizeof(T2) * (P.lmax + 1)) + sizeof(T) * (P.lmax + 1);
  const int pairs_per_cta = SYN_THREADS * NP;
  dim3 grid((P.npairs + pairs_per_cta - 1) / pairs_per_cta, P.lmax + 1);
  k_legendre_synth<T, NP><<<grid, SYN_THREADS, smem, P.stream>>>(
      P.pairs, P.npairs, P.lmax, P.rc, P.rc32, P.rg, P.seed_l, P.seed_u, xs, F, st,
      lstatic);
}

template <typename T, int NP>
static void anal_variant(const Plan &P, const typename Vec2<T>::type *G, double2 *x,
                         const SolverState *st, int mode, int lstatic, const double2 *src,
                         typename Vec2<T>::type *xs_out) {
  typedef typename Vec2<T>::type T2;
  const size_t smem =
      align16(sizeof(T2) * (P.lmax + 1) * ANA_WARPS) + sizeof(T) * (P.lmax + 1);
  k_legendre_anal<T, NP><<<P.lmax + 1, ANA_THREADS, smem, P.stream>>>(
      P.pairs, P.npairs, P.lmax, P.rc, P.rc32, P.rg, P.seed_l, P.seed_u, P.cl_d, P.omega,
      G, x, P.partials, src, xs_out, st, mode, lstatic);
}

// ring pairs per thread: the autotuner's choice for this plan and precision
template <typename T2>
wf_status launch_legendre_synth(const Plan &P, const T2 *xs, T2 *F,
                                const SolverState *st, int lstatic) {
  typedef typename Kernels<T2>::T T;
  const int np = P.syn_np[sizeof(T) == 4];
  ++P.nlaunch;
  switch (np) {
    case 1: synth_variant<T, 1>(P, xs, F, st, lstatic); break;
    case 4: synth_variant<T, 4>(P, xs, F, st, lstatic); break;
    default: synth_variant<T, 2>(P, xs, F, st, lstatic); break;
  }
  WF_CUDA(cudaGetLastError());
  return WF_OK;
}

template <typename T2>
wf_status launch_legendre_anal(const Plan &P, const T2 *G, double2 *x,
                               const SolverState *st, int mode, int lstatic,
                               const double2 *src, T2 *xs_out) {
  typedef typename Kernels<T2>::T T;
  const int np = P.ana_np[sizeof(T) == 4];
  ++P.nlaunch;
  switch (np) {
    case 2: anal_variant<T, 2>(P, G, x, st, mode, lstatic, src, xs_out); break;
    case 4: anal_variant<T, 4>(P, G, x, st, mode, lstatic, src, xs_out); break;
    case 16: anal_variant<T, 16>(P, G, x, st, mode, lstatic, src, xs_out); break;
    default: anal_variant<T, 8>(P, G, x, st, mode, lstatic, src, xs_out); break;
  }
  WF_CUDA(cudaGetLastError());
  return WF_OK;
}

template <typename T, int NP>
static cudaError_t set_big_smem_synth(int big) {
  return cudaFuncSetAttribute(k_legendre_synth<T, NP>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, big);
}
template <typename T, int NP>
static cudaError_t set_big_smem_anal(int big) {
  return cudaFuncSetAttribute(k_legendre_anal<T, NP>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, big);
}

wf_status init_legendre_attributes() {
  const int big = 220 * 1024;
  WF_CUDA((set_big_smem_synth<double, 1>(big)));
  WF_CUDA((set_big_smem_synth<double, 2>(big)));
  WF_CUDA((set_big_smem_synth<double, 4>(big)));
  WF_CUDA((set_big_smem_synth<float, 1>(big)));
  WF_CUDA((set_big_smem_synth<float, 2>(big)));
  WF_CUDA((set_big_smem_synth<float, 4>(big)));
  WF_CUDA((set_big_smem_anal<double, 2>(big)));
  WF_CUDA((set_big_smem_anal<double, 4>(big)));
  WF_CUDA((set_big_smem_anal<double, 8>(big)));
  WF_CUDA((set_big_smem_anal<double, 16>(big)));
  WF_CUDA((set_big_smem_anal<float, 2>(big)));
  WF_CUDA((set_big_smem_anal<float, 4>(big)));
  WF_CUDA((set_big_smem_anal<float, 8>(big)));
  WF_CUDA((set_big_smem_anal<float, 16>(big)));
  return WF_OK;
}

// xs = g_lm x_lm in the transform precision (the synthesis input)
template <typename T2>
__global__ void k_prescale(const double2 *__restrict__ x, const double *__restrict__ rg,
                           long n, T2 *__restrict__ xs) {
  typedef typename Scalar<T2>::type T;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long)gridDim.x * blockDim.x)
    xs[i] = Vec2<T>::make((T)(rg[i] * x[i].x), (T)(rg[i] * x[i].y));
}

template <typename T2>
wf_status launch_prescale(const Plan &P, const double2 *x, T2 *xs) {
  ++P.nlaunch;
  k_prescale<T2><<<304, 256, 0, P.stream>>>(x, P.rg, P.nalm, xs);
  WF_CUDA(cudaGetLastError());
  return WF_OK;
}

template wf_status launch_prescale<double2>(const Plan &, const double2 *, double2 *);
template wf_status launch_prescale<float2>(const Plan &, const double2 *, float2 *);
template wf_status launch_legendre_synth<double2>(const Plan &, const double2 *,
                                                  double2 *, const SolverState *,
                                                  int);
template wf_status launch_legendre_synth<float2>(const Plan &, const float2 *,
                                                 float2 *, const SolverState *, int);
template wf_status launch_legendre_anal<double2>(const Plan &, const double2 *,
                                                 double2 *, const SolverState *,
                                                 int, int, const double2 *, double2 *);
template wf_status launch_legendre_anal<float2>(const Plan &, const float2 *,
                                                double2 *, const SolverState *,
                                                int, int, const double2 *, float2 *);

}  // namespace wf
