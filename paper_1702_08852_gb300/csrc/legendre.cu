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
// Work split: synthesis -- one CTA row per m, one thread per NP ring pairs,
// a warp-uniform loop over l (pairs with a later seed stay at u = 0 until
// their seed is injected).  Analysis -- one CTA per m, warps own tiles of
// ring pairs, each warp accumulates 16 l values x (re, im) per lane and
// reduces them across the warp with a 31-shuffle transpose-reduction; per-warp
// partial sums (shared memory, or global scratch rows) are combined in a
// fixed order at the end (deterministic).  The analysis of the solver fuses
// the truncated-spectrum filter f_l = Sbar_l / (Sbar_l + xi Omega), Sbar_l =
// max(C_l - mu Omega, 0) (Eq. 15, App. B) and the partial sums of the Cauchy
// norms.  Launch variants (pairs per thread, packed f32x2 pairs of rings,
// queue scheduling, global accumulators) are picked per geometry by the
// autotuner; the FP32 variants run the sign-folded recurrence below, and the
// double-float kernels at the end of the file serve the mixed solver's
// anchor steps.
#include <limits.h>

#include <algorithm>
#include <atomic>

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

// One step of the recurrence.  FP64: u_l = c_l z u_{l-1} - u_{l-2}.  FP32
// runs the sign-folded s_l = eps_l u_l, eps_l = (-1)^floor(l/2), which obeys
// s_l = c'_l z s_{l-1} + s_{l-2} with the table c'_l = +-c_l (plan.cu): the
// same roundings, no negated operand.  The FP32 kernels therefore take seeds
// times eps, give ring sums in s-units (the epilogue multiplies by eps_l)
// and read a synthesis input pre-multiplied by eps_l.  In FP32, z = cos(theta)
// is carried as zh + zl (two floats): rounding z alone to FP32 displaces a
// ring near the pole by ~6e-8 / sin(theta) rad, a phase error of l times that.
__device__ __forceinline__ double rec_step(double c, double zh, double, double u1,
                                           double u2) {
  return fma(c * zh, u1, -u2);
}
__device__ __forceinline__ float rec_step(float c, float zh, float zl, float u1,
                                          float u2) {
  const float a = c * u1;
  return fmaf(a, zh, fmaf(a, zl, u2));
}
// eps_l of the FP32 sign folding (1 in FP64)
template <typename T>
__device__ __forceinline__ double fold_sign(int l) {
  return (sizeof(T) == 4 && ((l >> 1) & 1)) ? -1.0 : 1.0;
}

// Packed FP32 pairs (sm_100 family f32x2 arithmetic): one instruction does
// the operation for two rings, each half rounded as the scalar instruction.
__device__ __forceinline__ void fma2(float &dx, float &dy, float ax, float ay, float bx,
                                     float by, float cx, float cy) {
  asm("{\n .reg .b64 ra, rb, rc, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
      " mov.b64 rc, {%6, %7};\n fma.rn.f32x2 rd, ra, rb, rc;\n mov.b64 {%0, %1}, rd;\n}"
      : "=f"(dx), "=f"(dy)
      : "f"(ax), "f"(ay), "f"(bx), "f"(by), "f"(cx), "f"(cy));
}
__device__ __forceinline__ void mul2(float &dx, float &dy, float ax, float ay, float bx,
                                     float by) {
  asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
      " mul.rn.f32x2 rd, ra, rb;\n mov.b64 {%0, %1}, rd;\n}"
      : "=f"(dx), "=f"(dy)
      : "f"(ax), "f"(ay), "f"(bx), "f"(by));
}
// the FP32 recurrence step for rings j, j' at once (same roundings as
// rec_step); cx, cy both hold c_l (a register pair when loaded as one)
__device__ __forceinline__ void rec_step2(float cx, float cy, float zh0, float zh1,
                                          float zl0, float zl1, float u10, float u11,
                                          float u20, float u21, float &s0, float &s1) {
  float a0, a1, t0, t1;
  mul2(a0, a1, cx, cy, u10, u11);
  fma2(t0, t1, a0, a1, zl0, zl1, u20, u21);
  fma2(s0, s1, a0, a1, zh0, zh1, t0, t1);
}
__device__ __forceinline__ void rec_step2(float c, float zh0, float zh1, float zl0,
                                          float zl1, float u10, float u11, float u20,
                                          float u21, float &s0, float &s1) {
  float a0, a1, t0, t1;
  mul2(a0, a1, c, c, u10, u11);
  fma2(t0, t1, a0, a1, zl0, zl1, u20, u21);
  fma2(s0, s1, a0, a1, zh0, zh1, t0, t1);
}
template <typename T>
__device__ __forceinline__ void split_z(double z, T &zh, T &zl) {
  zh = (T)z;
  zl = (T)(z - (double)zh);
}
// z (as zh + zl) and the two seed values of ring pair k at (m, k) = mk: FP32
// from the plan's FP32 tables (s-units), FP64 from the pair and seed_u
template <typename T>
__device__ __forceinline__ void ring_seed(const RingPair *__restrict__ pairs,
                                          const double2 *__restrict__ seed_u,
                                          const Tab32 &t32, int k, long mk, T &zh, T &zl,
                                          T &s0, T &s1) {
  if constexpr (sizeof(T) == 4) {
    const float2 s = t32.seed_s[mk];
    zh = t32.zh[k];
    zl = t32.zl[k];
    s0 = s.x;
    s1 = s.y;
  } else {
    split_z<T>(pairs[k].z, zh, zl);
    const double2 su = seed_u[mk];
    s0 = su.x;
    s1 = su.y;
  }
}

static inline size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }
__device__ __forceinline__ size_t align16d(size_t b) { return (b + 15) & ~(size_t)15; }

// ------------------------------------------------------------------ synthesis
constexpr int SYN_THREADS = 128;

// DUP (with X2): the coefficient and input tables are kept duplicated in
// shared memory, (c, c) and (x_re, x_re, x_im, x_im), so that each packed
// operand pair arrives from one load instead of a load and a copy.
template <typename T, int NP, bool X2 = false, bool DUP = false>
__global__ void __launch_bounds__(SYN_THREADS)
    k_legendre_synth(const RingPair *__restrict__ pairs, int npairs, int lmax,
                     const double *__restrict__ rc, const float *__restrict__ rc32,
                     const double *__restrict__ rg, const int *__restrict__ seed_l,
                     const double2 *__restrict__ seed_u,
                     const typename Vec2<T>::type *__restrict__ xs,
                     typename Vec2<T>::type *__restrict__ F,
                     const SolverState *__restrict__ st, int lstatic, const Tab32 t32) {
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
  float4 *sx4 = reinterpret_cast<float4 *>(smraw);                 // DUP layout
  float2 *sc2 = reinterpret_cast<float2 *>(smraw + sizeof(float4) * nl);
  const long base = lm_index(lmax, m, m);
  for (int j = threadIdx.x; j < nl; j += blockDim.x) {
    const long i = base + j;
    if constexpr (DUP) {
      const float c = rc32[i];
      const float2 x = reinterpret_cast<const float2 *>(xs)[i];
      sc2[j] = make_float2(c, c);
      sx4[j] = make_float4(x.x, x.x, x.y, x.y);
    } else {
      sc[j] = coef<T>(rc, rc32, i);
      sx[j] = xs[i];
    }
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
      ls[j] = seed_l[(long)m * npairs + k];
      ring_seed<T>(pairs, seed_u, t32, k, (long)m * npairs + k, zh[j], zl[j], s0[j], s1[j]);
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
        T c;
        T2 xv;
        if constexpr (DUP) {
          c = sc2[li].x;
          xv = Vec2<T>::make(sx4[li].x, sx4[li].z);
        } else {
          c = sc[li];
          xv = sx[li];
        }
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
      if constexpr (DUP) {
        // (c_l, c_l, c_l+1, c_l+1) and (x_re, x_re, x_im, x_im) for l, l+1
        const float4 cq = *reinterpret_cast<const float4 *>(sc2 + (l - m));
        const float4 xa = sx4[l - m], xb = sx4[l + 1 - m];
#pragma unroll
        for (int jp = 0; jp < NP / 2; ++jp) {
          const int j0 = 2 * jp, j1 = 2 * jp + 1;
          float w0, w1, v0, v1;
          rec_step2(cq.x, cq.y, zh[j0], zh[j1], zl[j0], zl[j1], u1[j0], u1[j1], u2[j0],
                    u2[j1], w0, w1);
          fma2(er[j0], er[j1], w0, w1, xa.x, xa.y, er[j0], er[j1]);
          fma2(ei[j0], ei[j1], w0, w1, xa.z, xa.w, ei[j0], ei[j1]);
          rec_step2(cq.z, cq.w, zh[j0], zh[j1], zl[j0], zl[j1], w0, w1, u1[j0], u1[j1], v0,
                    v1);
          fma2(orr[j0], orr[j1], v0, v1, xb.x, xb.y, orr[j0], orr[j1]);
          fma2(oi[j0], oi[j1], v0, v1, xb.z, xb.w, oi[j0], oi[j1]);
          u2[j0] = w0;
          u2[j1] = w1;
          u1[j0] = v0;
          u1[j1] = v1;
        }
        continue;
      }
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
      if constexpr (X2) {
        // rings (2 jp, 2 jp + 1) in packed f32x2 pairs
        static_assert(sizeof(T) == 4 && NP % 2 == 0, "packed pairs are FP32, NP even");
#pragma unroll
        for (int jp = 0; jp < NP / 2; ++jp) {
          const int j0 = 2 * jp, j1 = 2 * jp + 1;
          float w0, w1, v0, v1;
          rec_step2(c0, zh[j0], zh[j1], zl[j0], zl[j1], u1[j0], u1[j1], u2[j0], u2[j1], w0,
                    w1);
          fma2(er[j0], er[j1], w0, w1, x0.x, x0.x, er[j0], er[j1]);
          fma2(ei[j0], ei[j1], w0, w1, x0.y, x0.y, ei[j0], ei[j1]);
          rec_step2(c1, zh[j0], zh[j1], zl[j0], zl[j1], w0, w1, u1[j0], u1[j1], v0, v1);
          fma2(orr[j0], orr[j1], v0, v1, x1.x, x1.x, orr[j0], orr[j1]);
          fma2(oi[j0], oi[j1], v0, v1, x1.y, x1.y, oi[j0], oi[j1]);
          u2[j0] = w0;
          u2[j1] = w1;
          u1[j0] = v0;
          u1[j1] = v1;
        }
      } else {
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
    }
    if (l <= L) {
      T c0;
      T2 x0;
      if constexpr (DUP) {
        c0 = sc2[l - m].x;
        x0 = Vec2<T>::make(sx4[l - m].x, sx4[l - m].z);
      } else {
        c0 = sc[l - m];
        x0 = sx[l - m];
      }
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


// v[0..NV) per lane (NV = 16 or 32) -> lane i returns the sum over lanes of
// v[i / R], R = 32 / NV (R lanes end with each value)
template <typename T, int NV>
__device__ __forceinline__ T transpose_reduce(T (&v)[NV], int lane) {
  constexpr int R = 32 / NV;
#pragma unroll
  for (int s = 16; s >= R; s >>= 1) {
    const int h = s / R;
    const bool upper = (lane & s) != 0;
#pragma unroll
    for (int j = 0; j < h; ++j) {
      const T send = upper ? v[j] : v[j + h];
      const T keep = upper ? v[j + h] : v[j];
      v[j] = keep + __shfl_xor_sync(0xffffffffu, send, s);
    }
  }
#pragma unroll
  for (int s = R / 2; s >= 1; s >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], s);
  return v[0];
}

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

// Cross-lane sum of NV FP32 values per lane through shared memory, the same
// totals as transpose_reduce<float, NV> (lane holds the total of value index
// lane / (32 / NV)): each lane stores its NV values as one row (16-byte
// stores; the row stride NV + 4 floats keeps them conflict-free), then sums
// one column over its share of the rows (the lanes sharing a column start at
// rotated rows, so they read different banks), then the shares by shuffles.
// 4 stores, NV loads and NV adds per lane per chunk, against the shuffle
// transpose's NV shuffles, NV adds and ~2 NV selects.  sb: this warp's
// 32 x (NV + 4) floats.
constexpr bool ANA_SMEM_REDUCE = true;
template <int NV>
__device__ __forceinline__ float smem_reduce(const float (&v)[NV], int lane, float *sb) {
  constexpr int STR = NV + 4;
  constexpr int R = 32 / NV;  // lanes per total
  constexpr int S = NV;       // rows each of them sums (32 / R)
  __syncwarp();               // the previous chunk's reads are done
  float4 *row = reinterpret_cast<float4 *>(sb + lane * STR);
#pragma unroll
  for (int q = 0; q < NV / 4; ++q)
    row[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
  __syncwarp();
  const int o = lane / R, sub = lane % R;
  float acc = 0.f;
#pragma unroll
  for (int k = 0; k < S; ++k) acc += sb[(sub * S + ((k + sub) % S)) * STR + o];
#pragma unroll
  for (int sh = R / 2; sh >= 1; sh >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, sh);
  return acc;
}

// One chunk of LCHUNK consecutive l for NP ring pairs per lane: v[2 jj] and
// v[2 jj + 1] receive this lane's contribution (re, im) to a_{lc+jj, m}.
// INJ: some lane of the warp still has its seed (ls, ls + 1) in or after this
// chunk.  TAIL: the chunk runs past L (l > L contributes 0).  In FP32 full
// chunks the coefficients c_l come from shared memory in 16-byte loads
// (lc - m is a multiple of LCHUNK and the table starts 16-byte aligned).
// SS: the seed values are read from shared memory (ssm: this lane's entry of
// ring 0, ring j at ssm[32 j]) where a seed may enter, instead of being held
// in registers for the whole tile.
template <typename T, int NP, bool INJ, bool TAIL, bool X2 = false, int LC = LCHUNK,
          bool SS = false>
__device__ __forceinline__ void anal_chunk(T (&v)[2 * LC], int lc, int L, int m,
                                           const T *__restrict__ sc, const T (&zh)[NP],
                                           const T (&zl)[NP], T (&u1)[NP], T (&u2)[NP],
                                           const T (&s0)[NP], const T (&s1)[NP],
                                           const int (&ls)[NP], const T (&pr)[NP],
                                           const T (&pim)[NP], const T (&qr)[NP],
                                           const T (&qim)[NP],
                                           const float2 *__restrict__ ssm = nullptr) {
  // FP32 full chunks: the 16 coefficients in four 16-byte loads
  constexpr bool VEC = sizeof(T) == 4 && !TAIL;
  T cc[VEC ? LC : 1];
  if constexpr (VEC) {
    const uint4 *s4 = reinterpret_cast<const uint4 *>(sc + (lc - m));
#pragma unroll
    for (int q = 0; q < LC / 4; ++q) {
      const uint4 w = s4[q];
      memcpy(&cc[4 * q], &w, 16);
    }
  }
#pragma unroll
  for (int jj = 0; jj < LC; ++jj) {
    const int l = lc + jj;
    // two partial sums (even, odd j) halve the dependent FMA chain
    T a_re = (T)0, a_im = (T)0, b_re = (T)0, b_im = (T)0;
    if (!TAIL || l <= L) {
      T c;
      if constexpr (VEC)
        c = cc[jj];
      else
        c = sc[l - m];
      if constexpr (X2) {
        // rings (2 jp, 2 jp + 1) in packed pairs; with more than two pairs
        // the partial sums a, b hold the even / odd pair of each group of
        // four rings (shorter dependent chains), with two pairs one packed
        // sum (fewer adds to merge)
        static_assert(sizeof(T) == 4 && NP % 2 == 0, "packed pairs are FP32, NP even");
        float ar0 = 0.f, ar1 = 0.f, ai0 = 0.f, ai1 = 0.f;
        float br0 = 0.f, br1 = 0.f, bi0 = 0.f, bi1 = 0.f;
#pragma unroll
        for (int jp = 0; jp < NP / 2; ++jp) {
          const int j0 = 2 * jp, j1 = 2 * jp + 1;
          float w0, w1;
          rec_step2(c, zh[j0], zh[j1], zl[j0], zl[j1], u1[j0], u1[j1], u2[j0], u2[j1], w0,
                    w1);
          if (INJ) {
            if constexpr (SS) {
              const float2 e0 = ssm[32 * j0], e1 = ssm[32 * j1];
              w0 = (l == ls[j0]) ? e0.x : w0;
              w0 = (l == ls[j0] + 1) ? e0.y : w0;
              w1 = (l == ls[j1]) ? e1.x : w1;
              w1 = (l == ls[j1] + 1) ? e1.y : w1;
            } else {
              w0 = (l == ls[j0]) ? s0[j0] : w0;
              w0 = (l == ls[j0] + 1) ? s1[j0] : w0;
              w1 = (l == ls[j1]) ? s0[j1] : w1;
              w1 = (l == ls[j1] + 1) ? s1[j1] : w1;
            }
          }
          u2[j0] = u1[j0];
          u2[j1] = u1[j1];
          u1[j0] = w0;
          u1[j1] = w1;
          const bool ev = (jj & 1) == 0;
          if (NP <= 4 || (jp & 1) == 0) {
            fma2(ar0, ar1, w0, w1, ev ? pr[j0] : qr[j0], ev ? pr[j1] : qr[j1], ar0, ar1);
            fma2(ai0, ai1, w0, w1, ev ? pim[j0] : qim[j0], ev ? pim[j1] : qim[j1], ai0, ai1);
          } else {
            fma2(br0, br1, w0, w1, ev ? pr[j0] : qr[j0], ev ? pr[j1] : qr[j1], br0, br1);
            fma2(bi0, bi1, w0, w1, ev ? pim[j0] : qim[j0], ev ? pim[j1] : qim[j1], bi0, bi1);
          }
        }
        if constexpr (NP <= 4) {
          a_re = ar0 + ar1;
          a_im = ai0 + ai1;
        } else {
          a_re = (ar0 + ar1) + (br0 + br1);
          a_im = (ai0 + ai1) + (bi0 + bi1);
        }
      } else {
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
        // FP32: two partial sums (shorter dependent chains); FP64 is bound
        // by its pipe's throughput, so one sum saves the merging adds
        if (sizeof(T) == 8 || (j & 1) == 0) {
          a_re = fma(u, pre, a_re);
          a_im = fma(u, pim_, a_im);
        } else {
          b_re = fma(u, pre, b_re);
          b_im = fma(u, pim_, b_im);
        }
      }
      }
    }
    if constexpr (sizeof(T) == 8) {
      v[2 * jj] = a_re;
      v[2 * jj + 1] = a_im;
    } else {
      v[2 * jj] = a_re + b_re;
      v[2 * jj + 1] = a_im + b_im;
    }
  }
}

// Epilogue of one coefficient (l, m), index i: a = Omega g_l (sr, si) (the
// ring sums in u-units; FP32: s-units, times eps_l here), then in ANA_FILTER mode the source term of an
// anchored stage, the filter f_l = Sbar / (Sbar + xi Omega) and the Cauchy
// partial sums (weight wm = 1 for m = 0, 2 else); writes x and xs_out.
template <typename T>
__device__ __forceinline__ void anal_finish(long i, int l, double sr, double si,
                                            double wm, int mode,
                                            const double *__restrict__ rg,
                                            const double *__restrict__ cl, double omega,
                                            double xi, double mu,
                                            const double2 *__restrict__ src,
                                            const double2 *__restrict__ xa,
                                            double2 *__restrict__ x,
                                            typename Vec2<T>::type *__restrict__ xs_out,
                                            double &num, double &den, double &dx) {
  const double s = omega * rg[i] * fold_sign<T>(l);  // ring sums are in s-units
  double ar = s * sr, ai = s * si;
  if (mode == ANA_FILTER) {
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
    if (xa) {  // anchored stage: ||x_a + delta||^2
      const double2 b = xa[i];
      const double tr = ar + b.x, ti = ai + b.y;
      dx += wm * (tr * tr + ti * ti);
    }
  }
  x[i] = make_double2(ar, ai);
  if (xs_out) {  // the synthesis input g a (times eps_l in FP32)
    const double gs = rg[i] * fold_sign<T>(l);
    xs_out[i] = Vec2<T>::make((T)(gs * ar), (T)(gs * ai));
  }
}

// The same epilogue for the FP32 kernels in FP32 arithmetic (this part's
// FP64 pipe is ~1/64 of its FP32 pipe, and a division per coefficient
// showed): ring sums in s-units times Omega g_l eps_l, the filter from the
// FP32 C_l, om = Omega, xio = xi Omega, muo = mu Omega.  Only the Cauchy
// differences against the FP64 iterate stay in FP64 (unweighted: the
// caller multiplies by wm once).
__device__ __forceinline__ void anal_finish32(long i, int l, float sr, float si, int mode,
                                              const Tab32 &t32, float om, float xio,
                                              float muo, const double2 *__restrict__ src,
                                              const double2 *__restrict__ xa,
                                              double2 *__restrict__ x,
                                              float2 *__restrict__ xs_out, double &num,
                                              double &den, double &dx) {
  const float g = t32.rg[i];
  float ar = om * (g * sr), ai = om * (g * si);
  if (mode == ANA_FILTER) {
    const float sbar = fmaxf(t32.cl[l] - muo, 0.f);
    const float f = sbar > 0.f ? sbar / (sbar + xio) : 0.f;
    if (src) {  // harmonic source term of a correction solve
      const double2 sv = src[i];
      ar = fmaf(xio, (float)sv.x, ar);
      ai = fmaf(xio, (float)sv.y, ai);
    }
    ar *= f;
    ai *= f;
    const double2 old = x[i];
    const double ard = ar, aid = ai;
    const double dr = ard - old.x, di = aid - old.y;
    num = fma(dr, dr, fma(di, di, num));
    den = fma(ard, ard, fma(aid, aid, den));
    if (xa) {  // anchored stage: ||x_a + delta||^2
      const double2 b = xa[i];
      const double tr = ard + b.x, ti = aid + b.y;
      dx = fma(tr, tr, fma(ti, ti, dx));
    }
  }
  x[i] = make_double2(ar, ai);
  if (xs_out) xs_out[i] = make_float2(g * ar, g * ai);  // the synthesis input
}

// coefficients of this m above the band (l > L) are zero
template <typename T>
__device__ __forceinline__ void anal_zero_above(int m, int L, int lmax, long base,
                                                double wm, int mode,
                                                double2 *__restrict__ x,
                                                typename Vec2<T>::type *__restrict__ xs_out,
                                                double &num) {
  const int lz = max(m, L + 1);
  for (int l = lz + (int)threadIdx.x; l <= lmax; l += ANA_THREADS) {
    const long i = base + (l - m);
    if (mode == ANA_FILTER) {
      const double2 old = x[i];
      num += wm * (old.x * old.x + old.y * old.y);
    }
    x[i] = make_double2(0.0, 0.0);
    if (xs_out) xs_out[i] = Vec2<T>::make((T)0, (T)0);
  }
}

// block sums of the Cauchy partials -> partials[2m], partials[2m + 1] and
// (anchored stages) partials[2 (lmax + 1) + m] (fixed order: lanes by
// xor-butterfly, then warps in index order)
__device__ __forceinline__ void anal_partials(double num, double den, double dx, int m,
                                              int lmax, double *__restrict__ partials) {
  __shared__ double wsum[3][ANA_WARPS];
  for (int o = 16; o > 0; o >>= 1) {
    num += __shfl_xor_sync(0xffffffffu, num, o);
    den += __shfl_xor_sync(0xffffffffu, den, o);
    dx += __shfl_xor_sync(0xffffffffu, dx, o);
  }
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    wsum[0][warp] = num;
    wsum[1][warp] = den;
    wsum[2][warp] = dx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0, c = 0.0;
    for (int w = 0; w < ANA_WARPS; ++w) {
      a += wsum[0][w];
      b += wsum[1][w];
      c += wsum[2][w];
    }
    partials[2 * m] = a;
    partials[2 * m + 1] = b;
    partials[2 * (lmax + 1) + m] = c;
  }
}

// GACC: the per-warp accumulators live in global memory (scratch rows
// [warp][alm], L2-resident) instead of shared memory, so shared memory no
// longer caps the CTAs per SM; each chunk's old value is loaded before the
// chunk's arithmetic and written back after its reduction.
// LC: l values per chunk (16, or 8 to free registers for more ring pairs).
// SS (with GACC): each lane's seed values go to shared memory after the
// tile load (the lane reads back only its own entries), freeing 2 NP
// registers; that kernel is compiled for 4 CTAs per SM.
template <typename T, int NP, bool X2, bool GACC, int LC, bool SS>
__device__ __forceinline__ void
    anal_body(const RingPair *__restrict__ pairs, int npairs, int lmax,
                    const double *__restrict__ rc, const float *__restrict__ rc32,
                    const double *__restrict__ rg, const int *__restrict__ seed_l,
                    const double2 *__restrict__ seed_u,
                    const double *__restrict__ cl, double omega,
                    const typename Vec2<T>::type *__restrict__ G,
                    double2 *__restrict__ x, double *__restrict__ partials,
                    const double2 *__restrict__ src,
                    typename Vec2<T>::type *__restrict__ xs_out,
                    const SolverState *__restrict__ st, int mode, int lstatic,
                    T *__restrict__ gacc, long nalm, const Tab32 &t32) {
  typedef typename Vec2<T>::type T2;
  const int m = blockIdx.x;
  int L = lstatic;
  double xi = 0.0, mu = 0.0;
  const double2 *xa = nullptr;  // anchored stage: the anchor iterate x_a
  if (st) {
    if (st->done) return;
    L = st->lcur;
    xi = st->xi;
    mu = filter_mu(*st, st->mu);  // the signal step's truncation
    xa = st->xa;
  }
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long base = lm_index(lmax, m, m);
  const double wm = (m == 0) ? 1.0 : 2.0;
  double num = 0.0, den = 0.0, dx = 0.0;

  if (m <= L) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int nl = L - m + 1;
    T2 *acc = reinterpret_cast<T2 *>(smraw);  // [ANA_WARPS][nl]
    T *sc = reinterpret_cast<T *>(smraw + (GACC ? 0 : align16d(sizeof(T2) * nl * ANA_WARPS)));
    static_assert(!SS || (GACC && sizeof(T) == 4), "shared seeds: FP32 with GACC");
    float2 *ssm = SS ? reinterpret_cast<float2 *>(smraw + align16d(sizeof(T) * (lmax + 1))) +
                           warp * 32 * NP + lane
                     : nullptr;
    for (int j = tid; j < nl; j += ANA_THREADS) sc[j] = coef<T>(rc, rc32, base + j);
    if constexpr (GACC) {
      for (int w = 0; w < ANA_WARPS; ++w)
        for (int j = tid; j < nl; j += ANA_THREADS)
          reinterpret_cast<T2 *>(gacc)[(long)w * nalm + base + j] = Vec2<T>::make((T)0, (T)0);
    } else {
      for (int j = tid; j < nl * ANA_WARPS; j += ANA_THREADS)
        acc[j] = Vec2<T>::make((T)0, (T)0);
    }
    __syncthreads();
    T2 *myacc = GACC ? reinterpret_cast<T2 *>(gacc) + (long)warp * nalm + base
                     : acc + (long)warp * nl;
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
          ls[j] = seed_l[(long)m * npairs + k];
          ring_seed<T>(pairs, seed_u, t32, k, (long)m * npairs + k, zh[j], zl[j], s0[j],
                       s1[j]);
          if constexpr (SS) ssm[32 * j] = make_float2((float)s0[j], (float)s1[j]);
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
          if constexpr (SS) ssm[32 * j] = make_float2(0.f, 0.f);
        }
        if (ls[j] <= L) {
          lmin = min(lmin, ls[j]);
          linj = max(linj, ls[j] + 1);
        }
      }
      lmin = warp_min(lmin);
      linj = warp_max(linj);
      if (lmin > L) continue;
      const int lc0 = m + ((lmin - m) / LC) * LC;
      constexpr int R = 16 / LC;  // lanes holding each reduced value
      for (int lc = lc0; lc <= L; lc += LC) {
        T v[2 * LC];
        // three specialisations of the chunk body: seeds still to come in
        // this warp (selects on every step), a full chunk with every seed of
        // the warp already in (the plain recurrence: 5 FP instructions per
        // term), and the last, partial chunk
        const int idx = lane / R;             // this lane's value after the reduction
        const int lmine = lc + (idx >> 1);
        const bool writer = (lane % R) == 0;
        T *mine = reinterpret_cast<T *>(myacc + (lmine - m)) + (idx & 1);
        T old = (T)0;
        if (GACC && writer && lmine <= L) old = *mine;  // in flight during the chunk
        if (lc + LC - 1 > L)
          anal_chunk<T, NP, true, true, X2, LC, SS>(v, lc, L, m, sc, zh, zl, u1, u2, s0, s1,
                                                    ls, pr, pim, qr, qim, ssm);
        else if (lc <= linj)
          anal_chunk<T, NP, true, false, X2, LC, SS>(v, lc, L, m, sc, zh, zl, u1, u2, s0,
                                                     s1, ls, pr, pim, qr, qim, ssm);
        else
          anal_chunk<T, NP, false, false, X2, LC, SS>(v, lc, L, m, sc, zh, zl, u1, u2, s0,
                                                      s1, ls, pr, pim, qr, qim, ssm);
        T tot;
        if constexpr (sizeof(T) == 4 && ANA_SMEM_REDUCE) {
          __shared__ __align__(16) float red_sm[ANA_WARPS][32 * (2 * LC + 4)];
          tot = smem_reduce<2 * LC>(v, lane, red_sm[warp]);
        } else {
          tot = transpose_reduce<T, 2 * LC>(v, lane);
        }
        if (writer && lmine <= L) {
          if constexpr (GACC)
            *mine = old + tot;
          else
            *mine += tot;
        }
      }
    }
    __syncthreads();
    const T2 *accr = GACC ? reinterpret_cast<const T2 *>(gacc) + base : acc;
    const long wstride = GACC ? nalm : nl;
    if constexpr (sizeof(T) == 4) {
      const float om = (float)omega, xio = (float)(xi * omega), muo = (float)(mu * omega);
      double nu = 0.0, de = 0.0, dxu = 0.0;
      for (int j = tid; j < nl; j += ANA_THREADS) {
        float sr = 0.f, si = 0.f;
#pragma unroll
        for (int w = 0; w < ANA_WARPS; ++w) {
          sr += accr[w * wstride + j].x;
          si += accr[w * wstride + j].y;
        }
        anal_finish32(base + j, m + j, sr, si, mode, t32, om, xio, muo, src, xa, x, xs_out,
                      nu, de, dxu);
      }
      num = wm * nu;
      den = wm * de;
      dx = wm * dxu;
    } else {
      for (int j = tid; j < nl; j += ANA_THREADS) {
        double sr = 0.0, si = 0.0;
#pragma unroll
        for (int w = 0; w < ANA_WARPS; ++w) {
          sr += (double)accr[w * wstride + j].x;
          si += (double)accr[w * wstride + j].y;
        }
        anal_finish<T>(base + j, m + j, sr, si, wm, mode, rg, cl, omega, xi, mu, src, xa, x,
                       xs_out, num, den, dx);
      }
    }
  }
  anal_zero_above<T>(m, L, lmax, base, wm, mode, x, xs_out, num);
  if (mode == ANA_FILTER) anal_partials(num, den, dx, m, lmax, partials);
}

#define WF_ANAL_PARAMS(T)                                                                 \
  const RingPair *__restrict__ pairs, int npairs, int lmax, const double *__restrict__ rc, \
      const float *__restrict__ rc32, const double *__restrict__ rg,                       \
      const int *__restrict__ seed_l, const double2 *__restrict__ seed_u,                  \
      const double *__restrict__ cl, double omega,                                         \
      const typename Vec2<T>::type *__restrict__ G, double2 *__restrict__ x,              \
      double *__restrict__ partials, const double2 *__restrict__ src,                      \
      typename Vec2<T>::type *__restrict__ xs_out, const SolverState *__restrict__ st,     \
      int mode, int lstatic, T *__restrict__ gacc, long nalm, const Tab32 t32
#define WF_ANAL_ARGS                                                                       \
  pairs, npairs, lmax, rc, rc32, rg, seed_l, seed_u, cl, omega, G, x, partials, src, xs_out, \
      st, mode, lstatic, gacc, nalm, t32

template <typename T, int NP, bool X2 = false, bool GACC = false, int LC = LCHUNK>
__global__ void __launch_bounds__(ANA_THREADS) k_legendre_anal(WF_ANAL_PARAMS(T)) {
  anal_body<T, NP, X2, GACC, LC, false>(WF_ANAL_ARGS);
}
template <int NP>
__global__ void __launch_bounds__(ANA_THREADS, 4) k_legendre_anal_ss(WF_ANAL_PARAMS(float)) {
  anal_body<float, NP, true, true, 8, true>(WF_ANAL_ARGS);
}
#undef WF_ANAL_PARAMS
#undef WF_ANAL_ARGS

// ------------------------------------------------- analysis, queue-scheduled
// The same contraction with the work split into items (m, tile of 32 NP ring
// pairs), ordered heaviest first (m ascending).  Each warp takes items from
// a device counter until none is left, so no warp waits for another (the
// per-m CTA above waits at its barriers for its slowest warp, and a CTA per m
// leaves the triangle's small-m rows to the end).  An item writes its
// per-chunk warp sums for l in [lstart, L] to scratch[tile][i] (FP32
// complex) and lstart to ana_lstart; k_anal_combine then adds the tiles of
// each (l, m) in tile order (deterministic) and runs the epilogue.
constexpr int ANA_Q_CTAS_PER_SM = 8;  // upper bound; the occupancy decides

template <typename T, int NP>
__global__ void __launch_bounds__(ANA_THREADS)
    k_legendre_anal_q(const RingPair *__restrict__ pairs, int npairs, int lmax, long nalm,
                      const double *__restrict__ rc, const float *__restrict__ rc32,
                      const int *__restrict__ seed_l, const double2 *__restrict__ seed_u,
                      const typename Vec2<T>::type *__restrict__ G, T *__restrict__ scratch,
                      int *__restrict__ lstart, int *__restrict__ counter,
                      const SolverState *__restrict__ st, int lstatic, const Tab32 t32) {
  int L = lstatic;
  if (st) {
    if (st->done) return;
    L = st->lcur;
  }
  if (L < 0) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int sc_stride = (lmax + 4) & ~3;  // 16-byte aligned rows
  T *sc = reinterpret_cast<T *>(smraw) + (long)warp * sc_stride;
  constexpr int TP = 32 * NP;
  const int ntiles = (npairs + TP - 1) / TP;
  const int nitems = (L + 1) * ntiles;
  const long stride = lmax + 1;
  for (;;) {
    int item = 0;
    if (lane == 0) item = atomicAdd(counter, 1);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= nitems) break;
    const int m = item / ntiles, tile = item - m * ntiles;
    const long base = lm_index(lmax, m, m);
    const int pair0 = tile * TP;
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
        ls[j] = seed_l[(long)m * npairs + k];
        ring_seed<T>(pairs, seed_u, t32, k, (long)m * npairs + k, zh[j], zl[j], s0[j], s1[j]);
        const typename Vec2<T>::type gn = G[rp.ringN * stride + m];
        typename Vec2<T>::type gs = Vec2<T>::make((T)0, (T)0);
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
    const int lc0 = lmin <= L ? m + ((lmin - m) / LCHUNK) * LCHUNK : L + 1;
    if (lane == 0) lstart[(long)m * ntiles + tile] = lc0;
    if (lmin > L) continue;
    __syncwarp();  // the previous item's reads of sc are done
    for (int j = lane; j <= L - m; j += 32) sc[j] = coef<T>(rc, rc32, base + j);
    __syncwarp();
    T *out = scratch + 2 * ((long)tile * nalm + base - m);  // out[2 l + re/im]
    for (int lc = lc0; lc <= L; lc += LCHUNK) {
      T v[32];
      if (lc + LCHUNK - 1 > L)
        anal_chunk<T, NP, true, true>(v, lc, L, m, sc, zh, zl, u1, u2, s0, s1, ls, pr,
                                      pim, qr, qim);
      else if (lc <= linj)
        anal_chunk<T, NP, true, false>(v, lc, L, m, sc, zh, zl, u1, u2, s0, s1, ls, pr,
                                       pim, qr, qim);
      else
        anal_chunk<T, NP, false, false>(v, lc, L, m, sc, zh, zl, u1, u2, s0, s1, ls, pr,
                                        pim, qr, qim);
      const T tot = transpose_reduce32<T>(v, lane);
      const int l = lc + (lane >> 1);
      if (l <= L) out[2 * l + (lane & 1)] = tot;
    }
  }
}

// Sum the tiles of every (l, m) of one m in tile order and finish as the
// per-m kernel does.  Block 0 resets the queue counter for the next launch
// (the analysis kernel has finished: same stream).
template <typename T>
__global__ void __launch_bounds__(ANA_THREADS)
    k_anal_combine(int lmax, long nalm, int ntiles, const T *__restrict__ scratch,
                   const int *__restrict__ lstart, int *__restrict__ counter,
                   const double *__restrict__ rg, const double *__restrict__ cl,
                   double omega, double2 *__restrict__ x, double *__restrict__ partials,
                   const double2 *__restrict__ src,
                   typename Vec2<T>::type *__restrict__ xs_out,
                   const SolverState *__restrict__ st, int mode, int lstatic,
                   const Tab32 t32) {
  const int m = blockIdx.x;
  int L = lstatic;
  double xi = 0.0, mu = 0.0;
  const double2 *xa = nullptr;  // anchored stage: the anchor iterate x_a
  if (st) {
    if (st->done) return;
    L = st->lcur;
    xi = st->xi;
    mu = filter_mu(*st, st->mu);  // the signal step's truncation
    xa = st->xa;
  }
  if (m == 0 && threadIdx.x == 0) *counter = 0;
  const long base = lm_index(lmax, m, m);
  const double wm = (m == 0) ? 1.0 : 2.0;
  double num = 0.0, den = 0.0, dx = 0.0;
  if (m <= L) {
    if constexpr (sizeof(T) == 4) {  // FP32 tiles: the FP32 epilogue
      const float om = (float)omega, xio = (float)(xi * omega), muo = (float)(mu * omega);
      double nu = 0.0, de = 0.0, dxu = 0.0;
      for (int j = threadIdx.x; j <= L - m; j += ANA_THREADS) {
        const int l = m + j;
        float sr = 0.f, si = 0.f;
        for (int t = 0; t < ntiles; ++t) {
          if (l < __ldg(lstart + (long)m * ntiles + t)) continue;
          const T *p = scratch + 2 * ((long)t * nalm + base + j);
          sr += p[0];
          si += p[1];
        }
        anal_finish32(base + j, l, sr, si, mode, t32, om, xio, muo, src, xa, x, xs_out, nu, de,
                      dxu);
      }
      num = wm * nu;
      den = wm * de;
      dx = wm * dxu;
    } else {
      for (int j = threadIdx.x; j <= L - m; j += ANA_THREADS) {
        const int l = m + j;
        double sr = 0.0, si = 0.0;
        for (int t = 0; t < ntiles; ++t) {
          if (l < __ldg(lstart + (long)m * ntiles + t)) continue;
          const T *p = scratch + 2 * ((long)t * nalm + base + j);
          sr += (double)p[0];
          si += (double)p[1];
        }
        anal_finish<T>(base + j, l, sr, si, wm, mode, rg, cl, omega, xi, mu, src, xa, x, xs_out,
                       num, den, dx);
      }
    }
  }
  anal_zero_above<T>(m, L, lmax, base, wm, mode, x, xs_out, num);
  if (mode == ANA_FILTER) anal_partials(num, den, dx, m, lmax, partials);
}

// ------------------------------------------- double-float (df64) kernels
// The anchors of the mixed solver need the FP64 iteration map to ~1e-10, not
// to FP64's last bit, and this part's FP64 pipe is ~1/64 of its FP32 pipe.
// These kernels carry every value as an unevaluated sum hi + lo of two
// floats (~48-bit significand: products by FMA two-product, sums by
// two-sum, Dekker/Knuth), so the same transforms run on the FP32 pipe.
// Inputs and outputs are FP64 (double2), the recurrence is the FP64 one
// (u-convention, table rc), the analysis writes per-tile FP64 partial sums
// that k_anal_combine<double> adds in tile order.  Every operation is an
// explicit _rn intrinsic or fmaf, so nothing is contracted or reassociated.
struct dd {
  float hi, lo;
};
__device__ __forceinline__ dd dd_of(double x) {
  const float h = (float)x;
  return {h, (float)(x - (double)h)};
}
__device__ __forceinline__ double dd_val(dd a) { return (double)a.hi + (double)a.lo; }
// (s, e) with |s| >= |e| -> normalised pair
__device__ __forceinline__ dd dd_quick(float s, float e) {
  const float h = __fadd_rn(s, e);
  return {h, __fsub_rn(e, __fsub_rn(h, s))};
}
__device__ __forceinline__ dd dd_add(dd a, dd b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  return dd_quick(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ dd dd_sub(dd a, dd b) { return dd_add(a, {-b.hi, -b.lo}); }
__device__ __forceinline__ dd dd_mul(dd a, dd b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  return dd_quick(p, e);
}
// acc += u x with acc kept unnormalised (hi carries the running sum, lo the
// accumulated rounding errors); read it with dd_val
__device__ __forceinline__ void dd_acc(dd &acc, dd u, dd x) {
  const float p = __fmul_rn(u.hi, x.hi);
  float e = fmaf(u.hi, x.hi, -p);
  e = fmaf(u.hi, x.lo, fmaf(u.lo, x.hi, e));
  const float s = __fadd_rn(acc.hi, p);
  const float bb = __fsub_rn(s, acc.hi);
  const float err = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  acc.hi = s;
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(err, e));
}
// u_l = c_l z u_{l-1} - u_{l-2}: t = c u_{l-1} in double-float, then the
// product t z (two-product, unnormalised) and the difference with u_{l-2}
// (two-sum) with one final normalisation
__device__ __forceinline__ dd dd_rec(dd c, dd z, dd u1, dd u2) {
  const dd t = dd_mul(c, u1);
  const float p = __fmul_rn(t.hi, z.hi);
  float e = fmaf(t.hi, z.hi, -p);
  e = fmaf(t.hi, z.lo, fmaf(t.lo, z.hi, e));
  const float s = __fsub_rn(p, u2.hi);
  const float bb = __fsub_rn(s, p);
  const float err = __fadd_rn(__fsub_rn(p, __fsub_rn(s, bb)), __fsub_rn(-u2.hi, bb));
  return dd_quick(s, __fadd_rn(__fsub_rn(e, u2.lo), err));
}

constexpr int DD_NP_SYN = 2, DD_NP_ANA = 4;

// (kh + kl) + (rh + rl) for unnormalised double-float sums: a two-sum of
// the hi parts whose rounding error joins the lo parts
__device__ __forceinline__ void dd_add_unnorm(float &kh, float &kl, float rh, float rl) {
  const float t = __fadd_rn(kh, rh);
  const float bb = __fsub_rn(t, kh);
  const float e = __fadd_rn(__fsub_rn(kh, __fsub_rn(t, bb)), __fsub_rn(rh, bb));
  kh = t;
  kl = __fadd_rn(__fadd_rn(kl, rl), e);
}

// Cross-lane sum of NV double-float values per lane (vh + vl): the
// transpose-reduce of transpose_reduce<T, NV> in double-float; lane i holds
// the total of value index i / (32 / NV).  FP32 pipe only: this part's FP64
// pipe runs at ~1/64 of the FP32 rate.
template <int NV>
__device__ __forceinline__ dd transpose_reduce_dd(float (&vh)[NV], float (&vl)[NV], int lane) {
  constexpr int R = 32 / NV;
#pragma unroll
  for (int s = 16; s >= R; s >>= 1) {
    const int h = s / R;
    const bool upper = (lane & s) != 0;
#pragma unroll
    for (int j = 0; j < h; ++j) {
      const float sh = upper ? vh[j] : vh[j + h];
      const float sl = upper ? vl[j] : vl[j + h];
      float kh = upper ? vh[j + h] : vh[j];
      float kl = upper ? vl[j + h] : vl[j];
      dd_add_unnorm(kh, kl, __shfl_xor_sync(0xffffffffu, sh, s),
                    __shfl_xor_sync(0xffffffffu, sl, s));
      vh[j] = kh;
      vl[j] = kl;
    }
  }
#pragma unroll
  for (int s = R / 2; s >= 1; s >>= 1)
    dd_add_unnorm(vh[0], vl[0], __shfl_xor_sync(0xffffffffu, vh[0], s),
                  __shfl_xor_sync(0xffffffffu, vl[0], s));
  return {vh[0], vl[0]};
}

// l values per chunk of the double-float analysis: its chunk body (LC l x
// DD_NP_ANA ring pairs of double-float arithmetic, fully unrolled) must fit
// the instruction cache (16 l: ~3500 instructions, stalled on instruction
// fetch)
constexpr int DD_LC_ANA = 8;


// synthesis: as k_legendre_synth (one CTA row per m, one thread per
// DD_NP_SYN ring pairs), E/O parity sums in df64
__global__ void __launch_bounds__(SYN_THREADS)
    k_legendre_synth_dd(const RingPair *__restrict__ pairs, int npairs, int lmax,
                        const float2 *__restrict__ rcdd, const int *__restrict__ seed_l,
                        const double2 *__restrict__ seed_u, const float4 *__restrict__ xs,
                        float4 *__restrict__ F, const SolverState *__restrict__ st,
                        int lstatic) {
  constexpr int NP = DD_NP_SYN;
  const int m = blockIdx.y;
  int L = lstatic;
  if (st) {
    if (st->done) return;
    L = st->lcur;
  }
  if (m > L) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int nl = L - m + 1;
  dd *sxr = reinterpret_cast<dd *>(smraw);
  dd *sxi = sxr + nl;
  dd *sc = sxi + nl;
  const long base = lm_index(lmax, m, m);
  for (int j = threadIdx.x; j < nl; j += blockDim.x) {
    const float4 xv = xs[base + j];
    const float2 cv = rcdd[base + j];
    sxr[j] = {xv.x, xv.y};
    sxi[j] = {xv.z, xv.w};
    sc[j] = {cv.x, cv.y};
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int pair0 = (blockIdx.x * (SYN_THREADS / 32) + warp) * 32 * NP;
  if (pair0 >= npairs) return;
  const dd zero = {0.f, 0.f};
  dd z[NP], u1[NP], u2[NP], s0[NP], s1[NP], er[NP], ei[NP], orr[NP], oi[NP];
  int ls[NP];
  int lmin = INT_MAX, linj = -1;
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    const int k = pair0 + lane + 32 * j;
    u1[j] = u2[j] = er[j] = ei[j] = orr[j] = oi[j] = zero;
    z[j] = s0[j] = s1[j] = zero;
    ls[j] = INT_MAX - 2;
    if (k < npairs) {
      z[j] = dd_of(pairs[k].z);
      ls[j] = seed_l[(long)m * npairs + k];
      const double2 su = seed_u[(long)m * npairs + k];
      s0[j] = dd_of(su.x);
      s1[j] = dd_of(su.y);
    }
    if (ls[j] <= L) {
      lmin = min(lmin, ls[j]);
      linj = max(linj, ls[j] + 1);
    }
  }
  lmin = warp_min(lmin);
  linj = warp_max(linj);
  // one l at a time: seeds may enter (inj), parity of l - m picks the sums
  auto step = [&](int l, bool inj) {
    const dd c = sc[l - m], xr = sxr[l - m], xi = sxi[l - m];
    const bool even = ((l - m) & 1) == 0;
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      dd u = dd_rec(c, z[j], u1[j], u2[j]);
      if (inj) {
        u = (l == ls[j]) ? s0[j] : u;
        u = (l == ls[j] + 1) ? s1[j] : u;
      }
      u2[j] = u1[j];
      u1[j] = u;
      if (even) {
        dd_acc(er[j], u, xr);
        dd_acc(ei[j], u, xi);
      } else {
        dd_acc(orr[j], u, xr);
        dd_acc(oi[j], u, xi);
      }
    }
  };
  int l = lmin;
  for (; l <= L && l <= linj; ++l) step(l, true);
  if (l <= L && ((l - m) & 1)) step(l++, false);
  // plain recurrence two l at a time (l - m even, then odd): the same
  // operations in the same order, without the parity branch and with the
  // u_{l-1}, u_{l-2} rotation left to register renaming
  for (; l + 1 <= L; l += 2) {
    const dd c0 = sc[l - m], xr0 = sxr[l - m], xi0 = sxi[l - m];
    const dd c1 = sc[l + 1 - m], xr1 = sxr[l + 1 - m], xi1 = sxi[l + 1 - m];
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      const dd w = dd_rec(c0, z[j], u1[j], u2[j]);
      dd_acc(er[j], w, xr0);
      dd_acc(ei[j], w, xi0);
      const dd v = dd_rec(c1, z[j], w, u1[j]);
      dd_acc(orr[j], v, xr1);
      dd_acc(oi[j], v, xi1);
      u2[j] = w;
      u1[j] = v;
    }
  }
  if (l <= L) step(l, false);
  const long stride = lmax + 1;
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    const int k = pair0 + lane + 32 * j;
    if (k >= npairs) continue;
    const RingPair &rp = pairs[k];
    // north = E + O, south = E - O, as double-float pairs (re hi, re lo,
    // im hi, im lo): the double-float ring transform reads them unconverted
    const dd nr = dd_add(er[j], orr[j]), ni = dd_add(ei[j], oi[j]);
    F[rp.ringN * stride + m] = make_float4(nr.hi, nr.lo, ni.hi, ni.lo);
    if (rp.ringS >= 0) {
      const dd sr = dd_sub(er[j], orr[j]), si = dd_sub(ei[j], oi[j]);
      F[rp.ringS * stride + m] = make_float4(sr.hi, sr.lo, si.hi, si.lo);
    }
  }
}

// analysis: queue-scheduled like k_legendre_anal_q; per (m, tile of 32
// DD_NP_ANA ring pairs) item, per chunk of DD_LC_ANA l the lane's df64 sums
// are reduced across the warp in double-float (transpose_reduce_dd) and
// rounded to FP64 once per output
__global__ void __launch_bounds__(ANA_THREADS)
    k_legendre_anal_dd(const RingPair *__restrict__ pairs, int npairs, int lmax, long nalm,
                       const float2 *__restrict__ rcdd, const int *__restrict__ seed_l,
                       const double2 *__restrict__ seed_u, const float4 *__restrict__ G,
                       double *__restrict__ scratch, int *__restrict__ lstart,
                       int *__restrict__ counter, const SolverState *__restrict__ st,
                       int lstatic) {
  constexpr int NP = DD_NP_ANA;
  int L = lstatic;
  if (st) {
    if (st->done) return;
    L = st->lcur;
  }
  if (L < 0) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  extern __shared__ __align__(16) unsigned char smraw[];
  dd *sc = reinterpret_cast<dd *>(smraw) + (long)warp * (lmax + 1);
  constexpr int TP = 32 * NP;
  const int ntiles = (npairs + TP - 1) / TP;
  const int nitems = (L + 1) * ntiles;
  const long stride = lmax + 1;
  const dd zero = {0.f, 0.f};
  for (;;) {
    int item = 0;
    if (lane == 0) item = atomicAdd(counter, 1);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= nitems) break;
    const int m = item / ntiles, tile = item - m * ntiles;
    const long base = lm_index(lmax, m, m);
    const int pair0 = tile * TP;
    dd z[NP], u1[NP], u2[NP], s0[NP], s1[NP], pr[NP], pim[NP], qr[NP], qim[NP];
    int ls[NP];
    int lmin = INT_MAX, linj = -1;
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      const int k = pair0 + lane + 32 * j;
      u1[j] = u2[j] = z[j] = s0[j] = s1[j] = pr[j] = pim[j] = qr[j] = qim[j] = zero;
      ls[j] = INT_MAX - 2;
      if (k < npairs) {
        const RingPair &rp = pairs[k];
        z[j] = dd_of(rp.z);
        ls[j] = seed_l[(long)m * npairs + k];
        const double2 su = seed_u[(long)m * npairs + k];
        s0[j] = dd_of(su.x);
        s1[j] = dd_of(su.y);
        // ring coefficients as double-float pairs (re hi, re lo, im hi, im lo)
        const float4 gn = G[rp.ringN * stride + m];
        float4 gs = make_float4(0.f, 0.f, 0.f, 0.f);
        if (rp.ringS >= 0) gs = G[rp.ringS * stride + m];
        const dd nre = {gn.x, gn.y}, nim = {gn.z, gn.w};
        const dd sre = {gs.x, gs.y}, sim = {gs.z, gs.w};
        pr[j] = dd_add(nre, sre);
        pim[j] = dd_add(nim, sim);
        qr[j] = dd_sub(nre, sre);
        qim[j] = dd_sub(nim, sim);
      }
      if (ls[j] <= L) {
        lmin = min(lmin, ls[j]);
        linj = max(linj, ls[j] + 1);
      }
    }
    lmin = warp_min(lmin);
    linj = warp_max(linj);
    constexpr int LC = DD_LC_ANA;
    const int lc0 = lmin <= L ? m + ((lmin - m) / LC) * LC : L + 1;
    if (lane == 0) lstart[(long)m * ntiles + tile] = lc0;
    if (lmin > L) continue;
    __syncwarp();
    for (int j = lane; j <= L - m; j += 32) {
      const float2 cv = rcdd[base + j];
      sc[j] = {cv.x, cv.y};
    }
    __syncwarp();
    double *out = scratch + 2 * ((long)tile * nalm + base - m);  // out[2 l + re/im]
    for (int lc = lc0; lc <= L; lc += LC) {
      float vh[2 * LC], vl[2 * LC];
      const bool inj = lc <= linj;
#pragma unroll
      for (int jj = 0; jj < LC; ++jj) {
        const int l = lc + jj;
        dd ar = zero, ai = zero;
        if (l <= L) {
          const dd c = sc[l - m];
          const bool even = (jj & 1) == 0;  // lc - m is a multiple of LC (even)
#pragma unroll
          for (int j = 0; j < NP; ++j) {
            dd u = dd_rec(c, z[j], u1[j], u2[j]);
            if (inj) {
              u = (l == ls[j]) ? s0[j] : u;
              u = (l == ls[j] + 1) ? s1[j] : u;
            }
            u2[j] = u1[j];
            u1[j] = u;
            dd_acc(ar, u, even ? pr[j] : qr[j]);
            dd_acc(ai, u, even ? pim[j] : qim[j]);
          }
        }
        vh[2 * jj] = ar.hi;
        vl[2 * jj] = ar.lo;
        vh[2 * jj + 1] = ai.hi;
        vl[2 * jj + 1] = ai.lo;
      }
      const dd tot = transpose_reduce_dd<2 * LC>(vh, vl, lane);
      constexpr int R = 16 / LC;  // lanes holding each total
      const int idx = lane / R;
      const int l = lc + (idx >> 1);
      if (lane % R == 0 && l <= L) out[2 * l + (idx & 1)] = dd_val(tot);
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

static Tab32 tab32(const Plan &P) {
  return {P.seed_s32, P.zs32, P.zs32 + P.npairs, P.rg32, P.cl32};
}

template <typename T, int NP, bool X2 = false, bool DUP = false>
static void synth_variant(const Plan &P, const typename Vec2<T>::type *xs,
                          typename Vec2<T>::type *F, const SolverState *st, int lstatic) {
  typedef typename Vec2<T>::type T2;
  const size_t smem = DUP ? (sizeof(float4) + sizeof(float2)) * (P.lmax + 1)
                          : align16(sizeof(T2) * (P.lmax + 1)) + sizeof(T) * (P.lmax + 1);
  const int pairs_per_cta = SYN_THREADS * NP;
  dim3 grid((P.npairs + pairs_per_cta - 1) / pairs_per_cta, P.lmax + 1);
  k_legendre_synth<T, NP, X2, DUP><<<grid, SYN_THREADS, smem, P.stream>>>(
      P.pairs, P.npairs, P.lmax, P.rc, P.rc32, P.rg, P.seed_l, P.seed_u, xs, F, st,
      lstatic, tab32(P));
}

template <typename T, int NP, bool X2 = false, bool GACC = false, int LC = LCHUNK>
static void anal_variant(const Plan &P, const typename Vec2<T>::type *G, double2 *x,
                         const SolverState *st, int mode, int lstatic, const double2 *src,
                         typename Vec2<T>::type *xs_out) {
  typedef typename Vec2<T>::type T2;
  const size_t smem = (GACC ? 0 : align16(sizeof(T2) * (P.lmax + 1) * ANA_WARPS)) +
                      sizeof(T) * (P.lmax + 1);
  k_legendre_anal<T, NP, X2, GACC, LC><<<P.lmax + 1, ANA_THREADS, smem, P.stream>>>(
      P.pairs, P.npairs, P.lmax, P.rc, P.rc32, P.rg, P.seed_l, P.seed_u, P.cl_d, P.omega,
      G, x, P.partials, src, xs_out, st, mode, lstatic,
      GACC ? reinterpret_cast<T *>(P.ana_scratch) : nullptr, P.nalm, tab32(P));
}
// packed FP32 analysis, 8-l chunks, global accumulators, seeds in shared memory
template <int NP>
static void anal_ss_variant(const Plan &P, const float2 *G, double2 *x,
                            const SolverState *st, int mode, int lstatic, const double2 *src,
                            float2 *xs_out) {
  const size_t smem = align16(sizeof(float) * (P.lmax + 1)) + sizeof(float2) * ANA_THREADS * NP;
  k_legendre_anal_ss<NP><<<P.lmax + 1, ANA_THREADS, smem, P.stream>>>(
      P.pairs, P.npairs, P.lmax, P.rc, P.rc32, P.rg, P.seed_l, P.seed_u, P.cl_d, P.omega,
      G, x, P.partials, src, xs_out, st, mode, lstatic,
      reinterpret_cast<float *>(P.ana_scratch), P.nalm, tab32(P));
}

// queue-scheduled FP32 analysis: persistent grid of ANA_Q_CTAS_PER_SM CTAs
// per SM, then the per-m combine
template <int NP>
static wf_status anal_queue_variant(const Plan &P, const float2 *G, double2 *x,
                                    const SolverState *st, int mode, int lstatic,
                                    const double2 *src, float2 *xs_out) {
  const int sc_stride = (P.lmax + 4) & ~3;
  const size_t smem = sizeof(float) * sc_stride * ANA_WARPS;
  const int ntiles = (P.npairs + 32 * NP - 1) / (32 * NP);
  // one resident wave: CTAs per SM from the occupancy calculator (queried
  // once; the first call comes from the autotuner, outside graph capture)
  static std::atomic<int> per_sm_cache[2] = {0, 0};
  int per_sm = per_sm_cache[NP == 8].load();
  if (per_sm == 0) {
    int n = 0;
    WF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_legendre_anal_q<float, NP>,
                                                          ANA_THREADS, smem));
    per_sm = std::max(1, std::min(n, ANA_Q_CTAS_PER_SM));
    per_sm_cache[NP == 8].store(per_sm);
  }
  k_legendre_anal_q<float, NP><<<P.num_sms * per_sm, ANA_THREADS, smem, P.stream>>>(
      P.pairs, P.npairs, P.lmax, P.nalm, P.rc, P.rc32, P.seed_l, P.seed_u, G,
      P.ana_scratch, P.ana_lstart, P.ana_counter, st, lstatic, tab32(P));
  WF_CUDA(cudaGetLastError());
  ++P.nlaunch;
  k_anal_combine<float><<<P.lmax + 1, ANA_THREADS, 0, P.stream>>>(
      P.lmax, P.nalm, ntiles, P.ana_scratch, P.ana_lstart, P.ana_counter, P.rg, P.cl_d,
      P.omega, x, P.partials, src, xs_out, st, mode, lstatic, tab32(P));
  WF_CUDA(cudaGetLastError());
  return WF_OK;
}

// ring pairs per thread: the autotuner's choice for this plan and precision
template <typename T2>
wf_status launch_legendre_synth(const Plan &P, const T2 *xs, T2 *F,
                                const SolverState *st, int lstatic) {
  typedef typename Kernels<T2>::T T;
  const int np = P.syn_np[sizeof(T) == 4];
  ++P.nlaunch;
  if constexpr (sizeof(T) == 4) {
    if (P.syn_x2) {
      if (P.syn_x2 == 2)
        synth_variant<T, 2, true, true>(P, xs, F, st, lstatic);
      else if (np == 4)
        synth_variant<T, 4, true>(P, xs, F, st, lstatic);
      else
        synth_variant<T, 2, true>(P, xs, F, st, lstatic);
      WF_CUDA(cudaGetLastError());
      return WF_OK;
    }
  }
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
  if constexpr (sizeof(T) == 4) {
    if (P.ana_queue) {
      const float2 *g = reinterpret_cast<const float2 *>(G);
      float2 *xo = reinterpret_cast<float2 *>(xs_out);
      return np == 4 ? anal_queue_variant<4>(P, g, x, st, mode, lstatic, src, xo)
                     : anal_queue_variant<8>(P, g, x, st, mode, lstatic, src, xo);
    }
    if (P.ana_x2 && P.ana_gacc == 3) {  // 8-l chunks, seeds in shared memory
      anal_ss_variant<8>(P, reinterpret_cast<const float2 *>(G), x, st, mode, lstatic, src,
                         reinterpret_cast<float2 *>(xs_out));
      WF_CUDA(cudaGetLastError());
      return WF_OK;
    }
    if (P.ana_x2 && P.ana_gacc == 2) {  // 8-l chunks
      if (np == 8)
        anal_variant<T, 8, true, true, 8>(P, G, x, st, mode, lstatic, src, xs_out);
      else if (np == 6)
        anal_variant<T, 6, true, true, 8>(P, G, x, st, mode, lstatic, src, xs_out);
      else
        anal_variant<T, 4, true, true, 8>(P, G, x, st, mode, lstatic, src, xs_out);
      WF_CUDA(cudaGetLastError());
      return WF_OK;
    }
    if (P.ana_x2 && P.ana_gacc) {
      if (np == 6)
        anal_variant<T, 6, true, true>(P, G, x, st, mode, lstatic, src, xs_out);
      else
        anal_variant<T, 4, true, true>(P, G, x, st, mode, lstatic, src, xs_out);
      WF_CUDA(cudaGetLastError());
      return WF_OK;
    }
    if (P.ana_x2) {
      if (np == 4)
        anal_variant<T, 4, true>(P, G, x, st, mode, lstatic, src, xs_out);
      else if (np == 6)
        anal_variant<T, 6, true>(P, G, x, st, mode, lstatic, src, xs_out);
      else
        anal_variant<T, 8, true>(P, G, x, st, mode, lstatic, src, xs_out);
      WF_CUDA(cudaGetLastError());
      return WF_OK;
    }
  }
  switch (np) {
    case 2: anal_variant<T, 2>(P, G, x, st, mode, lstatic, src, xs_out); break;
    case 4: anal_variant<T, 4>(P, G, x, st, mode, lstatic, src, xs_out); break;
    case 16: anal_variant<T, 16>(P, G, x, st, mode, lstatic, src, xs_out); break;
    default: anal_variant<T, 8>(P, G, x, st, mode, lstatic, src, xs_out); break;
  }
  WF_CUDA(cudaGetLastError());
  return WF_OK;
}

// double-float transforms for the anchors of the mixed solver (FP64 in and
// out; see the kernels above)
wf_status launch_legendre_synth_dd(const Plan &P, const float4 *xs, float4 *F,
                                   const SolverState *st, int lstatic) {
  const size_t smem = 3 * sizeof(dd) * (P.lmax + 1);
  const int pairs_per_cta = SYN_THREADS * DD_NP_SYN;
  dim3 grid((P.npairs + pairs_per_cta - 1) / pairs_per_cta, P.lmax + 1);
  ++P.nlaunch;
  k_legendre_synth_dd<<<grid, SYN_THREADS, smem, P.stream>>>(
      P.pairs, P.npairs, P.lmax, P.rcdd, P.seed_l, P.seed_u, xs, F, st, lstatic);
  WF_CUDA(cudaGetLastError());
  return WF_OK;
}

wf_status launch_legendre_anal_dd(const Plan &P, const float4 *G, double2 *x,
                                  const SolverState *st, int mode, int lstatic,
                                  const double2 *src, double2 *xs_out) {
  const size_t smem = sizeof(dd) * (P.lmax + 1) * ANA_WARPS;
  const int ntiles = (P.npairs + 32 * DD_NP_ANA - 1) / (32 * DD_NP_ANA);
  // one resident wave (occupancy queried once; the anchor steps that call
  // this are plain launches, never captured)
  static std::atomic<int> per_sm_cache{0};
  int per_sm = per_sm_cache.load();
  if (per_sm == 0) {
    int n = 0;
    WF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_legendre_anal_dd,
                                                          ANA_THREADS, smem));
    per_sm = std::max(1, std::min(n, ANA_Q_CTAS_PER_SM));
    per_sm_cache.store(per_sm);
  }
  double *scratch = reinterpret_cast<double *>(P.ana_scratch);
  ++P.nlaunch;
  k_legendre_anal_dd<<<P.num_sms * per_sm, ANA_THREADS, smem, P.stream>>>(
      P.pairs, P.npairs, P.lmax, P.nalm, P.rcdd, P.seed_l, P.seed_u, G, scratch,
      P.ana_lstart, P.ana_counter, st, lstatic);
  WF_CUDA(cudaGetLastError());
  ++P.nlaunch;
  k_anal_combine<double><<<P.lmax + 1, ANA_THREADS, 0, P.stream>>>(
      P.lmax, P.nalm, ntiles, scratch, P.ana_lstart, P.ana_counter, P.rg, P.cl_d, P.omega,
      x, P.partials, src, xs_out, st, mode, lstatic, Tab32{});
  WF_CUDA(cudaGetLastError());
  return WF_OK;
}

// Dynamic shared memory limit of a kernel: `big`, less what its own static
// shared memory (the FP32 analysis kernels' reduction buffer) takes of the
// per-block limit.
template <typename K>
static cudaError_t set_dyn_smem(K kern, int big) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kern);
  if (e != cudaSuccess) return e;
  int dev = 0, optin = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) !=
      cudaSuccess)
    return e;
  const int room = optin - (int)fa.sharedSizeBytes;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              big < room ? big : room);
}

template <typename T, int NP, bool X2 = false, bool DUP = false>
static cudaError_t set_big_smem_synth(int big) {
  return set_dyn_smem(k_legendre_synth<T, NP, X2, DUP>, big);
}

template <typename T, int NP, bool X2 = false, bool GACC = false, int LC = LCHUNK>
static cudaError_t set_big_smem_anal(int big) {
  return set_dyn_smem(k_legendre_anal<T, NP, X2, GACC, LC>, big);
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
  WF_CUDA((set_big_smem_synth<float, 2, true>(big)));
  WF_CUDA((set_big_smem_synth<float, 4, true>(big)));
  WF_CUDA((set_big_smem_synth<float, 2, true, true>(big)));
  WF_CUDA((set_big_smem_anal<float, 4, true>(big)));
  WF_CUDA((set_big_smem_anal<float, 8, true>(big)));
  WF_CUDA((set_big_smem_anal<float, 6, true>(big)));
  WF_CUDA((set_big_smem_anal<float, 4, true, true>(big)));
  WF_CUDA((set_big_smem_anal<float, 6, true, true>(big)));
  WF_CUDA((set_big_smem_anal<float, 8, true, true, 8>(big)));
  WF_CUDA((set_big_smem_anal<float, 6, true, true, 8>(big)));
  WF_CUDA((set_big_smem_anal<float, 4, true, true, 8>(big)));
  WF_CUDA(set_dyn_smem(k_legendre_anal_ss<8>, big));
  WF_CUDA(set_dyn_smem(k_legendre_synth_dd, big));
  WF_CUDA(set_dyn_smem(k_legendre_anal_dd, big));
  WF_CUDA(set_dyn_smem(k_legendre_anal_q<float, 4>, big));
  WF_CUDA(set_dyn_smem(k_legendre_anal_q<float, 8>, big));
  return WF_OK;
}

// xs = g_lm x_lm in the transform precision (the synthesis input; FP32
// also times eps_l); one block per m
template <typename T2>
__global__ void k_prescale(const double2 *__restrict__ x, const double *__restrict__ rg,
                           int lmax, T2 *__restrict__ xs) {
  typedef typename Scalar<T2>::type T;
  const int m = blockIdx.x;
  const long base = lm_index(lmax, m, m) - m;
  for (int l = m + threadIdx.x; l <= lmax; l += blockDim.x) {
    const long i = base + l;
    const double gs = rg[i] * fold_sign<T>(l);
    xs[i] = Vec2<T>::make((T)(gs * x[i].x), (T)(gs * x[i].y));
  }
}

template <typename T2>
wf_status launch_prescale(const Plan &P, const double2 *x, T2 *xs) {
  ++P.nlaunch;
  k_prescale<T2><<<P.lmax + 1, 128, 0, P.stream>>>(x, P.rg, P.lmax, xs);
  WF_CUDA(cudaGetLastError());
  return WF_OK;
}

// the synthesis input of the double-float transforms: g_lm x_lm (FP64
// product) as double-float pairs (re hi, re lo, im hi, im lo)
__global__ void k_prescale_dd(const double2 *__restrict__ x, const double *__restrict__ rg,
                              int lmax, float4 *__restrict__ xs) {
  const int m = blockIdx.x;
  const long base = lm_index(lmax, m, m) - m;
  for (int l = m + threadIdx.x; l <= lmax; l += blockDim.x) {
    const long i = base + l;
    const dd re = dd_of(rg[i] * x[i].x), im = dd_of(rg[i] * x[i].y);
    xs[i] = make_float4(re.hi, re.lo, im.hi, im.lo);
  }
}

wf_status launch_prescale_dd(const Plan &P, const double2 *x, float4 *xs) {
  ++P.nlaunch;
  k_prescale_dd<<<P.lmax + 1, 128, 0, P.stream>>>(x, P.rg, P.lmax, xs);
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
