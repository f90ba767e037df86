// group.cu -- Legendre transforms of a group of maps that share one
// geometry (Nside, lmax), contracted on the fifth-generation tensor cores.
//
// For one m the Legendre step of every map of the group is one dense
// product (Sect. 2.2's Y and Omega Y^T, split by the parity of l - m as in
// legendre.cu):
//   analysis   a_lm[b] = Omega sum_k lam_lm(z_k) P^p_m[k][b],
//              P^p_m = G_N[m] + (-1)^p G_S[m]                 (p = (l-m) & 1)
//              -> (rows l) x (K = ring pairs) times (K x N),
//   synthesis  E^p_m[k][b] = sum_{l: (l-m)&1 = p} lam_lm(z_k) a_lm[b],
//              F_N = E^0 + E^1, F_S = E^0 - E^1
//              -> (rows = ring pairs) x (K = l) times (K x N),
// with N = 2 x maps (real and imaginary parts as columns).  One table of
// lam_lm(z_k) per geometry, built once from the plan's FP64 recurrence, feeds
// both; the maps' ring coefficients are the product's N side, so the table is
// read once per call however many maps the group holds.
//
// Arithmetic: 3xTF32.  Every FP32 operand x is split into hi = x cut to TF32
// and lo = (x - hi) cut to TF32; kind::tf32 MMAs form A_hi B_hi + A_hi B_lo +
// A_lo B_hi with FP32 accumulation in tensor memory (the dropped A_lo B_lo
// and the cut of lo are below 2^-21 relative), so the products carry about
// FP32 accuracy.
//
// Data layout: each operand tile is stored pre-tiled in global memory as the
// tensor core reads it from shared memory -- chunks of K = 16 columns, each
// a block of 8-row x 16-byte core matrices, rows outer -- so one bulk copy
// (cp.async.bulk, the TMA engine) per operand and chunk moves it, and the
// shared-memory descriptors need no swizzling.  Only the rows a tile holds
// (rounded up to 8) are stored and copied.
//
// Kernel: one CTA of 128 threads per work item: one m and one 128-row tile
// (analysis: 128 l of each parity; synthesis: 128 ring pairs), the two
// parities accumulated side by side in tensor memory.  Thread 0 issues the
// copies of a multi-stage ring of chunk buffers and the MMAs (one elected
// thread per CTA) and commits each chunk's MMAs to the barrier that frees
// its buffer; the four warps read the accumulators out of tensor memory
// (tcgen05.ld, one lane per row) for the epilogue.  Two CTAs share an SM
// (up to 64 maps per launch), so one's epilogue overlaps the other's
// copies and products.  Every barrier wait is bounded: on a timeout the
// kernel sets an error word, waits (bounded) for its copies in flight, frees
// its tensor memory and returns.
#include <algorithm>
#include <vector>

#include "tc05.cuh"
#include "wf_internal.cuh"

namespace wf {

using namespace tc05;

constexpr int GT = 128;          // rows of a tile (MMA M)
constexpr int GKC = 16;          // K columns per chunk
constexpr int G_THREADS = 128;
constexpr int G_MAX_MAPS = 128;  // maps per launch (N = 2 maps <= 256)
constexpr long G_SPINS = 1L << 22;

// One work item of the contraction: two K segments (the parities p = 0, 1
// of one m) accumulated into two tensor-memory accumulators.
struct GItem {
  long a_off[2];   // float offset of the segment's first A chunk block
  long b_unit[2];  // the segment's first B chunk block starts at b_unit x N floats
  int k[2];        // K extent of the segment (a multiple of 8; 0 = empty)
  int rows[2];     // valid rows of the segment's tile
  int r8[2];       // rows rounded up to 8 (rows stored per chunk block)
  int m, tile;
};

// offset of element (row i, column j) inside a chunk block of kc columns
__host__ __device__ inline long core_off(int i, int j, int kc) {
  return ((long)(i >> 3) * (kc >> 2) + (j >> 2)) * 32 + (i & 7) * 4 + (j & 3);
}

__device__ __forceinline__ long glm_index(int lmax, int l, int m) {
  return (long)m * (2 * lmax + 1 - m) / 2 + l;
}

// number of l with l - m = p (mod 2), m <= l <= lmax
__host__ __device__ inline int par_count(int lmax, int m, int p) {
  return m + p > lmax ? 0 : (lmax - m - p) / 2 + 1;
}
__host__ __device__ inline int round8(int x) { return (x + 7) & ~7; }

__device__ __forceinline__ void split4(const float (&v)[4], float4 &h, float4 &l) {
  h.x = tf32_trunc(v[0]); l.x = tf32_trunc(v[0] - h.x);
  h.y = tf32_trunc(v[1]); l.y = tf32_trunc(v[1] - h.y);
  h.z = tf32_trunc(v[2]); l.z = tf32_trunc(v[2] - h.z);
  h.w = tf32_trunc(v[3]); l.w = tf32_trunc(v[3] - h.w);
}

// Per-plan state of the grouped transforms (built by the first call).
struct GroupState {
  int npairs = 0, k8 = 0;        // ring pairs, rounded up to 8
  std::vector<GItem> ana_h, syn_h;
  GItem *ana = nullptr, *syn = nullptr;
  int *ana_first = nullptr;      // [lmax+1] first analysis item of m
  int *syn_first = nullptr;      // [lmax+1] first synthesis item of m
  float *ta_hi = nullptr, *ta_lo = nullptr;  // analysis table (A of the analysis)
  float *ts_hi = nullptr, *ts_lo = nullptr;  // synthesis table
  long ta_floats = 0, ts_floats = 0;
  long *xoff = nullptr;          // [(lmax+1) * 2] synthesis B block start / N
  long xoff_total = 0;
  // per-call operands, grown on demand
  int cap_maps = 0;
  float *b_hi = nullptr, *b_lo = nullptr;     // B of the analysis or synthesis
  long b_floats = 0;
  float2 *ring = nullptr;        // [maps][nring][lmax+1] G or F, per map
  int *err = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
};

// ------------------------------------------------------------- table build
// lam_lm(z_k) from the FP64 recurrence of the plan's tables (u from the
// seeds at seed_l, lam = g u; lam = 0 below the seed, |lam| < 2^-100 there),
// split and scattered into both tables.  One thread per (m, pair).
__global__ void k_group_tables(const RingPair *__restrict__ pairs, int npairs, int lmax,
                               const double *__restrict__ rc, const double *__restrict__ rg,
                               const int *__restrict__ seed_l,
                               const double2 *__restrict__ seed_u,
                               const GItem *__restrict__ ana, const int *__restrict__ ana_first,
                               const GItem *__restrict__ syn, const int *__restrict__ syn_first,
                               int k8, float *ta_hi, float *ta_lo, float *ts_hi, float *ts_lo) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = blockIdx.y;
  if (k >= npairs) return;
  const long mk = (long)m * npairs + k;
  const int ls = seed_l[mk];
  if (ls > lmax) return;
  const double2 su = seed_u[mk];
  const double z = pairs[k].z;
  // analysis: column k % GKC of chunk k / GKC
  const int ca = k / GKC, ja = k % GKC, kca = min(GKC, k8 - GKC * ca);
  // synthesis: row k % 128 of pair tile k / 128
  const int ts = k / GT, is = k % GT;
  double u1 = 0.0, u2 = 0.0;
  for (int l = ls; l <= lmax; ++l) {
    const long i = glm_index(lmax, l, m);
    double u;
    if (l == ls) u = su.x;
    else if (l == ls + 1) u = su.y;
    else u = fma(rc[i] * z, u1, -u2);
    u2 = u1;
    u1 = u;
    const double lam = rg[i] * u;
    const float hi = tf32_trunc((float)lam);
    const float lo = tf32_trunc((float)(lam - (double)hi));
    const int p = (l - m) & 1, j = (l - m - p) >> 1;
    {
      const GItem &it = ana[ana_first[m] + j / GT];
      const long o = it.a_off[p] + (long)ca * it.r8[p] * GKC + core_off(j % GT, ja, kca);
      ta_hi[o] = hi;
      ta_lo[o] = lo;
    }
    {
      const GItem &it = syn[syn_first[m] + ts];
      const int kp = it.k[p];
      const int c = j / GKC, kc = min(GKC, kp - GKC * c);
      const long o = it.a_off[p] + (long)c * it.r8[p] * GKC + core_off(is, j % GKC, kc);
      ts_hi[o] = hi;
      ts_lo[o] = lo;
    }
  }
}

// ------------------------------------------------------------ operand packs
// analysis B: P^p_m[k][n] (n = 2 b + 0 / 1 for re / im) of 8 consecutive m,
// one K chunk and 4 maps per CTA: the ring coefficients are read in runs of
// 8 m and staged in shared memory; each (m, p) block of the 4 maps' 8 rows
// is written as whole 128-byte core matrices.
constexpr int PACK_THREADS = 256;
__global__ void __launch_bounds__(PACK_THREADS)
    k_group_pack_ana(const RingPair *__restrict__ pairs, int npairs, int lmax, int k8, int N,
                     int nmaps, const float2 *__restrict__ G, long gstride, float *bh,
                     float *bl) {
  __shared__ float2 sg[4][2][GKC][8];  // [map][north, south][pair][m]
  const int m0 = 8 * blockIdx.x, c = blockIdx.y, g = blockIdx.z;
  const int kc = min(GKC, k8 - GKC * c);
  for (int t = threadIdx.x; t < 4 * 2 * GKC * 8; t += blockDim.x) {
    const int mm = t & 7, kk = (t >> 3) % GKC, s = ((t >> 3) / GKC) & 1, b4 = t / (16 * GKC);
    const int b = 4 * g + b4, k = GKC * c + kk, m = m0 + mm;
    float2 v = make_float2(0.f, 0.f);
    if (b < nmaps && k < npairs && m <= lmax) {
      const int ring = s == 0 ? pairs[k].ringN : pairs[k].ringS;
      if (ring >= 0) v = G[(long)b * gstride + (long)ring * (lmax + 1) + m];
    }
    sg[b4][s][kk][mm] = v;
  }
  __syncthreads();
  const int nki = kc / 4;
  for (int t = threadIdx.x; t < 8 * 2 * nki * 8; t += blockDim.x) {
    const int r = t & 7, ki = (t >> 3) % nki, rest = (t >> 3) / nki;
    const int p = rest & 1, mm = rest >> 1, m = m0 + mm;
    if (m > lmax || par_count(lmax, m, p) == 0) continue;
    const int b4 = r >> 1, ri = r & 1;
    float v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float2 gn = sg[b4][0][4 * ki + u][mm], gs = sg[b4][1][4 * ki + u][mm];
      const float a = ri == 0 ? gn.x : gn.y, b = ri == 0 ? gs.x : gs.y;
      v[u] = p == 0 ? a + b : a - b;
    }
    float4 h, l;
    split4(v, h, l);
    const long o = (long)(2 * m + p) * N * k8 + (long)c * N * GKC + core_off(8 * g + r, 4 * ki, kc);
    *reinterpret_cast<float4 *>(bh + o) = h;
    *reinterpret_cast<float4 *>(bl + o) = l;
  }
}

// synthesis B: X^p_m[n][j] = a_{m+p+2j, m}[b] (re / im); one thread per
// (m, parity, 4 consecutive j, map)
__global__ void k_group_pack_syn(int lmax, long nalm, int N, const long *__restrict__ xoff,
                                 const double2 *__restrict__ alm, float *bh, float *bl) {
  const int m = blockIdx.y, b = blockIdx.z;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int p = t & 1, q = t >> 1;
  const int cnt = par_count(lmax, m, p);
  const int kp = round8(cnt);
  if (4 * q >= kp) return;
  const double2 *ab = alm + (long)b * nalm;
  float re[4], im[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int j = 4 * q + u;
    double2 a = make_double2(0.0, 0.0);
    if (j < cnt) a = ab[glm_index(lmax, m + p + 2 * j, m)];
    re[u] = (float)a.x;
    im[u] = (float)a.y;
  }
  const int c = (4 * q) / GKC, kc = min(GKC, kp - GKC * c), j0 = (4 * q) % GKC;
  const long base = xoff[2 * m + p] * N + (long)c * N * GKC;
  float4 h, l;
  split4(re, h, l);
  *reinterpret_cast<float4 *>(bh + base + core_off(2 * b, j0, kc)) = h;
  *reinterpret_cast<float4 *>(bl + base + core_off(2 * b, j0, kc)) = l;
  split4(im, h, l);
  *reinterpret_cast<float4 *>(bh + base + core_off(2 * b + 1, j0, kc)) = h;
  *reinterpret_cast<float4 *>(bl + base + core_off(2 * b + 1, j0, kc)) = l;
}

// ------------------------------------------------------------- contraction
// Both modes accumulate segment p into tensor-memory columns [p N, p N + N).
// MODE 0 (analysis) epilogue: a_lm = Omega D_p for l = m + p + 2 j;
// MODE 1 (synthesis): F_N = D0 + D1, F_S = D0 - D1.
struct GOut {
  double2 *alm;          // analysis: [maps][nalm]
  float2 *F;             // synthesis: [maps][nring][lmax+1]
  const RingPair *pairs;
  long nalm, fstride;    // per-map strides of alm and F
  double omega;
  int lmax, nmaps;
};

template <int MODE>
__global__ void __launch_bounds__(G_THREADS, 2)
    k_group_mma(const GItem *__restrict__ items, const float *__restrict__ a_hi,
                const float *__restrict__ a_lo, const float *__restrict__ b_hi,
                const float *__restrict__ b_lo, int N, int stages, uint32_t tmem_cols,
                GOut out, int *err) {
  extern __shared__ __align__(128) unsigned char gsm[];
  uint64_t *bars = reinterpret_cast<uint64_t *>(gsm);  // full[4], empty[4], done
  uint32_t *slot = reinterpret_cast<uint32_t *>(gsm + 9 * 8);
  unsigned char *buf = gsm + 128;
  const uint32_t a_bytes_max = GT * GKC * 4, b_bytes_max = (uint32_t)N * GKC * 4;
  const uint32_t stage_bytes = 2 * a_bytes_max + 2 * b_bytes_max;
  const int tid = threadIdx.x, warp = tid >> 5;
  const GItem it = items[blockIdx.x];

  if (tid == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(smem_u32(&bars[s]), 1);
      mbar_init(smem_u32(&bars[4 + s]), 1);
    }
    mbar_init(smem_u32(&bars[8]), 1);
    fence_barrier_init();
  }
  if (warp == 0) tmem_alloc(smem_u32(slot), tmem_cols);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tbase = *slot;

  const int c0 = (it.k[0] + GKC - 1) / GKC;
  const int C = c0 + (it.k[1] + GKC - 1) / GKC;

  if (tid == 0) {
    const uint32_t idesc = idesc_tf32(GT, N);
    int issued = 0, consumed = 0;
    bool ok = true;
    // chunk i -> its segment, chunk index and width
    // (segment fields selected without indexing, so they stay in registers)
    auto chunk = [&](int i, int &seg, int &c, int &kc) {
      seg = i < c0 ? 0 : 1;
      c = seg == 0 ? i : i - c0;
      kc = min(GKC, (seg ? it.k[1] : it.k[0]) - GKC * c);
    };
    auto issue = [&](int i) {
      int seg, c, kc;
      chunk(i, seg, c, kc);
      const int s = i % stages;
      const int r8 = seg ? it.r8[1] : it.r8[0];
      const uint32_t ab = (uint32_t)r8 * kc * 4, bb = (uint32_t)N * kc * 4;
      unsigned char *sb = buf + (size_t)s * stage_bytes;
      const uint32_t full = smem_u32(&bars[s]);
      mbar_arrive_expect_tx(full, 2 * (ab + bb));
      const long ao = (seg ? it.a_off[1] : it.a_off[0]) + (long)c * r8 * GKC;
      const long bo = (seg ? it.b_unit[1] : it.b_unit[0]) * N + (long)c * N * GKC;
      bulk_g2s(smem_u32(sb), a_hi + ao, ab, full);
      bulk_g2s(smem_u32(sb + a_bytes_max), a_lo + ao, ab, full);
      bulk_g2s(smem_u32(sb + 2 * a_bytes_max), b_hi + bo, bb, full);
      bulk_g2s(smem_u32(sb + 2 * a_bytes_max + b_bytes_max), b_lo + bo, bb, full);
      ++issued;
    };
    for (int i = 0; i < min(stages, C); ++i) issue(i);
    for (int i = 0; i < C && ok; ++i) {
      // refill the buffer of the previous chunk once its MMAs are done, before
      // waiting for this chunk: all stages' copies stay in flight
      if (i >= 1 && i - 1 + stages < C) {
        const int sp = (i - 1) % stages;
        if (!mbar_wait(smem_u32(&bars[4 + sp]), ((i - 1) / stages) & 1, G_SPINS)) {
          ok = false;
          break;
        }
        issue(i - 1 + stages);
      }
      const int s = i % stages;
      if (!mbar_wait(smem_u32(&bars[s]), (i / stages) & 1, G_SPINS)) {
        ok = false;
        break;
      }
      ++consumed;
      fence_after_sync();
      int seg, c, kc;
      chunk(i, seg, c, kc);
      const uint32_t sa = smem_u32(buf + (size_t)s * stage_bytes);
      const uint32_t sal = sa + a_bytes_max, sbh = sa + 2 * a_bytes_max,
                     sbl = sbh + b_bytes_max;
      const uint32_t lbo = 128, sbo = (uint32_t)kc * 32;
      const uint32_t d = tbase + (uint32_t)(seg * N);
      for (int st = 0; st < kc / 8; ++st) {
        const uint32_t o = st * 256;
        const uint64_t ah = smem_desc(sa + o, lbo, sbo), al = smem_desc(sal + o, lbo, sbo);
        const uint64_t bh = smem_desc(sbh + o, lbo, sbo), bl = smem_desc(sbl + o, lbo, sbo);
        mma_tf32(d, ah, bh, idesc, (c > 0 || st > 0) ? 1u : 0u);
        mma_tf32(d, ah, bl, idesc, 1u);
        mma_tf32(d, al, bh, idesc, 1u);
      }
      mma_commit(smem_u32(&bars[4 + s]));
    }
    mma_commit(smem_u32(&bars[8]));
    if (!ok) {
      atomicExch(err, 1);
      // copies still in flight land before the CTA leaves
      for (int i = consumed; i < issued; ++i)
        mbar_wait(smem_u32(&bars[i % stages]), (i / stages) & 1, G_SPINS);
    }
  }
  __syncwarp();
  const bool done = mbar_wait(smem_u32(&bars[8]), 0, G_SPINS);
  if (!done) atomicExch(err, 2);
  fence_after_sync();

  if (done) {
    const int row = tid;  // tensor-memory lane = tile row
    const uint32_t lane_addr = tbase + ((uint32_t)(warp * 32) << 16);
    const bool has_odd = it.k[1] > 0;
    if constexpr (MODE == 0) {
      const int j = it.tile * GT + row;
      const bool v0 = row < it.rows[0], v1 = row < it.rows[1];
      const long i0 = glm_index(out.lmax, it.m + 2 * j, it.m);
      for (int c = 0; c < N; c += 16) {
        float e[16], o[16];
        tmem_ld16(lane_addr + c, e);
        if (has_odd) tmem_ld16(lane_addr + N + c, o);
        tmem_wait_ld();
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int b = c / 2 + q;
          if (b >= out.nmaps) continue;
          double2 *ab = out.alm + (long)b * out.nalm + i0;
          if (v0) ab[0] = make_double2(out.omega * e[2 * q], out.omega * e[2 * q + 1]);
          if (v1) ab[1] = make_double2(out.omega * o[2 * q], out.omega * o[2 * q + 1]);
        }
      }
    } else {
      const int k = it.tile * GT + row;
      const bool valid = row < it.rows[0];
      int ring_n = 0, ring_s = -1;
      if (valid) {
        ring_n = out.pairs[k].ringN;
        ring_s = out.pairs[k].ringS;
      }
      for (int c = 0; c < N; c += 16) {
        float e[16], o[16];
        tmem_ld16(lane_addr + c, e);
        if (has_odd) tmem_ld16(lane_addr + N + c, o);
        tmem_wait_ld();
        if (valid) {
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int b = c / 2 + q;
            if (b >= out.nmaps) continue;
            const float er = e[2 * q], ei = e[2 * q + 1];
            const float orr = has_odd ? o[2 * q] : 0.f, oi = has_odd ? o[2 * q + 1] : 0.f;
            float2 *Fb = out.F + (long)b * out.fstride;
            Fb[(long)ring_n * (out.lmax + 1) + it.m] = make_float2(er + orr, ei + oi);
            if (ring_s >= 0)
              Fb[(long)ring_s * (out.lmax + 1) + it.m] = make_float2(er - orr, ei - oi);
          }
        }
      }
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    fence_after_sync();
    tmem_dealloc(tbase, tmem_cols);
  }
}

// ------------------------------------------------------------------- host
static inline int round16(int x) { return (x + 15) & ~15; }
static inline uint32_t pow2_cols(int c) {
  uint32_t n = 32;
  while ((int)n < c) n <<= 1;
  return n;
}
static size_t stage_bytes(int N) { return 2 * (size_t)GT * GKC * 4 + 2 * (size_t)N * GKC * 4; }
// Up to N = 128 two CTAs share an SM (their accumulators, 2 N columns each,
// fit the 512 tensor-memory columns together; shared memory <= 113 KB each);
// above, one CTA per SM with a deeper ring of chunk buffers.
static int stage_count(int N) {
  const size_t avail = (N <= 128 ? 113 * 1024 : 220 * 1024) - 128;
  return (int)std::max<size_t>(2, std::min<size_t>(4, avail / stage_bytes(N)));
}
static size_t smem_bytes(int N) { return 128 + stage_count(N) * stage_bytes(N); }

void free_group(Plan &P) {
  GroupState *g = P.group;
  if (!g) return;
  void *bufs[] = {g->ana, g->syn, g->ana_first, g->syn_first, g->ta_hi, g->ta_lo, g->ts_hi,
                  g->ts_lo, g->xoff, g->b_hi, g->b_lo, g->ring, g->err};
  for (void *b : bufs)
    if (b) cudaFree(b);
  for (cudaEvent_t e : g->ev)
    if (e) cudaEventDestroy(e);
  delete g;
  P.group = nullptr;
}

template <typename T>
static wf_status upload(T **dst, const std::vector<T> &v) {
  WF_CUDA(cudaMalloc(dst, sizeof(T) * std::max<size_t>(1, v.size())));
  if (!v.empty())
    WF_CUDA(cudaMemcpy(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
  return WF_OK;
}

// work items, offsets and the two lam tables of the plan's geometry
static wf_status build_group(Plan &P) {
  GroupState *g = new (std::nothrow) GroupState();
  if (!g) {
    set_error("group transforms: out of host memory");
    return WF_ERR_CUDA;
  }
  P.group = g;
  const int L = P.lmax;
  g->npairs = P.npairs;
  g->k8 = round8(P.npairs);
  std::vector<int> ana_first(L + 1, 0), syn_first(L + 1, 0);
  std::vector<long> xoff(2 * (L + 1), 0);
  long xo = 0;
  for (int m = 0; m <= L; ++m)
    for (int p = 0; p < 2; ++p) {
      xoff[2 * m + p] = xo;
      xo += round8(par_count(L, m, p));
    }
  g->xoff_total = xo;
  long ta = 0, ts = 0;
  for (int m = 0; m <= L; ++m) {
    ana_first[m] = (int)g->ana_h.size();
    for (int t = 0; t * GT < par_count(L, m, 0); ++t) {
      GItem it{};
      for (int p = 0; p < 2; ++p) {
        it.rows[p] = std::max(0, std::min(GT, par_count(L, m, p) - t * GT));
        it.r8[p] = round8(it.rows[p]);
        it.k[p] = it.rows[p] > 0 ? g->k8 : 0;
        it.a_off[p] = ta;
        ta += (long)it.r8[p] * it.k[p];
        it.b_unit[p] = (long)(2 * m + p) * g->k8;
      }
      it.m = m;
      it.tile = t;
      g->ana_h.push_back(it);
    }
  }
  for (int m = 0; m <= L; ++m) {
    syn_first[m] = (int)g->syn_h.size();
    for (int t = 0; t * GT < P.npairs; ++t) {
      GItem it{};
      for (int p = 0; p < 2; ++p) {
        it.rows[p] = std::min(GT, P.npairs - t * GT);
        it.r8[p] = round8(it.rows[p]);
        it.k[p] = round8(par_count(L, m, p));
        it.a_off[p] = ts;
        ts += (long)it.r8[p] * it.k[p];
        it.b_unit[p] = xoff[2 * m + p];
      }
      it.m = m;
      it.tile = t;
      g->syn_h.push_back(it);
    }
  }
  g->ta_floats = ta;
  g->ts_floats = ts;
  WF_TRY(upload(&g->ana, g->ana_h));
  WF_TRY(upload(&g->syn, g->syn_h));
  WF_TRY(upload(&g->ana_first, ana_first));
  WF_TRY(upload(&g->syn_first, syn_first));
  WF_TRY(upload(&g->xoff, xoff));
  float **tabs[4] = {&g->ta_hi, &g->ta_lo, &g->ts_hi, &g->ts_lo};
  for (int i = 0; i < 4; ++i) {
    const size_t n = (size_t)(i < 2 ? ta : ts);
    WF_CUDA(cudaMalloc(tabs[i], sizeof(float) * std::max<size_t>(1, n)));
    WF_CUDA(cudaMemsetAsync(*tabs[i], 0, sizeof(float) * n, P.stream));
  }
  WF_CUDA(cudaMalloc(&g->err, sizeof(int)));
  WF_CUDA(cudaMemsetAsync(g->err, 0, sizeof(int), P.stream));
  for (auto &e : g->ev) WF_CUDA(cudaEventCreate(&e));
  WF_CUDA(cudaFuncSetAttribute(k_group_mma<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem_bytes(2 * G_MAX_MAPS)));
  WF_CUDA(cudaFuncSetAttribute(k_group_mma<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem_bytes(2 * G_MAX_MAPS)));
  dim3 grid((P.npairs + 127) / 128, L + 1);
  ++P.nlaunch;
  k_group_tables<<<grid, 128, 0, P.stream>>>(P.pairs, P.npairs, L, P.rc, P.rg, P.seed_l,
                                             P.seed_u, g->ana, g->ana_first, g->syn,
                                             g->syn_first, g->k8, g->ta_hi, g->ta_lo,
                                             g->ts_hi, g->ts_lo);
  WF_CUDA(cudaGetLastError());
  WF_CUDA(cudaStreamSynchronize(P.stream));
  return WF_OK;
}

// operand buffers for up to nmaps maps per launch
static wf_status reserve_group(Plan &P, int nmaps) {
  GroupState *g = P.group;
  if (nmaps <= g->cap_maps) return WF_OK;
  if (g->b_hi) cudaFree(g->b_hi);
  if (g->b_lo) cudaFree(g->b_lo);
  if (g->ring) cudaFree(g->ring);
  g->b_hi = g->b_lo = nullptr;
  g->ring = nullptr;
  g->cap_maps = 0;
  const int N = round16(2 * nmaps);
  const long fb_ana = (long)2 * (P.lmax + 1) * g->k8 * N;
  const long fb_syn = g->xoff_total * N;
  g->b_floats = std::max(fb_ana, fb_syn);
  WF_CUDA(cudaMalloc(&g->b_hi, sizeof(float) * g->b_floats));
  WF_CUDA(cudaMalloc(&g->b_lo, sizeof(float) * g->b_floats));
  WF_CUDA(cudaMemsetAsync(g->b_hi, 0, sizeof(float) * g->b_floats, P.stream));
  WF_CUDA(cudaMemsetAsync(g->b_lo, 0, sizeof(float) * g->b_floats, P.stream));
  WF_CUDA(cudaMalloc(&g->ring, sizeof(float2) * (size_t)nmaps * P.nring * (P.lmax + 1)));
  g->cap_maps = nmaps;
  return WF_OK;
}

static wf_status check_group_err(Plan &P) {
  int e = 0;
  WF_CUDA(cudaMemcpyAsync(&e, P.group->err, sizeof(int), cudaMemcpyDeviceToHost, P.stream));
  WF_CUDA(cudaStreamSynchronize(P.stream));
  if (e) {
    WF_CUDA(cudaMemset(P.group->err, 0, sizeof(int)));
    set_error("grouped Legendre contraction: a barrier wait timed out");
    return WF_ERR_TIMEOUT;
  }
  return WF_OK;
}

// one timed launch of the contraction; records time, algorithmic flops and
// the bytes of its operands and result
template <int MODE>
static wf_status launch_mma(Plan &P, int nb, GOut out) {
  GroupState *g = P.group;
  const int N = round16(2 * nb);
  const std::vector<GItem> &items = MODE == 0 ? g->ana_h : g->syn_h;
  const uint32_t cols = pow2_cols(2 * N);
  WF_CUDA(cudaEventRecord(g->ev[0], P.stream));
  ++P.nlaunch;
  k_group_mma<MODE><<<(unsigned)items.size(), G_THREADS, smem_bytes(N), P.stream>>>(
      MODE == 0 ? g->ana : g->syn, MODE == 0 ? g->ta_hi : g->ts_hi,
      MODE == 0 ? g->ta_lo : g->ts_lo, g->b_hi, g->b_lo, N, stage_count(N), cols, out, g->err);
  WF_CUDA(cudaGetLastError());
  WF_CUDA(cudaEventRecord(g->ev[1], P.stream));
  WF_CUDA(cudaEventSynchronize(g->ev[1]));
  float ms = 0.f;
  WF_CUDA(cudaEventElapsedTime(&ms, g->ev[0], g->ev[1]));
  double terms = 0.0, bytes = 0.0;
  for (const GItem &it : items)
    for (int s = 0; s < 2; ++s) {
      terms += (double)it.rows[s] * (MODE == 0 ? P.npairs : it.k[s]);
      bytes += 8.0 * it.r8[s] * it.k[s];  // A hi + lo
    }
  // B hi + lo once, result once
  if (MODE == 0) {
    bytes += 8.0 * 2 * (P.lmax + 1) * g->k8 * N + 16.0 * nb * P.nalm;
  } else {
    bytes += 8.0 * g->xoff_total * N + 8.0 * nb * (double)P.nring * (P.lmax + 1);
  }
  P.group_ms += ms;
  P.group_launches += 1;
  P.group_flop += 2.0 * terms * 2 * nb;
  P.group_bytes += bytes;
  return check_group_err(P);
}

// build_group, leaving no half-built state behind on failure
static wf_status ensure_group(Plan &P) {
  if (P.group) return WF_OK;
  const wf_status s = build_group(P);
  if (s != WF_OK) free_group(P);
  return s;
}

wf_status map2alm_group(Plan &P, int nmaps, const double *maps, double *alm) {
  if (nmaps == 0) return WF_OK;
  WF_TRY(ensure_group(P));
  GroupState *g = P.group;
  WF_TRY(reserve_group(P, std::min(nmaps, G_MAX_MAPS)));
  const long fstride = (long)P.nring * (P.lmax + 1);
  for (int b0 = 0; b0 < nmaps; b0 += G_MAX_MAPS) {
    const int nb = std::min(G_MAX_MAPS, nmaps - b0);
    const int N = round16(2 * nb);
    WF_TRY(launch_ring_batch32(P, RING_ANALYSIS, nullptr, g->ring, maps + (long)b0 * P.npix,
                               nullptr, nb, fstride, P.npix));
    dim3 grid((P.lmax + 8) / 8, (g->k8 + GKC - 1) / GKC, (nb + 3) / 4);
    ++P.nlaunch;
    k_group_pack_ana<<<grid, PACK_THREADS, 0, P.stream>>>(P.pairs, P.npairs, P.lmax, g->k8, N,
                                                          nb, g->ring, fstride, g->b_hi,
                                                          g->b_lo);
    WF_CUDA(cudaGetLastError());
    GOut out{};
    out.alm = reinterpret_cast<double2 *>(alm) + (long)b0 * P.nalm;
    out.pairs = P.pairs;
    out.nalm = P.nalm;
    out.fstride = fstride;
    out.omega = P.omega;
    out.lmax = P.lmax;
    out.nmaps = nb;
    WF_TRY(launch_mma<0>(P, nb, out));
  }
  return WF_OK;
}

wf_status alm2map_group(Plan &P, int nmaps, const double *alm, double *maps) {
  if (nmaps == 0) return WF_OK;
  WF_TRY(ensure_group(P));
  GroupState *g = P.group;
  WF_TRY(reserve_group(P, std::min(nmaps, G_MAX_MAPS)));
  const long fstride = (long)P.nring * (P.lmax + 1);
  const int qmax = round8(par_count(P.lmax, 0, 0)) / 4;
  for (int b0 = 0; b0 < nmaps; b0 += G_MAX_MAPS) {
    const int nb = std::min(G_MAX_MAPS, nmaps - b0);
    const int N = round16(2 * nb);
    dim3 grid((2 * qmax + 127) / 128, P.lmax + 1, nb);
    ++P.nlaunch;
    k_group_pack_syn<<<grid, 128, 0, P.stream>>>(
        P.lmax, P.nalm, N, g->xoff, reinterpret_cast<const double2 *>(alm) + (long)b0 * P.nalm,
        g->b_hi, g->b_lo);
    WF_CUDA(cudaGetLastError());
    GOut out{};
    out.F = g->ring;
    out.pairs = P.pairs;
    out.nalm = P.nalm;
    out.fstride = fstride;
    out.omega = P.omega;
    out.lmax = P.lmax;
    out.nmaps = nb;
    WF_TRY(launch_mma<1>(P, nb, out));
    WF_TRY(launch_ring_batch32(P, RING_SYNTH, g->ring, nullptr, nullptr,
                               maps + (long)b0 * P.npix, nb, fstride, P.npix));
  }
  return WF_OK;
}

}  // namespace wf
