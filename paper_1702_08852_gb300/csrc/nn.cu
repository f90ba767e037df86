// nn.cu -- the learned warm start: a small network that maps (d, log sigma^2,
// mask) to an initial messenger field t0 and initial signal coefficients a0,
// with its forward pass, backward pass and Adam update as CUDA kernels.
//
// Network (weights kept in FP32, used rounded to BF16 when bf16 = 1; all
// accumulation in FP32):
//   input channels per pixel (observed: 1 - m, masked: m = 1):
//     c0 = (1-m) d / sigma_d, c1 = (1-m) (log sigma^2 - mu) / s, c2 = m
//   per-ring circular 1-D convolutions (kernel K, zero-based taps centred):
//     h1 = relu(W1 * c + b1)   (3 -> H channels)
//     h2 = relu(W2 * h1 + b2)  (H -> H)
//     r  = W3 * h2 + b3        (H -> 1)
//   t0 = (1-m) d + sigma_d r                       (messenger warm start)
//   a  = Omega Y^T t0                              (FP32 transform)
//   per-l MLP on features f_l = (l/lmax, log C_l, log P_d(l)/C_l,
//   log alpha Omega / C_l): q_l = sigmoid(V3 relu(V2 relu(V1 f_l + c1) + c2) + c3)
//   a0_lm = q_l a_lm                               (signal warm start)
// Loss: L = sum w |a0 - a*|^2 / sum w |a*|^2 against the solver's solution a*
// (real-basis weights w = 1 for m = 0, 2 for m > 0).
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "wf_internal.cuh"

struct wf_net_s;

namespace wf {

struct RingSpan {
  long start;
  int n;
};

struct Net {
  Plan *P = nullptr;
  int H = 16, K = 9, Hm = 32, bf16 = 1;
  long npar = 0, nconv = 0, nmlp = 0;
  long oW1, ob1, oW2, ob2, oW3, ob3, oV1, oc1, oV2, oc2, oV3, oc3;
  float *par = nullptr, *grad = nullptr, *am = nullptr, *av = nullptr;
  long step = 0;
  RingSpan *rings = nullptr;
  int nring = 0;
  float *in = nullptr, *h1 = nullptr, *h2 = nullptr, *r = nullptr;   // activations
  float *g1 = nullptr, *g2 = nullptr, *g3 = nullptr;                 // their gradients
  double *t0 = nullptr, *dmask = nullptr, *gmap = nullptr;
  double2 *a = nullptr, *ad = nullptr, *a0 = nullptr, *b = nullptr;
  float *feat = nullptr, *m1 = nullptr, *m2 = nullptr, *q = nullptr, *dq = nullptr;
  float *mpart = nullptr;   // [lmax+1][nmlp] per-l gradient contributions
  float *wpart = nullptr;   // conv weight-gradient partials
  double *red = nullptr;
  double sig_d = 1.0, mu_log = 0.0, sd_log = 1.0;
  int have_grad = 0;
};

constexpr int NN_THREADS = 256;
constexpr int NN_CHUNKS = 64;   // ring chunks of the weight-gradient reduction
constexpr int NN_MAXC = 32;     // max channels
constexpr int NN_MAXK = 15;     // max kernel width
constexpr int NN_MAXHM = 64;    // max MLP width
constexpr int NN_FEAT = 4;

__device__ __forceinline__ float wround(float w, int bf16) {
  return bf16 ? __bfloat162float(__float2bfloat16_rn(w)) : w;
}

// ---------------------------------------------------------------- inputs
__global__ void k_nn_stats(const double *d, const double *nvar, long npix, double *out) {
  __shared__ double s[4][NN_THREADS];
  double a = 0, b = 0, c = 0, n = 0;
  for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < npix;
       p += (long)gridDim.x * blockDim.x) {
    const double v = nvar[p];
    if (isinf(v)) continue;
    const double lg = log(v);
    a += d[p] * d[p];
    b += lg;
    c += lg * lg;
    n += 1.0;
  }
  s[0][threadIdx.x] = a;
  s[1][threadIdx.x] = b;
  s[2][threadIdx.x] = c;
  s[3][threadIdx.x] = n;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k)
      for (int j = 0; j < 4; ++j) s[j][threadIdx.x] += s[j][threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int j = 0; j < 4; ++j) out[4 * blockIdx.x + j] = s[j][0];
}

__global__ void k_nn_inputs(const double *d, const double *nvar, long npix, double sig_d,
                            double mu, double sd, float *in, double *dmask) {
  for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < npix;
       p += (long)gridDim.x * blockDim.x) {
    const double v = nvar[p];
    const bool m = isinf(v);
    in[p] = m ? 0.f : (float)(d[p] / sig_d);
    in[npix + p] = m ? 0.f : (float)((log(v) - mu) / sd);
    in[2 * npix + p] = m ? 1.f : 0.f;
    dmask[p] = m ? 0.0 : d[p];
  }
}

// ---------------------------------------------------------------- convolution
// out[co][p] = b[co] + sum_{ci,k} W[co][ci][k] in[ci][ring(p, j + k - K/2)],
// optionally ReLU; one CTA per ring, weights in shared memory.
__global__ void k_nn_conv_fwd(const RingSpan *rings, const float *__restrict__ in, int cin,
                              const float *__restrict__ W, const float *__restrict__ bias,
                              int cout, int K, int relu, int bf16, long npix,
                              float *__restrict__ out) {
  extern __shared__ float sw[];
  const int nw = cout * cin * K;
  for (int i = threadIdx.x; i < nw; i += blockDim.x) sw[i] = wround(W[i], bf16);
  for (int i = threadIdx.x; i < cout; i += blockDim.x) sw[nw + i] = wround(bias[i], bf16);
  __syncthreads();
  const RingSpan rs = rings[blockIdx.x];
  const int h = K / 2;
  for (int j = threadIdx.x; j < rs.n; j += blockDim.x) {
    float acc[NN_MAXC];
    for (int co = 0; co < cout; ++co) acc[co] = sw[nw + co];
    for (int ci = 0; ci < cin; ++ci) {
      const float *src = in + (long)ci * npix + rs.start;
      for (int k = 0; k < K; ++k) {
        int jj = (j + k - h) % rs.n;
        if (jj < 0) jj += rs.n;
        const float v = src[jj];
        const float *wk = sw + ci * K + k;
        for (int co = 0; co < cout; ++co) acc[co] = fmaf(wk[co * cin * K], v, acc[co]);
      }
    }
    for (int co = 0; co < cout; ++co) {
      const float o = relu ? fmaxf(acc[co], 0.f) : acc[co];
      out[(long)co * npix + rs.start + j] = o;
    }
  }
}

// gin[ci][p] = mask(p) * sum_{co,k} W[co][ci][k] gout[co][ring(p, j - (k - K/2))]
// with mask = (act[ci][p] > 0) when act is given (ReLU of the layer below)
__global__ void k_nn_conv_bwd_data(const RingSpan *rings, const float *__restrict__ gout,
                                   int cout, const float *__restrict__ W, int cin, int K,
                                   int bf16, const float *__restrict__ act, long npix,
                                   float *__restrict__ gin) {
  extern __shared__ float sw[];
  const int nw = cout * cin * K;
  for (int i = threadIdx.x; i < nw; i += blockDim.x) sw[i] = wround(W[i], bf16);
  __syncthreads();
  const RingSpan rs = rings[blockIdx.x];
  const int h = K / 2;
  for (int j = threadIdx.x; j < rs.n; j += blockDim.x) {
    float acc[NN_MAXC];
    for (int ci = 0; ci < cin; ++ci) acc[ci] = 0.f;
    for (int co = 0; co < cout; ++co) {
      const float *src = gout + (long)co * npix + rs.start;
      for (int k = 0; k < K; ++k) {
        int jj = (j - (k - h)) % rs.n;
        if (jj < 0) jj += rs.n;
        const float g = src[jj];
        const float *wk = sw + co * cin * K + k;
        for (int ci = 0; ci < cin; ++ci) acc[ci] = fmaf(wk[ci * K], g, acc[ci]);
      }
    }
    for (int ci = 0; ci < cin; ++ci) {
      const long p = (long)ci * npix + rs.start + j;
      float v = acc[ci];
      if (act && !(act[p] > 0.f)) v = 0.f;
      gin[p] = v;
    }
  }
}

// partial sums of dW[co][ci][k] = sum_p gout[co][p] in[ci][ring(p, j + k - K/2)]
// (ci = cin: the bias, sum_p gout[co][p]) over the rings of chunk blockIdx.y
__global__ void k_nn_conv_wgrad(const RingSpan *rings, int nring,
                                const float *__restrict__ gout, const float *__restrict__ in,
                                int cin, int K, long npix, float *__restrict__ part) {
  const int co = blockIdx.x / (cin + 1), ci = blockIdx.x % (cin + 1);
  const int chunk = blockIdx.y;
  const int r0 = (int)((long)nring * chunk / NN_CHUNKS);
  const int r1 = (int)((long)nring * (chunk + 1) / NN_CHUNKS);
  const int h = K / 2;
  float acc[NN_MAXK];
  for (int k = 0; k < K; ++k) acc[k] = 0.f;
  for (int r = r0; r < r1; ++r) {
    const RingSpan rs = rings[r];
    const float *go = gout + (long)co * npix + rs.start;
    const float *x = in + (long)ci * npix + rs.start;
    for (int j = threadIdx.x; j < rs.n; j += blockDim.x) {
      const float g = go[j];
      if (ci == cin) {
        acc[0] += g;
      } else {
        for (int k = 0; k < K; ++k) {
          int jj = (j + k - h) % rs.n;
          if (jj < 0) jj += rs.n;
          acc[k] = fmaf(g, x[jj], acc[k]);
        }
      }
    }
  }
  __shared__ float red[NN_THREADS];
  const int nk = ci == cin ? 1 : K;
  for (int k = 0; k < nk; ++k) {
    red[threadIdx.x] = acc[k];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) part[((long)blockIdx.x * NN_CHUNKS + chunk) * NN_MAXK + k] = red[0];
    __syncthreads();
  }
}

// fixed-order sum over chunks into the gradient vector
__global__ void k_nn_wgrad_reduce(const float *part, int cout, int cin, int K, float *gW,
                                  float *gb) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int nW = cout * cin * K;
  if (t < nW) {
    const int co = t / (cin * K), ci = (t / K) % cin, k = t % K;
    const long row = (long)(co * (cin + 1) + ci) * NN_CHUNKS;
    float s = 0.f;
    for (int c = 0; c < NN_CHUNKS; ++c) s += part[(row + c) * NN_MAXK + k];
    gW[t] = s;
  } else if (t < nW + cout) {
    const int co = t - nW;
    const long row = (long)(co * (cin + 1) + cin) * NN_CHUNKS;
    float s = 0.f;
    for (int c = 0; c < NN_CHUNKS; ++c) s += part[(row + c) * NN_MAXK];
    gb[co] = s;
  }
}

__global__ void k_nn_make_t0(const double *dmask, const float *r, double sig_d, long npix,
                             double *t0) {
  for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < npix;
       p += (long)gridDim.x * blockDim.x)
    t0[p] = dmask[p] + sig_d * (double)r[p];
}

// ---------------------------------------------------------------- harmonic MLP
__device__ __forceinline__ long nn_idx(int lmax, int l, int m) {
  return (long)m * (2 * lmax + 1 - m) / 2 + l;
}

__global__ void k_nn_features(const double2 *ad, const double *cl, int lmax, double aom,
                              float *feat) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l > lmax) return;
  double pd = 0.0;
  for (int m = 0; m <= l; ++m) {
    const double2 v = ad[nn_idx(lmax, l, m)];
    pd += (m == 0 ? 1.0 : 2.0) * (v.x * v.x + v.y * v.y);
  }
  pd /= (2.0 * l + 1.0);
  const double c = cl[l] + 1e-30;
  feat[NN_FEAT * l + 0] = (float)((double)l / lmax);
  feat[NN_FEAT * l + 1] = (float)fmin(fmax(log10(c) / 10.0, -4.0), 4.0);
  feat[NN_FEAT * l + 2] = (float)fmin(fmax(log10((pd + 1e-30) / c) / 5.0, -4.0), 4.0);
  feat[NN_FEAT * l + 3] = (float)fmin(fmax(log10(aom / c) / 5.0, -4.0), 4.0);
}

// one thread per l: q_l = sigmoid(V3 relu(V2 relu(V1 f + c1) + c2) + c3)
__global__ void k_nn_mlp_fwd(const float *feat, const float *par, long oV1, long oc1,
                             long oV2, long oc2, long oV3, long oc3, int Hm, int lmax,
                             int bf16, float *m1, float *m2, float *q) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l > lmax) return;
  float f[NN_FEAT], a1[NN_MAXHM], a2[NN_MAXHM];
  for (int i = 0; i < NN_FEAT; ++i) f[i] = feat[NN_FEAT * l + i];
  for (int o = 0; o < Hm; ++o) {
    float s = wround(par[oc1 + o], bf16);
    for (int i = 0; i < NN_FEAT; ++i) s = fmaf(wround(par[oV1 + o * NN_FEAT + i], bf16), f[i], s);
    a1[o] = fmaxf(s, 0.f);
    m1[(long)l * Hm + o] = a1[o];
  }
  for (int o = 0; o < Hm; ++o) {
    float s = wround(par[oc2 + o], bf16);
    for (int i = 0; i < Hm; ++i) s = fmaf(wround(par[oV2 + o * Hm + i], bf16), a1[i], s);
    a2[o] = fmaxf(s, 0.f);
    m2[(long)l * Hm + o] = a2[o];
  }
  float s = wround(par[oc3], bf16);
  for (int i = 0; i < Hm; ++i) s = fmaf(wround(par[oV3 + i], bf16), a2[i], s);
  q[l] = 1.f / (1.f + expf(-s));
}

// a0 = q_l a
__global__ void k_nn_gain(const double2 *a, const float *q, int lmax, double2 *a0) {
  const int m = blockIdx.x;
  for (int l = m + threadIdx.x; l <= lmax; l += blockDim.x) {
    const long i = nn_idx(lmax, l, m);
    a0[i] = make_double2(q[l] * a[i].x, q[l] * a[i].y);
  }
}

// per-m partial sums of sum w |a0 - a*|^2 and sum w |a*|^2
__global__ void k_nn_loss(const double2 *a0, const double2 *at, int lmax, double *part) {
  __shared__ double s0[128], s1[128];
  const int m = blockIdx.x;
  const double w = m == 0 ? 1.0 : 2.0;
  double e = 0.0, n = 0.0;
  for (int l = m + threadIdx.x; l <= lmax; l += blockDim.x) {
    const long i = nn_idx(lmax, l, m);
    const double dx = a0[i].x - at[i].x, dy = a0[i].y - at[i].y;
    e += w * (dx * dx + dy * dy);
    n += w * (at[i].x * at[i].x + at[i].y * at[i].y);
  }
  s0[threadIdx.x] = e;
  s1[threadIdx.x] = n;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) {
      s0[threadIdx.x] += s0[threadIdx.x + k];
      s1[threadIdx.x] += s1[threadIdx.x + k];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * m] = s0[0];
    part[2 * m + 1] = s1[0];
  }
}

// dL/dq_l = sum_m w 2 Re(conj(a0 - a*) a) / norm;  b = 2 q (a0 - a*) / norm
__global__ void k_nn_dq(const double2 *a0, const double2 *at, const double2 *a,
                        const float *q, int lmax, double inv_norm, float *dq, double2 *b) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l > lmax) return;
  double s = 0.0;
  for (int m = 0; m <= l; ++m) {
    const long i = nn_idx(lmax, l, m);
    const double w = m == 0 ? 1.0 : 2.0;
    const double dx = a0[i].x - at[i].x, dy = a0[i].y - at[i].y;
    s += w * 2.0 * (dx * a[i].x + dy * a[i].y);
    b[i] = make_double2(2.0 * q[l] * dx * inv_norm, 2.0 * q[l] * dy * inv_norm);
  }
  dq[l] = (float)(s * inv_norm);
}

// per-l contributions to the MLP gradient, row l of mpart
__global__ void k_nn_mlp_bwd(const float *feat, const float *par, long oV1, long oV2,
                             long oV3, int Hm, int lmax, int bf16, const float *m1,
                             const float *m2, const float *q, const float *dq,
                             long nmlp, float *mpart) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l > lmax) return;
  float *g = mpart + (long)l * nmlp;
  // local offsets inside the MLP block: V1, c1, V2, c2, V3, c3
  const long lV1 = 0, lc1 = lV1 + (long)Hm * NN_FEAT, lV2 = lc1 + Hm,
             lc2 = lV2 + (long)Hm * Hm, lV3 = lc2 + Hm, lc3 = lV3 + Hm;
  const float qq = q[l];
  const float dz = dq[l] * qq * (1.f - qq);  // through the sigmoid
  float d2[NN_MAXHM], d1[NN_MAXHM];
  g[lc3] = dz;
  for (int i = 0; i < Hm; ++i) {
    const float a2 = m2[(long)l * Hm + i];
    g[lV3 + i] = dz * a2;
    d2[i] = a2 > 0.f ? dz * wround(par[oV3 + i], bf16) : 0.f;
  }
  for (int i = 0; i < Hm; ++i) d1[i] = 0.f;
  for (int o = 0; o < Hm; ++o) {
    g[lc2 + o] = d2[o];
    for (int i = 0; i < Hm; ++i) {
      const float a1 = m1[(long)l * Hm + i];
      g[lV2 + (long)o * Hm + i] = d2[o] * a1;
      d1[i] = fmaf(wround(par[oV2 + (long)o * Hm + i], bf16), d2[o], d1[i]);
    }
  }
  for (int o = 0; o < Hm; ++o) {
    const float a1 = m1[(long)l * Hm + o];
    const float dd = a1 > 0.f ? d1[o] : 0.f;
    g[lc1 + o] = dd;
    for (int i = 0; i < NN_FEAT; ++i) g[lV1 + (long)o * NN_FEAT + i] = dd * feat[NN_FEAT * l + i];
  }
}

__global__ void k_nn_rows_sum(const float *mpart, int rows, long ncol, float *out) {
  const long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncol) return;
  float s = 0.f;
  for (int r = 0; r < rows; ++r) s += mpart[(long)r * ncol + c];
  out[c] = s;
}

// gradient of L w.r.t. the last conv output r: sig_d * Omega * (Y b)
__global__ void k_nn_gmap(const double *gmap, double scale, long npix, float *g3) {
  for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < npix;
       p += (long)gridDim.x * blockDim.x)
    g3[p] = (float)(scale * gmap[p]);
}

__global__ void k_nn_adam(float *par, const float *grad, float *m, float *v, long n,
                          float lr, float b1, float b2, float eps, float c1, float c2) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long)gridDim.x * blockDim.x) {
    const float g = grad[i];
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    par[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// ---------------------------------------------------------------- host
static void free_net_buffers(Net *N) {
  if (!N) return;
  void *bufs[] = {N->par, N->grad, N->am, N->av, N->rings, N->in, N->h1, N->h2, N->r,
                  N->g1, N->g2, N->g3, N->t0, N->dmask, N->gmap, N->a, N->ad, N->a0,
                  N->b, N->feat, N->m1, N->m2, N->q, N->dq, N->mpart, N->wpart, N->red};
  for (void *b : bufs)
    if (b) cudaFree(b);
}

static wf_status net_alloc(Net &N) {
  Plan &P = *N.P;
  const long np = P.npix;
  N.nring = P.nring;
  std::vector<RingSpan> rs(P.nring);
  for (const RingPair &p : P.pairs_h) {
    rs[p.ringN] = {p.ofsN, p.nphi};
    if (p.ringS >= 0) rs[p.ringS] = {p.ofsS, p.nphi};
  }
  WF_CUDA(cudaMalloc(&N.rings, sizeof(RingSpan) * P.nring));
  WF_CUDA(cudaMemcpy(N.rings, rs.data(), sizeof(RingSpan) * P.nring, cudaMemcpyHostToDevice));
  const int H = N.H, K = N.K, Hm = N.Hm;
  long o = 0;
  N.oW1 = o; o += (long)H * 3 * K; N.ob1 = o; o += H;
  N.oW2 = o; o += (long)H * H * K; N.ob2 = o; o += H;
  N.oW3 = o; o += (long)H * K;     N.ob3 = o; o += 1;
  N.nconv = o;
  N.oV1 = o; o += (long)Hm * NN_FEAT; N.oc1 = o; o += Hm;
  N.oV2 = o; o += (long)Hm * Hm;      N.oc2 = o; o += Hm;
  N.oV3 = o; o += Hm;                 N.oc3 = o; o += 1;
  N.npar = o;
  N.nmlp = N.npar - N.nconv;
  WF_CUDA(cudaMalloc(&N.par, sizeof(float) * N.npar));
  WF_CUDA(cudaMalloc(&N.grad, sizeof(float) * N.npar));
  WF_CUDA(cudaMalloc(&N.am, sizeof(float) * N.npar));
  WF_CUDA(cudaMalloc(&N.av, sizeof(float) * N.npar));
  WF_CUDA(cudaMemset(N.par, 0, sizeof(float) * N.npar));
  WF_CUDA(cudaMemset(N.am, 0, sizeof(float) * N.npar));
  WF_CUDA(cudaMemset(N.av, 0, sizeof(float) * N.npar));
  WF_CUDA(cudaMalloc(&N.in, sizeof(float) * 3 * np));
  WF_CUDA(cudaMalloc(&N.h1, sizeof(float) * H * np));
  WF_CUDA(cudaMalloc(&N.h2, sizeof(float) * H * np));
  WF_CUDA(cudaMalloc(&N.r, sizeof(float) * np));
  WF_CUDA(cudaMalloc(&N.g1, sizeof(float) * H * np));
  WF_CUDA(cudaMalloc(&N.g2, sizeof(float) * H * np));
  WF_CUDA(cudaMalloc(&N.g3, sizeof(float) * np));
  WF_CUDA(cudaMalloc(&N.t0, sizeof(double) * np));
  WF_CUDA(cudaMalloc(&N.dmask, sizeof(double) * np));
  WF_CUDA(cudaMalloc(&N.gmap, sizeof(double) * np));
  WF_CUDA(cudaMalloc(&N.a, sizeof(double2) * P.nalm));
  WF_CUDA(cudaMalloc(&N.ad, sizeof(double2) * P.nalm));
  WF_CUDA(cudaMalloc(&N.a0, sizeof(double2) * P.nalm));
  WF_CUDA(cudaMalloc(&N.b, sizeof(double2) * P.nalm));
  WF_CUDA(cudaMalloc(&N.feat, sizeof(float) * NN_FEAT * (P.lmax + 1)));
  WF_CUDA(cudaMalloc(&N.m1, sizeof(float) * Hm * (P.lmax + 1)));
  WF_CUDA(cudaMalloc(&N.m2, sizeof(float) * Hm * (P.lmax + 1)));
  WF_CUDA(cudaMalloc(&N.q, sizeof(float) * (P.lmax + 1)));
  WF_CUDA(cudaMalloc(&N.dq, sizeof(float) * (P.lmax + 1)));
  WF_CUDA(cudaMalloc(&N.mpart, sizeof(float) * N.nmlp * (P.lmax + 1)));
  const long wrows = (long)H * 4 + (long)H * (H + 1) + (H + 1);
  WF_CUDA(cudaMalloc(&N.wpart, sizeof(float) * wrows * NN_CHUNKS * NN_MAXK));
  WF_CUDA(cudaMalloc(&N.red, sizeof(double) * 4 * 304 + sizeof(double) * 2 * (P.lmax + 1)));
  return WF_OK;
}

// forward pass for data d: t0, a, q, a0 in the net's buffers
static wf_status net_forward(Net &N, const double *d) {
  Plan &P = *N.P;
  const long np = P.npix;
  cudaStream_t s = P.stream;
  k_nn_stats<<<304, NN_THREADS, 0, s>>>(d, P.nvar, np, N.red);
  WF_CUDA(cudaGetLastError());
  std::vector<double> h(4 * 304);
  WF_CUDA(cudaMemcpyAsync(h.data(), N.red, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s));
  WF_CUDA(cudaStreamSynchronize(s));
  double a = 0, b = 0, c = 0, n = 0;
  for (int i = 0; i < 304; ++i) {
    a += h[4 * i];
    b += h[4 * i + 1];
    c += h[4 * i + 2];
    n += h[4 * i + 3];
  }
  N.sig_d = n > 0 && a > 0 ? sqrt(a / n) : 1.0;
  N.mu_log = n > 0 ? b / n : 0.0;
  const double var = n > 0 ? c / n - N.mu_log * N.mu_log : 1.0;
  N.sd_log = var > 1e-24 ? sqrt(var) : 1.0;
  k_nn_inputs<<<304, NN_THREADS, 0, s>>>(d, P.nvar, np, N.sig_d, N.mu_log, N.sd_log, N.in,
                                         N.dmask);
  const int H = N.H, K = N.K;
  k_nn_conv_fwd<<<N.nring, NN_THREADS, sizeof(float) * (H * 3 * K + H), s>>>(
      N.rings, N.in, 3, N.par + N.oW1, N.par + N.ob1, H, K, 1, N.bf16, np, N.h1);
  k_nn_conv_fwd<<<N.nring, NN_THREADS, sizeof(float) * (H * H * K + H), s>>>(
      N.rings, N.h1, H, N.par + N.oW2, N.par + N.ob2, H, K, 1, N.bf16, np, N.h2);
  k_nn_conv_fwd<<<N.nring, NN_THREADS, sizeof(float) * (H * K + 1), s>>>(
      N.rings, N.h2, H, N.par + N.oW3, N.par + N.ob3, 1, K, 0, N.bf16, np, N.r);
  k_nn_make_t0<<<304, NN_THREADS, 0, s>>>(N.dmask, N.r, N.sig_d, np, N.t0);
  WF_CUDA(cudaGetLastError());
  WF_TRY(map2alm_f32(P, N.t0, reinterpret_cast<double *>(N.a)));
  WF_TRY(map2alm_f32(P, N.dmask, reinterpret_cast<double *>(N.ad)));
  const int lb = (P.lmax + 128) / 128;
  k_nn_features<<<lb, 128, 0, s>>>(N.ad, P.cl_d, P.lmax, P.alpha * P.omega, N.feat);
  k_nn_mlp_fwd<<<lb, 128, 0, s>>>(N.feat, N.par, N.oV1, N.oc1, N.oV2, N.oc2, N.oV3, N.oc3,
                                  N.Hm, P.lmax, N.bf16, N.m1, N.m2, N.q);
  k_nn_gain<<<P.lmax + 1, 128, 0, s>>>(N.a, N.q, P.lmax, N.a0);
  WF_CUDA(cudaGetLastError());
  P.nlaunch += 11;
  return WF_OK;
}

static wf_status net_loss_grad(Net &N, const double *d, const double2 *at, double *loss) {
  Plan &P = *N.P;
  const long np = P.npix;
  cudaStream_t s = P.stream;
  WF_TRY(net_forward(N, d));
  double *part = N.red + 4 * 304;
  k_nn_loss<<<P.lmax + 1, 128, 0, s>>>(N.a0, at, P.lmax, part);
  WF_CUDA(cudaGetLastError());
  std::vector<double> h(2 * (P.lmax + 1));
  WF_CUDA(cudaMemcpyAsync(h.data(), part, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s));
  WF_CUDA(cudaStreamSynchronize(s));
  double e = 0, nn = 0;
  for (int m = 0; m <= P.lmax; ++m) {
    e += h[2 * m];
    nn += h[2 * m + 1];
  }
  const double inv = nn > 0 ? 1.0 / nn : 0.0;
  if (loss) *loss = e * inv;
  const int lb = (P.lmax + 128) / 128;
  // harmonic MLP
  k_nn_dq<<<lb, 128, 0, s>>>(N.a0, at, N.a, N.q, P.lmax, inv, N.dq, N.b);
  k_nn_mlp_bwd<<<lb, 128, 0, s>>>(N.feat, N.par, N.oV1, N.oV2, N.oV3, N.Hm, P.lmax, N.bf16,
                                  N.m1, N.m2, N.q, N.dq, N.nmlp, N.mpart);
  k_nn_rows_sum<<<(unsigned)((N.nmlp + 127) / 128), 128, 0, s>>>(N.mpart, P.lmax + 1, N.nmlp,
                                                                 N.grad + N.nconv);
  WF_CUDA(cudaGetLastError());
  // back through a = Omega Y^T t0: dL/dt0 = Omega Y b, dL/dr = sig_d dL/dt0
  WF_TRY(alm2map_f32(P, reinterpret_cast<const double *>(N.b), N.gmap));
  k_nn_gmap<<<304, NN_THREADS, 0, s>>>(N.gmap, N.sig_d * P.omega, np, N.g3);
  const int H = N.H, K = N.K;
  float *wp = N.wpart;
  // layer 3 (H -> 1, no ReLU)
  k_nn_conv_wgrad<<<dim3(1 * (H + 1), NN_CHUNKS), NN_THREADS, 0, s>>>(N.rings, N.nring, N.g3,
                                                                    N.h2, H, K, np, wp);
  k_nn_wgrad_reduce<<<(H * K + 1 + 127) / 128, 128, 0, s>>>(wp, 1, H, K, N.grad + N.oW3,
                                                            N.grad + N.ob3);
  k_nn_conv_bwd_data<<<N.nring, NN_THREADS, sizeof(float) * H * K, s>>>(
      N.rings, N.g3, 1, N.par + N.oW3, H, K, N.bf16, N.h2, np, N.g2);
  // layer 2 (H -> H, ReLU)
  k_nn_conv_wgrad<<<dim3(H * (H + 1), NN_CHUNKS), NN_THREADS, 0, s>>>(N.rings, N.nring, N.g2,
                                                                    N.h1, H, K, np, wp);
  k_nn_wgrad_reduce<<<(H * H * K + H + 127) / 128, 128, 0, s>>>(wp, H, H, K, N.grad + N.oW2,
                                                                N.grad + N.ob2);
  k_nn_conv_bwd_data<<<N.nring, NN_THREADS, sizeof(float) * H * H * K, s>>>(
      N.rings, N.g2, H, N.par + N.oW2, H, K, N.bf16, N.h1, np, N.g1);
  // layer 1 (3 -> H, ReLU; no gradient into the inputs)
  k_nn_conv_wgrad<<<dim3(H * 4, NN_CHUNKS), NN_THREADS, 0, s>>>(N.rings, N.nring, N.g1, N.in,
                                                              3, K, np, wp);
  k_nn_wgrad_reduce<<<(H * 3 * K + H + 127) / 128, 128, 0, s>>>(wp, H, 3, K, N.grad + N.oW1,
                                                                N.grad + N.ob1);
  WF_CUDA(cudaGetLastError());
  P.nlaunch += 14;
  N.have_grad = 1;
  return WF_OK;
}

}  // namespace wf

struct wf_net_s : public wf::Net {};

using namespace wf;

extern "C" {

wf_status wf_net_create(wf_net_t *out, wf_plan_t plan, int channels, int kernel, int hidden,
                        int bf16) {
  if (!out || !plan) {
    set_error("wf_net_create: NULL argument");
    return WF_ERR_ARG;
  }
  *out = nullptr;
  if (channels < 1 || channels > NN_MAXC || kernel < 1 || kernel > NN_MAXK ||
      (kernel & 1) == 0 || hidden < 1 || hidden > NN_MAXHM) {
    set_error("wf_net_create: channels in [1, 32], odd kernel in [1, 15], hidden in [1, 64]");
    return WF_ERR_ARG;
  }
  if (!plan->has_noise) {
    set_error("wf_net_create: the plan needs noise and mask");
    return WF_ERR_STATE;
  }
  {
    const int big = 100 * 1024;
    WF_CUDA(cudaFuncSetAttribute(k_nn_conv_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 big));
    WF_CUDA(cudaFuncSetAttribute(k_nn_conv_bwd_data,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  }
  wf_net_s *N = new wf_net_s();
  N->P = plan;
  N->H = channels;
  N->K = kernel;
  N->Hm = hidden;
  N->bf16 = bf16 ? 1 : 0;
  wf_status s = net_alloc(*N);
  if (s != WF_OK) {
    free_net_buffers(N);
    delete N;
    return s;
  }
  *out = N;
  return WF_OK;
}

long wf_net_num_params(wf_net_t net) { return net ? net->npar : 0; }

wf_status wf_net_set_params(wf_net_t net, const float *host, long n) {
  if (!net || !host || n != net->npar) {
    set_error("wf_net_set_params: wrong size or NULL");
    return WF_ERR_ARG;
  }
  WF_CUDA(cudaMemcpy(net->par, host, sizeof(float) * n, cudaMemcpyHostToDevice));
  WF_CUDA(cudaMemset(net->am, 0, sizeof(float) * n));
  WF_CUDA(cudaMemset(net->av, 0, sizeof(float) * n));
  net->step = 0;
  return WF_OK;
}

wf_status wf_net_get_params(wf_net_t net, float *host, long n) {
  if (!net || !host || n != net->npar) {
    set_error("wf_net_get_params: wrong size or NULL");
    return WF_ERR_ARG;
  }
  WF_CUDA(cudaMemcpy(host, net->par, sizeof(float) * n, cudaMemcpyDeviceToHost));
  return WF_OK;
}

wf_status wf_net_forward(wf_net_t net, const double *d_dev, double *t0_dev,
                         double *alm0_dev) {
  if (!net || !d_dev) {
    set_error("wf_net_forward: NULL argument");
    return WF_ERR_ARG;
  }
  Plan &P = *net->P;
  WF_TRY(net_forward(*net, d_dev));
  if (t0_dev)
    WF_CUDA(cudaMemcpyAsync(t0_dev, net->t0, sizeof(double) * P.npix,
                            cudaMemcpyDeviceToDevice, P.stream));
  if (alm0_dev)
    WF_CUDA(cudaMemcpyAsync(alm0_dev, net->a0, sizeof(double2) * P.nalm,
                            cudaMemcpyDeviceToDevice, P.stream));
  WF_CUDA(cudaStreamSynchronize(P.stream));
  return WF_OK;
}

wf_status wf_net_loss_grad(wf_net_t net, const double *d_dev, const double *alm_target_dev,
                           double *loss, float *grad_host) {
  if (!net || !d_dev || !alm_target_dev) {
    set_error("wf_net_loss_grad: NULL argument");
    return WF_ERR_ARG;
  }
  WF_TRY(net_loss_grad(*net, d_dev, reinterpret_cast<const double2 *>(alm_target_dev), loss));
  if (grad_host)
    WF_CUDA(cudaMemcpyAsync(grad_host, net->grad, sizeof(float) * net->npar,
                            cudaMemcpyDeviceToHost, net->P->stream));
  WF_CUDA(cudaStreamSynchronize(net->P->stream));
  return WF_OK;
}

wf_status wf_net_adam_step(wf_net_t net, float lr, float beta1, float beta2, float eps) {
  if (!net || !net->have_grad) {
    set_error("wf_net_adam_step: no gradient (call wf_net_loss_grad first)");
    return WF_ERR_STATE;
  }
  net->step += 1;
  const float c1 = 1.f - powf(beta1, (float)net->step);
  const float c2 = 1.f - powf(beta2, (float)net->step);
  k_nn_adam<<<64, 256, 0, net->P->stream>>>(net->par, net->grad, net->am, net->av, net->npar,
                                            lr, beta1, beta2, eps, c1, c2);
  WF_CUDA(cudaGetLastError());
  net->P->nlaunch += 1;
  WF_CUDA(cudaStreamSynchronize(net->P->stream));
  return WF_OK;
}

void wf_net_destroy(wf_net_t net) {
  if (!net) return;
  free_net_buffers(net);
  delete net;
}

}  // extern "C"
