// Learned per-band choice of alpha.
//
// The paper picks one alpha for the whole spectrum by the discrepancy principle (Sec. 4).  The
// learned rule maps per-band statistics of the data to one alpha per radial band of frequencies:
//   features   f_b = log10( sum_{k in b} sum_planes |U~_k|^2 / (count_b delta^2) ): the data power per
//              frequency of band b over that of white noise of total norm delta (the unnormalised
//              spectrum of such noise has expected power delta^2 per frequency, summed over planes);
//   network    y = W3 tanh(W2 tanh(W1 x + b1) + b2) + b3 with x = f / 4 and y_b = (log10 alpha_b + 4.5) / 3.5;
//              weights in BF16 for the forward and backward kernels, FP32 master copy and Adam state;
//   targets    for data made from a known zeta, the candidate alpha that minimises the error of zeta~ in
//              each band; for M = 1 the Tikhonov solution of a frequency of class c is zeta~ = d a U~ with
//              d = 1 / (n_c + alpha s^2), n_c = ||a||^2 (a real), so
//              E_b(alpha) = sum_{c in b} [ n_c P_c d^2 - 2 d X_c + Z_c ]
//              with P_c = sum wt |U~|^2, X_c = sum wt Re(conj(U~) a^T zeta~_true), Z_c = sum wt ||zeta~_true||^2.
// Inside fr3d_invert (FR3D_ALPHA_LEARNED) the rule is one kernel in place of the alpha sweep: band
// power sums (deterministic block partials, the last block finishes), features, network, nearest
// candidate per band, all in FP32.
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <new>
#include <vector>

#include "ops.cuh"

namespace fr3d {

struct Mlp {
  int nin = 0, nh = 0, nout = 0, np = 0;
  float* master = nullptr;          // [np] FP32 parameters
  __nv_bfloat16* w = nullptr;       // [np] BF16 copy used by the kernels
  float* m = nullptr;               // Adam first moment
  float* v = nullptr;               // Adam second moment
  float* grad = nullptr;            // [np]
  float* acts = nullptr;            // [cap][2 nh + nout] activations of the last batch
  float* dh = nullptr;              // [cap][2 nh + nout] backward scratch
  int cap = 0;
  int step = 0;
};

}  // namespace fr3d

struct fr3d_mlp {
  fr3d::Mlp m;
};

namespace fr3d {

namespace {

// parameter offsets: W1 [nh][nin], b1 [nh], W2 [nh][nh], b2 [nh], W3 [nout][nh], b3 [nout]
struct Off {
  int w1, b1, w2, b2, w3, b3, np;
};
__host__ __device__ inline Off offsets(int nin, int nh, int nout) {
  Off o;
  o.w1 = 0;
  o.b1 = o.w1 + nh * nin;
  o.w2 = o.b1 + nh;
  o.b2 = o.w2 + nh * nh;
  o.w3 = o.b2 + nh;
  o.b3 = o.w3 + nout * nh;
  o.np = o.b3 + nout;
  return o;
}

constexpr float kFeatScale = 0.25f;   // x = f / 4
constexpr float kLogShift = 4.5f;     // y = (log10 alpha + 4.5) / 3.5
constexpr float kLogScale = 3.5f;
constexpr int kMaxHidden = 96;        // widest hidden layer of a network
constexpr int kMaxParams = FR3D_MAX_BANDS * kMaxHidden * 2 + kMaxHidden * kMaxHidden + 2 * kMaxHidden + FR3D_MAX_BANDS;
constexpr int kLearnedThreads = 256;

__device__ inline float bf(const __nv_bfloat16* w, int i) { return __bfloat162float(w[i]); }

// ------------------------------------------------------------------ network kernels
// one dense layer for a batch: out[s][u] = act(b[u] + sum_i W[u][i] in[s][i]); thread per (s, u)
__global__ void k_dense(const __nv_bfloat16* __restrict__ w, int wo, int bo, const float* __restrict__ in, int ldi,
                        int nin, float* __restrict__ out, int ldo, int nout, int B, int act) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B * nout) return;
  const int s = t / nout, u = t % nout;
  float acc = bf(w, bo + u);
  for (int i = 0; i < nin; ++i) acc = fmaf(bf(w, wo + u * nin + i), in[s * ldi + i], acc);
  out[s * ldo + u] = act ? tanhf(acc) : acc;
}

// dy = 2 (y - t) / (B nout) and the mean squared error, one block of 256 threads
__global__ void k_mse(const float* __restrict__ y, int ldy, const float* __restrict__ t, int nout, int B,
                      float* __restrict__ dy, int lddy, float* __restrict__ loss) {
  __shared__ float red[256];
  float s = 0.f;
  for (int e = threadIdx.x; e < B * nout; e += blockDim.x) {
    const int b = e / nout, o = e % nout;
    const float d = y[b * ldy + o] - t[e];
    dy[b * lddy + o] = 2.f * d / (float)(B * nout);
    s = fmaf(d, d, s);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if ((int)threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0 && loss) *loss = red[0] / (float)(B * nout);
}

// weight gradient of a layer: g[wo + u nin + i] = sum_s dout[s][u] in[s][i]; g[bo + u] = sum_s dout[s][u]
__global__ void k_wgrad(const float* __restrict__ dout, int ldd, const float* __restrict__ in, int ldi, int nin,
                        int nout, int B, float* __restrict__ g, int wo, int bo) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nout * (nin + 1)) return;
  const int u = t / (nin + 1), i = t % (nin + 1);
  float acc = 0.f;
  if (i < nin) {
    for (int s = 0; s < B; ++s) acc = fmaf(dout[s * ldd + u], in[s * ldi + i], acc);
    g[wo + u * nin + i] = acc;
  } else {
    for (int s = 0; s < B; ++s) acc += dout[s * ldd + u];
    g[bo + u] = acc;
  }
}

// input gradient through a tanh layer: din[s][i] = (1 - h[s][i]^2) sum_u dout[s][u] W[u][i]
__global__ void k_dgrad(const __nv_bfloat16* __restrict__ w, int wo, const float* __restrict__ dout, int ldd,
                        int nout, const float* __restrict__ h, int ldh, int nin, int B, float* __restrict__ din,
                        int lddi) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B * nin) return;
  const int s = t / nin, i = t % nin;
  float acc = 0.f;
  for (int u = 0; u < nout; ++u) acc = fmaf(dout[s * ldd + u], bf(w, wo + u * nin + i), acc);
  const float hv = h[s * ldh + i];
  din[s * lddi + i] = acc * (1.f - hv * hv);
}

// Adam (Kingma & Ba 2015), beta1 0.9, beta2 0.999, eps 1e-8; b1c, b2c = bias corrections of this step
__global__ void k_adam(float* __restrict__ master, __nv_bfloat16* __restrict__ w, float* __restrict__ m,
                       float* __restrict__ v, const float* __restrict__ g, int np, float lr, float b1c, float b2c) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= np) return;
  const float gi = g[t];
  const float mi = 0.9f * m[t] + 0.1f * gi;
  const float vi = 0.999f * v[t] + 0.001f * gi * gi;
  m[t] = mi;
  v[t] = vi;
  const float p = master[t] - lr * (mi / b1c) / (sqrtf(vi / b2c) + 1e-8f);
  master[t] = p;
  w[t] = __float2bfloat16(p);
}

__global__ void k_to_bf16(const float* __restrict__ a, __nv_bfloat16* __restrict__ b, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) b[t] = __float2bfloat16(a[t]);
}

int forward_batch(Mlp& M, const float* X, int B, cudaStream_t st) {
  const Off o = offsets(M.nin, M.nh, M.nout);
  const int ld = 2 * M.nh + M.nout;
  float* h1 = M.acts;
  float* h2 = M.acts + M.nh;
  float* y = M.acts + 2 * M.nh;
  k_dense<<<(B * M.nh + 127) / 128, 128, 0, st>>>(M.w, o.w1, o.b1, X, M.nin, M.nin, h1, ld, M.nh, B, 1);
  k_dense<<<(B * M.nh + 127) / 128, 128, 0, st>>>(M.w, o.w2, o.b2, h1, ld, M.nh, h2, ld, M.nh, B, 1);
  k_dense<<<(B * M.nout + 127) / 128, 128, 0, st>>>(M.w, o.w3, o.b3, h2, ld, M.nh, y, ld, M.nout, B, 0);
  FR3D_CUDA_TRY(cudaGetLastError());
  return FR3D_OK;
}

int ensure_cap(Mlp& M, int B) {
  if (B <= M.cap) return FR3D_OK;
  if (M.acts) cudaFree(M.acts);
  if (M.dh) cudaFree(M.dh);
  M.acts = M.dh = nullptr;
  M.cap = 0;
  const size_t per = (size_t)(2 * M.nh + M.nout);
  FR3D_CUDA_TRY(cudaMalloc(&M.acts, sizeof(float) * per * B));
  FR3D_CUDA_TRY(cudaMalloc(&M.dh, sizeof(float) * per * B));
  M.cap = B;
  return FR3D_OK;
}

int gradient(Mlp& M, const float* X, const float* T, int B, float* loss, cudaStream_t st) {
  FR3D_TRY(forward_batch(M, X, B, st));
  const Off o = offsets(M.nin, M.nh, M.nout);
  const int ld = 2 * M.nh + M.nout;
  float* h1 = M.acts;
  float* h2 = M.acts + M.nh;
  float* y = M.acts + 2 * M.nh;
  float* d1 = M.dh;
  float* d2 = M.dh + M.nh;
  float* dy = M.dh + 2 * M.nh;
  k_mse<<<1, 256, 0, st>>>(y, ld, T, M.nout, B, dy, ld, loss);
  k_wgrad<<<(M.nout * (M.nh + 1) + 127) / 128, 128, 0, st>>>(dy, ld, h2, ld, M.nh, M.nout, B, M.grad, o.w3, o.b3);
  k_dgrad<<<(B * M.nh + 127) / 128, 128, 0, st>>>(M.w, o.w3, dy, ld, M.nout, h2, ld, M.nh, B, d2, ld);
  k_wgrad<<<(M.nh * (M.nh + 1) + 127) / 128, 128, 0, st>>>(d2, ld, h1, ld, M.nh, M.nh, B, M.grad, o.w2, o.b2);
  k_dgrad<<<(B * M.nh + 127) / 128, 128, 0, st>>>(M.w, o.w2, d2, ld, M.nh, h1, ld, M.nh, B, d1, ld);
  k_wgrad<<<(M.nh * (M.nin + 1) + 127) / 128, 128, 0, st>>>(d1, ld, X, M.nin, M.nin, M.nh, B, M.grad, o.w1, o.b1);
  FR3D_CUDA_TRY(cudaGetLastError());
  return FR3D_OK;
}

// SplitMix64 (Steele, Lea & Flood 2014): the generator of the seeded initial weights
uint64_t splitmix64(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// ------------------------------------------------------------------ band statistics
struct BandConst {
  float lc[FR3D_MAX_BANDS];       // log10(count_b delta^2), formed on the host in FP64
};
struct AlphaLog {
  float lg[FR3D_MAX_ALPHAS];      // log10 of the candidates
};

// band of the half-spectrum bin (kx, ky)
__device__ __forceinline__ int bin_band(const unsigned char* __restrict__ cband, int nb, int kx, int ky, int n) {
  return nb > 1 ? (int)__ldg(cband + class_of(kx, ky, n)) : 0;
}

// sum over the block's threads of red[b][t] for every band b < nb, into tot[b] (fixed order: a
// butterfly within each warp, then the warp totals in warp order); ends with a barrier
__device__ void block_band_sum(float (*red)[kLearnedThreads], float (*wsum)[kLearnedThreads / 32], int nb,
                               float* tot, int tid) {
  const int warp = tid >> 5, lane = tid & 31;
  __syncthreads();
  for (int b = 0; b < nb; ++b) {
    float v = red[b][tid];
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
    if (lane == 0) wsum[b][warp] = v;
  }
  __syncthreads();
  if (tid < nb) {
    float s = 0.f;
#pragma unroll
    for (int w = 0; w < kLearnedThreads / 32; ++w) s += wsum[tid][w];
    tot[tid] = s;
  }
  __syncthreads();
}

// largest power of two <= v (v >= 1), capped at 32: lanes that share one output of a layer
__device__ __forceinline__ int lanes_per_output(int v) {
  int g = 1;
  while (g * 2 <= v && g < 32) g *= 2;
  return g;
}

// out[u] = act(b[u] + sum_i W[u][i] in[i]) for u < nout with G = lanes_per_output(256 / nout) adjacent
// lanes per output (a butterfly over the G lanes finishes each sum); every thread reaches the barrier
__device__ void dense_layer(const __nv_bfloat16* w, int wo, int bo, const float* in, int nin, float* out, int nout,
                            bool act, int tid) {
  const int G = lanes_per_output(kLearnedThreads / nout);
  const int u = tid / G, g = tid % G;
  float a = 0.f;
  if (u < nout)
    for (int i = g; i < nin; i += G) a = fmaf(bf(w, wo + u * nin + i), in[i], a);
  for (int m = G / 2; m > 0; m >>= 1) a += __shfl_xor_sync(0xffffffffu, a, m);
  if (u < nout && g == 0) {
    a += bf(w, bo + u);
    out[u] = act ? tanhf(a) : a;
  }
  __syncthreads();
}

// Band power sums of the half spectrum Uh (nplanes planes of (n/2+1) x n bins, weights 1 on the kx = 0
// and kx = n/2 rows, 2 elsewhere), block partials, and in the last block: the network input x_b = f_b / 4
// (to feat, if given), and with a network the per-band candidate indices.  info (if given) receives
// FR3D_INFO_NONFINITE and FR3D_INFO_LEARNED_OUT_OF_RANGE bits.
// Everything is FP32: every sum is pairwise (a few bins per thread, then butterflies over lanes, warps
// and blocks), so its relative error stays near 1e-6, far below what a log10 feature resolves, and the
// serial tail of the last block runs on the FP32 pipe (FP64 is a small fraction of it on this GPU).
__global__ void __launch_bounds__(kLearnedThreads) k_learned_alpha(
    const float4* __restrict__ Uh4, int n4, int ps2, int n, const unsigned char* __restrict__ cband, int nb,
    BandConst bc, float* __restrict__ partials, unsigned* __restrict__ counter, float* __restrict__ feat,
    const __nv_bfloat16* __restrict__ w, int nh, AlphaLog al, int na, int* __restrict__ aidx,
    int* __restrict__ info) {
  __shared__ __align__(16) union {
    float red[FR3D_MAX_BANDS][kLearnedThreads];
    __nv_bfloat16 w[kMaxParams];
    uint4 w16[(kMaxParams + 7) / 8];
  } sm;
  __shared__ float wsum[FR3D_MAX_BANDS][kLearnedThreads / 32];
  __shared__ float tot[FR3D_MAX_BANDS], x[FR3D_MAX_BANDS], h1[kMaxHidden], h2[kMaxHidden], y[FR3D_MAX_BANDS];
  __shared__ int flags;
  __shared__ bool last;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int b = 0; b < nb; ++b) sm.red[b][tid] = 0.f;
  for (int e4 = blockIdx.x * kLearnedThreads + tid; e4 < n4; e4 += gridDim.x * kLearnedThreads) {
    const float4 u = __ldg(Uh4 + e4);
    const int e = (e4 % ps2) * 2;                 // bin of u.x, u.y; u.z, u.w is bin e + 1 (same row)
    const int kx = e / n, ky = e % n;
    const float wt = (kx == 0 || 2 * kx == n) ? 1.f : 2.f;
    sm.red[bin_band(cband, nb, kx, ky, n)][tid] += wt * fmaf(u.x, u.x, u.y * u.y);
    sm.red[bin_band(cband, nb, kx, ky + 1, n)][tid] += wt * fmaf(u.z, u.z, u.w * u.w);
  }
  block_band_sum(sm.red, wsum, nb, tot, tid);
  if (tid < nb) partials[blockIdx.x * nb + tid] = tot[tid];
  __threadfence();
  __syncthreads();
  if (tid == 0) last = atomicAdd(counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  // every other block has finished: let a programmatically launched successor start its set-up
  pdl_release();
  {
    // the partials of blocks tid and tid + 256 (the grid has at most 2 * 256 blocks), all loads in flight
    float v0[FR3D_MAX_BANDS], v1[FR3D_MAX_BANDS];
    const int g = (int)gridDim.x;
#pragma unroll
    for (int b = 0; b < FR3D_MAX_BANDS; ++b) {
      v0[b] = (b < nb && tid < g) ? __ldcg(partials + tid * nb + b) : 0.f;
      v1[b] = (b < nb && tid + kLearnedThreads < g) ? __ldcg(partials + (tid + kLearnedThreads) * nb + b) : 0.f;
    }
#pragma unroll
    for (int b = 0; b < FR3D_MAX_BANDS; ++b)
      if (b < nb) sm.red[b][tid] = v0[b] + v1[b];
  }
  if (tid == 0) flags = 0;
  block_band_sum(sm.red, wsum, nb, tot, tid);
  if (tid < nb) {
    const float s = tot[tid];
    if (!isfinite(s)) atomicOr(&flags, FR3D_INFO_NONFINITE);
    x[tid] = (log10f(fmaxf(s, 1e-37f)) - bc.lc[tid]) * kFeatScale;
    if (feat) feat[tid] = x[tid];
  }
  if (tid == 0) *counter = 0u;
  __syncthreads();
  if (!w) {
    if (tid == 0 && info) *info = flags;
    return;
  }
  // network: weights staged in shared memory (over the reduction buffer), then three layers
  const Off o = offsets(nb, nh, nb);
  {
    // 16-byte pieces, all loads of a thread in flight before the stores (the allocation is 256-byte
    // aligned; the last partial piece is copied element by element)
    constexpr int kPer = ((kMaxParams + 7) / 8 + kLearnedThreads - 1) / kLearnedThreads;
    const int n16 = o.np / 8;
    const uint4* w16 = reinterpret_cast<const uint4*>(w);
    uint4 v[kPer];
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
      const int e = tid + i * kLearnedThreads;
      if (e < n16) v[i] = __ldg(w16 + e);
    }
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
      const int e = tid + i * kLearnedThreads;
      if (e < n16) sm.w16[e] = v[i];
    }
    for (int i = n16 * 8 + tid; i < o.np; i += kLearnedThreads) sm.w[i] = w[i];
  }
  __syncthreads();
  dense_layer(sm.w, o.w1, o.b1, x, nb, h1, nh, true, tid);
  dense_layer(sm.w, o.w2, o.b2, h1, nh, h2, nh, true, tid);
  dense_layer(sm.w, o.w3, o.b3, h2, nh, y, nb, false, tid);
  // nearest candidate in log10 alpha, one warp per band (ties: the smaller index)
  for (int b = warp; b < nb; b += kLearnedThreads / 32) {
    const float la = y[b] * kLogScale - kLogShift;
    float bd = 3.4e38f;
    int best = 0x7fffffff;
    for (int k = lane; k < na; k += 32) {
      const float d = fabsf(al.lg[k] - la);
      if (d < bd) {
        bd = d;
        best = k;
      }
    }
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) {
      const float od = __shfl_xor_sync(0xffffffffu, bd, m);
      const int ok = __shfl_xor_sync(0xffffffffu, best, m);
      if (od < bd || (od == bd && ok < best)) {
        bd = od;
        best = ok;
      }
    }
    if (lane == 0) {
      aidx[b] = best;
      if (!(la >= al.lg[0] - 0.5f && la <= al.lg[na - 1] + 0.5f)) atomicOr(&flags, FR3D_INFO_LEARNED_OUT_OF_RANGE);
    }
  }
  __syncthreads();
  if (tid == 0 && info) *info = flags;
}

// ------------------------------------------------------------------ training targets
__device__ inline void class_pq_l(int c, int& p, int& q) {
  p = (int)((sqrtf(8.f * (float)c + 1.f) - 1.f) * 0.5f);
  while ((p + 1) * (p + 2) / 2 <= c) ++p;
  while (p * (p + 1) / 2 > c) --p;
  q = c - p * (p + 1) / 2;
}

// Per class c, summed over its members (half-spectrum weights wt) and the Q planes:
//   P_c = sum wt |U~|^2,  X_c = sum wt Re(conj(U~) a^T zeta~_true),  Z_c = sum wt ||zeta~_true||^2,
// with a = A^(c) (FP64 table) and zeta~_true the spectra of the M' planes of each source parameter.
// X is formed in the spectral domain so that strongly attenuated classes (tiny ||a||) carry no
// rounding error from a spatial round trip.
__global__ void k_class_stats(const float2* __restrict__ Uh, const float2* __restrict__ Zh,
                              const double* __restrict__ A64, long ps, int Q, int Mp, int n, int Cn,
                              double* __restrict__ P, double* __restrict__ X, double* __restrict__ Z) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= Cn) return;
  int p, q;
  class_pq_l(c, p, q);
  int kxs[4], kys[4], nm = 0;
  kxs[nm] = p;
  kys[nm++] = q;
  if (q != 0 && 2 * q != n) {
    kxs[nm] = p;
    kys[nm++] = n - q;
  }
  if (p != q) {
    kxs[nm] = q;
    kys[nm++] = p;
    if (p != 0 && 2 * p != n) {
      kxs[nm] = q;
      kys[nm++] = n - p;
    }
  }
  const double* a = A64 + (long)c * Mp;
  double sp = 0.0, sx = 0.0, sz = 0.0;
  for (int mi = 0; mi < nm; ++mi) {
    const double wt = (kxs[mi] == 0 || 2 * kxs[mi] == n) ? 1.0 : 2.0;
    const long o = (long)kxs[mi] * n + kys[mi];
    for (int pl = 0; pl < Q; ++pl) {
      const float2 u = __ldg(Uh + pl * ps + o);
      double cr = 0.0, ci = 0.0, zz = 0.0;
      for (int j = 0; j < Mp; ++j) {
        const float2 z = __ldg(Zh + ((long)pl * Mp + j) * ps + o);
        cr += a[j] * z.x;
        ci += a[j] * z.y;
        zz += (double)z.x * z.x + (double)z.y * z.y;
      }
      sp += wt * ((double)u.x * u.x + (double)u.y * u.y);
      sx += wt * (u.x * cr + u.y * ci);
      sz += wt * zz;
    }
  }
  P[c] = sp;
  X[c] = sx;
  Z[c] = sz;
}

struct AlphaVal {
  double a[FR3D_MAX_ALPHAS];
};

// block partials of E_b(alpha_k) over a chunk of classes; thread per candidate
__global__ void k_band_err_partial(const double* __restrict__ P, const double* __restrict__ X,
                                   const double* __restrict__ Z, const double* __restrict__ nrm,
                                   const double* __restrict__ s2,
                                   const unsigned char* __restrict__ cband, int Cn, int nb, int chunk, AlphaVal av,
                                   int na, double* __restrict__ partials) {
  const int k = threadIdx.x;
  if (k >= na) return;
  double acc[FR3D_MAX_BANDS];
  for (int b = 0; b < nb; ++b) acc[b] = 0.0;
  const double as2 = av.a[k] * (*s2);
  const int c1 = min(Cn, (int)(blockIdx.x + 1) * chunk);
  for (int c = blockIdx.x * chunk; c < c1; ++c) {
    const int b = nb > 1 ? (int)cband[c] : 0;
    const double d = 1.0 / (nrm[c] + as2);
    acc[b] += nrm[c] * P[c] * d * d - 2.0 * d * X[c] + Z[c];
  }
  for (int b = 0; b < nb; ++b) partials[((long)blockIdx.x * nb + b) * na + k] = acc[b];
}

__global__ void k_band_err_finish(const double* __restrict__ partials, int nblk, int nb, AlphaVal av, int na,
                                  double* __restrict__ err, int* __restrict__ idx, float* __restrict__ target) {
  __shared__ double E[FR3D_MAX_BANDS][FR3D_MAX_ALPHAS];
  const int k = threadIdx.x;
  if (k < na)
    for (int b = 0; b < nb; ++b) {
      double s = 0.0;
      for (int blk = 0; blk < nblk; ++blk) s += partials[((long)blk * nb + b) * na + k];
      E[b][k] = s;
      if (err) err[b * na + k] = s;
    }
  __syncthreads();
  if (k < nb) {
    int best = 0;
    for (int j = 1; j < na; ++j)
      if (E[k][j] < E[k][best]) best = j;
    idx[k] = best;
    if (target) target[k] = (float)((log10(av.a[best]) + kLogShift) / kLogScale);
  }
}

// data spectrum of U (FP32, [Q][1][n][n]) into Uh (half spectrum, Q planes)
int spectrum(Handle* H, const float* U, int Q, float2* Uh, cudaStream_t st) {
  FR3D_TRY(Ops<float>::row_r2c(H, U, (long)H->n * H->n, Uh, Q, st));
  FR3D_TRY(Ops<float>::col_plain(H, Uh, Uh, Q, false, st));
  return FR3D_OK;
}

}  // namespace

bool learned_net_fits(const fr3d_mlp* net, int nb) {
  return net && net->m.nin == nb && net->m.nout == nb && net->m.nh <= kMaxHidden;
}

int learned_alpha(Handle* H, const float2* Uh, int nplanes, int nb, double delta, const double* alphas, int na,
                  const fr3d_mlp* net, int* aidx, float* feat, int* info, cudaStream_t st) {
  std::vector<double> count;
  FR3D_TRY(ensure_bands(H, nb, &count));
  FR3D_TRY(ensure_partials(H));
  BandConst bc;
  for (int b = 0; b < nb; ++b) bc.lc[b] = (float)log10(count[b] * delta * delta);
  AlphaLog al;
  for (int k = 0; k < na; ++k) al.lg[k] = (float)log10(alphas[k]);
  const long ps2 = (long)(H->n / 2 + 1) * H->n / 2;
  const long n4 = ps2 * nplanes;
  if (n4 > 0x7fffffffL) return FR3D_ERR_UNSUPPORTED_SIZE;
  long blocks = (n4 + 2 * kLearnedThreads - 1) / (2 * kLearnedThreads);
  blocks = std::max(1L, std::min(blocks, 2L * 152));   // at most 2 * kLearnedThreads (the last block's loads)
  k_learned_alpha<<<(int)blocks, kLearnedThreads, 0, st>>>(
      reinterpret_cast<const float4*>(Uh), (int)n4, (int)ps2, H->n, H->cband, nb, bc,
      reinterpret_cast<float*>(H->partials), H->counter, feat, net ? net->m.w : nullptr, net ? net->m.nh : 0, al,
      na, aidx, info);
  FR3D_CUDA_TRY(cudaGetLastError());
  return FR3D_OK;
}

}  // namespace fr3d

using fr3d::Mlp;

extern "C" int fr3d_mlp_create(int n_in, int n_hidden, int n_out, unsigned long long seed, fr3d_mlp** out) {
  if (!out) return FR3D_ERR_INVALID_ARG;
  *out = nullptr;
  if (n_in < 1 || n_in > FR3D_MAX_BANDS || n_out < 1 || n_out > FR3D_MAX_BANDS || n_hidden < 1 ||
      n_hidden > fr3d::kMaxHidden)
    return FR3D_ERR_INVALID_ARG;
  fr3d_mlp* h = new (std::nothrow) fr3d_mlp();
  if (!h) return FR3D_ERR_OOM;
  Mlp& M = h->m;
  M.nin = n_in;
  M.nh = n_hidden;
  M.nout = n_out;
  const fr3d::Off o = fr3d::offsets(n_in, n_hidden, n_out);
  M.np = o.np;
  // Glorot-uniform weights, zero biases
  std::vector<float> p(M.np, 0.f);
  uint64_t s = seed;
  auto uni = [&](double lim) { return (float)(((double)(fr3d::splitmix64(s) >> 11) * 0x1.0p-53 * 2.0 - 1.0) * lim); };
  for (int i = 0; i < n_hidden * n_in; ++i) p[o.w1 + i] = uni(sqrt(6.0 / (n_in + n_hidden)));
  for (int i = 0; i < n_hidden * n_hidden; ++i) p[o.w2 + i] = uni(sqrt(6.0 / (2 * n_hidden)));
  for (int i = 0; i < n_out * n_hidden; ++i) p[o.w3 + i] = uni(sqrt(6.0 / (n_hidden + n_out)));
  cudaError_t e = cudaMalloc(&M.master, sizeof(float) * M.np);
  if (e == cudaSuccess) e = cudaMalloc(&M.w, sizeof(__nv_bfloat16) * M.np);
  if (e == cudaSuccess) e = cudaMalloc(&M.m, sizeof(float) * M.np);
  if (e == cudaSuccess) e = cudaMalloc(&M.v, sizeof(float) * M.np);
  if (e == cudaSuccess) e = cudaMalloc(&M.grad, sizeof(float) * M.np);
  if (e == cudaSuccess) e = cudaMemcpy(M.master, p.data(), sizeof(float) * M.np, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(M.m, 0, sizeof(float) * M.np);
  if (e == cudaSuccess) e = cudaMemset(M.v, 0, sizeof(float) * M.np);
  if (e == cudaSuccess) {
    fr3d::k_to_bf16<<<(M.np + 255) / 256, 256>>>(M.master, M.w, M.np);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    fr3d_mlp_destroy(h);
    return e == cudaErrorMemoryAllocation ? FR3D_ERR_OOM : FR3D_ERR_CUDA;
  }
  *out = h;
  return FR3D_OK;
}

extern "C" void fr3d_mlp_destroy(fr3d_mlp* h) {
  if (!h) return;
  cudaDeviceSynchronize();
  Mlp& M = h->m;
  void* ps[] = {M.master, M.w, M.m, M.v, M.grad, M.acts, M.dh};
  for (void* p : ps)
    if (p) cudaFree(p);
  delete h;
}

extern "C" int fr3d_mlp_query(const fr3d_mlp* h, int* n_in, int* n_hidden, int* n_out, int* n_params) {
  if (!h) return FR3D_ERR_INVALID_ARG;
  if (n_in) *n_in = h->m.nin;
  if (n_hidden) *n_hidden = h->m.nh;
  if (n_out) *n_out = h->m.nout;
  if (n_params) *n_params = h->m.np;
  return FR3D_OK;
}

extern "C" int fr3d_mlp_get_params(fr3d_mlp* h, float* host) {
  if (!h || !host) return FR3D_ERR_INVALID_ARG;
  FR3D_CUDA_TRY(cudaDeviceSynchronize());
  FR3D_CUDA_TRY(cudaMemcpy(host, h->m.master, sizeof(float) * h->m.np, cudaMemcpyDeviceToHost));
  return FR3D_OK;
}

extern "C" int fr3d_mlp_set_params(fr3d_mlp* h, const float* host) {
  if (!h || !host) return FR3D_ERR_INVALID_ARG;
  Mlp& M = h->m;
  FR3D_CUDA_TRY(cudaDeviceSynchronize());
  FR3D_CUDA_TRY(cudaMemcpy(M.master, host, sizeof(float) * M.np, cudaMemcpyHostToDevice));
  FR3D_CUDA_TRY(cudaMemset(M.m, 0, sizeof(float) * M.np));
  FR3D_CUDA_TRY(cudaMemset(M.v, 0, sizeof(float) * M.np));
  M.step = 0;
  fr3d::k_to_bf16<<<(M.np + 255) / 256, 256>>>(M.master, M.w, M.np);
  FR3D_CUDA_TRY(cudaGetLastError());
  FR3D_CUDA_TRY(cudaDeviceSynchronize());
  return FR3D_OK;
}

extern "C" int fr3d_mlp_forward(fr3d_mlp* h, const float* X, int B, float* Y, void* stream) {
  if (!h || !X || !Y || B < 1) return FR3D_ERR_INVALID_ARG;
  Mlp& M = h->m;
  FR3D_TRY(fr3d::ensure_cap(M, B));
  cudaStream_t st = (cudaStream_t)stream;
  FR3D_TRY(fr3d::forward_batch(M, X, B, st));
  FR3D_CUDA_TRY(cudaMemcpy2DAsync(Y, sizeof(float) * M.nout, M.acts + 2 * M.nh, sizeof(float) * (2 * M.nh + M.nout),
                                  sizeof(float) * M.nout, B, cudaMemcpyDeviceToDevice, st));
  return FR3D_OK;
}

extern "C" int fr3d_mlp_gradient(fr3d_mlp* h, const float* X, const float* T, int B, float* grad, float* loss,
                                 void* stream) {
  if (!h || !X || !T || B < 1) return FR3D_ERR_INVALID_ARG;
  Mlp& M = h->m;
  FR3D_TRY(fr3d::ensure_cap(M, B));
  cudaStream_t st = (cudaStream_t)stream;
  FR3D_TRY(fr3d::gradient(M, X, T, B, loss, st));
  if (grad) FR3D_CUDA_TRY(cudaMemcpyAsync(grad, M.grad, sizeof(float) * M.np, cudaMemcpyDeviceToDevice, st));
  return FR3D_OK;
}

extern "C" int fr3d_mlp_train_step(fr3d_mlp* h, const float* X, const float* T, int B, float lr, float* loss,
                                   void* stream) {
  if (!h || !X || !T || B < 1 || !(lr > 0.f) || !isfinite(lr)) return FR3D_ERR_INVALID_ARG;
  Mlp& M = h->m;
  FR3D_TRY(fr3d::ensure_cap(M, B));
  cudaStream_t st = (cudaStream_t)stream;
  FR3D_TRY(fr3d::gradient(M, X, T, B, loss, st));
  ++M.step;
  const float b1c = (float)(1.0 - pow(0.9, (double)M.step));
  const float b2c = (float)(1.0 - pow(0.999, (double)M.step));
  fr3d::k_adam<<<(M.np + 255) / 256, 256, 0, st>>>(M.master, M.w, M.m, M.v, M.grad, M.np, lr, b1c, b2c);
  FR3D_CUDA_TRY(cudaGetLastError());
  return FR3D_OK;
}

extern "C" int fr3d_band_features(fr3d_handle* h, const float* U, int Q, int n_bands, double delta, float* feat,
                                  void* stream) {
  if (!h || !U || Q < 1 || !feat || n_bands < 1 || n_bands > FR3D_MAX_BANDS || !(delta > 0) || !isfinite(delta))
    return FR3D_ERR_INVALID_ARG;
  if (h->padded) return FR3D_ERR_UNSUPPORTED_SIZE;   // periodic box only
  fr3d::Handle* H = &h->h;
  if (H->M != 1) return FR3D_ERR_UNSUPPORTED_SIZE;
  cudaStream_t st = (cudaStream_t)stream;
  const long ps = (long)(H->n / 2 + 1) * H->n;
  FR3D_TRY(fr3d::ensure_ws(H, sizeof(float2) * ps * Q));
  float2* Uh = reinterpret_cast<float2*>(H->ws);
  FR3D_TRY(fr3d::spectrum(H, U, Q, Uh, st));
  const double dummy = 1.0;
  return fr3d::learned_alpha(H, Uh, Q, n_bands, delta, &dummy, 1, nullptr, nullptr, feat, nullptr, st);
}

extern "C" int fr3d_band_alpha_targets(fr3d_handle* h, const float* U, const float* zeta_true, int Q,
                                       const double* alphas, int n_alpha, int n_bands, int* idx, float* target,
                                       double* err, void* stream) {
  if (h && h->padded) return FR3D_ERR_UNSUPPORTED_SIZE;   // periodic box only
  if (!h || !U || !zeta_true || Q < 1 || !alphas || n_alpha < 1 || n_alpha > FR3D_MAX_ALPHAS || n_bands < 1 ||
      n_bands > FR3D_MAX_BANDS || !idx)
    return FR3D_ERR_INVALID_ARG;
  for (int k = 0; k < n_alpha; ++k)
    if (!(alphas[k] > 0) || !isfinite(alphas[k]) || (k > 0 && !(alphas[k] > alphas[k - 1])))
      return FR3D_ERR_INVALID_ARG;
  fr3d::Handle* H = &h->h;
  if (H->M != 1) return FR3D_ERR_UNSUPPORTED_SIZE;
  cudaStream_t st = (cudaStream_t)stream;
  const long ps = (long)(H->n / 2 + 1) * H->n;
  auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t ub = up(sizeof(float2) * ps * Q), zb = up(sizeof(float2) * ps * Q * H->Mp);
  FR3D_TRY(fr3d::ensure_ws(H, ub + zb + 3 * sizeof(double) * H->C));
  float2* Uh = reinterpret_cast<float2*>(H->ws);
  float2* Zh = reinterpret_cast<float2*>((char*)H->ws + ub);
  double* P = reinterpret_cast<double*>((char*)H->ws + ub + zb);
  double* X = P + H->C;
  double* Z = X + H->C;
  FR3D_TRY(fr3d::ensure_bands(H, n_bands, nullptr));
  FR3D_TRY(fr3d::ensure_partials(H));
  FR3D_TRY(fr3d::spectrum(H, U, Q, Uh, st));
  FR3D_TRY(fr3d::spectrum(H, zeta_true, Q * H->Mp, Zh, st));
  fr3d::k_class_stats<<<(H->C + 127) / 128, 128, 0, st>>>(Uh, Zh, H->A64, ps, Q, H->Mp, H->n, H->C, P, X, Z);
  fr3d::AlphaVal av;
  for (int k = 0; k < n_alpha; ++k) av.a[k] = alphas[k];
  const int chunk = 64;
  const int nblk = (H->C + chunk - 1) / chunk;   // ensure_partials holds ceil(C / 64) * 128 * 16 doubles
  fr3d::k_band_err_partial<<<nblk, 128, 0, st>>>(P, X, Z, H->nrm, H->s2, H->cband, H->C, n_bands, chunk, av,
                                                 n_alpha, H->partials);
  fr3d::k_band_err_finish<<<1, 128, 0, st>>>(H->partials, nblk, n_bands, av, n_alpha, err, idx, target);
  FR3D_CUDA_TRY(cudaGetLastError());
  return FR3D_OK;
}
