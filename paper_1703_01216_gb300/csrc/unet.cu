// The learned post-corrector (fr3d_unet_*): a 4-level 3D U-Net of base width 16 that maps the Tikhonov
// reconstruction of Algorithm 1 to a corrected xi, trained and run on the GPU.  The paper has no network;
// the learned part of the benchmark suite asks for one to put back what the normal solution leaves out
// (with one observation plane, M' - 1 depth directions per frequency, Assumption U of Sec. 4).
//
// Network (the FP64 oracle restates it): level 0 conv(1 -> 16), conv(16 -> 16); levels 1, 2: average
// pooling by 2, conv(w_{l-1} -> w_l), conv(w_l -> w_l); level 3 (bottom): pooling, three conv to 128
// channels; going up, nearest upsampling by 2 concatenated with the encoder output of the level,
// conv(w_{l+1} + w_l -> w_l), conv(w_l -> w_l); every conv 3 x 3 x 3 with bias and leaky ReLU (slope 0.01);
// a 1 x 1 x 1 head 16 -> 1 added to the input.  Inputs are scaled by in_scale inside (x_s = in_scale x),
// the prediction is returned in the caller's units; the loss is the batch mean of ||y - t||^2 / ||t||^2.
//
// Storage: FP32 master parameters, gradients and Adam moments; BF16 weight images (forward and input
// gradient, see unet_conv.cu) rebuilt after every update; BF16 activations and activation gradients in
// the padded channel-chunked layout of unet_conv.cu (zero halos and guards, allocated once per network
// for its maximum batch).  Convolutions and their gradients run on the tensor cores (unet_conv.cu); the
// pooling, upsampling, head, loss, reductions and Adam are the CUDA-core kernels below.  Every reduction
// has a fixed order (block partials, then one ordered pass), so results do not depend on the run.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "ops.cuh"
#include "tc.cuh"
#include "unet.cuh"

namespace fr3d {

namespace {

constexpr int kL = 4;
constexpr int kWidth[kL] = {16, 32, 64, 128};
constexpr int kGuard = 128;
constexpr int kNumConv = 15;
constexpr long kWgRange = 4096;   // voxels per weight-gradient CTA

struct Level {
  int D, H, W, Hp, Wp;
  long Vp, Vs, p_first, p_last;
  int ntiles;
};

Level make_level(int D, int H, int W) {
  Level l;
  l.D = D;
  l.H = H;
  l.W = W;
  l.Hp = H + 2;
  l.Wp = W + 2;
  l.Vp = (long)(D + 2) * l.Hp * l.Wp;
  l.Vs = l.Vp + kGuard;
  const long hw = (long)l.Hp * l.Wp;
  l.p_first = hw + l.Wp + 1;
  l.p_last = l.Vp - 1 - (hw + l.Wp + 1);
  l.ntiles = (int)((l.p_last - l.p_first + 128) / 128);
  return l;
}

// tensor ids
enum {
  T_X = 0,
  T_E1 = 1,     // + l (0..2): encoder conv 1 output
  T_CAT = 4,    // + l (0..2): [upsampled w_{l+1} | encoder output w_l]
  T_P = 7,      // + l - 1 (l = 1..3): pooled input of level l
  T_B = 10,     // + 0..2: bottom conv outputs
  T_D1 = 13,    // + l: decoder conv 1 output
  T_D2 = 16,    // + l: decoder conv 2 output
  T_N = 19
};

struct TensorDesc {
  int C = 0, lvl = 0;
};

struct Layer {
  int ci = 0, ci_pad = 0, co = 0, lvl = 0;
  long woff = 0;                  // w [co][ci][27] at woff, b [co] at woff + co ci 27 (flat parameters)
  int in_t = 0, in_off = 0;       // input tensor and channel offset
  int out_t = 0, out_off = 0;
  int dgrad = 0;                  // 0 none, 1 with the leaky derivative of the input, 2 plain
  size_t img_f = 0, img_b = 0;    // byte offsets of the weight images
};

}  // namespace

struct Unet {
  int dev = 0;
  int D = 0, H = 0, W = 0, Bmax = 0;
  float in_scale = 1.f;
  Level lv[kL];
  TensorDesc td[T_N];
  unsigned char* t[T_N] = {};     // activations
  unsigned char* g[T_N] = {};     // activation gradients
  size_t tbytes[T_N] = {};
  Layer layer[kNumConv];
  long n_params = 0;
  long head_off = 0;
  float* params = nullptr;        // FP32 master
  float* grads = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  int adam_t = 0;
  unsigned char* imgs = nullptr;  // BF16 weight images
  size_t img_bytes = 0;
  float* y = nullptr;             // scaled prediction [Bmax][D][H][W]
  float* partials = nullptr;      // weight-gradient partials
  size_t partial_floats = 0;
  float* red = nullptr;           // small reduction buffers
  size_t red_floats = 0;
  double* lossbuf = nullptr;      // [Bmax][2] sums, [1] loss
  int* err = nullptr;
};

namespace {

__device__ __forceinline__ float bfv(uint32_t u, int hi) { return __uint_as_float(hi ? (u & 0xFFFF0000u) : (u << 16)); }
__device__ __forceinline__ uint32_t pk(float a, float b) {
  return (uint32_t)tc::bf16_rn(a) | ((uint32_t)tc::bf16_rn(b) << 16);
}
__device__ __forceinline__ void unpack8(const uint4& q, float* f) {
  const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    f[2 * k] = bfv(w[k], 0);
    f[2 * k + 1] = bfv(w[k], 1);
  }
}
__device__ __forceinline__ uint4 pack8(const float* f) {
  return make_uint4(pk(f[0], f[1]), pk(f[2], f[3]), pk(f[4], f[5]), pk(f[6], f[7]));
}
__device__ __forceinline__ float bf16r(float x) { return tc::bf16_val(tc::bf16_rn(x)); }

struct LevelArg {
  int D, H, W, Hp, Wp;
  long Vs;
};
LevelArg larg(const Level& l) { return LevelArg{l.D, l.H, l.W, l.Hp, l.Wp, l.Vs}; }

__device__ __forceinline__ long ppos(const LevelArg& L, int d, int h, int w) {
  return ((long)(d + 1) * L.Hp + (h + 1)) * L.Wp + (w + 1);
}

// x_s = in_scale x into channel 0 of the input tensor (16 channels, the other 15 stay zero)
__global__ void k_pack_input(const float* __restrict__ x, int B, LevelArg L, float s, unsigned char* __restrict__ X) {
  const long nvox = (long)L.D * L.H * L.W;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < (long)B * nvox; i += (long)gridDim.x * blockDim.x) {
    const int b = (int)(i / nvox);
    long r = i - (long)b * nvox;
    const int w = (int)(r % L.W);
    r /= L.W;
    const int h = (int)(r % L.H), d = (int)(r / L.H);
    float f[8] = {bf16r(s * x[i]), 0, 0, 0, 0, 0, 0, 0};
    *reinterpret_cast<uint4*>(X + (((long)b * 2) * L.Vs + ppos(L, d, h, w)) * 16) = pack8(f);
  }
}

// average pooling by 2: dst (level l+1, chunks [0, nc)) from src (level l, chunks [soff, soff + nc))
__global__ void k_pool(const unsigned char* __restrict__ src, int s_chunks, int soff, LevelArg Ls,
                       unsigned char* __restrict__ dst, int d_chunks, LevelArg Ld, int nc, int B) {
  const long nvox = (long)Ld.D * Ld.H * Ld.W;
  const long total = (long)B * nc * nvox;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    long r = i;
    const int w = (int)(r % Ld.W);
    r /= Ld.W;
    const int h = (int)(r % Ld.H);
    r /= Ld.H;
    const int d = (int)(r % Ld.D);
    r /= Ld.D;
    const int j = (int)(r % nc), b = (int)(r / nc);
    float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const unsigned char* sp = src + ((long)b * s_chunks + soff + j) * Ls.Vs * 16;
    for (int c = 0; c < 8; ++c) {
      float f[8];
      unpack8(*reinterpret_cast<const uint4*>(sp + ppos(Ls, 2 * d + (c >> 2), 2 * h + ((c >> 1) & 1), 2 * w + (c & 1)) * 16), f);
#pragma unroll
      for (int k = 0; k < 8; ++k) acc[k] += f[k];
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] *= 0.125f;
    *reinterpret_cast<uint4*>(dst + (((long)b * d_chunks + j) * Ld.Vs + ppos(Ld, d, h, w)) * 16) = pack8(acc);
  }
}

// nearest upsampling by 2: dst (level l, chunks [0, nc)) from src (level l+1, chunks [0, nc))
__global__ void k_up(const unsigned char* __restrict__ src, int s_chunks, LevelArg Ls, unsigned char* __restrict__ dst,
                     int d_chunks, LevelArg Ld, int nc, int B) {
  const long nvox = (long)Ld.D * Ld.H * Ld.W;
  const long total = (long)B * nc * nvox;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    long r = i;
    const int w = (int)(r % Ld.W);
    r /= Ld.W;
    const int h = (int)(r % Ld.H);
    r /= Ld.H;
    const int d = (int)(r % Ld.D);
    r /= Ld.D;
    const int j = (int)(r % nc), b = (int)(r / nc);
    const uint4 q = *reinterpret_cast<const uint4*>(src + (((long)b * s_chunks + j) * Ls.Vs + ppos(Ls, d / 2, h / 2, w / 2)) * 16);
    *reinterpret_cast<uint4*>(dst + (((long)b * d_chunks + j) * Ld.Vs + ppos(Ld, d, h, w)) * 16) = q;
  }
}

// gradient of the upsampling, times the leaky derivative of the upsampled tensor (its only consumer):
// gs[parent] = bf16(leaky'(s[parent]) * bf16(sum over the 8 children of gd))
__global__ void k_up_backward(const unsigned char* __restrict__ gd, int d_chunks, LevelArg Ld,
                              const unsigned char* __restrict__ s, unsigned char* __restrict__ gs, int s_chunks,
                              LevelArg Ls, int nc, int B) {
  const long nvox = (long)Ls.D * Ls.H * Ls.W;
  const long total = (long)B * nc * nvox;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    long r = i;
    const int w = (int)(r % Ls.W);
    r /= Ls.W;
    const int h = (int)(r % Ls.H);
    r /= Ls.H;
    const int d = (int)(r % Ls.D);
    r /= Ls.D;
    const int j = (int)(r % nc), b = (int)(r / nc);
    float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const unsigned char* gp = gd + ((long)b * d_chunks + j) * Ld.Vs * 16;
    for (int c = 0; c < 8; ++c) {
      float f[8];
      unpack8(*reinterpret_cast<const uint4*>(gp + ppos(Ld, 2 * d + (c >> 2), 2 * h + ((c >> 1) & 1), 2 * w + (c & 1)) * 16), f);
#pragma unroll
      for (int k = 0; k < 8; ++k) acc[k] += f[k];
    }
    const long o = (((long)b * s_chunks + j) * Ls.Vs + ppos(Ls, d, h, w)) * 16;
    float m[8];
    unpack8(*reinterpret_cast<const uint4*>(s + o), m);
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = bf16r(acc[k]) * (m[k] > 0.f ? 1.f : kLeaky);
    *reinterpret_cast<uint4*>(gs + o) = pack8(acc);
  }
}

// gradient of an encoder output (consumed by the pooling and the skip connection), in place in the skip
// gradient: g = bf16(leaky'(s) * (bf16(gp[parent] / 8) + g))
__global__ void k_pool_backward(const unsigned char* __restrict__ gp, int p_chunks, LevelArg Lp,
                                const unsigned char* __restrict__ s, unsigned char* __restrict__ g, int c_chunks,
                                int coff, LevelArg Lc, int nc, int B) {
  const long nvox = (long)Lc.D * Lc.H * Lc.W;
  const long total = (long)B * nc * nvox;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    long r = i;
    const int w = (int)(r % Lc.W);
    r /= Lc.W;
    const int h = (int)(r % Lc.H);
    r /= Lc.H;
    const int d = (int)(r % Lc.D);
    r /= Lc.D;
    const int j = (int)(r % nc), b = (int)(r / nc);
    float up[8], sk[8], m[8];
    unpack8(*reinterpret_cast<const uint4*>(gp + (((long)b * p_chunks + j) * Lp.Vs + ppos(Lp, d / 2, h / 2, w / 2)) * 16), up);
    const long o = (((long)b * c_chunks + coff + j) * Lc.Vs + ppos(Lc, d, h, w)) * 16;
    unpack8(*reinterpret_cast<const uint4*>(g + o), sk);
    unpack8(*reinterpret_cast<const uint4*>(s + o), m);
#pragma unroll
    for (int k = 0; k < 8; ++k) sk[k] = (bf16r(up[k] * 0.125f) + sk[k]) * (m[k] > 0.f ? 1.f : kLeaky);
    *reinterpret_cast<uint4*>(g + o) = pack8(sk);
  }
}

// head: y_s = x_s + b + sum_c w_c h_c (FP32), optional prediction y_s / s in the caller's units, and
// per-block partial sums of (y_s - t_s)^2 and t_s^2 for each sample (when t is given)
constexpr int kHeadThreads = 256;
__global__ void __launch_bounds__(kHeadThreads) k_head_forward(const unsigned char* __restrict__ Hd, LevelArg L,
                                                               const float* __restrict__ x, const float* __restrict__ t,
                                                               const float* __restrict__ wb, float s, int B,
                                                               float* __restrict__ ys, float* __restrict__ out,
                                                               float* __restrict__ part) {
  __shared__ float red[2][kHeadThreads];
  const long nvox = (long)L.D * L.H * L.W;
  const int b = blockIdx.y;
  float w[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) w[c] = bf16r(wb[c]);
  const float bias = wb[16];
  float e2 = 0.f, t2 = 0.f;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < nvox; i += (long)gridDim.x * blockDim.x) {
    long r = i;
    const int ww = (int)(r % L.W);
    r /= L.W;
    const int h = (int)(r % L.H), d = (int)(r / L.H);
    const long p = ppos(L, d, h, ww);
    float a[8], c2[8];
    unpack8(*reinterpret_cast<const uint4*>(Hd + (((long)b * 2) * L.Vs + p) * 16), a);
    unpack8(*reinterpret_cast<const uint4*>(Hd + (((long)b * 2 + 1) * L.Vs + p) * 16), c2);
    float acc = bias;
#pragma unroll
    for (int k = 0; k < 8; ++k) acc = fmaf(w[k], a[k], fmaf(w[8 + k], c2[k], acc));
    const long gi = (long)b * nvox + i;
    const float y = bf16r(s * x[gi]) + acc;
    ys[gi] = y;
    if (out) out[gi] = y / s;
    if (t) {
      const float tv = s * t[gi];
      e2 += (y - tv) * (y - tv);
      t2 += tv * tv;
    }
  }
  if (!part) return;
  red[0][threadIdx.x] = e2;
  red[1][threadIdx.x] = t2;
  __syncthreads();
  for (int k = kHeadThreads / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) {
      red[0][threadIdx.x] += red[0][threadIdx.x + k];
      red[1][threadIdx.x] += red[1][threadIdx.x + k];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[((long)b * gridDim.x + blockIdx.x) * 2] = red[0][0];
    part[((long)b * gridDim.x + blockIdx.x) * 2 + 1] = red[1][0];
  }
}

// loss = mean_b e2_b / t2_b (FP64 over the block partials in order); keeps t2_b for the gradient
__global__ void k_loss(const float* __restrict__ part, int nblk, int B, double* __restrict__ sums, float* __restrict__ loss) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double l = 0.0;
  for (int b = 0; b < B; ++b) {
    double e2 = 0.0, t2 = 0.0;
    for (int k = 0; k < nblk; ++k) {
      e2 += part[((long)b * nblk + k) * 2];
      t2 += part[((long)b * nblk + k) * 2 + 1];
    }
    sums[2 * b] = e2;
    sums[2 * b + 1] = t2;
    l += e2 / t2;
  }
  if (loss) *loss = (float)(l / B);
}

// head backward: dy = 2 (y_s - t_s) / (B t2_b); gradient of the head input h (bf16(leaky'(h) bf16(w dy)))
// and per-block partials of the head's weight and bias gradients sum dy h_c, sum dy
__global__ void __launch_bounds__(kHeadThreads) k_head_backward(const unsigned char* __restrict__ Hd, LevelArg L,
                                                                const float* __restrict__ ys, const float* __restrict__ t,
                                                                const float* __restrict__ wb, float s, int B,
                                                                const double* __restrict__ sums,
                                                                unsigned char* __restrict__ G, float* __restrict__ part) {
  __shared__ float red[kHeadThreads];
  const long nvox = (long)L.D * L.H * L.W;
  const int b = blockIdx.y;
  float w[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) w[c] = bf16r(wb[c]);
  const float scale = (float)(2.0 / ((double)B * sums[2 * b + 1]));
  float acc[17];
#pragma unroll
  for (int c = 0; c < 17; ++c) acc[c] = 0.f;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < nvox; i += (long)gridDim.x * blockDim.x) {
    long r = i;
    const int ww = (int)(r % L.W);
    r /= L.W;
    const int h = (int)(r % L.H), d = (int)(r / L.H);
    const long p = ppos(L, d, h, ww);
    const long gi = (long)b * nvox + i;
    const float dy = scale * (ys[gi] - s * t[gi]);
    for (int half = 0; half < 2; ++half) {
      const long o = (((long)b * 2 + half) * L.Vs + p) * 16;
      float a[8], gg[8];
      unpack8(*reinterpret_cast<const uint4*>(Hd + o), a);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        acc[8 * half + k] = fmaf(dy, a[k], acc[8 * half + k]);
        gg[k] = bf16r(w[8 * half + k] * dy) * (a[k] > 0.f ? 1.f : kLeaky);
      }
      *reinterpret_cast<uint4*>(G + o) = pack8(gg);
    }
    acc[16] += dy;
  }
  for (int c = 0; c < 17; ++c) {
    red[threadIdx.x] = acc[c];
    __syncthreads();
    for (int k = kHeadThreads / 2; k > 0; k >>= 1) {
      if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
      __syncthreads();
    }
    if (threadIdx.x == 0) part[((long)b * gridDim.x + blockIdx.x) * 17 + c] = red[0];
    __syncthreads();
  }
}

__global__ void k_head_grad_reduce(const float* __restrict__ part, int nblk, int B, float* __restrict__ g) {
  const int c = threadIdx.x;
  if (c >= 17) return;
  double s = 0.0;
  for (int b = 0; b < B; ++b)
    for (int k = 0; k < nblk; ++k) s += part[((long)b * nblk + k) * 17 + c];
  g[c] = (float)s;
}

// bias gradient partials: per chunk j and block, the sum over positions [p_first, p_last] of each of
// the chunk's 8 channels (halo positions hold zeros)
constexpr int kBiasThreads = 256;
__global__ void __launch_bounds__(kBiasThreads) k_bias_partials(const unsigned char* __restrict__ G, int chunks, int off,
                                                                long Vs, long p0, long p1, int B, float* __restrict__ part) {
  __shared__ float red[8][kBiasThreads];
  const int j = blockIdx.y;
  float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  const long span = p1 - p0 + 1;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < (long)B * span; i += (long)gridDim.x * blockDim.x) {
    const int b = (int)(i / span);
    const long p = p0 + (i - (long)b * span);
    float f[8];
    unpack8(*reinterpret_cast<const uint4*>(G + (((long)b * chunks + off + j) * Vs + p) * 16), f);
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] += f[k];
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) red[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int s = kBiasThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
#pragma unroll
      for (int k = 0; k < 8; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < 8) part[((long)j * gridDim.x + blockIdx.x) * 8 + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void k_bias_reduce(const float* __restrict__ part, int nblk, int co, float* __restrict__ db) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= co) return;
  const int j = o / 8, k = o % 8;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += part[((long)j * nblk + b) * 8 + k];
  db[o] = (float)s;
}

// weight gradient: canonical dW[o][c][tap] (c < ci) = sum over the ranges of the partials (fixed order)
__global__ void k_wgrad_reduce(const float* __restrict__ part, long nranges, int co, int ci, int ci_pad,
                               float* __restrict__ dW) {
  const long total = (long)co * ci * 27;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const int tap = (int)(i % 27);
    const long oc = i / 27;
    const int c = (int)(oc % ci), o = (int)(oc / ci);
    double s = 0.0;
    for (long r = 0; r < nranges; ++r) s += part[((r * 27 + tap) * co + o) * (long)ci_pad + c];
    dW[i] = (float)s;
  }
}

// weight images from the FP32 master (see unet_conv.cu): forward [ae][c pair][f][o][2][8][8] and input
// gradient [ae][o pair][f][c][2][8][8] holding W[o][c][2 - a][2 - e][2 - f]
__global__ void k_images(const float* __restrict__ w, int co, int ci, int ci_pad, uint16_t* __restrict__ fwd,
                         uint16_t* __restrict__ bwd) {
  const long total = 27L * co * ci_pad;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    // forward image element i: ((((ae * cpairs + cp) * 3 + f) * co + o) * 16 + h * 8 + cc) with o = 8g + r
    {
      const int cc = (int)(i & 7), r = (int)((i >> 3) & 7), h = (int)((i >> 6) & 1);
      long rest = i >> 7;                     // (((ae * cpairs + cp) * 3 + f) * (co / 8) + g)
      const int g8 = (int)(rest % (co / 8));
      rest /= co / 8;
      const int f = (int)(rest % 3);
      rest /= 3;
      const int cpairs = ci_pad / 16;
      const int cp = (int)(rest % cpairs), ae = (int)(rest / cpairs);
      const int o = 8 * g8 + r, c = cp * 16 + h * 8 + cc;
      const float v = c < ci ? w[((long)o * ci + c) * 27 + ae * 3 + f] : 0.f;
      fwd[i] = tc::bf16_rn(v);
    }
    // input-gradient image element i: rows c (ci_pad), columns o (co)
    {
      const int cc = (int)(i & 7), r = (int)((i >> 3) & 7), h = (int)((i >> 6) & 1);
      long rest = i >> 7;
      const int g8 = (int)(rest % (ci_pad / 8));
      rest /= ci_pad / 8;
      const int f = (int)(rest % 3);
      rest /= 3;
      const int opairs = co / 16;
      const int op = (int)(rest % opairs), ae = (int)(rest / opairs);
      const int c = 8 * g8 + r, o = op * 16 + h * 8 + cc;
      const int a = ae / 3, e = ae % 3;
      const float v = c < ci ? w[((long)o * ci + c) * 27 + (2 - a) * 9 + (2 - e) * 3 + (2 - f)] : 0.f;
      bwd[i] = tc::bf16_rn(v);
    }
  }
}

__global__ void k_adam_unet(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, long n, float lr, float c1, float c2) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = 0.9f * m[i] + 0.1f * gi;
    const float vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
  }
}

int grid_for(long n, int threads = 256) { return (int)std::max<long>(1, std::min<long>((n + threads - 1) / threads, 152L * 8)); }

// ---------------------------------------------------------------------------------------- host side
int build_images(Unet* U, cudaStream_t st) {
  for (int k = 0; k < kNumConv; ++k) {
    const Layer& Ly = U->layer[k];
    k_images<<<grid_for(27L * Ly.co * Ly.ci_pad), 256, 0, st>>>(U->params + Ly.woff, Ly.co, Ly.ci, Ly.ci_pad,
                                                                 reinterpret_cast<uint16_t*>(U->imgs + Ly.img_f),
                                                                 reinterpret_cast<uint16_t*>(U->imgs + Ly.img_b));
  }
  FR3D_CUDA_TRY(cudaGetLastError());
  return FR3D_OK;
}

ConvArgs conv_args(const Unet* U, int lvl, int B) {
  ConvArgs a{};
  const Level& L = U->lv[lvl];
  a.B = B;
  a.D = L.D;
  a.H = L.H;
  a.W = L.W;
  a.Hp = L.Hp;
  a.Wp = L.Wp;
  a.Vs = L.Vs;
  a.p_first = L.p_first;
  a.p_last = L.p_last;
  a.ntiles = L.ntiles;
  a.err = U->err;
  return a;
}

int conv_forward(Unet* U, int k, int B, cudaStream_t st) {
  const Layer& Ly = U->layer[k];
  ConvArgs a = conv_args(U, Ly.lvl, B);
  a.x = U->t[Ly.in_t];
  a.x_chunks = U->td[Ly.in_t].C / 8;
  a.x_off = Ly.in_off / 8;
  a.Cin = Ly.ci_pad;
  a.wimg = U->imgs + Ly.img_f;
  a.N = Ly.co;
  a.y = U->t[Ly.out_t];
  a.y_chunks = U->td[Ly.out_t].C / 8;
  a.y_off = Ly.out_off / 8;
  a.bias = U->params + Ly.woff + (long)Ly.co * Ly.ci * 27;
  a.mode = kConvFwd;
  return conv3_launch(a, st);
}

int conv_backward(Unet* U, int k, int B, cudaStream_t st) {
  const Layer& Ly = U->layer[k];
  const Level& L = U->lv[Ly.lvl];
  // weight gradient partials, then the ordered reduction into the canonical gradient
  WgradArgs w{};
  w.g = U->g[Ly.out_t];
  w.g_chunks = U->td[Ly.out_t].C / 8;
  w.g_off = Ly.out_off / 8;
  w.Cout = Ly.co;
  w.x = U->t[Ly.in_t];
  w.x_chunks = U->td[Ly.in_t].C / 8;
  w.x_off = Ly.in_off / 8;
  w.Cin = Ly.ci_pad;
  w.ndw = 3 * Ly.co <= 128 ? 3 : 1;
  w.B = B;
  w.Hp = L.Hp;
  w.Wp = L.Wp;
  w.Vs = L.Vs;
  w.p_first = L.p_first;
  w.p_last = L.p_last;
  w.range = kWgRange;
  w.ranges_per_sample = wgrad_ranges_per_sample(L.p_first, L.p_last, kWgRange);
  w.partials = U->partials;
  w.err = U->err;
  const long nranges = (long)B * w.ranges_per_sample;
  if ((size_t)(nranges * 27 * Ly.co * Ly.ci_pad) > U->partial_floats) return FR3D_ERR_UNSUPPORTED_SIZE;
  FR3D_TRY(wgrad3_launch(w, st));
  k_wgrad_reduce<<<grid_for((long)Ly.co * Ly.ci * 27), 256, 0, st>>>(U->partials, nranges, Ly.co, Ly.ci, Ly.ci_pad,
                                                                        U->grads + Ly.woff);
  // bias gradient
  const int nblk = 64;
  k_bias_partials<<<dim3(nblk, Ly.co / 8), kBiasThreads, 0, st>>>(U->g[Ly.out_t], U->td[Ly.out_t].C / 8,
                                                                   Ly.out_off / 8, L.Vs, L.p_first, L.p_last, B,
                                                                   U->red);
  k_bias_reduce<<<1, 128, 0, st>>>(U->red, nblk, Ly.co, U->grads + Ly.woff + (long)Ly.co * Ly.ci * 27);
  FR3D_CUDA_TRY(cudaGetLastError());
  // input gradient
  if (Ly.dgrad) {
    ConvArgs a = conv_args(U, Ly.lvl, B);
    a.x = U->g[Ly.out_t];
    a.x_chunks = U->td[Ly.out_t].C / 8;
    a.x_off = Ly.out_off / 8;
    a.Cin = Ly.co;
    a.wimg = U->imgs + Ly.img_b;
    a.N = Ly.ci_pad;
    a.y = U->g[Ly.in_t];
    a.y_chunks = U->td[Ly.in_t].C / 8;
    a.y_off = Ly.in_off / 8;
    a.mode = Ly.dgrad == 1 ? kConvDgradMask : kConvDgradPlain;
    a.mask = U->t[Ly.in_t];
    a.mask_chunks = U->td[Ly.in_t].C / 8;
    a.mask_off = Ly.in_off / 8;
    FR3D_TRY(conv3_launch(a, st));
  }
  return FR3D_OK;
}

int forward(Unet* U, const float* x, int B, const float* t, float* out, cudaStream_t st) {
  const Level& L0 = U->lv[0];
  k_pack_input<<<grid_for((long)B * L0.D * L0.H * L0.W), 256, 0, st>>>(x, B, larg(L0), U->in_scale, U->t[T_X]);
  FR3D_CUDA_TRY(cudaGetLastError());
  FR3D_TRY(conv_forward(U, 0, B, st));
  FR3D_TRY(conv_forward(U, 1, B, st));
  for (int l = 1; l < kL; ++l) {
    const int src = T_CAT + l - 1;
    const int nc = kWidth[l - 1] / 8;
    const long nv = (long)B * nc * U->lv[l].D * U->lv[l].H * U->lv[l].W;
    k_pool<<<grid_for(nv), 256, 0, st>>>(U->t[src], U->td[src].C / 8, kWidth[l] / 8, larg(U->lv[l - 1]),
                                         U->t[T_P + l - 1], nc, larg(U->lv[l]), nc, B);
    FR3D_CUDA_TRY(cudaGetLastError());
    FR3D_TRY(conv_forward(U, 2 * l, B, st));
    FR3D_TRY(conv_forward(U, 2 * l + 1, B, st));
    if (l == kL - 1) FR3D_TRY(conv_forward(U, 8, B, st));
  }
  for (int l = kL - 2; l >= 0; --l) {
    const int src = l == kL - 2 ? T_B + 2 : T_D2 + l + 1;
    const int nc = kWidth[l + 1] / 8;
    const long nv = (long)B * nc * U->lv[l].D * U->lv[l].H * U->lv[l].W;
    k_up<<<grid_for(nv), 256, 0, st>>>(U->t[src], U->td[src].C / 8, larg(U->lv[l + 1]), U->t[T_CAT + l],
                                       U->td[T_CAT + l].C / 8, larg(U->lv[l]), nc, B);
    FR3D_CUDA_TRY(cudaGetLastError());
    const int k = 9 + 2 * (kL - 2 - l);
    FR3D_TRY(conv_forward(U, k, B, st));
    FR3D_TRY(conv_forward(U, k + 1, B, st));
  }
  const int nblk = 128;
  k_head_forward<<<dim3(nblk, B), kHeadThreads, 0, st>>>(U->t[T_D2], larg(L0), x, t, U->params + U->head_off,
                                                         U->in_scale, B, U->y, out, t ? U->red : nullptr);
  FR3D_CUDA_TRY(cudaGetLastError());
  return FR3D_OK;
}

int backward(Unet* U, const float* t, int B, float* loss, cudaStream_t st) {
  const Level& L0 = U->lv[0];
  const int nblk = 128;
  k_loss<<<1, 32, 0, st>>>(U->red, nblk, B, U->lossbuf, loss);
  k_head_backward<<<dim3(nblk, B), kHeadThreads, 0, st>>>(U->t[T_D2], larg(L0), U->y, t, U->params + U->head_off,
                                                          U->in_scale, B, U->lossbuf, U->g[T_D2], U->red);
  k_head_grad_reduce<<<1, 32, 0, st>>>(U->red, nblk, B, U->grads + U->head_off);
  FR3D_CUDA_TRY(cudaGetLastError());
  for (int l = 0; l <= kL - 2; ++l) {
    const int k = 9 + 2 * (kL - 2 - l);
    FR3D_TRY(conv_backward(U, k + 1, B, st));
    FR3D_TRY(conv_backward(U, k, B, st));
    const int dst = l == kL - 2 ? T_B + 2 : T_D2 + l + 1;
    const int nc = kWidth[l + 1] / 8;
    const long nv = (long)B * nc * U->lv[l + 1].D * U->lv[l + 1].H * U->lv[l + 1].W;
    k_up_backward<<<grid_for(nv), 256, 0, st>>>(U->g[T_CAT + l], U->td[T_CAT + l].C / 8, larg(U->lv[l]), U->t[dst],
                                                U->g[dst], U->td[dst].C / 8, larg(U->lv[l + 1]), nc, B);
    FR3D_CUDA_TRY(cudaGetLastError());
  }
  FR3D_TRY(conv_backward(U, 8, B, st));
  FR3D_TRY(conv_backward(U, 7, B, st));
  FR3D_TRY(conv_backward(U, 6, B, st));
  for (int l = kL - 2; l >= 0; --l) {
    const int nc = kWidth[l] / 8;
    const long nv = (long)B * nc * U->lv[l].D * U->lv[l].H * U->lv[l].W;
    k_pool_backward<<<grid_for(nv), 256, 0, st>>>(U->g[T_P + l], nc, larg(U->lv[l + 1]), U->t[T_CAT + l] +
                                                  0, U->g[T_CAT + l], U->td[T_CAT + l].C / 8, kWidth[l + 1] / 8,
                                                  larg(U->lv[l]), nc, B);
    FR3D_CUDA_TRY(cudaGetLastError());
    FR3D_TRY(conv_backward(U, 2 * l + 1, B, st));
    FR3D_TRY(conv_backward(U, 2 * l, B, st));
  }
  return FR3D_OK;
}

int check_input(const Unet* U, const void* x, int B) {
  if (!x || B < 1 || B > U->Bmax) return FR3D_ERR_INVALID_ARG;
  int dev = -1;
  FR3D_CUDA_TRY(cudaGetDevice(&dev));
  return dev == U->dev ? FR3D_OK : FR3D_ERR_INVALID_ARG;
}

uint64_t splitmix(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace

}  // namespace fr3d

struct fr3d_unet {
  fr3d::Unet u;
};

using fr3d::Unet;

static void unet_free(Unet* U) {
  for (int i = 0; i < fr3d::T_N; ++i) {
    if (U->t[i]) cudaFree(U->t[i]);
    if (U->g[i]) cudaFree(U->g[i]);
  }
  void* ps[] = {U->params, U->grads, U->m, U->v, U->imgs, U->y, U->partials, U->red, U->lossbuf, U->err};
  for (void* p : ps)
    if (p) cudaFree(p);
}

extern "C" int fr3d_unet_create(int depth, int height, int width, int max_batch, float in_scale,
                                unsigned long long seed, fr3d_unet** out) {
  using namespace fr3d;
  if (!out || max_batch < 1 || !(in_scale > 0.f) || !isfinite(in_scale)) return FR3D_ERR_INVALID_ARG;
  if (depth < 8 || height < 8 || width < 8 || depth % 8 || height % 8 || width % 8 || depth > 256 || height > 512 ||
      width > 512)
    return FR3D_ERR_UNSUPPORTED_SIZE;
  fr3d_unet* h = new (std::nothrow) fr3d_unet();
  if (!h) return FR3D_ERR_OOM;
  Unet* U = &h->u;
  int rc = FR3D_OK;
  do {
    if (cudaGetDevice(&U->dev) != cudaSuccess) {
      rc = FR3D_ERR_CUDA;
      break;
    }
    U->D = depth;
    U->H = height;
    U->W = width;
    U->Bmax = max_batch;
    U->in_scale = in_scale;
    for (int l = 0; l < kL; ++l) U->lv[l] = make_level(depth >> l, height >> l, width >> l);
    // tensors
    U->td[T_X] = {16, 0};
    for (int l = 0; l < kL - 1; ++l) {
      U->td[T_E1 + l] = {kWidth[l], l};
      U->td[T_CAT + l] = {kWidth[l + 1] + kWidth[l], l};
      U->td[T_D1 + l] = {kWidth[l], l};
      U->td[T_D2 + l] = {kWidth[l], l};
    }
    for (int l = 1; l < kL; ++l) U->td[T_P + l - 1] = {kWidth[l - 1], l};
    for (int k = 0; k < 3; ++k) U->td[T_B + k] = {kWidth[kL - 1], kL - 1};
    for (int i = 0; i < T_N && rc == FR3D_OK; ++i) {
      const size_t b = (size_t)max_batch * (U->td[i].C / 8) * U->lv[U->td[i].lvl].Vs * 16;
      U->tbytes[i] = b;
      if (cudaMalloc(&U->t[i], b) != cudaSuccess || cudaMalloc(&U->g[i], b) != cudaSuccess ||
          cudaMemset(U->t[i], 0, b) != cudaSuccess || cudaMemset(U->g[i], 0, b) != cudaSuccess)
        rc = FR3D_ERR_OOM;
    }
    if (rc) break;
    // layers in the oracle's order
    struct Spec {
      int ci, co, lvl, in_t, in_off, out_t, out_off, dgrad;
    };
    const Spec sp[kNumConv] = {
        {1, 16, 0, T_X, 0, T_E1 + 0, 0, 0},
        {16, 16, 0, T_E1 + 0, 0, T_CAT + 0, 32, 1},
        {16, 32, 1, T_P + 0, 0, T_E1 + 1, 0, 2},
        {32, 32, 1, T_E1 + 1, 0, T_CAT + 1, 64, 1},
        {32, 64, 2, T_P + 1, 0, T_E1 + 2, 0, 2},
        {64, 64, 2, T_E1 + 2, 0, T_CAT + 2, 128, 1},
        {64, 128, 3, T_P + 2, 0, T_B + 0, 0, 2},
        {128, 128, 3, T_B + 0, 0, T_B + 1, 0, 1},
        {128, 128, 3, T_B + 1, 0, T_B + 2, 0, 1},
        {192, 64, 2, T_CAT + 2, 0, T_D1 + 2, 0, 2},
        {64, 64, 2, T_D1 + 2, 0, T_D2 + 2, 0, 1},
        {96, 32, 1, T_CAT + 1, 0, T_D1 + 1, 0, 2},
        {32, 32, 1, T_D1 + 1, 0, T_D2 + 1, 0, 1},
        {48, 16, 0, T_CAT + 0, 0, T_D1 + 0, 0, 2},
        {16, 16, 0, T_D1 + 0, 0, T_D2 + 0, 0, 1},
    };
    long off = 0;
    size_t ioff = 0, pmax = 0;
    for (int k = 0; k < kNumConv; ++k) {
      Layer& Ly = U->layer[k];
      Ly.ci = sp[k].ci;
      Ly.ci_pad = std::max(16, sp[k].ci);
      Ly.co = sp[k].co;
      Ly.lvl = sp[k].lvl;
      Ly.in_t = sp[k].in_t;
      Ly.in_off = sp[k].in_off;
      Ly.out_t = sp[k].out_t;
      Ly.out_off = sp[k].out_off;
      Ly.dgrad = sp[k].dgrad;
      Ly.woff = off;
      off += (long)Ly.co * Ly.ci * 27 + Ly.co;
      const size_t ib = 27 * (size_t)Ly.co * Ly.ci_pad * 2;
      Ly.img_f = ioff;
      ioff += (ib + 255) & ~(size_t)255;
      Ly.img_b = ioff;
      ioff += (ib + 255) & ~(size_t)255;
      const Level& L = U->lv[Ly.lvl];
      const size_t nr = (size_t)max_batch * wgrad_ranges_per_sample(L.p_first, L.p_last, kWgRange);
      pmax = std::max(pmax, nr * 27 * Ly.co * Ly.ci_pad);
    }
    U->head_off = off;
    U->n_params = off + kWidth[0] + 1;
    U->img_bytes = ioff;
    U->partial_floats = pmax;
    U->red_floats = (size_t)std::max(128 * 17 * max_batch, 64 * 16 * 8);
    const size_t np = (size_t)U->n_params;
    if (cudaMalloc(&U->params, np * 4) != cudaSuccess || cudaMalloc(&U->grads, np * 4) != cudaSuccess ||
        cudaMalloc(&U->m, np * 4) != cudaSuccess || cudaMalloc(&U->v, np * 4) != cudaSuccess ||
        cudaMalloc(&U->imgs, ioff) != cudaSuccess ||
        cudaMalloc(&U->y, (size_t)max_batch * depth * height * width * 4) != cudaSuccess ||
        cudaMalloc(&U->partials, pmax * 4) != cudaSuccess || cudaMalloc(&U->red, U->red_floats * 4) != cudaSuccess ||
        cudaMalloc(&U->lossbuf, sizeof(double) * 2 * (max_batch + 1)) != cudaSuccess ||
        cudaMalloc(&U->err, sizeof(int)) != cudaSuccess) {
      rc = FR3D_ERR_OOM;
      break;
    }
    // He-normal weights (std sqrt(2 / (27 ci))) from SplitMix64 + Box-Muller, zero biases, zero head
    std::vector<float> p(np, 0.f);
    uint64_t s = seed;
    for (int k = 0; k < kNumConv; ++k) {
      const Layer& Ly = U->layer[k];
      const double sd = sqrt(2.0 / (27.0 * Ly.ci));
      for (long i = 0; i < (long)Ly.co * Ly.ci * 27; ++i) {
        const double u1 = ((splitmix(s) >> 11) + 1.0) * (1.0 / 9007199254740993.0);
        const double u2 = (splitmix(s) >> 11) * (1.0 / 9007199254740992.0);
        p[Ly.woff + i] = (float)(sd * sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2));
      }
    }
    if (cudaMemcpy(U->params, p.data(), np * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(U->m, 0, np * 4) != cudaSuccess || cudaMemset(U->v, 0, np * 4) != cudaSuccess ||
        cudaMemset(U->grads, 0, np * 4) != cudaSuccess || cudaMemset(U->err, 0, sizeof(int)) != cudaSuccess) {
      rc = FR3D_ERR_CUDA;
      break;
    }
    rc = build_images(U, 0);
    if (rc == FR3D_OK && cudaDeviceSynchronize() != cudaSuccess) rc = FR3D_ERR_CUDA;
  } while (0);
  if (rc != FR3D_OK) {
    unet_free(U);
    delete h;
    return rc;
  }
  *out = h;
  return FR3D_OK;
}

extern "C" void fr3d_unet_destroy(fr3d_unet* net) {
  if (!net) return;
  unet_free(&net->u);
  delete net;
}

extern "C" int fr3d_unet_query(const fr3d_unet* net, int* n_params) {
  if (!net) return FR3D_ERR_INVALID_ARG;
  if (n_params) *n_params = (int)net->u.n_params;
  return FR3D_OK;
}

extern "C" int fr3d_unet_get_params(fr3d_unet* net, float* params) {
  if (!net || !params) return FR3D_ERR_INVALID_ARG;
  FR3D_CUDA_TRY(cudaDeviceSynchronize());
  FR3D_CUDA_TRY(cudaMemcpy(params, net->u.params, sizeof(float) * net->u.n_params, cudaMemcpyDeviceToHost));
  return FR3D_OK;
}

extern "C" int fr3d_unet_set_params(fr3d_unet* net, const float* params) {
  if (!net || !params) return FR3D_ERR_INVALID_ARG;
  Unet* U = &net->u;
  const size_t b = sizeof(float) * U->n_params;
  FR3D_CUDA_TRY(cudaDeviceSynchronize());
  FR3D_CUDA_TRY(cudaMemcpy(U->params, params, b, cudaMemcpyHostToDevice));
  FR3D_CUDA_TRY(cudaMemset(U->m, 0, b));
  FR3D_CUDA_TRY(cudaMemset(U->v, 0, b));
  U->adam_t = 0;
  FR3D_TRY(fr3d::build_images(U, 0));
  FR3D_CUDA_TRY(cudaDeviceSynchronize());
  return FR3D_OK;
}

extern "C" int fr3d_unet_forward(fr3d_unet* net, const float* x, int B, float* y, void* stream) {
  if (!net || !y) return FR3D_ERR_INVALID_ARG;
  FR3D_TRY(fr3d::check_input(&net->u, x, B));
  return fr3d::forward(&net->u, x, B, nullptr, y, (cudaStream_t)stream);
}

extern "C" int fr3d_unet_gradient(fr3d_unet* net, const float* x, const float* t, int B, float* grad, float* loss,
                                  void* stream) {
  if (!net || !t) return FR3D_ERR_INVALID_ARG;
  FR3D_TRY(fr3d::check_input(&net->u, x, B));
  Unet* U = &net->u;
  cudaStream_t st = (cudaStream_t)stream;
  FR3D_TRY(fr3d::forward(U, x, B, t, nullptr, st));
  FR3D_TRY(fr3d::backward(U, t, B, loss, st));
  if (grad) FR3D_CUDA_TRY(cudaMemcpyAsync(grad, U->grads, sizeof(float) * U->n_params, cudaMemcpyDeviceToDevice, st));
  return FR3D_OK;
}

extern "C" int fr3d_unet_train_step(fr3d_unet* net, const float* x, const float* t, int B, float lr, float* loss,
                                    void* stream) {
  if (!net || !t || !(lr > 0.f) || !isfinite(lr)) return FR3D_ERR_INVALID_ARG;
  FR3D_TRY(fr3d::check_input(&net->u, x, B));
  Unet* U = &net->u;
  cudaStream_t st = (cudaStream_t)stream;
  FR3D_TRY(fr3d::forward(U, x, B, t, nullptr, st));
  FR3D_TRY(fr3d::backward(U, t, B, loss, st));
  ++U->adam_t;
  const float c1 = 1.f - powf(0.9f, (float)U->adam_t), c2 = 1.f - powf(0.999f, (float)U->adam_t);
  fr3d::k_adam_unet<<<fr3d::grid_for(U->n_params), 256, 0, st>>>(U->params, U->m, U->v, U->grads, U->n_params, lr, c1,
                                                                   c2);
  FR3D_CUDA_TRY(cudaGetLastError());
  return fr3d::build_images(U, st);
}

extern "C" int fr3d_unet_error_flags(fr3d_unet* net, int* flags) {
  if (!net || !flags) return FR3D_ERR_INVALID_ARG;
  FR3D_CUDA_TRY(cudaDeviceSynchronize());
  FR3D_CUDA_TRY(cudaMemcpy(flags, net->u.err, sizeof(int), cudaMemcpyDeviceToHost));
  return FR3D_OK;
}
