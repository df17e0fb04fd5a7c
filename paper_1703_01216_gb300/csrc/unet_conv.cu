// The U-Net post-corrector's 3 x 3 x 3 convolutions on the tensor cores (tcgen05, BF16 operands, FP32
// accumulation in TMEM), as implicit GEMMs over a padded, channel-chunked activation layout.
//
// Activation layout ("CP"): per sample and per chunk of 8 channels, one plane of Vs voxels of 16 bytes
// (8 BF16 channels), Vs = (D + 2)(H + 2)(W + 2) + 128: the volume with a one-voxel zero halo on every
// side, linearised (w fastest), plus 128 zero guard voxels.  A tap (a, e, f) of the 3 x 3 x 3 stencil is
// then a constant shift s(a, e, f) = (a - 1) Hp Wp + (e - 1) Wp + (f - 1) of the linear position, with
// the zero padding supplied by the halo; outputs are computed for 128 consecutive positions at a time
// (an MMA tile of M = 128 rows) and only the interior ones are stored.
//
// Forward and input-gradient kernel (k_conv3): D[p][n] = sum over taps and input channels of
// X[p + s(tap)][c] * Wimg[tap][n][c].  Per (a, e) and 16 input channels one pipeline stage holds a slab of
// 130 positions of two channel chunks (two bulk copies; the three f taps are the same slab with the
// operand's start moved by 16 bytes) and the three taps' weights (one bulk copy of a prepared image):
// three MMAs of K = 16.  The input gradient is the same kernel with the image of the flipped, transposed
// weights (the adjoint of a correlation is the correlation with the flipped kernel).
// Weight-gradient kernel (k_wgrad3): dW[tap][o][c] = sum_p G[p][o] X[p + s(tap)][c], a GEMM whose K is the
// voxels: both operands come straight from CP planes, which hold 8 channels per 16 bytes, i.e. they are
// MN-major operands (the instruction descriptor's transpose bits).  The rows stack the three f taps of a
// (a, e) pair (each the output gradient shifted by one voxel) when 3 Cout <= 128.
#include <math.h>

#include <algorithm>
#include <mutex>

#include "ops.cuh"
#include "tc.cuh"
#include "unet.cuh"

namespace fr3d {

namespace {

constexpr long kPolls = 1L << 22;
constexpr uint32_t kSleepNs = 1000;   // suspend-time hint of the waits: a waiting thread parks (bound: kPolls * 1 us)
constexpr int kConvStages = 4;
constexpr int kSlabPos = 130;                   // positions of one (a, e) slab: 128 + the two f neighbours
constexpr int kSlabBytes = kSlabPos * 16;       // one channel chunk of a slab
// MN-major shared-memory descriptor: byte strides between core matrices along MN (channel chunks) and
// along K (groups of 8 voxels)
constexpr uint32_t kMnStrideMN_LBO = 0;         // 0: the MN stride goes in the SBO field, the K stride in LBO (measured)

__device__ __forceinline__ uint64_t desc_mn(uint32_t saddr, uint32_t mn_stride, uint32_t k_stride) {
  return kMnStrideMN_LBO ? tc::desc_kmajor(saddr, mn_stride, k_stride) : tc::desc_kmajor(saddr, k_stride, mn_stride);
}
__host__ __device__ constexpr uint32_t idesc_mn(int M, int N) {
  return tc::idesc_bf16(M, N) | (1u << 15) | (1u << 16);
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = __uint_as_float(r[k]);
}

__device__ __forceinline__ bool interior(long p, int Hp, int Wp, int D, int H, int W) {
  const long hw = (long)Hp * Wp;
  const int d = (int)(p / hw);
  const long rem = p - (long)d * hw;
  const int h = (int)(rem / Wp), w = (int)(rem - (long)h * Wp);
  return d >= 1 && d <= D && h >= 1 && h <= H && w >= 1 && w <= W;
}

__device__ __forceinline__ uint32_t pack2(float a, float b) {
  return (uint32_t)tc::bf16_rn(a) | ((uint32_t)tc::bf16_rn(b) << 16);
}
__device__ __forceinline__ float lo16(uint32_t u) { return __uint_as_float(u << 16); }
__device__ __forceinline__ float hi16(uint32_t u) { return __uint_as_float(u & 0xFFFF0000u); }

__device__ __forceinline__ int flag(const int* f) { return *reinterpret_cast<const volatile int*>(f); }

__host__ __device__ __forceinline__ uint32_t tmem_cols(int n) {
  uint32_t c = 32;
  while ((int)c < n) c <<= 1;
  return c;
}

// ------------------------------------------------------------------------------------------ k_conv3
__global__ void __launch_bounds__(128) k_conv3(ConvArgs a) {
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ __align__(8) uint64_t full[kConvStages], empty[kConvStages], done;
  __shared__ uint32_t tbase;
  __shared__ int sabort;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int N = a.N;
  const int bBytes = 3 * N * 32;
  const int stage = ((2 * kSlabBytes + bBytes) + 127) & ~127;
  const int cpairs = a.Cin / 16, niter = 9 * cpairs;
  const uint32_t ncols = tmem_cols(N);
  if (tid == 0) {
    for (int s = 0; s < kConvStages; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    tc::mbar_init(&done, 1);
    tc::mbar_fence_init();
    sabort = 0;
  }
  if (warp == 0) tc::tmem_alloc(&tbase, ncols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tbase;
  const long HW = (long)a.Hp * a.Wp;
  const uint32_t idesc = tc::idesc_bf16(128, N);
  long g = 0;           // pipeline uses so far (all tiles of this CTA)
  uint32_t tcount = 0;  // tiles so far
  const long ntot = (long)a.B * a.ntiles;
  for (long t = blockIdx.x; t < ntot; t += gridDim.x, ++tcount) {
    const int b = (int)(t / a.ntiles);
    const long p0 = a.p_first + (t - (long)b * a.ntiles) * 128;
    if (tid == 0) {
      // producer
      for (int it = 0; it < niter && !flag(&sabort); ++it) {
        const long gi = g + it;
        const int s = (int)(gi % kConvStages);
        const long use = gi / kConvStages;
        if (use > 0 && !tc::mbar_wait_sleep(&empty[s], (uint32_t)((use - 1) & 1), kPolls, kSleepNs)) {
          sabort = 1;
          break;
        }
        const int ae = it / cpairs, cp = it - ae * cpairs;
        const long off = (long)(ae / 3 - 1) * HW + (long)(ae % 3 - 1) * a.Wp - 1;
        unsigned char* st = sm + (size_t)s * stage;
        tc::mbar_arrive_expect_tx(&full[s], (uint32_t)(2 * kSlabBytes + bBytes));
        for (int h = 0; h < 2; ++h) {
          const long chunk = (long)b * a.x_chunks + a.x_off + 2 * cp + h;
          tc::bulk_g2s(st + h * kSlabBytes, a.x + (chunk * a.Vs + p0 + off) * 16, kSlabBytes, &full[s]);
        }
        tc::bulk_g2s(st + 2 * kSlabBytes, a.wimg + (size_t)it * bBytes, (uint32_t)bBytes, &full[s]);
      }
    } else if (tid == 32) {
      // MMA issuer
      for (int it = 0; it < niter && !flag(&sabort); ++it) {
        const long gi = g + it;
        const int s = (int)(gi % kConvStages);
        if (!tc::mbar_wait_sleep(&full[s], (uint32_t)((gi / kConvStages) & 1), kPolls, kSleepNs)) {
          sabort = 1;
          break;
        }
        tc::fence_after_sync();
        const uint32_t st = tc::smem_addr(sm + (size_t)s * stage);
        for (int f = 0; f < 3; ++f) {
          const uint64_t da = tc::desc_kmajor(st + 16 * f, kSlabBytes, 128);
          const uint64_t db = tc::desc_kmajor(st + 2 * kSlabBytes + f * N * 32, 128, 256);
          tc::mma_bf16(tmem, da, db, idesc, it > 0 || f > 0);
        }
        tc::mma_commit(&empty[s]);
      }
      tc::mma_commit(&done);
    }
    g += niter;
    __syncwarp();
    const bool ok = tc::mbar_wait_sleep(&done, tcount & 1u, kPolls, kSleepNs);
    if (!ok) sabort = 1;
    tc::fence_after_sync();
    __syncthreads();
    if (sabort) break;
    // epilogue: row tid = position p0 + tid
    const long p = p0 + tid;
    const bool valid = p <= a.p_last && interior(p, a.Hp, a.Wp, a.D, a.H, a.W);
    const uint32_t tw = tmem + ((uint32_t)(warp * 32) << 16);
    for (int j = 0; j < N / 8; ++j) {
      float v[8];
      tmem_ld8(tw + 8 * j, v);
      if (!valid) continue;
      if (a.mode == kConvFwd) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const float z = v[k] + (a.bias ? a.bias[8 * j + k] : 0.f);
          v[k] = z > 0.f ? z : kLeaky * z;
        }
      } else if (a.mode == kConvDgradMask) {
        const uint4 m = *reinterpret_cast<const uint4*>(
            a.mask + (((long)b * a.mask_chunks + a.mask_off + j) * a.Vs + p) * 16);
        const uint32_t mw[4] = {m.x, m.y, m.z, m.w};
        // the gradient is stored (rounded) first, then scaled by the leaky derivative and rounded again,
        // as the two steps of the chain rule store it
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          v[2 * k] = tc::bf16_val(tc::bf16_rn(v[2 * k]));
          v[2 * k + 1] = tc::bf16_val(tc::bf16_rn(v[2 * k + 1]));
          if (!(lo16(mw[k]) > 0.f)) v[2 * k] *= kLeaky;
          if (!(hi16(mw[k]) > 0.f)) v[2 * k + 1] *= kLeaky;
        }
      }
      uint4 o;
      o.x = pack2(v[0], v[1]);
      o.y = pack2(v[2], v[3]);
      o.z = pack2(v[4], v[5]);
      o.w = pack2(v[6], v[7]);
      *reinterpret_cast<uint4*>(a.y + (((long)b * a.y_chunks + a.y_off + j) * a.Vs + p) * 16) = o;
    }
    tc::fence_before_sync();
    __syncthreads();
  }
  if (sabort) {
    if (tid == 0 && a.err) atomicOr(a.err, FR3D_INFO_TIMEOUT);
    tc::mbar_wait(&done, tcount & 1u, kPolls);   // give in-flight MMAs a bounded chance to finish
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, ncols);
}

// ------------------------------------------------------------------------------------------ k_wgrad3
constexpr int kWgStages = 3;
constexpr int kWgVox = 64;                      // voxels (K) per stage: four MMAs of K = 16 (a multiple of 16 dividing the range)
constexpr int kWgPlane = kWgVox * 16;           // bytes of one channel chunk of a stage

__global__ void __launch_bounds__(128) k_wgrad3(WgradArgs a) {
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ __align__(8) uint64_t full[kWgStages], empty[kWgStages], done;
  __shared__ uint32_t tbase;
  __shared__ int sabort;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int N = a.Cin;
  const int gc = a.Cout / 8;                     // output-gradient chunks per f tap
  const int rows_loaded = a.ndw * gc;            // row groups with data (the rest stay zero)
  const int aBytes = 16 * kWgPlane;              // 128 rows
  const int bBytes = (N / 8) * kWgPlane;
  const int stage = aBytes + bBytes;
  const uint32_t ncols = tmem_cols(N);
  const int ntg = a.ndw == 3 ? 9 : 27;
  const int tg = blockIdx.x % ntg;
  const long r = blockIdx.x / ntg;
  const int b = (int)(r / a.ranges_per_sample);
  const long v0 = a.p_first + (r - (long)b * a.ranges_per_sample) * a.range;
  const long v1 = min(v0 + a.range, a.p_last + 1);
  const int nst = v1 > v0 ? (int)((v1 - v0 + kWgVox - 1) / kWgVox) : 0;
  const int ae = a.ndw == 3 ? tg : tg / 3, fsel = a.ndw == 3 ? 0 : tg % 3;
  const long HW = (long)a.Hp * a.Wp;
  const long xoff = (long)(ae / 3 - 1) * HW + (long)(ae % 3 - 1) * a.Wp + (a.ndw == 3 ? 0 : fsel - 1);
  // zero every stage once (the unused row groups of A are read as zeros)
  for (int e = tid; e < kWgStages * stage / 16; e += 128) reinterpret_cast<uint4*>(sm)[e] = make_uint4(0, 0, 0, 0);
  tc::fence_proxy_async();
  if (tid == 0) {
    for (int s = 0; s < kWgStages; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    tc::mbar_init(&done, 1);
    tc::mbar_fence_init();
    sabort = 0;
  }
  if (warp == 0) tc::tmem_alloc(&tbase, ncols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tbase;
  const uint32_t idesc = idesc_mn(128, N);
  if (warp == 0) {
    // producer warp: lane 0 waits for the stage and posts its byte count, then the lanes issue the
    // stage's copies (rows_loaded gradient chunks, N / 8 input chunks), one copy per lane
    const int lane = tid & 31;
    const int ncopy = rows_loaded + N / 8;
    for (int it = 0; it < nst; ++it) {
      const int s = it % kWgStages;
      const int use = it / kWgStages;
      int stop = 0;
      if (lane == 0) {
        stop = flag(&sabort);
        if (!stop && use > 0 && !tc::mbar_wait_sleep(&empty[s], (uint32_t)((use - 1) & 1), kPolls, kSleepNs)) {
          sabort = 1;
          stop = 1;
        }
        if (!stop) tc::mbar_arrive_expect_tx(&full[s], (uint32_t)(ncopy * kWgPlane));
      }
      stop = __shfl_sync(0xffffffffu, stop, 0);
      __syncwarp();   // the byte count is posted before any copy of the stage is issued
      if (stop) break;
      const long v = v0 + (long)it * kWgVox;
      unsigned char* st = sm + (size_t)s * stage;
      for (int k = lane; k < ncopy; k += 32) {
        if (k < rows_loaded) {
          // A: row group (fi, c) = output gradient chunk c at positions v - (fi - 1) (ndw = 3), or c at v
          const int fi = k / gc, c = k - fi * gc;
          const long pos = v - (a.ndw == 3 ? fi - 1 : 0);
          const long chunk = (long)b * a.g_chunks + a.g_off + c;
          tc::bulk_g2s(st + k * kWgPlane, a.g + (chunk * a.Vs + pos) * 16, kWgPlane, &full[s]);
        } else {
          // B: input chunk c at positions v + the (a, e[, f]) shift
          const int c = k - rows_loaded;
          const long chunk = (long)b * a.x_chunks + a.x_off + c;
          tc::bulk_g2s(st + aBytes + c * kWgPlane, a.x + (chunk * a.Vs + v + xoff) * 16, kWgPlane, &full[s]);
        }
      }
    }
  } else if (tid == 32) {
    for (int it = 0; it < nst && !flag(&sabort); ++it) {
      const int s = it % kWgStages;
      if (!tc::mbar_wait_sleep(&full[s], (uint32_t)((it / kWgStages) & 1), kPolls, kSleepNs)) {
        sabort = 1;
        break;
      }
      tc::fence_after_sync();
      const uint32_t st = tc::smem_addr(sm + (size_t)s * stage);
      for (int k = 0; k < kWgVox / 16; ++k) {
        const uint64_t da = desc_mn(st + 256 * k, kWgPlane, 128);
        const uint64_t db = desc_mn(st + aBytes + 256 * k, kWgPlane, 128);
        tc::mma_bf16(tmem, da, db, idesc, it > 0 || k > 0);
      }
      tc::mma_commit(&empty[s]);
    }
    tc::mma_commit(&done);
  }
  __syncwarp();
  const bool ok = nst == 0 || tc::mbar_wait_sleep(&done, 0u, kPolls, kSleepNs);
  if (!ok) sabort = 1;
  tc::fence_after_sync();
  __syncthreads();
  // epilogue: row tid = (fi, o) of the stacked taps; partials [r][tap][o][c]
  const uint32_t tw = tmem + ((uint32_t)(warp * 32) << 16);
  const bool row_ok = tid < rows_loaded * 8 && !sabort;
  const int fi = tid / a.Cout, o = tid - fi * a.Cout;
  const int tap = a.ndw == 3 ? ae * 3 + fi : ae * 3 + fsel;
  float* dst = a.partials + ((r * 27 + tap) * (long)a.Cout + o) * N;
  for (int j = 0; j < N / 8; ++j) {
    float v[8];
    tmem_ld8(tw + 8 * j, v);
    if (!row_ok) continue;
    if (nst == 0)
      for (int k = 0; k < 8; ++k) v[k] = 0.f;
    *reinterpret_cast<float4*>(dst + 8 * j) = make_float4(v[0], v[1], v[2], v[3]);
    *reinterpret_cast<float4*>(dst + 8 * j + 4) = make_float4(v[4], v[5], v[6], v[7]);
  }
  if (sabort) {
    if (tid == 0 && a.err) atomicOr(a.err, FR3D_INFO_TIMEOUT);
    if (nst > 0) tc::mbar_wait(&done, 0u, kPolls);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, ncols);
}

std::mutex g_conv_mu;

int launch_cfg(const void* kern, size_t smem, int ncols, int* occ_out) {
  std::lock_guard<std::mutex> lock(g_conv_mu);
  FR3D_TRY(smem_optin(kern, smem));
  int occ = 0;
  occ = resident_ctas(kern, 128, smem);
  // the resident CTAs of an SM must not ask for more than its 512 TMEM columns together
  const int cap = 512 / ncols;
  while (occ > cap) {
    smem += 8192;
    FR3D_TRY(smem_optin(kern, smem));
    occ = resident_ctas(kern, 128, smem);
  }
  if (occ < 1) return FR3D_ERR_UNSUPPORTED_SIZE;
  *occ_out = occ;
  return (int)smem;
}

}  // namespace

int conv3_launch(const ConvArgs& a, cudaStream_t st) {
  if (a.Cin % 16 || a.N % 16 || a.N < 16 || a.N > 256) return FR3D_ERR_UNSUPPORTED_SIZE;
  const int bBytes = 3 * a.N * 32;
  const size_t stage = ((2 * kSlabBytes + bBytes) + 127) & ~127;
  int occ = 0;
  const int smem = launch_cfg(reinterpret_cast<const void*>(k_conv3), stage * kConvStages, (int)tmem_cols(a.N), &occ);
  if (smem < 0) return smem;
  int dev = 0, sms = 0;
  FR3D_CUDA_TRY(cudaGetDevice(&dev));
  FR3D_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const long ntot = (long)a.B * a.ntiles;
  const int grid = (int)std::max<long>(1, std::min<long>(ntot, (long)occ * sms));
  k_conv3<<<grid, 128, smem, st>>>(a);
  FR3D_CUDA_TRY(cudaGetLastError());
  return FR3D_OK;
}

int wgrad3_launch(const WgradArgs& a, cudaStream_t st) {
  if (a.Cin % 16 || a.Cin > 256 || a.Cout % 8 || a.ndw * a.Cout > 128) return FR3D_ERR_UNSUPPORTED_SIZE;
  const size_t stage = 16 * kWgPlane + (a.Cin / 8) * kWgPlane;
  int occ = 0;
  const int smem = launch_cfg(reinterpret_cast<const void*>(k_wgrad3), stage * kWgStages, (int)tmem_cols(a.Cin), &occ);
  if (smem < 0) return smem;
  const int ntg = a.ndw == 3 ? 9 : 27;
  const long grid = (long)ntg * a.B * a.ranges_per_sample;
  k_wgrad3<<<(unsigned)grid, 128, smem, st>>>(a);
  FR3D_CUDA_TRY(cudaGetLastError());
  return FR3D_OK;
}

int wgrad_ranges_per_sample(long p_first, long p_last, long range) { return (int)((p_last - p_first + range) / range); }

}  // namespace fr3d
