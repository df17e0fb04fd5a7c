// Per-class contractions of the M > 1 path on the tensor cores (BF16 operands, FP32 accumulation):
// the dense products of Eq. (6)'s small systems that the FP32 path runs on CUDA cores (multi.cu):
//     projection   p = U_c^T U~          (rows: eigen-components i, contraction over observation depths k)
//     solve        zeta~ = W_c^T (g p)   (rows: depths j of R, contraction over components i, g = g(alpha))
//     forward      U~ = A_c zeta~ / n^2  (rows: observation depths i, contraction over depths j)
// For a class c the right-hand sides are its member bins (up to 4), real and imaginary parts and every
// source parameter q: 8 Q columns.  Two classes share one 128-row MMA tile: the table of class 2c fills
// rows 0-63 and that of 2c+1 rows 64-127, the columns of both classes side by side (16 Q columns); the
// diagonal blocks are the two products (the off-diagonal ones are computed and discarded).
//
// Data movement per pair: one bulk asynchronous copy (TMA engine) per class table, which is stored in
// global memory as the exact shared-memory image of the MMA operand (core-matrix layout of tc.cuh, one
// contiguous blob per class); the right-hand sides gathered from the spectra by all threads, rounded to
// BF16 and written into the B operand; 2-8 tcgen05.mma of K = 16 into a TMEM accumulator issued by one
// thread; the epilogue reads each thread's TMEM lane (one output row) and scatters it to the spectra.
// Split mode (FR3D_PREC_BF16X3): table and data are each the sum of two BF16 numbers (hi + lo, lo the
// rounded remainder), and the products hi*hi + hi*lo + lo*hi accumulate in the same TMEM tile.
#include <math.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "classes.cuh"
#include "ops.cuh"
#include "tc.cuh"

namespace fr3d {

namespace {

constexpr long kWaitPolls = 1L << 22;   // bounded mbarrier waits (a poll suspends for a short slice)
constexpr uint32_t kSleepNs = 200;      // suspend-time hint of the pipeline waits (at most about 0.8 s in all)

struct TcAlphas {
  double a[FR3D_MAX_ALPHAS];
};

// right-hand-side scaling of the contraction (per class and contraction index)
enum TcScale { kScaleNone = 0, kScaleSolve = 1, kScaleConst = 2 };

struct TcArgs {
  const uint16_t* hi;   // [C][blob] BF16 tables (shared-memory image)
  const uint16_t* lo;   // [C][blob] remainders (split mode) or null
  int blob;             // bytes per class table: Rg * Kc * 128
  int Kc;               // 8-column chunks of the contraction index in a table row group
  int R, K;             // output rows per column and contraction length (<= 64 each)
  int C, n, Q;
  long ps;              // half-spectrum plane stride (bins)
  const float2* in;     // right-hand-side planes, plane q * K + k
  float2* out;          // output planes, q * R + r (jq = 0) or r * Q + q (jq = 1)
  int jq;
  int scale;            // TcScale
  float cscale;         // kScaleConst factor
  const double* lam;    // kScaleSolve: [C][K] eigenvalues
  const unsigned char* cband;
  int nb;
  const int* aidx;
  int na;
  const double* s2;
  int ra;
  float inv_n2;
  double* Pc;           // [C][R] class powers sum wt |out|^2, or null
  int* info;            // FR3D_INFO_TIMEOUT is OR-ed in when a bounded wait gives up (may be null)
};

struct TcLayout {
  int sboA, aRegion, nsteps, KcB, ncolc, N, sboB, bRegion, ncols_tmem;
};

__host__ __device__ inline TcLayout tc_layout(int Kc, int Q) {
  TcLayout L;
  L.sboA = Kc * 128;
  L.aRegion = 16 * L.sboA + 128;   // 16 row groups + one core matrix of zeros read past the last row group
  L.nsteps = (Kc + 1) / 2;
  L.KcB = 2 * L.nsteps;
  L.ncolc = 8 * Q;
  L.N = 2 * L.ncolc;
  L.sboB = L.KcB * 128;
  L.bRegion = (L.N / 8) * L.sboB;
  int c = 32;
  while (c < 2 * L.N) c <<= 1;   // two accumulators (consecutive pairs)
  L.ncols_tmem = c;
  return L;
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

// byte offset of element (row, col) in a core-matrix operand with `chunks` 8-column chunks per row group
__device__ __forceinline__ int cm_off(int row, int col, int chunks) {
  return ((row >> 3) * chunks + (col >> 3)) * 128 + (row & 7) * 16 + (col & 7) * 2;
}

// One CTA = 8 warps over its pairs j (pair blockIdx.x + j gridDim.x), stage j % kTcStages, TMEM
// accumulator j % 2, warp-specialised:
//   producer warps 4-7: for every pair, once its stage is free (the MMAs of the pair kTcStages earlier
//     have completed), request its class tables (one bulk copy per class, thread 128), gather and round
//     its right-hand sides into the stage (loads of a thread issued together) and arrive on the stage's
//     "operands ready" barrier; they run up to kTcStages pairs ahead of the MMAs;
//   consumer warps 0-3: thread 0 waits for the stage's tables and right-hand sides, issues the pair's
//     MMAs into accumulator j % 2 and commits twice (accumulator ready; stage free); then all 128
//     consumer threads read the accumulator (one output row each) and scatter it, and meet on a named
//     barrier before the accumulator is written again.
constexpr int kTcStages = 3;
constexpr int kTcCtaThreads = 256;

__device__ __forceinline__ int tc_flag(const int* f) { return *reinterpret_cast<const volatile int*>(f); }
__device__ __forceinline__ void consumer_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_addr(bar)) : "memory");
}

struct PairInfo {
  long bin[2][4];
  float wt[2][4];
  int nm[2], cls[2];
};

__device__ __forceinline__ void pair_info(int pair, int C, int n, PairInfo& I) {
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const int c = 2 * pair + s;
    I.cls[s] = c < C ? c : -1;
    int kxs[4], kys[4];
    float wts[4];
    int nm = 0;
    if (c < C) nm = class_members(c, n, kxs, kys, wts);
    I.nm[s] = nm;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      I.bin[s][m] = m < nm ? (long)kxs[m] * n + kys[m] : 0;
      I.wt[s][m] = m < nm ? wts[m] : 0.f;
    }
  }
}

template <bool SPLIT>
__global__ void __launch_bounds__(kTcCtaThreads) k_tc_contract(TcArgs a, TcAlphas al) {
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ __align__(8) uint64_t full_tma[kTcStages], full_b[kTcStages], empty[kTcStages], acc_ready[2];
  __shared__ uint32_t tbase;
  __shared__ int sbad, cstop;
  __shared__ int sidx[FR3D_MAX_BANDS];
  const TcLayout L = tc_layout(a.Kc, a.Q);
  const int stage_bytes = (SPLIT ? 2 : 1) * (L.aRegion + L.bRegion);
  auto sA = [&](int st, int h) { return sm + (size_t)st * stage_bytes + h * L.aRegion; };
  auto sB = [&](int st, int h) { return sm + (size_t)st * stage_bytes + (SPLIT ? 2 : 1) * L.aRegion + h * L.bRegion; };
  const int tid = threadIdx.x, warp = tid >> 5;
  const int npairs = (a.C + 1) / 2;
  const int nloc = blockIdx.x < npairs ? (npairs - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  auto pair_of = [&](int j) { return (int)blockIdx.x + j * (int)gridDim.x; };
  // zero every table region once: rows past R, chunks past K and the tail are never copied
  for (int e = tid; e < kTcStages * stage_bytes / 16; e += kTcCtaThreads)
    reinterpret_cast<uint4*>(sm)[e] = make_uint4(0, 0, 0, 0);
  tc::fence_proxy_async();   // the zeros are ordered before the bulk copies into the same regions
  if (a.scale == kScaleSolve)
    for (int b = tid; b < max(a.nb, 1); b += kTcCtaThreads) sidx[b] = min(max(a.aidx[b], 0), a.na - 1);
  if (tid == 0) {
    for (int st = 0; st < kTcStages; ++st) {
      tc::mbar_init(&full_tma[st], 1);
      tc::mbar_init(&full_b[st], 128);
      tc::mbar_init(&empty[st], 1);
    }
    tc::mbar_init(&acc_ready[0], 1);
    tc::mbar_init(&acc_ready[1], 1);
    tc::mbar_fence_init();
    sbad = 0;
    cstop = 0;
  }
  if (warp == 0) tc::tmem_alloc(&tbase, L.ncols_tmem);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tbase;
  const uint32_t idesc = tc::idesc_bf16(128, L.N);

  if (warp >= 4) {
    // ------------------------------------------------------------------ producers
    const int ptid = tid - 128;
    const int njobs = 2 * a.Q * 4 * L.KcB;   // (class, source parameter, member, 8-index chunk)
    for (int j = 0; j < nloc && !tc_flag(&sbad); ++j) {
      const int st = j % kTcStages, use = j / kTcStages;
      if (use > 0 && !tc::mbar_wait_sleep(&empty[st], (uint32_t)((use - 1) & 1), kWaitPolls, kSleepNs)) {
        sbad = 1;
        break;
      }
      const int pair = pair_of(j);
      if (ptid == 0) {
        const int nv = (2 * pair + 1 < a.C) ? 2 : 1;
        tc::mbar_arrive_expect_tx(&full_tma[st], (uint32_t)(nv * a.blob * (SPLIT ? 2 : 1)));
        for (int s = 0; s < nv; ++s) {
          const long c = 2L * pair + s;
          tc::bulk_g2s(sA(st, 0) + s * 8 * L.sboA, reinterpret_cast<const unsigned char*>(a.hi) + c * a.blob,
                       (uint32_t)a.blob, &full_tma[st]);
          if (SPLIT)
            tc::bulk_g2s(sA(st, 1) + s * 8 * L.sboA, reinterpret_cast<const unsigned char*>(a.lo) + c * a.blob,
                         (uint32_t)a.blob, &full_tma[st]);
        }
      }
      PairInfo I;
      pair_info(pair, a.C, a.n, I);
      // right-hand sides: job (s, q, m, kc) gathers the contraction indices k = 8 kc .. 8 kc + 7 of member m
      // of class s and source parameter q (8 loads in flight), scales and rounds them to BF16 and writes
      // one 16-byte core-matrix row each for the real and the imaginary column
      for (int jb = ptid; jb < njobs; jb += 128) {
        const int kc = jb % L.KcB;
        int r = jb / L.KcB;
        const int m = r & 3;
        r >>= 2;
        const int q = r % a.Q, s = r / a.Q;
        const int c = I.cls[s];
        const bool live = c >= 0 && m < I.nm[s];
        const long bin = I.bin[s][m];
        float2 v[8];
        double lv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int k = 8 * kc + u;
          const bool ok = live && k < a.K;
          v[u] = ok ? __ldg(a.in + ((long)q * a.K + k) * a.ps + bin) : make_float2(0.f, 0.f);
          lv[u] = (ok && a.scale == kScaleSolve) ? __ldg(a.lam + (long)c * a.K + k) : 0.0;
        }
        double t = 0.0;
        if (live && a.scale == kScaleSolve) t = al.a[sidx[a.nb > 1 ? (int)a.cband[c] : 0]] * (*a.s2);
        uint32_t hx[4], hy[4], lx[4], ly[4];
#pragma unroll
        for (int u = 0; u < 8; u += 2) {
          uint16_t h[2][2], l[2][2];
#pragma unroll
          for (int w = 0; w < 2; ++w) {
            float f = 1.f;
            if (live && 8 * kc + u + w < a.K && a.scale == kScaleSolve) {
              const double lam = lv[u + w];
              float gi;
              if (a.ra == FR3D_RA_TSVD) gi = (lam >= t && lam > 0.0) ? __frcp_rn((float)lam) : 0.f;
              else gi = __frcp_rn((float)(lam + t));
              f = gi * a.inv_n2;
            } else if (a.scale == kScaleConst) {
              f = a.cscale;
            }
            const float x = v[u + w].x * f, y = v[u + w].y * f;
            h[0][w] = tc::bf16_rn(x);
            h[1][w] = tc::bf16_rn(y);
            l[0][w] = SPLIT ? tc::bf16_rn(x - tc::bf16_val(h[0][w])) : (uint16_t)0;
            l[1][w] = SPLIT ? tc::bf16_rn(y - tc::bf16_val(h[1][w])) : (uint16_t)0;
          }
          hx[u / 2] = (uint32_t)h[0][0] | ((uint32_t)h[0][1] << 16);
          hy[u / 2] = (uint32_t)h[1][0] | ((uint32_t)h[1][1] << 16);
          lx[u / 2] = (uint32_t)l[0][0] | ((uint32_t)l[0][1] << 16);
          ly[u / 2] = (uint32_t)l[1][0] | ((uint32_t)l[1][1] << 16);
        }
        const int col = s * L.ncolc + q * 8 + 2 * m;
        *reinterpret_cast<uint4*>(sB(st, 0) + cm_off(col, 8 * kc, L.KcB)) = make_uint4(hx[0], hx[1], hx[2], hx[3]);
        *reinterpret_cast<uint4*>(sB(st, 0) + cm_off(col + 1, 8 * kc, L.KcB)) = make_uint4(hy[0], hy[1], hy[2], hy[3]);
        if (SPLIT) {
          *reinterpret_cast<uint4*>(sB(st, 1) + cm_off(col, 8 * kc, L.KcB)) = make_uint4(lx[0], lx[1], lx[2], lx[3]);
          *reinterpret_cast<uint4*>(sB(st, 1) + cm_off(col + 1, 8 * kc, L.KcB)) =
              make_uint4(ly[0], ly[1], ly[2], ly[3]);
        }
      }
      tc::fence_proxy_async();   // this thread's operand writes before the MMAs read them
      mbar_arrive(&full_b[st]);
    }
  } else {
    // ------------------------------------------------------------------ consumers
    // thread 0 issues the MMAs of pair j + 1 before the epilogue of pair j (accumulators alternate), so
    // each pair's MMAs run while the previous pair is written out
    auto issue = [&](int j) {   // thread 0 only; false if a wait gave up
      const int st = j % kTcStages, use = j / kTcStages;
      const uint32_t acc = tmem + (uint32_t)((j & 1) * (L.ncols_tmem / 2));
      if (tc_flag(&sbad) || !tc::mbar_wait_sleep(&full_tma[st], (uint32_t)(use & 1), kWaitPolls, kSleepNs) ||
          !tc::mbar_wait_sleep(&full_b[st], (uint32_t)(use & 1), kWaitPolls, kSleepNs))
        return false;
      tc::fence_after_sync();
      const uint32_t a0 = tc::smem_addr(sA(st, 0)), b0 = tc::smem_addr(sB(st, 0));
      for (int k = 0; k < L.nsteps; ++k)
        tc::mma_bf16(acc, tc::desc_kmajor(a0 + 256 * k, 128, L.sboA), tc::desc_kmajor(b0 + 256 * k, 128, L.sboB),
                     idesc, k > 0);
      if (SPLIT) {
        const uint32_t a1 = tc::smem_addr(sA(st, 1)), b1 = tc::smem_addr(sB(st, 1));
        for (int k = 0; k < L.nsteps; ++k) {
          tc::mma_bf16(acc, tc::desc_kmajor(a0 + 256 * k, 128, L.sboA), tc::desc_kmajor(b1 + 256 * k, 128, L.sboB),
                       idesc, true);
          tc::mma_bf16(acc, tc::desc_kmajor(a1 + 256 * k, 128, L.sboA), tc::desc_kmajor(b0 + 256 * k, 128, L.sboB),
                       idesc, true);
        }
      }
      tc::mma_commit(&acc_ready[j & 1]);
      tc::mma_commit(&empty[st]);
      return true;
    };
    if (tid == 0 && nloc > 0 && !issue(0)) sbad = 1;
    for (int j = 0; j < nloc; ++j) {
      const int ab = j & 1;
      const uint32_t acc = tmem + (uint32_t)(ab * (L.ncols_tmem / 2));
      // accumulator (j + 1) % 2 was read by the epilogue of pair j - 1, which ended at the last barrier
      if (tid == 0 && j + 1 < nloc && !issue(j + 1)) sbad = 1;
      __syncwarp();
      bool done = !tc_flag(&sbad) && tc::mbar_wait_sleep(&acc_ready[ab], (uint32_t)((j >> 1) & 1), kWaitPolls, kSleepNs);
      done = __all_sync(0xffffffffu, done);   // the TMEM loads below are warp-collective
      if (!done) sbad = 1;
      tc::fence_after_sync();
      if (done) {
        // epilogue of pair j: thread tid owns TMEM lane tid = row tid: slot tid / 64, row r = tid % 64
        PairInfo I;
        pair_info(pair_of(j), a.C, a.n, I);
        const int s = warp >> 1, r = tid & 63, c = I.cls[s];
        const uint32_t tw = acc + ((uint32_t)(warp * 32) << 16) + (uint32_t)(s * L.ncolc);
        float pw = 0.f;
        for (int q = 0; q < a.Q; ++q) {
          float v[8];
          tmem_ld8(tw + 8 * q, v);   // warp-uniform address: every lane loads, rows past R are dropped
          if (c >= 0 && r < a.R) {
            for (int m = 0; m < I.nm[s]; ++m) {
              const float2 y = make_float2(v[2 * m], v[2 * m + 1]);
              const long plane = a.jq ? (long)r * a.Q + q : (long)q * a.R + r;
              a.out[plane * a.ps + I.bin[s][m]] = y;
              pw = fmaf(I.wt[s][m], y.x * y.x + y.y * y.y, pw);
            }
          }
        }
        if (a.Pc && c >= 0 && r < a.R) a.Pc[(long)c * a.R + r] = (double)pw;
      }
      tc::fence_before_sync();
      if (tid == 0) cstop = tc_flag(&sbad);
      consumer_sync();   // every row of accumulator j % 2 is read before the MMAs of pair j + 2 reuse it
      if (cstop) break;  // the same decision for every consumer thread (written before the barrier)
    }
  }
  __syncthreads();
  if (sbad) {
    // a wait gave up: report it and give in-flight copies and MMAs a bounded chance to land
    if (tid == 0 && a.info) atomicOr(a.info, FR3D_INFO_TIMEOUT);
    tc::mbar_wait(&acc_ready[0], 0, 1024);
    tc::mbar_wait(&acc_ready[1], 0, 1024);
    __syncthreads();
  }
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, L.ncols_tmem);
}

// Class tables in the core-matrix image: element (r, k) of class c's R x K table (zeros outside).
// kind 0: U_c^T from Ut [C][k][i] (r = i); 1: W_c^T from W [C][i][j] (r = j, k = i); 2: A_c from A64
// [C][i][j] (r = i, k = j).  hi = BF16(v), lo = BF16(v - hi).
__global__ void k_tc_tables(const float* __restrict__ f32, const double* __restrict__ f64, int kind, int C, int M,
                            int Mp, int R, int K, int Kc, int Rg, uint16_t* __restrict__ hi, uint16_t* __restrict__ lo) {
  const int blob_el = Rg * Kc * 64;
  const long total = (long)C * blob_el;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const long c = idx / blob_el;
    const int e = (int)(idx - c * blob_el);
    // e enumerates the blob in storage order: (row group, chunk, row in group, column in chunk)
    const int cc = e & 7, rr = (e >> 3) & 7, chunk = (e >> 6) % Kc, g = (e >> 6) / Kc;
    const int r = 8 * g + rr, k = 8 * chunk + cc;
    double v = 0.0;
    if (r < R && k < K) {
      if (kind == 0) v = f32[(c * M + k) * M + r];
      else if (kind == 1) v = f32[(c * M + k) * Mp + r];
      else v = f64[(c * M + r) * Mp + k];
    }
    const float vf = (float)v;
    const uint16_t h = tc::bf16_rn(vf);
    hi[idx] = h;
    if (lo) lo[idx] = tc::bf16_rn((float)(v - (double)tc::bf16_val(h)));
  }
}

}  // namespace

bool tc_precision(int p) { return p == FR3D_PREC_BF16TC || p == FR3D_PREC_BF16X3; }

// Tables of one kind, built on first use (synchronous; allocates).
int ensure_tc_tables(Handle* H, int kind, cudaStream_t st) {
  if (H->tc_hi[kind]) return FR3D_OK;
  const int M = H->M, Mp = H->Mp, C = H->C;
  const int R = kind == 1 ? Mp : M, K = kind == 2 ? Mp : M;
  if (R > 64 || K > 64) return FR3D_ERR_UNSUPPORTED_SIZE;
  if (kind < 2) FR3D_TRY(ensure_multi_tables(H, st));
  const int Rg = (R + 7) / 8, Kc = (K + 7) / 8;
  const size_t blob = (size_t)Rg * Kc * 128;
  uint16_t *hi = nullptr, *lo = nullptr;
  cudaError_t e = cudaMalloc(&hi, blob * C);
  if (e == cudaSuccess) e = cudaMalloc(&lo, blob * C);
  if (e != cudaSuccess) {
    cudaFree(hi);
    cudaFree(lo);
    return e == cudaErrorMemoryAllocation ? FR3D_ERR_OOM : FR3D_ERR_CUDA;
  }
  const float* f32 = kind == 0 ? H->mUt : (kind == 1 ? H->mW : nullptr);
  k_tc_tables<<<152 * 8, 256, 0, st>>>(f32, H->A64, kind, C, M, Mp, R, K, Kc, Rg, hi, lo);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) {
    cudaFree(hi);
    cudaFree(lo);
    return FR3D_ERR_CUDA;
  }
  H->tc_hi[kind] = hi;
  H->tc_lo[kind] = lo;
  H->tc_blob[kind] = (int)blob;
  H->tc_kc[kind] = Kc;
  return FR3D_OK;
}

namespace {

// dynamic shared memory and grid of one launch; the shared memory is raised where needed so that the
// resident CTAs of an SM never ask for more than its 512 TMEM columns together
struct TcLaunch {
  size_t smem;
  int grid;
};
std::mutex g_tc_mu;

int tc_launch_config(const void* kern, const TcLayout& L, bool split, int npairs, TcLaunch* out) {
  int dev = 0, sms = 0;
  FR3D_CUDA_TRY(cudaGetDevice(&dev));
  FR3D_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  size_t smem = (size_t)kTcStages * (split ? 2 : 1) * (L.aRegion + L.bRegion);
  const int max_ctas = 512 / L.ncols_tmem;
  int occ = 0;
  std::lock_guard<std::mutex> lock(g_tc_mu);
  for (;;) {
    FR3D_TRY(smem_optin(kern, smem));
    occ = resident_ctas(kern, kTcCtaThreads, smem);
    if (occ <= max_ctas) break;
    smem += 4096;
  }
  if (occ < 1) return FR3D_ERR_UNSUPPORTED_SIZE;
  out->smem = smem;   // (occupancy computed for kTcCtaThreads threads)
  out->grid = std::max(1, std::min(npairs, occ * sms));
  return FR3D_OK;
}

int tc_run(const TcArgs& a, const TcAlphas& al, bool split, cudaStream_t st) {
  const TcLayout L = tc_layout(a.Kc, a.Q);
  const int npairs = (a.C + 1) / 2;
  const void* kern = split ? reinterpret_cast<const void*>(k_tc_contract<true>)
                           : reinterpret_cast<const void*>(k_tc_contract<false>);
  TcLaunch lc;
  FR3D_TRY(tc_launch_config(kern, L, split, npairs, &lc));
  if (split) k_tc_contract<true><<<lc.grid, kTcCtaThreads, lc.smem, st>>>(a, al);
  else k_tc_contract<false><<<lc.grid, kTcCtaThreads, lc.smem, st>>>(a, al);
  FR3D_CUDA_TRY(cudaGetLastError());
  return FR3D_OK;
}

TcArgs base_args(const Handle* H, int kind, bool split, int Q) {
  TcArgs a{};
  a.hi = H->tc_hi[kind];
  a.lo = split ? H->tc_lo[kind] : nullptr;
  a.blob = H->tc_blob[kind];
  a.Kc = H->tc_kc[kind];
  a.C = H->C;
  a.n = H->n;
  a.Q = Q;
  a.ps = (long)(H->n / 2 + 1) * H->n;
  a.inv_n2 = (float)(1.0 / ((double)H->n * H->n));
  return a;
}

}  // namespace

int tc_max_q() { return 16; }

// p = U_c^T U~ in place in Uh [q][i] planes, class powers to Pc [C][M]
int tc_project(Handle* H, float2* Uh, int Q, double* Pc, bool split, int* info, cudaStream_t st) {
  FR3D_TRY(ensure_tc_tables(H, 0, st));
  TcArgs a = base_args(H, 0, split, Q);
  a.R = H->M;
  a.K = H->M;
  a.in = Uh;
  a.out = Uh;
  a.scale = kScaleNone;
  a.Pc = Pc;
  a.info = info;
  return tc_run(a, TcAlphas{}, split, st);
}

// zeta~_j = sum_i W_c[i][j] g_i p_i / n^2 into Zs ([q][j] planes, or [j][q] when jq)
int tc_solve(Handle* H, const float2* P, int Q, const int* aidx, const double* alphas, int na, int ra, int nb,
             float2* Zs, int jq, bool split, int* info, cudaStream_t st) {
  FR3D_TRY(ensure_tc_tables(H, 1, st));
  TcArgs a = base_args(H, 1, split, Q);
  a.R = H->Mp;
  a.K = H->M;
  a.in = P;
  a.out = Zs;
  a.jq = jq;
  a.scale = kScaleSolve;
  a.lam = H->mlam;
  a.cband = H->cband;
  a.nb = nb;
  a.aidx = aidx;
  a.na = na;
  a.s2 = H->s2;
  a.ra = ra;
  a.info = info;
  TcAlphas al{};
  for (int k = 0; k < na; ++k) al.a[k] = alphas[k];
  return tc_run(a, al, split, st);
}

// U~_i = sum_j A_c[i][j] zeta~_j / n^2 for one source parameter (Zh [j] planes -> Uh [i] planes)
int tc_forward(Handle* H, const float2* Zh, float2* Uh, bool split, cudaStream_t st) {
  FR3D_TRY(ensure_tc_tables(H, 2, st));
  TcArgs a = base_args(H, 2, split, 1);
  a.R = H->M;
  a.K = H->Mp;
  a.in = Zh;
  a.out = Uh;
  a.scale = kScaleConst;
  a.cscale = a.inv_n2;
  return tc_run(a, TcAlphas{}, split, st);
}

}  // namespace fr3d
