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

constexpr int kTcThreads = 128;
constexpr long kWaitPolls = 1L << 22;   // bounded mbarrier waits (a poll suspends for a short slice)

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
  while (c < L.N) c <<= 1;
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

template <bool SPLIT>
__global__ void __launch_bounds__(kTcThreads) k_tc_contract(TcArgs a, TcAlphas al) {
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ __align__(8) uint64_t bar_tma, bar_mma;
  __shared__ uint32_t tbase;
  __shared__ int sbad;
  __shared__ long sbin[2][4];
  __shared__ float swt[2][4];
  __shared__ int snm[2], scls[2];
  __shared__ float gsc[2][64];
  const TcLayout L = tc_layout(a.Kc, a.Q);
  unsigned char* sA[2] = {sm, sm + L.aRegion};
  unsigned char* sB[2] = {sm + (SPLIT ? 2 : 1) * L.aRegion, sm + (SPLIT ? 2 : 1) * L.aRegion + L.bRegion};
  const int tid = threadIdx.x, warp = tid >> 5;
  // zero the table regions once: the rows past R, the chunks past K and the tail are never copied and
  // must hold finite values (they meet zero right-hand-side entries or feed discarded rows)
  for (int e = tid; e < (SPLIT ? 2 : 1) * L.aRegion / 16; e += kTcThreads)
    reinterpret_cast<uint4*>(sm)[e] = make_uint4(0, 0, 0, 0);
  tc::fence_proxy_async();   // the zeros are ordered before the bulk copies into the same region
  if (tid == 0) {
    tc::mbar_init(&bar_tma, 1);
    tc::mbar_init(&bar_mma, 1);
    tc::mbar_fence_init();
    sbad = 0;
  }
  if (warp == 0) tc::tmem_alloc(&tbase, L.ncols_tmem);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tbase;
  const int npairs = (a.C + 1) / 2;
  const uint32_t idesc = tc::idesc_bf16(128, L.N);
  uint32_t phase = 0;
  for (int pair = blockIdx.x; pair < npairs; pair += gridDim.x, phase ^= 1u) {
    // class tables of the pair: one bulk copy per class (and per split half)
    if (tid < 2) {
      const int c = 2 * pair + tid;
      scls[tid] = c < a.C ? c : -1;
      int kxs[4], kys[4];
      float wts[4];
      int nm = 0;
      if (c < a.C) nm = class_members(c, a.n, kxs, kys, wts);
      snm[tid] = nm;
      for (int m = 0; m < 4; ++m) {
        sbin[tid][m] = m < nm ? (long)kxs[m] * a.n + kys[m] : 0;
        swt[tid][m] = m < nm ? wts[m] : 0.f;
      }
    }
    if (tid == 0) {
      const int nv = (2 * pair + 1 < a.C) ? 2 : 1;
      tc::mbar_arrive_expect_tx(&bar_tma, (uint32_t)(nv * a.blob * (SPLIT ? 2 : 1)));
      for (int s = 0; s < nv; ++s) {
        const long c = 2L * pair + s;
        unsigned char* dst = sA[0] + s * 8 * L.sboA;
        tc::bulk_g2s(dst, reinterpret_cast<const unsigned char*>(a.hi) + c * a.blob, (uint32_t)a.blob, &bar_tma);
        if (SPLIT)
          tc::bulk_g2s(sA[1] + s * 8 * L.sboA, reinterpret_cast<const unsigned char*>(a.lo) + c * a.blob,
                       (uint32_t)a.blob, &bar_tma);
      }
    }
    __syncthreads();
    // per-class scaling of the right-hand sides
    if (a.scale == kScaleSolve) {
      for (int e = tid; e < 2 * a.K; e += kTcThreads) {
        const int s = e / a.K, k = e - s * a.K, c = scls[s];
        float g = 0.f;
        if (c >= 0) {
          const int ki = min(max(a.aidx[a.nb > 1 ? (int)a.cband[c] : 0], 0), a.na - 1);
          const double t = al.a[ki] * (*a.s2);
          const double l = a.lam[(long)c * a.K + k];
          float gi;
          if (a.ra == FR3D_RA_TSVD) gi = (l >= t && l > 0.0) ? __frcp_rn((float)l) : 0.f;
          else gi = __frcp_rn((float)(l + t));
          g = gi * a.inv_n2;
        }
        gsc[s][k] = g;
      }
      __syncthreads();
    }
    // B operand: column (slot s, q, member m, re/im), contraction index k; zeros outside the data
    {
      const int kpad = 8 * L.KcB;
      const int total = 2 * a.Q * kpad * 4;
      for (int e = tid; e < total; e += kTcThreads) {
        const int m = e & 3;
        int rest = e >> 2;
        const int k = rest % kpad;
        rest /= kpad;
        const int q = rest % a.Q, s = rest / a.Q;
        float2 v = make_float2(0.f, 0.f);
        if (scls[s] >= 0 && k < a.K && m < snm[s]) {
          v = a.in[((long)q * a.K + k) * a.ps + sbin[s][m]];
          const float f = a.scale == kScaleSolve ? gsc[s][k] : (a.scale == kScaleConst ? a.cscale : 1.f);
          v.x *= f;
          v.y *= f;
        }
        const int col = s * L.ncolc + q * 8 + 2 * m;
        const uint16_t hx = tc::bf16_rn(v.x), hy = tc::bf16_rn(v.y);
        *reinterpret_cast<uint16_t*>(sB[0] + cm_off(col, k, L.KcB)) = hx;
        *reinterpret_cast<uint16_t*>(sB[0] + cm_off(col + 1, k, L.KcB)) = hy;
        if (SPLIT) {
          *reinterpret_cast<uint16_t*>(sB[1] + cm_off(col, k, L.KcB)) = tc::bf16_rn(v.x - tc::bf16_val(hx));
          *reinterpret_cast<uint16_t*>(sB[1] + cm_off(col + 1, k, L.KcB)) = tc::bf16_rn(v.y - tc::bf16_val(hy));
        }
      }
    }
    tc::fence_proxy_async();
    __syncthreads();
    // tables landed?  (every thread waits, so a give-up is seen by all)
    const bool got = tc::mbar_wait(&bar_tma, phase, kWaitPolls);
    if (!got) sbad = 1;
    __syncthreads();
    if (sbad) break;
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t a0 = tc::smem_addr(sA[0]), b0 = tc::smem_addr(sB[0]);
      for (int st = 0; st < L.nsteps; ++st) {
        const uint64_t da = tc::desc_kmajor(a0 + 256 * st, 128, L.sboA);
        const uint64_t db = tc::desc_kmajor(b0 + 256 * st, 128, L.sboB);
        tc::mma_bf16(tmem, da, db, idesc, st > 0);
      }
      if (SPLIT) {
        const uint32_t a1 = tc::smem_addr(sA[1]), b1 = tc::smem_addr(sB[1]);
        for (int st = 0; st < L.nsteps; ++st) {
          tc::mma_bf16(tmem, tc::desc_kmajor(a0 + 256 * st, 128, L.sboA), tc::desc_kmajor(b1 + 256 * st, 128, L.sboB),
                       idesc, true);
          tc::mma_bf16(tmem, tc::desc_kmajor(a1 + 256 * st, 128, L.sboA), tc::desc_kmajor(b0 + 256 * st, 128, L.sboB),
                       idesc, true);
        }
      }
      tc::mma_commit(&bar_mma);
    }
    const bool done = tc::mbar_wait(&bar_mma, phase, kWaitPolls);
    if (!done) sbad = 1;
    tc::fence_after_sync();
    __syncthreads();
    if (sbad) break;
    // epilogue: thread tid owns TMEM lane tid = row tid of the tile: slot tid / 64, row r = tid % 64
    {
      const int s = warp >> 1, r = tid & 63, c = scls[s];
      const uint32_t tw = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(s * L.ncolc);
      float pw = 0.f;
      for (int q = 0; q < a.Q; ++q) {
        float v[8];
        tmem_ld8(tw + 8 * q, v);   // warp-uniform address: every lane loads, rows past R are dropped
        if (c >= 0 && r < a.R) {
          for (int m = 0; m < snm[s]; ++m) {
            const float2 y = make_float2(v[2 * m], v[2 * m + 1]);
            const long plane = a.jq ? (long)r * a.Q + q : (long)q * a.R + r;
            a.out[plane * a.ps + sbin[s][m]] = y;
            pw = fmaf(swt[s][m], y.x * y.x + y.y * y.y, pw);
          }
        }
      }
      if (a.Pc && c >= 0 && r < a.R) a.Pc[(long)c * a.R + r] = (double)pw;
    }
    tc::fence_before_sync();
    __syncthreads();
  }
  if (sbad) {
    // a wait gave up: report it, give in-flight copies and MMAs a bounded chance to land, release TMEM
    if (tid == 0 && a.info) atomicOr(a.info, FR3D_INFO_TIMEOUT);
    tc::mbar_wait(&bar_tma, phase, kWaitPolls);
    tc::mbar_wait(&bar_mma, phase, kWaitPolls);
    tc::fence_before_sync();
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
  size_t smem = (size_t)(split ? 2 : 1) * (L.aRegion + L.bRegion);
  const int max_ctas = 512 / L.ncols_tmem;
  int occ = 0;
  std::lock_guard<std::mutex> lock(g_tc_mu);
  for (;;) {
    FR3D_TRY(smem_optin(kern, smem));
    FR3D_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kTcThreads, smem));
    if (occ <= max_ctas) break;
    smem += 4096;
  }
  if (occ < 1) return FR3D_ERR_UNSUPPORTED_SIZE;
  out->smem = smem;
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
  if (split) k_tc_contract<true><<<lc.grid, kTcThreads, lc.smem, st>>>(a, al);
  else k_tc_contract<false><<<lc.grid, kTcThreads, lc.smem, st>>>(a, al);
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
