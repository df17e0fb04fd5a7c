// Fused Algorithm 1 steps 2-4 for M = 1 (FP32): per depth z'_j, the Tikhonov weights, the inverse
// 2D DFT of every source parameter's spectrum and the combination xi = sum_q W_q zeta_q, in one
// kernel with no spectrum intermediate in global memory.
//
// One thread-block cluster of CL CTAs handles one depth j.
//   set-up        CTA r stages the solve weights w_j(kx, ky) = A_j / (n^2 (||A||^2 + alpha s^2))
//                 (Eq. (6) with M = 1) of the columns it owns in shared memory; they do not depend
//                 on the source parameter q.
//   For each q:
//   column phase  the n/2 + 1 columns kx of the half spectrum are handled as n/2 complex columns:
//                 column 0 carries kx = 0 in its real part and kx = n/2 in its imaginary part (both
//                 are Hermitian in ky, so their inverse column DFTs are real and one complex DFT
//                 yields both).  CTA r owns columns [r n/(2 CL), (r + 1) n/(2 CL)), loads
//                 U~_q w_j and runs the inverse column DFTs along ky in shared memory;
//   row phase     after a cluster barrier, CTA r owns rows [r n/CL, (r + 1) n/CL); it reads each
//                 row's spectrum from the owners' shared memory (distributed shared memory), forms
//                 the length-n/2 complex sequence of the real inverse, transforms it and
//                 accumulates W_q zeta_q in shared memory, W_q = V0_q / sum_q' V0_q'^2 read from a
//                 per-voxel table that depends only on the geometry and the sources;
//   a second cluster barrier lets the peers finish reading before the next q overwrites.
// After the last q the accumulated xi of the owned rows is stored.  ZETA mode stores zeta_q.
// Global loads are issued in unrolled batches so that several are in flight per thread.
#pragma once

#include <cooperative_groups.h>

#include "common.cuh"
#include "fft2d.cuh"
#include "../../include/fr3d.h"

namespace fr3d {

namespace cg = cooperative_groups;

// Split cluster barrier: arrive without ordering memory and wait later.  The caller arrives only after
// it has consumed every value it read from peer shared memory, so those reads are complete.
__device__ __forceinline__ void cluster_arrive_relaxed() {
  asm volatile("barrier.cluster.arrive.relaxed.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.aligned;\n" ::: "memory"); }

// CL: CTAs per cluster (above 8 a non-portable cluster size), NT: threads, RB: rows per row batch,
// MINB: resident CTAs per SM that the register budget is sized for; GACC: accumulate xi in the output
// array (L2-resident read-modify-write) instead of shared memory
struct FusedCfgBase {
  static constexpr bool GACC = false;
};
template <int N> struct FusedCfg;
template <> struct FusedCfg<16> : FusedCfgBase { static constexpr int CL = 1, NT = 128, RB = 16, MINB = 4; };
template <> struct FusedCfg<24> : FusedCfgBase { static constexpr int CL = 1, NT = 96, RB = 24, MINB = 4; };
template <> struct FusedCfg<32> : FusedCfgBase { static constexpr int CL = 1, NT = 128, RB = 32, MINB = 4; };
template <> struct FusedCfg<48> : FusedCfgBase { static constexpr int CL = 1, NT = 128, RB = 48, MINB = 3; };
template <> struct FusedCfg<64> : FusedCfgBase { static constexpr int CL = 2, NT = 256, RB = 32, MINB = 2; };
template <> struct FusedCfg<96> : FusedCfgBase { static constexpr int CL = 2, NT = 256, RB = 48, MINB = 2; };
template <> struct FusedCfg<128> : FusedCfgBase { static constexpr int CL = 4, NT = 256, RB = 32, MINB = 2; };
template <> struct FusedCfg<192> : FusedCfgBase { static constexpr int CL = 8, NT = 256, RB = 8, MINB = 2; };
template <> struct FusedCfg<256> : FusedCfgBase { static constexpr int CL = 8, NT = 256, RB = 16, MINB = 2; };
template <> struct FusedCfg<384> : FusedCfgBase { static constexpr int CL = 8, NT = 512, RB = 16, MINB = 1; };

// Tile variants of the fused inverse (chosen at run time by the autotuner in fused_f32.cu):
//   V = 0  the table above;
//   V = 1  xi accumulated in the output array, row batches twice as tall when they divide the rows;
//   V = 2  xi accumulated in the output array, row batches as in the table;
//   V = 3  one row batch of all the CTA's rows, so that every thread owns the same outputs for every
//          source parameter: xi accumulated in registers and written once.
// All variants perform the same arithmetic in the same order: their outputs are bit-identical.
constexpr int kFusedVariants = 4;
// Variants 1 and 2 in XI mode read the output array back for every q (accumulator in the output
// array); 0 and 3 write every output once.
constexpr bool fused_rereads_output(int v) { return v == 1 || v == 2; }
template <int N, int V> struct FusedCfgV {
  using B = FusedCfg<N>;
  static constexpr int CL = B::CL, NT = B::NT, MINB = B::MINB;
  static constexpr int RB = V == 3 ? N / CL
                          : (V == 1 && (N / CL) % (2 * B::RB) == 0 && (2 * B::RB * (N / 2)) % NT == 0)
                                ? 2 * B::RB : B::RB;
  static constexpr bool GACC = V == 0 ? B::GACC : V != 3;
  static constexpr bool RACC = V == 3;
  static constexpr bool SACC = !GACC && !RACC;   // xi accumulated in shared memory
};

template <int N, int V = 0> struct FusedGeom {
  using Cf = FusedCfgV<N, V>;
  static constexpr int CL = Cf::CL, NT = Cf::NT, RB = Cf::RB;
  static constexpr int L = N / 2;
  static constexpr int CPC = L / CL;                   // packed columns per CTA
  static constexpr int NRW = N / CL;                   // rows per CTA
  static constexpr int NB = NRW / RB;                  // row batches
  static constexpr int SSC = Smem<float2, N>::ss;      // column stride in shared memory
  static constexpr int SSR = Smem<float2, L>::ss;      // row stride
  static constexpr int EPT = RB * L / NT;              // complex outputs per thread per batch
  static constexpr int NSPL = RB * (L / 2 + 1);        // Hermitian-split pairs per batch
  // shared memory: columns, rows, twiddles, pass tables (length n, n/2), weights (+ the kx = n/2
  // weights), xi accumulator
  static constexpr int PTC = passtw_size<N>(), PTR = passtw_size<L>();
  static constexpr size_t smem_zeta = sizeof(float2) * ((size_t)CPC * SSC + (size_t)RB * SSR + N + PTC + PTR) +
                                      sizeof(float) * (size_t)(CPC + 1) * N;
  static constexpr size_t smem_xi = smem_zeta + (Cf::SACC ? sizeof(float) * (size_t)NRW * N : 0);
  static_assert(L % CL == 0, "column split");
  static_assert(NRW % RB == 0, "row batches");
  static_assert((RB * L) % NT == 0, "outputs per thread");
  static_assert((CPC * N) % NT == 0, "column loads per thread");
};

struct FusedArgs {
  const float2* Uh;    // [Q][n/2+1][n] data spectra
  const float* A;      // [M' = j][n/2+1][n] dense kernel table
  const float* Dd;     // [n_alpha][n/2+1][n] dense solve weights
  const int* aidx;     // chosen row of Dd per band (clamped to [0, na))
  int na;              // rows of Dd
  const unsigned char* bbin;   // [n/2+1][n] band of every half-spectrum bin (nb > 1)
  int nb;              // bands (1: one alpha for the whole spectrum)
  const float* W;      // [Q][M'][n][n] combination weights V0_q / sum_q' V0_q'^2 (XI mode)
  float* out;          // XI: [M'][n][n]; ZETA: [Q][M'][n][n]
  const float2* tw_n;  // length-n twiddles
  int Q, j0, Mp;
  const float2* Zs;    // NULL, or solved spectra [Q][M'][n/2+1][n] (1/n^2 folded in): then A, Dd, aidx
                       // are not read and the column phase transforms Zs directly (M > 1 path)
  int* info = nullptr; // NULL or the caller's info word: a variant whose bounded waits give up ORs
                       // FR3D_INFO_TIMEOUT into it
};

// PRE: the column phase transforms the solved spectra a.Zs (M > 1 path) instead of weighting U~.
template <int N, int MODE, int V, bool PRE = false>
__device__ __forceinline__ void inv_fused_body(const FusedArgs& a, int jl) {
  using G = FusedGeom<N, V>;
  constexpr int CL = G::CL, NT = G::NT, RB = G::RB, L = G::L;
  constexpr int CPC = G::CPC, NRW = G::NRW, NB = G::NB, SSC = G::SSC, SSR = G::SSR;
  constexpr int CLD = CPC * N / NT;           // column elements per thread
  constexpr int CB = divisor_at_most(CLD, 8);  // loads in flight per batch
  static_assert(CLD % CB == 0, "load batches");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* colbuf = reinterpret_cast<float2*>(smem_raw);
  float2* rowbuf = colbuf + CPC * SSC;
  float2* tws = rowbuf + RB * SSR;           // exp(-2 pi i t / n), t < n
  float2* ptc = tws + N;                     // pass tables, length n (columns)
  float2* ptr = ptc + G::PTC;                // pass tables, length n/2 (rows)
  float* wsm = reinterpret_cast<float*>(ptr + G::PTR);   // [CPC][n] weights of the owned columns, then w(n/2, .)
  // XI with the shared-memory accumulator only: [NRW][n/2] pairs of the owned rows
  float2* accs = reinterpret_cast<float2*>(wsm + (CPC + 1) * N);
  const int tid = threadIdx.x;
  int r = 0;
  if constexpr (CL > 1) r = (int)cg::this_cluster().block_rank();
  const int j = a.j0 + jl;
  const int c0 = r * CPC;
  const int y0 = r * NRW;
  const long ps = (long)(L + 1) * N;

  // ---------------- set-up: twiddles and the q-invariant solve weights of the owned columns
  // The twiddle tables depend on nothing the previous kernel writes: they are built before waiting on
  // it (with a programmatic launch this kernel may start while the alpha rule finishes).
  for (int e = tid; e < N; e += NT) tws[e] = __ldg(a.tw_n + e);
  build_passtw<N, 1, NT>(ptc, a.tw_n, tid);
  build_passtw<L, 2, NT>(ptr, a.tw_n, tid);
  pdl_wait();
  __shared__ int s_aidx[FR3D_MAX_BANDS];
  if (tid < a.nb) s_aidx[tid] = min(max(a.aidx[tid], 0), a.na - 1);   // a caller-given index stays in the table
  __syncthreads();
  {
    const float* Aj = a.A + (long)j * ps;
    const float* drow = a.Dd + (long)s_aidx[0] * ps;
    // solve weight of bin o = kx n + ky: row aidx[band(o)] of Dd (one row when nb = 1); with bands the
    // band indices of all of this thread's bins are fetched first, then every weight in one round
    if constexpr (PRE) {
      // solved spectra: no weights
    } else if (a.nb == 1) {
#pragma unroll
      for (int b0 = 0; b0 < CLD; b0 += CB) {
        float wa[CB], wd[CB];
#pragma unroll
        for (int i = 0; i < CB; ++i) {
          const long o = (long)c0 * N + tid + (b0 + i) * NT;   // columns c0.. are contiguous
          wa[i] = __ldg(Aj + o);
          wd[i] = __ldg(drow + o);
        }
#pragma unroll
        for (int i = 0; i < CB; ++i) wsm[tid + (b0 + i) * NT] = __fmul_rn(wa[i], wd[i]);
      }
      if (r == 0)
        for (int e = tid; e < N; e += NT)
          wsm[CPC * N + e] = __fmul_rn(__ldg(Aj + (long)L * N + e), __ldg(drow + (long)L * N + e));
    } else {
#pragma unroll
      for (int b0 = 0; b0 < CLD; b0 += CB) {
        int bb[CB];
        float wa[CB], wd[CB];
#pragma unroll
        for (int i = 0; i < CB; ++i) bb[i] = __ldg(a.bbin + (long)c0 * N + tid + (b0 + i) * NT);
#pragma unroll
        for (int i = 0; i < CB; ++i) {
          const long o = (long)c0 * N + tid + (b0 + i) * NT;
          wa[i] = __ldg(Aj + o);
          wd[i] = __ldg(a.Dd + (long)s_aidx[bb[i]] * ps + o);
        }
#pragma unroll
        for (int i = 0; i < CB; ++i) wsm[tid + (b0 + i) * NT] = __fmul_rn(wa[i], wd[i]);
      }
      if (r == 0)
        for (int e = tid; e < N; e += NT) {
          const long o = (long)L * N + e;
          wsm[CPC * N + e] = __fmul_rn(__ldg(Aj + o), __ldg(a.Dd + (long)s_aidx[__ldg(a.bbin + o)] * ps + o));
        }
    }
  }
  __syncthreads();

  // X(kx, y) after the column phase, from the shared memory of the column's owner (kx in [0, n/2])
  auto xat = [&](int kx, int y) -> float2 {
    const int c = kx == L ? 0 : kx;
    const int o = c / CPC, idx = (c - o * CPC) * SSC + pidx<float2>(y);
    float2 v;
    if constexpr (CL == 1) {
      v = colbuf[idx];
    } else {
      if (o == r) v = colbuf[idx];
      else v = *cg::this_cluster().map_shared_rank(colbuf + idx, (unsigned)o);
    }
    if (kx == 0) return make_float2(v.x, 0.f);   // packed column 0: real part is kx = 0
    if (kx == L) return make_float2(v.y, 0.f);   // imaginary part is kx = n/2
    return v;
  };

  // register accumulator of xi (variant 3): element [k][rr] is the output that butterfly tid + k NT of
  // the last row pass writes as its rr-th value (the same rows and columns for every q: one row batch)
  using LPo = LastPass<L>;
  constexpr bool RACC = MODE == 1 && G::Cf::RACC;
  constexpr int KRA = RACC ? (RB * LPo::BPS + NT - 1) / NT : 1, RRA = RACC ? LPo::R : 1;
  static_assert(!RACC || NB == 1, "the register accumulator needs one row batch");
  float2 racc[KRA][RRA];
#pragma unroll
  for (int k = 0; k < KRA; ++k)
#pragma unroll
    for (int rr = 0; rr < RRA; ++rr) racc[k][rr] = make_float2(0.f, 0.f);

  for (int q = 0; q < a.Q; ++q) {
    const float2* Zq = a.Uh + (long)q * ps;
    // the peers' reads of this CTA's columns for q - 1 are done (arrive below) before overwriting
    if constexpr (CL > 1)
      if (q > 0) cluster_wait();
    // ---------------- column phase: U~_q w_j loaded straight into the registers of the first pass of
    // the inverse column DFTs (no shared-memory round trip for the input)
    const float2* Zj = PRE ? a.Zs + ((long)q * a.Mp + j) * ps : nullptr;
    auto ldc = [&](int col, int ky) -> float2 {
      const int e = col * N + ky;
      if constexpr (PRE) {        // solved spectrum of depth j (M > 1 path)
        float2 v = __ldg(Zj + (long)c0 * N + e);
        if (r == 0 && col == 0) {
          const float2 un = __ldg(Zj + (long)L * N + ky);
          v.x -= un.y;
          v.y += un.x;
        }
        return v;
      }
      const float2 u = __ldg(Zq + (long)c0 * N + e);
      const float w = wsm[e];
      float2 v = make_float2(__fmul_rn(u.x, w), __fmul_rn(u.y, w));
      if (r == 0 && col == 0) {   // packed column 0: add i w(n/2, ky) U~(n/2, ky)
        const float2 un = __ldg(Zq + (long)L * N + ky);
        const float wl = wsm[CPC * N + ky];
        v.x = __fmaf_rn(-un.y, wl, v.x);
        v.y = __fmaf_rn(un.x, wl, v.y);
      }
      return v;
    };
    first_pass_from<N, true, CPC, NT>(colbuf, SSC, ldc, tid);
    fft_passes<N, true, CPC, NT, 1, Plan<N>::np, Plan<N>::radix(0)>(colbuf, SSC, ptc, tid);
    if constexpr (CL > 1) cg::this_cluster().sync();
    // ---------------- row phase
#pragma unroll 1
    for (int b = 0; b < NB; ++b) {
      // combination weights of this batch in the layout of the last row pass (butterfly (row, jq) owns
      // outputs jq + rr NS), requested now so that the HBM latency overlaps the split and the passes
      using LPr = LastPass<L>;
      constexpr int KR = (RB * LPr::BPS + NT - 1) / NT;
      float2 wv[KR][LPr::R];
      if constexpr (MODE == 1) {
        const float2* wq = reinterpret_cast<const float2*>(a.W + (((long)q * a.Mp + j) * N + y0 + b * RB) * N);
#pragma unroll
        for (int k = 0; k < KR; ++k) {
          const int bb = tid + k * NT;
          if ((RB * LPr::BPS) % NT == 0 || bb < RB * LPr::BPS) {
            const int sr = bb / LPr::BPS, jq = bb % LPr::BPS;
#pragma unroll
            for (int rr = 0; rr < LPr::R; ++rr) wv[k][rr] = __ldg(wq + sr * L + jq + rr * LPr::NS);
          }
        }
      }
      // Hermitian split Z'[k] = (X[k] + conj X[L-k]) + i w^-k (X[k] - conj X[L-k]), pairs (k, L - k)
      constexpr int SIT = (G::NSPL + NT - 1) / NT;
      float2 xa[SIT], xb[SIT];
#pragma unroll
      for (int i = 0; i < SIT; ++i) {
        const int e = tid + i * NT;
        if (G::NSPL % NT == 0 || e < G::NSPL) {
          const int row = e % RB, k = e / RB, y = y0 + b * RB + row;
          xa[i] = xat(k, y);
          xb[i] = xat(L - k, y);
        }
      }
#pragma unroll
      for (int i = 0; i < SIT; ++i) {
        const int e = tid + i * NT;
        if (G::NSPL % NT == 0 || e < G::NSPL) {
          const int row = e % RB, k = e / RB;
          float2* rw = rowbuf + row * SSR;
          {
            const float2 sum = cadd(xa[i], cconj(xb[i])), dif = csub(xa[i], cconj(xb[i]));
            rw[pidx<float2>(k)] = cadd(sum, cmul_mi<true>(cmul(cconj(tws[k]), dif)));
          }
          if (k != 0 && 2 * k != L) {
            const float2 sum = cadd(xb[i], cconj(xa[i])), dif = csub(xb[i], cconj(xa[i]));
            rw[pidx<float2>(L - k)] = cadd(sum, cmul_mi<true>(cmul(cconj(tws[L - k]), dif)));
          }
        }
      }
      // every value read from the peers' columns for this q has been consumed above (the loads are
      // complete), so the arrival needs no memory ordering; the peers wait on it before they overwrite
      // their columns (next q) or exit
      if constexpr (CL > 1)
        if (b == NB - 1) cluster_arrive_relaxed();
      __syncthreads();
      fft_passes<L, true, RB, NT, 0, Plan<L>::np - 1>(rowbuf, SSR, ptr, tid);
      if constexpr (RACC) {
        // fmaf(w, v, 0) for q = 0, as in the accumulators of the other variants
        auto emit = [&](int, int, float2 v, int k, int rr) {
          racc[k][rr] = make_float2(fmaf(wv[k][rr].x, v.x, racc[k][rr].x), fmaf(wv[k][rr].y, v.y, racc[k][rr].y));
        };
        last_pass_to<L, true, RB, NT>(rowbuf, SSR, ptr, emit, tid);
      } else if constexpr (MODE == 1) {
        float2* acb = accs + b * RB * L;
        if constexpr (G::Cf::GACC) acb = reinterpret_cast<float2*>(a.out + ((long)j * N + y0 + b * RB) * N);
        auto emit = [&](int sr, int t, float2 v, int k, int rr) {
          float2* ac = acb + sr * L + t;
          const float2 prev = q == 0 ? make_float2(0.f, 0.f) : *ac;
          *ac = make_float2(fmaf(wv[k][rr].x, v.x, prev.x), fmaf(wv[k][rr].y, v.y, prev.y));
        };
        last_pass_to<L, true, RB, NT>(rowbuf, SSR, ptr, emit, tid);
      } else {
        float2* o = reinterpret_cast<float2*>(a.out + (((long)q * a.Mp + j) * N + y0 + b * RB) * N);
        auto emit = [&](int sr, int t, float2 v, int, int) { o[sr * L + t] = v; };
        last_pass_to<L, true, RB, NT>(rowbuf, SSR, ptr, emit, tid);
      }
      __syncthreads();
    }
  }
  if constexpr (RACC) {
    // xi of the owned rows, in the positions the last row pass produced them
    float2* ov = reinterpret_cast<float2*>(a.out + ((long)j * N + y0) * N);
#pragma unroll
    for (int k = 0; k < KRA; ++k) {
      const int bb = tid + k * NT;
      if ((RB * LPo::BPS) % NT == 0 || bb < RB * LPo::BPS) {
        const int sr = bb / LPo::BPS, jq = bb - sr * LPo::BPS;
#pragma unroll
        for (int rr = 0; rr < RRA; ++rr) ov[sr * L + jq + rr * LPo::NS] = racc[k][rr];
      }
    }
  }
  // no CTA leaves while a peer may still read its shared memory
  if constexpr (CL > 1) cluster_wait();
  if constexpr (MODE == 1 && G::Cf::SACC) {
    // xi of the owned rows; the last barrier of the q loop ordered every accumulator write first
    float2* ov = reinterpret_cast<float2*>(a.out + ((long)j * N + y0) * N);
#pragma unroll 4
    for (int e = tid; e < NRW * L; e += NT) ov[e] = accs[e];
  }
}

// Both kernels are launched with a cluster dimension of FusedCfg<N>::CL (launch_clustered).
template <int N, int MODE, int V, bool PRE = false>
__global__ void __launch_bounds__(FusedCfg<N>::NT, FusedCfg<N>::MINB) k_inv_fused(FusedArgs a) {
  inv_fused_body<N, MODE, V, PRE>(a, (int)blockIdx.x / FusedCfg<N>::CL);
}

// Batched instances of one grid size n: cluster c handles depth map[c].y of instance map[c].x.
template <int N, int MODE, int V>
__global__ void __launch_bounds__(FusedCfg<N>::NT, FusedCfg<N>::MINB)
    k_inv_fused_batched(const FusedArgs* __restrict__ inst, const int2* __restrict__ map) {
  const int2 m = map[blockIdx.x / FusedCfg<N>::CL];
  const FusedArgs a = inst[m.x];
  inv_fused_body<N, MODE, V>(a, m.y);
}

// Launch `kern` on `clusters` clusters of CL CTAs (a runtime cluster dimension; sizes above the
// portable 8 are allowed once per kernel, on the first launch, which happens outside any capture).
template <int CL, class K, class... Args>
int launch_clustered(K kern, int clusters, int nt, size_t sm, cudaStream_t st, Args... args) {
  FR3D_TRY(smem_optin(reinterpret_cast<const void*>(kern), sm));
  if constexpr (CL > 8) {
    static bool allowed = false;
    if (!allowed) {
      FR3D_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
      allowed = true;
    }
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(clusters * CL);
  cfg.blockDim = dim3(nt);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = st;
  // cluster dimension, and a programmatic launch: the kernel may start while the previous kernel in the
  // stream finishes (it builds its twiddle tables, then waits for that kernel before reading its output)
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  FR3D_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, args...));
  return FR3D_OK;
}

// Launchers of variant V for every supported n (defined in fused_v<V>.cu), and of the solved-spectra
// form (variant 1, fused_pre.cu).
template <int V> int fused_launch(int n, bool xi, const FusedArgs& a, int nj, cudaStream_t st);
int fused_launch_pre(int n, bool xi, const FusedArgs& a, int nj, cudaStream_t st);
template <int V>
int fused_launch_batched(int n, bool xi, const FusedArgs* inst, const int2* map, int nclusters, cudaStream_t st);

// Definitions shared by the fused_v<V>.cu files.
#define FR3D_FUSED_VARIANT(V)                                                                                   \
  template <int N, int MODE>                                                                                    \
  static int launch_one_##V(const FusedArgs& a, int nj, cudaStream_t st) {                                      \
    using G = FusedGeom<N, V>;                                                                                  \
    constexpr size_t sm = MODE == 1 ? G::smem_xi : G::smem_zeta;                                                \
    return launch_clustered<G::CL>(k_inv_fused<N, MODE, V>, nj, G::NT, sm, st, a);                              \
  }                                                                                                             \
  template <int N, int MODE>                                                                                    \
  static int launch_batched_##V(const FusedArgs* inst, const int2* map, int ncl, cudaStream_t st) {             \
    using G = FusedGeom<N, V>;                                                                                  \
    constexpr size_t sm = MODE == 1 ? G::smem_xi : G::smem_zeta;                                                \
    return launch_clustered<G::CL>(k_inv_fused_batched<N, MODE, V>, ncl, G::NT, sm, st, inst, map);             \
  }                                                                                                             \
  template <>                                                                                                   \
  int fused_launch<V>(int n, bool xi, const FusedArgs& a, int nj, cudaStream_t st) {                            \
    switch (n) {                                                                                                \
      FR3D_FUSED_CASES(launch_one_##V, (a, nj, st))                                                             \
    }                                                                                                           \
    return FR3D_ERR_UNSUPPORTED_SIZE;                                                                           \
  }                                                                                                             \
  template <>                                                                                                   \
  int fused_launch_batched<V>(int n, bool xi, const FusedArgs* inst, const int2* map, int ncl, cudaStream_t st) { \
    switch (n) {                                                                                                \
      FR3D_FUSED_CASES(launch_batched_##V, (inst, map, ncl, st))                                                \
    }                                                                                                           \
    return FR3D_ERR_UNSUPPORTED_SIZE;                                                                           \
  }
#define FR3D_FUSED_CASE(F, ARGS, N) \
  case N: return xi ? F<N, 1> ARGS : F<N, 0> ARGS;
#define FR3D_FUSED_CASES(F, ARGS)                                                                 \
  FR3D_FUSED_CASE(F, ARGS, 16) FR3D_FUSED_CASE(F, ARGS, 24) FR3D_FUSED_CASE(F, ARGS, 32)         \
  FR3D_FUSED_CASE(F, ARGS, 48) FR3D_FUSED_CASE(F, ARGS, 64) FR3D_FUSED_CASE(F, ARGS, 96)         \
  FR3D_FUSED_CASE(F, ARGS, 128) FR3D_FUSED_CASE(F, ARGS, 192) FR3D_FUSED_CASE(F, ARGS, 256)      \
  FR3D_FUSED_CASE(F, ARGS, 384)

}  // namespace fr3d
