// Several observation depths (M > 1): the per-frequency systems A^(m) zeta~ = U~^(m) of Eq. (6) are
// M x M' instead of rows, so step 2 needs more than a division per frequency class.
//
// Cold (once per handle, FP64): for every frequency class c the Gram matrix G_c = A_c A_c^T (M x M) and
// its eigendecomposition G_c = U_c diag(lambda_c) U_c^T by the cyclic Jacobi method (rotation pairs of a
// round are disjoint, so their angles come from the same G and the rotations apply together), and
// W_c = U_c^T A_c (M x M').  With p = U_c^T U~ the Tikhonov solution and its squared residual are
//     zeta~ = A_c^T (G_c + alpha s^2 I)^-1 U~ = W_c^T diag(g) p,   g_i = 1 / (lambda_i + alpha s^2),
//     ||A_c zeta~ - U~||^2 = sum_i (alpha s^2 / (lambda_i + alpha s^2))^2 |p_i|^2,
// (the dual form of the Tikhonov normal equation, an exact identity for any M, M'), and the truncated
// SVD keeps the components with lambda_i >= alpha s^2: g_i = 1 / lambda_i, residual weight 0, else 0 and 1.
// Hot path (FP32 data, FP64 sums): data FFT of all Q M planes; per class the projection p = U_c^T U~ in
// place and the class powers P_ci = sum wt |p_i|^2; the alpha rule over sum_c sum_i F(lambda_ci) P_ci;
// per class the solve zeta~_j = sum_i W_c[i][j] g_i p_i written as spectra [q][j][bin]; the fused
// inverse DFT + combination reading those spectra.
#include <math.h>

#include <algorithm>
#include <vector>

#include "classes.cuh"
#include "fused.cuh"
#include "ops.cuh"

namespace fr3d {

namespace {

constexpr int kMaxM = FR3D_MAX_OBS_DEPTHS;  // observation depths handled by the M > 1 path
constexpr int kSweeps = 30;                // Jacobi sweep limit (convergence is checked every sweep)

// One CTA per class.  Shared memory: G [Me][Me], U [Me][Me] (Me = M rounded up to even), FP64.
__global__ void __launch_bounds__(256) k_class_eig(const double* __restrict__ A64, int M, int Mp, int Cn,
                                                   double* __restrict__ lam, float* __restrict__ Ut,
                                                   float* __restrict__ W, int* __restrict__ sweeps_out) {
  extern __shared__ double smd[];
  const int c = blockIdx.x;
  const int Me = (M + 1) & ~1;
  double* G = smd;                 // [Me][Me]
  double* U = G + Me * Me;         // [Me][Me], column i = eigenvector i
  __shared__ double cs[kMaxM / 2 + 1][2];
  __shared__ int pr[kMaxM / 2 + 1][2];
  __shared__ double off_s, diag_s;
  __shared__ double red[256][2];
  const int tid = threadIdx.x, nt = blockDim.x;
  const double* A = A64 + (long)c * M * Mp;
  // G = A A^T; when M is odd the pad is a zero row/column in G and an identity row/column in U (the
  // pad never couples)
  for (int e = tid; e < Me * Me; e += nt) {
    const int a = e / Me, b = e % Me;
    double s = 0.0;
    if (a < M && b < M)
      for (int j = 0; j < Mp; ++j) s = fma(A[(long)a * Mp + j], A[(long)b * Mp + j], s);
    G[e] = s;
    U[e] = a == b ? 1.0 : 0.0;
  }
  __syncthreads();
  int sweep = 0;
  for (; sweep < kSweeps; ++sweep) {
    // convergence: off-diagonal mass against the diagonal (block reduction)
    {
      double off = 0.0, dg = 0.0;
      for (int e = tid; e < Me * Me; e += nt) {
        const double v = G[e] * G[e];
        if (e / Me == e % Me) dg += v;
        else off += v;
      }
      red[tid][0] = off;
      red[tid][1] = dg;
      __syncthreads();
      for (int k = nt / 2; k > 0; k >>= 1) {
        if (tid < k) {
          red[tid][0] += red[tid + k][0];
          red[tid][1] += red[tid + k][1];
        }
        __syncthreads();
      }
      if (tid == 0) {
        off_s = red[0][0];
        diag_s = red[0][1];
      }
      __syncthreads();
    }
    if (!(off_s > 1e-30 * diag_s) || Me == 1) break;
    // round-robin tournament: Me - 1 rounds of Me / 2 disjoint pairs
    for (int round = 0; round < Me - 1; ++round) {
      if (tid < Me / 2) {
        // player positions: 0 fixed, the others rotate
        auto player = [&](int pos) { return pos == 0 ? 0 : 1 + (pos - 1 + round) % (Me - 1); };
        int p = player(tid), q = player(Me - 1 - tid);
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        pr[tid][0] = p;
        pr[tid][1] = q;
        const double gpq = G[p * Me + q], gpp = G[p * Me + p], gqq = G[q * Me + q];
        double cth = 1.0, sth = 0.0;
        if (gpq != 0.0) {
          // rotation that zeroes G[p][q] (Rutishauser's stable form)
          const double tau = (gqq - gpp) / (2.0 * gpq);
          const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
          cth = 1.0 / sqrt(1.0 + t * t);
          sth = t * cth;
        }
        cs[tid][0] = cth;
        cs[tid][1] = sth;
      }
      __syncthreads();
      // rows: G <- J^T G (pair k rotates rows p, q at every column b)
      for (int e = tid; e < (Me / 2) * Me; e += nt) {
        const int k = e / Me, b = e % Me;
        const int p = pr[k][0], q = pr[k][1];
        const double cth = cs[k][0], sth = cs[k][1];
        const double gp = G[p * Me + b], gq = G[q * Me + b];
        G[p * Me + b] = cth * gp - sth * gq;
        G[q * Me + b] = sth * gp + cth * gq;
      }
      __syncthreads();
      // columns: G <- G J, and U <- U J
      for (int e = tid; e < (Me / 2) * Me; e += nt) {
        const int k = e / Me, a = e % Me;
        const int p = pr[k][0], q = pr[k][1];
        const double cth = cs[k][0], sth = cs[k][1];
        const double gp = G[a * Me + p], gq = G[a * Me + q];
        G[a * Me + p] = cth * gp - sth * gq;
        G[a * Me + q] = sth * gp + cth * gq;
        const double up = U[a * Me + p], uq = U[a * Me + q];
        U[a * Me + p] = cth * up - sth * uq;
        U[a * Me + q] = sth * up + cth * uq;
      }
      __syncthreads();
    }
  }
  // lambda_i = G[i][i] (clamped at 0: the Gram matrix is positive semidefinite), Ut[i][k] = U[k][i],
  // W[i][j] = sum_k U[k][i] A[k][j]
  for (int i = tid; i < M; i += nt) lam[(long)c * M + i] = fmax(G[i * Me + i], 0.0);
  for (int e = tid; e < M * M; e += nt) {
    const int k = e / M, i = e % M;   // stored [k][i]: component i's eigenvector, contiguous over i
    Ut[(long)c * M * M + e] = (float)U[k * Me + i];
  }
  for (int e = tid; e < M * Mp; e += nt) {
    const int i = e / Mp, j = e % Mp;
    double s = 0.0;
    for (int k = 0; k < M; ++k) s = fma(U[k * Me + i], A[(long)k * Mp + j], s);
    W[(long)c * M * Mp + e] = (float)s;
  }
  if (tid == 0 && sweeps_out) atomicMax(sweeps_out, sweep);
}

// Projection p = U_c^T U~ in place for every member bin and plane set q, and the class powers
// P_ci = sum over members and q of wt |p_i|^2 (FP32 terms in a fixed order, stored in FP64).
// Uh planes are [q][i] (plane q M + i).  One warp per class: the class's member values of a plane set
// are gathered into the warp's shared-memory slice, lane l owns components i = l, l + 32, and the
// eigenvector table (stored [k][i]) streams from global memory in coalesced rows, each element
// feeding every member.  Classes own disjoint bins, so the in-place writes never meet another
// class's reads.
constexpr int kPerCta = 8;                      // warps (classes) per CTA
constexpr int kRows = (kMaxM + 31) / 32;        // components (or depths) per lane
constexpr int kBatch = 4;                       // table rows per batch of the double-buffered stream
__global__ void __launch_bounds__(256) k_project(float2* __restrict__ Uh, long ps, int Q, int M, int n, int Cn,
                                                 const float* __restrict__ Ut, double* __restrict__ Pc) {
  __shared__ float2 xs[kPerCta][4 * kMaxM];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = blockIdx.x * kPerCta + warp;
  if (c >= Cn) return;   // a whole warp; the kernel synchronises warps only
  int kxs[4], kys[4];
  float wts[4];
  const int nm = class_members(c, n, kxs, kys, wts);
  long bin[4];
  for (int m = 0; m < 4; ++m) bin[m] = m < nm ? (long)kxs[m] * n + kys[m] : 0;
  float2* x = xs[warp];
  const float* Uc = Ut + (long)c * M * M;
  float pw[kRows];
#pragma unroll
  for (int r = 0; r < kRows; ++r) pw[r] = 0.f;
  // table rows k0 .. k0 + kBatch - 1 into buffer b (zeros past M); the arithmetic of a batch in k order
  float ub[2][kBatch][kRows];
  auto load = [&](int b, int k0) {
#pragma unroll
    for (int j = 0; j < kBatch; ++j)
#pragma unroll
      for (int r = 0; r < kRows; ++r) {
        const int k = k0 + j, i = lane + 32 * r;
        ub[b][j][r] = (k < M && i < M) ? __ldg(Uc + (long)k * M + i) : 0.f;
      }
  };
  for (int q = 0; q < Q; ++q) {
    load(0, 0);   // the first batch is in flight during the gather
    for (int e = lane; e < nm * M; e += 32) {
      const int m = e / M, k = e - m * M;
      x[e] = Uh[((long)q * M + k) * ps + bin[m]];
    }
    __syncwarp();
    float2 y[kRows][4];
#pragma unroll
    for (int r = 0; r < kRows; ++r)
#pragma unroll
      for (int m = 0; m < 4; ++m) y[r][m] = make_float2(0.f, 0.f);
    auto fma_batch = [&](int b, int k0) {
#pragma unroll
      for (int j = 0; j < kBatch; ++j) {
        const int k = k0 + j;
        if (k < M) {
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            if (m < nm) {
              const float2 xv = x[m * M + k];
#pragma unroll
              for (int r = 0; r < kRows; ++r) {
                y[r][m].x = fmaf(ub[b][j][r], xv.x, y[r][m].x);
                y[r][m].y = fmaf(ub[b][j][r], xv.y, y[r][m].y);
              }
            }
          }
        }
      }
    };
    // double-buffered stream: the next batch is requested before the current one is used
    for (int k0 = 0; k0 < M; k0 += 2 * kBatch) {
      load(1, k0 + kBatch);
      fma_batch(0, k0);
      load(0, k0 + 2 * kBatch);
      fma_batch(1, k0 + kBatch);
    }
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
      const int i = lane + 32 * r;
      if (i < M) {
#pragma unroll
        for (int m = 0; m < 4; ++m)
          if (m < nm) {
            Uh[((long)q * M + i) * ps + bin[m]] = y[r][m];
            pw[r] = fmaf(wts[m], y[r][m].x * y[r][m].x + y[r][m].y * y[r][m].y, pw[r]);
          }
      }
    }
    __syncwarp();   // the x reads are done before the next plane set is gathered
  }
#pragma unroll
  for (int r = 0; r < kRows; ++r) {
    const int i = lane + 32 * r;
    if (i < M) Pc[(long)c * M + i] = (double)pw[r];
  }
}

struct MAlphas {
  double a[FR3D_MAX_ALPHAS];
};

// residual weight of component (lambda, t = alpha s^2): Tikhonov (t / (lambda + t))^2, TSVD [lambda < t]
__device__ inline float resid_weight(float lam, float t, int ra) {
  if (ra == FR3D_RA_TSVD) return lam < t ? 1.f : 0.f;
  const float f = __fdividef(t, lam + t);   // within 2 ulp: far inside the curves' 1e-5 bound
  return f * f;
}

constexpr int kMCPB = 64;   // classes per block of the residual sums
constexpr int kMThreads = 1024;   // threads of the residual-sum blocks

// Block partials of r_b^2(alpha_k) * n^2 = sum_{c in b} sum_i F(lambda_ci, alpha_k) P_ci: the sum over
// i in FP32 (M terms), over classes in FP64; S = kMThreads / n_alpha threads per candidate take every S-th
// class, their sums are added in a fixed order.
__global__ void __launch_bounds__(kMThreads) k_alpha_m_partial(
    const double* __restrict__ lam, const double* __restrict__ Pc, int M, int Cn,
    const unsigned char* __restrict__ cband, int nb, MAlphas al, const double* __restrict__ s2, int na, int ra,
    double* __restrict__ partials) {
  __shared__ float sl[kMCPB * kMaxM], sp[kMCPB * kMaxM];
  __shared__ double red[kMThreads];
  __shared__ unsigned char sb[kMCPB];
  const int c0 = blockIdx.x * kMCPB, ncl = min(kMCPB, Cn - c0);
  for (int e = threadIdx.x; e < ncl * M; e += blockDim.x) {
    sl[e] = (float)lam[(long)c0 * M + e];
    sp[e] = (float)Pc[(long)c0 * M + e];
  }
  for (int e = threadIdx.x; e < ncl; e += blockDim.x) sb[e] = nb > 1 ? cband[c0 + e] : 0;
  __syncthreads();
  const int S = kMThreads / na, k = threadIdx.x % na, sub = threadIdx.x / na;
  const float t = (float)(al.a[k] * (*s2));
  for (int b = 0; b < nb; ++b) {
    double acc = 0.0;
    if (sub < S)
      for (int cc = sub; cc < ncl; cc += S) {
        if (sb[cc] != b) continue;
        float f = 0.f;
        for (int i = 0; i < M; ++i) f = fmaf(resid_weight(sl[cc * M + i], t, ra), sp[cc * M + i], f);
        acc += (double)f;
      }
    red[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x < na) {
      double s = 0.0;
      for (int q = 0; q < S; ++q) s += red[q * na + threadIdx.x];
      partials[((long)blockIdx.x * nb + b) * na + threadIdx.x] = s;
    }
    __syncthreads();
  }
}

// Sum of the partials (fixed order), r^2 = sum / n^2, and the discrepancy choice per band (one warp
// per band: ballots of r^2 <= thr, the largest index wins).
struct MThr {
  double t[FR3D_MAX_BANDS];
};
__global__ void __launch_bounds__(256) k_alpha_m_finish(const double* __restrict__ partials, int nblk, int nb, int na,
                                                        double inv_n2, MThr thr, int* __restrict__ aidx,
                                                        double* __restrict__ res_out, int* __restrict__ info,
                                                        int keep) {
  __shared__ double r2[FR3D_MAX_BANDS * FR3D_MAX_ALPHAS];
  __shared__ int flg[FR3D_MAX_BANDS];
  const int tid = threadIdx.x, O = nb * na;
  for (int o = tid; o < O; o += blockDim.x) {
    double s = 0.0;
    for (int blk = 0; blk < nblk; ++blk) s += partials[(long)blk * O + o];
    r2[o] = s * inv_n2;
    if (res_out) res_out[o] = s * inv_n2;
  }
  __syncthreads();
  const int warp = tid >> 5, lane = tid & 31;
  for (int b = warp; b < nb; b += blockDim.x / 32) {
    int best = -1, ok = 0, flags = 0;
    for (int k0 = 0; k0 < na; k0 += 32) {
      const int k = k0 + lane;
      bool good = false, bad = false;
      if (k < na) {
        const double v = r2[b * na + k];
        bad = ((__double_as_longlong(v) >> 52) & 0x7ff) == 0x7ff;
        good = v <= thr.t[b];
      }
      const unsigned bg = __ballot_sync(0xffffffffu, good);
      if (__ballot_sync(0xffffffffu, bad)) flags |= FR3D_INFO_NONFINITE;
      if (bg) best = k0 + 31 - __clz(bg);
      ok += __popc(bg);
    }
    if (best < 0) {
      best = 0;
      flags |= FR3D_INFO_ALPHA_NONE_SATISFIES;
    } else if (ok == na) {
      flags |= FR3D_INFO_ALPHA_ALL_SATISFY;
    }
    if (lane == 0) {
      aidx[b] = best;
      flg[b] = flags;
    }
  }
  __syncthreads();
  if (tid == 0) {
    int flags = 0;
    for (int b = 0; b < nb; ++b) flags |= flg[b];
    if (info) *info = flags | (*info & keep);   // keep: bits set earlier in this call (cleared at its start)
  }
}

// zeta~_j(bin, q) = sum_i W_c[i][j] g_i p_i(bin, q) / n^2 with g_i of the class's band alpha, written to
// the spectra Zs [q][j][bin] (jq = 0: the fused inverse's order) or [j][q][bin] (jq = 1: the order of the
// two-pass inverse).  One warp per class: the scaled projected data g_i p_i of the members
// for one q sit in the warp's shared-memory slice, lane l owns depths j = j0 + l, j0 + l + 32 of a
// 64-depth chunk, and W_c (stored [i][j]) streams from global memory in coalesced rows, each element
// feeding every member.
__global__ void __launch_bounds__(256) k_solve_m(const float2* __restrict__ P, long ps, int Q, int M, int Mp, int n,
                                                 int Cn, const double* __restrict__ lam, const float* __restrict__ W,
                                                 const unsigned char* __restrict__ cband, int nb,
                                                 const int* __restrict__ aidx, int na, MAlphas al,
                                                 const double* __restrict__ s2, int ra, double inv_n2,
                                                 float2* __restrict__ Zs, int jq) {
  constexpr int kJ = 2;   // depths per lane in a chunk of 64
  __shared__ float2 xs[kPerCta][4 * kMaxM];
  __shared__ float gs[kPerCta][kMaxM];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = blockIdx.x * kPerCta + warp;
  if (c >= Cn) return;   // a whole warp; the kernel synchronises warps only
  int kxs[4], kys[4];
  float wts[4];
  const int nm = class_members(c, n, kxs, kys, wts);
  long bin[4];
  for (int m = 0; m < 4; ++m) bin[m] = m < nm ? (long)kxs[m] * n + kys[m] : 0;
  float2* x = xs[warp];
  float* g = gs[warp];
  {
    const int k = min(max(aidx[nb > 1 ? (int)cband[c] : 0], 0), na - 1);   // caller-given indices stay in range
    const double t = al.a[k] * (*s2);
    // the TSVD keep decision in FP64 (against the candidate's level), the reciprocal in FP32 (the
    // weights multiply FP32 data and tables)
    for (int i = lane; i < M; i += 32) {
      const double l = lam[(long)c * M + i];
      float gi;
      if (ra == FR3D_RA_TSVD) gi = (l >= t && l > 0.0) ? __frcp_rn((float)l) : 0.f;
      else gi = __frcp_rn((float)(l + t));
      g[i] = gi * (float)inv_n2;
    }
  }
  __syncwarp();
  const float* Wc = W + (long)c * M * Mp;
  for (int q = 0; q < Q; ++q) {
    for (int e = lane; e < nm * M; e += 32) {
      const int m = e / M, i = e - m * M;
      const float2 v = P[((long)q * M + i) * ps + bin[m]];
      x[e] = make_float2(v.x * g[i], v.y * g[i]);
    }
    __syncwarp();
    for (int j0 = 0; j0 < Mp; j0 += 32 * kJ) {
      // rows i0 .. i0 + kBatch - 1 of this depth chunk into buffer b (zeros past M or M')
      float wb[2][kBatch][kJ];
      auto load = [&](int b, int i0) {
#pragma unroll
        for (int u = 0; u < kBatch; ++u)
#pragma unroll
          for (int t = 0; t < kJ; ++t) {
            const int i = i0 + u, jj = j0 + lane + 32 * t;
            wb[b][u][t] = (i < M && jj < Mp) ? __ldg(Wc + (long)i * Mp + jj) : 0.f;
          }
      };
      float2 z[kJ][4];
#pragma unroll
      for (int t = 0; t < kJ; ++t)
#pragma unroll
        for (int m = 0; m < 4; ++m) z[t][m] = make_float2(0.f, 0.f);
      auto fma_batch = [&](int b, int i0) {
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
          const int i = i0 + u;
          if (i < M) {
#pragma unroll
            for (int m = 0; m < 4; ++m) {
              if (m < nm) {
                const float2 xv = x[m * M + i];
#pragma unroll
                for (int t = 0; t < kJ; ++t) {
                  z[t][m].x = fmaf(wb[b][u][t], xv.x, z[t][m].x);
                  z[t][m].y = fmaf(wb[b][u][t], xv.y, z[t][m].y);
                }
              }
            }
          }
        }
      };
      // double-buffered stream: the next batch is requested before the current one is used
      load(0, 0);
      for (int i0 = 0; i0 < M; i0 += 2 * kBatch) {
        load(1, i0 + kBatch);
        fma_batch(0, i0);
        load(0, i0 + 2 * kBatch);
        fma_batch(1, i0 + kBatch);
      }
#pragma unroll
      for (int t = 0; t < kJ; ++t) {
        const int jj = j0 + lane + 32 * t;
        if (jj < Mp)
#pragma unroll
          for (int m = 0; m < 4; ++m)
            if (m < nm) Zs[(jq ? (long)jj * Q + q : (long)q * Mp + jj) * ps + bin[m]] = z[t][m];
      }
    }
    __syncwarp();   // the x reads are done before the next q is gathered
  }
}

}  // namespace

// Eigen tables of every class (built on the first call with M > 1, synchronously).
int ensure_multi_tables(Handle* H, cudaStream_t st) {
  if (H->mlam) return FR3D_OK;
  const int M = H->M, Mp = H->Mp, C = H->C;
  double* lam = nullptr;
  float *Ut = nullptr, *W = nullptr;
  int* sweeps = nullptr;
  cudaError_t e = cudaMalloc(&lam, sizeof(double) * C * M);
  if (e == cudaSuccess) e = cudaMalloc(&Ut, sizeof(float) * C * M * M);
  if (e == cudaSuccess) e = cudaMalloc(&W, sizeof(float) * (size_t)C * M * Mp);
  if (e == cudaSuccess) e = cudaMalloc(&sweeps, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(sweeps, 0, sizeof(int), st);
  const int Me = (M + 1) & ~1;
  const size_t sm = sizeof(double) * 2 * Me * Me;
  int rc = e == cudaSuccess ? FR3D_OK : (e == cudaErrorMemoryAllocation ? FR3D_ERR_OOM : FR3D_ERR_CUDA);
  if (rc == FR3D_OK) rc = smem_optin(reinterpret_cast<const void*>(k_class_eig), sm);
  if (rc == FR3D_OK) {
    k_class_eig<<<C, 256, sm, st>>>(H->A64, M, Mp, C, lam, Ut, W, sweeps);
    int sw = 0;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&sw, sweeps, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      rc = FR3D_ERR_CUDA;
    H->m_sweeps = sw;
  }
  cudaFree(sweeps);
  if (rc != FR3D_OK) {
    cudaFree(lam);
    cudaFree(Ut);
    cudaFree(W);
    return rc;
  }
  H->mlam = lam;
  H->mUt = Ut;
  H->mW = W;
  return FR3D_OK;
}

// workspace of invert_multi: data spectra [Q][M], solved spectra [Q][M'], class powers [C][M]
size_t multi_ws_bytes(const Handle* H, int Q) {
  const size_t ps = (size_t)(H->n / 2 + 1) * H->n;
  auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
  return up(sizeof(float2) * ps * Q * H->M) + up(sizeof(float2) * ps * Q * H->Mp) + up(sizeof(double) * H->C * H->M);
}

namespace {

struct MultiWs {
  float2* Uh;   // [Q][M] half spectra, projected in place
  float2* Zs;   // [Q][M'] solved spectra
  double* Pc;   // [C][M] class powers
};

size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }

int multi_ws(Handle* H, int Q, bool with_zs, MultiWs* w) {
  const long ps = (long)(H->n / 2 + 1) * H->n;
  const size_t ub = up256(sizeof(float2) * ps * Q * H->M);
  const size_t zb = with_zs ? up256(sizeof(float2) * ps * Q * H->Mp) : 0;
  const size_t pb = up256(sizeof(double) * H->C * H->M);
  FR3D_TRY(ensure_ws(H, std::max(ub + zb + pb, with_zs ? multi_ws_bytes(H, Q) : 0)));
  w->Uh = reinterpret_cast<float2*>(H->ws);
  w->Zs = with_zs ? reinterpret_cast<float2*>((char*)H->ws + ub) : nullptr;
  w->Pc = reinterpret_cast<double*>((char*)H->ws + ub + zb);
  return FR3D_OK;
}

// data spectra of every (q, i) plane and their projection onto the class eigenvectors
int multi_data(Handle* H, const float* U, int Q, const MultiWs& w, int precision, int* info, int* launches,
               cudaStream_t st) {
  const long ps = (long)(H->n / 2 + 1) * H->n;
  FR3D_TRY(Ops<float>::row_r2c(H, U, (long)H->n * H->n, w.Uh, Q * H->M, st));
  prof_mark(H, kStRowR2C, st);
  FR3D_TRY(Ops<float>::col_plain(H, w.Uh, w.Uh, Q * H->M, false, st));
  prof_mark(H, kStColFwd, st);
  if (tc_precision(precision)) {
    FR3D_TRY(tc_project(H, w.Uh, Q, w.Pc, precision == FR3D_PREC_BF16X3, info, st));
  } else {
    k_project<<<(H->C + kPerCta - 1) / kPerCta, 32 * kPerCta, 0, st>>>(w.Uh, ps, Q, H->M, H->n, H->C, H->mUt, w.Pc);
    FR3D_CUDA_TRY(cudaGetLastError());
  }
  prof_mark(H, kStOther, st);
  *launches += 3;
  return FR3D_OK;
}

int multi_alpha(Handle* H, const MultiWs& w, const double* alphas, int na, int ra, int nb, const double* thr2,
                int* aidx, double* residuals, int* info, int keep, cudaStream_t st) {
  FR3D_TRY(ensure_partials(H));
  MAlphas al;
  for (int k = 0; k < na; ++k) al.a[k] = alphas[k];
  const int nblk = (H->C + kMCPB - 1) / kMCPB;
  k_alpha_m_partial<<<nblk, kMThreads, 0, st>>>(H->mlam, w.Pc, H->M, H->C, H->cband, nb, al, H->s2, na, ra, H->partials);
  MThr t;
  for (int b = 0; b < nb; ++b) t.t[b] = thr2[b];
  k_alpha_m_finish<<<1, 256, 0, st>>>(H->partials, nblk, nb, na, 1.0 / ((double)H->n * H->n), t, aidx, residuals,
                                      info, keep);
  FR3D_CUDA_TRY(cudaGetLastError());
  prof_mark(H, kStAlpha, st);
  return FR3D_OK;
}

}  // namespace

// Algorithm 1 for M > 1 (FP32 data and FFTs, FP64 eigen tables and residual sums).
// The combination table (XI) is built by the caller.
int invert_multi(Handle* H, const float* U, int Q, const fr3d_invert_opts* o, float* out, const SrcHost& src,
                 cudaStream_t st) {
  FR3D_TRY(ensure_multi_tables(H, st));
  const int nb = o->n_bands > 1 ? o->n_bands : 1;
  std::vector<double> count;
  FR3D_TRY(ensure_bands(H, nb, &count));
  MultiWs w;
  FR3D_TRY(multi_ws(H, Q, true, &w));
  const bool tcp = tc_precision(o->precision);
  if (tcp) {
    FR3D_TRY(ensure_tc_tables(H, 0, st));
    FR3D_TRY(ensure_tc_tables(H, 1, st));
  }
  int launches = 0;
  prof_begin(H, st);
  // the tensor-core kernels OR a time-out bit into info: clear it first
  if (tcp && o->info) {
    FR3D_CUDA_TRY(cudaMemsetAsync(o->info, 0, sizeof(int), st));
    ++launches;
  }
  FR3D_TRY(multi_data(H, U, Q, w, o->precision, o->info, &launches, st));
  MAlphas al;
  const int* aidx;
  if (o->alpha_mode == FR3D_ALPHA_FIXED) {
    al.a[0] = o->alpha;
    aidx = H->zero_idx;
    if (o->alpha_idx) FR3D_CUDA_TRY(cudaMemsetAsync(o->alpha_idx, 0, sizeof(int), st));
    if (o->info && !tcp) FR3D_CUDA_TRY(cudaMemsetAsync(o->info, 0, sizeof(int), st));
  } else {
    for (int k = 0; k < o->n_alpha; ++k) al.a[k] = o->alphas[k];
    if (o->alpha_mode == FR3D_ALPHA_DISCREPANCY) {
      int* idx = o->alpha_idx ? o->alpha_idx : H->idx_scratch;
      double thr2[FR3D_MAX_BANDS];
      band_thresholds(H, o, nb, thr2);
      FR3D_TRY(multi_alpha(H, w, o->alphas, o->n_alpha, o->ra, nb, thr2, idx, o->residuals, o->info,
                           tcp ? FR3D_INFO_TIMEOUT : 0, st));
      launches += 2;
      aidx = idx;
    } else {
      aidx = o->alpha_idx;
      if (o->info && !tcp) FR3D_CUDA_TRY(cudaMemsetAsync(o->info, 0, sizeof(int), st));
    }
  }
  const long ps = (long)(H->n / 2 + 1) * H->n;
  const int na = o->alpha_mode == FR3D_ALPHA_FIXED ? 1 : o->n_alpha;
  const bool fused = fused_supported(H->n);
  if (tcp) {
    FR3D_TRY(tc_solve(H, w.Uh, Q, aidx, al.a, na, o->ra, nb, w.Zs, fused ? 0 : 1, o->precision == FR3D_PREC_BF16X3,
                      o->info, st));
  } else {
    k_solve_m<<<(H->C + kPerCta - 1) / kPerCta, 32 * kPerCta, 0, st>>>(
        w.Uh, ps, Q, H->M, H->Mp, H->n, H->C, H->mlam, H->mW, H->cband, nb, aidx, na, al, H->s2, o->ra,
        1.0 / ((double)H->n * H->n), w.Zs, fused ? 0 : 1);
    FR3D_CUDA_TRY(cudaGetLastError());
  }
  prof_mark(H, kStColSolve, st);
  if (fused) {
    FR3D_TRY(inv_fused_presolved_f32(H, w.Zs, H->wtab, out, Q, o->output, st));
    prof_mark(H, kStFused, st);
    H->last_launches = launches + 2;
    return FR3D_OK;
  }
  // other sizes: the inverse column pass in place, then the row pass with the source combination (XI)
  // or per source (ZETA); the solved spectra already carry 1/n^2
  FR3D_TRY(Ops<float>::col_plain(H, w.Zs, w.Zs, Q * H->Mp, true, st));
  prof_mark(H, kStColInv, st);
  if (o->output == FR3D_OUT_XI)
    FR3D_TRY(Ops<float>::row_c2r_xi(H, w.Zs, out, H->Mp, Q, 0, src, st));
  else
    FR3D_TRY(Ops<float>::row_c2r_plain(H, w.Zs, out, H->Mp * Q, Q, 0, H->Mp, st));
  prof_mark(H, kStRowC2R, st);
  H->last_launches = launches + 3;
  return FR3D_OK;
}

// Discrepancy choice alone for M > 1 (fr3d_choose_alpha): data FFT, projection, residual sums.
int choose_multi(Handle* H, const float* U, int Q, const double* alphas, int na, double delta, double tau,
                 int precision, int* aidx, double* residuals, int* info, cudaStream_t st) {
  FR3D_TRY(ensure_multi_tables(H, st));
  FR3D_TRY(ensure_bands(H, 1, nullptr));
  const bool tcp = tc_precision(precision);
  if (tcp) FR3D_TRY(ensure_tc_tables(H, 0, st));
  MultiWs w;
  FR3D_TRY(multi_ws(H, Q, false, &w));
  int launches = 0;
  prof_begin(H, st);
  if (tcp && info) {
    FR3D_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(int), st));
    ++launches;
  }
  FR3D_TRY(multi_data(H, U, Q, w, precision, info, &launches, st));
  const double thr2 = (tau * delta) * (tau * delta);
  FR3D_TRY(multi_alpha(H, w, alphas, na, FR3D_RA_TIKHONOV, 1, &thr2, aidx, residuals, info,
                       tcp ? FR3D_INFO_TIMEOUT : 0, st));
  H->last_launches = launches + 2;
  return FR3D_OK;
}

}  // namespace fr3d
