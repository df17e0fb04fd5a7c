// Per-precision kernel launchers (included once per precision by ops_f32.cu / ops_f64.cu).
#pragma once

#include <cooperative_groups.h>

#include <type_traits>

#include "fft2d.cuh"
#include "ops.cuh"

namespace fr3d {

#define FR3D_FOR_EACH_N(X) X(16) X(24) X(32) X(48) X(64) X(96) X(128) X(192) X(256) X(384) X(512)

template <typename K> static int set_smem(K kernel, size_t bytes) {
  return smem_optin(reinterpret_cast<const void*>(kernel), bytes);
}

template <typename T> static const typename cpx<T>::t* tw_of(const Handle* H, int L) {
  const int off = twiddle_offset(H, L);
  if constexpr (sizeof(T) == 4) return H->tw32 + off;
  else return H->tw64 + off;
}

constexpr int kSmallGrid = 2 * 152;  // below this many CTAs with the large tile, use the small one

template <typename T, int N, int TY, class PM = StridedPlanes<T>>
static int row_r2c_t(const Handle* H, const PM& pm, int nplanes, cudaStream_t st) {
  constexpr size_t sm = row_r2c_smem<T, N, TY>();
  auto kern = k_row_r2c<T, N, TY, PM>;
  FR3D_TRY(set_smem(kern, sm));
  dim3 grid(N / TY, nplanes);
  kern<<<grid, kThreads, sm, st>>>(pm, tw_of<T>(H, N));
  return cudaGetLastError() == cudaSuccess ? FR3D_OK : FR3D_ERR_CUDA;
}

template <typename T, int N>
static int row_r2c_n(const Handle* H, const T* in, long in_ps, typename cpx<T>::t* out, int nplanes, cudaStream_t st) {
  constexpr int TY = RowTile<T, N>::v;
  const StridedPlanes<T> pm{in, in_ps, out, (long)(N / 2 + 1) * N};
  if ((long)nplanes * (N / TY) < kSmallGrid && SmallTile<N>::row < TY)
    return row_r2c_t<T, N, SmallTile<N>::row>(H, pm, nplanes, st);
  return row_r2c_t<T, N, TY>(H, pm, nplanes, st);
}

template <typename T, int N, bool INV, class Op, int TC>
static int col_t(const Handle* H, const Op& op, int nplanes, cudaStream_t st) {
  constexpr size_t sm = col_smem<T, N, TC>();
  auto kern = k_col_fft<T, N, INV, Op, TC>;
  FR3D_TRY(set_smem(kern, sm));
  dim3 grid((N / 2 + 1 + TC - 1) / TC, nplanes);
  kern<<<grid, kThreads, sm, st>>>(op, tw_of<T>(H, N));
  return cudaGetLastError() == cudaSuccess ? FR3D_OK : FR3D_ERR_CUDA;
}

template <typename T, int N, bool INV, class Op>
static int col_n(const Handle* H, const Op& op, int nplanes, cudaStream_t st) {
  constexpr int TC = ColTile<T, N>::v;
  if ((long)nplanes * ((N / 2 + TC) / TC) < kSmallGrid && SmallTile<N>::col < TC)
    return col_t<T, N, INV, Op, SmallTile<N>::col>(H, op, nplanes, st);
  return col_t<T, N, INV, Op, TC>(H, op, nplanes, st);
}

template <typename T, int N, int MODE>
static int row_c2r_n(const Handle* H, const typename cpx<T>::t* in, T* out, int nplanes, int Q, int j0,
                     int out_stride, const SrcHost& src, cudaStream_t st) {
  constexpr size_t sm = row_c2r_smem<T, N, MODE>();
  auto kern = k_row_c2r<T, N, MODE>;
  FR3D_TRY(set_smem(kern, sm));
  typename SrcOf<T>::t s;
  s.pts = reinterpret_cast<decltype(s.pts)>(src.pts);
  s.L = src.L;
  s.coef = (T)src.coef;
  RowGeom g{H->x0, H->y0, H->h};
  const T* zr;
  if constexpr (sizeof(T) == 4) zr = H->zr32;
  else zr = H->zr64;
  dim3 grid(N / row_c2r_tile<T, N, MODE>(), nplanes);
  kern<<<grid, kThreads, sm, st>>>(in, out, Q, j0, out_stride, s, g, zr, tw_of<T>(H, N / 2), tw_of<T>(H, N));
  return cudaGetLastError() == cudaSuccess ? FR3D_OK : FR3D_ERR_CUDA;
}

template <typename T>
int Ops<T>::row_r2c(const Handle* H, const T* in, long in_ps, C* out, int nplanes, cudaStream_t st) {
  switch (H->n) {
#define X(N) \
  case N: return row_r2c_n<T, N>(H, in, in_ps, out, nplanes, st);
    FR3D_FOR_EACH_N(X)
#undef X
  }
  return FR3D_ERR_UNSUPPORTED_SIZE;
}

template <typename T>
int Ops<T>::col_plain(const Handle* H, const C* in, C* out, int nplanes, bool inverse, cudaStream_t st) {
  ColPlain<T> op{in, out, (long)(H->n / 2 + 1) * H->n};
  switch (H->n) {
#define X(N)                                                         \
  case N:                                                            \
    return inverse ? col_n<T, N, true>(H, op, nplanes, st) : col_n<T, N, false>(H, op, nplanes, st);
    FR3D_FOR_EACH_N(X)
#undef X
  }
  return FR3D_ERR_UNSUPPORTED_SIZE;
}

template <typename T>
int Ops<T>::col_solve1(const Handle* H, const C* Uh, C* out, const T* A, const T* D, const int* aidx, int nb, int Q,
                       int j0, int nj, cudaStream_t st) {
  ColSolve1<T> op;
  op.cband = H->cband;
  op.nb = nb;
  op.Uh = Uh;
  op.out = out;
  op.A = A;
  op.D = D;
  op.aidx = aidx;
  op.ps = (long)(H->n / 2 + 1) * H->n;
  op.Q = Q;
  op.j0 = j0;
  op.n = H->n;
  op.Cn = H->C;
  op.drow = nullptr;
  switch (H->n) {
#define X(N) \
  case N: return col_n<T, N, true>(H, op, nj * Q, st);
    FR3D_FOR_EACH_N(X)
#undef X
  }
  return FR3D_ERR_UNSUPPORTED_SIZE;
}

template <typename T>
int Ops<T>::row_c2r_plain(const Handle* H, const C* in, T* out, int nplanes, int Q, int j0, int out_stride,
                          cudaStream_t st) {
  SrcHost none{nullptr, 0, 0.0};
  switch (H->n) {
#define X(N) \
  case N: return row_c2r_n<T, N, 0>(H, in, out, nplanes, Q, j0, out_stride, none, st);
    FR3D_FOR_EACH_N(X)
#undef X
  }
  return FR3D_ERR_UNSUPPORTED_SIZE;
}

template <typename T>
int Ops<T>::row_c2r_xi(const Handle* H, const C* in, T* out, int nj, int Q, int j0, const SrcHost& src,
                       cudaStream_t st) {
  switch (H->n) {
#define X(N) \
  case N: return row_c2r_n<T, N, 1>(H, in, out, nj, Q, j0, 0, src, st);
    FR3D_FOR_EACH_N(X)
#undef X
  }
  return FR3D_ERR_UNSUPPORTED_SIZE;
}

// ---------------------------------------------------------------- forward contraction (Eq. (5)-(6))
template <typename T, typename C>
__global__ void k_contract_fwd(const C* __restrict__ Zh, C* __restrict__ Uh, const T* __restrict__ A, int Q, int M,
                               int Mp, long ps, T inv_n2) {
  const long total = (long)Q * M * ps;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const long bin = idx % ps;
    const int qi = (int)(idx / ps);
    const int q = qi / M, i = qi - q * M;
    const C* z = Zh + (long)q * Mp * ps + bin;
    const T* a = A + (long)i * Mp * ps + bin;
    T re = 0, im = 0;
    for (int j = 0; j < Mp; ++j) {
      const T w = a[(long)j * ps];
      const C v = z[(long)j * ps];
      re += w * v.x;
      im += w * v.y;
    }
    C r;
    r.x = re * inv_n2;
    r.y = im * inv_n2;
    Uh[idx] = r;
  }
}

template <typename T>
int Ops<T>::contract_fwd(const Handle* H, const C* Zh, C* Uh, const T* A, int Q, cudaStream_t st) {
  const long ps = (long)(H->n / 2 + 1) * H->n;
  const long total = (long)Q * H->M * ps;
  const int blocks = (int)std::min<long>((total + 255) / 256, 152L * 16);
  k_contract_fwd<T, C><<<blocks, 256, 0, st>>>(Zh, Uh, A, Q, H->M, H->Mp, ps, (T)(1.0 / ((double)H->n * H->n)));
  return cudaGetLastError() == cudaSuccess ? FR3D_OK : FR3D_ERR_CUDA;
}

// ---------------------------------------------------------------- zeta = xi V0 (Sec. 2)
template <typename T, typename S>
__global__ void k_zeta_from_xi(const T* __restrict__ xi, T* __restrict__ zeta, int Q, int Mp, int n, S src,
                               RowGeom g, const T* __restrict__ zr) {
  const long plane = (long)n * n;
  const long total = (long)Q * Mp * plane;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const long pix = idx % plane;
    const int qj = (int)(idx / plane);
    const int q = qj / Mp, j = qj - q * Mp;
    const int a = (int)(pix % n), b = (int)(pix / n);
    const T x = (T)g.x0 + ((T)a + (T)0.5) * (T)g.h, y = (T)g.y0 + ((T)b + (T)0.5) * (T)g.h;
    zeta[idx] = xi[(long)j * plane + pix] * v0_at(src, q, x, y, zr[j]);
  }
}

template <typename T>
int Ops<T>::zeta_from_xi(const Handle* H, const T* xi, T* zeta, int Q, const SrcHost& src, cudaStream_t st) {
  typename SrcOf<T>::t s;
  s.pts = reinterpret_cast<decltype(s.pts)>(src.pts);
  s.L = src.L;
  s.coef = (T)src.coef;
  RowGeom g{H->x0, H->y0, H->h};
  const T* zr;
  if constexpr (sizeof(T) == 4) zr = H->zr32;
  else zr = H->zr64;
  const long total = (long)Q * H->Mp * H->n * H->n;
  const int blocks = (int)std::min<long>((total + 255) / 256, 152L * 16);
  k_zeta_from_xi<T><<<blocks, 256, 0, st>>>(xi, zeta, Q, H->Mp, H->n, s, g, zr);
  return cudaGetLastError() == cudaSuccess ? FR3D_OK : FR3D_ERR_CUDA;
}

// ---------------------------------------------------------------- discrepancy principle (Sec. 4)
// (p, q) of class c = p (p + 1) / 2 + q, q <= p (exact integer correction of a float estimate)
__device__ __forceinline__ void class_pq(int c, int& p, int& q) {
  p = (int)((sqrtf(8.f * (float)c + 1.f) - 1.f) * 0.5f);
  while ((p + 1) * (p + 2) / 2 <= c) ++p;
  while (p * (p + 1) / 2 > c) --p;
  q = c - p * (p + 1) / 2;
}

__device__ __forceinline__ double sq_abs(float2 v) { return (double)fmaf(v.x, v.x, v.y * v.y); }
__device__ __forceinline__ double sq_abs(double2 v) { return fma(v.x, v.x, v.y * v.y); }

constexpr int kAlphaCPB = 64;  // classes per block
constexpr int kAlphaSplit = 4; // threads per class in the power gather
constexpr int kAlphaGroup = 8;   // blocks per group of the two-level reduction
static_assert(kAlphaCPB == 64 && kAlphaGroup == 8,
              "ensure_partials sizes the partial-sum buffer for 64 classes per block and 8 blocks per group");
static_assert(256 / kAlphaSplit >= kAlphaCPB, "every class of a block has its gather threads");

// Per band b of frequency classes (one band: the whole spectrum),
//   r_b^2(alpha_k) = n^-2 sum_{c in b} Ft[c][k] P[c]  (Parseval; M = 1 closed form of the residual),
// with P[c] the data power of class c: every stored half-spectrum bin of the class, weighted 1 on
// the kx = 0 and kx = n/2 columns and 2 elsewhere (their mirror bins are not stored), summed over
// planes.  The discrepancy rule picks, per band, the largest alpha_k with r_b^2 <= thr2.t[b].
// Deterministic: fixed-order partial sums per block; per group of kAlphaGroup consecutive blocks, in
// block order, by the group's last block to finish (an atomic ticket per group); over the groups, in
// group order, by the last group to finish.  The tickets leave the blocks free to land on distinct
// SMs (an 8-block cluster per group placed two blocks on some SMs and added two cluster barriers).
// FP64 runs at a small fraction of the FP32 rate on this GPU, so the serial parts avoid FP64 chains:
// the choice is a warp ballot per band rather than a loop over candidates.
struct BandThr {
  double t[FR3D_MAX_BANDS];
};

// blocks of the alpha rule for Cn classes: one per kAlphaCPB classes
inline int alpha_blocks(int Cn) { return (Cn + kAlphaCPB - 1) / kAlphaCPB; }
__host__ __device__ inline int alpha_groups(int nblk) { return (nblk + kAlphaGroup - 1) / kAlphaGroup; }
// the group tickets of the alpha rule in the handle's partial-sum buffer (tables.cu)
unsigned* alpha_tickets(const Handle* H);

template <typename C>
__device__ __forceinline__ void alpha_choose_body(const C* __restrict__ Uh, long ps, int nplanes, int n, int Cn,
                                                  const double* __restrict__ Ft, int na, const BandThr& thr2,
                                                  const unsigned char* __restrict__ cband, int nb, double inv_n2,
                                                  double* __restrict__ partials, unsigned* __restrict__ counter,
                                                  int* __restrict__ aidx, double* __restrict__ res_out,
                                                  int* __restrict__ info, unsigned* __restrict__ gticket, int blk,
                                                  int nblk) {
  // partials: [nblk][O] block sums, then [groups][O] group sums; gticket: one ticket per group
  // (alpha_tickets); counter: the ticket over the groups.  Every ticket is zero between launches.
  // Accumulation types: the class power P[c] is summed in the data's precision (at most 4 nplanes
  // positive terms); the residual sums F[c][k] P[c] over classes and blocks are FP64.
  using A = typename std::conditional<std::is_same<C, float2>::value, float, double>::type;
  __shared__ double sP[kAlphaCPB];
  __shared__ unsigned char sB[kAlphaCPB];
  __shared__ int present[FR3D_MAX_BANDS];
  __shared__ double red[256];
  __shared__ double sPart[FR3D_MAX_BANDS * FR3D_MAX_ALPHAS];   // this block's sums; later the r^2 curves
  __shared__ int flg[FR3D_MAX_BANDS];
  __shared__ bool last;
  extern __shared__ double sF[];             // [kAlphaCPB][na] slab of Ft for this block's classes
  const int tid = threadIdx.x;
  const int c0 = blk * kAlphaCPB;
  const int nF = max(0, min(kAlphaCPB, Cn - c0)) * na;
  const double* slab = Ft + (long)c0 * na;
  const int O = nb * na;
  if (tid < FR3D_MAX_BANDS) present[tid] = 0;
  // one round of global loads: this thread's share of the class powers and of the filter slab
  const int cl = tid / kAlphaSplit, sub = tid % kAlphaSplit, c = c0 + cl;
  const bool own = cl < kAlphaCPB;            // threads past the block's classes gather nothing
  int kxs[4] = {0, 0, 0, 0}, kys[4] = {0, 0, 0, 0}, nm = 0;
  if (own && c < Cn) {
    int p, q;
    class_pq(c, p, q);
    // members (kx, ky) of the class in the half spectrum
    kxs[nm] = p; kys[nm++] = q;
    if (q != 0 && 2 * q != n) { kxs[nm] = p; kys[nm++] = n - q; }
    if (p != q) {
      kxs[nm] = q; kys[nm++] = p;
      if (p != 0 && 2 * p != n) { kxs[nm] = q; kys[nm++] = n - p; }
    }
  }
  double f[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const int e = tid + i * 256;
    f[i] = e < nF ? __ldg(slab + e) : 0.0;
  }
  A acc = 0;
  for (int pl0 = sub; pl0 < nplanes; pl0 += 2 * kAlphaSplit) {
    A s[4][2];
#pragma unroll
    for (int mi = 0; mi < 4; ++mi)
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int pl = pl0 + u * kAlphaSplit;
        const C v = (mi < nm && pl < nplanes) ? __ldg(Uh + pl * ps + (long)kxs[mi] * n + kys[mi]) : C{0, 0};
        s[mi][u] = v.x * v.x + v.y * v.y;
      }
#pragma unroll
    for (int mi = 0; mi < 4; ++mi)
      if (mi < nm) acc += ((kxs[mi] == 0 || 2 * kxs[mi] == n) ? A(1) : A(2)) * (s[mi][0] + s[mi][1]);
  }
  // the kAlphaSplit threads of a class are adjacent lanes: combine them in a fixed order
#pragma unroll
  for (int m = 1; m < kAlphaSplit; m <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, m);
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const int e = tid + i * 256;
    if (e < nF) sF[e] = f[i];
  }
  // slabs longer than 16 loads per thread (more than 64 candidates) finish here
  for (int e = tid + 16 * 256; e < nF; e += 256) sF[e] = __ldg(slab + e);
  if (sub == 0 && own) {
    sP[cl] = (double)acc;
    const int b = (c < Cn && nb > 1) ? (int)cband[c] : 0;
    sB[cl] = (unsigned char)b;
    if (c < Cn) present[b] = 1;
  }
  __syncthreads();
  // per band: this block's sums of F[c][k] P[c] (S threads per candidate, fixed order)
  const int S = 256 / na;
  for (int b = 0; b < nb; ++b) {
    if (present[b]) {
      if (tid < S * na) {
        const int k = tid % na, sb = tid / na;
        double a2 = 0.0;
        for (int cc = sb; cc < kAlphaCPB; cc += S)
          if (c0 + cc < Cn && sB[cc] == b) a2 = fma(sF[cc * na + k], sP[cc], a2);
        red[tid] = a2;
      }
      __syncthreads();
    }
    if (tid < na) {
      double s = 0.0;
      if (present[b])
        for (int sb = 0; sb < S; ++sb) s += red[sb * na + tid];
      sPart[b * na + tid] = s;
    }
    __syncthreads();
  }
  // level 1: this block's sums, then a ticket of its group; the group's last block adds the group's
  // block sums in block order
  const int ngr = alpha_groups(nblk);
  double* gpart = partials + (long)nblk * O;
  for (int o = tid; o < O; o += 256) partials[(long)blk * O + o] = sPart[o];
  __threadfence();
  __syncthreads();
  const int g = blk / kAlphaGroup;
  const int gsz = min(kAlphaGroup, nblk - g * kAlphaGroup);
  if (tid == 0) last = atomicAdd(gticket + g, 1u) == (unsigned)(gsz - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int o = tid; o < O; o += 256) {
    double v[kAlphaGroup];
#pragma unroll
    for (int q = 0; q < kAlphaGroup; ++q) v[q] = q < gsz ? __ldcg(partials + (long)(g * kAlphaGroup + q) * O + o) : 0.0;
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < kAlphaGroup; ++q)
      if (q < gsz) s += v[q];
    gpart[(long)g * O + o] = s;
  }
  // level 2: a ticket over the groups
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    gticket[g] = 0u;
    last = atomicAdd(counter, 1u) == (unsigned)(ngr - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // every other block has finished: let a programmatically launched successor start its set-up
  pdl_release();
  // the last group: r^2 per (band, candidate) over the group sums (24 loads in flight per round)
  for (int o = tid; o < O; o += 256) {
    double s = 0.0;
    for (int g0 = 0; g0 < ngr; g0 += 24) {
      double v[24];
#pragma unroll
      for (int i = 0; i < 24; ++i) v[i] = g0 + i < ngr ? __ldcg(gpart + (long)(g0 + i) * O + o) : 0.0;
#pragma unroll
      for (int i = 0; i < 24; ++i) s += v[i];
    }
    s *= inv_n2;
    sPart[o] = s;
    if (res_out) res_out[o] = s;
  }
  __syncthreads();
  // choice per band, one warp per band: ballots of r^2 <= thr over the candidates, largest index wins
  const int warp = tid >> 5, lane = tid & 31;
  for (int b = warp; b < nb; b += 8) {
    int best = -1, ok = 0, flags = 0;
    for (int k0 = 0; k0 < na; k0 += 32) {
      const int k = k0 + lane;
      bool good = false, bad = false;
      if (k < na) {
        const double v = sPart[b * na + k];
        const long long bits = __double_as_longlong(v);
        bad = ((bits >> 52) & 0x7ff) == 0x7ff;      // Inf or NaN
        good = v <= thr2.t[b];
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
    if (info) *info = flags;
    *counter = 0u;
  }
}

template <typename C>
__global__ void __launch_bounds__(256) k_alpha_choose(const C* __restrict__ Uh, long ps, int nplanes, int n, int Cn,
                                                      const double* __restrict__ Ft, int na, BandThr thr2,
                                                      const unsigned char* __restrict__ cband, int nb, double inv_n2,
                                                      double* __restrict__ partials, unsigned* __restrict__ counter,
                                                      int* __restrict__ aidx, double* __restrict__ res_out,
                                                      int* __restrict__ info, unsigned* __restrict__ gticket) {
  alpha_choose_body(Uh, ps, nplanes, n, Cn, Ft, na, thr2, cband, nb, inv_n2, partials, counter, aidx, res_out, info,
                    gticket, (int)blockIdx.x, (int)gridDim.x);
}

template <typename T>
int Ops<T>::alpha_choose(Handle* H, const C* Uh, int nplanes, int n_alpha, const double* thr2, int nb, int* aidx,
                         double* residuals, int* info, cudaStream_t st) {
  const int blocks = alpha_blocks(H->C);
  FR3D_TRY(ensure_partials(H));
  const long ps = (long)(H->n / 2 + 1) * H->n;
  const size_t sm = sizeof(double) * kAlphaCPB * n_alpha;
  FR3D_TRY(set_smem(k_alpha_choose<C>, sm));
  BandThr t;
  for (int b = 0; b < nb; ++b) t.t[b] = thr2[b];
  k_alpha_choose<C><<<blocks, 256, sm, st>>>(Uh, ps, nplanes, H->n, H->C, H->Ft, n_alpha, t, H->cband, nb,
                                            1.0 / ((double)H->n * H->n), H->partials, H->counter, aidx, residuals,
                                            info, alpha_tickets(H));
  return cudaGetLastError() == cudaSuccess ? FR3D_OK : FR3D_ERR_CUDA;
}

}  // namespace fr3d
