// Steps 2-4 of Algorithm 1 at M = 1 (FP32) as two streaming passes through HBM: the fifth variant of the
// inverse that the autotuner weighs against the fused cluster kernel (fused.cuh).
//
// Pass 1 (k_inv2_col): per source parameter q, depth j and tile of CA frequency columns kx: the solve
// (U~_q(kx, ky) times w_j(kx, ky) = A_j(kx, ky) D_alpha(kx, ky), 1/n^2 folded into D) loaded straight into the
// first pass of the inverse DFT along ky, the other passes in shared memory, and the result written as
// rows of the intermediate T[q][j][y][kx] (kx = 0 carries kx = 0 in its real part and kx = n/2 in its
// imaginary part: both columns are Hermitian in ky, so one complex DFT gives both).
// Pass 2 (k_inv2_row): per depth j and batch of RB rows y: for every q the row's n/2 values of T, the
// Hermitian split into one n/2-point complex sequence, the inverse DFT, and (xi output) the combination
// sum_q W_q(x) zeta_q(x) accumulated in registers and written once (zeta output: each q written).
// Every pass reads and writes HBM with whole rows (no clusters, no distributed shared memory): its
// bytes are the two-pass figure of the inverse (the intermediate written and read once) plus the
// combination table.
#include "fused.cuh"
#include "ops.cuh"

namespace fr3d {

namespace {

constexpr int kColThreads = 256;
constexpr int kRowThreads = 128;
constexpr int kRB = 8;   // rows per block of pass 2

template <int N> struct Inv2Geom {
  static constexpr int L = N / 2;
  static constexpr int CA = L <= 16 ? L : (L % 16 == 0 ? 16 : 12);   // columns per block of pass 1
  static constexpr int SSC = PaddedLen<N, float2>::v + 1;            // odd: transposed reads free of conflicts
  static constexpr int SSR = PaddedLen<L, float2>::v;
  static constexpr int PTC = passtw_size<N>() > 0 ? passtw_size<N>() : 1;
  static constexpr int PTR = passtw_size<L>() > 0 ? passtw_size<L>() : 1;
  static constexpr size_t smem_col = sizeof(float2) * ((size_t)CA * SSC + PTC);
  static constexpr size_t smem_row = sizeof(float2) * ((size_t)kRB * SSR + N + PTR);
};

struct Inv2Args {
  const float2* Uh;            // [Q][n/2+1][n] data spectra
  const float* A;              // [M'][n/2+1][n] dense kernel table
  const float* Dd;             // [n_alpha][n/2+1][n] solve weights (1/n^2 folded in)
  const int* aidx;
  int na;
  const unsigned char* bbin;   // [n/2+1][n] band of every bin (nb > 1)
  int nb;
  const float* W;              // [Q][M'][n][n] combination weights (XI)
  float* out;
  const float2* tw_n;          // length-n twiddles
  float2* T;                   // [Q][nj][n][n/2] intermediate
  int Q, j0, nj, Mp;
};

template <int N>
__global__ void __launch_bounds__(kColThreads) k_inv2_col(Inv2Args a) {
  using G = Inv2Geom<N>;
  constexpr int L = G::L, CA = G::CA, SSC = G::SSC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* colbuf = reinterpret_cast<float2*>(smem_raw);
  float2* ptc = colbuf + CA * SSC;
  __shared__ int s_aidx[FR3D_MAX_BANDS];
  const int tid = threadIdx.x;
  const int plane = blockIdx.x;              // q * nj + jl
  const int q = plane / a.nj, jl = plane - q * a.nj, j = a.j0 + jl;
  const int c0 = blockIdx.y * CA;
  const long ps = (long)(L + 1) * N;
  build_passtw<N, 1, kColThreads>(ptc, a.tw_n, tid);
  pdl_wait();
  if (tid < a.nb) s_aidx[tid] = min(max(a.aidx[tid], 0), a.na - 1);
  __syncthreads();
  const float2* Uq = a.Uh + (long)q * ps;
  const float* Aj = a.A + (long)j * ps;
  auto wt = [&](long o) -> float {
    const int row = a.nb > 1 ? s_aidx[__ldg(a.bbin + o)] : s_aidx[0];
    return __fmul_rn(__ldg(Aj + o), __ldg(a.Dd + (long)row * ps + o));
  };
  auto ldc = [&](int s, int ky) -> float2 {
    const long o = (long)(c0 + s) * N + ky;
    const float2 u = __ldg(Uq + o);
    const float w = wt(o);
    float2 v = make_float2(__fmul_rn(u.x, w), __fmul_rn(u.y, w));
    if (c0 + s == 0) {   // packed column 0: add i w(n/2, ky) U~(n/2, ky)
      const long oL = (long)L * N + ky;
      const float2 un = __ldg(Uq + oL);
      const float wl = wt(oL);
      v.x = __fmaf_rn(-un.y, wl, v.x);
      v.y = __fmaf_rn(un.x, wl, v.y);
    }
    return v;
  };
  first_pass_from<N, true, CA, kColThreads>(colbuf, SSC, ldc, tid);
  fft_passes<N, true, CA, kColThreads, 1, Plan<N>::np, Plan<N>::radix(0)>(colbuf, SSC, ptc, tid);
  // rows of T: CA consecutive columns per row y (coalesced writes; the odd stride keeps the reads of
  // consecutive columns in distinct banks)
  float2* Tp = a.T + (long)plane * N * L;
  for (int e = tid; e < CA * N; e += kColThreads) {
    const int y = e / CA, s = e - y * CA;
    Tp[(long)y * L + c0 + s] = colbuf[s * SSC + pidx<float2>(y)];
  }
}

template <int N, int MODE>
__global__ void __launch_bounds__(kRowThreads) k_inv2_row(Inv2Args a) {
  using G = Inv2Geom<N>;
  constexpr int L = G::L, SSR = G::SSR;
  using LP = LastPass<L>;
  constexpr int NBF = kRB * LP::BPS;                       // butterflies of the last pass
  constexpr int KR = (NBF + kRowThreads - 1) / kRowThreads;
  constexpr int NK = L / 2 + 1;                            // Hermitian-split pairs (k, L - k), k <= L/2
  constexpr int NSPL = kRB * NK;
  constexpr int SIT = (NSPL + kRowThreads - 1) / kRowThreads;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* rowbuf = reinterpret_cast<float2*>(smem_raw);
  float2* tws = rowbuf + kRB * SSR;
  float2* ptr = tws + N;
  const int tid = threadIdx.x;
  const int jl = blockIdx.x, j = a.j0 + jl;
  const int y0 = blockIdx.y * kRB;
  for (int e = tid; e < N; e += kRowThreads) tws[e] = __ldg(a.tw_n + e);
  build_passtw<L, 2, kRowThreads>(ptr, a.tw_n, tid);
  pdl_wait();
  __syncthreads();
  float2 acc[KR][LP::R];
#pragma unroll
  for (int k = 0; k < KR; ++k)
#pragma unroll
    for (int rr = 0; rr < LP::R; ++rr) acc[k][rr] = make_float2(0.f, 0.f);
  // loads of source parameter q: the split pairs X(k), X(L - k) of every row (column 0 packed), those of
  // q + 1 in flight while q is transformed, and the combination weights in the layout of the last pass,
  // requested before the split
  float2 xa[SIT], xb[SIT], wv[KR][LP::R];
  auto load_w = [&](int q) {
    if constexpr (MODE == 1) {
      const float2* wq = reinterpret_cast<const float2*>(a.W + (((long)q * a.Mp + j) * N + y0) * N);
#pragma unroll
      for (int k = 0; k < KR; ++k) {
        const int b = tid + k * kRowThreads;
        if (NBF % kRowThreads == 0 || b < NBF) {
          const int sr = b / LP::BPS, jq = b % LP::BPS;
#pragma unroll
          for (int rr = 0; rr < LP::R; ++rr) wv[k][rr] = __ldg(wq + sr * L + jq + rr * LP::NS);
        }
      }
    }
  };
  auto load_q = [&](int q, float2 (&ya)[SIT], float2 (&yb)[SIT]) {
    const float2* Tq = a.T + ((long)(q * a.nj + jl) * N + y0) * L;
#pragma unroll
    for (int i = 0; i < SIT; ++i) {
      const int e = tid + i * kRowThreads;
      if (NSPL % kRowThreads == 0 || e < NSPL) {
        const int row = e / NK, k = e - row * NK;   // consecutive threads: consecutive k of one row
        const float2 u = __ldg(Tq + (long)row * L + k);
        const float2 v = __ldg(Tq + (long)row * L + (k == 0 ? 0 : L - k));
        ya[i] = k == 0 ? make_float2(u.x, 0.f) : u;                     // X(0): real part of column 0
        yb[i] = k == 0 ? make_float2(v.y, 0.f) : v;                     // X(L): its imaginary part
      }
    }
  };
  load_q(0, xa, xb);
  for (int q = 0; q < a.Q; ++q) {
    load_w(q);         // in flight during the split and the passes
    __syncthreads();   // the previous q's last pass has read rowbuf
    // Hermitian split Z'[k] = (X[k] + conj X[L-k]) + i w^-k (X[k] - conj X[L-k]), pairs (k, L - k)
#pragma unroll
    for (int i = 0; i < SIT; ++i) {
      const int e = tid + i * kRowThreads;
      if (NSPL % kRowThreads == 0 || e < NSPL) {
        const int row = e / NK, k = e - row * NK;
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
    if (q + 1 < a.Q) load_q(q + 1, xa, xb);
    __syncthreads();
    fft_passes<L, true, kRB, kRowThreads, 0, Plan<L>::np - 1>(rowbuf, SSR, ptr, tid);
    if constexpr (MODE == 1) {
      auto emit = [&](int, int, float2 v, int k, int rr) {
        acc[k][rr] = make_float2(fmaf(wv[k][rr].x, v.x, acc[k][rr].x), fmaf(wv[k][rr].y, v.y, acc[k][rr].y));
      };
      last_pass_to<L, true, kRB, kRowThreads>(rowbuf, SSR, ptr, emit, tid);
    } else {
      float2* oq = reinterpret_cast<float2*>(a.out + (((long)q * a.Mp + j) * N + y0) * N);
      auto emit = [&](int sr, int t, float2 v, int, int) { oq[sr * L + t] = v; };
      last_pass_to<L, true, kRB, kRowThreads>(rowbuf, SSR, ptr, emit, tid);
    }
  }
  if constexpr (MODE == 1) {
    float2* oj = reinterpret_cast<float2*>(a.out + ((long)j * N + y0) * N);
#pragma unroll
    for (int k = 0; k < KR; ++k) {
      const int b = tid + k * kRowThreads;
      if (NBF % kRowThreads == 0 || b < NBF) {
        const int sr = b / LP::BPS, jq = b % LP::BPS;
#pragma unroll
        for (int rr = 0; rr < LP::R; ++rr) oj[sr * L + jq + rr * LP::NS] = acc[k][rr];
      }
    }
  }
}

template <int N>
int inv2_launch_n(const Inv2Args& a, bool xi, cudaStream_t st) {
  using G = Inv2Geom<N>;
  FR3D_TRY(smem_optin(reinterpret_cast<const void*>(k_inv2_col<N>), G::smem_col));
  const void* rk = xi ? reinterpret_cast<const void*>(k_inv2_row<N, 1>) : reinterpret_cast<const void*>(k_inv2_row<N, 0>);
  FR3D_TRY(smem_optin(rk, G::smem_row));
  k_inv2_col<N><<<dim3(a.Q * a.nj, G::L / G::CA), kColThreads, G::smem_col, st>>>(a);
  FR3D_CUDA_TRY(cudaGetLastError());
  if (xi) k_inv2_row<N, 1><<<dim3(a.nj, N / kRB), kRowThreads, G::smem_row, st>>>(a);
  else k_inv2_row<N, 0><<<dim3(a.nj, N / kRB), kRowThreads, G::smem_row, st>>>(a);
  FR3D_CUDA_TRY(cudaGetLastError());
  return FR3D_OK;
}

}  // namespace

size_t inv2_scratch_bytes(int n, int Q, int nj) { return sizeof(float2) * (size_t)Q * nj * n * (n / 2); }

// The two-pass inverse for the fused inverse's arguments; T: scratch of inv2_scratch_bytes.
int inv2_launch(int n, bool xi, const FusedArgs& f, int nj, float2* T, cudaStream_t st) {
  Inv2Args a;
  a.Uh = f.Uh;
  a.A = f.A;
  a.Dd = f.Dd;
  a.aidx = f.aidx;
  a.na = f.na;
  a.bbin = f.bbin;
  a.nb = f.nb;
  a.W = f.W;
  a.out = f.out;
  a.tw_n = f.tw_n;
  a.T = T;
  a.Q = f.Q;
  a.j0 = f.j0;
  a.nj = nj;
  a.Mp = f.Mp;
  switch (n) {
    case 16: return inv2_launch_n<16>(a, xi, st);
    case 24: return inv2_launch_n<24>(a, xi, st);
    case 32: return inv2_launch_n<32>(a, xi, st);
    case 48: return inv2_launch_n<48>(a, xi, st);
    case 64: return inv2_launch_n<64>(a, xi, st);
    case 96: return inv2_launch_n<96>(a, xi, st);
    case 128: return inv2_launch_n<128>(a, xi, st);
    case 192: return inv2_launch_n<192>(a, xi, st);
    case 256: return inv2_launch_n<256>(a, xi, st);
    case 384: return inv2_launch_n<384>(a, xi, st);
  }
  return FR3D_ERR_UNSUPPORTED_SIZE;
}

}  // namespace fr3d
