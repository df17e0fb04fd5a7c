// Batched mixed-radix (2, 3, 4, 8, 16) complex FFTs on shared memory.
//
// Every 2D transform of Algorithm 1 (steps 1 and 3) is built from one
// primitive: a CTA transforms NSEQ sequences of compile-time length L held in
// shared memory.  Each pass is a Stockham autosort step of radix R: a thread
// gathers R elements at stride L/R into registers, twiddles them, runs an
// R-point DFT in registers and scatters the results so that the output of the
// last pass is in natural order.  Passes are in place: every thread first reads
// all of its butterflies, the CTA synchronises, then every thread writes.
// The number of butterflies a thread owns per pass is a compile-time constant,
// so all of them stay in registers.
#pragma once

#include <cuda_runtime.h>

namespace fr3d {

template <typename T> struct cpx;
template <> struct cpx<float> { using t = float2; };
template <> struct cpx<double> { using t = double2; };

__device__ __forceinline__ float2 cmk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 cmk(double a, double b) { return make_double2(a, b); }
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
// Products and fused multiply-adds with their rounding pinned (the compiler may not contract them
// differently in different kernels), so that every kernel built from these butterflies computes the
// same bits for the same inputs.
__device__ __forceinline__ float fmul_p(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double fmul_p(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fma_p(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_p(double a, double b, double c) { return __fma_rn(a, b, c); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  C r;
  r.x = fma_p(a.x, b.x, -fmul_p(a.y, b.y));
  r.y = fma_p(a.x, b.y, fmul_p(a.y, b.x));
  return r;
}
// float2: the two lanes in one packed FP32x2 operation (one instruction, each lane rounded to nearest
// like the scalar form, so the results are the same bits).  A translation unit that defines
// FR3D_SCALAR_COMPLEX_ADDS before including this header keeps the scalar form (its kernels then use
// fewer registers; the device code of every unit is self-contained, so units may differ).
#ifndef FR3D_SCALAR_COMPLEX_ADDS
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(*reinterpret_cast<const unsigned long long*>(&a)),
      "l"(*reinterpret_cast<const unsigned long long*>(&b)));
  return *reinterpret_cast<const float2*>(&r);
}
#endif
template <typename C> __device__ __forceinline__ C cconj(C a) { a.y = -a.y; return a; }
// multiply by -i (forward) or +i (inverse)
template <bool INV, typename C> __device__ __forceinline__ C cmul_mi(C a) {
  C r;
  if (INV) { r.x = -a.y; r.y = a.x; } else { r.x = a.y; r.y = -a.x; }
  return r;
}
template <typename C, typename S> __device__ __forceinline__ C cscale(C a, S s) {
  a.x = fmul_p(a.x, s);
  a.y = fmul_p(a.y, s);
  return a;
}

// cos and sin of 2 pi n / 16, n = 0..15 (exact decimal expansions of the 16th roots of unity)
#define FR3D_C1 0.92387953251128675613
#define FR3D_S1 0.38268343236508977173
#define FR3D_R2 0.70710678118654752440

template <typename C, int R, int n, bool INV>
__device__ __forceinline__ C twiddle_const(C a) {
  // a * exp(-+ 2 pi i n / R) for R in {8, 16}
  constexpr int m = n * (16 / R);  // index in 16ths of a turn
  using T = decltype(a.x);
  if constexpr (m == 0) {
    return a;
  } else if constexpr (m == 4) {
    return cmul_mi<INV>(a);
  } else {
    constexpr double cs[16] = {1.0, FR3D_C1, FR3D_R2, FR3D_S1, 0.0, -FR3D_S1, -FR3D_R2, -FR3D_C1,
                               -1.0, -FR3D_C1, -FR3D_R2, -FR3D_S1, 0.0, FR3D_S1, FR3D_R2, FR3D_C1};
    constexpr double sn[16] = {0.0, FR3D_S1, FR3D_R2, FR3D_C1, 1.0, FR3D_C1, FR3D_R2, FR3D_S1,
                               0.0, -FR3D_S1, -FR3D_R2, -FR3D_C1, -1.0, -FR3D_C1, -FR3D_R2, -FR3D_S1};
    const T c = (T)cs[m];
    const T s = INV ? (T)sn[m] : (T)(-sn[m]);
    C r;
    r.x = fma_p(a.x, c, -fmul_p(a.y, s));
    r.y = fma_p(a.x, s, fmul_p(a.y, c));
    return r;
  }
}

// R-point DFT in registers, natural order in and out.  Forward: exp(-2 pi i nk/R); inverse: exp(+...).
template <int R, bool INV> struct Dft;

template <bool INV> struct Dft<1, INV> {
  template <typename C> static __device__ __forceinline__ void run(C*) {}
};
template <bool INV> struct Dft<2, INV> {
  template <typename C> static __device__ __forceinline__ void run(C* v) {
    C a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};
template <bool INV> struct Dft<3, INV> {
  template <typename C> static __device__ __forceinline__ void run(C* v) {
    using T = decltype(v[0].x);
    const T h3 = (T)0.86602540378443864676;  // sin(2 pi / 3)
    C s = cadd(v[1], v[2]);
    C d = csub(v[1], v[2]);
    C m = csub(v[0], cscale(s, (T)0.5));
    C t = cmul_mi<INV>(cscale(d, h3));  // -i h3 d (forward)
    v[0] = cadd(v[0], s);
    v[1] = cadd(m, t);
    v[2] = csub(m, t);
  }
};
template <bool INV> struct Dft<4, INV> {
  template <typename C> static __device__ __forceinline__ void run(C* v) {
    C a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
    C c = cadd(v[1], v[3]), d = cmul_mi<INV>(csub(v[1], v[3]));
    v[0] = cadd(a, c);
    v[2] = csub(a, c);
    v[1] = cadd(b, d);
    v[3] = csub(b, d);
  }
};

template <int R, int n, bool INV> struct DifStep {
  template <typename C> static __device__ __forceinline__ void run(C* v, C* e, C* o) {
    if constexpr (n < R / 2) {
      e[n] = cadd(v[n], v[n + R / 2]);
      o[n] = twiddle_const<C, R, n, INV>(csub(v[n], v[n + R / 2]));
      DifStep<R, n + 1, INV>::run(v, e, o);
    }
  }
};

// radix 8 and 16: one decimation-in-frequency radix-2 step, then two half-size DFTs
template <int R, bool INV> struct DftDif {
  template <typename C> static __device__ __forceinline__ void run(C* v) {
    C e[R / 2], o[R / 2];
    DifStep<R, 0, INV>::run(v, e, o);
    Dft<R / 2, INV>::run(e);
    Dft<R / 2, INV>::run(o);
#pragma unroll
    for (int k = 0; k < R / 2; ++k) {
      v[2 * k] = e[k];
      v[2 * k + 1] = o[k];
    }
  }
};
template <bool INV> struct Dft<8, INV> {
  template <typename C> static __device__ __forceinline__ void run(C* v) { DftDif<8, INV>::run(v); }
};
template <bool INV> struct Dft<16, INV> {
  template <typename C> static __device__ __forceinline__ void run(C* v) { DftDif<16, INV>::run(v); }
};

// Radix schedule per transform length (product of the radices = L, applied first to last).
template <int L> struct Plan;
#define FR3D_PLAN(L_, NP_, R0_, R1_, R2_)                                        \
  template <> struct Plan<L_> {                                                \
    static constexpr int np = NP_;                                             \
    static constexpr int radix(int p) { return p == 0 ? R0_ : (p == 1 ? R1_ : R2_); } \
  };
FR3D_PLAN(8, 1, 8, 1, 1)
FR3D_PLAN(12, 2, 4, 3, 1)
FR3D_PLAN(16, 1, 16, 1, 1)
FR3D_PLAN(24, 2, 8, 3, 1)
FR3D_PLAN(32, 2, 8, 4, 1)
FR3D_PLAN(48, 2, 16, 3, 1)
FR3D_PLAN(64, 2, 8, 8, 1)
FR3D_PLAN(96, 3, 8, 4, 3)
FR3D_PLAN(128, 2, 16, 8, 1)
FR3D_PLAN(192, 3, 16, 4, 3)
FR3D_PLAN(256, 2, 16, 16, 1)
FR3D_PLAN(384, 3, 16, 8, 3)
FR3D_PLAN(512, 3, 8, 8, 8)
#undef FR3D_PLAN

// Shared-memory layout: sequences of length L stored contiguously with one pad element
// every 2^PSH elements (PSH = 4 for 8-byte, 3 for 16-byte complex: one pad per 128 B).
template <typename C> struct PadShift { static constexpr int v = sizeof(C) == 8 ? 4 : 3; };
template <int L, typename C> struct PaddedLen { static constexpr int v = L + (L >> PadShift<C>::v); };
template <typename C> __device__ __forceinline__ int pidx(int e) { return e + (e >> PadShift<C>::v); }

// Per-pass twiddle tables.  Pass p of length L (radix R_p, NS_p = product of the earlier radices)
// with NS_p > 1 needs w^(r jj L/(NS_p R_p)) for r in [1, R_p) and jj in [0, NS_p), w = exp(-2 pi i / L).
// They are stored pass after pass as blocks [r - 1][jj]: a warp's lanes (consecutive jj) read
// consecutive entries, so shared-memory reads are free of bank conflicts.
template <int L> constexpr int passtw_offset(int p) {
  int off = 0, ns = 1;
  for (int i = 0; i < p; ++i) {
    const int R = Plan<L>::radix(i);
    if (ns > 1) off += (R - 1) * ns;
    ns *= R;
  }
  return off;
}
template <int L> constexpr int passtw_size() { return passtw_offset<L>(Plan<L>::np); }

// Fill the pass tables of length L from tw_g[t] = exp(-2 pi i t / (TS L)), t < TS L (global memory).
template <int L, int TS, int NTHR, typename C>
__device__ __forceinline__ void build_passtw(C* dst, const C* __restrict__ tw_g, int tid) {
  constexpr int NP = Plan<L>::np;
  int ns = 1, off = 0;
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    const int R = Plan<L>::radix(p);
    if (ns > 1) {
      const int cnt = (R - 1) * ns, step = L / (ns * R);
      for (int e = tid; e < cnt; e += NTHR) {
        const int r = e / ns + 1, jj = e % ns;
        dst[off + e] = __ldg(tw_g + r * jj * step * TS);
      }
      off += cnt;
    }
    ns *= R;
  }
}

// One Stockham pass.  Butterfly j of a sequence reads elements j + r L/R (r < R), multiplies
// element r by w^(r (j mod NS) L/(NS R)), with w = exp(-+2 pi i / L), taken from the pass table
// twp = [r - 1][j mod NS], and writes the R-point DFT to positions (j / NS) NS R + (j mod NS) + r NS.
template <int L, int R, int NS, bool INV, int NSEQ, int NTHR, typename C>
__device__ __forceinline__ void stockham_pass(C* buf, int sstride, const C* __restrict__ twp, int tid) {
  constexpr int BPS = L / R;
  constexpr int NB = NSEQ * BPS;
  constexpr int K = (NB + NTHR - 1) / NTHR;
  constexpr bool EXACT = (K * NTHR == NB);
  C v[K][R];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int b = tid + k * NTHR;
    if (EXACT || b < NB) {
      const int s = b / BPS, j = b - s * BPS;
      const int jj = j % NS;
      C* base = buf + s * sstride;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        C x = base[pidx<C>(j + r * BPS)];
        if (NS > 1 && r > 0) {
          C w = twp[(r - 1) * NS + jj];
          if (INV) w = cconj(w);
          x = cmul(x, w);
        }
        v[k][r] = x;
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int b = tid + k * NTHR;
    if (EXACT || b < NB) {
      const int s = b / BPS, j = b - s * BPS;
      const int jj = j % NS;
      Dft<R, INV>::run(v[k]);
      C* base = buf + s * sstride;
      const int d0 = (j / NS) * NS * R + jj;
#pragma unroll
      for (int r = 0; r < R; ++r) base[pidx<C>(d0 + r * NS)] = v[k][r];
    }
  }
  __syncthreads();
}

// Pass 0 (NS = 1, no twiddles) fed from registers: element t of sequence s comes from ld(s, t) (for
// example a global load) instead of shared memory, so the input never makes a shared-memory round trip.
// Writes the pass's output to buf and synchronises.
template <int L, bool INV, int NSEQ, int NTHR, class Ld, typename C>
__device__ __forceinline__ void first_pass_from(C* buf, int sstride, Ld ld, int tid) {
  constexpr int R = Plan<L>::radix(0);
  constexpr int BPS = L / R;
  constexpr int NB = NSEQ * BPS;
  constexpr int K = (NB + NTHR - 1) / NTHR;
  constexpr bool EXACT = (K * NTHR == NB);
  C v[K][R];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int b = tid + k * NTHR;
    if (EXACT || b < NB) {
      const int s = b / BPS, j = b - s * BPS;
#pragma unroll
      for (int r = 0; r < R; ++r) v[k][r] = ld(s, j + r * BPS);
    }
  }
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int b = tid + k * NTHR;
    if (EXACT || b < NB) {
      const int s = b / BPS, j = b - s * BPS;
      Dft<R, INV>::run(v[k]);
      C* base = buf + s * sstride;
#pragma unroll
      for (int r = 0; r < R; ++r) base[pidx<C>(j * R + r)] = v[k][r];
    }
  }
  __syncthreads();
}

// Geometry of the last pass of an L-point FFT: butterfly b = tid + k NTHR of NSEQ sequences owns the
// outputs t = j + r NS (r < R) of sequence s = b / BPS, j = b mod BPS.
template <int L> struct LastPass {
  static constexpr int NP = Plan<L>::np;
  static constexpr int R = Plan<L>::radix(NP - 1);
  static constexpr int BPS = L / R;
  static constexpr int NS = L / R;
};

// The last pass of an L-point FFT whose earlier passes are done (data in buf): the outputs go to
// emit(s, t, value, k, r) instead of back to shared memory, so no barrier follows the reads.
template <int L, bool INV, int NSEQ, int NTHR, class Em, typename C>
__device__ __forceinline__ void last_pass_to(const C* buf, int sstride, const C* __restrict__ twp, Em emit, int tid) {
  using LP = LastPass<L>;
  constexpr int R = LP::R, BPS = LP::BPS, NS = LP::NS;
  constexpr int NB = NSEQ * BPS;
  constexpr int K = (NB + NTHR - 1) / NTHR;
  constexpr bool EXACT = (K * NTHR == NB);
  const C* tw = twp + passtw_offset<L>(LP::NP - 1);
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int b = tid + k * NTHR;
    if (EXACT || b < NB) {
      const int s = b / BPS, j = b - s * BPS;
      const C* base = buf + s * sstride;
      C v[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        C x = base[pidx<C>(j + r * BPS)];
        if (NS > 1 && r > 0) {
          C w = tw[(r - 1) * NS + j];
          if (INV) w = cconj(w);
          x = cmul(x, w);
        }
        v[r] = x;
      }
      Dft<R, INV>::run(v);
#pragma unroll
      for (int r = 0; r < R; ++r) emit(s, j + r * NS, v[r], k, r);
    }
  }
}

// Passes P0 .. P1 - 1 of an L-point FFT (NS = product of the radices before P0).
template <int L, bool INV, int NSEQ, int NTHR, int P0, int P1, int NS = 1, typename C>
__device__ __forceinline__ void fft_passes(C* buf, int sstride, const C* __restrict__ twp, int tid) {
  if constexpr (P0 < P1) {
    constexpr int R = Plan<L>::radix(P0);
    stockham_pass<L, R, NS, INV, NSEQ, NTHR>(buf, sstride, twp + passtw_offset<L>(P0), tid);
    fft_passes<L, INV, NSEQ, NTHR, P0 + 1, P1, NS * R>(buf, sstride, twp, tid);
  }
}

// All passes of an L-point FFT on NSEQ sequences (stride sstride); twp = pass tables of length L.
template <int L, bool INV, int NSEQ, int NTHR, int P = 0, int NS = 1, typename C>
__device__ __forceinline__ void fft_smem(C* buf, int sstride, const C* __restrict__ twp, int tid) {
  if constexpr (P < Plan<L>::np) {
    constexpr int R = Plan<L>::radix(P);
    stockham_pass<L, R, NS, INV, NSEQ, NTHR>(buf, sstride, twp + passtw_offset<L>(P), tid);
    fft_smem<L, INV, NSEQ, NTHR, P + 1, NS * R>(buf, sstride, twp, tid);
  }
}

}  // namespace fr3d
