// 2D real transforms over (x, y) for Algorithm 1 steps 1 and 3 and the forward operator of Eq. (5).
//
// Layouts in device memory:
//   real volume      [plane][y][x]            (x fastest, n floats per row)
//   half spectrum    [plane][kx][ky]          kx in [0, n/2], ky in [0, n): one contiguous column of
//                                             n complex values per kx, (n/2 + 1) n per plane
// A forward 2D transform is a row pass (real-to-complex along x, written transposed into the
// half-spectrum layout) followed by a column pass (complex along ky, contiguous).  The inverse
// runs the column pass first and then the complex-to-real row pass.  The row passes use the
// standard packing of a length-n real sequence into a length-n/2 complex one
// (z[m] = x[2m] + i x[2m+1]) and its Hermitian split.  All transforms are unnormalised.
#pragma once

#include "common.cuh"
#include "fft_engine.cuh"

namespace fr3d {

constexpr int kThreads = 256;

template <typename C, int L> struct Smem {
  // odd row stride (in elements) holding L + 1 padded elements: conflict-free column access
  static constexpr int pl = L + (L >> PadShift<C>::v) + 1;
  static constexpr int ss = (pl % 2 == 0) ? pl + 1 : pl;
};

// largest divisor of n that is <= cap (>= 1)
constexpr int divisor_at_most(int n, int cap) {
  int d = cap < 1 ? 1 : (cap > n ? n : cap);
  while (n % d != 0) --d;
  return d;
}
template <typename T, int N> struct RowTile {
  static constexpr int v = divisor_at_most(N, (sizeof(T) == 4 ? 8192 : 4096) / N);
};
template <typename T, int N> struct ColTile {
  static constexpr int v0 = (sizeof(T) == 4 ? 4096 : 2048) / N;
  static constexpr int v1 = v0 < 1 ? 1 : v0;
  static constexpr int v = v1 > N / 2 + 1 ? N / 2 + 1 : v1;
};

// Copy TOTAL elements with NT threads, element e = tid + i NT, issuing B loads before their stores
// so that several global loads are in flight per thread (ld(e) -> value, st(e, value)).
template <int TOTAL, int NT, int B, typename LD, typename ST>
__device__ __forceinline__ void batched_copy(int tid, LD ld, ST st) {
  constexpr int IT = (TOTAL + NT - 1) / NT;
  constexpr bool FULL = TOTAL % NT == 0;
#pragma unroll
  for (int b0 = 0; b0 < IT; b0 += B) {
    decltype(ld(0)) v[B];
#pragma unroll
    for (int i = 0; i < B; ++i) {
      const int e = tid + (b0 + i) * NT;
      if (b0 + i < IT && (FULL || e < TOTAL)) v[i] = ld(e);
    }
#pragma unroll
    for (int i = 0; i < B; ++i) {
      const int e = tid + (b0 + i) * NT;
      if (b0 + i < IT && (FULL || e < TOTAL)) st(e, v[i]);
    }
  }
}

// ---------------------------------------------------------------- row pass, real -> half spectrum
// Plane maps: in(p) -> the real n x n plane p, out(p) -> its half spectrum [kx][ky].
template <typename T> struct StridedPlanes {
  const T* in;
  long in_ps;
  typename cpx<T>::t* out;
  long out_ps;
  __device__ const T* src(int p) const { return in + p * in_ps; }
  __device__ typename cpx<T>::t* dst(int p) const { return out + p * out_ps; }
};
struct PlanePtr {            // one entry per plane of a batch of instances
  const float* in;
  float2* out;
};
struct TablePlanes {
  const PlanePtr* t;
  __device__ const float* src(int p) const { return t[p].in; }
  __device__ float2* dst(int p) const { return t[p].out; }
};

// in: planes of n x n reals; out: [plane][kx][y] complex.  One CTA transforms TY rows of a plane.
template <typename T, int N, int TY, class PM>
__global__ void __launch_bounds__(kThreads) k_row_r2c(PM pm, const typename cpx<T>::t* __restrict__ tw_full) {
  using C = typename cpx<T>::t;
  constexpr int L = N / 2, SS = Smem<C, L>::ss, STS = TY + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tws = reinterpret_cast<C*>(smem_raw);       // exp(-2 pi i t / n), t < n
  C* ptw = tws + N;                              // pass tables of the length-n/2 transform
  C* buf = ptw + passtw_size<L>();
  C* stg = buf + TY * SS;
  const int tid = threadIdx.x, plane = blockIdx.y, y0 = blockIdx.x * TY;
  const C* src = reinterpret_cast<const C*>(pm.src(plane) + (long)y0 * N);
  for (int e = tid; e < N; e += kThreads) tws[e] = __ldg(tw_full + e);
  build_passtw<L, 2, kThreads>(ptw, tw_full, tid);
  batched_copy<TY * L, kThreads, 8>(
      tid, [&](int e) { return __ldg(src + e); },
      [&](int e, C v) { buf[(e / L) * SS + pidx<C>(e % L)] = v; });
  __syncthreads();
  fft_smem<L, false, TY, kThreads>(buf, SS, ptw, tid);
  const T half = (T)0.5;
  for (int e = tid; e < TY * (L + 1); e += kThreads) {
    const int k = e / TY, r = e - k * TY;
    const C zk = buf[r * SS + pidx<C>(k == L ? 0 : k)];
    const C zc = cconj(buf[r * SS + pidx<C>(k == 0 ? 0 : L - k)]);
    const C E = cscale(cadd(zk, zc), half);
    const C O = cmul_mi<false>(cscale(csub(zk, zc), half));  // (Z[k] - conj Z[L-k]) / (2i)
    stg[k * STS + r] = cadd(E, cmul(tws[k], O));  // X[k] = E[k] + w^k O[k]
  }
  __syncthreads();
  C* dst = pm.dst(plane) + y0;
  for (int e = tid; e < TY * (L + 1); e += kThreads) {
    const int k = e / TY, r = e - k * TY;
    dst[(long)k * N + r] = stg[k * STS + r];
  }
}

// ---------------------------------------------------------------- column pass along ky
// Op supplies: src(plane) -> const C*, dst(plane) -> C*, and load(plane, kx, ky, value) -> C
// (a per-bin multiplier for the solve).  One CTA transforms TC consecutive columns of one plane.
template <typename T, int N, bool INV, class Op, int TC>
__global__ void __launch_bounds__(kThreads) k_col_fft(Op op, const typename cpx<T>::t* __restrict__ tw) {
  using C = typename cpx<T>::t;
  constexpr int SS = Smem<C, N>::ss, H1 = N / 2 + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* ptw = reinterpret_cast<C*>(smem_raw);       // pass tables of the length-n transform
  C* buf = ptw + passtw_size<N>();
  const int tid = threadIdx.x, plane = blockIdx.y, c0 = blockIdx.x * TC;
  build_passtw<N, 1, kThreads>(ptw, tw, tid);
  op.begin(plane);
  const C* src = op.src(plane);
  batched_copy<TC * N, kThreads, 8>(
      tid,
      [&](int e) {
        const int kx = c0 + e / N;
        return kx < H1 ? src[(long)c0 * N + e] : cmk((T)0, (T)0);
      },
      [&](int e, C v) {
        const int col = e / N, ky = e - col * N, kx = c0 + col;
        buf[col * SS + pidx<C>(ky)] = kx < H1 ? op.load(plane, kx, ky, v) : v;
      });
  __syncthreads();
  fft_smem<N, INV, TC, kThreads>(buf, SS, ptw, tid);
  C* dst = op.dst(plane);
  for (int e = tid; e < TC * N; e += kThreads) {
    const int col = e / N, ky = e - col * N, kx = c0 + col;
    if (kx < H1) dst[(long)kx * N + ky] = buf[col * SS + pidx<C>(ky)];
  }
}

// plain forward/inverse column pass, plane p -> plane p
template <typename T> struct ColPlain {
  using C = typename cpx<T>::t;
  const C* in;
  C* out;
  long ps;
  __device__ void begin(int) {}
  __device__ const C* src(int p) const { return in + p * ps; }
  __device__ C* dst(int p) const { return out + p * ps; }
  __device__ C load(int, int, int, C v) const { return v; }
};

// forward column pass over a table of planes (batched instances), in place
struct ColTable {
  const PlanePtr* t;
  __device__ void begin(int) {}
  __device__ const float2* src(int p) const { return t[p].out; }
  __device__ float2* dst(int p) const { return t[p].out; }
  __device__ float2 load(int, int, int, float2 v) const { return v; }
};

// Solve for M = 1 fused into the inverse column pass (Eq. (6) with a single observation depth):
// zeta~_j(k) = A_j(k) U~_q(k) / (n^2 (||A(k)||^2 + alpha s^2)).  Output plane p = jc Q + q holds
// depth j = j0 + jc of source parameter q.
template <typename T> struct ColSolve1 {
  using C = typename cpx<T>::t;
  const C* Uh;        // [Q][H1][n]
  C* out;             // [chunk Q][H1][n]
  const T* A;         // [M' = j][H1][n]
  const T* D;         // [n_alpha][C]
  const int* aidx;    // chosen row of D per band
  const unsigned char* cband;  // band of every class (nb > 1)
  long ps;
  int Q, j0, n, Cn, nb;
  const T* drow;
  __device__ void begin(int) { drow = D + (long)(*aidx) * Cn; }
  __device__ const C* src(int p) const { return Uh + (p % Q) * ps; }
  __device__ C* dst(int p) const { return out + p * ps; }
  __device__ C load(int p, int kx, int ky, C v) const {
    const int j = j0 + p / Q;
    const int c = class_of(kx, ky, n);
    const T d = nb == 1 ? drow[c] : D[(long)aidx[cband[c]] * Cn + c];
    const T w = A[(long)j * ps + (long)kx * n + ky] * d;
    return cscale(v, w);
  }
};

// ---------------------------------------------------------------- row pass, half spectrum -> real
struct Src32 {
  const float4* pts;  // [Q * L] point sources
  int L;              // points per source parameter
  float coef;         // -A0 / (4 pi)
};
struct Src64 {
  const double* pts;  // [Q * L * 3]
  int L;
  double coef;
};

template <typename T> struct SrcOf;
template <> struct SrcOf<float> { using t = Src32; };
template <> struct SrcOf<double> { using t = Src64; };

__device__ __forceinline__ float v0_at(const Src32& s, int q, float x, float y, float z) {
  float acc = 0.f;
  const float4* p = s.pts + q * s.L;
  for (int l = 0; l < s.L; ++l) {
    const float4 a = __ldg(p + l);
    const float dx = x - a.x, dy = y - a.y, dz = z - a.z;
    acc += rsqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
  }
  return s.coef * acc;
}
// 1 / sqrt(r2) in FP64 by Newton-Raphson for the reciprocal square root, y <- y (3 - r2 y^2) / 2, from
// the single-precision estimate: each step squares the relative error (about 1e-7 -> 1e-14 -> below
// the FP64 rounding), so two steps reach FP64 accuracy with a few FMAs instead of an FP64 square root
// and division.  Arguments outside the single-precision range take the direct form.
__device__ __forceinline__ double rsqrt_fp64(double r2) {
  if (!(r2 > 1e-30 && r2 < 1e30)) return 1.0 / sqrt(r2);
  double y = (double)rsqrtf((float)r2);
  const double h = 0.5 * r2;
  y = y * fma(-h * y, y, 1.5);
  y = y * fma(-h * y, y, 1.5);
  return y;
}

__device__ __forceinline__ double v0_at(const Src64& s, int q, double x, double y, double z) {
  double acc = 0.0;
  const double* p = s.pts + 3 * q * s.L;
  for (int l = 0; l < s.L; ++l) {
    const double dx = x - __ldg(p + 3 * l), dy = y - __ldg(p + 3 * l + 1), dz = z - __ldg(p + 3 * l + 2);
    acc += rsqrt_fp64(fma(dx, dx, fma(dy, dy, dz * dz)));
  }
  return s.coef * acc;
}

struct RowGeom {
  double x0, y0, h;  // voxel-centred grid x_a = x0 + (a + 1/2) h
};

// MODE 0 (plain): input plane ip -> output plane (ip % Q) * out_stride + j0 + ip / Q.
// MODE 1 (xi):   output plane j0 + blockIdx.y <- sum over q of V0_q * (input plane blockIdx.y Q + q),
//                divided by sum_q V0_q^2 (Algorithm 1 step 4, several q).
template <typename T, int N, int MODE>
__global__ void __launch_bounds__(kThreads) k_row_c2r(const typename cpx<T>::t* __restrict__ in, T* __restrict__ out,
                                                     int Q, int j0, int out_stride,
                                                     typename SrcOf<T>::t src, RowGeom g, const T* __restrict__ zr,
                                                     const typename cpx<T>::t* __restrict__ tw_half,
                                                     const typename cpx<T>::t* __restrict__ tw_full) {
  using C = typename cpx<T>::t;
  constexpr int L = N / 2, TY0 = RowTile<T, N>::v, TY = (MODE == 1 && TY0 % 2 == 0) ? TY0 / 2 : TY0;
  constexpr int SS = Smem<C, L>::ss;
  constexpr int EPT = (TY * L + kThreads - 1) / kThreads;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tws = reinterpret_cast<C*>(smem_raw);       // exp(-2 pi i t / n), t < n
  C* ptw = tws + N;                              // pass tables of the length-n/2 transform
  C* buf = ptw + passtw_size<L>();
  const int tid = threadIdx.x, y0 = blockIdx.x * TY;
  const long ps = (long)(L + 1) * N;
  for (int e = tid; e < N; e += kThreads) tws[e] = __ldg(tw_full + e);
  build_passtw<L, 2, kThreads>(ptw, tw_full, tid);
  T num[EPT][2], den[EPT][2];
  if (MODE == 1) {
#pragma unroll
    for (int i = 0; i < EPT; ++i) num[i][0] = num[i][1] = den[i][0] = den[i][1] = (T)0;
  }
  const int nq = MODE == 1 ? Q : 1;
  for (int q = 0; q < nq; ++q) {
    const int ip = MODE == 1 ? blockIdx.y * Q + q : blockIdx.y;
    const C* s = in + ip * ps + y0;
    for (int e = tid; e < TY * (L + 1); e += kThreads) {
      const int k = e / TY, r = e - k * TY;
      buf[r * SS + pidx<C>(k)] = s[(long)k * N + r];
    }
    __syncthreads();
    // Hermitian split: Z'[k] = (X[k] + conj X[L-k]) + i w^-k (X[k] - conj X[L-k]); pairs (k, L-k) in one thread
    for (int e = tid; e < TY * (L / 2 + 1); e += kThreads) {
      const int r = e / (L / 2 + 1), k = e - r * (L / 2 + 1);
      C* row = buf + r * SS;
      const C a = row[pidx<C>(k)], b = row[pidx<C>(L - k)];
      {
        const C sum = cadd(a, cconj(b)), dif = csub(a, cconj(b));
        const C t = cmul_mi<true>(cmul(cconj(tws[k]), dif));
        row[pidx<C>(k)] = cadd(sum, t);
      }
      if (k != 0 && 2 * k != L) {
        const C sum = cadd(b, cconj(a)), dif = csub(b, cconj(a));
        const C t = cmul_mi<true>(cmul(cconj(tws[L - k]), dif));
        row[pidx<C>(L - k)] = cadd(sum, t);
      }
    }
    __syncthreads();
    fft_smem<L, true, TY, kThreads>(buf, SS, ptw, tid);
    if (MODE == 0) {
      const int jc = ip / Q, qq = ip - jc * Q;
      T* o = out + ((long)qq * out_stride + j0 + jc) * N * N + (long)y0 * N;
      C* oc = reinterpret_cast<C*>(o);
      for (int e = tid; e < TY * L; e += kThreads) {
        const int r = e / L, m = e - r * L;
        oc[(long)r * L + m] = buf[r * SS + pidx<C>(m)];
      }
    } else {
      const T z = zr[j0 + blockIdx.y];
      const T yy0 = (T)g.y0, xx0 = (T)g.x0, hh = (T)g.h;
#pragma unroll
      for (int i = 0; i < EPT; ++i) {
        const int e = tid + i * kThreads;
        if (EPT * kThreads == TY * L || e < TY * L) {
          const int r = e / L, m = e - r * L;
          const C v = buf[r * SS + pidx<C>(m)];
          const T y = yy0 + ((T)(y0 + r) + (T)0.5) * hh;
          const T xa = xx0 + ((T)(2 * m) + (T)0.5) * hh, xb = xa + hh;
          const T va = v0_at(src, q, xa, y, z), vb = v0_at(src, q, xb, y, z);
          num[i][0] += va * v.x;
          num[i][1] += vb * v.y;
          den[i][0] += va * va;
          den[i][1] += vb * vb;
        }
      }
    }
    __syncthreads();
  }
  if (MODE == 1) {
    T* o = out + (long)(j0 + blockIdx.y) * N * N + (long)y0 * N;
    C* oc = reinterpret_cast<C*>(o);
#pragma unroll
    for (int i = 0; i < EPT; ++i) {
      const int e = tid + i * kThreads;
      if (EPT * kThreads == TY * L || e < TY * L) {
        const int r = e / L, m = e - r * L;
        oc[(long)r * L + m] = cmk(num[i][0] / den[i][0], num[i][1] / den[i][1]);
      }
    }
  }
}

template <typename T, int N, int TY> constexpr size_t row_r2c_smem() {
  using C = typename cpx<T>::t;
  constexpr int L = N / 2;
  return sizeof(C) * ((size_t)N + passtw_size<L>() + (size_t)TY * Smem<C, L>::ss + (size_t)(L + 1) * (TY + 1));
}
template <typename T, int N, int TC> constexpr size_t col_smem() {
  using C = typename cpx<T>::t;
  return sizeof(C) * ((size_t)passtw_size<N>() + (size_t)TC * Smem<C, N>::ss);
}
// small tiles for transforms of few planes (more CTAs in flight)
template <int N> struct SmallTile {
  static constexpr int row = divisor_at_most(N, 8);
  static constexpr int col = 4;
};
template <typename T, int N, int MODE> constexpr int row_c2r_tile() {
  constexpr int TY0 = RowTile<T, N>::v;
  return (MODE == 1 && TY0 % 2 == 0) ? TY0 / 2 : TY0;
}
template <typename T, int N, int MODE> constexpr size_t row_c2r_smem() {
  using C = typename cpx<T>::t;
  return sizeof(C) * ((size_t)N + passtw_size<N / 2>() + (size_t)row_c2r_tile<T, N, MODE>() * Smem<C, N / 2>::ss);
}

}  // namespace fr3d
