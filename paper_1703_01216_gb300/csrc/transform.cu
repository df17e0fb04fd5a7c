// Algorithm 1 step 1 for the kernel (Sec. 5): the discrete transform of K = d/dz (1/r) (or of 1/r)
// sampled at the periodic lags, in FP64, and the per-frequency tables of Eq. (6).
//
// The sampled kernel is even in x and in y, so its DFT is the 2D cosine sum
//   K~(k1, k2) = h^2 sum_{a, b = 0}^{n/2} c_a c_b K(a h, b h, dz) cos(2 pi k1 a / n) cos(2 pi k2 b / n)
// with c = 1 at lags 0 and n/2 and 2 elsewhere (the two lags +-a of the periodic box), evaluated
// as two small dense products per depth difference.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <utility>
#include <vector>

#include "common.cuh"

namespace fr3d {

namespace {

constexpr double kTwoPi = 6.283185307179586476925286766559;

__global__ void k_samples(double* __restrict__ Ks, int H1, double h, const double* __restrict__ dz, int nij,
                          int kind) {
  const long total = (long)nij * H1 * H1;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int a = (int)(idx % H1);
    const int b = (int)((idx / H1) % H1);
    const int ij = (int)(idx / ((long)H1 * H1));
    const double x = a * h, y = b * h, z = dz[ij];
    const double r2 = x * x + y * y + z * z;
    // K = d/dz (1/r) = -z / r^3 (Eq. (4)), or 1/r (the first equation of Sec. 3, for V2 data)
    Ks[idx] = kind == FR3D_K_INV_R ? 1.0 / sqrt(r2) : -z / (r2 * sqrt(r2));
  }
}

// Batched FP64 product  Out_z[i][j] = scale * sum_k A_z[i][k] * B_z(k, j),  B_z(k, j) = B[j][k] if BT else B[k][j].
// Plain 16 x 16 shared-memory tiles (cold path, once per geometry).
template <bool BT>
__global__ void k_dgemm(const double* __restrict__ A, long sA, const double* __restrict__ B, long sB,
                        double* __restrict__ Out, long sO, int n, double scale) {
  __shared__ double ta[16][17], tb[16][17];
  const int z = blockIdx.z;
  A += z * sA;
  B += z * sB;
  Out += z * sO;
  const int i = blockIdx.y * 16 + threadIdx.y, j = blockIdx.x * 16 + threadIdx.x;
  double acc = 0.0;
  for (int k0 = 0; k0 < n; k0 += 16) {
    const int ka = k0 + threadIdx.x, kb = k0 + threadIdx.y;
    ta[threadIdx.y][threadIdx.x] = (i < n && ka < n) ? A[(long)i * n + ka] : 0.0;
    if (BT)
      tb[threadIdx.y][threadIdx.x] = (j < n && kb < n) ? B[(long)j * n + kb] : 0.0;
    else
      tb[threadIdx.y][threadIdx.x] = (j < n && kb < n) ? B[(long)kb * n + j] : 0.0;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) acc = fma(ta[threadIdx.y][k], tb[k][threadIdx.x], acc);
    __syncthreads();
  }
  if (i < n && j < n) Out[(long)i * n + j] = scale * acc;
}

// A64[c][i][j] = nu_j K~(p, q; z_i - z'_j) for class c = (p, q), and ||A^(c)||_F^2.
__global__ void k_classes(const double* __restrict__ Kh, int H1, int C, int M, int Mp,
                          const double* __restrict__ nu, double* __restrict__ A64, double* __restrict__ nrm) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  int p = (int)((sqrt(8.0 * c + 1.0) - 1.0) * 0.5);
  while ((p + 1) * (p + 2) / 2 <= c) ++p;
  while (p * (p + 1) / 2 > c) --p;
  const int q = c - p * (p + 1) / 2;
  double s = 0.0;
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < Mp; ++j) {
      const double v = nu[j] * Kh[((long)(i * Mp + j) * H1 + p) * H1 + q];
      A64[((long)c * M + i) * Mp + j] = v;
      s = fma(v, v, s);
    }
  nrm[c] = s;
}

__global__ void k_max(const double* __restrict__ v, int n, double* __restrict__ out) {
  __shared__ double red[256];
  double m = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, v[i]);
  red[threadIdx.x] = m;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

template <typename T>
__global__ void k_dense(const double* __restrict__ A64, int n, int M, int Mp, T* __restrict__ out) {
  // out[(i Mp + j)][kx][ky] = A64[class(kx, ky)][i][j]
  const int H1 = n / 2 + 1;
  const long total = (long)M * Mp * H1 * n;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int ky = (int)(idx % n);
    const int kx = (int)((idx / n) % H1);
    const int ij = (int)(idx / ((long)n * H1));
    out[idx] = (T)A64[(long)class_of(kx, ky, n) * M * Mp + ij];
  }
}

bool supported_n(int n) {
  if (n < 16 || n > 512) return false;
  int m = n;
  while (m % 2 == 0) m /= 2;
  while (m % 3 == 0) m /= 3;
  if (m != 1) return false;
  bool a = false, b = false;
  for (int i = 0; i < kNumLengths; ++i) {
    if (kLengths[i] == n) a = true;
    if (kLengths[i] == n / 2) b = true;
  }
  return a && b;
}

}  // namespace

int twiddle_offset(const Handle* H, int L) {
  for (int i = 0; i < kNumLengths; ++i)
    if (kLengths[i] == L) return H->tw_off[i];
  return -1;
}

// CTAs of `kernel` that fit on one SM by its registers, threads and shared memory (the device's full
// per-SM shared memory; the occupancy calculator's answer depends on the carveout it assumes).
int resident_ctas(const void* kernel, int threads, size_t dyn_smem) {
  cudaFuncAttributes fa;
  int dev = 0, smem_sm = 0, regs_sm = 0, thr_sm = 0, blk_sm = 0, reserved = 0;
  if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&blk_sm, cudaDevAttrMaxBlocksPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  const int warps = (threads + 31) / 32;
  const int regs_warp = ((fa.numRegs * 32 + 255) / 256) * 256;   // allocation unit of 256 registers
  int n = std::min(blk_sm, thr_sm / std::max(threads, 1));
  if (regs_warp > 0) n = std::min(n, regs_sm / (regs_warp * warps));
  const size_t per = dyn_smem + fa.sharedSizeBytes + (size_t)reserved;
  if (per > 0) n = std::min<int>(n, (int)(smem_sm / per));
  return std::max(n, 1);
}

int smem_optin(const void* kernel, size_t bytes) {
  // static shared memory counts against the same 48 KB default, so opt in whenever dynamic memory
  // is used (at most once per kernel and device)
  if (bytes == 0) return FR3D_OK;
  struct Entry {
    const void* k;
    int dev;
    size_t bytes;
  };
  static std::mutex mu;
  static std::vector<Entry> done;
  int dev = 0;
  FR3D_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  for (auto& d : done)
    if (d.k == kernel && d.dev == dev) {
      if (d.bytes >= bytes) return FR3D_OK;
      FR3D_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
      d.bytes = bytes;
      return FR3D_OK;
    }
  FR3D_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  done.push_back({kernel, dev, bytes});
  return FR3D_OK;
}

int ensure_ws(Handle* H, size_t bytes) {
  if (bytes <= H->ws_bytes) return FR3D_OK;
  if (H->ws) {
    cudaFree(H->ws);
    H->ws = nullptr;
    H->ws_bytes = 0;
  }
  FR3D_CUDA_TRY(cudaMalloc(&H->ws, bytes));
  H->ws_bytes = bytes;
  return FR3D_OK;
}

int build_dense64(Handle* H, cudaStream_t st) {
  if (H->A64d) return FR3D_OK;
  const int H1 = H->n / 2 + 1;
  const size_t cnt = (size_t)H->M * H->Mp * H1 * H->n;
  FR3D_CUDA_TRY(cudaMalloc(&H->A64d, cnt * sizeof(double)));
  k_dense<double><<<1024, 256, 0, st>>>(H->A64, H->n, H->M, H->Mp, H->A64d);
  FR3D_CUDA_TRY(cudaGetLastError());
  return FR3D_OK;
}

static int kernel_transform_impl(const fr3d_geometry* g, Handle* H, cudaStream_t st) {
  const int n = g->nx;
  H->n = n;
  H->M = g->nzy;
  H->Mp = g->nzr;
  H->C = num_classes(n);
  H->kind = g->kernel_kind;
  H->x0 = g->x0;
  H->y0 = g->y0;
  H->h = g->hx;
  H->zr.assign(g->zr, g->zr + g->nzr);
  H->zy.assign(g->zy, g->zy + g->nzy);
  H->nu.resize(g->nzr);
  for (int j = 0; j < g->nzr; ++j) {
    if (g->nu) H->nu[j] = g->nu[j];
    else H->nu[j] = g->nzr > 1 ? fabs(g->zr[1] - g->zr[0]) : 1.0;
  }
  H->create_stream = st;
  FR3D_CUDA_TRY(cudaGetDevice(&H->dev));

  // twiddles
  int total = 0;
  for (int i = 0; i < kNumLengths; ++i) {
    H->tw_off[i] = total;
    total += kLengths[i];
  }
  std::vector<float2> t32(total);
  std::vector<double2> t64(total);
  for (int i = 0; i < kNumLengths; ++i) {
    const int L = kLengths[i];
    for (int t = 0; t < L; ++t) {
      const double ang = kTwoPi * (double)t / (double)L;
      const double c = cos(ang), s = -sin(ang);
      t64[H->tw_off[i] + t] = make_double2(c, s);
      t32[H->tw_off[i] + t] = make_float2((float)c, (float)s);
    }
  }
  FR3D_CUDA_TRY(cudaMalloc(&H->tw32, total * sizeof(float2)));
  FR3D_CUDA_TRY(cudaMalloc(&H->tw64, total * sizeof(double2)));
  FR3D_CUDA_TRY(cudaMemcpy(H->tw32, t32.data(), total * sizeof(float2), cudaMemcpyHostToDevice));
  FR3D_CUDA_TRY(cudaMemcpy(H->tw64, t64.data(), total * sizeof(double2), cudaMemcpyHostToDevice));

  const int H1 = n / 2 + 1;
  const int nij = H->M * H->Mp;
  std::vector<double> dz(nij), cw((size_t)H1 * H1);
  std::vector<float> zr32(H->Mp);
  for (int j = 0; j < H->Mp; ++j) zr32[j] = (float)H->zr[j];
  for (int i = 0; i < H->M; ++i)
    for (int j = 0; j < H->Mp; ++j) dz[i * H->Mp + j] = H->zy[i] - H->zr[j];
  for (int k = 0; k < H1; ++k)
    for (int a = 0; a < H1; ++a) {
      const double ca = (a == 0 || 2 * a == n) ? 1.0 : 2.0;
      const long t = ((long)k * a) % n;
      cw[(size_t)k * H1 + a] = ca * cos(kTwoPi * (double)t / (double)n);
    }
  double *d_dz = nullptr, *d_cw = nullptr, *d_ks = nullptr, *d_s = nullptr, *d_kh = nullptr, *d_nu = nullptr;
  const size_t plane = (size_t)H1 * H1;
  int rc = FR3D_OK;
  do {
#define TRYB(x)                                                   \
  {                                                               \
    cudaError_t e_ = (x);                                         \
    if (e_ != cudaSuccess) {                                      \
      rc = e_ == cudaErrorMemoryAllocation ? FR3D_ERR_OOM : FR3D_ERR_CUDA; \
      break;                                                      \
    }                                                             \
  }
    TRYB(cudaMalloc(&d_dz, nij * sizeof(double)));
    TRYB(cudaMalloc(&d_nu, H->Mp * sizeof(double)));
    TRYB(cudaMalloc(&d_cw, plane * sizeof(double)));
    TRYB(cudaMalloc(&d_ks, nij * plane * sizeof(double)));
    TRYB(cudaMalloc(&d_s, nij * plane * sizeof(double)));
    TRYB(cudaMalloc(&d_kh, nij * plane * sizeof(double)));
    TRYB(cudaMalloc(&H->A64, (size_t)H->C * nij * sizeof(double)));
    TRYB(cudaMalloc(&H->nrm, (size_t)H->C * sizeof(double)));
    TRYB(cudaMalloc(&H->s2, sizeof(double)));
    TRYB(cudaMalloc(&H->A32, (size_t)nij * H1 * n * sizeof(float)));
    TRYB(cudaMalloc(&H->zr64, H->Mp * sizeof(double)));
    TRYB(cudaMalloc(&H->zr32, H->Mp * sizeof(float)));
    TRYB(cudaMalloc(&H->counter, sizeof(unsigned)));
    TRYB(cudaMalloc(&H->idx_scratch, sizeof(int) * FR3D_MAX_BANDS));
    TRYB(cudaMalloc(&H->zero_idx, sizeof(int)));
    TRYB(cudaMalloc(&H->info_scratch, sizeof(int)));
    TRYB(cudaMemsetAsync(H->counter, 0, sizeof(unsigned), st));
    TRYB(cudaMemsetAsync(H->zero_idx, 0, sizeof(int), st));
    TRYB(cudaMemcpyAsync(d_dz, dz.data(), nij * sizeof(double), cudaMemcpyHostToDevice, st));
    TRYB(cudaMemcpyAsync(d_nu, H->nu.data(), H->Mp * sizeof(double), cudaMemcpyHostToDevice, st));
    TRYB(cudaMemcpyAsync(d_cw, cw.data(), plane * sizeof(double), cudaMemcpyHostToDevice, st));
    TRYB(cudaMemcpyAsync(H->zr64, H->zr.data(), H->Mp * sizeof(double), cudaMemcpyHostToDevice, st));
    TRYB(cudaMemcpyAsync(H->zr32, zr32.data(), H->Mp * sizeof(float), cudaMemcpyHostToDevice, st));
    k_samples<<<1024, 256, 0, st>>>(d_ks, H1, H->h, d_dz, nij, H->kind);
    dim3 blk(16, 16), grd((H1 + 15) / 16, (H1 + 15) / 16, nij);
    // S[ij][b][k1] = sum_a Ks[ij][b][a] cw[k1][a]
    k_dgemm<true><<<grd, blk, 0, st>>>(d_ks, plane, d_cw, 0, d_s, plane, H1, 1.0);
    // Kh[ij][k2][k1] = h^2 sum_b cw[k2][b] S[ij][b][k1]
    k_dgemm<false><<<grd, blk, 0, st>>>(d_cw, 0, d_s, plane, d_kh, plane, H1, H->h * H->h);
    k_classes<<<(H->C + 127) / 128, 128, 0, st>>>(d_kh, H1, H->C, H->M, H->Mp, d_nu, H->A64, H->nrm);
    k_max<<<1, 256, 0, st>>>(H->nrm, H->C, H->s2);
    k_dense<float><<<1024, 256, 0, st>>>(H->A64, n, H->M, H->Mp, H->A32);
    TRYB(cudaGetLastError());
    TRYB(cudaMemcpyAsync(&H->s2_host, H->s2, sizeof(double), cudaMemcpyDeviceToHost, st));
    TRYB(cudaStreamSynchronize(st));
    H->synced = true;
#undef TRYB
  } while (0);
  cudaFree(d_dz);
  cudaFree(d_nu);
  cudaFree(d_cw);
  cudaFree(d_ks);
  cudaFree(d_s);
  cudaFree(d_kh);
  return rc;
}

void handle_free(Handle* H) {
  void* ptrs[] = {H->A64, H->nrm, H->s2, H->A32, H->A64d, H->tw32, H->tw64, H->Ft, H->D32, H->D64,
                  H->Dfix32, H->Dfix64, H->zr64, H->zr32, H->wtab, H->Dd32, H->Ddfix32, H->pts32, H->pts64, H->counter, H->idx_scratch, H->zero_idx,
                  H->info_scratch, H->partials, H->cband, H->bbin, H->mlam, H->mUt, H->mW, H->rhs_buf, H->ws,
                  H->inv2_buf, H->qctl};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (int k = 0; k < 3; ++k) {
    if (H->tc_hi[k]) cudaFree(H->tc_hi[k]);
    if (H->tc_lo[k]) cudaFree(H->tc_lo[k]);
  }
  for (int i = 0; i < Handle::kMaxEv; ++i)
    if (H->ev[i]) cudaEventDestroy(H->ev[i]);
  if (H->pi) fr3d_handle_destroy(H->pi);
  H->pi = nullptr;
}

int validate_geometry(const fr3d_geometry* g) {
  if (!g || !g->zr || !g->zy || g->nzr < 1 || g->nzy < 1) return FR3D_ERR_INVALID_ARG;
  if (g->kernel_kind != FR3D_K_DZ_INV_R && g->kernel_kind != FR3D_K_INV_R) return FR3D_ERR_INVALID_ARG;
  if (g->nx != g->ny || !supported_n(g->nx)) return FR3D_ERR_UNSUPPORTED_SIZE;
  if (g->pad != 1 && g->pad != 2) return FR3D_ERR_UNSUPPORTED_SIZE;
  if (g->pad == 2 && !supported_n(2 * g->nx)) return FR3D_ERR_UNSUPPORTED_SIZE;
  if (!(g->hx > 0) || g->hx != g->hy || !isfinite(g->x0) || !isfinite(g->y0)) return FR3D_ERR_BAD_GEOMETRY;
  for (int i = 0; i < g->nzy; ++i)
    for (int j = 0; j < g->nzr; ++j) {
      const double d = g->zy[i] - g->zr[j];
      if (!(d != 0.0) || !isfinite(d)) return FR3D_ERR_BAD_GEOMETRY;  // R and Y must be disjoint (Sec. 1)
    }
  if (g->nu)
    for (int j = 0; j < g->nzr; ++j)
      if (!isfinite(g->nu[j])) return FR3D_ERR_BAD_GEOMETRY;
  return FR3D_OK;
}

}  // namespace fr3d

extern "C" int fr3d_kernel_transform(const fr3d_geometry* geom, fr3d_handle** out, void* stream) {
  if (!out) return FR3D_ERR_INVALID_ARG;
  *out = nullptr;
  int rc = fr3d::validate_geometry(geom);
  if (rc != FR3D_OK) return rc;
  fr3d_handle* h = new (std::nothrow) fr3d_handle();
  if (!h) return FR3D_ERR_OOM;
  if (geom->pad == 2) {
    // the zero-padded box: an inner handle of the 2n x 2n grid with the same spacing and origin; this
    // handle keeps the n x n sizes (pad.cu)
    fr3d_geometry g2 = *geom;
    g2.nx = g2.ny = 2 * geom->nx;
    g2.pad = 1;
    rc = fr3d_kernel_transform(&g2, &h->padded, stream);
    if (rc != FR3D_OK) {
      delete h;
      return rc;
    }
    h->h.n = geom->nx;
    h->h.M = geom->nzy;
    h->h.Mp = geom->nzr;
    h->h.dev = h->padded->h.dev;
    h->h.s2_host = h->padded->h.s2_host;
    *out = h;
    return FR3D_OK;
  }
  rc = fr3d::kernel_transform_impl(geom, &h->h, (cudaStream_t)stream);
  if (rc != FR3D_OK) {
    fr3d::handle_free(&h->h);
    delete h;
    return rc;
  }
  *out = h;
  return FR3D_OK;
}

extern "C" void fr3d_handle_destroy(fr3d_handle* h) {
  if (!h) return;
  cudaDeviceSynchronize();
  if (h->padded) fr3d_handle_destroy(h->padded);
  fr3d::handle_free(&h->h);
  delete h;
}

extern "C" int fr3d_handle_query(fr3d_handle* h, int* n, int* m, int* mp, double* s2) {
  if (!h) return FR3D_ERR_INVALID_ARG;
  if (n) *n = h->h.n;
  if (m) *m = h->h.M;
  if (mp) *mp = h->h.Mp;
  if (s2) *s2 = h->h.s2_host;
  return FR3D_OK;
}
