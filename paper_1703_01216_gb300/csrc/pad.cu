// The zero-padded box (pad = 2, Sec. 5: the plane replaced by the square Pi_xy, here twice the grid
// of R in x and y): a handle of an n x n grid with pad = 2 owns an inner handle of the 2n x 2n periodic
// box with the same spacing.  Data and unknowns sit in the box's low n x n corner with zeros elsewhere,
// so the box's circular convolution equals the aperiodic one over R; the inversion runs on the box
// (its frequencies, its alpha scale, its residuals) and the result is cropped back to R.  The entry
// points below embed their inputs into the handle's workspace, call the inner handle and crop.
#include <algorithm>

#include "common.cuh"
#include "ops.cuh"

namespace fr3d {

namespace {

// dst[p][y][x] (2n x 2n) = src[p][y][x] for y, x < n, 0 elsewhere
template <typename T>
__global__ void k_embed(const T* __restrict__ src, T* __restrict__ dst, long planes, int n) {
  const long N2 = 2L * n, per = N2 * N2, total = planes * per;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    const long p = e / per, r = e - p * per, y = r / N2, x = r - y * N2;
    dst[e] = (y < n && x < n) ? src[(p * n + y) * n + x] : T(0);
  }
}

// dst[p][y][x] (n x n) = src[p][y][x] of the 2n x 2n planes
template <typename T>
__global__ void k_crop(const T* __restrict__ src, T* __restrict__ dst, long planes, int n) {
  const long N2 = 2L * n, per = (long)n * n, total = planes * per;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    const long p = e / per, r = e - p * per, y = r / n, x = r - y * n;
    dst[e] = src[(p * N2 + y) * N2 + x];
  }
}

int grid_of(long total) { return (int)std::max<long>(1, std::min<long>((total + 255) / 256, 152L * 16)); }

int embed(const void* src, void* dst, long planes, int n, int precision, cudaStream_t st) {
  const long total = planes * 4L * n * n;
  if (precision == FR3D_PREC_FP64)
    k_embed<double><<<grid_of(total), 256, 0, st>>>((const double*)src, (double*)dst, planes, n);
  else
    k_embed<float><<<grid_of(total), 256, 0, st>>>((const float*)src, (float*)dst, planes, n);
  return cudaGetLastError() == cudaSuccess ? FR3D_OK : FR3D_ERR_CUDA;
}

int crop(const void* src, void* dst, long planes, int n, int precision, cudaStream_t st) {
  const long total = planes * (long)n * n;
  if (precision == FR3D_PREC_FP64)
    k_crop<double><<<grid_of(total), 256, 0, st>>>((const double*)src, (double*)dst, planes, n);
  else
    k_crop<float><<<grid_of(total), 256, 0, st>>>((const float*)src, (float*)dst, planes, n);
  return cudaGetLastError() == cudaSuccess ? FR3D_OK : FR3D_ERR_CUDA;
}

size_t elem_of(int precision) { return precision == FR3D_PREC_FP64 ? sizeof(double) : sizeof(float); }
size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }

// Workspace slices of the outer handle: bytes[i] each, 256-byte aligned
template <int K>
int slices(fr3d_handle* h, const size_t (&bytes)[K], void* (&out)[K]) {
  size_t total = 0;
  for (int i = 0; i < K; ++i) total += up256(bytes[i]);
  FR3D_TRY(ensure_ws(&h->h, total));
  char* p = static_cast<char*>(h->h.ws);
  for (int i = 0; i < K; ++i) {
    out[i] = p;
    p += up256(bytes[i]);
  }
  return FR3D_OK;
}

}  // namespace

int padded_fwd_apply(fr3d_handle* h, const void* zeta, int Q, void* U, int precision, cudaStream_t st) {
  if (Q < 1) return FR3D_ERR_INVALID_ARG;
  const int n = h->h.n;
  const size_t plane = 4 * (size_t)n * n * elem_of(precision);
  void* w[2];
  FR3D_TRY(slices<2>(h, {plane * Q * h->h.Mp, plane * Q * h->h.M}, w));
  FR3D_TRY(embed(zeta, w[0], (long)Q * h->h.Mp, n, precision, st));
  FR3D_TRY(fr3d_fwd_apply(h->padded, w[0], Q, w[1], precision, st));
  FR3D_TRY(crop(w[1], U, (long)Q * h->h.M, n, precision, st));
  h->h.last_launches = h->padded->h.last_launches + 2;
  return FR3D_OK;
}

int padded_zeta_from_xi(fr3d_handle* h, const void* xi, const fr3d_sources* sources, void* zeta, int precision,
                        cudaStream_t st) {
  if (!sources || sources->q < 1) return FR3D_ERR_INVALID_ARG;
  const int n = h->h.n, Q = sources->q;
  const size_t plane = 4 * (size_t)n * n * elem_of(precision);
  void* w[2];
  FR3D_TRY(slices<2>(h, {plane * h->h.Mp, plane * Q * h->h.Mp}, w));
  FR3D_TRY(embed(xi, w[0], h->h.Mp, n, precision, st));
  FR3D_TRY(fr3d_zeta_from_xi(h->padded, w[0], sources, w[1], precision, st));
  FR3D_TRY(crop(w[1], zeta, (long)Q * h->h.Mp, n, precision, st));
  h->h.last_launches = h->padded->h.last_launches + 2;
  return FR3D_OK;
}

int padded_choose_alpha(fr3d_handle* h, const void* U, int Q, const double* alphas, int n_alpha, double delta,
                        double tau, int precision, int* alpha_idx, double* residuals, int* info, cudaStream_t st) {
  if (Q < 1) return FR3D_ERR_INVALID_ARG;
  const int n = h->h.n;
  void* w[1];
  FR3D_TRY(slices<1>(h, {4 * (size_t)n * n * elem_of(precision) * Q * h->h.M}, w));
  FR3D_TRY(embed(U, w[0], (long)Q * h->h.M, n, precision, st));
  FR3D_TRY(fr3d_choose_alpha(h->padded, w[0], Q, alphas, n_alpha, delta, tau, precision, alpha_idx, residuals, info,
                             st));
  h->h.last_launches = h->padded->h.last_launches + 1;
  return FR3D_OK;
}

int padded_invert(fr3d_handle* h, const void* U, int Q, const fr3d_invert_opts* o, void* out, cudaStream_t st) {
  if (!o || Q < 1) return FR3D_ERR_INVALID_ARG;
  const int n = h->h.n;
  const size_t plane = 4 * (size_t)n * n * elem_of(o->precision);
  const long out_planes = (long)(o->output == FR3D_OUT_XI ? 1 : Q) * h->h.Mp;
  void* w[2];
  FR3D_TRY(slices<2>(h, {plane * Q * h->h.M, plane * out_planes}, w));
  FR3D_TRY(embed(U, w[0], (long)Q * h->h.M, n, o->precision, st));
  FR3D_TRY(fr3d_invert(h->padded, w[0], Q, o, w[1], st));
  FR3D_TRY(crop(w[1], out, out_planes, n, o->precision, st));
  h->h.last_launches = h->padded->h.last_launches + 2;
  return FR3D_OK;
}

int padded_invert_host(fr3d_handle* h, const void* U_host, int Q, const fr3d_invert_opts* o, void* out_host,
                       cudaStream_t st) {
  if (!o || Q < 1) return FR3D_ERR_INVALID_ARG;
  const int n = h->h.n;
  const size_t e = elem_of(o->precision), plane = (size_t)n * n * e;
  const long in_planes = (long)Q * h->h.M, out_planes = (long)(o->output == FR3D_OUT_XI ? 1 : Q) * h->h.Mp;
  void* w[4];
  FR3D_TRY(slices<4>(h, {plane * in_planes, 4 * plane * in_planes, 4 * plane * out_planes, plane * out_planes}, w));
  FR3D_CUDA_TRY(cudaMemcpyAsync(w[0], U_host, plane * in_planes, cudaMemcpyHostToDevice, st));
  FR3D_TRY(embed(w[0], w[1], in_planes, n, o->precision, st));
  FR3D_TRY(fr3d_invert(h->padded, w[1], Q, o, w[2], st));
  FR3D_TRY(crop(w[2], w[3], out_planes, n, o->precision, st));
  FR3D_CUDA_TRY(cudaMemcpyAsync(out_host, w[3], plane * out_planes, cudaMemcpyDeviceToHost, st));
  FR3D_CUDA_TRY(cudaStreamSynchronize(st));
  h->h.last_launches = h->padded->h.last_launches + 2;
  return FR3D_OK;
}

}  // namespace fr3d
