// Per-call tables of the Tikhonov solve (Sec. 5) that depend only on the geometry and on alpha:
// for every frequency class c and candidate alpha_k, with the regulariser alpha s^2,
//   D[k][c]  = 1 / (n^2 (||A^(c)||^2 + alpha_k s^2))             (solve weight, M = 1)
//   Ft[c][k] = (alpha_k s^2 / (||A^(c)||^2 + alpha_k s^2))^2     (residual filter, M = 1)
// They are cached in the handle and rebuilt only when the candidate list changes.
#include <string.h>

#include "ops.cuh"

namespace fr3d {

namespace {

struct AlphaList {
  double a[FR3D_MAX_ALPHAS];
};

__global__ void k_alpha_tables(AlphaList al, int na, const double* __restrict__ nrm, const double* __restrict__ s2,
                               int Cn, double inv_n2, double* __restrict__ Ft, float* __restrict__ D32,
                               double* __restrict__ D64) {
  const int total = na * Cn;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    const int c = idx / na, k = idx - c * na;
    const double as2 = al.a[k] * (*s2);
    const double d = 1.0 / (nrm[c] + as2);
    const double f = as2 * d;
    if (Ft) Ft[(long)c * na + k] = f * f;
    D64[(long)k * Cn + c] = d * inv_n2;
    D32[(long)k * Cn + c] = (float)(d * inv_n2);
  }
}

}  // namespace

int alpha_tables(Handle* H, const double* alphas, int n_alpha, cudaStream_t st) {
  if ((int)H->alpha_key.size() == n_alpha && memcmp(H->alpha_key.data(), alphas, n_alpha * sizeof(double)) == 0)
    return FR3D_OK;
  if (H->alpha_cap < n_alpha) {
    cudaFree(H->Ft);
    cudaFree(H->D32);
    cudaFree(H->D64);
    H->Ft = nullptr;
    H->D32 = nullptr;
    H->D64 = nullptr;
    H->alpha_cap = 0;
    FR3D_CUDA_TRY(cudaMalloc(&H->Ft, sizeof(double) * H->C * FR3D_MAX_ALPHAS));
    FR3D_CUDA_TRY(cudaMalloc(&H->D32, sizeof(float) * H->C * FR3D_MAX_ALPHAS));
    FR3D_CUDA_TRY(cudaMalloc(&H->D64, sizeof(double) * H->C * FR3D_MAX_ALPHAS));
    H->alpha_cap = FR3D_MAX_ALPHAS;
  }
  AlphaList al;
  for (int k = 0; k < n_alpha; ++k) al.a[k] = alphas[k];
  const double inv_n2 = 1.0 / ((double)H->n * H->n);
  const int total = n_alpha * H->C;
  k_alpha_tables<<<(total + 255) / 256, 256, 0, st>>>(al, n_alpha, H->nrm, H->s2, H->C, inv_n2, H->Ft, H->D32, H->D64);
  FR3D_CUDA_TRY(cudaGetLastError());
  H->alpha_key.assign(alphas, alphas + n_alpha);
  return FR3D_OK;
}

int fixed_table(Handle* H, double alpha, cudaStream_t st) {
  if (H->fixed_key == alpha && H->Dfix32) return FR3D_OK;
  if (!H->Dfix32) {
    FR3D_CUDA_TRY(cudaMalloc(&H->Dfix32, sizeof(float) * H->C));
    FR3D_CUDA_TRY(cudaMalloc(&H->Dfix64, sizeof(double) * H->C));
  }
  AlphaList al;
  al.a[0] = alpha;
  const double inv_n2 = 1.0 / ((double)H->n * H->n);
  k_alpha_tables<<<(H->C + 255) / 256, 256, 0, st>>>(al, 1, H->nrm, H->s2, H->C, inv_n2, nullptr, H->Dfix32,
                                                     H->Dfix64);
  FR3D_CUDA_TRY(cudaGetLastError());
  H->fixed_key = alpha;
  return FR3D_OK;
}

}  // namespace fr3d
