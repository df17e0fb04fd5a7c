// Right-hand side of Eq. (7) from the measured z-derivative of V2 on Y (Sec. 3, Sec. 6):
//     U(x) = 2 pi dV2/dx3(x) + (A2 / 2) sum_l d/dx3 (1/|x - x_l|) - A0 / (4 pi c0^2) I(x),
//     I(x) = sum_l integral over Pi of d/dx3 (1/|x - x'|) / |x' - x_l| dx',
// with R^3 replaced by the box Pi (Sec. 5; the paper simulates its data over Pi, Sec. 6).  I is the
// discrete operator of Eq. (4) on Pi's depth grid applied to the density f(x') = sum_l 1/|x' - x_l|;
// the kernels here build f and combine the three terms.
#include <math.h>

#include "ops.cuh"

namespace fr3d {

namespace {

// f[q][k][y][x] = sum_l 1 / |(x_a, y_b, zp_k) - x_{q,l}| (FP64 sums, FP32 result)
__global__ void k_pi_density(float* __restrict__ f, int Q, int npi, int n, double x0, double h, double half,
                             const double* __restrict__ pts, int L) {
  const long plane = (long)n * n, total = (long)Q * npi * plane;
  const double dz = 2.0 * half / npi;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int q = (int)(idx / (npi * plane));
    const int k = (int)((idx / plane) % npi);
    const long pix = idx % plane;
    const double x = x0 + ((double)(pix % n) + 0.5) * h, y = x0 + ((double)(pix / n) + 0.5) * h;
    const double z = -half + ((double)k + 0.5) * dz;
    double s = 0.0;
    for (int l = 0; l < L; ++l) {
      const double* p = pts + ((long)q * L + l) * 3;
      const double ddx = x - p[0], ddy = y - p[1], ddz = z - p[2];
      s += 1.0 / sqrt(ddx * ddx + ddy * ddy + ddz * ddz);
    }
    f[idx] = (float)s;
  }
}

struct Depths {
  double z[FR3D_MAX_OBS_DEPTHS];
};

// U = 2 pi d + (A2 / 2) sum_l K(x - x_l) - coef I, K = d/dx3 (1/r) = -dz / r^3 (FP64 per point)
__global__ void k_rhs_combine(const float* __restrict__ d, const float* __restrict__ I, float* __restrict__ U, int Q,
                              int M, int n, double x0, double h, Depths zy, const double* __restrict__ pts, int L,
                              double a2half, double coef) {
  const long plane = (long)n * n, total = (long)Q * M * plane;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int q = (int)(idx / (M * plane));
    const int i = (int)((idx / plane) % M);
    const long pix = idx % plane;
    const double x = x0 + ((double)(pix % n) + 0.5) * h, y = x0 + ((double)(pix / n) + 0.5) * h;
    double s = 0.0;
    for (int l = 0; l < L; ++l) {
      const double* p = pts + ((long)q * L + l) * 3;
      const double ddx = x - p[0], ddy = y - p[1], ddz = zy.z[i] - p[2];
      const double r2 = ddx * ddx + ddy * ddy + ddz * ddz;
      s -= ddz / (r2 * sqrt(r2));
    }
    U[idx] = (float)(6.283185307179586476925286766559 * (double)d[idx] + a2half * s - coef * (double)I[idx]);
  }
}

}  // namespace

int rhs_pi_density(float* f, int Q, int npi, int n, double x0, double h, double half, const double* pts, int L,
                   cudaStream_t st) {
  const long total = (long)Q * npi * n * n;
  const int blocks = (int)std::min<long>((total + 255) / 256, 152L * 16);
  k_pi_density<<<blocks, 256, 0, st>>>(f, Q, npi, n, x0, h, half, pts, L);
  FR3D_CUDA_TRY(cudaGetLastError());
  return FR3D_OK;
}

int rhs_combine(const Handle* H, const float* d, const float* I, float* U, int Q, const double* pts, int L,
                double A2, double coef, cudaStream_t st) {
  Depths zy;
  for (int i = 0; i < H->M; ++i) zy.z[i] = H->zy[i];
  const long total = (long)Q * H->M * H->n * H->n;
  const int blocks = (int)std::min<long>((total + 255) / 256, 152L * 16);
  k_rhs_combine<<<blocks, 256, 0, st>>>(d, I, U, Q, H->M, H->n, H->x0, H->h, zy, pts, L, 0.5 * A2, coef);
  FR3D_CUDA_TRY(cudaGetLastError());
  return FR3D_OK;
}

}  // namespace fr3d
