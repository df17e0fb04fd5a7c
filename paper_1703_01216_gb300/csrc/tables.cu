// Per-call tables of the Tikhonov solve (Sec. 5) that depend only on the geometry and on alpha:
// for every frequency class c and candidate alpha_k, with the regulariser alpha s^2,
//   D[k][c]  = 1 / (n^2 (||A^(c)||^2 + alpha_k s^2))             (solve weight, M = 1)
//   Ft[c][k] = (alpha_k s^2 / (||A^(c)||^2 + alpha_k s^2))^2     (residual filter, M = 1)
// They are cached in the handle and rebuilt only when the candidate list changes; D also has a
// dense copy in the half-spectrum layout for the fused inverse.
#include <math.h>
#include <string.h>

#include <vector>

#include "ops.cuh"

namespace fr3d {

namespace {

struct AlphaList {
  double a[FR3D_MAX_ALPHAS];
};

// Per class c (M = 1, a = A^(c), n_c = ||a||^2) and candidate k, the solution of a frequency of the class
// is zeta~ = D a U~ (with the inverse DFT's 1/n^2 folded into D) and its squared residual is Ft |U~|^2:
//   Tikhonov (ra = 0): D = 1 / (n_c + alpha s^2),            Ft = (alpha s^2 / (n_c + alpha s^2))^2;
//   TSVD     (ra = 1): D = 1 / n_c if n_c >= alpha s^2 else 0, Ft = 0 if kept else 1
// (the single singular value of the 1 x M' system is sqrt(n_c); kept, the fit is exact).
__global__ void k_alpha_tables(AlphaList al, int na, int ra, const double* __restrict__ nrm,
                               const double* __restrict__ s2, int Cn, double inv_n2, double* __restrict__ Ft,
                               float* __restrict__ D32, double* __restrict__ D64) {
  const int total = na * Cn;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    const int c = idx / na, k = idx - c * na;
    const double as2 = al.a[k] * (*s2);
    double d, f2;
    if (ra == FR3D_RA_TSVD) {
      const bool keep = nrm[c] >= as2;
      d = keep ? 1.0 / nrm[c] : 0.0;
      f2 = keep ? 0.0 : 1.0;
    } else {
      d = 1.0 / (nrm[c] + as2);
      const double f = as2 * d;
      f2 = f * f;
    }
    if (Ft) Ft[(long)c * na + k] = f2;
    D64[(long)k * Cn + c] = d * inv_n2;
    D32[(long)k * Cn + c] = (float)(d * inv_n2);
  }
}

// dense per-bin copy of the solve weights: Dd[k][kx][ky] = D[k][class(kx, ky)]
__global__ void k_dense_d(const float* __restrict__ D, int na, int Cn, int n, float* __restrict__ Dd) {
  const long ps = (long)(n / 2 + 1) * n, total = na * ps;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int k = (int)(idx / ps);
    const long bin = idx % ps;
    Dd[idx] = D[(long)k * Cn + class_of((int)(bin / n), (int)(bin % n), n)];
  }
}

// bbin[o] = band of the class of half-spectrum bin o = kx n + ky
__global__ void k_bin_bands(const unsigned char* __restrict__ cband, int n, int ps, unsigned char* __restrict__ bbin) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o < ps) bbin[o] = cband[class_of(o / n, o % n, n)];
}

}  // namespace

int alpha_tables(Handle* H, const double* alphas, int n_alpha, int ra, cudaStream_t st) {
  if (H->alpha_ra == ra && (int)H->alpha_key.size() == n_alpha &&
      memcmp(H->alpha_key.data(), alphas, n_alpha * sizeof(double)) == 0)
    return FR3D_OK;
  if (H->alpha_cap < n_alpha) {
    cudaFree(H->Ft);
    cudaFree(H->D32);
    cudaFree(H->D64);
    cudaFree(H->Dd32);
    H->Ft = nullptr;
    H->D32 = nullptr;
    H->D64 = nullptr;
    H->Dd32 = nullptr;
    H->alpha_cap = 0;
    const size_t ps = (size_t)(H->n / 2 + 1) * H->n;
    FR3D_CUDA_TRY(cudaMalloc(&H->Ft, sizeof(double) * H->C * n_alpha));
    FR3D_CUDA_TRY(cudaMalloc(&H->D32, sizeof(float) * H->C * n_alpha));
    FR3D_CUDA_TRY(cudaMalloc(&H->D64, sizeof(double) * H->C * n_alpha));
    FR3D_CUDA_TRY(cudaMalloc(&H->Dd32, sizeof(float) * ps * n_alpha));
    H->alpha_cap = n_alpha;
  }
  AlphaList al;
  for (int k = 0; k < n_alpha; ++k) al.a[k] = alphas[k];
  const double inv_n2 = 1.0 / ((double)H->n * H->n);
  const int total = n_alpha * H->C;
  k_alpha_tables<<<(total + 255) / 256, 256, 0, st>>>(al, n_alpha, ra, H->nrm, H->s2, H->C, inv_n2, H->Ft, H->D32,
                                                      H->D64);
  k_dense_d<<<1024, 256, 0, st>>>(H->D32, n_alpha, H->C, H->n, H->Dd32);
  FR3D_CUDA_TRY(cudaGetLastError());
  H->alpha_key.assign(alphas, alphas + n_alpha);
  H->alpha_ra = ra;
  return FR3D_OK;
}

// The handle's partial-sum buffer: data, then the alpha rule's group tickets at a fixed offset.
// Data: the alpha rule's [blocks][O] block sums and [groups][O] group sums (blocks of 64 classes,
// groups of 8 blocks, O <= FR3D_MAX_ALPHAS * FR3D_MAX_BANDS); the M > 1 rule's [blocks of 64
// classes][bands][alphas]; the learned rule's at most 2 * 152 blocks of FR3D_MAX_BANDS sums.
// Tickets: one unsigned per group, zero between launches (zeroed here, reset by the launch that
// used them).
static long partial_data_doubles(int C) {
  const long blocks = (C + 63) / 64, groups = (blocks + 7) / 8;
  return std::max((blocks + groups) * (long)FR3D_MAX_ALPHAS * FR3D_MAX_BANDS, 2L * 152 * FR3D_MAX_BANDS);
}

int ensure_partials(Handle* H) {
  const long data = partial_data_doubles(H->C);
  const long groups = ((H->C + 63) / 64 + 7) / 8;
  const long need = data + (groups + 1) / 2;
  if (H->partial_cap >= need) return FR3D_OK;
  if (H->partials) cudaFree(H->partials);
  H->partials = nullptr;
  H->partial_cap = 0;
  FR3D_CUDA_TRY(cudaMalloc(&H->partials, sizeof(double) * need));
  FR3D_CUDA_TRY(cudaMemset(H->partials + data, 0, sizeof(double) * (need - data)));
  FR3D_CUDA_TRY(cudaDeviceSynchronize());
  H->partial_cap = (int)need;
  return FR3D_OK;
}

unsigned* alpha_tickets(const Handle* H) { return reinterpret_cast<unsigned*>(H->partials + partial_data_doubles(H->C)); }

// Radial band of frequency class (p, q): floor(nb |k| / |k|max) with |k| = sqrt(p^2 + q^2) and
// |k|max = sqrt(2) n/2 (clamped to nb - 1).  count[b] = number of grid frequencies in band b (each
// class counts its members with the weights of the stored half spectrum: 1 on the kx = 0 and
// kx = n/2 columns, 2 elsewhere).
int ensure_bands(Handle* H, int nb, std::vector<double>* count) {
  if (H->cband_nb != nb || !H->cband) {
    const int n = H->n;
    std::vector<unsigned char> band(H->C);
    std::vector<double> cnt(nb, 0.0);
    const double rmax = sqrt(2.0) * (n / 2);
    for (int p = 0; p <= n / 2; ++p)
      for (int q = 0; q <= p; ++q) {
        const int c = p * (p + 1) / 2 + q;
        int b = (int)(nb * sqrt((double)p * p + (double)q * q) / rmax);
        if (b > nb - 1) b = nb - 1;
        band[c] = (unsigned char)b;
        auto wt = [&](int kx) { return (kx == 0 || 2 * kx == n) ? 1.0 : 2.0; };
        double w = wt(p);
        if (q != 0 && 2 * q != n) w += wt(p);
        if (p != q) {
          w += wt(q);
          if (p != 0 && 2 * p != n) w += wt(q);
        }
        cnt[b] += w;
      }
    if (!H->cband) FR3D_CUDA_TRY(cudaMalloc(&H->cband, H->C));
    FR3D_CUDA_TRY(cudaMemcpy(H->cband, band.data(), H->C, cudaMemcpyHostToDevice));
    const int ps = (n / 2 + 1) * n;
    if (!H->bbin) FR3D_CUDA_TRY(cudaMalloc(&H->bbin, ps));
    k_bin_bands<<<(ps + 255) / 256, 256>>>(H->cband, n, ps, H->bbin);
    FR3D_CUDA_TRY(cudaGetLastError());
    FR3D_CUDA_TRY(cudaDeviceSynchronize());
    H->cband_nb = nb;
    H->band_count = cnt;
  }
  if (count) *count = H->band_count;
  return FR3D_OK;
}

int fixed_table(Handle* H, double alpha, int ra, cudaStream_t st) {
  if (H->fixed_key == alpha && H->fixed_ra == ra && H->Dfix32) return FR3D_OK;
  if (!H->Dfix32) {
    FR3D_CUDA_TRY(cudaMalloc(&H->Dfix32, sizeof(float) * H->C));
    FR3D_CUDA_TRY(cudaMalloc(&H->Dfix64, sizeof(double) * H->C));
    FR3D_CUDA_TRY(cudaMalloc(&H->Ddfix32, sizeof(float) * (size_t)(H->n / 2 + 1) * H->n));
  }
  AlphaList al;
  al.a[0] = alpha;
  const double inv_n2 = 1.0 / ((double)H->n * H->n);
  k_alpha_tables<<<(H->C + 255) / 256, 256, 0, st>>>(al, 1, ra, H->nrm, H->s2, H->C, inv_n2, nullptr, H->Dfix32,
                                                     H->Dfix64);
  k_dense_d<<<256, 256, 0, st>>>(H->Dfix32, 1, H->C, H->n, H->Ddfix32);
  FR3D_CUDA_TRY(cudaGetLastError());
  H->fixed_key = alpha;
  H->fixed_ra = ra;
  return FR3D_OK;
}

}  // namespace fr3d
