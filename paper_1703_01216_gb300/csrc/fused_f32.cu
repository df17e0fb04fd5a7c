// Launchers of the fused inverse (fused.cuh) and of the 1 / sum_q V0_q^2 table.
#include "fused.cuh"
#include "ops.cuh"

namespace fr3d {

// W_q = V0_q / sum_q' V0_q'^2 on the R grid (Algorithm 1 step 4 for several source parameters),
// in FP64, stored as FP32; depends only on the geometry and the sources
__global__ void k_wtab(float* __restrict__ W, int Q, int Mp, int n, Src64 src, double x0, double y0, double h,
                       const double* __restrict__ zr) {
  const long plane = (long)n * n, total = (long)Mp * plane;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int j = (int)(idx / plane);
    const long pix = idx % plane;
    const double x = x0 + ((double)(pix % n) + 0.5) * h, y = y0 + ((double)(pix / n) + 0.5) * h;
    double s = 0.0;
    for (int q = 0; q < Q; ++q) {
      const double v = v0_at(src, q, x, y, zr[j]);
      s += v * v;
    }
    for (int q = 0; q < Q; ++q) W[(long)q * total + idx] = (float)(v0_at(src, q, x, y, zr[j]) / s);
  }
}

namespace {

// Launch `kern` on `clusters` clusters of CL CTAs (a runtime cluster dimension; sizes above the
// portable 8 are allowed once per kernel, on the first launch, which happens outside any capture).
template <int CL, class K, class... Args>
int launch_clustered(K kern, int clusters, int nt, size_t sm, cudaStream_t st, Args... args) {
  FR3D_TRY(smem_optin(reinterpret_cast<const void*>(kern), sm));
  if constexpr (CL > 8) {
    static bool allowed = false;
    if (!allowed) {
      FR3D_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
      allowed = true;
    }
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(clusters * CL);
  cfg.blockDim = dim3(nt);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  FR3D_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, args...));
  return FR3D_OK;
}

template <int N, int MODE>
int launch_fused(const Handle* H, const FusedArgs& a, int nj, cudaStream_t st) {
  using G = FusedGeom<N>;
  constexpr size_t sm = MODE == 1 ? G::smem_xi : G::smem_zeta;
  return launch_clustered<G::CL>(k_inv_fused<N, MODE>, nj, G::NT, sm, st, a);
}

}  // namespace

bool fused_supported(int n) {
  switch (n) {
    case 16: case 24: case 32: case 48: case 64: case 96: case 128: case 192: case 256: case 384:
      return true;
  }
  return false;
}

int inv_fused_f32(const Handle* H, const float2* Uh, const float* Dd, const int* aidx, int nb, const float* W,
                  float* out, int Q, int j0, int nj, int output, cudaStream_t st) {
  FusedArgs a;
  a.Uh = Uh;
  a.A = H->A32;
  a.Dd = Dd;
  a.aidx = aidx;
  a.cband = H->cband;
  a.nb = nb;
  a.W = W;
  a.out = out;
  a.tw_n = H->tw32 + twiddle_offset(H, H->n);
  a.Q = Q;
  a.j0 = j0;
  a.Mp = H->Mp;
  const bool xi = output == FR3D_OUT_XI;
  switch (H->n) {
#define X(N) \
  case N: return xi ? launch_fused<N, 1>(H, a, nj, st) : launch_fused<N, 0>(H, a, nj, st);
    X(16) X(24) X(32) X(48) X(64) X(96) X(128) X(192) X(256) X(384)
#undef X
  }
  return FR3D_ERR_UNSUPPORTED_SIZE;
}

namespace {
template <int N, int MODE>
int launch_fused_batched(const FusedArgs* inst, const int2* map, int nclusters, cudaStream_t st) {
  using G = FusedGeom<N>;
  constexpr size_t sm = MODE == 1 ? G::smem_xi : G::smem_zeta;
  return launch_clustered<G::CL>(k_inv_fused_batched<N, MODE>, nclusters, G::NT, sm, st, inst, map);
}
}  // namespace

int inv_fused_batched_f32(int n, const FusedArgs* inst, const int2* map, int nclusters, int output, cudaStream_t st) {
  const bool xi = output == FR3D_OUT_XI;
  switch (n) {
#define X(N) \
  case N: return xi ? launch_fused_batched<N, 1>(inst, map, nclusters, st) : launch_fused_batched<N, 0>(inst, map, nclusters, st);
    X(16) X(24) X(32) X(48) X(64) X(96) X(128) X(192) X(256) X(384)
#undef X
  }
  return FR3D_ERR_UNSUPPORTED_SIZE;
}

void fused_args_f32(const Handle* H, const float2* Uh, const float* Dd, const int* aidx, int nb, const float* W,
                    float* out, int Q, FusedArgs* a) {
  a->Uh = Uh;
  a->A = H->A32;
  a->Dd = Dd;
  a->aidx = aidx;
  a->cband = H->cband;
  a->nb = nb;
  a->W = W;
  a->out = out;
  a->tw_n = H->tw32 + twiddle_offset(H, H->n);
  a->Q = Q;
  a->j0 = 0;
  a->Mp = H->Mp;
}

int build_wtab(const Handle* H, float* W, int Q, const double* pts64, int L, double coef, cudaStream_t st) {
  Src64 s;
  s.pts = pts64;
  s.L = L;
  s.coef = coef;
  const long total = (long)H->Mp * H->n * H->n;
  const int blocks = (int)std::min<long>((total + 255) / 256, 152L * 16);
  k_wtab<<<blocks, 256, 0, st>>>(W, Q, H->Mp, H->n, s, H->x0, H->y0, H->h, H->zr64);
  return cudaGetLastError() == cudaSuccess ? FR3D_OK : FR3D_ERR_CUDA;
}

}  // namespace fr3d
