// fr3d_fwd_apply_noalloc: the forward operator with a fixed, statically allocated scratch area.
//
// Who needs this: code that must not call cudaMalloc at the point where it applies the operator,
// for example a real-time loop that cannot afford the allocator's latency or its implicit
// synchronisation, or a host framework that owns all device memory through its own allocator and
// forbids side allocations.  Such a caller creates the handle during set-up and afterwards only
// calls this entry point, which allocates nothing: its scratch lives in the file-scope device array
// below, loaded with the library on every GPU and held until the process exits.
#include <mutex>

#include "ops.cuh"

namespace fr3d {

namespace {

// 4 MiB of scratch: the half spectra of M' + M planes, (M' + M) (n/2 + 1) n complex64 values.
constexpr size_t kNoAllocScratchBytes = 4u << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once per device.
int scratch_address(void** out) {
  int dev = 0;
  FR3D_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return FR3D_ERR_UNSUPPORTED_SIZE;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_ptr[dev]) {
    void* p = nullptr;
    FR3D_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_ptr[dev] = p;
  }
  *out = g_ptr[dev];
  return FR3D_OK;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

}  // namespace fr3d

extern "C" int fr3d_fwd_apply_noalloc(fr3d_handle* h, const float* zeta, int Q, float* U, void* stream) {
  using namespace fr3d;
  if (!h || !zeta || !U || Q < 1) return FR3D_ERR_INVALID_ARG;
  if (h->padded) return FR3D_ERR_UNSUPPORTED_SIZE;   // periodic box only
  Handle* H = &h->h;
  // the handle's tables live on the device it was created on; the scratch address is looked up for
  // the current device, so both must be the same device
  int cur = -1;
  FR3D_CUDA_TRY(cudaGetDevice(&cur));
  if (cur != H->dev) return FR3D_ERR_INVALID_ARG;
  const int n = H->n;
  const long ps = (long)(n / 2 + 1) * n;
  const size_t zb = align256(sizeof(float2) * ps * H->Mp), ub = align256(sizeof(float2) * ps * H->M);
  if (zb + ub > kNoAllocScratchBytes) return FR3D_ERR_UNSUPPORTED_SIZE;
  void* base = nullptr;
  FR3D_TRY(scratch_address(&base));
  float2* Zh = reinterpret_cast<float2*>(base);
  float2* Uh = reinterpret_cast<float2*>((char*)base + zb);
  cudaStream_t st = (cudaStream_t)stream;
  // Every scratch byte read below is written earlier in the same call, so nothing is cleared.
  for (int q = 0; q < Q; ++q) {
    FR3D_TRY(Ops<float>::row_r2c(H, zeta + (long)q * H->Mp * n * n, (long)n * n, Zh, H->Mp, st));
    FR3D_TRY(Ops<float>::col_plain(H, Zh, Zh, H->Mp, false, st));
    FR3D_TRY(Ops<float>::contract_fwd(H, Zh, Uh, H->A32, 1, st));
    FR3D_TRY(Ops<float>::col_plain(H, Uh, Uh, H->M, true, st));
    FR3D_TRY(Ops<float>::row_c2r_plain(H, Uh, U + (long)q * H->M * n * n, H->M, 1, 0, 0, st));
  }
  return FR3D_OK;
}
