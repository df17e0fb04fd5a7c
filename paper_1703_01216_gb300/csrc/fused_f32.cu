// Launchers of the fused inverse (fused.cuh), its tile-variant autotuner, and the combination table.
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>

#include "fused.cuh"
#include "ops.cuh"

namespace fr3d {

// W_q = V0_q / sum_q' V0_q'^2 on the R grid (Algorithm 1 step 4 for several source parameters), stored
// as FP32 for the FP32 fused inverse; depends only on the geometry and the sources.  With
// V0_q = coef a_q, a_q = sum_l 1/|x - x_l|: W_q = a_q / (coef sum_q' a_q'^2).  The coordinate
// differences are taken in FP64 (no cancellation near a source), a_q and the sum of squares in FP32
// (relative error ~1e-7, the order of the table's own FP32 rounding), the scale 1/(coef sum) once per
// voxel in FP64 (any A0).
__device__ __forceinline__ float a_w(const Src64& s, int q, double x, double y, double z) {
  float acc = 0.f;
  const double* p = s.pts + 3 * q * s.L;
  for (int l = 0; l < s.L; ++l) {
    const float dx = (float)(x - __ldg(p + 3 * l)), dy = (float)(y - __ldg(p + 3 * l + 1)),
                dz = (float)(z - __ldg(p + 3 * l + 2));
    acc += rsqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
  }
  return acc;
}

__global__ void k_wtab(float* __restrict__ W, int Q, int Mp, int n, Src64 src, double x0, double y0, double h,
                       const double* __restrict__ zr) {
  const long plane = (long)n * n, total = (long)Mp * plane;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int j = (int)(idx / plane);
    const long pix = idx % plane;
    const double x = x0 + ((double)(pix % n) + 0.5) * h, y = y0 + ((double)(pix / n) + 0.5) * h;
    // every a_q once (the first kWtabKeep kept for the second loop, the rest evaluated again)
    constexpr int kWtabKeep = 16;
    float keep[kWtabKeep];
    float s = 0.f;
    for (int q = 0; q < Q; ++q) {
      const float a = a_w(src, q, x, y, zr[j]);
      if (q < kWtabKeep) keep[q] = a;
      s = fmaf(a, a, s);
    }
    const double scale = 1.0 / (src.coef * (double)s);
    for (int q = 0; q < Q; ++q)
      W[(long)q * total + idx] = (float)((double)(q < kWtabKeep ? keep[q] : a_w(src, q, x, y, zr[j])) * scale);
  }
}

namespace {

// ---------------- autotuner of the fused inverse's tile variant
// Mode 0: always variant 0; 1: on the first call for a shape (device, n, depths, Q, output) outside a
// stream capture, time every variant on the call's own arguments (one warm-up and three timed launches
// each; all variants produce the same bits) and keep the fastest for later calls; 2 + v: always
// variant v.  Calls inside a capture use the tuned choice if there is one, else variant 0.
std::atomic<int> g_tune_mode{1};
struct TuneKey {
  int dev, n, nj, Q, xi, once;   // once: only variants that write every output once (mapped host output)
  bool operator<(const TuneKey& o) const {
    return std::tie(dev, n, nj, Q, xi, once) < std::tie(o.dev, o.n, o.nj, o.Q, o.xi, o.once);
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tuned;

// variants 0-3: the fused cluster kernel's tiles; 4: the two-pass inverse (inv2p.cu), whose intermediate
// lives in the handle's inv2 buffer (grown outside stream captures only); 5: the persistent tile queue
// (inv_queue.cu: n = 256, xi output), through the same intermediate and the handle's queue counters
constexpr int kInvVariants = kFusedVariants + 2;

int ensure_inv2(Handle* H, int Q, int nj, cudaStream_t st, bool* ok) {
  const size_t need = inv2_scratch_bytes(H->n, Q, nj);
  *ok = H->inv2_cap >= need;
  if (*ok) return FR3D_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  FR3D_CUDA_TRY(cudaStreamIsCapturing(st, &cs));
  if (cs != cudaStreamCaptureStatusNone) return FR3D_OK;   // no allocation inside a capture
  FR3D_CUDA_TRY(cudaStreamSynchronize(st));
  if (H->inv2_buf) cudaFree(H->inv2_buf);
  H->inv2_buf = nullptr;
  H->inv2_cap = 0;
  FR3D_CUDA_TRY(cudaMalloc(&H->inv2_buf, need));
  H->inv2_cap = need;
  *ok = true;
  return FR3D_OK;
}

// the queue counters of variant 5 (zeroed once here; every launch leaves them zeroed)
int ensure_qctl(Handle* H, int nj, int Q, cudaStream_t st, bool* ok) {
  const size_t need = inv_queue_ctl_ints(nj, Q);
  *ok = H->qctl_n >= need;
  if (*ok) return FR3D_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  FR3D_CUDA_TRY(cudaStreamIsCapturing(st, &cs));
  if (cs != cudaStreamCaptureStatusNone) return FR3D_OK;
  FR3D_CUDA_TRY(cudaStreamSynchronize(st));
  if (H->qctl) cudaFree(H->qctl);
  H->qctl = nullptr;
  H->qctl_n = 0;
  FR3D_CUDA_TRY(cudaMalloc(&H->qctl, need * sizeof(int)));
  FR3D_CUDA_TRY(cudaMemset(H->qctl, 0, need * sizeof(int)));
  H->qctl_n = need;
  *ok = true;
  return FR3D_OK;
}

int launch_variant(Handle* H, int v, int n, bool xi, const FusedArgs& a, int nj, cudaStream_t st) {
  switch (v) {
    case 0: return fused_launch<0>(n, xi, a, nj, st);
    case 1: return fused_launch<1>(n, xi, a, nj, st);
    case 2: return fused_launch<2>(n, xi, a, nj, st);
    case 3: return fused_launch<3>(n, xi, a, nj, st);
    case 4: {
      bool ok = false;
      FR3D_TRY(ensure_inv2(H, a.Q, nj, st, &ok));
      if (!ok) return fused_launch<3>(n, xi, a, nj, st);   // inside a capture without the buffer
      return inv2_launch(n, xi, a, nj, H->inv2_buf, st);
    }
    case 5: {
      // other sizes and outputs, and a first call inside a capture: the register-accumulator tile
      if (!inv_queue_supported(n, xi) || a.Zs) return fused_launch<3>(n, xi, a, nj, st);
      bool ok = false, okc = false;
      FR3D_TRY(ensure_inv2(H, a.Q, nj, st, &ok));
      FR3D_TRY(ensure_qctl(H, nj, a.Q, st, &okc));
      if (!ok || !okc) return fused_launch<3>(n, xi, a, nj, st);
      return inv_queue_launch(n, a, nj, H->inv2_buf, H->qctl, st);
    }
  }
  return FR3D_ERR_INVALID_ARG;
}

// once: the output lives in page-locked host memory that the kernel writes over the host link; the
// tuner then times only the variants that write every output once (a forced variant is still used).
int choose_variant(Handle* H, const FusedArgs& a, int nj, bool xi, bool once, cudaStream_t st, int* v_out) {
  const int mode = g_tune_mode.load();
  if (mode >= 2) {
    *v_out = std::min(mode - 2, kInvVariants - 1);
    return FR3D_OK;
  }
  *v_out = 0;
  if (mode == 0) return FR3D_OK;
  once = once && xi;
  const TuneKey key{H->dev, H->n, nj, a.Q, xi ? 1 : 0, once ? 1 : 0};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) {
      *v_out = it->second;
      return FR3D_OK;
    }
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  FR3D_CUDA_TRY(cudaStreamIsCapturing(st, &cs));
  if (cs != cudaStreamCaptureStatusNone) return FR3D_OK;
  cudaEvent_t e0, e1;
  FR3D_CUDA_TRY(cudaEventCreate(&e0));
  FR3D_CUDA_TRY(cudaEventCreate(&e1));
  int best = 0, st_ok = FR3D_OK;
  float best_ms = 3.4e38f;
  for (int v = 0; v < kInvVariants && st_ok == FR3D_OK; ++v) {
    if (once && v < kFusedVariants && fused_rereads_output(v)) {
      H->fused_tune_ms[v] = 0.f;
      continue;
    }
    st_ok = launch_variant(H, v, H->n, xi, a, nj, st);
    if (st_ok == FR3D_OK && cudaEventRecord(e0, st) != cudaSuccess) st_ok = FR3D_ERR_CUDA;
    for (int rep = 0; rep < 3 && st_ok == FR3D_OK; ++rep) st_ok = launch_variant(H, v, H->n, xi, a, nj, st);
    if (st_ok == FR3D_OK && cudaEventRecord(e1, st) != cudaSuccess) st_ok = FR3D_ERR_CUDA;
    if (st_ok == FR3D_OK && cudaEventSynchronize(e1) != cudaSuccess) st_ok = FR3D_ERR_CUDA;
    float ms = 0.f;
    if (st_ok == FR3D_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) st_ok = FR3D_ERR_CUDA;
    if (st_ok != FR3D_OK) break;
    ms /= 3.f;
    H->fused_tune_ms[v] = ms;
    if (ms < best_ms) {
      best_ms = ms;
      best = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  FR3D_TRY(st_ok);
  H->fused_tuned = 1;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tuned[key] = best;
  *v_out = best;
  return FR3D_OK;
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
                  float* out, int Q, int j0, int nj, int output, cudaStream_t st, bool out_host_mapped, int* info) {
  FusedArgs a;
  a.Uh = Uh;
  a.A = H->A32;
  a.Dd = Dd;
  a.aidx = aidx;
  a.na = Dd == H->Ddfix32 ? 1 : std::max(1, (int)H->alpha_key.size());
  a.bbin = H->bbin;
  a.nb = nb;
  a.W = W;
  a.out = out;
  a.tw_n = H->tw32 + twiddle_offset(H, H->n);
  a.Q = Q;
  a.j0 = j0;
  a.Mp = H->Mp;
  a.Zs = nullptr;
  a.info = info;
  const bool xi = output == FR3D_OUT_XI;
  int v = 0;
  FR3D_TRY(choose_variant(const_cast<Handle*>(H), a, nj, xi, out_host_mapped, st, &v));
  const_cast<Handle*>(H)->fused_var = v;
  return launch_variant(const_cast<Handle*>(H), v, H->n, xi, a, nj, st);
}

namespace {
int launch_batched_variant(int v, int n, bool xi, const FusedArgs* inst, const int2* map, int ncl, cudaStream_t st) {
  switch (v) {
    case 0: return fused_launch_batched<0>(n, xi, inst, map, ncl, st);
    case 1: return fused_launch_batched<1>(n, xi, inst, map, ncl, st);
    case 2: return fused_launch_batched<2>(n, xi, inst, map, ncl, st);
    case 3: return fused_launch_batched<3>(n, xi, inst, map, ncl, st);
  }
  return FR3D_ERR_INVALID_ARG;
}
}  // namespace

int inv_fused_batched_f32(int n, const FusedArgs* inst, const int2* map, int nclusters, int output, int variant,
                          cudaStream_t st) {
  return launch_batched_variant(std::min(std::max(variant, 0), kFusedVariants - 1), n, output == FR3D_OUT_XI, inst,
                                map, nclusters, st);
}

int fused_tune_mode_get() { return g_tune_mode.load(); }

// Time every variant of a batched group's fused launch (1 warm-up + 2 timed launches each) and return
// the fastest in *best.  Synchronises the stream.
int fused_tune_batched(int n, const FusedArgs* inst, const int2* map, int nclusters, int output, cudaStream_t st,
                       int* best, float* best_ms) {
  const bool xi = output == FR3D_OUT_XI;
  cudaEvent_t e0, e1;
  FR3D_CUDA_TRY(cudaEventCreate(&e0));
  FR3D_CUDA_TRY(cudaEventCreate(&e1));
  int rc = FR3D_OK, bv = 0;
  float bms = 3.4e38f;
  for (int v = 0; v < kFusedVariants && rc == FR3D_OK; ++v) {
    rc = launch_batched_variant(v, n, xi, inst, map, nclusters, st);
    if (rc == FR3D_OK && cudaEventRecord(e0, st) != cudaSuccess) rc = FR3D_ERR_CUDA;
    for (int k = 0; k < 2 && rc == FR3D_OK; ++k) rc = launch_batched_variant(v, n, xi, inst, map, nclusters, st);
    if (rc == FR3D_OK && cudaEventRecord(e1, st) != cudaSuccess) rc = FR3D_ERR_CUDA;
    if (rc == FR3D_OK && cudaEventSynchronize(e1) != cudaSuccess) rc = FR3D_ERR_CUDA;
    float ms = 0.f;
    if (rc == FR3D_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = FR3D_ERR_CUDA;
    if (rc == FR3D_OK && ms < bms) {
      bms = ms;
      bv = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  FR3D_TRY(rc);
  *best = bv;
  if (best_ms) *best_ms = bms / 2.f;   // per launch
  return FR3D_OK;
}

int inv_fused_presolved_f32(const Handle* H, const float2* Zs, const float* W, float* out, int Q, int output,
                            cudaStream_t st) {
  FusedArgs a;
  a.Uh = nullptr;
  a.A = nullptr;
  a.Dd = nullptr;
  a.aidx = H->zero_idx;
  a.na = 1;
  a.bbin = nullptr;
  a.nb = 1;
  a.W = W;
  a.out = out;
  a.tw_n = H->tw32 + twiddle_offset(H, H->n);
  a.Q = Q;
  a.j0 = 0;
  a.Mp = H->Mp;
  a.Zs = Zs;
  const_cast<Handle*>(H)->fused_var = 1;
  return fused_launch_pre(H->n, output == FR3D_OUT_XI, a, H->Mp, st);
}

void fused_args_f32(const Handle* H, const float2* Uh, const float* Dd, const int* aidx, int nb, const float* W,
                    float* out, int Q, FusedArgs* a) {
  a->Uh = Uh;
  a->A = H->A32;
  a->Dd = Dd;
  a->aidx = aidx;
  a->na = Dd == H->Ddfix32 ? 1 : std::max(1, (int)H->alpha_key.size());
  a->bbin = H->bbin;
  a->nb = nb;
  a->W = W;
  a->out = out;
  a->tw_n = H->tw32 + twiddle_offset(H, H->n);
  a->Q = Q;
  a->j0 = 0;
  a->Mp = H->Mp;
  a->Zs = nullptr;
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

extern "C" int fr3d_autotune_mode(int mode) {
  if (mode < -1 || mode > 1 + fr3d::kInvVariants) return FR3D_ERR_INVALID_ARG;
  if (mode == -1) return fr3d::g_tune_mode.load();
  return fr3d::g_tune_mode.exchange(mode);
}

extern "C" int fr3d_autotune_query(fr3d_handle* h, int* variant, float* ms, int cap) {
  if (!h) return FR3D_ERR_INVALID_ARG;
  if (h->padded) return fr3d_autotune_query(h->padded, variant, ms, cap);
  const fr3d::Handle* H = &h->h;
  if (variant) *variant = H->fused_var;
  if (ms)
    for (int v = 0; v < std::min(cap, fr3d::kInvVariants); ++v) ms[v] = H->fused_tuned ? H->fused_tune_ms[v] : 0.f;
  return fr3d::kInvVariants;
}
