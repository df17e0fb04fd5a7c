// Shared host/device declarations of the fr3d library (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <vector>

#include "../../include/fr3d.h"

namespace fr3d {

#define FR3D_CUDA_TRY(expr)                              \
  do {                                                   \
    cudaError_t e_ = (expr);                             \
    if (e_ != cudaSuccess) {                             \
      if (e_ == cudaErrorMemoryAllocation) return FR3D_ERR_OOM; \
      return FR3D_ERR_CUDA;                              \
    }                                                    \
  } while (0)

#define FR3D_TRY(expr)        \
  do {                        \
    int s_ = (expr);          \
    if (s_ < 0) return s_;    \
  } while (0)

// Transform lengths with a radix plan (fft_engine.cuh); the 2D grid n must have n and n/2 in it.
static const int kLengths[] = {8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256, 384, 512};
static const int kNumLengths = 13;

// Frequency classes: (kx, ky) of the half spectrum (kx in [0, n/2], ky in [0, n)) folded by the
// symmetries of the sampled kernel (k -> -k per axis and kx <-> ky on a square grid):
// u = kx, v = min(ky, n - ky), class (p, q) = (max, min), index p (p + 1) / 2 + q.
__host__ __device__ __forceinline__ int class_of(int kx, int ky, int n) {
  int v = ky <= n - ky ? ky : n - ky;
  int p = kx > v ? kx : v, q = kx > v ? v : kx;
  return p * (p + 1) / 2 + q;
}
__host__ __device__ __forceinline__ int num_classes(int n) { return (n / 2 + 1) * (n / 2 + 2) / 2; }

struct Handle {
  int dev = 0;
  int n = 0, M = 0, Mp = 0, C = 0;
  int kind = FR3D_K_DZ_INV_R;  // kernel of the equation (fr3d_geometry.kernel_kind)
  double x0 = 0, y0 = 0, h = 0;
  std::vector<double> zr, nu, zy;
  // kernel tables (owned)
  double* A64 = nullptr;      // [C][M][Mp]   nu_j K~(class c; z_i - z'_j)
  double* nrm = nullptr;      // [C]          ||A^(c)||_F^2
  double* s2 = nullptr;       // [1]          max_c nrm[c]
  float* A32 = nullptr;       // [M][Mp][n/2+1][n]   dense per half-spectrum bin
  double* A64d = nullptr;     // same, FP64 (built on the first FP64 call)
  double* zr64 = nullptr;     // [Mp] depths of R on the device
  float* zr32 = nullptr;
  double s2_host = -1.0;
  // twiddles exp(-2 pi i t / L) for every supported L, FP32 and FP64
  float2* tw32 = nullptr;
  double2* tw64 = nullptr;
  int tw_off[kNumLengths] = {0};
  // alpha tables, keyed by the candidate list
  std::vector<double> alpha_key;
  int alpha_ra = -1;          // regularising algorithm of the alpha tables (FR3D_RA_*)
  double* Ft = nullptr;       // [C][n_alpha]  ((alpha s^2) / (nrm + alpha s^2))^2
  float* D32 = nullptr;       // [n_alpha][C]  1 / (n^2 (nrm + alpha s^2))
  float* Dd32 = nullptr;      // [n_alpha][n/2+1][n]  the same per half-spectrum bin
  double* D64 = nullptr;      // [n_alpha][C]
  int alpha_cap = 0;
  // fixed-alpha table
  double fixed_key = -1.0;
  int fixed_ra = -1;
  float* Dfix32 = nullptr;    // [C]
  float* Ddfix32 = nullptr;   // [n/2+1][n]
  double* Dfix64 = nullptr;   // [C]
  // sources, keyed by content
  std::vector<double> src_key;
  float4* pts32 = nullptr;    // [Q*L] (x, y, z, 0)
  float* wtab = nullptr;      // [Q][M'][n][n] V0_q / sum_q' V0_q'^2 for src_key (built on demand)
  std::vector<double> wtab_key;
  size_t wtab_cap = 0;
  double* pts64 = nullptr;    // [Q*L*3]
  int src_cap = 0;
  // small device words
  unsigned* counter = nullptr;   // last-block counter (self-resetting)
  int* idx_scratch = nullptr;    // chosen alpha index when the caller passes none
  int* zero_idx = nullptr;       // constant 0
  int* info_scratch = nullptr;
  double* partials = nullptr;    // [blocks][bands][n_alpha]
  int partial_cap = 0;
  unsigned char* cband = nullptr; // [C] radial band of every class for cband_nb bands
  int cband_nb = 0;
  std::vector<double> band_count; // grid frequencies per band (sum of the classes' member weights)
  unsigned char* bbin = nullptr;  // [n/2+1][n] radial band of every half-spectrum bin for cband_nb bands
  // several observation depths (M > 1): per class the Gram eigenvalues, eigenvectors U and W = U^T A (multi.cu)
  double* mlam = nullptr;      // [C][M]
  float* mUt = nullptr;        // [C][k][i]: the eigenvectors (component i along observation depth k)
  float* mW = nullptr;         // [C][M][M']
  int m_sweeps = 0;            // Jacobi sweeps the slowest class needed
  // tensor-core tables (tc_contract.cu), per kind (0 projection U^T, 1 solve W^T, 2 forward A): BF16
  // class blobs in the MMA operand's shared-memory image, and the BF16 remainders (split mode)
  uint16_t* tc_hi[3] = {nullptr, nullptr, nullptr};
  uint16_t* tc_lo[3] = {nullptr, nullptr, nullptr};
  int tc_blob[3] = {0, 0, 0};
  int tc_kc[3] = {0, 0, 0};
  // right-hand side of Eq. (7): the handle of the box Pi's geometry (same grid, Pi's depths as the
  // unknown depths) and its buffers (density on Pi, integral term on Y)
  fr3d_handle* pi = nullptr;
  int pi_n = 0;
  double pi_half = 0.0;
  void* rhs_buf = nullptr;
  size_t rhs_bytes = 0;
  // workspace
  void* ws = nullptr;
  size_t ws_bytes = 0;
  int last_launches = 0;
  // fused-inverse tile variant of the last call, and the autotuner's timings (ms) if it ran
  int fused_var = 0;
  int fused_tuned = 0;
  float fused_tune_ms[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  // intermediate of the two-pass and the tile-queue inverses (inv2p.cu, inv_queue.cu): Q M' n n/2 complex,
  // grown outside captures; the tile queue's counters (zeroed at allocation, left zeroed by every launch)
  float2* inv2_buf = nullptr;
  size_t inv2_cap = 0;
  int* qctl = nullptr;
  size_t qctl_n = 0;
  // stage profiling: events recorded between consecutive launches of one call
  static constexpr int kMaxEv = 96;
  bool prof_on = false;
  cudaEvent_t ev[kMaxEv] = {};
  int ev_kind[kMaxEv] = {0};
  int n_ev = 0;
  cudaStream_t create_stream = nullptr;
  bool synced = false;
};

// Programmatic dependent launch.  A kernel launched with programmatic stream serialisation may start
// while the kernel before it in the stream is still running: before pdl_wait() it may read only data
// that no kernel of the current call writes; pdl_wait() returns once that kernel has completed and its
// writes are visible (at once for an ordinary launch).  pdl_release() lets this kernel's programmatic
// successor start; a successor starts only after every block of this kernel has released it (or
// exited), so all of this kernel's blocks are resident by then.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

// launch-count bookkeeping (host)
struct Launches {
  int n = 0;
  void add(int k = 1) { n += k; }
};

int ensure_ws(Handle* H, size_t bytes);

// Opt a kernel in to `bytes` of dynamic shared memory (beyond the 48 KB default that static and
// dynamic shared memory share) once per (kernel, device); later calls are a lookup, so launches
// inside a stream capture make no attribute call.  Returns an error if bytes exceed the device limit.
int smem_optin(const void* kernel, size_t bytes);
// CTAs of `kernel` that fit on one SM by registers, threads and the device's per-SM shared memory
int resident_ctas(const void* kernel, int threads, size_t dyn_smem);

// stage kinds reported by fr3d_profile_read
enum StageKind { kStRowR2C = 0, kStColFwd = 1, kStAlpha = 2, kStColSolve = 3, kStRowC2R = 4, kStTable = 5,
                 kStContract = 6, kStColInv = 7, kStOther = 8, kStFused = 9 };
// Inside a stream capture an event is recorded with cudaEventRecordExternal so that it becomes a
// graph node and a replayed graph records the stage events too; outside a capture it is a plain
// record.  A failed record stops the tracing of this call (n_ev = 0) and clears the error.
inline bool prof_record(cudaEvent_t e, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(st, &cs);
  const cudaError_t r = cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(e, st, cudaEventRecordExternal)
                                                            : cudaEventRecord(e, st);
  if (r != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return true;
}
inline void prof_begin(Handle* H, cudaStream_t st) {
  H->n_ev = 0;
  if (!H->prof_on) return;
  if (prof_record(H->ev[0], st)) H->n_ev = 1;
}
inline void prof_mark(Handle* H, int kind, cudaStream_t st) {
  if (!H->prof_on || H->n_ev <= 0 || H->n_ev >= Handle::kMaxEv) return;
  H->ev_kind[H->n_ev - 1] = kind;
  if (prof_record(H->ev[H->n_ev], st)) ++H->n_ev;
  else H->n_ev = 0;
}
int twiddle_offset(const Handle* H, int L);

}  // namespace fr3d

struct fr3d_handle {
  fr3d::Handle h;
  // pad = 2: the handle of the 2n x 2n box (pad.cu); h then carries the n x n geometry's sizes and the
  // workspace of the embedded inputs and results
  fr3d_handle* padded = nullptr;
};
