// Batched inversion of many independent instances of uneven size (grid n, depths M', sources Q):
// a batch plan groups the instances by n and runs Algorithm 1 with three launches per group (data
// row pass, data column pass, inverse), each covering all instances of the group through device
// tables of per-plane, per-instance and per-cluster descriptors, and one alpha-rule launch over the
// instances of every group (the rule's kernel takes the grid size per instance).  The plan
// is built once (tables, workspaces, descriptors); running it only launches kernels, so it can be
// captured in a CUDA graph.
#include <string.h>

#include <algorithm>
#include <map>
#include <new>
#include <vector>

#include "fused.cuh"
#include "ops_impl.cuh"

namespace fr3d {

struct AlphaInst {
  const float2* Uh;
  const double* Ft;
  const unsigned char* cband;
  double* partials;
  unsigned* counter;
  unsigned* tickets;
  int* aidx;
  double* res;
  int* info;
  BandThr thr2;
  double inv_n2;   // 1 / n^2
  long ps;         // plane stride of the data spectra, (n/2 + 1) n
  int n, Cn;       // grid size and its frequency classes
  int nplanes, na, nb, bstart, nblk;
};

// The alpha rule of every instance of a plan, all grid sizes, in one launch.  Each instance owns
// alpha_blocks(Cn) consecutive blocks of the grid (the table is ordered by first block) and its own
// partial sums and tickets.  A plan's grid is many waves of blocks, each a chain of dependent
// steps, so four blocks per SM (64 registers, a 64-byte spill) run faster than two at 98 registers.
__global__ void __launch_bounds__(256, 4) k_alpha_batched(const AlphaInst* __restrict__ inst, int ninst) {
  int lo = 0, hi = ninst - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (inst[mid].bstart <= (int)blockIdx.x) lo = mid;
    else hi = mid - 1;
  }
  const AlphaInst a = inst[lo];
  alpha_choose_body<float2>(a.Uh, a.ps, a.nplanes, a.n, a.Cn, a.Ft, a.na, a.thr2, a.cband, a.nb, a.inv_n2, a.partials,
                            a.counter, a.aidx, a.res, a.info, a.tickets, (int)blockIdx.x - a.bstart, a.nblk);
}

int inv_fused_batched_f32(int n, const FusedArgs* inst, const int2* map, int nclusters, int output, int variant,
                          cudaStream_t st);
int fused_tune_mode_get();
int fused_tune_batched(int n, const FusedArgs* inst, const int2* map, int nclusters, int output, cudaStream_t st,
                       int* best, float* best_ms);
void fused_args_f32(const Handle* H, const float2* Uh, const float* Dd, const int* aidx, int nb, const float* W,
                    float* out, int Q, FusedArgs* a);
int prepare_instance_f32(Handle* H, int Q, const fr3d_invert_opts* o, float2** Uh, const float** Dd, const int** aidx,
                         cudaStream_t st);

namespace {

struct Group {
  int n = 0;
  const Handle* H0 = nullptr;
  int nplanes = 0, nclusters = 0;
  int var = -1;   // inverse variant (-1: not chosen yet; 5: the tile queue)
  size_t off_planes = 0, off_fused = 0, off_map = 0;
  // the tile queue over the group's instances (n = 256, xi output, plan form): its descriptor table in
  // the plan's tables, its counters and intermediates in the plan's queue buffer
  int qn = 0, qtotal = 0, qncnt = 0;
  size_t off_queue = 0;
  int* qctl = nullptr;
  int* qcnt = nullptr;
};

// Bytes of the queue buffer for the instances of a group (4 launch counters, the depth counters, the
// intermediates), laid out by queue_layout.
bool queue_group(int n, int output) { return output == FR3D_OUT_XI && inv_queue_supported(n, true); }

// the data transform of a group: row and column passes over all its instances' planes
template <int N>
int run_group_pre_n(const Group& g, const unsigned char* dev, cudaStream_t st) {
  const PlanePtr* planes = reinterpret_cast<const PlanePtr*>(dev + g.off_planes);
  constexpr int TY = SmallTile<N>::row, TC = SmallTile<N>::col;
  FR3D_TRY((row_r2c_t<float, N, TY, TablePlanes>(g.H0, TablePlanes{planes}, g.nplanes, st)));
  FR3D_TRY((col_t<float, N, false, ColTable, TC>(g.H0, ColTable{planes}, g.nplanes, st)));
  return FR3D_OK;
}

int run_group_pre(const Group& g, const unsigned char* dev, cudaStream_t st) {
  switch (g.n) {
#define X(N) \
  case N: return run_group_pre_n<N>(g, dev, st);
    X(16) X(24) X(32) X(48) X(64) X(96) X(128) X(192) X(256) X(384)
#undef X
  }
  return FR3D_ERR_UNSUPPORTED_SIZE;
}

const FusedArgs* fused_of(const Group& g, const unsigned char* dev) {
  return reinterpret_cast<const FusedArgs*>(dev + g.off_fused);
}
const int2* map_of(const Group& g, const unsigned char* dev) { return reinterpret_cast<const int2*>(dev + g.off_map); }

size_t al(size_t v) { return (v + 255) & ~(size_t)255; }

// The alpha rule over all groups: one table of every discrepancy-rule instance, in group order.
struct AlphaPlan {
  size_t off = 0;   // the table's offset in the plan's device tables
  int ninst = 0, nblk = 0, max_na = 0;
};

int run_alpha(const AlphaPlan& a, const unsigned char* dev, cudaStream_t st) {
  if (a.ninst == 0) return FR3D_OK;
  const size_t sm = sizeof(double) * kAlphaCPB * a.max_na;
  FR3D_TRY(smem_optin(reinterpret_cast<const void*>(k_alpha_batched), sm));
  k_alpha_batched<<<a.nblk, 256, sm, st>>>(reinterpret_cast<const AlphaInst*>(dev + a.off), a.ninst);
  FR3D_CUDA_TRY(cudaGetLastError());
  return FR3D_OK;
}

}  // namespace

struct Batch {
  std::vector<Group> groups;
  AlphaPlan alpha;
  unsigned char* dev = nullptr;
  unsigned char* qbuf = nullptr;   // the tile queue's counters and intermediates (zeroed once)
  int output = FR3D_OUT_XI;
  int launches = 0;
};

}  // namespace fr3d

struct fr3d_batch {
  fr3d::Batch b;
};

namespace fr3d {
namespace {

size_t spectra_bytes(const fr3d_instance& I) {
  const int n = I.handle->h.n;
  return al(sizeof(float2) * (size_t)I.Q * (n / 2 + 1) * n);
}

// Validate the instances, prepare every handle's tables (cold; allocates) and group them by grid size.
// With ext = true the data spectra are laid out from offset 0 of a caller workspace (uh[i] = offsets).
int batch_prepare(const fr3d_instance* inst, int n, bool ext, std::vector<float2*>& uh, std::vector<const float*>& dd,
                  std::vector<const int*>& ai, std::map<int, std::vector<int>>& by_n, size_t* spectra_total,
                  cudaStream_t st) {
  const int output = inst[0].opts ? inst[0].opts->output : FR3D_OUT_XI;
  size_t off = 0;
  for (int i = 0; i < n; ++i) {
    const fr3d_instance& I = inst[i];
    if (!I.handle || !I.U || !I.out || !I.opts || I.Q < 1) return FR3D_ERR_INVALID_ARG;
    if (I.handle->padded) return FR3D_ERR_UNSUPPORTED_SIZE;   // periodic box only
    for (int k = 0; k < i; ++k)
      if (inst[k].handle == I.handle) return FR3D_ERR_INVALID_ARG;   // one set of tables and scratch per handle
    if (I.opts->output != output || I.opts->precision != FR3D_PREC_FP32) return FR3D_ERR_INVALID_ARG;
    Handle* H = &I.handle->h;
    if (H->M != 1 || !fused_supported(H->n)) return FR3D_ERR_UNSUPPORTED_SIZE;
    FR3D_TRY(prepare_instance_f32(H, I.Q, I.opts, ext ? nullptr : &uh[i], &dd[i], &ai[i], st));
    if (ext) {
      uh[i] = reinterpret_cast<float2*>(off);
      off += spectra_bytes(I);
    }
    by_n[H->n].push_back(i);
  }
  *spectra_total = off;
  return FR3D_OK;
}

}  // namespace
}  // namespace fr3d

namespace fr3d {
namespace {

// Descriptor tables of the groups (host image; device offsets relative to the table's start).
// qbuf: the plan's queue buffer (device), or null (no tile queue: the one-shot workspace form).
void build_descriptors(const fr3d_instance* inst, const std::map<int, std::vector<int>>& by_n,
                       const std::vector<float2*>& uh, const std::vector<const float*>& dd,
                       const std::vector<const int*>& ai, std::vector<unsigned char>& host, std::vector<Group>& groups,
                       AlphaPlan& ap, unsigned char* qbuf = nullptr) {
  std::vector<AlphaInst> alph;
  auto put = [&](const void* p, size_t bytes) {
    const size_t off = al(host.size());
    host.resize(off + bytes);
    memcpy(host.data() + off, p, bytes);
    return off;
  };
  for (auto& kv : by_n) {
    Group g;
    g.n = kv.first;
    g.H0 = &inst[kv.second[0]].handle->h;
    std::vector<PlanePtr> planes;
    std::vector<FusedArgs> fa;
    std::vector<int2> map;
    const long ps = (long)(g.n / 2 + 1) * g.n;
    for (int idx : kv.second) {
      const fr3d_instance& I = inst[idx];
      Handle* H = &I.handle->h;
      for (int q = 0; q < I.Q; ++q) planes.push_back({I.U + (long)q * g.n * g.n, uh[idx] + q * ps});
      if (I.opts->alpha_mode == FR3D_ALPHA_DISCREPANCY) {
        AlphaInst a;
        a.Uh = uh[idx];
        a.Ft = H->Ft;
        a.nb = I.opts->n_bands > 1 ? I.opts->n_bands : 1;
        a.cband = H->cband;
        band_thresholds(H, I.opts, a.nb, a.thr2.t);
        a.partials = H->partials;
        a.counter = H->counter;
        a.tickets = alpha_tickets(H);
        a.aidx = const_cast<int*>(ai[idx]);
        a.res = I.opts->residuals;
        a.info = I.opts->info;
        a.inv_n2 = 1.0 / ((double)g.n * g.n);
        a.ps = ps;
        a.n = g.n;
        a.Cn = H->C;
        a.nplanes = I.Q;
        a.na = I.opts->n_alpha;
        a.bstart = ap.nblk;
        a.nblk = alpha_blocks(H->C);
        ap.nblk += a.nblk;
        ap.max_na = std::max(ap.max_na, a.na);
        alph.push_back(a);
      }
      FusedArgs f;
      fused_args_f32(H, uh[idx], dd[idx], ai[idx], I.opts->n_bands > 1 ? I.opts->n_bands : 1, H->wtab, I.out, I.Q, &f);
      for (int j = 0; j < H->Mp; ++j) map.push_back(make_int2((int)fa.size(), j));
      fa.push_back(f);
    }
    g.nplanes = (int)planes.size();
    g.nclusters = (int)map.size();
    if (qbuf && queue_group(g.n, inst[kv.second[0]].opts->output)) {
      // [4 launch counters][2 M' depth counters per instance][intermediates, 256-byte aligned]
      int ncnt = 0;
      for (int idx : kv.second) ncnt += 2 * inst[idx].handle->h.Mp;
      g.qctl = reinterpret_cast<int*>(qbuf);
      g.qcnt = g.qctl + 4;
      unsigned char* tp = qbuf + al(sizeof(int) * (4 + (size_t)ncnt));
      std::vector<unsigned char> qt(inv_queue_inst_bytes() * kv.second.size());
      int tick = 0, c = 0, k = 0;
      for (int idx : kv.second) {
        const fr3d_instance& I = inst[idx];
        const int mp = I.handle->h.Mp;
        tick += inv_queue_make_inst(qt.data() + k * inv_queue_inst_bytes(), fa[k], reinterpret_cast<float2*>(tp),
                                    g.qcnt + c, mp, tick);
        tp += al(inv2_scratch_bytes(g.n, I.Q, mp));
        c += 2 * mp;
        ++k;
      }
      g.qn = k;
      g.qtotal = tick;
      g.qncnt = ncnt;
      g.off_queue = put(qt.data(), qt.size());
    }
    g.off_planes = put(planes.data(), planes.size() * sizeof(PlanePtr));
    g.off_fused = put(fa.data(), fa.size() * sizeof(FusedArgs));
    g.off_map = put(map.data(), map.size() * sizeof(int2));
    groups.push_back(g);
  }
  ap.ninst = (int)alph.size();
  ap.off = alph.empty() ? 0 : put(alph.data(), alph.size() * sizeof(AlphaInst));
}

// bytes of the plan's queue buffer (the tile queue of its n = 256 group, xi output), 0 if none
size_t queue_bytes(const fr3d_instance* inst, const std::map<int, std::vector<int>>& by_n) {
  size_t b = 0;
  for (auto& kv : by_n) {
    if (!queue_group(kv.first, inst[kv.second[0]].opts->output)) continue;
    size_t ncnt = 0;
    for (int idx : kv.second) ncnt += 2 * (size_t)inst[idx].handle->h.Mp;
    b += al(sizeof(int) * (4 + ncnt));
    for (int idx : kv.second) b += al(inv2_scratch_bytes(kv.first, inst[idx].Q, inst[idx].handle->h.Mp));
  }
  return b;
}

// the inverse of a group: the tile queue (variant 5, where the plan has one) or a fused tile variant
int run_inverse(const Group& g, const unsigned char* dev, int output, int v, cudaStream_t st) {
  if (v == 5 && g.qn > 0)
    return inv_queue_launch_table(dev + g.off_queue, g.qn, g.qctl, g.qcnt, g.qncnt, g.qtotal, st);
  return inv_fused_batched_f32(g.n, fused_of(g, dev), map_of(g, dev), g.nclusters, output, std::min(v, 3), st);
}

// per group: row pass, column pass, inverse; one alpha launch over all groups
int batch_launches(const std::vector<Group>& groups, const AlphaPlan& ap) {
  return 3 * (int)groups.size() + (ap.ninst > 0 ? 1 : 0);
}

}  // namespace
}  // namespace fr3d

extern "C" int fr3d_batch_create(const fr3d_instance* inst, int n, fr3d_batch** out, void* stream) {
  using namespace fr3d;
  if (!inst || n < 1 || !out) return FR3D_ERR_INVALID_ARG;
  *out = nullptr;
  cudaStream_t st = (cudaStream_t)stream;
  std::map<int, std::vector<int>> by_n;
  std::vector<float2*> uh(n);
  std::vector<const float*> dd(n);
  std::vector<const int*> ai(n);
  size_t spectra = 0;
  FR3D_TRY(batch_prepare(inst, n, false, uh, dd, ai, by_n, &spectra, st));
  Batch b;
  b.output = inst[0].opts->output;
  const size_t qb = queue_bytes(inst, by_n);
  if (qb > 0) {
    FR3D_CUDA_TRY(cudaMalloc(&b.qbuf, qb));
    cudaError_t e = cudaMemsetAsync(b.qbuf, 0, qb, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      cudaFree(b.qbuf);
      return FR3D_ERR_CUDA;
    }
  }
  std::vector<unsigned char> host;
  build_descriptors(inst, by_n, uh, dd, ai, host, b.groups, b.alpha, b.qbuf);
  if (cudaMalloc(&b.dev, al(host.size())) != cudaSuccess) {
    cudaFree(b.qbuf);
    return FR3D_ERR_OOM;
  }
  {
    cudaError_t e = cudaMemcpyAsync(b.dev, host.data(), host.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      cudaFree(b.dev);
      cudaFree(b.qbuf);
      return FR3D_ERR_CUDA;
    }
  }
  b.launches = batch_launches(b.groups, b.alpha);
  fr3d_batch* h = new (std::nothrow) fr3d_batch();
  if (!h) {
    cudaFree(b.dev);
    cudaFree(b.qbuf);
    return FR3D_ERR_OOM;
  }
  h->b = std::move(b);
  *out = h;
  return FR3D_OK;
}

extern "C" int fr3d_batch_run(fr3d_batch* h, void* stream) {
  using namespace fr3d;
  if (!h) return FR3D_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int mode = fused_tune_mode_get();
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  FR3D_CUDA_TRY(cudaStreamIsCapturing(st, &cs));
  for (auto& g : h->b.groups) FR3D_TRY(run_group_pre(g, h->b.dev, st));
  FR3D_TRY(run_alpha(h->b.alpha, h->b.dev, st));
  for (auto& g : h->b.groups) {
    int v = mode >= 2 ? mode - 2 : 0;
    if (mode == 1) {
      if (g.var < 0 && cs == cudaStreamCaptureStatusNone) {
        // the first run outside a capture times the variants on this group (their launches leave
        // the group's outputs complete: every variant writes the same bits), the tile queue too
        float fms = 0.f;
        FR3D_TRY(fused_tune_batched(g.n, fused_of(g, h->b.dev), map_of(g, h->b.dev), g.nclusters, h->b.output, st,
                                    &g.var, &fms));
        if (g.qn > 0) {
          cudaEvent_t e0, e1;
          FR3D_CUDA_TRY(cudaEventCreate(&e0));
          FR3D_CUDA_TRY(cudaEventCreate(&e1));
          int rc = run_inverse(g, h->b.dev, h->b.output, 5, st);
          if (rc == FR3D_OK && cudaEventRecord(e0, st) != cudaSuccess) rc = FR3D_ERR_CUDA;
          for (int k = 0; k < 2 && rc == FR3D_OK; ++k) rc = run_inverse(g, h->b.dev, h->b.output, 5, st);
          if (rc == FR3D_OK && cudaEventRecord(e1, st) != cudaSuccess) rc = FR3D_ERR_CUDA;
          if (rc == FR3D_OK && cudaEventSynchronize(e1) != cudaSuccess) rc = FR3D_ERR_CUDA;
          float qms = 0.f;
          if (rc == FR3D_OK && cudaEventElapsedTime(&qms, e0, e1) != cudaSuccess) rc = FR3D_ERR_CUDA;
          cudaEventDestroy(e0);
          cudaEventDestroy(e1);
          FR3D_TRY(rc);
          if (qms / 2.f < fms) g.var = 5;
        }
        continue;
      }
      v = g.var < 0 ? 0 : g.var;
    }
    FR3D_TRY(run_inverse(g, h->b.dev, h->b.output, v, st));
  }
  return FR3D_OK;
}

extern "C" int fr3d_batch_launch_count(fr3d_batch* h) { return h ? h->b.launches : -1; }

extern "C" void fr3d_batch_destroy(fr3d_batch* h) {
  if (!h) return;
  cudaDeviceSynchronize();
  cudaFree(h->b.dev);
  cudaFree(h->b.qbuf);
  delete h;
}

// One-shot batched inversion in caller-provided device memory.  The query prepares every handle's
// tables (allocating them, synchronously) and returns the bytes the run needs: the data spectra of all
// instances and the descriptor tables.  The run allocates nothing when the handles' tables are already
// prepared for these options; it copies the descriptors into the workspace and launches the groups.
extern "C" int fr3d_invert_batched_workspace(const fr3d_instance* inst, int n, size_t* bytes, void* stream) {
  using namespace fr3d;
  if (!inst || n < 1 || !bytes) return FR3D_ERR_INVALID_ARG;
  std::map<int, std::vector<int>> by_n;
  std::vector<float2*> uh(n);
  std::vector<const float*> dd(n);
  std::vector<const int*> ai(n);
  size_t spectra = 0;
  FR3D_TRY(batch_prepare(inst, n, true, uh, dd, ai, by_n, &spectra, (cudaStream_t)stream));
  std::vector<unsigned char> host;
  std::vector<Group> groups;
  AlphaPlan ap;
  build_descriptors(inst, by_n, uh, dd, ai, host, groups, ap);
  *bytes = al(spectra) + al(host.size());
  return FR3D_OK;
}

extern "C" int fr3d_invert_batched(const fr3d_instance* inst, int n, void* workspace, size_t ws_bytes, void* stream) {
  using namespace fr3d;
  if (!inst || n < 1 || !workspace || reinterpret_cast<uintptr_t>(workspace) % 256) return FR3D_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  std::map<int, std::vector<int>> by_n;
  std::vector<float2*> uh(n);
  std::vector<const float*> dd(n);
  std::vector<const int*> ai(n);
  size_t spectra = 0;
  FR3D_TRY(batch_prepare(inst, n, true, uh, dd, ai, by_n, &spectra, st));
  unsigned char* base = static_cast<unsigned char*>(workspace);
  for (int i = 0; i < n; ++i) uh[i] = reinterpret_cast<float2*>(base + reinterpret_cast<size_t>(uh[i]));
  std::vector<unsigned char> host;
  std::vector<Group> groups;
  AlphaPlan ap;
  build_descriptors(inst, by_n, uh, dd, ai, host, groups, ap);
  const size_t need = al(spectra) + al(host.size());
  if (ws_bytes < need) return FR3D_ERR_INVALID_ARG;
  unsigned char* tables = base + al(spectra);
  // pageable source: the copy has staged the descriptors when the call returns
  FR3D_CUDA_TRY(cudaMemcpyAsync(tables, host.data(), host.size(), cudaMemcpyHostToDevice, st));
  const int mode = fused_tune_mode_get();
  const int v = mode >= 2 ? mode - 2 : 3;   // the forced tile, else the register-accumulator tile
  for (auto& g : groups) FR3D_TRY(run_group_pre(g, tables, st));
  FR3D_TRY(run_alpha(ap, tables, st));
  for (auto& g : groups)
    FR3D_TRY(inv_fused_batched_f32(g.n, fused_of(g, tables), map_of(g, tables), g.nclusters, inst[0].opts->output, v,
                                   st));
  return FR3D_OK;
}
