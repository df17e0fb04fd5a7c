// Steps 2-4 of Algorithm 1 at M = 1 (FP32) as one persistent launch over a queue of tiles: the sixth
// variant of the inverse that the autotuner weighs against the fused cluster kernel (fused.cuh) and the
// two-pass form (inv2p.cu).  n = 256.
//
// The work of a call is a list of tiles, taken in ticket order from one atomic counter:
//   column tile (j, t)  depth j, four pairs of packed columns (kx, n/2 - kx), which are each other's
//                       partners in the Hermitian split of the rows (the pair (0, n/4) is its own: column
//                       0 carries kx = 0 in its real part and kx = n/2 in its imaginary part, both
//                       Hermitian in ky, so one complex DFT gives both); for every source parameter q the
//                       solve U~_q w_j, the inverse DFT along ky, and the split
//                       Z'(kx, y) = (X[kx] + conj X[n/2-kx]) + i w^-kx (X[kx] - conj X[n/2-kx]) with the
//                       partner's value from the lane 16 apart, written to the intermediate
//                       T[j][q][y / 16][kx][y % 16];
//   row tile (j, b)     depth j, rows [16b, 16b + 16): for every q those rows of T, the n/2-point inverse
//                       row DFT and xi += W_q zeta_q in registers; xi written once.
// Ordering: the column tiles of depth j come `lag` depths before its row tiles in the ticket order.  A
// column tile counts itself on its depth's first counter once it has stored the first half of the q
// (a release), and on the second once it has stored all; a row tile requests the rows of the first half
// once all column tiles of its depth have counted on the first, and those of the second half once they
// have counted on the second (acquires, bounded).  Every waiting tile was ticketed after the tiles it
// waits for, which are running or finished and wait for nothing, so the queue cannot deadlock.  The
// intermediate of a depth is read about one tile duration after it is written, from L2; a row tile drops
// each line from L2 once it holds it in shared memory (no line is read twice, so none needs writing back
// to HBM), and the combination weights W, read once, are prefetched into L2 by bulk prefetches three q
// ahead and loaded into registers one q ahead with an evict-first policy.
// Staging: the inputs of every q (a column tile's 8 columns of U~_q, 16 KB, plus column n/2 in tile 0; a
// row tile's 16 rows of T, 16 KB) arrive by bulk copies two q ahead in double-buffered stages tracked by
// mbarriers.  Every wait (on a stage or a counter) is bounded: on expiry the kernel ORs
// FR3D_INFO_TIMEOUT into the caller's info word and lets every other wait end at once, so the launch
// always ends.
// The arithmetic of every output (the solve weights, the radix passes and their twiddles, the split, the
// order of the accumulation over q) is the fused kernel's, so all variants return the same bits.
#include <string.h>

#include <atomic>

#include "fused.cuh"
#include "ops.cuh"
#include "tc.cuh"

namespace fr3d {

namespace {

constexpr int kQThreads = 128;
constexpr int kQMinBlocks = 4;        // resident CTAs per SM the registers and shared memory are sized for
constexpr long kSpinLimit = 1L << 20;  // polls before a wait gives up (a counter poll sleeps at least 128 ns)

template <int N> struct QGeom {
  static constexpr int L = N / 2;
  static constexpr int CT = 8;                     // packed columns per column tile
  static constexpr int NCT = L / CT;               // column tiles per depth
  static constexpr int RB = 16;                    // rows per row tile
  static constexpr int NRT = N / RB;               // row tiles per depth
  static constexpr int SSC = PaddedLen<N, float2>::v;        // column stride (complex) of the column buffer
  static constexpr int SSR = PaddedLen<L, float2>::v + 1;    // row stride of the row buffer (odd)
  static constexpr int STG = CT * N;               // complex elements of one stage
  static constexpr int PTC = passtw_size<N>(), PTR = passtw_size<L>();
  static constexpr int BUF = CT * SSC > RB * SSR ? CT * SSC : RB * SSR;
  // per-tile tables: column tile = two stages of column n/2 + pass tables of length n; row tile = pass
  // tables of length n/2
  static constexpr int TABC = 2 * N + PTC, TABR = PTR;
  static constexpr int TAB = TABC > TABR ? TABC : TABR;
  static constexpr size_t head = 32;               // two mbarriers, the broadcast ticket
  static constexpr size_t smem = head + sizeof(float2) * (2 * (size_t)STG + BUF + TAB);
  static_assert(STG == RB * L, "a stage holds a column tile's columns or a row tile's rows");
  static_assert(CT * 16 == kQThreads, "one radix-16 butterfly per thread in the column passes");
  static_assert(Plan<L>::np == 2 && Plan<L>::radix(0) == 16, "the row DFT: a radix-16 first pass, then the last pass");
  static_assert(Plan<N>::np == 2 && Plan<N>::radix(0) == 16, "the column DFT: a radix-16 first pass, then the last pass");
};

// One instance of a launch (a call, or one instance of a batch).
struct QInst {
  FusedArgs f;
  float2* T;    // [nj][Q][n/16][n/2][16] intermediate
  int* cnt;     // [2 nj]: column tiles of depth j done with the first (2j) or with every (2j + 1) half of the q
  int nj, lag;
  int tick0;    // the instance's first ticket; its tickets follow each other
};

// The launch: the instances (one in the arguments, or a device table of several), the ticket counter and
// the flags that every instance shares.
struct QLaunch {
  int* ctl;          // [0] ticket, [1] CTAs finished, [2] a wait gave up
  int* cnt_all;      // every instance's counters, contiguous (reset with ctl by the last CTA)
  int ncnt, total;   // counter ints; tickets of the launch
  int withhold;      // test hook: column tiles do not count themselves (the row tiles' waits run out)
  int ninst;
  const QInst* tab;  // device table of ninst instances, or null: inst0
  QInst inst0;
};

// Tile of ticket k (depth j counted from the call's first depth j0): kind 0 = column tile, 1 = row tile.  Groups s = 0 .. nj - 1 + lag: the column tiles
// of depth s (s < nj), then the row tiles of depth s - lag (s >= lag).
template <int N>
__device__ __forceinline__ void decode_ticket(int k, int nj, int lag, int& kind, int& j, int& t) {
  using G = QGeom<N>;
  constexpr int NCT = G::NCT, NRT = G::NRT, NG = NCT + NRT;
  if (k < lag * NCT) {
    kind = 0;
    j = k / NCT;
    t = k - j * NCT;
    return;
  }
  k -= lag * NCT;
  if (k < (nj - lag) * NG) {
    const int s = lag + k / NG, w = k % NG;
    if (w < NCT) {
      kind = 0;
      j = s;
      t = w;
    } else {
      kind = 1;
      j = s - lag;
      t = w - NCT;
    }
    return;
  }
  k -= (nj - lag) * NG;
  kind = 1;
  j = nj - lag + k / NRT;
  t = k % NRT;
}

// source parameters of the first half (the first dependency step of a row tile)
__device__ __forceinline__ int half_q(int Q) { return Q > 1 ? Q / 2 : 1; }

// tickets of one instance
template <int N> __host__ __device__ inline int queue_tickets(int nj, int) {
  using G = QGeom<N>;
  return nj * (G::NCT + G::NRT);
}

__device__ __forceinline__ void report_timeout(const QLaunch& ql, const QInst& qa) {
  atomicExch(ql.ctl + 2, 1);
  if (qa.f.info) atomicOr(qa.f.info, FR3D_INFO_TIMEOUT);
}

// Wait until *c >= target (acquire), or a wait elsewhere has given up; false if this one gave up.
__device__ __forceinline__ bool wait_count(const QLaunch& ql, const QInst& qa, const int* c, int target) {
  const volatile int* gave_up = ql.ctl + 2;
  for (long it = 0; it < kSpinLimit; ++it) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(c) : "memory");
    if (v >= target) return true;
    if (*gave_up) return true;   // the results are flagged already; do not wait again
    __nanosleep(128);
  }
  report_timeout(ql, qa);
  return false;
}

__device__ __forceinline__ void stage_wait(const QLaunch& ql, const QInst& qa, uint64_t* bar, uint32_t& parity) {
  if (!tc::mbar_wait(bar, parity, kSpinLimit)) report_timeout(ql, qa);
  parity ^= 1u;
}

// order this thread's earlier shared-memory accesses (and, through a preceding barrier, the CTA's) before
// its next bulk copies into shared memory, which run in the async proxy
__device__ __forceinline__ void fence_proxy_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// the same for global memory: the intermediate, written by other CTAs' generic stores, read by bulk copies
__device__ __forceinline__ void fence_proxy_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

__device__ __forceinline__ uint64_t evict_first_policy() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ float2 ld_evict_first(const float2* a, uint64_t pol) {
  float2 v;
  asm volatile("ld.global.nc.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(v.x), "=f"(v.y) : "l"(a), "l"(pol));
  return v;
}
// drop a 128-byte line of L2 without writing it back (its contents are not needed again)
__device__ __forceinline__ void l2_discard(const void* a) { asm volatile("discard.global.L2 [%0], 128;" ::"l"(a) : "memory"); }

// Column of stage slot c of column tile t: warp w handles the pair p = 4t + w of columns whose
// Hermitian-split partners they are, p and n/2 - p (p >= 1), or column 0 (packed: also kx = n/2) and
// column n/4, which are their own partners (p = 0); slot 2w + s holds the pair's column s.
template <int N> __device__ __forceinline__ int pair_column(int t, int c) {
  constexpr int L = N / 2;
  const int p = (kQThreads / 32) * t + (c >> 1), s = c & 1;
  return p == 0 ? (s == 0 ? 0 : L / 2) : (s == 0 ? p : L - p);
}

template <int N>
__device__ __forceinline__ void column_tile(const QLaunch& ql, const QInst& qa, int j, int t, float2* stage, float2* colbuf,
                                            float2* tab, uint64_t* bar, uint32_t* par, const int* s_aidx, int tid) {
  using G = QGeom<N>;
  constexpr int L = G::L, CT = G::CT, SSC = G::SSC, STG = G::STG;
  static_assert(CT == 2 * (kQThreads / 32), "two columns per warp");
  const FusedArgs& a = qa.f;
  const long ps = (long)(L + 1) * N;
  float2* stL = tab;              // [2][n] column n/2 of U~_q (tile 0)
  float2* ptc = tab + 2 * N;      // pass tables of length n
  const int c = tid >> 4, jj = tid & 15;   // stage slot (column) and butterfly of the first pass
  const int kx = pair_column<N>(t, c);
  const bool pk = kx == 0;                 // packed column 0: also carries kx = n/2
  const bool self = t == 0 && (c >> 1) == 0;   // columns 0 and n/4 are their own split partners
  auto issue = [&](int q, int sl) {
    const float2* src = a.Uh + (long)q * ps;
    tc::mbar_arrive_expect_tx(&bar[sl], (uint32_t)(sizeof(float2) * (STG + (t == 0 ? N : 0))));
#pragma unroll
    for (int cc = 0; cc < CT; ++cc)
      tc::bulk_g2s(stage + sl * STG + cc * N, src + (long)pair_column<N>(t, cc) * N, (uint32_t)(sizeof(float2) * N),
                   &bar[sl]);
    if (t == 0) tc::bulk_g2s(stL + sl * N, src + (long)L * N, (uint32_t)(sizeof(float2) * N), &bar[sl]);
  };
  if (tid == 0) {
    fence_proxy_smem();
    issue(0, 0);
    if (a.Q > 1) issue(1, 1);
  }
  build_passtw<N, 1, kQThreads>(ptc, a.tw_n, tid);
  // q-invariant solve weights w_j of this thread's 16 bins (and of column n/2 at the same ky), as the
  // fused kernel stages them: A_j times the chosen row of the solve table; the split twiddle w^kx
  float w[16], wl[16];
  const float2 twk = __ldg(a.tw_n + kx);
  {
    const float* Aj = a.A + (long)(a.j0 + j) * ps;
    int row[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const long o = (long)kx * N + jj + 16 * r;
      row[r] = a.nb > 1 ? s_aidx[__ldg(a.bbin + o)] : s_aidx[0];
    }
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const long o = (long)kx * N + jj + 16 * r;
      w[r] = __fmul_rn(__ldg(Aj + o), __ldg(a.Dd + (long)row[r] * ps + o));
    }
#pragma unroll
    for (int r = 0; r < 16; ++r) wl[r] = 0.f;
    if (pk) {
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        const long o = (long)L * N + jj + 16 * r;
        const int rw = a.nb > 1 ? s_aidx[__ldg(a.bbin + o)] : s_aidx[0];
        wl[r] = __fmul_rn(__ldg(Aj + o), __ldg(a.Dd + (long)rw * ps + o));
      }
    }
  }
  float2* Tj = qa.T + (long)j * a.Q * N * L;
  for (int q = 0; q < a.Q; ++q) {
    const int sl = q & 1;
    stage_wait(ql, qa, &bar[sl], par[sl]);
    // first pass of the inverse column DFTs from the stage (butterfly jj of column c: bins jj + 16 r)
    const float2* sg = stage + sl * STG + c * N;
    float2 v[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const float2 u = sg[jj + 16 * r];
      float2 x = make_float2(__fmul_rn(u.x, w[r]), __fmul_rn(u.y, w[r]));
      if (pk) {   // add i w(n/2, ky) U~(n/2, ky)
        const float2 un = stL[sl * N + jj + 16 * r];
        x.x = __fmaf_rn(-un.y, wl[r], x.x);
        x.y = __fmaf_rn(un.x, wl[r], x.y);
      }
      v[r] = x;
    }
    Dft<16, true>::run(v);
#pragma unroll
    for (int r = 0; r < 16; ++r) colbuf[c * SSC + pidx<float2>(jj * 16 + r)] = v[r];
    __syncthreads();   // the column buffer is complete and the stage consumed
    if (tid == 0 && q + 2 < a.Q) {
      fence_proxy_smem();
      issue(q + 2, sl);
    }
    // last pass: X(kx, y) for y = jj + 16 r
    auto emit = [&](int, int, float2 val, int, int r) { v[r] = val; };
    last_pass_to<N, true, CT, kQThreads>(colbuf, SSC, ptc, emit, tid);
    // Hermitian split of the row sequences, Z'(kx, y) = (X[kx] + conj X[L-kx]) + i w^-kx (X[kx] - conj X[L-kx])
    // with X[L-kx] from the partner column (the lane 16 apart), stored to T[j][q][y / 16][kx][y % 16]
    float2* Tq = Tj + (long)q * N * L;
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const float2 own = v[r];
      float2 oth;
      oth.x = __shfl_xor_sync(0xffffffffu, own.x, 16);
      oth.y = __shfl_xor_sync(0xffffffffu, own.y, 16);
      float2 xa = own, xb = self ? own : oth;
      if (pk) {   // X(0) and X(n/2): the real and imaginary parts of column 0
        xa = make_float2(own.x, 0.f);
        xb = make_float2(own.y, 0.f);
      }
      const float2 sum = cadd(xa, cconj(xb)), dif = csub(xa, cconj(xb));
      const int y = jj + 16 * r;
      Tq[((long)(y >> 4) * L + kx) * 16 + (y & 15)] = cadd(sum, cmul_mi<true>(cmul(cconj(twk), dif)));
    }
    // release of a half of the q: every thread makes its own stores visible GPU-wide (a fence orders only
    // the issuing thread's writes; the barrier below only orders their issue), then one thread counts
    const bool release = q == half_q(a.Q) - 1 || q == a.Q - 1;
    if (release) __threadfence();
    __syncthreads();   // the column buffer is free again
    if (tid == 0 && release && !ql.withhold) {
      if (q == half_q(a.Q) - 1) atomicAdd(qa.cnt + 2 * j, 1);
      if (q == a.Q - 1) atomicAdd(qa.cnt + 2 * j + 1, 1);
    }
  }
}

template <int N>
__device__ __forceinline__ void row_tile(const QLaunch& ql, const QInst& qa, int j, int b, float2* stage, float2* rowbuf,
                                         float2* tab, uint64_t* bar, uint32_t* par, uint64_t pol, int tid) {
  using G = QGeom<N>;
  constexpr int L = G::L, RB = G::RB, SSR = G::SSR, STG = G::STG, NCT = G::NCT;
  using LP = LastPass<L>;
  constexpr int NBF = RB * LP::BPS;
  constexpr int KR = (NBF + kQThreads - 1) / kQThreads;
  const FusedArgs& a = qa.f;
  float2* ptr = tab;                          // pass tables of length n/2
  const float2* Tj = qa.T + (long)j * a.Q * N * L;
  // q's rows once every column tile of depth j has finished the half of the source parameters q is in
  auto issue = [&](int q, int sl) {
    if (q == 0 || q == half_q(a.Q)) {
      wait_count(ql, qa, qa.cnt + 2 * j + (q == 0 ? 0 : 1), NCT);
      fence_proxy_global();
    }
    fence_proxy_smem();
    tc::mbar_arrive_expect_tx(&bar[sl], (uint32_t)(sizeof(float2) * STG));
    tc::bulk_g2s(stage + sl * STG, Tj + ((long)q * (N / 16) + b) * L * 16, (uint32_t)(sizeof(float2) * STG), &bar[sl]);
  };
  if (tid == 0) {
    issue(0, 0);
    if (a.Q > 1) issue(1, 1);
  }
  build_passtw<L, 2, kQThreads>(ptr, a.tw_n, tid);
  float2 acc[KR][LP::R], wv[KR][LP::R];
#pragma unroll
  for (int k = 0; k < KR; ++k)
#pragma unroll
    for (int rr = 0; rr < LP::R; ++rr) acc[k][rr] = make_float2(0.f, 0.f);
  // combination weights of q in the layout of the last pass (butterfly (row, jq) owns outputs jq + rr NS)
  auto load_w = [&](int q) {
    const float2* wq = reinterpret_cast<const float2*>(a.W + (((long)q * a.Mp + a.j0 + j) * N + b * RB) * N);
#pragma unroll
    for (int k = 0; k < KR; ++k) {
      const int bb = tid + k * kQThreads;
      if (NBF % kQThreads == 0 || bb < NBF) {
        const int sr = bb / LP::BPS, jq = bb % LP::BPS;
#pragma unroll
        for (int rr = 0; rr < LP::R; ++rr) wv[k][rr] = ld_evict_first(wq + sr * L + jq + rr * LP::NS, pol);
      }
    }
  };
  auto prefetch_w = [&](int q) {   // the tile's rows of W_q into L2, so that the register loads hit there
    const float* src = a.W + (((long)q * a.Mp + a.j0 + j) * N + b * RB) * N;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"((uint32_t)(RB * N * sizeof(float)))
                 : "memory");
  };
  if (tid == 0)
    for (int q = 0; q < 3 && q < a.Q; ++q) prefetch_w(q);
  load_w(0);
  __syncthreads();   // tables
  for (int q = 0; q < a.Q; ++q) {
    const int sl = q & 1;
    stage_wait(ql, qa, &bar[sl], par[sl]);
    // the rows of T are in shared memory now: drop their lines from L2 (one 128-byte line per thread)
    static_assert(STG * sizeof(float2) == 128 * kQThreads, "one line per thread");
    l2_discard(Tj + ((long)q * (N / 16) + b) * L * 16 + tid * 16);
    float2* sg = stage + sl * STG;            // Z'[k][row], split by the column tiles
    // first pass (radix 16, no twiddles) from the stage into the row buffer, the threads running over the
    // rows first: butterfly jb of a row reads jb + (n/32) r and writes 16 jb + r
    {
      constexpr int BPS0 = L / 16;
      static_assert(RB * BPS0 == kQThreads, "one first-pass butterfly per thread");
      const int row = tid % RB, jb = tid / RB;
      float2 v[16];
#pragma unroll
      for (int r = 0; r < 16; ++r) v[r] = sg[(jb + BPS0 * r) * RB + row];
      Dft<16, true>::run(v);
      __syncthreads();   // every thread has finished the previous q's last pass, which read the row buffer
      float2* rw = rowbuf + row * SSR;
#pragma unroll
      for (int r = 0; r < 16; ++r) rw[pidx<float2>(16 * jb + r)] = v[r];
    }
    __syncthreads();   // the row buffer is complete and the stage consumed
    if (tid == 0 && q + 2 < a.Q) issue(q + 2, sl);
    // fmaf(w, v, 0) for q = 0, as in the accumulators of the other variants
    auto emit = [&](int, int, float2 v, int k, int rr) {
      acc[k][rr] = make_float2(fmaf(wv[k][rr].x, v.x, acc[k][rr].x), fmaf(wv[k][rr].y, v.y, acc[k][rr].y));
    };
    last_pass_to<L, true, RB, kQThreads>(rowbuf, SSR, ptr, emit, tid);
    if (tid == 0 && q + 3 < a.Q) prefetch_w(q + 3);
    if (q + 1 < a.Q) load_w(q + 1);   // in flight during the next q's split and passes
  }
  float2* ov = reinterpret_cast<float2*>(a.out + ((long)(a.j0 + j) * N + b * RB) * N);
#pragma unroll
  for (int k = 0; k < KR; ++k) {
    const int bb = tid + k * kQThreads;
    if (NBF % kQThreads == 0 || bb < NBF) {
      const int sr = bb / LP::BPS, jq = bb % LP::BPS;
#pragma unroll
      for (int rr = 0; rr < LP::R; ++rr) ov[sr * L + jq + rr * LP::NS] = acc[k][rr];
    }
  }
}

template <int N>
__global__ void __launch_bounds__(kQThreads, kQMinBlocks) k_inv_queue(QLaunch ql) {
  using G = QGeom<N>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  int* s_tick = reinterpret_cast<int*>(smem_raw + 16);
  float2* stage = reinterpret_cast<float2*>(smem_raw + G::head);
  float2* buf = stage + 2 * G::STG;
  float2* tab = buf + G::BUF;
  __shared__ int s_aidx[FR3D_MAX_BANDS];
  __shared__ __align__(16) int s_inst_raw[sizeof(QInst) / 4];   // the current tile's instance descriptor
  QInst& s_inst = *reinterpret_cast<QInst*>(s_inst_raw);
  const int tid = threadIdx.x;
  if (tid == 0) {
    tc::mbar_init(&bar[0], 1);
    tc::mbar_init(&bar[1], 1);
    tc::mbar_fence_init();
  }
  uint32_t par[2] = {0u, 0u};   // parity of each stage barrier's next completion
  const uint64_t pol = evict_first_policy();
  pdl_wait();   // the data spectra, the chosen alpha indices and the queue counters of the previous call
  int cur = -1;   // instance held in s_inst
  for (;;) {
    if (tid == 0) *s_tick = atomicAdd(ql.ctl, 1);
    __syncthreads();   // the ticket; also orders the previous tile's last reads before this tile's writes
    const int tick = *s_tick;
    if (tick >= ql.total) break;
    // the instance of the ticket (the table is ordered by first ticket)
    int inst = 0;
    if (ql.tab) {
      int lo = 0, hi = ql.ninst - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&ql.tab[mid].tick0) <= tick) lo = mid;
        else hi = mid - 1;
      }
      inst = lo;
    }
    if (inst != cur) {   // a uniform branch: every thread computed the same instance
      constexpr int W = sizeof(QInst) / 4;
      static_assert(sizeof(QInst) % 4 == 0 && W <= kQThreads, "the descriptor is copied one word per thread");
      const int* src = reinterpret_cast<const int*>(ql.tab ? &ql.tab[inst] : &ql.inst0);
      if (tid < W) s_inst_raw[tid] = src[tid];
      __syncthreads();
      if (tid < s_inst.f.nb) s_aidx[tid] = min(max(s_inst.f.aidx[tid], 0), s_inst.f.na - 1);
      __syncthreads();
      cur = inst;
    }
    int kind, j, t;
    decode_ticket<N>(tick - s_inst.tick0, s_inst.nj, s_inst.lag, kind, j, t);
    if (kind == 0) column_tile<N>(ql, s_inst, j, t, stage, buf, tab, bar, par, s_aidx, tid);
    else row_tile<N>(ql, s_inst, j, t, stage, buf, tab, bar, par, pol, tid);
    __syncthreads();   // before thread 0 overwrites the ticket
  }
  // the last CTA to finish resets the queue for the next launch
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(ql.ctl + 1, 1) == (int)gridDim.x - 1) {
      __threadfence();
      ql.ctl[0] = 0;
      ql.ctl[2] = 0;
      for (int e = 0; e < ql.ncnt; ++e) ql.cnt_all[e] = 0;
      __threadfence();
      ql.ctl[1] = 0;
    }
  }
}

}  // namespace

std::atomic<int> g_withhold{0};

bool inv_queue_supported(int n, bool xi) { return n == 256 && xi; }

size_t inv_queue_ctl_ints(int nj, int) { return 4 + 2 * (size_t)nj; }

namespace {

int queue_launch(const QLaunch& ql, cudaStream_t st) {
  using G = QGeom<256>;
  const void* kern = reinterpret_cast<const void*>(k_inv_queue<256>);
  FR3D_TRY(smem_optin(kern, G::smem));
  static int grid_per_sm = 0;
  if (grid_per_sm == 0) grid_per_sm = std::max(1, resident_ctas(kern, kQThreads, G::smem));
  int dev = 0, sms = 0;
  FR3D_CUDA_TRY(cudaGetDevice(&dev));
  FR3D_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(std::min(ql.total, grid_per_sm * sms));
  cfg.blockDim = dim3(kQThreads);
  cfg.dynamicSmemBytes = G::smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  FR3D_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_inv_queue<256>, ql));
  return FR3D_OK;
}

QInst make_inst(const FusedArgs& f, float2* T, int* cnt, int nj, int tick0) {
  QInst qi;
  qi.f = f;
  qi.T = T;
  qi.cnt = cnt;
  qi.nj = nj;
  qi.lag = std::min(36, nj);
  qi.tick0 = tick0;
  return qi;
}

}  // namespace

// T: the intermediate ([nj][Q][n][n/2] complex, inv2_scratch_bytes); ctl: inv_queue_ctl_ints(nj, Q) zeroed
// ints (the kernel leaves them zeroed): [0..3] the launch's counters, then the depth counters.
int inv_queue_launch(int n, const FusedArgs& f, int nj, float2* T, int* ctl, cudaStream_t st) {
  if (!inv_queue_supported(n, true) || f.Zs) return FR3D_ERR_UNSUPPORTED_SIZE;
  QLaunch ql = {};
  ql.inst0 = make_inst(f, T, ctl + 4, nj, 0);
  ql.ctl = ctl;
  ql.cnt_all = ctl + 4;
  ql.ncnt = 2 * nj;
  ql.total = queue_tickets<256>(nj, ql.inst0.lag);
  ql.withhold = g_withhold.load();
  ql.ninst = 1;
  ql.tab = nullptr;
  return queue_launch(ql, st);
}

size_t inv_queue_inst_bytes() { return sizeof(QInst); }

int inv_queue_make_inst(void* dst, const FusedArgs& f, float2* T, int* cnt, int nj, int tick0) {
  const QInst qi = make_inst(f, T, cnt, nj, tick0);
  memcpy(dst, &qi, sizeof(QInst));
  return queue_tickets<256>(nj, qi.lag);
}

int inv_queue_launch_table(const void* tab, int ninst, int* ctl, int* cnt_all, int ncnt, int total, cudaStream_t st) {
  QLaunch ql = {};
  ql.ctl = ctl;
  ql.cnt_all = cnt_all;
  ql.ncnt = ncnt;
  ql.total = total;
  ql.withhold = g_withhold.load();
  ql.ninst = ninst;
  ql.tab = static_cast<const QInst*>(tab);
  return queue_launch(ql, st);
}

}  // namespace fr3d

extern "C" int fr3d_test_withhold_queue_counts(int on) { return fr3d::g_withhold.exchange(on ? 1 : 0); }
