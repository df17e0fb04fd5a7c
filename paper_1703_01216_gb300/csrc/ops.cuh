// Host-side launchers of the per-precision kernels (internal interface between api.cu and
// ops_f32.cu / ops_f64.cu).
#pragma once

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace fr3d {

struct SrcHost {
  const void* pts;  // float4* (FP32) or double* (FP64), device
  int L;
  double coef;      // -A0 / (4 pi)
};

template <typename T> struct Ops {
  using C = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
  // row pass real -> half spectrum for nplanes planes (plane stride in_ps reals)
  static int row_r2c(const Handle* H, const T* in, long in_ps, C* out, int nplanes, cudaStream_t st);
  // column pass in place/out of place, plain
  static int col_plain(const Handle* H, const C* in, C* out, int nplanes, bool inverse, cudaStream_t st);
  // inverse column pass with the M = 1 Tikhonov weights; output planes jc * Q + q, jc < nj
  static int col_solve1(const Handle* H, const C* Uh, C* out, const T* A, const T* D, const int* aidx, int nb,
                        int Q, int j0, int nj, cudaStream_t st);
  // row pass half spectrum -> real; input plane ip -> output plane (ip % Q) * out_stride + j0 + ip / Q
  static int row_c2r_plain(const Handle* H, const C* in, T* out, int nplanes, int Q, int j0, int out_stride,
                           cudaStream_t st);
  // row pass with the combination xi = sum_q V0_q zeta_q / sum_q V0_q^2 for depths j0 .. j0 + nj - 1
  static int row_c2r_xi(const Handle* H, const C* in, T* out, int nj, int Q, int j0, const SrcHost& src,
                        cudaStream_t st);
  // U~[q][i] = (1/n^2) sum_j A[i][j] zeta~[q][j] for every half-spectrum bin
  static int contract_fwd(const Handle* H, const C* Zh, C* Uh, const T* A, int Q, cudaStream_t st);
  // zeta[q][j] = xi[j] * V0_q
  static int zeta_from_xi(const Handle* H, const T* xi, T* zeta, int Q, const SrcHost& src, cudaStream_t st);
  // discrepancy choice over the cached alpha tables (M = 1), per band (nb = 1: whole spectrum);
  // thr2[b] = (tau delta_b)^2
  static int alpha_choose(Handle* H, const C* Uh, int nplanes, int n_alpha, const double* thr2, int nb, int* aidx,
                          double* residuals, int* info, cudaStream_t st);
};

// fused inverse (FP32, M = 1): solve + inverse 2D DFT + combination for depths j0 .. j0 + nj - 1;
// out_host_mapped: out is the device address of page-locked host memory (the autotuner then keeps to
// the variants that write every output once)
bool fused_supported(int n);
int inv_fused_f32(const Handle* H, const float2* Uh, const float* Dd, const int* aidx, int nb, const float* W,
                  float* out, int Q, int j0, int nj, int output, cudaStream_t st, bool out_host_mapped = false,
                  int* info = nullptr);
// the two-pass inverse (inv2p.cu): column pass with the solve, row pass with the combination; T holds
// inv2_scratch_bytes(n, Q, nj)
struct FusedArgs;
size_t inv2_scratch_bytes(int n, int Q, int nj);
int inv2_launch(int n, bool xi, const FusedArgs& f, int nj, float2* T, cudaStream_t st);
// The persistent tile-queue inverse (inv_queue.cu): n = 256, xi output, U~ input (no solved spectra).
// T: the two-pass intermediate (inv2_scratch_bytes); ctl: inv_queue_ctl_ints(nj, Q) ints, zeroed once at
// allocation (every launch leaves them zeroed).
bool inv_queue_supported(int n, bool xi);
size_t inv_queue_ctl_ints(int nj, int Q);
int inv_queue_launch(int n, const FusedArgs& f, int nj, float2* T, int* ctl, cudaStream_t st);
// The same queue over several instances of n = 256 in one launch: every instance's descriptor (written to
// host memory by inv_queue_make_inst, which returns the instance's ticket count; tick0 = the tickets of the
// instances before it) in a device table; ctl: 4 zeroed ints; cnt_all: ncnt zeroed ints holding every
// instance's 2 nj counters (cnt); total = all tickets.  The launch leaves ctl and cnt_all zeroed.
size_t inv_queue_inst_bytes();
int inv_queue_make_inst(void* dst, const FusedArgs& f, float2* T, int* cnt, int nj, int tick0);
int inv_queue_launch_table(const void* tab, int ninst, int* ctl, int* cnt_all, int ncnt, int total, cudaStream_t st);
// W_q = V0_q / sum_q' V0_q'^2 on the R grid for the handle's cached sources
int build_wtab(const Handle* H, float* W, int Q, const double* pts64, int L, double coef, cudaStream_t st);

// alpha-rule partial sums buffer (per block, band and candidate)
int ensure_partials(Handle* H);
// band of every frequency class (cband) and of every half-spectrum bin (bbin) for nb radial bands,
// and the number of grid frequencies per band
int ensure_bands(Handle* H, int nb, std::vector<double>* count);

// learned per-band alpha (learned.cu): one launch computing the band features (to feat, if given)
// and, with a network, the per-band candidate indices (to aidx); info gets the INFO bits
bool learned_net_fits(const fr3d_mlp* net, int nb);
int learned_alpha(Handle* H, const float2* Uh, int nplanes, int nb, double delta, const double* alphas, int na,
                  const fr3d_mlp* net, int* aidx, float* feat, int* info, cudaStream_t st);

// several observation depths (multi.cu): eigen tables of every class, the inversion and the alpha
// choice, and the workspace bytes the inversion lays out from the start of the handle's workspace
int ensure_multi_tables(Handle* H, cudaStream_t st);
size_t multi_ws_bytes(const Handle* H, int Q);
// src: the point sources of the combination (XI output; used at sizes without the fused inverse)
int invert_multi(Handle* H, const float* U, int Q, const fr3d_invert_opts* o, float* out, const SrcHost& src,
                 cudaStream_t st);
int choose_multi(Handle* H, const float* U, int Q, const double* alphas, int na, double delta, double tau,
                 int precision, int* aidx, double* residuals, int* info, cudaStream_t st);
void band_thresholds(const Handle* H, const fr3d_invert_opts* o, int nb, double* thr2);
// fused inverse DFT + combination of already solved spectra Zs [Q][M'][n/2+1][n] (1/n^2 folded in)
int inv_fused_presolved_f32(const Handle* H, const float2* Zs, const float* W, float* out, int Q, int output,
                            cudaStream_t st);

// per-class dense products on the tensor cores (tc_contract.cu; M > 1, BF16 operands, FP32 accumulation;
// split = the hi + lo form of FR3D_PREC_BF16X3)
bool tc_precision(int precision);
int tc_max_q();
int ensure_tc_tables(Handle* H, int kind, cudaStream_t st);
int tc_project(Handle* H, float2* Uh, int Q, double* Pc, bool split, int* info, cudaStream_t st);
int tc_solve(Handle* H, const float2* P, int Q, const int* aidx, const double* alphas, int na, int ra, int nb,
             float2* Zs, int jq, bool split, int* info, cudaStream_t st);
int tc_forward(Handle* H, const float2* Zh, float2* Uh, bool split, cudaStream_t st);

// right-hand side of Eq. (7) (rhs.cu): the density sum_l 1/|x' - x_l| on the box Pi, and the combination
// U = 2 pi d + (A2 / 2) sum_l d/dx3 (1/|x - x_l|) - coef I on the observation grid
int rhs_pi_density(float* f, int Q, int npi, int n, double x0, double h, double half, const double* pts, int L,
                   cudaStream_t st);
int rhs_combine(const Handle* H, const float* d, const float* I, float* U, int Q, const double* pts, int L,
                double A2, double coef, cudaStream_t st);

// precision-independent table builders (alpha tables, fixed alpha)
int alpha_tables(Handle* H, const double* alphas, int n_alpha, int ra, cudaStream_t st);
int fixed_table(Handle* H, double alpha, int ra, cudaStream_t st);
int build_dense64(Handle* H, cudaStream_t st);

// pad = 2 handles (pad.cu): inputs embedded in the low corner of the 2n x 2n box, the inner handle's
// call, results cropped to n x n
int padded_fwd_apply(fr3d_handle* h, const void* zeta, int Q, void* U, int precision, cudaStream_t st);
int padded_zeta_from_xi(fr3d_handle* h, const void* xi, const fr3d_sources* sources, void* zeta, int precision,
                        cudaStream_t st);
int padded_choose_alpha(fr3d_handle* h, const void* U, int Q, const double* alphas, int n_alpha, double delta,
                        double tau, int precision, int* alpha_idx, double* residuals, int* info, cudaStream_t st);
int padded_invert(fr3d_handle* h, const void* U, int Q, const fr3d_invert_opts* o, void* out, cudaStream_t st);
int padded_invert_host(fr3d_handle* h, const void* U_host, int Q, const fr3d_invert_opts* o, void* out_host,
                       cudaStream_t st);

}  // namespace fr3d
