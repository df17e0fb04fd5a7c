// C ABI of the library (include/fr3d.h): argument checks, workspace planning and the launch
// sequences of Algorithm 1 (Sec. 4-5) and of the forward operator (Eq. (4)-(6)).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "ops.cuh"

namespace fr3d {

// (tau delta_b)^2 per band: the noise energy of a band is delta^2 times its share of the frequencies
// (white noise), so delta_b^2 = delta^2 (frequencies in band b) / n^2
void band_thresholds(const Handle* H, const fr3d_invert_opts* o, int nb, double* thr2) {
  const double t2 = (o->tau * o->delta) * (o->tau * o->delta);
  if (nb == 1) {
    thr2[0] = t2;
    return;
  }
  const double n2 = (double)H->n * H->n;
  for (int b = 0; b < nb; ++b) thr2[b] = t2 * H->band_count[b] / n2;
}

namespace {

constexpr double kFourPi = 12.566370614359172953850573533118;
constexpr size_t kChunkBytes = 128ull << 20;  // cap of the per-depth-chunk spectrum buffer

size_t align_up(size_t v) { return (v + 255) & ~(size_t)255; }

int ensure_sources(Handle* H, const fr3d_sources* s) {
  if (!s || s->q < 1 || s->n_points < 1 || !s->xyz) return FR3D_ERR_INVALID_ARG;
  if ((long)s->q * s->n_points > FR3D_MAX_SOURCE_POINTS) return FR3D_ERR_UNSUPPORTED_SIZE;
  if (!(s->A0 != 0.0) || !isfinite(s->A0)) return FR3D_ERR_INVALID_ARG;
  const int np = s->q * s->n_points;
  std::vector<double> key(3 + 3 * (size_t)np);
  key[0] = s->q;
  key[1] = s->n_points;
  key[2] = s->A0;
  for (int i = 0; i < 3 * np; ++i) {
    if (!isfinite(s->xyz[i])) return FR3D_ERR_INVALID_ARG;
    key[3 + i] = s->xyz[i];
  }
  if (key == H->src_key) return FR3D_OK;
  if (!H->pts32) {
    FR3D_CUDA_TRY(cudaMalloc(&H->pts32, sizeof(float4) * FR3D_MAX_SOURCE_POINTS));
    FR3D_CUDA_TRY(cudaMalloc(&H->pts64, sizeof(double) * 3 * FR3D_MAX_SOURCE_POINTS));
  }
  std::vector<float4> p32(np);
  for (int i = 0; i < np; ++i)
    p32[i] = make_float4((float)s->xyz[3 * i], (float)s->xyz[3 * i + 1], (float)s->xyz[3 * i + 2], 0.f);
  FR3D_CUDA_TRY(cudaMemcpy(H->pts32, p32.data(), sizeof(float4) * np, cudaMemcpyHostToDevice));
  FR3D_CUDA_TRY(cudaMemcpy(H->pts64, s->xyz, sizeof(double) * 3 * np, cudaMemcpyHostToDevice));
  H->src_key.swap(key);
  return FR3D_OK;
}

SrcHost src_host(const Handle* H, int precision, const fr3d_sources* s) {
  SrcHost r;
  r.pts = precision == FR3D_PREC_FP64 ? (const void*)H->pts64 : (const void*)H->pts32;
  r.L = s->n_points;
  r.coef = -s->A0 / kFourPi;  // V0 = -A0/(4 pi) sum_l 1/|x - x_l| (Sec. 6)
  return r;
}

bool valid_precision(int p) { return p == FR3D_PREC_FP32 || p == FR3D_PREC_FP64; }
// the calls with per-class dense products (forward operator, alpha rule, inversion) also take the
// tensor-core precisions, which exist for several observation depths only (M = 1 has no contraction)
bool valid_contract_precision(int p) { return valid_precision(p) || tc_precision(p); }
int check_tc(const Handle* H, int p, int Q) {
  if (!tc_precision(p)) return FR3D_OK;
  if (H->M < 2 || H->M > 64 || H->Mp > 64 || Q > tc_max_q()) return FR3D_ERR_UNSUPPORTED_SIZE;
  return FR3D_OK;
}

// combination weights W_q = V0_q / sum_q' V0_q'^2 for the cached sources (rebuilt when they change)
int ensure_wtab(Handle* H, const fr3d_sources* s, cudaStream_t st) {
  if (H->wtab && H->wtab_key == H->src_key) return FR3D_OK;
  const size_t need = sizeof(float) * (size_t)s->q * H->Mp * H->n * H->n;
  if (H->wtab_cap < need) {
    if (H->wtab) cudaFree(H->wtab);
    H->wtab = nullptr;
    H->wtab_cap = 0;
    FR3D_CUDA_TRY(cudaMalloc(&H->wtab, need));
    H->wtab_cap = need;
  }
  FR3D_TRY(build_wtab(H, H->wtab, s->q, H->pts64, s->n_points, -s->A0 / kFourPi, st));
  H->wtab_key = H->src_key;
  return FR3D_OK;
}

// ------------------------------------------------------------------ forward operator
template <typename T>
int fwd_impl(Handle* H, const T* zeta, int Q, T* U, cudaStream_t st) {
  using C = typename Ops<T>::C;
  const int n = H->n;
  const long ps = (long)(n / 2 + 1) * n;
  const size_t zb = align_up(sizeof(C) * ps * H->Mp), ub = align_up(sizeof(C) * ps * H->M);
  FR3D_TRY(ensure_ws(H, zb + ub));
  C* Zh = reinterpret_cast<C*>(H->ws);
  C* Uh = reinterpret_cast<C*>((char*)H->ws + zb);
  const T* A;
  if constexpr (sizeof(T) == 4) A = H->A32;
  else {
    FR3D_TRY(build_dense64(H, st));
    A = H->A64d;
  }
  int launches = 0;
  for (int q = 0; q < Q; ++q) {
    FR3D_TRY(Ops<T>::row_r2c(H, zeta + (long)q * H->Mp * n * n, (long)n * n, Zh, H->Mp, st));
    FR3D_TRY(Ops<T>::col_plain(H, Zh, Zh, H->Mp, false, st));
    FR3D_TRY(Ops<T>::contract_fwd(H, Zh, Uh, A, 1, st));
    FR3D_TRY(Ops<T>::col_plain(H, Uh, Uh, H->M, true, st));
    FR3D_TRY(Ops<T>::row_c2r_plain(H, Uh, U + (long)q * H->M * n * n, H->M, 1, 0, 0, st));
    launches += 5;
  }
  H->last_launches = launches;
  return FR3D_OK;
}

// the forward operator with the per-class products on the tensor cores (M > 1)
int fwd_impl_tc(Handle* H, const float* zeta, int Q, float* U, int precision, cudaStream_t st) {
  const int n = H->n;
  const long ps = (long)(n / 2 + 1) * n;
  FR3D_TRY(ensure_tc_tables(H, 2, st));
  const size_t zb = align_up(sizeof(float2) * ps * H->Mp), ub = align_up(sizeof(float2) * ps * H->M);
  FR3D_TRY(ensure_ws(H, zb + ub));
  float2* Zh = reinterpret_cast<float2*>(H->ws);
  float2* Uh = reinterpret_cast<float2*>((char*)H->ws + zb);
  int launches = 0;
  for (int q = 0; q < Q; ++q) {
    FR3D_TRY(Ops<float>::row_r2c(H, zeta + (long)q * H->Mp * n * n, (long)n * n, Zh, H->Mp, st));
    FR3D_TRY(Ops<float>::col_plain(H, Zh, Zh, H->Mp, false, st));
    FR3D_TRY(tc_forward(H, Zh, Uh, precision == FR3D_PREC_BF16X3, st));
    FR3D_TRY(Ops<float>::col_plain(H, Uh, Uh, H->M, true, st));
    FR3D_TRY(Ops<float>::row_c2r_plain(H, Uh, U + (long)q * H->M * n * n, H->M, 1, 0, 0, st));
    launches += 5;
  }
  H->last_launches = launches;
  return FR3D_OK;
}

// ------------------------------------------------------------------ data transform + alpha rule
template <typename T>
int data_fft(Handle* H, const T* U, int Q, typename Ops<T>::C* Uh, cudaStream_t st) {
  const int n = H->n;
  FR3D_TRY(Ops<T>::row_r2c(H, U, (long)n * n, Uh, Q * H->M, st));
  prof_mark(H, kStRowR2C, st);
  FR3D_TRY(Ops<T>::col_plain(H, Uh, Uh, Q * H->M, false, st));
  prof_mark(H, kStColFwd, st);
  return FR3D_OK;
}

int check_alphas(const double* alphas, int n_alpha) {
  if (!alphas || n_alpha < 1) return FR3D_ERR_INVALID_ARG;
  if (n_alpha > FR3D_MAX_ALPHAS) return FR3D_ERR_UNSUPPORTED_SIZE;
  for (int k = 0; k < n_alpha; ++k) {
    if (!(alphas[k] > 0) || !isfinite(alphas[k])) return FR3D_ERR_INVALID_ARG;
    if (k && !(alphas[k] > alphas[k - 1])) return FR3D_ERR_INVALID_ARG;
  }
  return FR3D_OK;
}

template <typename T>
int choose_impl(Handle* H, const T* U, int Q, const double* alphas, int n_alpha, double delta, double tau,
                int* alpha_idx, double* residuals, int* info, cudaStream_t st) {
  using C = typename Ops<T>::C;
  const long ps = (long)(H->n / 2 + 1) * H->n;
  FR3D_TRY(ensure_ws(H, align_up(sizeof(C) * ps * Q * H->M)));
  C* Uh = reinterpret_cast<C*>(H->ws);
  FR3D_TRY(data_fft<T>(H, U, Q, Uh, st));
  FR3D_TRY(alpha_tables(H, alphas, n_alpha, FR3D_RA_TIKHONOV, st));
  const double thr2 = (tau * delta) * (tau * delta);
  FR3D_TRY(Ops<T>::alpha_choose(H, Uh, Q * H->M, n_alpha, &thr2, 1, alpha_idx, residuals, info, st));
  H->last_launches = 3;
  return FR3D_OK;
}

// ------------------------------------------------------------------ Algorithm 1
struct InvertPlan {
  size_t uh_off, t_off, uin_off, out_off, total;
  int chunk;
};

template <typename T>
InvertPlan plan_invert(const Handle* H, int Q, bool host_io, int output) {
  using C = typename Ops<T>::C;
  const int n = H->n;
  const size_t ps_b = sizeof(C) * (size_t)(n / 2 + 1) * n;
  InvertPlan p;
  p.uh_off = 0;
  size_t off = align_up(ps_b * Q * H->M);
  const size_t per_j = ps_b * Q;
  const bool fused = sizeof(T) == 4 && fused_supported(n);
  const bool multi = sizeof(T) == 4 && H->M > 1;      // the M > 1 path lays out its own workspace first
  int chunk = fused ? 0 : (int)std::max<size_t>(1, std::min<size_t>(H->Mp, kChunkBytes / per_j));
  if (multi) off = multi_ws_bytes(H, Q);
  if (fused || multi) {
    p.chunk = H->Mp;
    p.t_off = off;
    p.uin_off = p.out_off = 0;
    if (host_io) {
      p.uin_off = off;
      off += align_up(sizeof(T) * (size_t)Q * H->M * n * n);
      p.out_off = off;
      off += align_up(sizeof(T) * (size_t)(output == FR3D_OUT_XI ? 1 : Q) * H->Mp * n * n);
    }
    p.total = off;
    return p;
  }
  const int nch = (H->Mp + chunk - 1) / chunk;
  chunk = (H->Mp + nch - 1) / nch;
  p.chunk = chunk;
  p.t_off = off;
  off += align_up(per_j * chunk);
  p.uin_off = p.out_off = 0;
  if (host_io) {
    p.uin_off = off;
    off += align_up(sizeof(T) * (size_t)Q * H->M * n * n);
    p.out_off = off;
    off += align_up(sizeof(T) * (size_t)(output == FR3D_OUT_XI ? 1 : Q) * H->Mp * n * n);
  }
  p.total = off;
  return p;
}

int check_invert_args(Handle* H, int Q, const fr3d_invert_opts* o) {
  if (!o || Q < 1) return FR3D_ERR_INVALID_ARG;
  if (!valid_contract_precision(o->precision)) return FR3D_ERR_INVALID_ARG;
  if (H->M > FR3D_MAX_OBS_DEPTHS) return FR3D_ERR_UNSUPPORTED_SIZE;
  FR3D_TRY(check_tc(H, o->precision, Q));
  if (H->M > 1) {
    // several observation depths: FP32 data (eigen tables, multi.cu; products on CUDA or tensor cores)
    if (o->precision == FR3D_PREC_FP64) return FR3D_ERR_UNSUPPORTED_SIZE;
    if (o->alpha_mode == FR3D_ALPHA_LEARNED) return FR3D_ERR_INVALID_ARG;
  }
  if (o->output != FR3D_OUT_XI && o->output != FR3D_OUT_ZETA) return FR3D_ERR_INVALID_ARG;
  if (o->n_bands < 0 || o->n_bands > FR3D_MAX_BANDS) return FR3D_ERR_INVALID_ARG;
  if (o->ra != FR3D_RA_TIKHONOV && o->ra != FR3D_RA_TSVD) return FR3D_ERR_INVALID_ARG;
  if (o->alpha_mode == FR3D_ALPHA_FIXED) {
    if (!(o->alpha > 0) || !isfinite(o->alpha)) return FR3D_ERR_INVALID_ARG;
    if (o->n_bands > 1) return FR3D_ERR_INVALID_ARG;
  } else if (o->alpha_mode == FR3D_ALPHA_DISCREPANCY) {
    FR3D_TRY(check_alphas(o->alphas, o->n_alpha));
    if (!(o->delta >= 0) || !isfinite(o->delta) || !(o->tau > 0) || !isfinite(o->tau)) return FR3D_ERR_INVALID_ARG;
  } else if (o->alpha_mode == FR3D_ALPHA_GIVEN) {
    FR3D_TRY(check_alphas(o->alphas, o->n_alpha));
    if (!o->alpha_idx) return FR3D_ERR_INVALID_ARG;
  } else if (o->alpha_mode == FR3D_ALPHA_LEARNED) {
    FR3D_TRY(check_alphas(o->alphas, o->n_alpha));
    if (!(o->delta > 0) || !isfinite(o->delta)) return FR3D_ERR_INVALID_ARG;
    if (o->precision != FR3D_PREC_FP32 || o->ra != FR3D_RA_TIKHONOV) return FR3D_ERR_INVALID_ARG;
    if (!learned_net_fits(o->net, o->n_bands > 1 ? o->n_bands : 1)) return FR3D_ERR_INVALID_ARG;
  } else {
    return FR3D_ERR_INVALID_ARG;
  }
  if (o->output == FR3D_OUT_XI) {
    if (!o->sources) return FR3D_ERR_INVALID_ARG;
    if (o->sources->q != Q) return FR3D_ERR_INVALID_ARG;
    FR3D_TRY(ensure_sources(H, o->sources));
  }
  return FR3D_OK;
}

template <typename T>
int invert_impl(Handle* H, const T* U, int Q, const fr3d_invert_opts* o, T* out, const InvertPlan& p,
                cudaStream_t st, bool out_host_mapped = false) {
  using C = typename Ops<T>::C;
  if constexpr (sizeof(T) == 4) {
    if (H->M > 1) {
      if (o->output == FR3D_OUT_XI && fused_supported(H->n)) FR3D_TRY(ensure_wtab(H, o->sources, st));
      const SrcHost src = o->output == FR3D_OUT_XI ? src_host(H, FR3D_PREC_FP32, o->sources) : SrcHost{};
      return invert_multi(H, U, Q, o, out, src, st);
    }
  }
  C* Uh = reinterpret_cast<C*>((char*)H->ws + p.uh_off);
  C* Tb = reinterpret_cast<C*>((char*)H->ws + p.t_off);
  int launches = 0;
  prof_begin(H, st);
  // step 1: 2D DFT of the data
  FR3D_TRY(data_fft<T>(H, U, Q, Uh, st));
  launches += 2;
  // step 2 (parameter): alpha
  const int* aidx;
  const T* D;
  const int nb = o->n_bands > 1 ? o->n_bands : 1;
  if (nb > 1) FR3D_TRY(ensure_bands(H, nb, nullptr));
  if (o->alpha_mode == FR3D_ALPHA_DISCREPANCY) {
    FR3D_TRY(alpha_tables(H, o->alphas, o->n_alpha, o->ra, st));
    prof_mark(H, kStTable, st);
    int* idx = o->alpha_idx ? o->alpha_idx : H->idx_scratch;
    double thr2[FR3D_MAX_BANDS];
    band_thresholds(H, o, nb, thr2);
    FR3D_TRY(Ops<T>::alpha_choose(H, Uh, Q * H->M, o->n_alpha, thr2, nb, idx, o->residuals, o->info, st));
    prof_mark(H, kStAlpha, st);
    launches += 1;
    aidx = idx;
    if constexpr (sizeof(T) == 4) D = H->D32;
    else D = H->D64;
  } else if (o->alpha_mode == FR3D_ALPHA_LEARNED) {
    FR3D_TRY(alpha_tables(H, o->alphas, o->n_alpha, o->ra, st));
    prof_mark(H, kStTable, st);
    int* idx = o->alpha_idx ? o->alpha_idx : H->idx_scratch;
    if constexpr (sizeof(T) == 4) {
      FR3D_TRY(learned_alpha(H, Uh, Q * H->M, nb, o->delta, o->alphas, o->n_alpha, o->net, idx, nullptr, o->info, st));
      D = H->D32;
    } else {
      return FR3D_ERR_INVALID_ARG;   // excluded by check_invert_args
    }
    prof_mark(H, kStAlpha, st);
    launches += 1;
    aidx = idx;
  } else if (o->alpha_mode == FR3D_ALPHA_GIVEN) {
    FR3D_TRY(alpha_tables(H, o->alphas, o->n_alpha, o->ra, st));
    prof_mark(H, kStTable, st);
    aidx = o->alpha_idx;
    if constexpr (sizeof(T) == 4) D = H->D32;
    else D = H->D64;
    if (o->info) FR3D_CUDA_TRY(cudaMemsetAsync(o->info, 0, sizeof(int), st));
  } else {
    FR3D_TRY(fixed_table(H, o->alpha, o->ra, st));
    prof_mark(H, kStTable, st);
    aidx = H->zero_idx;
    if constexpr (sizeof(T) == 4) D = H->Dfix32;
    else D = H->Dfix64;
    if (o->alpha_idx) FR3D_CUDA_TRY(cudaMemsetAsync(o->alpha_idx, 0, sizeof(int), st));
    if (o->info) FR3D_CUDA_TRY(cudaMemsetAsync(o->info, 0, sizeof(int), st));
  }
  if constexpr (sizeof(T) == 4) {
    if (fused_supported(H->n)) {
      // steps 2 (solve) + 3 (inverse DFT) + 4 (combination) fused, one launch for all depths
      if (o->output == FR3D_OUT_XI) {
        FR3D_TRY(ensure_wtab(H, o->sources, st));
        prof_mark(H, kStTable, st);
      }
      const float* Dd = o->alpha_mode == FR3D_ALPHA_FIXED ? H->Ddfix32 : H->Dd32;
      FR3D_TRY(inv_fused_f32(H, Uh, Dd, aidx, nb, H->wtab, out, Q, 0, H->Mp, o->output, st, out_host_mapped,
                             o->info));
      prof_mark(H, kStFused, st);
      H->last_launches = launches + 1;
      return FR3D_OK;
    }
  }
  const T* A;
  if constexpr (sizeof(T) == 4) A = H->A32;
  else {
    FR3D_TRY(build_dense64(H, st));
    A = H->A64d;
  }
  // step 2 (solve) + step 3 (inverse DFT) + step 4 (xi = zeta / V0), by chunks of depths
  for (int j0 = 0; j0 < H->Mp; j0 += p.chunk) {
    const int nj = std::min(p.chunk, H->Mp - j0);
    FR3D_TRY(Ops<T>::col_solve1(H, Uh, Tb, A, D, aidx, nb, Q, j0, nj, st));
    prof_mark(H, kStColSolve, st);
    if (o->output == FR3D_OUT_XI)
      FR3D_TRY(Ops<T>::row_c2r_xi(H, Tb, out, nj, Q, j0, src_host(H, o->precision, o->sources), st));
    else
      FR3D_TRY(Ops<T>::row_c2r_plain(H, Tb, out, nj * Q, Q, j0, H->Mp, st));
    prof_mark(H, kStRowC2R, st);
    launches += 2;
  }
  H->last_launches = launches;
  return FR3D_OK;
}

}  // namespace

// Everything a batched run of this instance needs, built now: sources, combination weights, alpha
// tables, the data-spectrum workspace and the alpha-rule partial sums.  Returns the spectrum buffer,
// the dense solve-weight table and the device word that will hold the chosen alpha index.
int prepare_instance_f32(Handle* H, int Q, const fr3d_invert_opts* o, float2** Uh, const float** Dd,
                         const int** aidx, cudaStream_t st) {
  FR3D_TRY(check_invert_args(H, Q, o));
  if (Uh) {   // data spectra in the handle's workspace (Uh = NULL: the caller provides them)
    const InvertPlan p = plan_invert<float>(H, Q, false, o->output);
    FR3D_TRY(ensure_ws(H, p.total));
    *Uh = reinterpret_cast<float2*>((char*)H->ws + p.uh_off);
  }
  if (o->output == FR3D_OUT_XI) FR3D_TRY(ensure_wtab(H, o->sources, st));
  const int nb = o->n_bands > 1 ? o->n_bands : 1;
  if (nb > 1) FR3D_TRY(ensure_bands(H, nb, nullptr));
  if (o->alpha_mode == FR3D_ALPHA_LEARNED) return FR3D_ERR_INVALID_ARG;   // not in batched plans
  if (o->alpha_mode == FR3D_ALPHA_DISCREPANCY || o->alpha_mode == FR3D_ALPHA_GIVEN) {
    FR3D_TRY(alpha_tables(H, o->alphas, o->n_alpha, o->ra, st));
    FR3D_TRY(ensure_partials(H));
    *Dd = H->Dd32;
    *aidx = o->alpha_idx ? o->alpha_idx : H->idx_scratch;
  } else {
    FR3D_TRY(fixed_table(H, o->alpha, o->ra, st));
    *Dd = H->Ddfix32;
    *aidx = H->zero_idx;
  }
  FR3D_CUDA_TRY(cudaStreamSynchronize(st));
  return FR3D_OK;
}

}  // namespace fr3d

using fr3d::Handle;

extern "C" int fr3d_fwd_apply(fr3d_handle* h, const void* zeta, int Q, void* U, int precision, void* stream) {
  if (!h || !zeta || !U || Q < 1 || !fr3d::valid_contract_precision(precision)) return FR3D_ERR_INVALID_ARG;
  FR3D_TRY(fr3d::check_tc(h->padded ? &h->padded->h : &h->h, precision, 1));
  if (h->padded) return fr3d::padded_fwd_apply(h, zeta, Q, U, precision, (cudaStream_t)stream);
  Handle* H = &h->h;
  cudaStream_t st = (cudaStream_t)stream;
  if (precision == FR3D_PREC_FP64) return fr3d::fwd_impl<double>(H, (const double*)zeta, Q, (double*)U, st);
  if (fr3d::tc_precision(precision)) return fr3d::fwd_impl_tc(H, (const float*)zeta, Q, (float*)U, precision, st);
  return fr3d::fwd_impl<float>(H, (const float*)zeta, Q, (float*)U, st);
}

extern "C" int fr3d_zeta_from_xi(fr3d_handle* h, const void* xi, const fr3d_sources* sources, void* zeta,
                                 int precision, void* stream) {
  if (!h || !xi || !zeta || !fr3d::valid_precision(precision)) return FR3D_ERR_INVALID_ARG;
  if (h->padded) return fr3d::padded_zeta_from_xi(h, xi, sources, zeta, precision, (cudaStream_t)stream);
  Handle* H = &h->h;
  FR3D_TRY(fr3d::ensure_sources(H, sources));
  cudaStream_t st = (cudaStream_t)stream;
  const fr3d::SrcHost s = fr3d::src_host(H, precision, sources);
  H->last_launches = 1;
  if (precision == FR3D_PREC_FP64)
    return fr3d::Ops<double>::zeta_from_xi(H, (const double*)xi, (double*)zeta, sources->q, s, st);
  return fr3d::Ops<float>::zeta_from_xi(H, (const float*)xi, (float*)zeta, sources->q, s, st);
}

extern "C" int fr3d_choose_alpha(fr3d_handle* h, const void* U, int Q, const double* alphas, int n_alpha,
                                 double delta, double tau, int precision, int* alpha_idx, double* residuals,
                                 int* info, void* stream) {
  if (!h || !U || Q < 1 || !alpha_idx || !fr3d::valid_contract_precision(precision))
    return FR3D_ERR_INVALID_ARG;
  FR3D_TRY(fr3d::check_alphas(alphas, n_alpha));
  if (h->padded)
    return fr3d::padded_choose_alpha(h, U, Q, alphas, n_alpha, delta, tau, precision, alpha_idx, residuals, info,
                                     (cudaStream_t)stream);
  if (!(delta >= 0) || !isfinite(delta) || !(tau > 0) || !isfinite(tau)) return FR3D_ERR_INVALID_ARG;
  Handle* H = &h->h;
  cudaStream_t st = (cudaStream_t)stream;
  FR3D_TRY(fr3d::check_tc(H, precision, Q));
  if (H->M > 1) {
    if (H->M > FR3D_MAX_OBS_DEPTHS || precision == FR3D_PREC_FP64) return FR3D_ERR_UNSUPPORTED_SIZE;
    return fr3d::choose_multi(H, (const float*)U, Q, alphas, n_alpha, delta, tau, precision, alpha_idx, residuals,
                              info, st);
  }
  if (precision == FR3D_PREC_FP64)
    return fr3d::choose_impl<double>(H, (const double*)U, Q, alphas, n_alpha, delta, tau, alpha_idx, residuals,
                                     info, st);
  return fr3d::choose_impl<float>(H, (const float*)U, Q, alphas, n_alpha, delta, tau, alpha_idx, residuals, info,
                                  st);
}

extern "C" int fr3d_invert(fr3d_handle* h, const void* U, int Q, const fr3d_invert_opts* opts, void* out,
                           void* stream) {
  if (!h || !U || !out) return FR3D_ERR_INVALID_ARG;
  if (h->padded) {
    FR3D_TRY(fr3d::check_invert_args(&h->padded->h, Q, opts));
    // the learned rule's features and training targets exist for the periodic box only
    if (opts->alpha_mode == FR3D_ALPHA_LEARNED) return FR3D_ERR_UNSUPPORTED_SIZE;
    return fr3d::padded_invert(h, U, Q, opts, out, (cudaStream_t)stream);
  }
  Handle* H = &h->h;
  FR3D_TRY(fr3d::check_invert_args(H, Q, opts));
  cudaStream_t st = (cudaStream_t)stream;
  if (opts->precision == FR3D_PREC_FP64) {
    const fr3d::InvertPlan p = fr3d::plan_invert<double>(H, Q, false, opts->output);
    FR3D_TRY(fr3d::ensure_ws(H, p.total));
    return fr3d::invert_impl<double>(H, (const double*)U, Q, opts, (double*)out, p, st);
  }
  const fr3d::InvertPlan p = fr3d::plan_invert<float>(H, Q, false, opts->output);
  FR3D_TRY(fr3d::ensure_ws(H, p.total));
  return fr3d::invert_impl<float>(H, (const float*)U, Q, opts, (float*)out, p, st);
}

// The device address of a host buffer of `bytes` bytes that lies in one page-locked, device-mapped
// range (cudaHostAlloc, cudaHostRegister), 16-byte aligned; nullptr otherwise (pageable memory).
static void* host_mapped_alias(const void* p, size_t bytes) {
  if (bytes == 0 || reinterpret_cast<uintptr_t>(p) % 16) return nullptr;
  cudaPointerAttributes a0, a1;
  const char* last = static_cast<const char*>(p) + (bytes - 1);
  if (cudaPointerGetAttributes(&a0, p) != cudaSuccess || cudaPointerGetAttributes(&a1, last) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a0.type != cudaMemoryTypeHost || a1.type != cudaMemoryTypeHost || !a0.devicePointer || !a1.devicePointer)
    return nullptr;
  if (static_cast<char*>(a1.devicePointer) - static_cast<char*>(a0.devicePointer) != (ptrdiff_t)(bytes - 1))
    return nullptr;
  return a0.devicePointer;
}

template <typename T>
static int invert_host_t(Handle* H, const void* U_host, int Q, const fr3d_invert_opts* o, void* out_host,
                         cudaStream_t st) {
  const fr3d::InvertPlan p = fr3d::plan_invert<T>(H, Q, true, o->output);
  FR3D_TRY(fr3d::ensure_ws(H, p.total));
  const int n = H->n;
  T* Ud = reinterpret_cast<T*>((char*)H->ws + p.uin_off);
  T* Od = reinterpret_cast<T*>((char*)H->ws + p.out_off);
  const size_t in_b = sizeof(T) * (size_t)Q * H->M * n * n;
  const size_t out_b = sizeof(T) * (size_t)(o->output == FR3D_OUT_XI ? 1 : Q) * H->Mp * n * n;
  // FP32, one observation depth: page-locked host buffers are used in place over the host link (the
  // first row pass reads U, the last kernel writes the result; each element crosses once), so the
  // transfers overlap the kernels instead of preceding and following them
  const T* Uin = Ud;
  T* Out = Od;
  if (sizeof(T) == 4 && H->M == 1) {
    if (void* m = host_mapped_alias(U_host, in_b)) Uin = static_cast<const T*>(m);
    if (void* m = host_mapped_alias(out_host, out_b)) Out = static_cast<T*>(m);
  }
  if (Uin == Ud) FR3D_CUDA_TRY(cudaMemcpyAsync(Ud, U_host, in_b, cudaMemcpyHostToDevice, st));
  FR3D_TRY(fr3d::invert_impl<T>(H, Uin, Q, o, Out, p, st, Out != Od));
  if (Out == Od) FR3D_CUDA_TRY(cudaMemcpyAsync(out_host, Od, out_b, cudaMemcpyDeviceToHost, st));
  FR3D_CUDA_TRY(cudaStreamSynchronize(st));
  return FR3D_OK;
}

extern "C" int fr3d_invert_host(fr3d_handle* h, const void* U_host, int Q, const fr3d_invert_opts* opts,
                                void* out_host, void* stream) {
  if (!h || !U_host || !out_host) return FR3D_ERR_INVALID_ARG;
  if (h->padded) {
    FR3D_TRY(fr3d::check_invert_args(&h->padded->h, Q, opts));
    if (opts->alpha_mode == FR3D_ALPHA_LEARNED) return FR3D_ERR_UNSUPPORTED_SIZE;
    return fr3d::padded_invert_host(h, U_host, Q, opts, out_host, (cudaStream_t)stream);
  }
  Handle* H = &h->h;
  FR3D_TRY(fr3d::check_invert_args(H, Q, opts));
  cudaStream_t st = (cudaStream_t)stream;
  if (opts->precision == FR3D_PREC_FP64) return invert_host_t<double>(H, U_host, Q, opts, out_host, st);
  return invert_host_t<float>(H, U_host, Q, opts, out_host, st);
}

extern "C" int fr3d_assemble_rhs(fr3d_handle* h, const float* dV2dz, int Q, const fr3d_sources* sources, double A2,
                                 double c0, int n_pi, double pi_half, float* U, void* stream) {
  if (!h || !dV2dz || !U || Q < 1 || !sources || sources->q != Q) return FR3D_ERR_INVALID_ARG;
  if (h->padded) return FR3D_ERR_UNSUPPORTED_SIZE;   // periodic box only
  if (n_pi < 2 || (n_pi & 1) || !(pi_half > 0) || !isfinite(pi_half) || !isfinite(A2) || !(c0 > 0) || !isfinite(c0))
    return FR3D_ERR_INVALID_ARG;
  Handle* H = &h->h;
  if (H->M > FR3D_MAX_OBS_DEPTHS) return FR3D_ERR_UNSUPPORTED_SIZE;
  FR3D_TRY(fr3d::ensure_sources(H, sources));
  const int L = sources->n_points;
  // no source point may sit on a node of Pi's grid (the density 1/|x' - x_l| would be infinite there)
  const double dzp = 2.0 * pi_half / n_pi;
  for (int e = 0; e < Q * L; ++e) {
    const double* p = sources->xyz + 3 * e;
    auto off = [](double v, double o, double step) {
      const double t = (v - o) / step - 0.5;
      return fabs(t - nearbyint(t)) * step;
    };
    const double dx = off(p[0], H->x0, H->h), dy = off(p[1], H->y0, H->h), dz = off(p[2], -pi_half, dzp);
    if (dx * dx + dy * dy + dz * dz < 1e-24 * (H->h * H->h)) return FR3D_ERR_BAD_GEOMETRY;
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (!H->pi || H->pi_n != n_pi || H->pi_half != pi_half) {
    if (H->pi) fr3d_handle_destroy(H->pi);
    H->pi = nullptr;
    std::vector<double> zp(n_pi), nu(n_pi, dzp);
    for (int k = 0; k < n_pi; ++k) zp[k] = -pi_half + (k + 0.5) * dzp;
    fr3d_geometry g;
    g.nx = g.ny = H->n;
    g.x0 = H->x0;
    g.y0 = H->y0;
    g.hx = g.hy = H->h;
    g.pad = 1;
    g.nzr = n_pi;
    g.zr = zp.data();
    g.nu = nu.data();
    g.nzy = H->M;
    g.zy = H->zy.data();
    g.kernel_kind = FR3D_K_DZ_INV_R;
    FR3D_TRY(fr3d_kernel_transform(&g, &H->pi, stream));   // rejects observation depths on Pi's grid
    H->pi_n = n_pi;
    H->pi_half = pi_half;
  }
  const size_t plane = (size_t)H->n * H->n;
  const size_t fb = (sizeof(float) * Q * n_pi * plane + 255) & ~(size_t)255;
  const size_t ib = sizeof(float) * Q * H->M * plane;
  if (H->rhs_bytes < fb + ib) {
    if (H->rhs_buf) cudaFree(H->rhs_buf);
    H->rhs_buf = nullptr;
    H->rhs_bytes = 0;
    FR3D_CUDA_TRY(cudaMalloc(&H->rhs_buf, fb + ib));
    H->rhs_bytes = fb + ib;
  }
  float* f = reinterpret_cast<float*>(H->rhs_buf);
  float* I = reinterpret_cast<float*>((char*)H->rhs_buf + fb);
  FR3D_TRY(fr3d::rhs_pi_density(f, Q, n_pi, H->n, H->x0, H->h, pi_half, H->pts64, L, st));
  FR3D_TRY(fr3d::fwd_impl<float>(&H->pi->h, f, Q, I, st));
  const double coef = sources->A0 / (4.0 * 3.14159265358979323846 * c0 * c0);
  FR3D_TRY(fr3d::rhs_combine(H, dV2dz, I, U, Q, H->pts64, L, A2, coef, st));
  H->last_launches = 2 + H->pi->h.last_launches;
  return FR3D_OK;
}

extern "C" int fr3d_last_launch_count(fr3d_handle* h) { return h ? h->h.last_launches : -1; }

extern "C" int fr3d_profile_enable(fr3d_handle* h, int enable) {
  if (!h) return FR3D_ERR_INVALID_ARG;
  if (h->padded) return fr3d_profile_enable(h->padded, enable);   // the stages of the box's calls
  Handle* H = &h->h;
  if (enable && !H->ev[0]) {
    for (int i = 0; i < Handle::kMaxEv; ++i) FR3D_CUDA_TRY(cudaEventCreate(&H->ev[i]));
  }
  H->prof_on = enable != 0;
  H->n_ev = 0;
  return FR3D_OK;
}

extern "C" int fr3d_profile_read(fr3d_handle* h, int* kinds, float* ms, int cap) {
  if (!h || (cap > 0 && (!kinds || !ms))) return FR3D_ERR_INVALID_ARG;
  if (h->padded) return fr3d_profile_read(h->padded, kinds, ms, cap);
  Handle* H = &h->h;
  if (H->n_ev < 2) return 0;
  FR3D_CUDA_TRY(cudaEventSynchronize(H->ev[H->n_ev - 1]));
  const int n = std::min(cap, H->n_ev - 1);
  for (int i = 0; i < n; ++i) {
    kinds[i] = H->ev_kind[i];
    FR3D_CUDA_TRY(cudaEventElapsedTime(&ms[i], H->ev[i], H->ev[i + 1]));
  }
  return n;
}

extern "C" const char* fr3d_status_string(int s) {
  switch (s) {
    case FR3D_OK: return "ok";
    case FR3D_ERR_INVALID_ARG: return "invalid argument";
    case FR3D_ERR_BAD_GEOMETRY: return "bad geometry (R and Y must be disjoint: every z_i - z'_j non-zero; h > 0)";
    case FR3D_ERR_UNSUPPORTED_SIZE: return "unsupported size";
    case FR3D_ERR_OOM: return "device allocation failed";
    case FR3D_ERR_CUDA: return "CUDA runtime error";
    case FR3D_ERR_TIMEOUT: return "bounded device wait gave up";
    case FR3D_ERR_NONFINITE_INPUT: return "non-finite input";
    default: return "unknown status";
  }
}
