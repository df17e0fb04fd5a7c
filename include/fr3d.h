/*
 * fr3d.h -- C ABI of the GB300 (sm_103a) FFT-Tikhonov inversion library.
 *
 * The library solves the linear first-kind Fredholm equation of Leonov &
 * Bakushinsky (arXiv 1703.01216), Eq. (4):
 *
 *     integral over R of K(x - x', y - y', z - z') zeta(x', y', z') dx' dy' dz' = U(x, y, z),
 *     (x, y, z) in Y,      K(x, y, z) = d/dz (1/r) = -z / (x^2 + y^2 + z^2)^(3/2),
 *
 * for the flat-layer geometry of Sec. 3 (R and Y horizontal slabs), with
 * Algorithm 1 of Sec. 4 in the finite-dimensional form of Sec. 5:
 *   step 1  2D DFT over (x, y) of the data and of the sampled kernel,
 *   step 2  per horizontal frequency m, a Tikhonov solution of the small system
 *           A^(m) zeta~^(m) = U~^(m) of Eq. (6), alpha by the discrepancy principle,
 *   step 3  inverse 2D DFT per depth z'_j,
 *   step 4  xi = zeta / V0, xi = 1/c0^2 - 1/c^2 (c = (1/c0^2 - xi)^(-1/2)).
 *
 * Conventions.  Horizontal grid: n x n voxel-centred points x_a = x0 + (a + 1/2) h
 * (same in y).  The box is periodic (pad = 1, the paper's discrete model of Sec. 5) or the
 * zero-padded box of twice the side (pad = 2: volumes stay n x n, the transforms run on 2n x 2n
 * with the inputs in the low corner and zeros elsewhere, and results are cropped to n x n).
 * Real volumes are row-major [plane][y][x] (x fastest).  The forward DFT is
 * unnormalised, the inverse carries 1/n^2; the continuous transform is
 * approximated by h^2 * DFT.  Depth grids: M' depths z'_j of R with quadrature
 * weights nu_j, and M observation depths z_i of Y; every z_i - z'_j must be
 * non-zero (R and Y are disjoint, Sec. 1).  The Tikhonov parameter is
 * dimensionless: the regulariser is alpha * s^2 with s^2 = max_m ||A^(m)||_F^2.
 *
 * Memory.  Data pointers (volumes, alpha_idx, residuals, info) are DEVICE
 * pointers owned by the caller unless stated otherwise; small parameter arrays
 * (depths, alphas, source points) are HOST pointers read during the call.  The
 * handle owns its device tables and a workspace that grows on the first call for
 * a new shape (so make that first call outside any stream capture).  Calls are
 * asynchronous on the given CUDA stream (NULL = legacy default stream); results
 * are valid once the stream has synchronised.  One handle serves one stream at a
 * time: concurrent calls on one handle share its workspace and race.
 *
 * Errors.  Every call returns an int status: FR3D_OK (0) or a negative
 * FR3D_ERR_* code; argument and geometry checks happen on the host before any
 * launch, so an error return means nothing was enqueued.  Conditions only the
 * device can see (alpha rule outcome, non-finite data) are reported as
 * FR3D_INFO_* bit flags in an optional device int.  No C++ exception crosses
 * this interface.
 */
#ifndef FR3D_H
#define FR3D_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define FR3D_OK 0
#define FR3D_ERR_INVALID_ARG (-1)      /* NULL pointer, negative count, bad enum */
#define FR3D_ERR_BAD_GEOMETRY (-2)     /* some z_i - z'_j == 0 (R and Y overlap), h <= 0 */
#define FR3D_ERR_UNSUPPORTED_SIZE (-3) /* n not 2^a 3^b in [16, 512], nx != ny, too many alphas/sources,
                                          pad not 1 or 2 (pad 2: 2n too), a call that keeps the
                                          periodic box made on a pad-2 handle */
#define FR3D_ERR_OOM (-4)              /* device allocation failed */
#define FR3D_ERR_CUDA (-5)             /* a CUDA runtime call failed */
#define FR3D_ERR_TIMEOUT (-6)          /* a bounded device wait gave up */
#define FR3D_ERR_NONFINITE_INPUT (-7)  /* reserved for synchronous checks */

/* ---- device-side info bits (OR-ed into *info when an info pointer is given) ---- */
#define FR3D_INFO_ALPHA_NONE_SATISFIES 1 /* no candidate met the bound: the smallest alpha was used */
#define FR3D_INFO_ALPHA_ALL_SATISFY 2    /* every candidate met the bound: the largest alpha was used */
#define FR3D_INFO_NONFINITE 4            /* the data spectrum held NaN/Inf */
#define FR3D_INFO_LEARNED_OUT_OF_RANGE 8 /* LEARNED: a band's predicted log10 alpha lay more than half a
                                            decade outside the candidate grid (the nearest end was used;
                                            the discrepancy rule is the fallback to run) */
#define FR3D_INFO_TIMEOUT 16             /* a bounded device wait (a tensor-core copy or MMA completion,
                                            or the tile-queue inverse's wait on a release) gave up: the
                                            outputs of this call are incomplete */

/* ---- enums ---- */
#define FR3D_K_DZ_INV_R 0 /* K = d/dz (1/r), Eq. (4) (the equation the paper solves) */
#define FR3D_K_INV_R 1    /* K = 1/r: the first equation Sec. 3 derives, for data V2 instead of its
                             z-derivative; the periodic box keeps every bin finite, including k = 0 */
#define FR3D_PREC_FP32 0  /* FP32 FFTs, FP64 alpha rule; data and outputs are float */
#define FR3D_PREC_FP64 1  /* FP64 throughout; data and outputs are double */
#define FR3D_PREC_BF16TC 2 /* M > 1 only: as FP32, but the per-class dense products of Eq. (6) (projection
                              onto the Gram eigenvectors, the solve, the forward operator) run on the
                              tensor cores with BF16 tables and right-hand sides and FP32 accumulation;
                              data and outputs are float.  Relative error per product ~ 2^-9. */
#define FR3D_PREC_BF16X3 3 /* as BF16TC with every table and right-hand side split into two BF16 numbers
                              (hi + lo) and three products (hi hi + hi lo + lo hi) per contraction:
                              relative error per product ~ 2^-16 */
#define FR3D_ALPHA_FIXED 0
#define FR3D_ALPHA_DISCREPANCY 1
#define FR3D_ALPHA_GIVEN 2        /* per-band indices into `alphas` supplied in alpha_idx (no sweep) */
#define FR3D_ALPHA_LEARNED 3      /* per-band alpha predicted by a trained network (fr3d_mlp, below) */
#define FR3D_RA_TIKHONOV 0 /* regularising algorithm: Tikhonov, regulariser alpha s^2 ||zeta~||^2 (Sec. 4) */
#define FR3D_RA_TSVD 1     /* truncated SVD per frequency (Sec. 5, the paper's best RA): singular values
                              with sigma^2 < alpha s^2 are dropped */
#define FR3D_OUT_ZETA 0   /* output zeta_q per source parameter: [Q][M'][n][n] */
#define FR3D_OUT_XI 1     /* output xi (Algorithm 1 step 4): [M'][n][n] */

#define FR3D_MAX_ALPHAS 128
#define FR3D_MAX_BANDS 16
#define FR3D_MAX_SOURCE_POINTS 256 /* total points over all source parameters q */
#define FR3D_MAX_OBS_DEPTHS 64     /* M (observation depths) of fr3d_invert; M > 1 needs FP32 */

/* Flat-layer geometry (Sec. 3: R = R^2 x [h, H], Y = R^2 x [h_Y, H_Y]; Sec. 5 grids). */
typedef struct fr3d_geometry {
  int nx, ny;              /* horizontal grid; nx == ny == n, n = 2^a 3^b with 16 <= n <= 512 */
  double x0, y0, hx, hy;   /* voxel-centred grid x_a = x0 + (a + 1/2) hx; hx == hy > 0 */
  int pad;                 /* box factor P: 1 (periodic box of side n h) or 2 (zero-padded box of side
                              2 n h; 2n must itself be a supported size, so n <= 256) */
  int nzr;                 /* M' >= 1: depths of R */
  const double* zr;        /* host [M'] depths z'_j */
  const double* nu;        /* host [M'] quadrature weights nu_j (NULL: midpoint, |z'_1 - z'_0|, or 1 if M' = 1) */
  int nzy;                 /* M >= 1: observation depths of Y */
  const double* zy;        /* host [M] depths z_i; z_i != z'_j for all i, j */
  int kernel_kind;         /* FR3D_K_DZ_INV_R or FR3D_K_INV_R */
} fr3d_geometry;

/* Point sources of the model example (Sec. 6): for source parameter q the field source is
 * sum_l delta(x - x_{q,l}); V0_q(x) = -A0/(4 pi) sum_l 1/|x - x_{q,l}| (points outside R and Y). */
typedef struct fr3d_sources {
  int q;                   /* number of source parameters Q >= 1 */
  int n_points;            /* points per source parameter L >= 1 (Q * L <= FR3D_MAX_SOURCE_POINTS) */
  const double* xyz;       /* host [Q][L][3] */
  double A0;               /* A0 = integral of g(t) dt, non-zero (Sec. 2, Assumption 5) */
} fr3d_sources;

typedef struct fr3d_handle fr3d_handle;
typedef struct fr3d_mlp fr3d_mlp;

typedef struct fr3d_invert_opts {
  int alpha_mode;          /* FR3D_ALPHA_FIXED or FR3D_ALPHA_DISCREPANCY */
  double alpha;            /* FIXED: alpha > 0 */
  const double* alphas;    /* DISCREPANCY: host [n_alpha], strictly increasing, > 0 */
  int n_alpha;             /* 1 .. FR3D_MAX_ALPHAS */
  double delta;            /* DISCREPANCY: data error level, ||U - U_exact|| over all data (>= 0) */
  double tau;              /* DISCREPANCY: threshold factor (e.g. 1.1); the largest alpha with
                              residual <= tau * delta is chosen */
  int output;              /* FR3D_OUT_ZETA or FR3D_OUT_XI */
  int precision;           /* FR3D_PREC_FP32 or FR3D_PREC_FP64 */
  const fr3d_sources* sources; /* required for FR3D_OUT_XI (sources->q == Q) */
  int* alpha_idx;          /* device int[max(1, n_bands)] or NULL: index of the chosen alpha per band
                              (0 for FIXED); for GIVEN it is the input (required) */
  double* residuals;       /* device double[max(1, n_bands)][n_alpha] or NULL: squared residuals
                              ||A zeta_alpha - U||^2 restricted to each band */
  int* info;               /* device int[1] or NULL: FR3D_INFO_* bits of this call (overwritten) */
  int n_bands;             /* 0 or 1: one alpha for the whole spectrum (the paper's global rule);
                              2..FR3D_MAX_BANDS: radial bands of |k| (band b holds the frequencies with
                              b <= n_bands |k| / (sqrt(2) n/2) < b + 1), each with its own alpha; the
                              discrepancy bound of band b is tau delta sqrt(frequencies in b / n^2)
                              (white noise).  DISCREPANCY and GIVEN (any M) and LEARNED (M = 1). */
  const fr3d_mlp* net;     /* LEARNED: the network (n_in == n_out == max(1, n_bands)); NULL otherwise */
  int ra;                  /* FR3D_RA_TIKHONOV (0, default) or FR3D_RA_TSVD: alpha (or each candidate) is
                              then the truncation level relative to s^2; every alpha mode but LEARNED */
} fr3d_invert_opts;

/* Step 1 for the kernel (Algorithm 1, Sec. 5): samples K at the periodic lags for every
 * z_i - z'_j, transforms them in FP64 and builds the tables A^(m) = [nu_j K~(w^(m), z_i - z'_j)]
 * of Eq. (6), ||A^(m)||_F^2 and s^2.  Allocates the handle (free with fr3d_handle_destroy).
 * The geometry's host arrays are copied; they may be freed after the call returns.
 * pad = 2: the tables are those of the 2n x 2n box (lags wrapped at 2n, frequencies 2 pi k/(2 n h),
 * s^2 of the box), so the box's circular sums equal the aperiodic sums over the n x n grid.
 * fr3d_fwd_apply, fr3d_zeta_from_xi, fr3d_choose_alpha, fr3d_invert and fr3d_invert_host take and
 * return n x n volumes on such a handle; the residuals and the discrepancy rule are those of the
 * box (A zeta against the zero-padded data over all (2n)^2 points, the data's zeros included), and the
 * per-band rules use the box's radial bands.  fr3d_fwd_apply_noalloc, fr3d_assemble_rhs,
 * fr3d_band_features, fr3d_band_alpha_targets, the batched plan and FR3D_ALPHA_LEARNED take
 * periodic-box handles only and return FR3D_ERR_UNSUPPORTED_SIZE for pad = 2. */
int fr3d_kernel_transform(const fr3d_geometry* geom, fr3d_handle** out, void* stream);
void fr3d_handle_destroy(fr3d_handle* h);

/* Sizes and the alpha scale of a handle (any pointer may be NULL).  Synchronises the
 * handle's creation stream on the first call. */
int fr3d_handle_query(fr3d_handle* h, int* n, int* m, int* mp, double* s2);

/* The discrete operator of Eq. (4) through Eq. (5)-(6): U_q = A zeta_q for q = 0..Q-1.
 * zeta: device [Q][M'][n][n]; U: device [Q][M][n][n]; float or double per precision. */
int fr3d_fwd_apply(fr3d_handle* h, const void* zeta, int Q, void* U, int precision, void* stream);

/* fr3d_fwd_apply (FP32 only) for callers that cannot allocate device memory at the point of the
 * call: for example a real-time loop that cannot afford the allocator's latency or its implicit
 * synchronisation, or a host framework that owns all device memory through its own allocator.
 * The paper has no counterpart; this is a deployment variant.  It allocates nothing: its scratch
 * is a static 4 MiB device array that the library holds on every GPU until the process exits, so
 * the request must satisfy 8 * (M' + M) * (n/2 + 1) * n <= 4 MiB (each term rounded up to
 * 256 bytes; at n = 256, M' + M <= 15); larger requests return FR3D_ERR_UNSUPPORTED_SIZE before
 * any launch.  The current device must be the handle's (else FR3D_ERR_INVALID_ARG).  The first
 * call on a device looks up the array's device address (no allocation); make that first call
 * before any stream capture.  All calls share the one array, so calls that overlap on the GPU
 * (other streams, other threads) race and corrupt each other; serialise them.  Nothing in the
 * array needs clearing: every byte a call reads was written earlier in that call.
 * zeta: device [Q][M'][n][n] float; U: device [Q][M][n][n] float. */
int fr3d_fwd_apply_noalloc(fr3d_handle* h, const float* zeta, int Q, float* U, void* stream);

/* zeta_q = xi * V0_q (Sec. 2, zeta = xi V0) for the point sources of Sec. 6.
 * xi: device [M'][n][n]; zeta: device [Q][M'][n][n]; Q = sources->q. */
int fr3d_zeta_from_xi(fr3d_handle* h, const void* xi, const fr3d_sources* sources, void* zeta,
                      int precision, void* stream);

/* Step 2's parameter choice alone: squared residuals r^2(alpha_k) = ||A zeta_alpha_k - U||^2
 * (summed over all q and all data points) and the discrepancy choice (Sec. 4): the largest
 * alpha_k with r <= tau * delta.  U: device [Q][M][n][n].  alpha_idx: device int[1];
 * residuals: device double[n_alpha] or NULL; info: device int[1] or NULL. */
int fr3d_choose_alpha(fr3d_handle* h, const void* U, int Q, const double* alphas, int n_alpha,
                      double delta, double tau, int precision, int* alpha_idx, double* residuals,
                      int* info, void* stream);

/* Algorithm 1 steps 1-4.  U: device [Q][M][n][n]; out: device [Q][M'][n][n] (ZETA) or
 * [M'][n][n] (XI).  The regularised normal solution of each frequency's system is the
 * Tikhonov minimiser of ||A zeta - U||^2 + alpha s^2 ||zeta||^2. */
int fr3d_invert(fr3d_handle* h, const void* U, int Q, const fr3d_invert_opts* opts, void* out,
                void* stream);

/* fr3d_invert with HOST buffers U (host [Q][M][n][n]) and out (host, the shape of fr3d_invert's
 * out); returns after the stream has synchronised.  FP32 with one observation depth (M = 1): a
 * buffer that lies in one page-locked, device-mapped range (cudaHostAlloc, cudaHostRegister) and
 * starts on a 16-byte boundary is used in place: the first row pass reads U and the last kernel
 * writes out over the host link, each element once.  Otherwise (pageable or unaligned memory,
 * FP64, M > 1) U is copied to the handle's workspace and the result copied back.  Both forms
 * give the same bits as fr3d_invert. */
int fr3d_invert_host(fr3d_handle* h, const void* U_host, int Q, const fr3d_invert_opts* opts,
                     void* out_host, void* stream);

/* ---- batched inversion of independent instances of uneven size ----
 * Each instance is one call of fr3d_invert (FP32, M = 1) with its own handle (geometry), data,
 * options and output; all instances of a batch use the same output kind.  Instances must have
 * distinct handles (a handle's workspace holds one instance's spectra).  A plan groups the
 * instances by grid size n and runs Algorithm 1 with three launches per group covering all of its
 * instances (data row pass, data column pass, inverse) and one alpha-rule launch covering the
 * instances of every group (fr3d_batch_launch_count: 3 per group + 1).  fr3d_batch_create
 * builds every table and workspace and uploads the descriptors (it synchronises `stream`); the
 * device pointers and options of the instances are fixed at creation.  fr3d_batch_run only
 * launches kernels (it can be captured in a CUDA graph); with the autotuner on (mode 1, below) its
 * first call outside a capture also times the fused variants and synchronises `stream`, so make
 * that call before capturing.  The paper has no batch form: this is
 * Algorithm 1 applied to many independent problems at once. */
typedef struct fr3d_instance {
  fr3d_handle* handle;            /* geometry and kernel tables (fr3d_kernel_transform) */
  const float* U;                 /* device [Q][1][n][n] data */
  int Q;                          /* source parameters of this instance */
  const fr3d_invert_opts* opts;   /* alpha rule, sources (XI), output; precision must be FP32 */
  float* out;                     /* device [M'][n][n] (XI) or [Q][M'][n][n] (ZETA) */
} fr3d_instance;
typedef struct fr3d_batch fr3d_batch;
int fr3d_batch_create(const fr3d_instance* inst, int n, fr3d_batch** out, void* stream);
int fr3d_batch_run(fr3d_batch* b, void* stream);
int fr3d_batch_launch_count(fr3d_batch* b);
void fr3d_batch_destroy(fr3d_batch* b);
/* One-shot form in caller-provided device memory: fr3d_invert_batched_workspace validates the instances,
 * prepares every handle's tables (allocating them; synchronous) and writes the workspace bytes the run
 * needs (the data spectra of all instances and the descriptor tables); fr3d_invert_batched then runs
 * the batch in `workspace` (device, 256-byte aligned, at least that many bytes, else
 * FR3D_ERR_INVALID_ARG), allocating nothing when called with the same instances and options.  It is
 * asynchronous on `stream`; the workspace must stay untouched until the stream has synchronised.  The
 * fused inverse uses the forced tile variant (autotuner mode 2 + v) or variant 3. */
int fr3d_invert_batched_workspace(const fr3d_instance* inst, int n, size_t* bytes, void* stream);
int fr3d_invert_batched(const fr3d_instance* inst, int n, void* workspace, size_t ws_bytes, void* stream);

/* ---- learned per-band alpha (FR3D_ALPHA_LEARNED) ----
 * The paper chooses one alpha by the discrepancy principle (Sec. 4); it has no learned rule.  This
 * one replaces the alpha sweep by a small network that maps per-band statistics of the data to one
 * alpha per radial band (the bands of fr3d_invert_opts.n_bands).  Features, per band b:
 *     f_b = log10( sum over the frequencies k of b and all planes of |U~_k|^2 / (count_b delta^2) ),
 * the data power per frequency over that of white noise of total norm delta.  Network:
 *     y = W3 tanh(W2 tanh(W1 x + b1) + b2) + b3,  x = f / 4,  y_b = (log10 alpha_b + 4.5) / 3.5,
 * parameters in one vector [W1 (n_hidden x n_in, row-major), b1, W2 (n_hidden x n_hidden), b2,
 * W3 (n_out x n_hidden), b3]; the kernels use a BF16 copy of the weights with FP32 arithmetic, the
 * update keeps an FP32 master copy (Adam, beta1 0.9, beta2 0.999, eps 1e-8, loss = mean squared
 * error).  Inference (inside fr3d_invert, LEARNED) takes per band the candidate of opts.alphas nearest
 * to the predicted log10 alpha; delta must be > 0; FP32 only; residuals are not written.
 * Training targets (fr3d_band_alpha_targets): for data U made from a known zeta (fr3d_fwd_apply plus
 * noise), the candidate minimising, per band, the error sum ||zeta~_alpha - zeta~_true||^2 of the
 * Tikhonov solution (M = 1: evaluated in closed form per frequency class, no solve).  X, T, Y: device [B][n_in] / [B][n_out] float; grad: device [n_params] float;
 * loss: device float; params: HOST [n_params] float.  A network serves one stream at a time. */
int fr3d_mlp_create(int n_in, int n_hidden, int n_out, unsigned long long seed, fr3d_mlp** out);
                          /* 1 <= n_in, n_out <= FR3D_MAX_BANDS, 1 <= n_hidden <= 96; Glorot-uniform
                             weights from SplitMix64(seed), zero biases; synchronous */
void fr3d_mlp_destroy(fr3d_mlp* net);
int fr3d_mlp_query(const fr3d_mlp* net, int* n_in, int* n_hidden, int* n_out, int* n_params);
int fr3d_mlp_get_params(fr3d_mlp* net, float* params);        /* synchronous */
int fr3d_mlp_set_params(fr3d_mlp* net, const float* params);  /* synchronous; resets the Adam state */
int fr3d_mlp_forward(fr3d_mlp* net, const float* X, int B, float* Y, void* stream);
/* loss (if non-NULL) and the gradient of the loss (copied to grad if non-NULL) for one batch */
int fr3d_mlp_gradient(fr3d_mlp* net, const float* X, const float* T, int B, float* grad, float* loss,
                      void* stream);
/* gradient + one Adam step with learning rate lr */
int fr3d_mlp_train_step(fr3d_mlp* net, const float* X, const float* T, int B, float lr, float* loss,
                        void* stream);
/* the network input x_b = f_b / 4 of data U (device [Q][1][n][n] float, M = 1) into feat (device
 * float[n_bands]) */
int fr3d_band_features(fr3d_handle* h, const float* U, int Q, int n_bands, double delta, float* feat,
                       void* stream);
/* per-band error-optimal candidate for data U (device [Q][1][n][n] float, M = 1) made from the known
 * zeta_true (device [Q][M'][n][n] float): idx (device int[n_bands]); target (device float[n_bands] or
 * NULL): y_b of the chosen candidate; err (device double[n_bands][n_alpha] or NULL): the error curves
 * E_b(alpha_k) = sum over the frequencies of band b, all q and all depths of |zeta~_alpha - zeta~_true|^2
 * (unnormalised spectra) */
int fr3d_band_alpha_targets(fr3d_handle* h, const float* U, const float* zeta_true, int Q,
                            const double* alphas, int n_alpha, int n_bands, int* idx, float* target,
                            double* err, void* stream);

/* ---- autotuner of the inverse (steps 2-4, FP32, M = 1) ----
 * The inverse has variants that compute the same bits: the fused cluster kernel's tiles (variant 0: the
 * built-in table of cluster size, threads and row-batch height per n with xi accumulated in shared
 * memory; 1: xi accumulated in the output array with taller row batches where they fit; 2: xi in the
 * output array, table batches; 3: one row batch of all a CTA's rows, xi accumulated in registers and
 * written once); 4: two streaming passes through an intermediate in a handle-owned buffer; 5: one
 * persistent launch over a queue of column and row tiles through the same intermediate, served from L2
 * (n = 256 with xi output; other shapes run variant 3).  Variants 4 and 5 allocate their buffer on the
 * first call outside a stream capture (inside a capture before that, they run variant 3).  Modes: 0 = always variant 0; 1 (default) = on the first fr3d_invert of a
 * shape (device, n, M', Q, output) made outside a stream capture, time every variant on that
 * call's own arguments (1 warm-up + 3 timed launches each, synchronising the stream once) and use
 * the fastest from then on, process-wide; 2 + v = always variant v.  A batched plan (mode 1) times
 * the variants of each grid-size group on its first fr3d_batch_run outside a capture and keeps the
 * fastest per group (that run's outputs are complete and identical).  The paper has no counterpart
 * (it fixes no tiling).
 * fr3d_autotune_mode(-1) returns the mode; otherwise it sets it and returns the previous one. */
int fr3d_autotune_mode(int mode);
/* The variant that the handle's last fused inverse used, and (ms, up to cap entries) the per-launch
 * times the tuner measured on this handle (0 if it did not tune here).  Returns the variant count. */
int fr3d_autotune_query(fr3d_handle* h, int* variant, float* ms, int cap);
/* Test hook of variant 5's bounded waits: while on != 0, its column tiles withhold the counts that release
 * the intermediate to the row tiles, so the row tiles' waits run out (after about a second): the call
 * still returns, with FR3D_INFO_TIMEOUT set in the info word, and its xi is not valid.  No fault and no
 * hang is involved; the next call with the hook off is exact again.  Returns the previous setting. */
int fr3d_test_withhold_queue_counts(int on);

/* ---- learned post-corrector: a 3D U-Net on the tensor cores (fr3d_unet) ----
 * The paper has no network.  This one post-corrects the reconstruction of fr3d_invert: with one observation
 * plane each frequency's system has rank one, so the regularised normal solution (Assumption U, Sec. 4)
 * keeps one depth direction per frequency, and a network trained on examples from the same forward
 * operator restores the others.  Architecture (4 levels, widths 16, 32, 64, 128; 1 902 081 parameters):
 * level 0 conv(1 -> 16), conv(16 -> 16); levels 1, 2: 2x average pooling, conv(w_{l-1} -> w_l), conv(w_l -> w_l);
 * level 3: pooling and three conv to 128; going up, 2x nearest upsampling concatenated (channels first)
 * with the encoder output of the level, conv(w_{l+1} + w_l -> w_l), conv(w_l -> w_l); every conv 3 x 3 x 3 with
 * zero padding, bias and leaky ReLU (slope 0.01); a 1 x 1 x 1 head 16 -> 1 added to the input:
 *     y = x + head(...),   with x = in_scale * xi_in and the prediction y / in_scale.
 * Loss: the batch mean of ||y - t||^2 / ||t||^2 (the squared relative L2 error).  Convolutions and their
 * gradients run on the tensor cores with BF16 weights and activations and FP32 accumulation; the update is
 * Adam (beta1 0.9, beta2 0.999, eps 1e-8) on FP32 master parameters.  Parameters in one flat vector, per
 * conv layer in the order above w [co][ci][3][3][3] then b [co], then the head w [16] and b [1].
 * Volumes: device FP32 [B][depth][height][width] (x fastest); depth, height and width multiples of 8
 * (three poolings), depth <= 256, height, width <= 512; 1 <= B <= max_batch.  The network owns its
 * activation buffers for max_batch samples (about 330 MB per sample at 32 x 128 x 128); one network serves
 * one stream at a time.  A bounded device wait that gives up sets FR3D_INFO_TIMEOUT in the flags
 * fr3d_unet_error_flags reads (synchronous). */
typedef struct fr3d_unet fr3d_unet;
int fr3d_unet_create(int depth, int height, int width, int max_batch, float in_scale, unsigned long long seed,
                     fr3d_unet** out);   /* He-normal conv weights from SplitMix64(seed), zero biases and head
                                            (the initial network is the identity); synchronous */
void fr3d_unet_destroy(fr3d_unet* net);
int fr3d_unet_query(const fr3d_unet* net, int* n_params);
int fr3d_unet_get_params(fr3d_unet* net, float* params);        /* host [n_params]; synchronous */
int fr3d_unet_set_params(fr3d_unet* net, const float* params);  /* host [n_params]; resets Adam; synchronous */
/* y: device [B][depth][height][width], the corrected volume (caller's units) */
int fr3d_unet_forward(fr3d_unet* net, const float* x, int B, float* y, void* stream);
/* loss (device float, or NULL) and gradient (device float[n_params], or NULL) for inputs x and targets t */
int fr3d_unet_gradient(fr3d_unet* net, const float* x, const float* t, int B, float* grad, float* loss,
                       void* stream);
/* gradient + one Adam step with learning rate lr */
int fr3d_unet_train_step(fr3d_unet* net, const float* x, const float* t, int B, float lr, float* loss,
                         void* stream);
int fr3d_unet_error_flags(fr3d_unet* net, int* flags);

/* Right-hand side of Eq. (7) (the form Eq. (3) takes for point sources, Sec. 6) from the measured
 * z-derivative of V2 on the observation depths:
 *     U_q = 2 pi dV2/dx3 + (A2 / 2) sum_l d/dx3 (1/|x - x_{q,l}|)
 *           - A0 / (4 pi c0^2) sum_l integral over Pi of d/dx3 (1/|x - x'|) / |x' - x_{q,l}| dx',
 * R^3 replaced by the box Pi (Sec. 5): horizontally the handle's periodic grid, vertically a midpoint
 * grid of n_pi (even) depths on [-pi_half, pi_half]; the integral is the discrete operator of Eq. (4)
 * on that depth grid (the paper simulates its data this way, Sec. 6).  A0 = sources->A0; A2 =
 * integral of t^2 g(t) dt (Sec. 2); c0 the background speed.  dV2dz and U: device [Q][M][n][n] float
 * (U may be dV2dz).  The first call for a (n_pi, pi_half) pair builds the kernel tables of Pi's
 * geometry (synchronous, allocates); an observation depth on Pi's depth grid is BAD_GEOMETRY, and so
 * is a source point on a node of Pi's grid. */
int fr3d_assemble_rhs(fr3d_handle* h, const float* dV2dz, int Q, const fr3d_sources* sources, double A2,
                      double c0, int n_pi, double pi_half, float* U, void* stream);

/* Number of kernel launches the last call on this handle enqueued (cache rebuilds excluded). */
int fr3d_last_launch_count(fr3d_handle* h);

/* Stage tracing.  When enabled, fr3d_invert records a CUDA event on its stream before its first
 * launch and after every launch.  fr3d_profile_read waits for the last event of the latest call
 * and writes, per launch interval i < min(cap, count), its stage kind and its duration in ms;
 * it returns the count.  Kinds: 0 data row pass, 1 data column pass, 2 alpha rule, 3 solve +
 * inverse column pass, 4 inverse row pass (+ xi), 5 table rebuild, 6 forward contraction,
 * 7 inverse column pass, 8 other, 9 fused solve + inverse DFT + combination. */
int fr3d_profile_enable(fr3d_handle* h, int enable);
int fr3d_profile_read(fr3d_handle* h, int* kinds, float* ms, int cap);

const char* fr3d_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* FR3D_H */
