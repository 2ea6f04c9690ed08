/*
 * cofem.h -- C ABI of libcofem, a GB300 (sm_103a) implementation of
 * covariance-free EM (CoFEM) for sparse Bayesian learning.
 *
 * Method (Lin, Song, Bilgic, Ba, "High-Dimensional Sparse Bayesian Learning
 * without Covariance Matrices"):
 *   model      z ~ N(0, diag(alpha)^-1), y ~ N(Phi z, beta^-1 I)      Sec. 2.1
 *   E-step     solve A X = B with A = beta Phi^T Phi + diag(alpha) and
 *              B = [beta Phi^T y | p_1 .. p_K] (K Rademacher probes)  Eq. (mat-eq)
 *              by conjugate gradients, one recurrence per column     Sec. 3.2
 *   estimate   s = (1/K) sum_k p_k . x_k                              Eq. (diag-estimate)
 *   M-step     alpha = 1 / (mu . mu + s)                              Eq. (mstep), Alg. 1
 *
 * Conventions for every entry point:
 *  - All array arguments named *_dev are DEVICE pointers owned by the caller;
 *    the library never frees them and keeps none of them past the call,
 *    except that an operator handle keeps the dictionary pointers it was
 *    created with (the caller keeps that memory alive while the handle lives).
 *  - Work is enqueued on the caller's CUDA stream (`stream`, a cudaStream_t
 *    passed as void*; NULL = legacy default stream).  Entry points that say
 *    "synchronous" wait for the stream before returning.
 *  - Multi-column vectors ("blocks") are column-major: column j of a block
 *    with leading dimension ld starts at element j*ld.  ld >= the column
 *    length and ld must be a multiple of 64.  Column 0 is the mean system
 *    (right-hand side beta Phi^T y, solution mu); columns 1..K are probes.
 *    The paper lists mu last; the order changes no result.
 *  - Vector precision is COFEM_F64 (double) or COFEM_F32 (float).  CG scalars
 *    (dot products, step sizes) are always double.  mu, s and alpha outputs
 *    are always double.
 *  - Errors are returned as cofem_status; nothing aborts.  Device-side faults
 *    of the method (non-finite values, CG breakdown) are recorded in an error
 *    word in the workspace and returned by the synchronous calls.  When a call
 *    fails its outputs are unspecified.
 */
#ifndef COFEM_H
#define COFEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  COFEM_OK = 0,
  COFEM_ERR_INVALID_ARG = 1,   /* bad size, null pointer, misaligned ld ... */
  COFEM_ERR_CUDA = 2,          /* a CUDA runtime call failed */
  COFEM_ERR_NONFINITE = 3,     /* NaN/Inf met in mu, s or a CG scalar */
  COFEM_ERR_BREAKDOWN = 4,     /* CG curvature p^T A p <= 0 */
  COFEM_ERR_TIMEOUT = 5,       /* a bounded device wait ran out */
  COFEM_ERR_UNSUPPORTED = 6,   /* combination not built (e.g. dtype/op) */
  COFEM_ERR_WORKSPACE = 7      /* workspace smaller than cofem_workspace_bytes */
} cofem_status;

typedef enum {
  COFEM_F64 = 0,
  COFEM_F32 = 1,
  COFEM_BF16 = 2,
  COFEM_FP8_E4M3 = 3
} cofem_dtype;

/* Human-readable name of a status code (static string). */
const char* cofem_status_string(cofem_status s);

/* Text of the last CUDA failure seen by this thread (call, error, source
 * line); empty if none.  Valid until the next failing call on the thread. */
const char* cofem_last_error(void);

/* ------------------------------------------------------------------------
 * Dictionary operators (Sec. 3.2: CG only needs Phi and Phi^T applied to
 * vectors; tau_D is the cost of one application).
 * ------------------------------------------------------------------------ */
typedef struct cofem_op cofem_op;

/* Dense Phi, N x D, row-major with leading dimension ld (elements, >= D,
 * multiple of 64 for BF16/FP8, of 4 for F32/F64).  phi_dev is 256-byte
 * aligned.  dtype F64 (only with F64 vectors), F32, BF16 or FP8_E4M3 (F32
 * vectors).  For FP8 each entry is one E4M3 byte q, standing for
 * phi = q x scale of its 128 x 128 tile; tile_scales_dev holds ceil(N/128)
 * x ceil(D/128) float scales (row-major), NULL for the other dtypes.  Every
 * product of an FP8 handle applies bf16(q x scale) (the FP8 value is exact
 * in FP32; the product is rounded to FP32, then to BF16, to nearest even):
 * the CG operator on the tensor cores, which needs a packed copy attached
 * (cofem_op_dense_attach_packed; without one an FP8 fit returns
 * COFEM_ERR_UNSUPPORTED), and beta Phi^T y, forward, adjoint and column norms
 * on the CUDA cores.  Writes a new handle to *out. */
cofem_status cofem_op_dense(int64_t N, int64_t D, cofem_dtype dtype,
                            const void* phi_dev, int64_t ld,
                            const float* tile_scales_dev, cofem_op** out);

/* BF16 and FP32 dictionaries: how the FP32 vectors meet Phi on the tensor
 * cores.  nterms 1..3: on the tensor cores (tcgen05), each FP32 vector is
 * split into nterms BF16 terms (x = x1 + x2 [+ x3], each term the BF16
 * rounding of the remainder), all products accumulate in FP32; 3 terms carry
 * the full 24-bit FP32 mantissa, 2 terms 16 bits.  nterms 0: CUDA cores.
 * Default 3 for BF16; an FP32 dictionary runs on the CUDA cores until a
 * packed copy is attached (cofem_op_dense_attach_packed), which sets 3 if
 * nterms was 0. */
cofem_status cofem_op_dense_set_terms(cofem_op* op, int32_t nterms);

/* Tensor-core pipeline shape of a BF16 dictionary's operator: shared-memory
 * ring depth (stages, 2..8; 0 = as deep as fits) and resident CTAs per SM
 * (1..4; 0 = 2).  Set explicitly, or let cofem_op_dense_autotune pick it.
 * Workspace sizes (cofem_workspace_bytes, cofem_apply_workspace_bytes)
 * depend on it: query them after choosing the shape. */
cofem_status cofem_op_dense_set_pipeline(cofem_op* op, int32_t stages, int32_t ctas_per_sm);

/* Output rows of one tensor-core work unit: 128 (default) or 256.  With 256
 * a CTA computes two 128-row output tiles from every B-operand stage it
 * loads (one tensor-memory accumulator each), halving the B-operand traffic
 * per byte of Phi; its accumulators then take all of an SM's tensor memory
 * when BN > 64, so one CTA runs per SM.  cofem_op_dense_autotune tries both.
 * Workspace sizes depend on it (query them after choosing). */
cofem_status cofem_op_dense_set_tile_rows(cofem_op* op, int32_t rows);

/* The tensor-core pipeline shape set on a dense handle (any pointer may be
 * NULL): stages (0 = as deep as fits), CTAs per SM (0 = 2), tile rows. */
cofem_status cofem_op_dense_get_pipeline(const cofem_op* op, int32_t* stages,
                                         int32_t* ctas_per_sm, int32_t* tile_rows);

/* Autotuner: times one operator application (ncols FP32 columns of made-up
 * data, 2 warm-up + 5 timed runs, CUDA events on `stream`) for every
 * pipeline shape that fits (stages, CTAs per SM, 128 or 256 tile rows),
 * keeps the fastest on the handle and returns it
 * (any output pointer may be NULL; best_us = mean microseconds per
 * application).  workspace_dev: >= cofem_op_dense_autotune_workspace_bytes,
 * 256-byte aligned.  Synchronous.  BF16 dictionaries on tensor cores only. */
size_t cofem_op_dense_autotune_workspace_bytes(const cofem_op* op, int32_t ncols);
cofem_status cofem_op_dense_autotune(cofem_op* op, int32_t ncols, void* workspace_dev,
                                     size_t workspace_bytes, void* stream,
                                     int32_t* best_stages, int32_t* best_ctas_per_sm,
                                     float* best_us);

/* BF16 dictionaries: a tile-major copy of Phi for the tensor-core operator.
 * cofem_dense_packed_bytes gives its size: ceil(N/128) * ceil(D/64) tiles of
 * 128 x 64 values (16 KB) each, a tile's rows 64 values long and contiguous,
 * tiles ordered by column block fastest, zero padded at the edges.
 * cofem_op_dense_attach_packed fills packed_dev (caller-owned, 256-byte
 * aligned, >= that size) from the handle's row-major Phi on `stream` and
 * makes operator applications read it: each tensor-memory load is then one
 * contiguous range of DRAM.  The row-major Phi stays in use for
 * cofem_op_forward/adjoint and for beta Phi^T y.  packed_dev = NULL
 * detaches.  Both buffers must outlive the handle's use. */
size_t cofem_dense_packed_bytes(int64_t N, int64_t D);
cofem_status cofem_op_dense_attach_packed(cofem_op* op, void* packed_dev,
                                          size_t packed_bytes, void* stream);

/* FP32 dictionaries on the tensor cores (Sec. 3.2's operator at FP32-class
 * precision, 4 bytes per entry like FP32 storage): the packed copy holds two
 * images of the layout above, 2 * cofem_dense_packed_bytes(N, D) bytes, the
 * first with hi = bf16(phi), the second with lo = bf16(phi - hi) (rounding to
 * nearest even), so every entry is applied as hi + lo: 16 significant bits,
 * a relative error of at most 2^-17 per entry.  Attaching it
 * (cofem_op_dense_attach_packed, same rules) moves the operator
 * applications of cofem_fit and cofem_op_apply to the tensor cores, both
 * terms accumulating into the same FP32 accumulator, and makes every other
 * product of the handle (beta Phi^T y in cofem_fit, cofem_op_forward,
 * cofem_op_adjoint, cofem_op_col_norms) use hi + lo too, so that the fit
 * solves one consistent system; detaching (NULL) returns all of them to
 * the FP32 entries on the CUDA cores.  cofem_op_dense_packed_bytes gives the
 * size the attach call needs for any dense operator (one image for BF16,
 * two for FP32, half an image -- one byte per entry -- for FP8, 0 for other
 * kinds). */
size_t cofem_op_dense_packed_bytes(const cofem_op* op);

/* FP8 E4M3 quantisation of an FP32 dictionary (phi_dev: N x D, leading
 * dimension ld) into one byte per entry (out_dev, leading dimension ld_out)
 * with a scale per 128 x 128 tile (scales_dev, ceil(N/128) x ceil(D/128)):
 * the tile's scale is the smallest power of two s with max |phi| / s <= 448
 * (1 for an all-zero tile), each byte e4m3(phi / s) rounded to nearest even
 * with saturation.  Power-of-two scales make q x s exact, so an FP8 handle
 * applies bf16(q x s) = the BF16 rounding of the quantised entry.
 * Asynchronous. */
cofem_status cofem_quantize_fp8_tiles(const float* phi_dev, int64_t N, int64_t D, int64_t ld,
                                      void* out_dev, int64_t ld_out, float* scales_dev,
                                      void* stream);

/* BF16 dictionaries on the tensor cores: bytes of Phi (a band of its first
 * columns) to keep resident in L2 across the two products of every operator
 * application, by loading that band with an evict-last and the rest with an
 * evict-first cache policy.  -1 = 60% of the device's L2; 0 (the default)
 * = stream all of Phi, which measured faster on GB300. */
cofem_status cofem_op_dense_set_l2_resident(cofem_op* op, int64_t bytes);

/* Circular convolutional Phi (Sec. 3.2 structured tau_D): signal length L,
 * C filters of T taps (filters_dev: C x T floats, row-major).  N = L,
 * D = C*L, coordinate d = c*L + m.
 *   (Phi z)[n]     = sum_c sum_j h[c][j] z_c[(n - j) mod L]
 *   (Phi^T w)_c[m] = sum_j h[c][j] w[(m + j) mod L]
 * L must be a multiple of 64 and at most 2^22; T <= 64; filters_dev
 * 4-byte aligned.  F32 vectors only. */
cofem_status cofem_op_conv1d(int64_t L, int32_t C, int32_t T,
                             const float* filters_dev, cofem_op** out);

/* on = 1: apply the convolutional Phi on the tensor cores with its filters
 * rounded to BF16 (the dictionary becomes the BF16 rounding of h, as a BF16
 * dense dictionary is; every entry point that uses Phi -- the operator, its
 * two products, the fits, the column norms -- then uses the rounded taps).
 * The products run as block Toeplitz GEMMs (tcgen05): blocks of 64 outputs,
 * the FP32 vectors as three BF16 terms (exact FP32 products), FP32
 * accumulation.  on = 0: FP32 filters on the CUDA cores (the default).
 * COFEM_ERR_INVALID_ARG for other operators.  Workspace sizes depend on it:
 * query them after choosing. */
cofem_status cofem_op_conv1d_set_tensor_cores(cofem_op* op, int32_t on);

/* Masked-DCT Phi (the structured dictionary of Sec. 4.2): Phi = M C^T, with C
 * the orthonormal DCT-II matrix of size D (C[k][n] = s_k cos(pi k (2n+1) /
 * 2D), s_0 = sqrt(1/D), s_k = sqrt(2/D)) and M the selection of the N
 * samples idx_dev[0..N-1] of its inverse:
 *   (Phi z)_i  = (C^T z)[idx[i]],     Phi^T w = C (w scattered to idx).
 * D a power of two, 16 <= D <= 2^22; 1 <= N <= D; idx_dev: N int32 device
 * values, strictly increasing in [0, D), owned by the caller and read at
 * every application (a violation is reported as COFEM_ERR_INVALID_ARG by
 * the fit, through the device error word).  F32 vectors only.  With a
 * learned warm start the fit computes ||phi_d||^2 from one DCT of the sample
 * mask (the closed form under cofem_op_col_norms_ws). */
cofem_status cofem_op_dct(int64_t D, int64_t N, const int32_t* idx_dev, cofem_op** out);

/* Releases a handle (NULL is ignored). */
void cofem_op_destroy(cofem_op* op);

/* N and D of an operator. */
cofem_status cofem_op_shape(const cofem_op* op, int64_t* N, int64_t* D);

/* ------------------------------------------------------------------------
 * Fit parameters (Algorithm 1 inputs y, Phi, beta, T_em, K; the solver
 * limits U and eps of Sec. 3.2).
 * ------------------------------------------------------------------------ */
typedef struct {
  int32_t K;                   /* probes per E-step, 1..64 */
  int32_t em_iters;            /* T_em */
  int32_t cg_max_iters;        /* U */
  int32_t fixed_cg_iters;      /* >0: run exactly this many CG iterations,
                                  ignoring cg_tol (parity mode); 0 = off */
  int32_t resid_replace_every; /* R > 0: every R CG iterations recompute the
                                  true residual r = B - A x; 0 = never */
  int32_t vec_dtype;           /* COFEM_F64 or COFEM_F32 */
  int32_t stop_rule;           /* 0: joint test ||R||_F / ||B||_F < cg_tol on
                                  the recursive residual (Sec. 3.2, the
                                  paper's); 1: per column -- column j is
                                  frozen (a_j = b_j = 0 from then on) once
                                  ||r_j|| / ||b_j|| < cg_tol, the solve ends
                                  when every column is frozen.  Ignored with
                                  fixed_cg_iters; 1 with mlp returns
                                  COFEM_ERR_UNSUPPORTED.  Other values:
                                  COFEM_ERR_INVALID_ARG. */
  int32_t tasks;               /* T >= 1 (0 = 1): tasks sharing alpha, the
                                  multi-task extension named in Sec. 5.
                                  cofem_fit then reads y_dev as T vectors of
                                  N (task t at y_dev + t N), solves for
                                  B = [beta Phi^T y_1 .. beta Phi^T y_T |
                                  p_1 .. p_K] (K + T <= 64 columns), writes
                                  mu_dev as T x D (task t at mu_dev + t D)
                                  and updates alpha_d = 1 / max(mean_t
                                  mu_td^2 + s_d, den_floor).  Not with mlp
                                  or cofem_fit_batched
                                  (COFEM_ERR_UNSUPPORTED). */
  double cg_tol;               /* eps: stop when ||R||_F / ||B||_F < eps */
  double alpha_init;           /* initial alpha (Alg. 1: 1) when
                                  t_offset == 0; ignored otherwise */
  double den_floor;            /* alpha = 1 / max(mu^2 + s, den_floor) */
  double support_threshold;    /* stats: support = #{alpha_d < threshold} */
  uint64_t seed;               /* probe seed */
  int64_t t_offset;            /* EM iterations already done: t runs
                                  t_offset+1 .. t_offset+em_iters; when > 0
                                  alpha_dev is read as the starting alpha */
  const void* mlp;             /* learned warm start / preconditioner (not in
                                  the paper): device pointer to the 1282 BF16
                                  weights of cofem_mlp_*, or NULL for plain CG.
                                  From the fit's second E-step on, each solve
                                  starts from X0 = [mu_hat | s_hat . p_k] with
                                  M^-1 = diag(s_hat) (preconditioned CG, same
                                  stop test); if it has not converged after
                                  cg_max_iters, plain CG from zero is run
                                  instead.  F32 vectors only. */
  int32_t solver;              /* E-step solver: 0 = the paper's column-wise
                                  CG (Sec. 3.2); 1 = block CG, a solver
                                  variant: the K + T columns share one block
                                  Krylov space (O'Leary 1980) in the
                                  residual-orthonormalised form R = Q C of
                                  Dubrulle (2001), same joint stop test
                                  ||R||_F / ||B||_F = ||C||_F / ||B||_F <
                                  cg_tol.  A direction of the residual block
                                  that becomes dependent (a zero y, a
                                  converged column combination) is dropped
                                  from the solve.  With resid_replace_every
                                  > 0, stop_rule 1, mlp or cofem_fit_batched:
                                  COFEM_ERR_UNSUPPORTED.  Other values:
                                  COFEM_ERR_INVALID_ARG. */
} cofem_params;

/* Fills *p with: K 20, em_iters 50, cg_max_iters 400, fixed 0, R 0, F32,
 * cg_tol 1e-6, alpha_init 1, den_floor 1e-12, support_threshold 1e6,
 * seed 0, t_offset 0, mlp NULL, solver 0. */
void cofem_params_default(cofem_params* p);

/* Per-EM-iteration statistics, host arrays of length em_iters (any may be
 * NULL): CG iterations, final recursive relative residual ||R||_F/||B||_F,
 * number of clamped denominators, support size, and (cofem_fit only; the
 * batched fit leaves it untouched) the device clock at the end of each EM
 * iteration's M-step in nanoseconds, counted from the fit's first kernel on
 * the device (%globaltimer, so host-side set-up between kernels counts). */
typedef struct {
  int32_t* cg_iters;
  double* relres;
  int32_t* clamps;
  int32_t* support;
  int64_t* end_ns;
} cofem_stats;

/* Learned path: number of fallbacks to plain CG in the last cofem_fit on
 * this thread (0 without a learned warm start). */
int32_t cofem_last_fit_fallbacks(void);

/* Bytes of device workspace cofem_fit needs for this operator and params
 * (256-byte aligned base required). */
cofem_status cofem_workspace_bytes(const cofem_op* op, const cofem_params* p,
                                   size_t* bytes);

/* Algorithm 1 (CovarianceFreeEM): b = beta Phi^T y once, then em_iters times
 * { draw probes, solve A X = B by column-wise CG, s = (1/K) sum p_k . x_k,
 *   alpha = 1 / max(mu^2 + s, den_floor) }.
 * y_dev: N values of vec_dtype (T x N with params.tasks = T > 1).  mu_dev:
 * D doubles (T x D with T tasks); s_dev, alpha_dev: D doubles each
 * (alpha_dev is also the input alpha when t_offset > 0).  stats: optional.
 * Synchronous: returns after the work on `stream` has finished, with the
 * device error word checked. */
cofem_status cofem_fit(const cofem_op* op, const void* y_dev, double beta,
                       const cofem_params* p, void* workspace_dev,
                       size_t workspace_bytes, double* mu_dev, double* s_dev,
                       double* alpha_dev, cofem_stats* stats, void* stream);

/* ------------------------------------------------------------------------
 * Many independent problems in one fit (each its own Algorithm 1).
 * ------------------------------------------------------------------------ */
typedef struct {
  int64_t N, D;          /* dictionary shape */
  const void* phi_dev;   /* BF16, N x D row-major, leading dimension ld (multiple
                            of 64), 256-byte aligned */
  int64_t ld;
  const void* y_dev;     /* N floats */
  double beta;           /* noise precision */
  uint64_t seed;         /* this problem's probe seed */
} cofem_problem;

/* Workspace of cofem_fit_batched: about the packed dictionaries (2 N D
 * bytes each) plus 4 (K+1) D floats of CG state per problem. */
cofem_status cofem_batched_workspace_bytes(int32_t n, const cofem_problem* problems,
                                           const cofem_params* p, size_t* bytes);

/* Algorithm 1 for n problems at once: every problem keeps its own
 * column-wise CG (own step sizes, own stop test ||R||_F/||B||_F < cg_tol,
 * own probes from its seed), the problems sharing each kernel launch; a
 * problem whose CG has stopped costs nothing until the next EM iteration.
 * FP32 vectors (p->vec_dtype must be COFEM_F32), BF16 dictionaries on the
 * tensor cores (3-term split); no residual replacement (must be 0).
 * p->mlp (the learned warm start, see cofem_params) runs per problem as in
 * cofem_fit: from the fit's second E-step on every problem starts from its
 * own X0 = [mu_hat | s_hat . p_k] with M^-1 = diag(s_hat), and a problem
 * whose preconditioned solve misses cg_tol within cg_max_iters is rerun as
 * plain CG from zero (its E-step counting both solves; the total over all
 * problems is cofem_last_fit_fallbacks); not with stop_rule 1
 * (COFEM_ERR_UNSUPPORTED).
 * mu_dev, s_dev, alpha_dev: sum_i D_i doubles each, problem i at offset
 * sum_{k<i} D_k (alpha_dev is read as the starting alpha when
 * t_offset > 0).  stats (optional): host arrays of n * em_iters values,
 * problem-major.  Synchronous. */
cofem_status cofem_fit_batched(int32_t n, const cofem_problem* problems,
                               const cofem_params* p, void* workspace_dev,
                               size_t workspace_bytes, double* mu_dev, double* s_dev,
                               double* alpha_dev, cofem_stats* stats, void* stream);

/* ------------------------------------------------------------------------
 * Learned warm start / preconditioner (not in the paper; plain CG stays the
 * fallback).  A per-coordinate MLP 4 -> 32 -> 32 -> 2 with tanh, 1282
 * parameters laid out W1 (32x4, row-major) | b1 (32) | W2 (32x32) | b2 (32)
 * | W3 (2x32) | b3 (2).  With c_d = beta ||phi_d||^2 + alpha_d its input is
 *   u = [ln alpha_d / 10, ln(beta ||phi_d||^2) / 10,
 *        asinh(mu_prev_d sqrt(c_d)) / 4, ln(max(s_prev_d c_d, 1e-6)) / 4]
 * and its output o gives mu_hat_d = sinh(4 o1) / sqrt(c_d) and
 * s_hat_d = exp(4 o2) / c_d; training targets are the same transforms of an
 * E-step's mu and s.  Training minimises the mean of 1/2 ||o - y||^2 with
 * Adam (beta1 0.9, beta2 0.999, eps 1e-8) on FP32 master weights; the
 * forward pass and inference use BF16 weights with FP32 arithmetic.
 * ------------------------------------------------------------------------ */

/* ||phi_d||^2 for every coordinate (D floats): dense and convolutional
 * dictionaries (the masked DCT's needs a workspace: COFEM_ERR_UNSUPPORTED
 * here, use cofem_op_col_norms_ws).  Asynchronous. */
cofem_status cofem_op_col_norms(const cofem_op* op, float* out_dev, void* stream);

/* The same for every operator kind, with a caller-owned device workspace of
 * at least cofem_col_norms_workspace_bytes(op) bytes, 256-byte aligned (0
 * bytes, and workspace_dev may be NULL, for dense and convolutional
 * dictionaries).  For the masked DCT (Phi = C^T[idx, :], C the orthonormal
 * DCT-II) cos^2 t = (1 + cos 2t) / 2 gives
 *   ||phi_d||^2 = (s_d^2 / 2) (N + T_d),  T_d = sum over kept n of
 *   cos(pi 2d (2n + 1) / 2D),
 * and T_d is read off X = C m, the DCT of the 0/1 sample mask m: X_{2d} /
 * s_{2d} for 2d < D, 0 for 2d = D, -X_{2D-2d} / s_{2D-2d} for 2d > D (one
 * FP32 transform: the transform's error, near log2(D) 2^-24 sqrt(N) in T_d,
 * is relative error log2(D) 2^-24 / sqrt(N) in ||phi_d||^2).
 * COFEM_ERR_WORKSPACE when workspace_bytes is too small.  Asynchronous. */
cofem_status cofem_col_norms_workspace_bytes(const cofem_op* op, size_t* bytes);
cofem_status cofem_op_col_norms_ws(const cofem_op* op, float* out_dev, void* workspace_dev,
                                   size_t workspace_bytes, void* stream);

/* Features u (D x 4 floats, row-major) from alpha, ||phi_d||^2, beta and the
 * previous E-step's mu, s (NULL: mu_prev = 0, s_prev = 1/c_d).  Async. */
cofem_status cofem_mlp_features(const double* alpha_dev, const float* phinorm2_dev,
                                double beta, const double* mu_prev_dev,
                                const double* s_prev_dev, int64_t D, float* U_dev,
                                void* stream);

/* Targets y (D x 2 floats) from an E-step's mu and s.  Asynchronous. */
cofem_status cofem_mlp_targets(const double* alpha_dev, const float* phinorm2_dev,
                               double beta, const double* mu_dev, const double* s_dev,
                               int64_t D, float* Y_dev, void* stream);

/* o = MLP(u) for n samples (U: n x 4, O: n x 2 floats); weights F32 or BF16.
 * Asynchronous. */
cofem_status cofem_mlp_forward(const void* weights_dev, cofem_dtype wdtype,
                               const float* U_dev, int64_t n, float* O_dev, void* stream);

/* Scratch of cofem_mlp_grad / cofem_mlp_adam_step for n samples. */
size_t cofem_mlp_train_workspace_bytes(int64_t n);

/* Gradient (1282 floats, parameter layout above) and loss (double) of the
 * mean loss over n samples, weights F32 or BF16.  Deterministic (fixed
 * reduction order).  Asynchronous. */
cofem_status cofem_mlp_grad(const void* weights_dev, cofem_dtype wdtype, const float* U_dev,
                            const float* Y_dev, int64_t n, float* grad_dev, double* loss_dev,
                            void* workspace_dev, size_t workspace_bytes, void* stream);

/* One Adam step on the n samples: forward/backward with the BF16 weights,
 * update of the FP32 master weights and moments (m, v), new BF16 copy.
 * step is 1-based; loss_dev (optional) receives the loss before the step.
 * Asynchronous. */
cofem_status cofem_mlp_adam_step(float* master_dev, float* m_dev, float* v_dev,
                                 void* weights_bf16_dev, const float* U_dev,
                                 const float* Y_dev, int64_t n, int32_t step, float lr,
                                 void* workspace_dev, size_t workspace_bytes,
                                 double* loss_dev, void* stream);

/* ------------------------------------------------------------------------
 * Individual hot-path steps (each is one of the kernels cofem_fit runs).
 * ------------------------------------------------------------------------ */

/* Probe block for EM iteration t (Sec. 3.1 Rademacher probes, Alg. 1
 * "draw p_1..p_K"): out[k*ld + d] = p_{k+1, d} in {+1, -1}, d < D, k < K,
 * from the counter-based hash
 *   s1 = mix64(mix64(seed) ^ t);  h = mix64(s1 ^ ((d << 8) | (k / 64)));
 *   p = (bit (k mod 64) of h) ? -1 : +1
 * with mix64 the SplitMix64 output function.  K <= 16384.  dtype F64/F32.
 * Asynchronous. */
cofem_status cofem_probe_fill(uint64_t seed, int64_t t, int32_t K, int64_t D,
                              cofem_dtype dtype, void* out_dev, int64_t ld,
                              void* stream);

/* Operator application Y = beta Phi^T (Phi X) + alpha . X over ncols
 * columns (the product A X of Eq. (mat-eq)).  X, Y: blocks of vec dtype
 * with leading dimension ld (>= D); entries d >= D of X must be zero, those
 * of Y are unspecified.  alpha_dev: D doubles.  workspace: at least
 * cofem_apply_workspace_bytes(op, vec, ncols), 256-byte aligned.
 * ncols <= 64.  Asynchronous. */
cofem_status cofem_apply_workspace_bytes(const cofem_op* op, cofem_dtype vec,
                                         int32_t ncols, size_t* bytes);
cofem_status cofem_op_apply(const cofem_op* op, cofem_dtype vec,
                            const void* x_dev, int64_t ld, int32_t ncols,
                            const double* alpha_dev, double beta, void* y_dev,
                            void* workspace_dev, size_t workspace_bytes,
                            void* stream);

/* cofem_op_apply with per-kernel timing (diagnostics): CUDA events recorded
 * on `stream` before the application and after each of its kernels; on
 * return kernel_ms[i] (i < *n_kernels <= max_kernels <= 16) holds the
 * elapsed milliseconds of the i-th kernel in launch order (tensor cores:
 * split, first product, reduce/split, second product).  Synchronous. */
cofem_status cofem_op_apply_timed(const cofem_op* op, cofem_dtype vec, const void* x_dev,
                                  int64_t ld, int32_t ncols, const double* alpha_dev,
                                  double beta, void* y_dev, void* workspace_dev,
                                  size_t workspace_bytes, void* stream, float* kernel_ms,
                                  int32_t max_kernels, int32_t* n_kernels);

/* cofem_op_apply without a workspace argument, for callers that may not
 * allocate device memory (for example a plugin inside an application that
 * owns the whole device memory pool, or a loop that must not synchronise on
 * an allocation).  The paper has no counterpart: this is a service of the
 * library, not a step of the method.  Scratch comes from a static device
 * array of cofem_noalloc_scratch_capacity() bytes (16 MiB) compiled into
 * the library; every GPU that loads the library holds it until exit.  A
 * problem whose scratch would exceed it returns COFEM_ERR_WORKSPACE (see
 * cofem_last_error for the sizes).  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) and must come before any
 * stream capture; the address is then kept for the life of the process, so
 * after a cudaDeviceReset of that device this entry point must not be called
 * again in the same process.  All calls share the array: calls whose GPU work overlaps
 * race and give wrong results; order them on one stream.  Same arguments and
 * results as cofem_op_apply.  Asynchronous. */
cofem_status cofem_op_apply_noalloc(const cofem_op* op, cofem_dtype vec,
                                    const void* x_dev, int64_t ld, int32_t ncols,
                                    const double* alpha_dev, double beta,
                                    void* y_dev, void* stream);
size_t cofem_noalloc_scratch_capacity(void);

/* Self-test of the bounded device waits (the paper has no counterpart).
 * Every tensor-core kernel gives up a wait on a shared-memory mbarrier after
 * a time limit, records COFEM_ERR_TIMEOUT in the device error word, frees
 * its tensor memory and exits, so that the context stays usable.  This call
 * runs the same wait routine in one CTA on an mbarrier that nothing arrives
 * on, with a limit of limit_ns nanoseconds (1e3 .. 1e9), and reads the
 * error word back.  Returns COFEM_ERR_TIMEOUT when the wait ran out (the
 * expected result), COFEM_OK if it completed, COFEM_ERR_INVALID_ARG for a
 * limit outside the range.  Synchronous on `stream`. */
cofem_status cofem_selftest_wait_timeout(int64_t limit_ns, void* stream);

/* Self-test of the CG update's bounded wait (the paper has no counterpart).
 * Where the fit folds the direction update into the CG update, every block
 * but the one that closes the iteration waits for that block, with a time
 * limit (2 s in a fit); a wait that runs out records COFEM_ERR_TIMEOUT, ends
 * the CG loops and returns, and every later update launch of the fit ends
 * them at once.  This call runs one such launch (2 columns of 4096 values, 8
 * blocks, all resident at once) in which no block is the closing one, with a
 * limit of limit_ns nanoseconds (1e3 .. 1e9), on workspace_dev (>=
 * cofem_selftest_cg_update_workspace_bytes(), any alignment; overwritten),
 * and reads the error word back.  Returns COFEM_ERR_TIMEOUT when the waits
 * ran out (the expected result), COFEM_ERR_INVALID_ARG for a limit outside
 * the range or a null workspace, COFEM_ERR_WORKSPACE if it is too small.
 * Synchronous on `stream`. */
/* Timing of the CG vector kernels outside a fit graph (diagnostics; the paper
 * has no counterpart).  Builds a synthetic CG state of ncols (2..64) FP32
 * columns of D values on workspace_dev (>= cofem_bench_cg_kernels_workspace_
 * bytes(D, ncols) bytes, any alignment; overwritten), then times `reps`
 * launches (after one warm-up launch) each of: the CG update x += a p,
 * r -= a q, r^T r with the direction update p = r + b p and P's three BF16
 * terms fused into the same launch where its grid is resident (as cofem_fit
 * launches it for the tensor-core operator), the stand-alone direction
 * update, and the fused diagonal estimate + M-step; CUDA events on
 * `stream`.  ms_out[0..2] = mean milliseconds per launch of each; ms_out[3]
 * = 1 if the update's launch held the direction update, 0 if its grid was
 * too large to be resident at once (the update alone was timed).
 * Synchronous. */
size_t cofem_bench_cg_kernels_workspace_bytes(int64_t D, int32_t ncols);
cofem_status cofem_bench_cg_kernels(int64_t D, int32_t ncols, int32_t reps, void* workspace_dev,
                                    size_t workspace_bytes, void* stream, float* ms_out);

/* Timing of the block-CG passes (params.solver = 1) outside a fit graph
 * (diagnostics; the paper has no counterpart).  On ncols (2..64) FP32
 * columns of D values in workspace_dev (>= cofem_bench_bcg_kernels_
 * workspace_bytes(D, ncols) bytes, any alignment; overwritten), with P,
 * Z = P and Q refilled before every timed launch: ms_out[0] the xi pass
 * (Gram P^T Z, xi, M), ms_out[1] the v pass (X and V updates, Gram V^T V,
 * stop test, Cholesky QR step), ms_out[2] the row pass (Q, P and P's BF16
 * terms), ms_out[3] the three back to back; mean milliseconds over `reps`
 * launches after one warm-up, CUDA events on `stream`.  Synchronous. */
size_t cofem_bench_bcg_kernels_workspace_bytes(int64_t D, int32_t ncols);
cofem_status cofem_bench_bcg_kernels(int64_t D, int32_t ncols, int32_t reps,
                                     void* workspace_dev, size_t workspace_bytes, void* stream,
                                     float* ms_out);

size_t cofem_selftest_cg_update_workspace_bytes(void);
cofem_status cofem_selftest_cg_update_timeout(int64_t limit_ns, void* workspace_dev,
                                              size_t workspace_bytes, void* stream);

/* The two halves: W = Phi Z (ncols columns of length N, leading dimension
 * ldw) and Z = Phi^T W (length D, leading dimension ldz).  Used for
 * b = beta Phi^T y.  Same workspace rule as cofem_op_apply. Asynchronous. */
cofem_status cofem_op_forward(const cofem_op* op, cofem_dtype vec,
                              const void* z_dev, int64_t ldz, int32_t ncols,
                              void* w_dev, int64_t ldw, void* workspace_dev,
                              size_t workspace_bytes, void* stream);
cofem_status cofem_op_adjoint(const cofem_op* op, cofem_dtype vec,
                              const void* w_dev, int64_t ldw, int32_t ncols,
                              void* z_dev, int64_t ldz, void* workspace_dev,
                              size_t workspace_bytes, void* stream);

/* Diagonal estimate and M-step from a solved block X (K+1 columns, vec
 * dtype, leading dimension ld) for EM iteration t (Eq. (diag-estimate),
 * Eq. (mstep) with s):  mu_d = X[0][d];  s_d = (1/K) sum_k p_kd X[k][d]
 * (probes as in cofem_probe_fill);  alpha_d = 1 / max(mu_d^2 + s_d,
 * den_floor).  counts_dev (2 int32, optional): number of clamped
 * denominators, number of alpha_d < support_threshold (accumulated: the
 * caller zeroes them).  Asynchronous. */
cofem_status cofem_diag_mstep(uint64_t seed, int64_t t, int32_t K, int64_t D,
                              cofem_dtype vec, const void* x_dev, int64_t ld,
                              double den_floor, double support_threshold,
                              double* mu_dev, double* s_dev, double* alpha_dev,
                              int32_t* counts_dev, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* COFEM_H */
