// Internal launcher declarations of libcofem.
#pragma once
#include "common.cuh"

namespace cofem {

int num_sms();   // SM count of the current device (cached per device)

// ---- CG / probe / M-step kernels (cg_kernels.cu) ----
template <typename V>
void launch_probe_fill(uint64_t key, int K, int64_t D, V* out, int64_t ld, cudaStream_t st);
template <typename V>
void launch_cg_init(const CgConf& cf, CgCtl* ctl, CgScalars* sc, V* X, V* R, V* P,
                    const V* bvec, double* part, cudaStream_t st);
// with_direction: also apply p = r + b p in the same launch when its grid
// fits on the GPU at once; returns whether it did (else the caller launches
// cg_direction after it).
template <typename V>
bool launch_cg_update(const CgConf& cf, CgCtl* ctl, CgScalars* sc, V* X, V* R, V* P,
                      const V* Q, const double* gparts, double* part, double* part2,
                      cudaStream_t st, bool with_direction);
template <typename V>
void launch_cg_init_warm(const CgConf& cf, CgCtl* ctl, CgScalars* sc, const V* X, V* R, V* P,
                         const V* Q, const V* bvec, double* pz, double* pr, double* pb,
                         cudaStream_t st);
void launch_warm_start(const CgConf& cf, const CgCtl* ctl, long long t_first,
                       const __nv_bfloat16* w, const double* alpha, const float* pn2,
                       const double* mu_prev, const double* s_prev, float* X, float* minv,
                       cudaStream_t st);
// Batched learned start (cofem_fit_batched with a network): one problem as
// the warm-start kernel sees it -- its D, block pitch and offsets into the
// concatenated vectors (X at xoff, per-coordinate arrays at aoff, BF16 terms
// at column boff1 of the split buffer), probe seed and beta.
struct BWarmProb {
  int64_t D, ld, xoff, aoff, boff1;
  uint64_t seed;
  double beta;
};
// X0 = [mu_hat | s_hat . p_k] and M^-1 = diag(s_hat) for every problem (X0 = 0
// and M^-1 = 1 at the fit's first E-step, *t == t_first), X0's BF16 terms
// (nt per value, rows split_row(j, t) of pitch split_ld), done[i] = 0.
// Grid: ceil(ld_max / 128) x nprob blocks of 128 threads.
void launch_batched_warm_start(int nprob, int K, int64_t ld_max, const BWarmProb* probs,
                               const long long* t, long long t_first, const __nv_bfloat16* w,
                               const double* alpha, const float* pn2, const double* mu_prev,
                               const double* s_prev, float* X, float* minv, int* done,
                               int split_nt, __nv_bfloat16* split_buf, int64_t split_ld,
                               cudaStream_t st);
// ||phi_d||^2 of a BF16 dictionary (N x D, leading dimension ld) into out[0..D).
void launch_col_norms_bf16(const void* phi, int64_t N, int64_t D, int64_t ld, float* out,
                           cudaStream_t st);
// cofem_last_fit_fallbacks of this thread (set by the batched fit).
void set_last_fit_fallbacks(int n);
// Self-test of the fused CG update's bounded wait (cg_kernels.cu): returns the
// error word after one launch in which no block closes the iteration, or -1
// on a CUDA error.  ws: cg_update_selftest_bytes() bytes.
size_t cg_update_selftest_bytes();
int cg_update_selftest(int64_t limit_ns, char* ws, cudaStream_t st);
// Timing of the CG vector kernels outside a fit graph (cg_kernels.cu).
size_t cg_kernels_bench_bytes(int64_t D, int ncols);
int cg_kernels_bench(int64_t D, int ncols, int reps, char* ws, cudaStream_t st, float* ms);

// ---- block CG (block_cg.cu) ----
// Workspace bytes of one block-CG solve with ncols columns of leading
// dimension ld (vector element size vec_bytes).
size_t bcg_state_bytes(int vec_bytes, int ncols, int64_t ld);
// Start of an E-step: X = 0, Q R-factor of B, P = Q.
template <typename V>
cudaError_t launch_bcg_start(const CgConf& cf, CgCtl* ctl, char* state, V* X, V* R, V* P,
                             const V* bvec, cudaStream_t st);
// One iteration after Z = A P: the xi and v gram passes (the second with
// the stop test) and the row pass.
// Timing of the block-CG passes outside a fit graph (block_cg.cu).
size_t bcg_bench_bytes(int64_t D, int ncols);
int bcg_kernels_bench(int64_t D, int ncols, int reps, char* ws, cudaStream_t st, float* ms);
template <typename V>
cudaError_t launch_bcg_iteration(const CgConf& cf, CgCtl* ctl, char* state, V* X, V* R, V* P,
                                 const V* Z, cudaStream_t st);

template <typename V>
void launch_cg_true_resid(const CgConf& cf, CgCtl* ctl, CgScalars* sc, V* R, const V* Q,
                          const V* bvec, double* part, double* part2, cudaStream_t st);
template <typename V>
void launch_cg_direction(const CgConf& cf, const CgCtl* ctl, const CgScalars* sc,
                         const V* R, V* P, cudaStream_t st);
template <typename V>
void launch_diag_mstep(const CgConf& cf, CgCtl* ctl, uint64_t key, const V* X, double* mu,
                       double* s, double* alpha, int32_t* counts, int32_t* st_iters,
                       double* st_relres, int32_t* st_clamps, int32_t* st_support,
                       cudaStream_t st);
template <typename V>
void launch_scale(V* x, int64_t n, double beta, cudaStream_t st);

// ---- convolutional dictionary (conv.cu); h64: C x 64 taps ----
void conv_forward(const float* h64, int C, int64_t L, const float* Z, int64_t ldz, int ncols,
                  float* W, int64_t ldw, cudaStream_t st);
int conv_adjoint(const float* h64, int C, int64_t L, const float* W, int64_t ldw, int ncols,
                 float* Y, int64_t ld, double beta, const double* alpha, const float* X,
                 double* dots, cudaStream_t st, const float* alpha32 = nullptr);
void conv_pad_filters(const float* h, int C, int T, float* h64, cudaStream_t st);
void conv_alpha_f32(const double* alpha, int64_t n, float* out, cudaStream_t st);
// ---- convolution on the tensor cores (conv_tc.cu): BF16 filters ----
// h64 = the BF16-rounded filters padded to 64 taps; img = the forward and
// adjoint Toeplitz tiles (conv_tc_image_bytes(C) bytes, 1024-byte aligned)
size_t conv_tc_image_bytes(int C);
void conv_tc_prepare(const float* h, int C, int T, float* h64, __nv_bfloat16* img,
                     cudaStream_t st);
void conv_tc_forward(int C, int64_t L, const float* Z, int64_t ldz, int ncols, float* W,
                     int64_t ldw, const __nv_bfloat16* img, int* err, cudaStream_t st);
int conv_tc_adjoint(int C, int64_t L, const float* W, int64_t ldw, int ncols, float* Y,
                    int64_t ld, double beta, const double* alpha, const float* alpha32,
                    const float* X, double* dots, const __nv_bfloat16* img, int* err,
                    cudaStream_t st);

// ---- masked DCT dictionary (dct.cu); idx: N strictly increasing sample indices ----
bool dct_size_ok(int64_t D);                      // D a power of two, 16 <= D <= 2^22
size_t dct_ws_bytes(int64_t D, int ncols);
// prepared: the mask and twiddle tables are already in ws (dct_prepare with
// the same D, idx, ncols and ws)
void dct_prepare(int64_t D, const int32_t* idx, int64_t N, int ncols, char* ws, int* err,
                 cudaStream_t st);
int dct_apply(int64_t D, const int32_t* idx, int64_t N, const float* X, int64_t ld, int ncols,
              float* Y, double beta, const double* alpha, const float* alpha32, double* dots,
              char* ws, int* err, cudaStream_t st, bool prepared = false);
void dct_forward(int64_t D, const int32_t* idx, int64_t N, const float* Z, int64_t ldz, int ncols,
                 float* W, int64_t ldw, char* ws, int* err, cudaStream_t st);
void dct_adjoint(int64_t D, const int32_t* idx, int64_t N, const float* W, int64_t ldw, int ncols,
                 float* Z, int64_t ldz, double beta, char* ws, int* err, cudaStream_t st);
// ||phi_d||^2, d < D, into out (closed form from one DCT of the mask);
// scratch: ones_buf (N floats), x_buf (D floats), ws (dct_ws_bytes(D, 1)).
void dct_col_norms(int64_t D, const int32_t* idx, int64_t N, float* ones_buf, float* x_buf,
                   char* ws, int* err, float* out, cudaStream_t st);

// ---- operator application ----
// Every operator application writes, besides its output, per-block partial
// dot products gamma_j = x_j^T (A x)_j into `dots` (layout [part][kMaxCols])
// and returns the number of parts used through *nparts (0 if dots == null).
struct ApplyArgs {
  const void* x;       // input block (vec dtype), leading dim ld
  void* y;             // output block
  int64_t ld;
  int ncols;
  const double* alpha; // D doubles (nullptr: no diagonal term)
  double beta;
  double* dots;        // [kMaxParts][kMaxCols] partials or nullptr
  char* ws;            // operator scratch
  size_t ws_bytes;
};

}  // namespace cofem
