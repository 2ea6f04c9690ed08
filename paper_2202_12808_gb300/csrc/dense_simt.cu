// Dense dictionary operator on CUDA cores: A X = beta Phi^T (Phi X) + alpha . X
// (Eq. (mat-eq)), as two tall-skinny products with split-K partial sums:
//   GEMM1  W_s = Phi[:, K-range s] X[K-range s, :]          (N x ncols)
//   reduce W   = sum_s W_s                                   (fixed order)
//   GEMM2  Q_s = Phi[K-range s, :]^T W[K-range s, :]         (D x ncols)
//   epilogue Y = beta sum_s Q_s + alpha . X, gamma_j partials = x_j^T y_j
// Used for FP64 dictionaries (F64 vectors) and as the CUDA-core path for
// F32 and BF16 dictionaries.  The tensor-core path is dense_tc.cu.
#include "dense.cuh"

namespace cofem {

constexpr int kBK = 32;

template <typename T> __device__ __forceinline__ float to_f(T v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) {
  return __bfloat162float(v);
}
template <> __device__ __forceinline__ float to_f<F32HiLo>(F32HiLo v) { return hilo_value(v.v); }

template <typename V, typename TA> __device__ __forceinline__ V cvt(TA v) {
  if constexpr (std::is_same<TA, double>::value) return (V)v;
  else return (V)to_f<TA>(v);
}

// C_s(m, j) = sum_{k in split s} A(m, k) B(k, j)
// A(m, k) = A_KMAJOR ? A[m*lda + k] : A[k*lda + m];  B(k, j) = B[j*ldb + k]
// C_s(m, j) -> C[s*split_stride + j*ldc + m]
template <typename TA, typename V, bool A_KMAJOR, int TM, int TN>
__global__ void __launch_bounds__(256)
tsgemm_kernel(int64_t M, int64_t Kdim, int ncols, const TA* __restrict__ A, int64_t lda,
              const V* __restrict__ B, int64_t ldb, V* __restrict__ C, int64_t ldc,
              int64_t split_stride, int64_t k_per_split) {
  pdl_wait();
  pdl_trigger();
  constexpr int BM = 16 * TM, BN = 16 * TN;
  __shared__ __align__(16) V As[kBK][BM + 4];
  __shared__ __align__(16) V Bs[kBK][BN];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t m0 = (int64_t)blockIdx.x * BM;
  const int s = blockIdx.y;
  const int64_t kbeg = (int64_t)s * k_per_split;
  const int64_t kend = min(Kdim, kbeg + k_per_split);
  V acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int t = 0; t < TN; ++t) acc[i][t] = V(0);

  for (int64_t k0 = kbeg; k0 < kend; k0 += kBK) {
#pragma unroll
    for (int i = 0; i < BM * kBK / 256; ++i) {
      const int idx = threadIdx.x + 256 * i;
      int mm, kk;
      if (A_KMAJOR) { kk = idx % kBK; mm = idx / kBK; }
      else { mm = idx % BM; kk = idx / BM; }
      const int64_t gm = m0 + mm, gk = k0 + kk;
      V v = V(0);
      if (gm < M && gk < kend)
        v = cvt<V, TA>(A_KMAJOR ? A[gm * lda + gk] : A[gk * lda + gm]);
      As[kk][mm] = v;
    }
    for (int idx = threadIdx.x; idx < BN * kBK; idx += 256) {
      const int kk = idx % kBK, jj = idx / kBK;
      const int64_t gk = k0 + kk;
      V v = V(0);
      if (jj < ncols && gk < kend) v = B[(int64_t)jj * ldb + gk];
      Bs[kk][jj] = v;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kBK; ++kk) {
      V a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty * TM + i];
#pragma unroll
      for (int t = 0; t < TN; ++t) b[t] = Bs[kk][tx + 16 * t];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int t = 0; t < TN; ++t) acc[i][t] = fma(a[i], b[t], acc[i][t]);
    }
    __syncthreads();
  }
  V* Cs = C + (int64_t)s * split_stride;
#pragma unroll
  for (int t = 0; t < TN; ++t) {
    const int j = tx + 16 * t;
    if (j >= ncols) continue;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int64_t gm = m0 + ty * TM + i;
      if (gm < M) Cs[(int64_t)j * ldc + gm] = acc[i][t];
    }
  }
}

// Y(m, j) = beta * sum_s P_s(m, j) [+ alpha_m X(m, j)];  dots[part][j] = X.Y
// Partials P_s have leading dimension ldp, X and Y have ldo (>= M); entries
// m in [M, ldo) of Y are written as zero.  Grid (blocks, ncols).
template <typename V>
__global__ void reduce_epilogue_kernel(int64_t M, int64_t ldp, int64_t ldo, int S,
                                       int64_t split_stride, const V* __restrict__ Pp,
                                       double beta, const double* __restrict__ alpha,
                                       const V* __restrict__ X, V* __restrict__ Y,
                                       double* dots) {
  pdl_wait();
  pdl_trigger();
  __shared__ double sh[32];
  const int j = blockIdx.y;
  typename AccOf<V>::T acc;
  for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < ldo;
       m += (int64_t)gridDim.x * blockDim.x) {
    V y = V(0);
    if (m < M) {
      V sum = V(0);
      for (int s = 0; s < S; ++s) sum += Pp[(int64_t)s * split_stride + (int64_t)j * ldp + m];
      y = (V)beta * sum;
      if (alpha) {
        const V xv = X[(int64_t)j * ldo + m];
        y = fma((V)alpha[m], xv, y);
        acc.add_prod(xv, y);
      }
    }
    Y[(int64_t)j * ldo + m] = y;
  }
  if (dots) {
    const double t = block_sum(acc, sh);
    if (threadIdx.x == 0) dots[(int64_t)blockIdx.x * kMaxCols + j] = t;
  }
}

// ------------------------------------------------------------- planning

static int pick_tn(int ncols) { return ncols <= 16 ? 1 : ncols <= 32 ? 2 : ncols <= 48 ? 3 : 4; }

template <typename V> static int pick_tm() { return sizeof(V) == 8 ? 4 : 8; }

static void split_plan(int64_t M, int64_t Kdim, int BM, int sms, int* S, int64_t* kps) {
  const int64_t mt = (M + BM - 1) / BM;
  int64_t kblocks = (Kdim + kBK - 1) / kBK;
  int64_t want = (2 * (int64_t)sms + mt - 1) / mt;
  if (want < 1) want = 1;
  if (want > kblocks) want = kblocks;
  if (want > 64) want = 64;
  int64_t per = (kblocks + want - 1) / want;
  *kps = per * kBK;
  *S = (int)((Kdim + *kps - 1) / *kps);
}

DenseSimtPlan dense_simt_plan(int64_t N, int64_t D, int ncols, int vec_bytes, int sms) {
  DenseSimtPlan p;
  const int BM = vec_bytes == 8 ? 64 : 128;
  p.ldw = round_up(N, kLdAlign);
  p.ld = round_up(D, kLdAlign);
  split_plan(N, D, BM, sms, &p.S1, &p.kps1);
  split_plan(D, N, BM, sms, &p.S2, &p.kps2);
  p.bytes_wpart = (size_t)p.S1 * ncols * p.ldw * vec_bytes;
  p.bytes_w = (size_t)ncols * p.ldw * vec_bytes;
  p.bytes_qpart = (size_t)p.S2 * ncols * p.ld * vec_bytes;
  return p;
}

static int epi_blocks(int64_t ld, int ncols, int sms) {
  int64_t need = (ld + 255) / 256;
  int64_t cap = (int64_t)8 * sms / ncols;
  if (cap < 1) cap = 1;
  int64_t b = need < cap ? need : cap;
  if (b > kMaxParts) b = kMaxParts;
  return (int)(b < 1 ? 1 : b);
}

template <typename TA, typename V, bool KM>
static void launch_tsgemm(int64_t M, int64_t Kdim, int ncols, const TA* A, int64_t lda,
                          const V* B, int64_t ldb, V* C, int64_t ldc, int64_t sstride,
                          int S, int64_t kps, cudaStream_t st) {
  constexpr int TM = sizeof(V) == 8 ? 4 : 8;
  const int BM = 16 * TM;
  dim3 g((unsigned)((M + BM - 1) / BM), S);
  switch (pick_tn(ncols)) {
    case 1: launch_k(tsgemm_kernel<TA, V, KM, TM, 1>, dim3(g), dim3(256), 0, st, M, Kdim, ncols, A, lda, B, ldb, C, ldc, sstride, kps); break;
    case 2: launch_k(tsgemm_kernel<TA, V, KM, TM, 2>, dim3(g), dim3(256), 0, st, M, Kdim, ncols, A, lda, B, ldb, C, ldc, sstride, kps); break;
    case 3: launch_k(tsgemm_kernel<TA, V, KM, TM, 3>, dim3(g), dim3(256), 0, st, M, Kdim, ncols, A, lda, B, ldb, C, ldc, sstride, kps); break;
    default: launch_k(tsgemm_kernel<TA, V, KM, TM, 4>, dim3(g), dim3(256), 0, st, M, Kdim, ncols, A, lda, B, ldb, C, ldc, sstride, kps); break;
  }
}

// W = Phi Z   (Z: D x ncols, ldz;  W: N x ncols, ldw)
template <typename TA, typename V>
void dense_simt_forward(const DenseDesc& op, const V* Z, int64_t ldz, int ncols, V* W,
                        int64_t ldw, char* ws, cudaStream_t st) {
  const int sms = num_sms();
  DenseSimtPlan p = dense_simt_plan(op.N, op.D, ncols, sizeof(V), sms);
  V* Wp = reinterpret_cast<V*>(ws);
  const int64_t sstride = (int64_t)ncols * p.ldw;
  launch_tsgemm<TA, V, true>(op.N, op.D, ncols, (const TA*)op.phi, op.ld, Z, ldz, Wp, p.ldw,
                             sstride, p.S1, p.kps1, st);
  apply_tick(st);
  dim3 g(epi_blocks(ldw, ncols, sms), ncols);
  launch_k(reduce_epilogue_kernel<V>, dim3(g), dim3(256), 0, st, op.N, p.ldw, ldw, p.S1, sstride, Wp, 1.0,
                                               nullptr, nullptr, W, nullptr);
  apply_tick(st);
}

// Y = beta Phi^T W [+ alpha . X]  (W: N x ncols, ldw;  X, Y: D x ncols, ld)
template <typename TA, typename V>
void dense_simt_adjoint(const DenseDesc& op, const V* W, int64_t ldw, int ncols, V* Y,
                        int64_t ld, double beta, const double* alpha, const V* X,
                        double* dots, int* nparts, char* ws, cudaStream_t st) {
  const int sms = num_sms();
  DenseSimtPlan p = dense_simt_plan(op.N, op.D, ncols, sizeof(V), sms);
  V* Qp = reinterpret_cast<V*>(ws + p.bytes_wpart + p.bytes_w);
  const int64_t sstride = (int64_t)ncols * p.ld;
  launch_tsgemm<TA, V, false>(op.D, op.N, ncols, (const TA*)op.phi, op.ld, W, ldw, Qp, p.ld,
                              sstride, p.S2, p.kps2, st);
  apply_tick(st);
  dim3 g(epi_blocks(ld, ncols, sms), ncols);
  launch_k(reduce_epilogue_kernel<V>, dim3(g), dim3(256), 0, st, op.D, p.ld, ld, p.S2, sstride, Qp, beta, alpha,
                                               X, Y, dots);
  apply_tick(st);
  if (nparts) *nparts = dots ? (int)g.x : 0;
}

// Y = beta Phi^T Phi X + alpha . X
template <typename TA, typename V>
void dense_simt_apply(const DenseDesc& op, const V* X, int64_t ld, int ncols, V* Y,
                      double beta, const double* alpha, double* dots, int* nparts, char* ws,
                      cudaStream_t st) {
  const int sms = num_sms();
  DenseSimtPlan p = dense_simt_plan(op.N, op.D, ncols, sizeof(V), sms);
  V* W = reinterpret_cast<V*>(ws + p.bytes_wpart);
  dense_simt_forward<TA, V>(op, X, ld, ncols, W, p.ldw, ws, st);
  dense_simt_adjoint<TA, V>(op, W, p.ldw, ncols, Y, ld, beta, alpha, X, dots, nparts, ws, st);
}

#define INST(TA, V)                                                                        \
  template void dense_simt_forward<TA, V>(const DenseDesc&, const V*, int64_t, int, V*,    \
                                          int64_t, char*, cudaStream_t);                   \
  template void dense_simt_adjoint<TA, V>(const DenseDesc&, const V*, int64_t, int, V*,    \
                                          int64_t, double, const double*, const V*,        \
                                          double*, int*, char*, cudaStream_t);             \
  template void dense_simt_apply<TA, V>(const DenseDesc&, const V*, int64_t, int, V*,      \
                                        double, const double*, double*, int*, char*,       \
                                        cudaStream_t);
INST(double, double)
INST(float, float)
INST(__nv_bfloat16, float)
INST(F32HiLo, float)

}  // namespace cofem
