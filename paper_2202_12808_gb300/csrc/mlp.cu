// Learned warm start and diagonal preconditioner for the E-step solve (the
// paper has no learned component; plain CG remains the fallback and its
// stop test decides the result).  A per-coordinate MLP 4 -> 32 -> 32 -> 2 (tanh,
// 1282 parameters, layout W1 32x4 | b1 | W2 32x32 | b2 | W3 2x32 | b3)
// maps normalised features of coordinate d, with c_d = beta ||phi_d||^2 +
// alpha_d,
//   u = [ln alpha_d / 10, ln(beta ||phi_d||^2) / 10,
//        asinh(mu_prev_d sqrt(c_d)) / 4, ln(max(s_prev_d c_d, 1e-6)) / 4]
// to o, read as mu_hat_d = sinh(4 o1) / sqrt(c_d), s_hat_d = exp(4 o2) / c_d.
// Inference uses BF16 weights with FP32 arithmetic; training keeps FP32
// master weights, runs the forward pass with the BF16 copy, and reduces the
// per-block gradients in a fixed order before an Adam step.
#include <cmath>

#include "dense.cuh"

namespace cofem {

constexpr int kMlpParams = 1282;
constexpr int oW1 = 0, ob1 = 128, oW2 = 160, ob2 = 1184, oW3 = 1216, ob3 = 1280;
constexpr int kTrainS = 128;            // samples per training block

template <typename TW> __device__ __forceinline__ float wf(TW v);
template <> __device__ __forceinline__ float wf<float>(float v) { return v; }
template <> __device__ __forceinline__ float wf<__nv_bfloat16>(__nv_bfloat16 v) {
  return __bfloat162float(v);
}

template <typename TW>
__device__ __forceinline__ void load_weights(const TW* w, float* sw) {
  for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) sw[i] = wf<TW>(w[i]);
  __syncthreads();
}

// Forward pass of one sample; the thread's hidden activations go to its
// own shared-memory rows r1, r2 (33 floats apart across threads, so the
// per-thread accesses hit distinct banks).
__device__ __forceinline__ void mlp_fwd(const float* sw, const float (&u)[4], float* r1,
                                        float* r2, float (&o)[2]) {
#pragma unroll 4
  for (int i = 0; i < 32; ++i) {
    float a = sw[ob1 + i];
#pragma unroll
    for (int k = 0; k < 4; ++k) a = fmaf(sw[oW1 + i * 4 + k], u[k], a);
    r1[i] = tanhf(a);
  }
#pragma unroll 2
  for (int i = 0; i < 32; ++i) {
    float a = sw[ob2 + i];
#pragma unroll 8
    for (int k = 0; k < 32; ++k) a = fmaf(sw[oW2 + i * 32 + k], r1[k], a);
    r2[i] = tanhf(a);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    float a = sw[ob3 + i];
#pragma unroll 8
    for (int k = 0; k < 32; ++k) a = fmaf(sw[oW3 + i * 32 + k], r2[k], a);
    o[i] = a;
  }
}

__device__ __forceinline__ void features(double alpha, float pn2, double beta, double mu_prev,
                                         double s_prev, float (&u)[4], double* c_out) {
  const double bp = beta * (double)pn2;
  const double c = bp + alpha;
  u[0] = (float)(log(alpha) / 10.0);
  u[1] = (float)(log(bp) / 10.0);
  u[2] = (float)(asinh(mu_prev * sqrt(c)) / 4.0);
  u[3] = (float)(log(fmax(s_prev * c, 1e-6)) / 4.0);
  *c_out = c;
}

__device__ __forceinline__ double wf_any(double v) { return v; }
__device__ __forceinline__ double wf_any(float v) { return v; }
__device__ __forceinline__ double wf_any(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ double wf_any(F32HiLo v) { return hilo_value(v.v); }

// ----------------------------------------------------- column norms of Phi
template <typename TA>
__global__ void col_norms_kernel(const TA* phi, int64_t N, int64_t D, int64_t ld, float* out) {
  pdl_wait();
  pdl_trigger();
  for (int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; d < D;
       d += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int64_t n = 0; n < N; ++n) {
      const double v = (double)wf_any(phi[n * ld + d]);
      acc += v * v;
    }
    out[d] = (float)acc;
  }
}

// -------------------------------------------------- features and targets
__global__ void features_kernel(const double* alpha, const float* pn2, double beta,
                                const double* mu_prev, const double* s_prev, int64_t D,
                                float* U) {
  pdl_wait();
  pdl_trigger();
  for (int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; d < D;
       d += (int64_t)gridDim.x * blockDim.x) {
    float u[4];
    double c;
    features(alpha[d], pn2[d], beta, mu_prev ? mu_prev[d] : 0.0,
             s_prev ? s_prev[d] : 1.0 / (beta * (double)pn2[d] + alpha[d]), u, &c);
#pragma unroll
    for (int k = 0; k < 4; ++k) U[d * 4 + k] = u[k];
  }
}

__global__ void targets_kernel(const double* alpha, const float* pn2, double beta,
                               const double* mu, const double* s, int64_t D, float* Y) {
  pdl_wait();
  pdl_trigger();
  for (int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; d < D;
       d += (int64_t)gridDim.x * blockDim.x) {
    const double c = beta * (double)pn2[d] + alpha[d];
    Y[d * 2] = (float)(asinh(mu[d] * sqrt(c)) / 4.0);
    Y[d * 2 + 1] = (float)(log(fmax(s[d] * c, 1e-6)) / 4.0);
  }
}

// ------------------------------------------------------------- inference
template <typename TW>
__global__ void mlp_forward_kernel(const TW* w, const float* U, int64_t n, float* O) {
  pdl_wait();
  pdl_trigger();
  __shared__ float sw[kMlpParams];
  __shared__ float rows[2][128 * 33];
  load_weights<TW>(w, sw);
  float* r1 = rows[0] + threadIdx.x * 33;
  float* r2 = rows[1] + threadIdx.x * 33;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float u[4] = {U[i * 4], U[i * 4 + 1], U[i * 4 + 2], U[i * 4 + 3]};
    float o[2];
    mlp_fwd(sw, u, r1, r2, o);
    O[i * 2] = o[0];
    O[i * 2 + 1] = o[1];
  }
}

// -------------------------------------------------------------- training
// One block = kTrainS samples: forward with weights w, backward of the mean
// loss 1/(2n) sum ||o - y||^2, per-block gradient (each parameter summed
// over the block's samples in order) -> gpart[block][param], loss -> lpart.
template <typename TW>
__global__ void __launch_bounds__(kTrainS)
mlp_train_kernel(const TW* w, const float* U, const float* Y, int64_t n, float* gpart,
                 double* lpart) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ float sm[];
  float* sw = sm;                                   // 1282 (+pad)
  float* su = sw + 1284;                            // S x 4
  float* sh1 = su + kTrainS * 4;                    // S x 33
  float* sh2 = sh1 + kTrainS * 33;
  float* sa2 = sh2 + kTrainS * 33;
  float* sa1 = sa2 + kTrainS * 33;
  float* sgo = sa1 + kTrainS * 33;                  // S x 2
  __shared__ double red[32];
  load_weights<TW>(w, sw);
  const int tid = threadIdx.x;
  const int64_t i = (int64_t)blockIdx.x * kTrainS + tid;
  const bool valid = i < n;
  float u[4] = {0.f, 0.f, 0.f, 0.f}, y[2] = {0.f, 0.f};
  if (valid) {
#pragma unroll
    for (int k = 0; k < 4; ++k) u[k] = U[i * 4 + k];
    y[0] = Y[i * 2];
    y[1] = Y[i * 2 + 1];
  }
  float* r1 = sh1 + tid * 33;
  float* r2 = sh2 + tid * 33;
  float o[2];
  mlp_fwd(sw, u, r1, r2, o);
  const float inv_n = 1.0f / (float)n;
  float go[2];
  double l = 0.0;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const float e = o[k] - y[k];
    go[k] = valid ? e * inv_n : 0.f;
    if (valid) l += 0.5 * (double)e * (double)e;
  }
  float* g2 = sa2 + tid * 33;
#pragma unroll 4
  for (int k = 0; k < 32; ++k) {
    const float g = sw[oW3 + k] * go[0] + sw[oW3 + 32 + k] * go[1];
    g2[k] = g * (1.f - r2[k] * r2[k]);
  }
#pragma unroll 2
  for (int k = 0; k < 32; ++k) {
    float g = 0.f;
#pragma unroll 8
    for (int j = 0; j < 32; ++j) g = fmaf(sw[oW2 + j * 32 + k], g2[j], g);
    sa1[tid * 33 + k] = g * (1.f - r1[k] * r1[k]);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) su[tid * 4 + k] = u[k];
  sgo[tid * 2] = go[0];
  sgo[tid * 2 + 1] = go[1];
  __syncthreads();
  for (int p = tid; p < kMlpParams; p += kTrainS) {
    float g = 0.f;
    if (p < ob1) {                               // W1[r][c] += ga1[r] u[c]
      const int r = p / 4, c = p % 4;
      for (int s = 0; s < kTrainS; ++s) g = fmaf(sa1[s * 33 + r], su[s * 4 + c], g);
    } else if (p < oW2) {
      const int r = p - ob1;
      for (int s = 0; s < kTrainS; ++s) g += sa1[s * 33 + r];
    } else if (p < ob2) {                        // W2[r][c] += ga2[r] h1[c]
      const int r = (p - oW2) / 32, c = (p - oW2) % 32;
      for (int s = 0; s < kTrainS; ++s) g = fmaf(sa2[s * 33 + r], sh1[s * 33 + c], g);
    } else if (p < oW3) {
      const int r = p - ob2;
      for (int s = 0; s < kTrainS; ++s) g += sa2[s * 33 + r];
    } else if (p < ob3) {                        // W3[r][c] += go[r] h2[c]
      const int r = (p - oW3) / 32, c = (p - oW3) % 32;
      for (int s = 0; s < kTrainS; ++s) g = fmaf(sgo[s * 2 + r], sh2[s * 33 + c], g);
    } else {
      const int r = p - ob3;
      for (int s = 0; s < kTrainS; ++s) g += sgo[s * 2 + r];
    }
    gpart[(int64_t)blockIdx.x * kMlpParams + p] = g;
  }
  const double bl = block_sum(l, red);
  if (tid == 0) lpart[blockIdx.x] = bl;
}

// Fixed-order sum of the block gradients; optional Adam step on the FP32
// master weights (and their BF16 copy).  One thread per parameter.
__global__ void mlp_reduce_adam_kernel(const float* gpart, int nblocks, const double* lpart,
                                       double inv_n, float* grad, double* loss, float* master,
                                       float* m, float* v, __nv_bfloat16* wbf, int step,
                                       float lr, float b1, float b2, float eps) {
  pdl_wait();
  pdl_trigger();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p == 0 && loss) {
    double l = 0.0;
    for (int b = 0; b < nblocks; ++b) l += lpart[b];
    *loss = l * inv_n;
  }
  if (p >= kMlpParams) return;
  float g = 0.f;
  for (int b = 0; b < nblocks; ++b) g += gpart[(int64_t)b * kMlpParams + p];
  if (grad) grad[p] = g;
  if (master && step > 0) {
    const float mm = b1 * m[p] + (1.f - b1) * g;
    const float vv = b2 * v[p] + (1.f - b2) * g * g;
    m[p] = mm;
    v[p] = vv;
    const float mh = mm / (1.f - powf(b1, (float)step));
    const float vh = vv / (1.f - powf(b2, (float)step));
    const float th = master[p] - lr * mh / (sqrtf(vh) + eps);
    master[p] = th;
    if (wbf) wbf[p] = __float2bfloat16_rn(th);
  }
}

// ------------------------------------------- warm start inside a fit
// At the first E-step of a fit (no previous mu, s) X0 = 0 and M^-1 = 1 (the
// preconditioned solve is then plain CG); afterwards X0 = [mu_hat | s_hat .
// p_k] and M^-1 = s_hat.  Writes X (all K+1 columns, zero padding) and minv.
__global__ void warm_start_kernel(CgConf cf, const CgCtl* ctl, long long t_first,
                                  const __nv_bfloat16* w, const double* alpha, const float* pn2,
                                  const double* mu_prev, const double* s_prev, float* X,
                                  float* minv) {
  pdl_wait();
  pdl_trigger();
  __shared__ float sw[kMlpParams];
  __shared__ float rows[2][128 * 33];
  load_weights<__nv_bfloat16>(w, sw);
  float* r1 = rows[0] + threadIdx.x * 33;
  float* r2 = rows[1] + threadIdx.x * 33;
  const bool first = ctl->t == t_first;
  const uint64_t key = probe_key(cf.seed, ctl->t);
  for (int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; d < cf.ld;
       d += (int64_t)gridDim.x * blockDim.x) {
    float m0 = 0.f, sh = 1.f;
    if (d < cf.D && !first) {
      float u[4], o[2];
      double c;
      features(alpha[d], pn2[d], cf.beta, mu_prev[d], s_prev[d], u, &c);
      mlp_fwd(sw, u, r1, r2, o);
      m0 = (float)(sinh(4.0 * (double)o[0]) / sqrt(c));
      sh = (float)(exp(4.0 * fmin(fmax((double)o[1], -10.0), 10.0)) / c);
    }
    if (d >= cf.D) { m0 = 0.f; sh = 0.f; }
    minv[d] = d < cf.D ? sh : 0.f;
    X[d] = m0;
    for (int w0 = 0; w0 * 64 < cf.K; ++w0) {
      const uint64_t h = d < cf.D ? probe_word(key, d, w0) : 0ull;
      const int kend = min(cf.K, (w0 + 1) * 64);
      for (int k = w0 * 64; k < kend; ++k) {
        const float pk = ((h >> (k & 63)) & 1ull) ? -1.f : 1.f;
        X[(int64_t)(k + 1) * cf.ld + d] = (d < cf.D && !first) ? sh * pk : 0.f;
      }
    }
  }
}

// The batched form of warm_start_kernel: blockIdx.y is the problem.
__global__ void batched_warm_start_kernel(int K, const BWarmProb* probs, const long long* tcur,
                                          long long t_first, const __nv_bfloat16* w,
                                          const double* alpha, const float* pn2,
                                          const double* mu_prev, const double* s_prev, float* X,
                                          float* minv, int* done, int split_nt,
                                          __nv_bfloat16* split_buf, int64_t split_ld) {
  pdl_wait();
  pdl_trigger();
  __shared__ float sw[kMlpParams];
  __shared__ float rows[2][128 * 33];
  const BWarmProb pb = probs[blockIdx.y];
  const int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if ((int64_t)blockIdx.x * blockDim.x >= pb.ld) return;       // whole block past this problem
  load_weights<__nv_bfloat16>(w, sw);
  if (blockIdx.x == 0 && threadIdx.x == 0) done[blockIdx.y] = 0;
  if (d >= pb.ld) return;
  float* r1 = rows[0] + threadIdx.x * 33;
  float* r2 = rows[1] + threadIdx.x * 33;
  const long long t = *tcur;
  const bool first = t == t_first;
  const uint64_t key = probe_key(pb.seed, t);
  float m0 = 0.f, sh = 1.f;
  if (d < pb.D && !first) {
    float u[4], o[2];
    double c;
    const int64_t a = pb.aoff + d;
    features(alpha[a], pn2[a], pb.beta, mu_prev[a], s_prev[a], u, &c);
    mlp_fwd(sw, u, r1, r2, o);
    m0 = (float)(sinh(4.0 * (double)o[0]) / sqrt(c));
    sh = (float)(exp(4.0 * fmin(fmax((double)o[1], -10.0), 10.0)) / c);
  }
  if (d >= pb.D) { m0 = 0.f; sh = 0.f; }
  if (d < pb.D) minv[pb.aoff + d] = sh;
  auto put = [&](int j, float v) {
    X[pb.xoff + (int64_t)j * pb.ld + d] = v;
    float r = v;
    for (int tt = 0; tt < split_nt; ++tt) {
      const __nv_bfloat16 o = __float2bfloat16_rn(r);
      r -= __bfloat162float(o);
      split_buf[(int64_t)split_row(j, tt, split_nt) * split_ld + pb.boff1 + d] = o;
    }
  };
  put(0, m0);
  for (int w0 = 0; w0 * 64 < K; ++w0) {
    const uint64_t h = d < pb.D ? probe_word(key, d, w0) : 0ull;
    const int kend = min(K, (w0 + 1) * 64);
    for (int k = w0 * 64; k < kend; ++k) {
      const float pk = ((h >> (k & 63)) & 1ull) ? -1.f : 1.f;
      put(k + 1, (d < pb.D && !first) ? sh * pk : 0.f);
    }
  }
}

void launch_batched_warm_start(int nprob, int K, int64_t ld_max, const BWarmProb* probs,
                               const long long* t, long long t_first, const __nv_bfloat16* w,
                               const double* alpha, const float* pn2, const double* mu_prev,
                               const double* s_prev, float* X, float* minv, int* done,
                               int split_nt, __nv_bfloat16* split_buf, int64_t split_ld,
                               cudaStream_t st) {
  const dim3 g((unsigned)((ld_max + 127) / 128), (unsigned)nprob);
  launch_k(batched_warm_start_kernel, g, dim3(128), 0, st, K, probs, t, t_first, w, alpha, pn2,
           mu_prev, s_prev, X, minv, done, split_nt, split_buf, split_ld);
}

void launch_warm_start(const CgConf& cf, const CgCtl* ctl, long long t_first,
                       const __nv_bfloat16* w, const double* alpha, const float* pn2,
                       const double* mu_prev, const double* s_prev, float* X, float* minv,
                       cudaStream_t st) {
  int64_t need = (cf.ld + 127) / 128;
  const unsigned blocks = (unsigned)(need < 2048 ? need : 2048);
  launch_k(warm_start_kernel, dim3(blocks), dim3(128), 0, st, cf, ctl, t_first, w, alpha, pn2,
           mu_prev, s_prev, X, minv);
}

}  // namespace cofem

// ================================================================== ABI
struct cofem_op;   // opaque here; the dense fields are reached through accessors

namespace cofem {
int op_is_dense(const cofem_op* op);
DenseDesc op_dense_desc(const cofem_op* op);
int op_conv_desc(const cofem_op* op, int64_t* L, int* C, int* T, const float** h, int* bf16);

// ||phi_d||^2 = sum_t h[c][t]^2 for d = c L + m (taps rounded to BF16 when
// the operator runs on the tensor cores)
__global__ void conv_col_norms_kernel(const float* h, int C, int T, int64_t L, int bf16,
                                      float* out) {
  pdl_wait();
  pdl_trigger();
  for (int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; d < (int64_t)C * L;
       d += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(d / L);
    double acc = 0.0;
    for (int t = 0; t < T; ++t) {
      float v = h[c * T + t];
      if (bf16) v = __bfloat162float(__float2bfloat16_rn(v));
      acc += (double)v * (double)v;
    }
    out[d] = (float)acc;
  }
}

static unsigned blocks_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  return (unsigned)(b < 4096 ? (b < 1 ? 1 : b) : 4096);
}

void launch_col_norms_bf16(const void* phi, int64_t N, int64_t D, int64_t ld, float* out,
                           cudaStream_t st) {
  launch_k(col_norms_kernel<__nv_bfloat16>, dim3(blocks_for(D, 256)), dim3(256), 0, st,
           (const __nv_bfloat16*)phi, N, D, ld, out);
}

cofem_status mlp_col_norms(const cofem_op* op, float* out, cudaStream_t st) {
  if (op_is_dense(op)) {
    const DenseDesc d = op_dense_desc(op);
    if (d.dtype == COFEM_FP8_E4M3)
      fp8_col_norms(d, out, st);
    else if (d.dtype == COFEM_F64)
      launch_k(col_norms_kernel<double>, dim3(blocks_for(d.D, 256)), dim3(256), 0, st,
               (const double*)d.phi, d.N, d.D, d.ld, out);
    else if (dense_applies_hilo(d))
      launch_k(col_norms_kernel<F32HiLo>, dim3(blocks_for(d.D, 256)), dim3(256), 0, st,
               (const F32HiLo*)d.phi, d.N, d.D, d.ld, out);
    else if (d.dtype == COFEM_F32)
      launch_k(col_norms_kernel<float>, dim3(blocks_for(d.D, 256)), dim3(256), 0, st,
               (const float*)d.phi, d.N, d.D, d.ld, out);
    else
      launch_k(col_norms_kernel<__nv_bfloat16>, dim3(blocks_for(d.D, 256)), dim3(256), 0, st,
               (const __nv_bfloat16*)d.phi, d.N, d.D, d.ld, out);
  } else {
    int64_t L;
    int C, T, bf16;
    const float* h;
    if (op_conv_desc(op, &L, &C, &T, &h, &bf16) != 0) return COFEM_ERR_UNSUPPORTED;
    launch_k(conv_col_norms_kernel, dim3(blocks_for((int64_t)C * L, 256)), dim3(256), 0, st, h, C,
             T, L, bf16, out);
  }
  return cudaGetLastError() == cudaSuccess ? COFEM_OK : COFEM_ERR_CUDA;
}

static size_t train_smem() {
  return (size_t)(1284 + kTrainS * 4 + 4 * kTrainS * 33 + kTrainS * 2) * sizeof(float);
}

}  // namespace cofem

using namespace cofem;

extern "C" cofem_status cofem_op_col_norms(const cofem_op* op, float* out_dev, void* stream) {
  if (!op || !out_dev) return COFEM_ERR_INVALID_ARG;
  return mlp_col_norms(op, out_dev, (cudaStream_t)stream);
}

extern "C" cofem_status cofem_mlp_features(const double* alpha_dev, const float* phinorm2_dev,
                                           double beta, const double* mu_prev_dev,
                                           const double* s_prev_dev, int64_t D, float* U_dev,
                                           void* stream) {
  if (!alpha_dev || !phinorm2_dev || !U_dev || D < 1 || !(beta > 0.0)) return COFEM_ERR_INVALID_ARG;
  launch_k(features_kernel, dim3(blocks_for(D, 256)), dim3(256), 0, (cudaStream_t)stream,
           alpha_dev, phinorm2_dev, beta, mu_prev_dev, s_prev_dev, D, U_dev);
  return cudaGetLastError() == cudaSuccess ? COFEM_OK : COFEM_ERR_CUDA;
}

extern "C" cofem_status cofem_mlp_targets(const double* alpha_dev, const float* phinorm2_dev,
                                          double beta, const double* mu_dev, const double* s_dev,
                                          int64_t D, float* Y_dev, void* stream) {
  if (!alpha_dev || !phinorm2_dev || !mu_dev || !s_dev || !Y_dev || D < 1)
    return COFEM_ERR_INVALID_ARG;
  launch_k(targets_kernel, dim3(blocks_for(D, 256)), dim3(256), 0, (cudaStream_t)stream,
           alpha_dev, phinorm2_dev, beta, mu_dev, s_dev, D, Y_dev);
  return cudaGetLastError() == cudaSuccess ? COFEM_OK : COFEM_ERR_CUDA;
}

extern "C" cofem_status cofem_mlp_forward(const void* weights_dev, cofem_dtype wdtype,
                                          const float* U_dev, int64_t n, float* O_dev,
                                          void* stream) {
  if (!weights_dev || !U_dev || !O_dev || n < 1) return COFEM_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (wdtype == COFEM_BF16)
    launch_k(mlp_forward_kernel<__nv_bfloat16>, dim3(blocks_for(n, 128)), dim3(128), 0, st,
             (const __nv_bfloat16*)weights_dev, U_dev, n, O_dev);
  else if (wdtype == COFEM_F32)
    launch_k(mlp_forward_kernel<float>, dim3(blocks_for(n, 128)), dim3(128), 0, st,
             (const float*)weights_dev, U_dev, n, O_dev);
  else
    return COFEM_ERR_INVALID_ARG;
  return cudaGetLastError() == cudaSuccess ? COFEM_OK : COFEM_ERR_CUDA;
}

extern "C" size_t cofem_mlp_train_workspace_bytes(int64_t n) {
  const int64_t nb = (n + kTrainS - 1) / kTrainS;
  return (size_t)(nb * kMlpParams * 4 + 255) / 256 * 256 + (size_t)(nb * 8 + 255) / 256 * 256;
}

// Shared by cofem_mlp_grad and cofem_mlp_adam_step.
static cofem_status train_pass(const void* w, cofem_dtype wdtype, const float* U, const float* Y,
                               int64_t n, void* ws, size_t ws_bytes, float* grad, double* loss,
                               float* master, float* m, float* v, __nv_bfloat16* wbf, int step,
                               float lr, cudaStream_t st) {
  if (!w || !U || !Y || n < 1 || !ws || ws_bytes < cofem_mlp_train_workspace_bytes(n))
    return COFEM_ERR_INVALID_ARG;
  const int64_t nb = (n + kTrainS - 1) / kTrainS;
  float* gpart = (float*)ws;
  double* lpart = (double*)((char*)ws + (size_t)(nb * kMlpParams * 4 + 255) / 256 * 256);
  const size_t sm = train_smem();
  cudaError_t e;
  if (wdtype == COFEM_BF16) {
    cudaFuncSetAttribute(mlp_train_kernel<__nv_bfloat16>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    e = launch_k(mlp_train_kernel<__nv_bfloat16>, dim3((unsigned)nb), dim3(kTrainS), sm, st,
                 (const __nv_bfloat16*)w, U, Y, n, gpart, lpart);
  } else if (wdtype == COFEM_F32) {
    cudaFuncSetAttribute(mlp_train_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sm);
    e = launch_k(mlp_train_kernel<float>, dim3((unsigned)nb), dim3(kTrainS), sm, st,
                 (const float*)w, U, Y, n, gpart, lpart);
  } else {
    return COFEM_ERR_INVALID_ARG;
  }
  if (e != cudaSuccess) return COFEM_ERR_CUDA;
  e = launch_k(mlp_reduce_adam_kernel, dim3((kMlpParams + 255) / 256), dim3(256), 0, st,
               (const float*)gpart, (int)nb, (const double*)lpart, 1.0 / (double)n, grad, loss,
               master, m, v, wbf, step, lr, 0.9f, 0.999f, 1e-8f);
  return e == cudaSuccess ? COFEM_OK : COFEM_ERR_CUDA;
}

extern "C" cofem_status cofem_mlp_grad(const void* weights_dev, cofem_dtype wdtype,
                                       const float* U_dev, const float* Y_dev, int64_t n,
                                       float* grad_dev, double* loss_dev, void* workspace_dev,
                                       size_t workspace_bytes, void* stream) {
  if (!grad_dev) return COFEM_ERR_INVALID_ARG;
  return train_pass(weights_dev, wdtype, U_dev, Y_dev, n, workspace_dev, workspace_bytes, grad_dev,
                    loss_dev, nullptr, nullptr, nullptr, nullptr, 0, 0.f, (cudaStream_t)stream);
}

extern "C" cofem_status cofem_mlp_adam_step(float* master_dev, float* m_dev, float* v_dev,
                                            void* weights_bf16_dev, const float* U_dev,
                                            const float* Y_dev, int64_t n, int32_t step, float lr,
                                            void* workspace_dev, size_t workspace_bytes,
                                            double* loss_dev, void* stream) {
  if (!master_dev || !m_dev || !v_dev || !weights_bf16_dev || step < 1) return COFEM_ERR_INVALID_ARG;
  return train_pass(weights_bf16_dev, COFEM_BF16, U_dev, Y_dev, n, workspace_dev, workspace_bytes,
                    nullptr, loss_dev, master_dev, m_dev, v_dev, (__nv_bfloat16*)weights_bf16_dev,
                    step, lr, (cudaStream_t)stream);
}
