// Host side of libcofem: operator handles, workspace layout, the per-EM-
// iteration CUDA graph of Algorithm 1, and the C ABI of include/cofem.h.
//
// One EM iteration is one graph launch:
//   init (probes hashed into B, X = 0, R = P = B, rho, ||B||)       Alg. 1 l.5-6
//   WHILE (not converged):                                           Sec. 3.2
//       Q = A P (+ gamma partials) ; a = rho / gamma ; x, r update
//       IF (residual replacement due): Q = A x ; r = B - Q
//       p = r + b p
//   diag estimate + M-step, statistics, t += 1                        Alg. 1 l.7-9
// The CG stop test runs on the device and drives the WHILE node through
// cudaGraphSetConditional, so the host never waits inside a fit.
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "dense.cuh"

struct cofem_op {
  int kind;                       // 0 dense, 1 conv, 2 masked DCT
  cofem::DenseDesc dense;
  int64_t L;
  int C, T;
  const float* filters;
  int conv_tc = 0;                // convolution on the tensor cores (BF16-rounded filters)
  int64_t dct_D, dct_N;           // masked DCT: D coefficients, N kept samples
  const int32_t* dct_idx;         // their indices (strictly increasing, caller's memory)
};

namespace cofem {

static thread_local std::string g_last_error;

static void set_error(const char* what, cudaError_t e, const char* file, int line) {
  char buf[512];
  snprintf(buf, sizeof(buf), "%s: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
  g_last_error = buf;
}

#define CK(x)                                                   \
  do {                                                          \
    cudaError_t e_ = (x);                                       \
    if (e_ != cudaSuccess) {                                    \
      cofem::set_error(#x, e_, __FILE__, __LINE__);             \
      return COFEM_ERR_CUDA;                                    \
    }                                                           \
  } while (0)

#define CKL()  CK(cudaGetLastError())

int num_sms() {
  static int cache[128] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 128) return 148;
  if (cache[dev] == 0) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    cache[dev] = n > 0 ? n : 148;
  }
  return cache[dev];
}

__global__ void ctl_init_kernel(CgCtl* ctl, long long t0) {
  pdl_wait();
  pdl_trigger();
  ctl->t = t0;
  ctl->em_index = 0;
  ctl->error = 0;
  unsigned long long now;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
  ctl->start_ns = now;
}

// alpha32[i] = (float)alpha[i]: the FP32 copy that the operators read
__global__ void alpha32_kernel(const double* alpha, int64_t n, float* alpha32) {
  pdl_wait();
  pdl_trigger();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    alpha32[i] = (float)alpha[i];
}

__global__ void fill_double_kernel(double* x, int64_t n, double v) {
  pdl_wait();
  pdl_trigger();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] = v;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static int vec_bytes(int vec) { return vec == COFEM_F64 ? 8 : 4; }

// ------------------------------------------------------------ operators

static bool use_tc(const cofem_op* op);

static bool op_supports(const cofem_op* op, int vec) {
  if (op->kind == 0) {
    if (vec == COFEM_F64) return op->dense.dtype == COFEM_F64;
    // FP8 dictionaries: tensor cores only (a packed copy attached)
    if (op->dense.dtype == COFEM_FP8_E4M3) return vec == COFEM_F32 && use_tc(op);
    if (vec == COFEM_F32) return op->dense.dtype == COFEM_F32 || op->dense.dtype == COFEM_BF16;
    return false;
  }
  return vec == COFEM_F32;     // convolution, masked DCT: FP32 vectors
}

// Convolution scratch: the filters padded to 64 taps (rounded to BF16 on the
// tensor cores), on the tensor cores the Toeplitz images (1024-aligned),
// then W (ncols x L floats), then an FP32 copy of alpha (C L floats) for
// applications given none.  The prefix does not depend on ncols, so tables
// prepared once (a fit) serve every application.
static size_t conv_prefix_bytes(const cofem_op* op) {
  size_t b = align256((size_t)op->C * 64 * sizeof(float));
  if (op->conv_tc) b = ((b + 1023) & ~(size_t)1023) + conv_tc_image_bytes(op->C);
  return b;
}
static __nv_bfloat16* conv_images(const cofem_op* op, char* ws) {
  return (__nv_bfloat16*)(ws + ((align256((size_t)op->C * 64 * sizeof(float)) + 1023) &
                                ~(size_t)1023));
}
static size_t conv_w_bytes(const cofem_op* op, int ncols) {
  return conv_prefix_bytes(op) + align256((size_t)ncols * op->L * sizeof(float)) +
         align256((size_t)op->C * op->L * sizeof(float));
}
static float* conv_alpha32_scratch(const cofem_op* op, char* ws, int ncols) {
  return (float*)(ws + conv_prefix_bytes(op) + align256((size_t)ncols * op->L * sizeof(float)));
}
static float* conv_w_scratch(const cofem_op* op, char* ws) {
  return (float*)(ws + conv_prefix_bytes(op));
}
// The filters the kernels read (taps as float4): the caller's in place when
// they are 64 taps long and 16-byte aligned and not rounded; otherwise the
// workspace copy, written here unless `prepared` (with the Toeplitz images
// on the tensor cores).
static const float* conv_filters64(const cofem_op* op, char* ws, cudaStream_t st,
                                   bool prepared = false) {
  if (!op->conv_tc && op->T == 64 && ((uintptr_t)op->filters & 15) == 0) return op->filters;
  float* h64 = (float*)ws;
  if (!prepared) {
    if (op->conv_tc) conv_tc_prepare(op->filters, op->C, op->T, h64, conv_images(op, ws), st);
    else conv_pad_filters(op->filters, op->C, op->T, h64, st);
  }
  return h64;
}

// Tensor cores: BF16 dictionaries (nterms > 0), and FP32 dictionaries with a
// packed two-term copy attached (Phi = hi + lo in BF16).
static bool use_tc(const cofem_op* op) {
  if (op->kind != 0 || op->dense.nterms <= 0) return false;
  if (op->dense.dtype == COFEM_BF16) return true;
  return (op->dense.dtype == COFEM_F32 || op->dense.dtype == COFEM_FP8_E4M3) && op->dense.packed;
}

// Scratch of one operator application.  For the tensor-core path it depends
// on the pipeline shape (split-K grows with CTAs per SM): `max_shape` sizes
// it for the largest shape the autotuner tries, otherwise for the handle's
// current shape.
static size_t op_ws_bytes(const cofem_op* op, int vec, int ncols, bool max_shape = false) {
  if (op->kind == 0) {
    DenseSimtPlan p = dense_simt_plan(op->dense.N, op->dense.D, ncols, vec_bytes(vec), num_sms());
    size_t b = align256(p.total());
    if (use_tc(op)) {
      DenseTcPlan q = dense_tc_plan(op->dense, ncols, num_sms());
      if (align256(q.total) > b) b = align256(q.total);
      for (int mt = 1; max_shape && mt <= 2; ++mt)
        for (int cps = 1; cps <= 4; ++cps) {
          DenseTcPlan r = dense_tc_plan(op->dense.N, op->dense.D, ncols, op->dense.nterms,
                                        num_sms(), cps, 0, op->dense.phi_terms, mt);
          if (align256(r.total) > b) b = align256(r.total);
        }
    }
    return b;
  }
  if (op->kind == 2) return dct_ws_bytes(op->dct_D, ncols);
  return conv_w_bytes(op, ncols);
}

// Y = beta Phi^T Phi X + alpha . X  (alpha may be null: no diagonal term)
static cofem_status op_apply(const cofem_op* op, int vec, const void* x, int64_t ld, int ncols,
                             const double* alpha, double beta, void* y, double* dots,
                             int* nparts, char* ws, cudaStream_t st, int* err = nullptr,
                             unsigned flags = 0u, const float* alpha32 = nullptr,
                             const int* gate = nullptr) {
  if (op->kind == 0) {
    const DenseDesc& d = op->dense;
    if (use_tc(op) && vec == COFEM_F32) {
      if (d.l2_resident_cols < 0) {
        // 60% of this device's L2 holds a fixed band of Phi's columns
        int dev = 0, l2 = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
        int64_t cols = (int64_t)(0.6 * (double)l2) / (d.N * 2) / 128 * 128;
        const_cast<cofem_op*>(op)->dense.l2_resident_cols = cols < d.D ? cols : d.D;
      }
      int rc = dense_tc_apply(d, d.nterms, (const float*)x, ld, ncols, (float*)y, beta, alpha,
                              dots, nparts, ws, err, flags, st, alpha32, gate);
      if (rc == 1) {
        g_last_error = "cuTensorMapEncodeTiled failed";
        return COFEM_ERR_CUDA;
      }
      CKL();
      return COFEM_OK;
    }
    if (vec == COFEM_F64)
      dense_simt_apply<double, double>(d, (const double*)x, ld, ncols, (double*)y, beta, alpha,
                                       dots, nparts, ws, st);
    else if (dense_applies_hilo(d))
      dense_simt_apply<F32HiLo, float>(d, (const float*)x, ld, ncols, (float*)y, beta, alpha,
                                       dots, nparts, ws, st);
    else if (d.dtype == COFEM_F32)
      dense_simt_apply<float, float>(d, (const float*)x, ld, ncols, (float*)y, beta, alpha,
                                     dots, nparts, ws, st);
    else
      dense_simt_apply<__nv_bfloat16, float>(d, (const float*)x, ld, ncols, (float*)y, beta,
                                             alpha, dots, nparts, ws, st);
    CKL();
    return COFEM_OK;
  }
  if (op->kind == 2) {
    const int np = dct_apply(op->dct_D, op->dct_idx, op->dct_N, (const float*)x, ld, ncols,
                             (float*)y, beta, alpha, vec == COFEM_F32 ? alpha32 : nullptr, dots,
                             ws, err, st, (flags & kApplyOpPrepared) != 0);
    if (nparts) *nparts = dots ? np : 0;
    CKL();
    return COFEM_OK;
  }
  const float* h64 = conv_filters64(op, ws, st, (flags & kApplyOpPrepared) != 0);
  float* W = conv_w_scratch(op, ws);
  const float* a32 = vec == COFEM_F32 ? alpha32 : nullptr;
  if (!a32 && alpha) {
    float* t = conv_alpha32_scratch(op, ws, ncols);
    conv_alpha_f32(alpha, (int64_t)op->C * op->L, t, st);
    a32 = t;
  }
  if (op->conv_tc) {
    const __nv_bfloat16* img = conv_images(op, ws);
    conv_tc_forward(op->C, op->L, (const float*)x, ld, ncols, W, op->L, img, err, st);
    const int np = conv_tc_adjoint(op->C, op->L, W, op->L, ncols, (float*)y, ld, beta, alpha,
                                   a32, (const float*)x, dots, img, err, st);
    if (nparts) *nparts = dots ? np : 0;
    CKL();
    return COFEM_OK;
  }
  conv_forward(h64, op->C, op->L, (const float*)x, ld, ncols, W, op->L, st);
  const int np = conv_adjoint(h64, op->C, op->L, W, op->L, ncols, (float*)y, ld, beta, alpha,
                              (const float*)x, dots, st, a32);
  if (nparts) *nparts = dots ? np : 0;
  CKL();
  return COFEM_OK;
}

// W = Phi Z
static cofem_status op_forward(const cofem_op* op, int vec, const void* z, int64_t ldz,
                               int ncols, void* w, int64_t ldw, char* ws, cudaStream_t st) {
  if (op->kind == 0) {
    const DenseDesc& d = op->dense;
    if (d.dtype == COFEM_FP8_E4M3)
      fp8_forward(d, (const float*)z, ldz, ncols, (float*)w, ldw, st);
    else if (vec == COFEM_F64)
      dense_simt_forward<double, double>(d, (const double*)z, ldz, ncols, (double*)w, ldw, ws, st);
    else if (dense_applies_hilo(d))
      dense_simt_forward<F32HiLo, float>(d, (const float*)z, ldz, ncols, (float*)w, ldw, ws, st);
    else if (d.dtype == COFEM_F32)
      dense_simt_forward<float, float>(d, (const float*)z, ldz, ncols, (float*)w, ldw, ws, st);
    else
      dense_simt_forward<__nv_bfloat16, float>(d, (const float*)z, ldz, ncols, (float*)w, ldw,
                                               ws, st);
    CKL();
    return COFEM_OK;
  }
  if (op->kind == 2) {
    dct_forward(op->dct_D, op->dct_idx, op->dct_N, (const float*)z, ldz, ncols, (float*)w, ldw,
                ws, nullptr, st);
    CKL();
    return COFEM_OK;
  }
  const float* h64 = conv_filters64(op, ws, st);
  conv_forward(h64, op->C, op->L, (const float*)z, ldz, ncols, (float*)w, ldw, st);
  CKL();
  return COFEM_OK;
}

// Z = beta Phi^T W
static cofem_status op_adjoint(const cofem_op* op, int vec, const void* w, int64_t ldw,
                               int ncols, void* z, int64_t ldz, double beta, char* ws,
                               cudaStream_t st) {
  if (op->kind == 0) {
    const DenseDesc& d = op->dense;
    if (d.dtype == COFEM_FP8_E4M3)
      fp8_adjoint(d, (const float*)w, ldw, ncols, (float*)z, ldz, beta, st);
    else if (vec == COFEM_F64)
      dense_simt_adjoint<double, double>(d, (const double*)w, ldw, ncols, (double*)z, ldz, beta,
                                         nullptr, nullptr, nullptr, nullptr, ws, st);
    else if (dense_applies_hilo(d))
      dense_simt_adjoint<F32HiLo, float>(d, (const float*)w, ldw, ncols, (float*)z, ldz, beta,
                                         nullptr, nullptr, nullptr, nullptr, ws, st);
    else if (d.dtype == COFEM_F32)
      dense_simt_adjoint<float, float>(d, (const float*)w, ldw, ncols, (float*)z, ldz, beta,
                                       nullptr, nullptr, nullptr, nullptr, ws, st);
    else
      dense_simt_adjoint<__nv_bfloat16, float>(d, (const float*)w, ldw, ncols, (float*)z, ldz,
                                               beta, nullptr, nullptr, nullptr, nullptr, ws, st);
    CKL();
    return COFEM_OK;
  }
  if (op->kind == 2) {
    dct_adjoint(op->dct_D, op->dct_idx, op->dct_N, (const float*)w, ldw, ncols, (float*)z, ldz,
                beta, ws, nullptr, st);
    CKL();
    return COFEM_OK;
  }
  const float* h64 = conv_filters64(op, ws, st);
  conv_adjoint(h64, op->C, op->L, (const float*)w, ldw, ncols, (float*)z, ldz, beta, nullptr,
               nullptr, nullptr, st);
  CKL();
  return COFEM_OK;
}

static int64_t op_N(const cofem_op* op) {
  return op->kind == 0 ? op->dense.N : op->kind == 2 ? op->dct_N : op->L;
}
static int64_t op_D(const cofem_op* op) {
  return op->kind == 0 ? op->dense.D : op->kind == 2 ? op->dct_D : (int64_t)op->C * op->L;
}

// --------------------------------------------------------------- layout

struct FitLayout {
  size_t ctl, sc, pdots, pvec, pvec2, pvec3, minv, pn2, alpha32, X, R, P, Q, b, yblk, st_iters,
      st_relres, st_clamps, st_support, st_end, bcg, opws;
  size_t total;
  int64_t ld;
};

// Tasks sharing alpha (1 = the paper's single-task model).
static int n_tasks(const cofem_params* p) { return p->tasks > 1 ? p->tasks : 1; }

static FitLayout fit_layout(const cofem_op* op, const cofem_params* p) {
  FitLayout L;
  const int T = n_tasks(p);
  const int ncols = p->K + T;
  const int vb = vec_bytes(p->vec_dtype);
  L.ld = round_up(op_D(op), kLdAlign);
  const size_t blk = align256((size_t)ncols * L.ld * vb);
  const int ne = p->em_iters > 0 ? p->em_iters : 1;
  size_t o = 0;
  L.ctl = o; o += align256(sizeof(CgCtl));
  L.sc = o; o += align256(sizeof(CgScalars));
  L.pdots = o; o += align256(sizeof(double) * kMaxParts * kMaxCols);
  L.pvec = o; o += align256(sizeof(double) * kMaxParts * kMaxCols);
  L.pvec2 = o; o += align256(sizeof(double) * kMaxParts * kMaxCols);
  L.pvec3 = o; o += align256(sizeof(double) * kMaxParts * kMaxCols);
  L.minv = o; o += align256((size_t)L.ld * sizeof(float));
  L.pn2 = o; o += align256((size_t)L.ld * sizeof(float));
  L.alpha32 = o; o += align256((size_t)L.ld * sizeof(float));
  L.X = o; o += blk;
  L.R = o; o += blk;
  L.P = o; o += blk;
  L.Q = o; o += blk;
  L.b = o; o += align256((size_t)T * L.ld * vb);
  // multi-task: the T observation vectors at a 64-element pitch
  L.yblk = o; o += T > 1 ? align256((size_t)T * round_up(op_N(op), kLdAlign) * vb) : 0;
  L.st_iters = o; o += align256(sizeof(int32_t) * ne);
  L.st_relres = o; o += align256(sizeof(double) * ne);
  L.st_clamps = o; o += align256(sizeof(int32_t) * ne);
  L.st_support = o; o += align256(sizeof(int32_t) * ne);
  L.st_end = o; o += align256(sizeof(int64_t) * ne);
  // block CG: its m x m matrices, counters and Gram partial sums
  L.bcg = o; o += p->solver == 1 ? align256(bcg_state_bytes(vb, ncols, L.ld)) : 0;
  L.opws = o;
  size_t ows = op_ws_bytes(op, p->vec_dtype, ncols);
  size_t ows1 = op_ws_bytes(op, p->vec_dtype, 1);
  o += ows > ows1 ? ows : ows1;
  L.total = o;
  return L;
}

static cofem_status check_params(const cofem_op* op, const cofem_params* p) {
  if (!op || !p) return COFEM_ERR_INVALID_ARG;
  if (p->K < 1 || p->tasks < 0 || p->K + n_tasks(p) > kMaxCols) return COFEM_ERR_INVALID_ARG;
  if (p->em_iters < 0 || p->cg_max_iters < 1 || p->fixed_cg_iters < 0) return COFEM_ERR_INVALID_ARG;
  if (p->resid_replace_every < 0) return COFEM_ERR_INVALID_ARG;
  if (p->vec_dtype != COFEM_F64 && p->vec_dtype != COFEM_F32) return COFEM_ERR_INVALID_ARG;
  if (!(p->cg_tol >= 0.0) || !(p->den_floor > 0.0)) return COFEM_ERR_INVALID_ARG;
  if (p->t_offset < 0) return COFEM_ERR_INVALID_ARG;
  if (p->stop_rule != 0 && p->stop_rule != 1) return COFEM_ERR_INVALID_ARG;
  if (p->solver != 0 && p->solver != 1) return COFEM_ERR_INVALID_ARG;
  if (!op_supports(op, p->vec_dtype)) return COFEM_ERR_UNSUPPORTED;
  // block CG: the joint stop test on its own recurrence, nothing else
  if (p->solver == 1 && (p->resid_replace_every > 0 || p->stop_rule != 0 || p->mlp))
    return COFEM_ERR_UNSUPPORTED;
  if (p->mlp && p->vec_dtype != COFEM_F32) return COFEM_ERR_UNSUPPORTED;
  if (p->mlp && p->stop_rule == 1) return COFEM_ERR_UNSUPPORTED;
  if (p->mlp && n_tasks(p) > 1) return COFEM_ERR_UNSUPPORTED;
  // the tensor-core operator writes one partial dot per 128-row tile of D
  // (plus one when two tiles share a unit and their count is odd)
  if (use_tc(op) && p->vec_dtype == COFEM_F32 && (op->dense.D + 127) / 128 + 1 > kMaxParts)
    return COFEM_ERR_UNSUPPORTED;
  return COFEM_OK;
}

static thread_local int g_last_fallbacks = 0;
void set_last_fit_fallbacks(int n) { g_last_fallbacks = n; }
cofem_status mlp_col_norms(const cofem_op* op, float* out, cudaStream_t st);

// ---------------------------------------------------------------- graph

struct Streams {
  cudaStream_t s[3] = {nullptr, nullptr, nullptr};
  ~Streams() {
    for (auto x : s)
      if (x) cudaStreamDestroy(x);
  }
};

static cofem_status add_conditional(cudaStream_t cs, cudaGraphConditionalHandle h,
                                    cudaGraphConditionalNodeType type, cudaGraph_t* body) {
  cudaStreamCaptureStatus status;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  CK(cudaStreamGetCaptureInfo(cs, &status, nullptr, &g, &deps, nullptr, &ndeps));
  if (status != cudaStreamCaptureStatusActive) return COFEM_ERR_CUDA;
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = type;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  CK(cudaGraphAddNode(&node, g, deps, nullptr, ndeps, &np));
  *body = np.conditional.phGraph_out[0];
  CK(cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  return COFEM_OK;
}

template <typename V>
static cofem_status build_em_graph(const cofem_op* op, const cofem_params* p, double beta,
                                   char* ws, const FitLayout& L, double* mu, double* s,
                                   double* alpha, cudaGraphExec_t* exec) {
  // structured operators: their tables were built once for the fit
  const unsigned prep = (op->kind == 2 || (op->kind == 1 && op->conv_tc)) ? kApplyOpPrepared : 0u;
  Streams ss;
  for (auto& x : ss.s) CK(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
  CgCtl* ctl = (CgCtl*)(ws + L.ctl);
  CgScalars* sc = (CgScalars*)(ws + L.sc);
  double* pdots = (double*)(ws + L.pdots);
  double* pvec = (double*)(ws + L.pvec);
  double* pvec2 = (double*)(ws + L.pvec2);
  double* pvec3 = (double*)(ws + L.pvec3);
  V* X = (V*)(ws + L.X);
  V* R = (V*)(ws + L.R);
  V* P = (V*)(ws + L.P);
  V* Q = (V*)(ws + L.Q);
  V* b = (V*)(ws + L.b);
  char* opws = ws + L.opws;
  const int ncols = p->K + n_tasks(p);
  const int vec = p->vec_dtype;

  CgConf cf;
  memset(&cf, 0, sizeof(cf));
  cf.D = op_D(op);
  cf.ld = L.ld;
  cf.ncols = ncols;
  cf.K = p->K;
  cf.T = n_tasks(p);
  cf.seed = p->seed;
  cf.tol = p->cg_tol;
  cf.max_iters = p->cg_max_iters;
  cf.fixed_iters = p->fixed_cg_iters;
  cf.stop_rule = p->fixed_cg_iters > 0 ? 0 : p->stop_rule;
  cf.replace_every = p->resid_replace_every;
  cf.beta = beta;
  cf.den_floor = p->den_floor;
  cf.support_threshold = p->support_threshold;
  cf.em_iters = p->em_iters;
  cf.st_end_ns = (long long*)(ws + L.st_end);
  float* alpha32 = vec == COFEM_F32 ? (float*)(ws + L.alpha32) : nullptr;
  cf.alpha32 = alpha32;
  if (use_tc(op) && vec == COFEM_F32) {
    // the CG kernels write P's BF16 terms straight into the operator's
    // split buffer, so the operator skips its own split of P
    DenseTcPlan tp = dense_tc_plan(op->dense, ncols, num_sms());
    cf.split_nt = op->dense.nterms;
    cf.split_rows = tp.BN;
    cf.split_buf = opws + tp.off_xs;
  }

  cudaStream_t cs = ss.s[0];
  CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
  cudaStreamCaptureStatus status;
  cudaGraph_t g = nullptr;
  CK(cudaStreamGetCaptureInfo(cs, &status, nullptr, &g, nullptr, nullptr, nullptr));
  cudaGraphConditionalHandle hw;
  CK(cudaGraphConditionalHandleCreate(&hw, g, 0, cudaGraphCondAssignDefault));
  cf.while_handle = (unsigned long long)hw;

  const bool learned = p->mlp != nullptr;
  cudaGraphConditionalHandle hf = 0;
  if (learned) {
    // warm start X0 and M^-1 from the network; Q = A X0; preconditioned start
    CK(cudaGraphConditionalHandleCreate(&hf, g, 0, cudaGraphCondAssignDefault));
    cf.fallback_handle = (unsigned long long)hf;
    cf.minv = (const float*)(ws + L.minv);
    if constexpr (sizeof(V) == 4) {
      launch_warm_start(cf, ctl, (long long)(p->t_offset + 1), (const __nv_bfloat16*)p->mlp,
                        alpha, (const float*)(ws + L.pn2), mu, s, (float*)X,
                        (float*)(ws + L.minv), cs);
    }
    CKL();
    cofem_status rw = op_apply(op, vec, X, L.ld, ncols, alpha, beta, Q, nullptr, nullptr, opws,
                               cs, &ctl->error, prep, alpha32);
    if (rw != COFEM_OK) return rw;
    launch_cg_init_warm<V>(cf, ctl, sc, X, R, P, Q, b, pvec, pvec2, pvec3, cs);
  } else if (p->solver == 1) {
    CK(launch_bcg_start<V>(cf, ctl, ws + L.bcg, X, R, P, b, cs));
  } else {
    launch_cg_init<V>(cf, ctl, sc, X, R, P, b, pvec, cs);
  }
  CKL();
  cudaGraph_t body = nullptr;
  cofem_status rc = add_conditional(cs, hw, cudaGraphCondTypeWhile, &body);
  if (rc != COFEM_OK) return rc;

  if (p->solver == 1) {
    // ---- block CG: Z = A P (into Q), then its gram passes and row pass
    cudaStream_t bs = ss.s[1];
    CK(cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    rc = op_apply(op, vec, P, L.ld, ncols, alpha, beta, Q, nullptr, nullptr, opws, bs,
                  &ctl->error, (cf.split_nt > 0 ? kApplyPresplit : 0u) | prep, alpha32);
    if (rc != COFEM_OK) return rc;
    CK(launch_bcg_iteration<V>(cf, ctl, ws + L.bcg, X, R, P, Q, bs));
    cudaGraph_t tmp;
    CK(cudaStreamEndCapture(bs, &tmp));
    launch_diag_mstep<V>(cf, ctl, 0, X, mu, s, alpha, nullptr, (int32_t*)(ws + L.st_iters),
                         (double*)(ws + L.st_relres), (int32_t*)(ws + L.st_clamps),
                         (int32_t*)(ws + L.st_support), cs);
    CKL();
    cudaGraph_t graph;
    CK(cudaStreamEndCapture(cs, &graph));
    cudaError_t e = cudaGraphInstantiate(exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      set_error("cudaGraphInstantiate", e, __FILE__, __LINE__);
      return COFEM_ERR_CUDA;
    }
    return COFEM_OK;
  }

  // ---- WHILE body.  Tensor-core operator with residual replacement: the
  // body is an inner WHILE loop of plain CG iterations, left when the
  // replacement is due (or the solve is done), followed by the replacement
  // (operator on X, true residual, stop test, direction), whose kernels run
  // only when it is due (gated on ctl->replace / ctl->run).  This keeps the
  // IF node's cost out of every iteration.  Otherwise one CG iteration, with
  // the replacement behind an IF node.
  const bool nested = p->resid_replace_every > 0 && use_tc(op) && vec == COFEM_F32;
  cudaGraphConditionalHandle hi = 0;
  if (nested) {
    cudaStream_t bs = ss.s[1];
    cudaGraphConditionalHandle hin;
    CK(cudaGraphConditionalHandleCreate(&hin, body, 1, cudaGraphCondAssignDefault));
    cf.inner_handle = (unsigned long long)hin;
    CK(cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    cudaGraph_t inner = nullptr;
    rc = add_conditional(bs, hin, cudaGraphCondTypeWhile, &inner);
    if (rc != COFEM_OK) return rc;
    {
      // two CG iterations per pass of the inner loop (half the loop's back
      // edges); the second copy's kernels return at once when the first
      // ended the solve or a replacement is due (ctl->run == 0)
      cudaStream_t is = ss.s[2];
      CK(cudaStreamBeginCaptureToGraph(is, inner, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
      for (int copy = 0; copy < 2; ++copy) {
        int nparts = 0;
        rc = op_apply(op, vec, P, L.ld, ncols, alpha, beta, Q, pdots, &nparts, opws, is,
                      &ctl->error, kApplyPresplit | prep, alpha32, copy ? &ctl->run : nullptr);
        if (rc != COFEM_OK) return rc;
        cf.gamma_parts = nparts;
        CgConf cc = cf;
        cc.gate_run = copy;
        if (!launch_cg_update<V>(cc, ctl, sc, X, R, P, Q, pdots, pvec, pvec2, is, true))
          launch_cg_direction<V>(cc, ctl, sc, R, P, is);
      }
      CKL();
      cudaGraph_t tmp;
      CK(cudaStreamEndCapture(is, &tmp));
    }
    rc = op_apply(op, vec, X, L.ld, ncols, alpha, beta, Q, nullptr, nullptr, opws, bs,
                  &ctl->error, prep, alpha32, &ctl->replace);
    if (rc != COFEM_OK) return rc;
    launch_cg_true_resid<V>(cf, ctl, sc, R, Q, b, pvec, pvec2, bs);
    launch_cg_direction<V>(cf, ctl, sc, R, P, bs);
    CKL();
    cudaGraph_t tmp;
    CK(cudaStreamEndCapture(bs, &tmp));
  } else {
    if (p->resid_replace_every > 0) {
      CK(cudaGraphConditionalHandleCreate(&hi, body, 0, cudaGraphCondAssignDefault));
      cf.if_handle = (unsigned long long)hi;
    }
    cudaStream_t bs = ss.s[1];
    CK(cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    int nparts = 0;
    rc = op_apply(op, vec, P, L.ld, ncols, alpha, beta, Q, pdots, &nparts, opws, bs,
                  &ctl->error, (cf.split_nt > 0 ? kApplyPresplit : 0u) | prep, alpha32);
    if (rc != COFEM_OK) return rc;
    cf.gamma_parts = nparts;
    // with a replacement IF node the direction update follows the IF (it
    // also closes a replacement iteration), so it stays a kernel of its own
    const bool fused = launch_cg_update<V>(cf, ctl, sc, X, R, P, Q, pdots, pvec, pvec2, bs,
                                           p->resid_replace_every <= 0);
    CKL();
    if (p->resid_replace_every > 0) {
      cudaGraph_t ibody = nullptr;
      rc = add_conditional(bs, hi, cudaGraphCondTypeIf, &ibody);
      if (rc != COFEM_OK) return rc;
      cudaStream_t is = ss.s[2];
      CK(cudaStreamBeginCaptureToGraph(is, ibody, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
      rc = op_apply(op, vec, X, L.ld, ncols, alpha, beta, Q, nullptr, nullptr, opws, is,
                    &ctl->error, prep, alpha32);
      if (rc != COFEM_OK) return rc;
      launch_cg_true_resid<V>(cf, ctl, sc, R, Q, b, pvec, pvec2, is);
      CKL();
      cudaGraph_t tmp;
      CK(cudaStreamEndCapture(is, &tmp));
    }
    if (!fused) launch_cg_direction<V>(cf, ctl, sc, R, P, bs);
    CKL();
    cudaGraph_t tmp;
    CK(cudaStreamEndCapture(bs, &tmp));
  }

  // ---- learned path: plain CG from zero when the preconditioned solve failed
  if (learned) {
    cudaGraph_t fbody = nullptr;
    rc = add_conditional(cs, hf, cudaGraphCondTypeIf, &fbody);
    if (rc != COFEM_OK) return rc;
    cudaStream_t fs = ss.s[1];
    CK(cudaStreamBeginCaptureToGraph(fs, fbody, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    cudaGraphConditionalHandle hw2;
    CK(cudaGraphConditionalHandleCreate(&hw2, fbody, 0, cudaGraphCondAssignDefault));
    CgConf pf = cf;
    pf.minv = nullptr;
    pf.fallback_handle = 0;
    pf.fallback_init = 1;
    pf.while_handle = (unsigned long long)hw2;
    pf.if_handle = 0;
    pf.inner_handle = 0;
    pf.replace_every = 0;
    launch_cg_init<V>(pf, ctl, sc, X, R, P, b, pvec, fs);
    CKL();
    cudaGraph_t fwhile = nullptr;
    rc = add_conditional(fs, hw2, cudaGraphCondTypeWhile, &fwhile);
    if (rc != COFEM_OK) return rc;
    cudaStream_t ws2 = ss.s[2];
    CK(cudaStreamBeginCaptureToGraph(ws2, fwhile, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    int np2 = 0;
    rc = op_apply(op, vec, P, L.ld, ncols, alpha, beta, Q, pdots, &np2, opws, ws2, &ctl->error,
                  (pf.split_nt > 0 ? kApplyPresplit : 0u) | prep, alpha32);
    if (rc != COFEM_OK) return rc;
    pf.gamma_parts = np2;
    if (!launch_cg_update<V>(pf, ctl, sc, X, R, P, Q, pdots, pvec, pvec2, ws2, true))
      launch_cg_direction<V>(pf, ctl, sc, R, P, ws2);
    CKL();
    cudaGraph_t tmp1, tmp2;
    CK(cudaStreamEndCapture(ws2, &tmp1));
    CK(cudaStreamEndCapture(fs, &tmp2));
  }

  // ---- after the solve: diagonal estimate + M-step + statistics
  launch_diag_mstep<V>(cf, ctl, 0, X, mu, s, alpha, nullptr, (int32_t*)(ws + L.st_iters),
                       (double*)(ws + L.st_relres), (int32_t*)(ws + L.st_clamps),
                       (int32_t*)(ws + L.st_support), cs);
  CKL();
  cudaGraph_t graph;
  CK(cudaStreamEndCapture(cs, &graph));
  cudaError_t e = cudaGraphInstantiate(exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    set_error("cudaGraphInstantiate", e, __FILE__, __LINE__);
    return COFEM_ERR_CUDA;
  }
  return COFEM_OK;
}

template <typename V>
static cofem_status fit_impl(const cofem_op* op, const void* y, double beta,
                             const cofem_params* p, char* ws, const FitLayout& L, double* mu,
                             double* s, double* alpha, cofem_stats* stats, cudaStream_t st) {
  const int64_t D = op_D(op), N = op_N(op);
  CK(cudaMemsetAsync(ws, 0, L.total, st));
  launch_k(ctl_init_kernel, dim3(1), dim3(1), 0, st, (CgCtl*)(ws + L.ctl), p->t_offset + 1);
  CKL();
  if (p->t_offset == 0) {
    launch_k(fill_double_kernel, dim3((unsigned)((D + 255) / 256 < 4096 ? (D + 255) / 256 : 4096)), dim3(256), 0, st, alpha, D, p->alpha_init);
    CKL();
  }
  if (p->vec_dtype == COFEM_F32) {
    // the M-step keeps this copy current from here on
    launch_k(alpha32_kernel, dim3((unsigned)((D + 255) / 256 < 4096 ? (D + 255) / 256 : 4096)), dim3(256), 0, st, (const double*)alpha, D, (float*)(ws + L.alpha32));
    CKL();
  }
  // b_t = beta Phi^T y_t  (once per fit: y and beta do not change); T > 1
  // tasks are first copied to a 64-element pitch
  const int T = n_tasks(p);
  const void* ysrc = y;
  int64_t ldy = N;
  if (T > 1) {
    ldy = round_up(N, kLdAlign);
    CK(cudaMemcpy2DAsync(ws + L.yblk, (size_t)ldy * sizeof(V), y, (size_t)N * sizeof(V),
                         (size_t)N * sizeof(V), (size_t)T, cudaMemcpyDeviceToDevice, st));
    ysrc = ws + L.yblk;
  }
  cofem_status rc = op_adjoint(op, p->vec_dtype, ysrc, ldy, T, ws + L.b, L.ld, beta,
                               ws + L.opws, st);
  if (rc != COFEM_OK) return rc;
  // the masked DCT's column norms for the learned start (one DCT of the
  // mask; X and R serve as scratch before the solve), then its mask and
  // twiddle tables, once per fit (the graph's applications reuse them)
  if (op->kind == 2 && p->mlp) {
    dct_col_norms(op->dct_D, op->dct_idx, op->dct_N, (float*)(ws + L.X), (float*)(ws + L.R),
                  ws + L.opws, &((CgCtl*)(ws + L.ctl))->error, (float*)(ws + L.pn2), st);
    CKL();
  }
  if (op->kind == 2) {
    dct_prepare(op->dct_D, op->dct_idx, op->dct_N, p->K + T, ws + L.opws,
                &((CgCtl*)(ws + L.ctl))->error, st);
    CKL();
  }

  if (p->mlp && op->kind != 2) {
    rc = mlp_col_norms(op, (float*)(ws + L.pn2), st);
    if (rc != COFEM_OK) return rc;
  }
  if (p->em_iters > 0) {
    cudaGraphExec_t exec = nullptr;
    rc = build_em_graph<V>(op, p, beta, ws, L, mu, s, alpha, &exec);
    if (rc != COFEM_OK) {
      if (exec) cudaGraphExecDestroy(exec);
      return rc;
    }
    for (int t = 0; t < p->em_iters; ++t) {
      cudaError_t e = cudaGraphLaunch(exec, st);
      if (e != cudaSuccess) {
        set_error("cudaGraphLaunch", e, __FILE__, __LINE__);
        cudaGraphExecDestroy(exec);
        return COFEM_ERR_CUDA;
      }
    }
    cudaError_t e = cudaStreamSynchronize(st);
    cudaGraphExecDestroy(exec);
    if (e != cudaSuccess) {
      set_error("cudaStreamSynchronize", e, __FILE__, __LINE__);
      return COFEM_ERR_CUDA;
    }
  } else {
    CK(cudaStreamSynchronize(st));
  }
  CgCtl hctl;
  CK(cudaMemcpy(&hctl, ws + L.ctl, sizeof(hctl), cudaMemcpyDeviceToHost));
  g_last_fallbacks = hctl.fallbacks;
  if (stats && p->em_iters > 0) {
    const int n = p->em_iters;
    if (stats->cg_iters) CK(cudaMemcpy(stats->cg_iters, ws + L.st_iters, 4 * n, cudaMemcpyDeviceToHost));
    if (stats->relres) CK(cudaMemcpy(stats->relres, ws + L.st_relres, 8 * n, cudaMemcpyDeviceToHost));
    if (stats->clamps) CK(cudaMemcpy(stats->clamps, ws + L.st_clamps, 4 * n, cudaMemcpyDeviceToHost));
    if (stats->support) CK(cudaMemcpy(stats->support, ws + L.st_support, 4 * n, cudaMemcpyDeviceToHost));
    if (stats->end_ns) CK(cudaMemcpy(stats->end_ns, ws + L.st_end, 8 * n, cudaMemcpyDeviceToHost));
  }
  if (hctl.error != 0) return (cofem_status)hctl.error;
  return COFEM_OK;
}

}  // namespace cofem

// ===================================================================== ABI
using namespace cofem;

extern "C" {

const char* cofem_status_string(cofem_status s) {
  switch (s) {
    case COFEM_OK: return "ok";
    case COFEM_ERR_INVALID_ARG: return "invalid argument";
    case COFEM_ERR_CUDA: return "CUDA error";
    case COFEM_ERR_NONFINITE: return "non-finite value";
    case COFEM_ERR_BREAKDOWN: return "CG breakdown (p^T A p <= 0)";
    case COFEM_ERR_TIMEOUT: return "device wait timed out";
    case COFEM_ERR_UNSUPPORTED: return "unsupported combination";
    case COFEM_ERR_WORKSPACE: return "workspace too small";
  }
  return "unknown status";
}

const char* cofem_last_error(void) { return g_last_error.c_str(); }

int32_t cofem_last_fit_fallbacks(void) { return g_last_fallbacks; }

cofem_status cofem_selftest_wait_timeout(int64_t limit_ns, void* stream) {
  if (limit_ns < 1000 || limit_ns > 1000000000) return COFEM_ERR_INVALID_ARG;
  const int r = wait_selftest(limit_ns, (cudaStream_t)stream);
  if (r < 0) {
    set_error("wait self-test", cudaGetLastError(), __FILE__, __LINE__);
    return COFEM_ERR_CUDA;
  }
  return r == 0 ? COFEM_OK : (cofem_status)r;
}

size_t cofem_bench_cg_kernels_workspace_bytes(int64_t D, int32_t ncols) {
  if (D < 1 || ncols < 2 || ncols > kMaxCols) return 0;
  return cg_kernels_bench_bytes(D, ncols);
}

cofem_status cofem_bench_cg_kernels(int64_t D, int32_t ncols, int32_t reps, void* workspace_dev,
                                    size_t workspace_bytes, void* stream, float* ms_out) {
  if (D < 1 || ncols < 2 || ncols > kMaxCols || reps < 1 || !workspace_dev || !ms_out)
    return COFEM_ERR_INVALID_ARG;
  if (workspace_bytes < cg_kernels_bench_bytes(D, ncols)) return COFEM_ERR_WORKSPACE;
  if (cg_kernels_bench(D, ncols, reps, (char*)workspace_dev, (cudaStream_t)stream, ms_out) != 0) {
    set_error("CG kernel timing", cudaGetLastError(), __FILE__, __LINE__);
    return COFEM_ERR_CUDA;
  }
  return COFEM_OK;
}

size_t cofem_bench_bcg_kernels_workspace_bytes(int64_t D, int32_t ncols) {
  if (D < 1 || ncols < 2 || ncols > kMaxCols) return 0;
  return bcg_bench_bytes(D, ncols);
}

cofem_status cofem_bench_bcg_kernels(int64_t D, int32_t ncols, int32_t reps, void* workspace_dev,
                                     size_t workspace_bytes, void* stream, float* ms_out) {
  if (D < 1 || ncols < 2 || ncols > kMaxCols || reps < 1 || !workspace_dev || !ms_out)
    return COFEM_ERR_INVALID_ARG;
  if (workspace_bytes < bcg_bench_bytes(D, ncols)) return COFEM_ERR_WORKSPACE;
  if (bcg_kernels_bench(D, ncols, reps, (char*)workspace_dev, (cudaStream_t)stream, ms_out) != 0) {
    set_error("block CG kernel timing", cudaGetLastError(), __FILE__, __LINE__);
    return COFEM_ERR_CUDA;
  }
  return COFEM_OK;
}

size_t cofem_selftest_cg_update_workspace_bytes(void) { return cg_update_selftest_bytes(); }

cofem_status cofem_selftest_cg_update_timeout(int64_t limit_ns, void* workspace_dev,
                                              size_t workspace_bytes, void* stream) {
  if (limit_ns < 1000 || limit_ns > 1000000000 || !workspace_dev) return COFEM_ERR_INVALID_ARG;
  if (workspace_bytes < cg_update_selftest_bytes()) return COFEM_ERR_WORKSPACE;
  const int r = cg_update_selftest(limit_ns, (char*)workspace_dev, (cudaStream_t)stream);
  if (r < 0) {
    set_error("CG update self-test", cudaGetLastError(), __FILE__, __LINE__);
    return COFEM_ERR_CUDA;
  }
  return r == 0 ? COFEM_OK : (cofem_status)r;
}

cofem_status cofem_op_dense(int64_t N, int64_t D, cofem_dtype dtype, const void* phi_dev,
                            int64_t ld, const float* tile_scales_dev, cofem_op** out) {
  if (!out || !phi_dev || N < 1 || D < 1 || ld < D) return COFEM_ERR_INVALID_ARG;
  if (dtype != COFEM_F64 && dtype != COFEM_F32 && dtype != COFEM_BF16 && dtype != COFEM_FP8_E4M3)
    return COFEM_ERR_INVALID_ARG;
  if (dtype == COFEM_FP8_E4M3 && (!tile_scales_dev || ((uintptr_t)tile_scales_dev & 3)))
    return COFEM_ERR_INVALID_ARG;
  if ((dtype == COFEM_BF16 || dtype == COFEM_FP8_E4M3) &&
      (ld % 64 != 0 || ((uintptr_t)phi_dev & 255)))
    return COFEM_ERR_INVALID_ARG;
  if ((uintptr_t)phi_dev & 15) return COFEM_ERR_INVALID_ARG;
  cofem_op* op = new cofem_op();
  op->kind = 0;
  op->dense.N = N;
  op->dense.D = D;
  op->dense.ld = ld;
  op->dense.dtype = dtype;
  op->dense.phi = phi_dev;
  op->dense.scales = tile_scales_dev;
  op->dense.nterms = (dtype == COFEM_BF16 || dtype == COFEM_FP8_E4M3) ? 3 : 0;
  op->dense.l2_resident_cols = 0;            // stream all of Phi (see the setter)
  op->dense.packed = nullptr;
  op->dense.tc_ctas_per_sm = 0;
  op->dense.tc_stages = 0;
  op->dense.phi_terms = dtype == COFEM_F32 ? 2 : 1;
  op->dense.tc_row_tiles = 1;
  *out = op;
  return COFEM_OK;
}

cofem_status cofem_op_dense_set_pipeline(cofem_op* op, int32_t stages, int32_t ctas_per_sm) {
  if (!op || op->kind != 0 || stages < 0 || stages > 8 || ctas_per_sm < 0 || ctas_per_sm > 4)
    return COFEM_ERR_INVALID_ARG;
  op->dense.tc_stages = stages;
  op->dense.tc_ctas_per_sm = ctas_per_sm;
  return COFEM_OK;
}

cofem_status cofem_op_dense_set_tile_rows(cofem_op* op, int32_t rows) {
  if (!op || op->kind != 0 || (rows != 128 && rows != 256)) return COFEM_ERR_INVALID_ARG;
  op->dense.tc_row_tiles = rows / 128;
  return COFEM_OK;
}

cofem_status cofem_op_dense_get_pipeline(const cofem_op* op, int32_t* stages,
                                         int32_t* ctas_per_sm, int32_t* tile_rows) {
  if (!op || op->kind != 0) return COFEM_ERR_INVALID_ARG;
  if (stages) *stages = op->dense.tc_stages;
  if (ctas_per_sm) *ctas_per_sm = op->dense.tc_ctas_per_sm;
  if (tile_rows) *tile_rows = 128 * (op->dense.tc_row_tiles > 1 ? 2 : 1);
  return COFEM_OK;
}

size_t cofem_dense_packed_bytes(int64_t N, int64_t D) {
  if (N < 1 || D < 1) return 0;
  return packed_bytes(N, D);
}

size_t cofem_op_dense_packed_bytes(const cofem_op* op) {
  if (!op || op->kind != 0) return 0;
  if (op->dense.dtype == COFEM_BF16) return packed_bytes(op->dense.N, op->dense.D);
  if (op->dense.dtype == COFEM_F32) return 2 * packed_bytes(op->dense.N, op->dense.D);
  if (op->dense.dtype == COFEM_FP8_E4M3) return packed_bytes(op->dense.N, op->dense.D) / 2;
  return 0;
}

cofem_status cofem_quantize_fp8_tiles(const float* phi_dev, int64_t N, int64_t D, int64_t ld,
                                      void* out_dev, int64_t ld_out, float* scales_dev,
                                      void* stream) {
  if (!phi_dev || !out_dev || !scales_dev || N < 1 || D < 1 || ld < D || ld_out < D)
    return COFEM_ERR_INVALID_ARG;
  fp8_quantize_tiles(phi_dev, N, D, ld, (uint8_t*)out_dev, ld_out, scales_dev,
                     (cudaStream_t)stream);
  CKL();
  return COFEM_OK;
}

cofem_status cofem_op_dense_attach_packed(cofem_op* op, void* packed_dev, size_t packed_bytes_,
                                          void* stream) {
  if (!op || op->kind != 0 ||
      (op->dense.dtype != COFEM_BF16 && op->dense.dtype != COFEM_F32 &&
       op->dense.dtype != COFEM_FP8_E4M3))
    return COFEM_ERR_INVALID_ARG;
  if (!packed_dev) { op->dense.packed = nullptr; return COFEM_OK; }
  if (((uintptr_t)packed_dev & 255) != 0) return COFEM_ERR_INVALID_ARG;
  if (packed_bytes_ < cofem_op_dense_packed_bytes(op)) return COFEM_ERR_WORKSPACE;
  if (op->dense.dtype == COFEM_F32) {
    dense_pack_f32_terms((const float*)op->dense.phi, op->dense.N, op->dense.D, op->dense.ld,
                         packed_dev, (cudaStream_t)stream);
    if (op->dense.nterms == 0) op->dense.nterms = 3;
  } else if (op->dense.dtype == COFEM_FP8_E4M3) {
    dense_pack_fp8(op->dense.phi, op->dense.N, op->dense.D, op->dense.ld, packed_dev,
                   (cudaStream_t)stream);
  } else {
    dense_pack_bf16(op->dense.phi, op->dense.N, op->dense.D, op->dense.ld, packed_dev,
                    (cudaStream_t)stream);
  }
  CKL();
  op->dense.packed = packed_dev;
  return COFEM_OK;
}

cofem_status cofem_op_dense_set_l2_resident(cofem_op* op, int64_t bytes) {
  if (!op || op->kind != 0) return COFEM_ERR_INVALID_ARG;
  if (bytes < 0) { op->dense.l2_resident_cols = -1; return COFEM_OK; }
  const int64_t esz = op->dense.dtype == COFEM_BF16 ? 2 : 4;
  int64_t cols = bytes / (op->dense.N * esz) / 128 * 128;
  op->dense.l2_resident_cols = cols < op->dense.D ? cols : op->dense.D;
  return COFEM_OK;
}

cofem_status cofem_op_dense_set_terms(cofem_op* op, int32_t nterms) {
  if (!op || op->kind != 0 ||
      (op->dense.dtype != COFEM_BF16 && op->dense.dtype != COFEM_F32 &&
       op->dense.dtype != COFEM_FP8_E4M3) ||
      nterms < 0 || nterms > 3 || (op->dense.dtype == COFEM_FP8_E4M3 && nterms != 3))
    return COFEM_ERR_INVALID_ARG;
  op->dense.nterms = nterms;
  return COFEM_OK;
}

cofem_status cofem_op_conv1d(int64_t L, int32_t C, int32_t T, const float* filters_dev,
                             cofem_op** out) {
  if (!out || !filters_dev || L < 64 || L % 64 != 0 || L > (int64_t)2048 * kMaxParts || C < 1 ||
      T < 1 || T > 64 || T > L || ((uintptr_t)filters_dev & 3))
    return COFEM_ERR_INVALID_ARG;
  cofem_op* op = new cofem_op();
  op->kind = 1;
  op->L = L;
  op->C = C;
  op->T = T;
  op->filters = filters_dev;
  *out = op;
  return COFEM_OK;
}

cofem_status cofem_op_conv1d_set_tensor_cores(cofem_op* op, int32_t on) {
  if (!op || op->kind != 1 || (on != 0 && on != 1)) return COFEM_ERR_INVALID_ARG;
  op->conv_tc = on;
  return COFEM_OK;
}

cofem_status cofem_op_dct(int64_t D, int64_t N, const int32_t* idx_dev, cofem_op** out) {
  if (!out || !idx_dev || !dct_size_ok(D) || N < 1 || N > D || ((uintptr_t)idx_dev & 3))
    return COFEM_ERR_INVALID_ARG;
  cofem_op* op = new cofem_op();
  op->kind = 2;
  op->dct_D = D;
  op->dct_N = N;
  op->dct_idx = idx_dev;
  *out = op;
  return COFEM_OK;
}

void cofem_op_destroy(cofem_op* op) { delete op; }

cofem_status cofem_op_shape(const cofem_op* op, int64_t* N, int64_t* D) {
  if (!op) return COFEM_ERR_INVALID_ARG;
  if (N) *N = op_N(op);
  if (D) *D = op_D(op);
  return COFEM_OK;
}

void cofem_params_default(cofem_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->K = 20;
  p->em_iters = 50;
  p->cg_max_iters = 400;
  p->vec_dtype = COFEM_F32;
  p->cg_tol = 1e-6;
  p->alpha_init = 1.0;
  p->den_floor = 1e-12;
  p->support_threshold = 1e6;
}

cofem_status cofem_workspace_bytes(const cofem_op* op, const cofem_params* p, size_t* bytes) {
  cofem_status rc = check_params(op, p);
  if (rc != COFEM_OK) return rc;
  if (!bytes) return COFEM_ERR_INVALID_ARG;
  *bytes = fit_layout(op, p).total;
  return COFEM_OK;
}

cofem_status cofem_fit(const cofem_op* op, const void* y_dev, double beta, const cofem_params* p,
                       void* workspace_dev, size_t workspace_bytes, double* mu_dev, double* s_dev,
                       double* alpha_dev, cofem_stats* stats, void* stream) {
  cofem_status rc = check_params(op, p);
  if (rc != COFEM_OK) return rc;
  if (!y_dev || !workspace_dev || !mu_dev || !s_dev || !alpha_dev) return COFEM_ERR_INVALID_ARG;
  if (!(beta > 0.0) || !isfinite(beta)) return COFEM_ERR_INVALID_ARG;
  if ((uintptr_t)workspace_dev & 255) return COFEM_ERR_INVALID_ARG;
  FitLayout L = fit_layout(op, p);
  if (workspace_bytes < L.total) return COFEM_ERR_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  if (p->vec_dtype == COFEM_F64)
    return fit_impl<double>(op, y_dev, beta, p, (char*)workspace_dev, L, mu_dev, s_dev,
                            alpha_dev, stats, st);
  return fit_impl<float>(op, y_dev, beta, p, (char*)workspace_dev, L, mu_dev, s_dev, alpha_dev,
                         stats, st);
}

cofem_status cofem_probe_fill(uint64_t seed, int64_t t, int32_t K, int64_t D, cofem_dtype dtype,
                              void* out_dev, int64_t ld, void* stream) {
  if (!out_dev || K < 1 || K > 16384 || D < 1 || ld < D || t < 0) return COFEM_ERR_INVALID_ARG;
  const uint64_t key = probe_key(seed, t);
  cudaStream_t st = (cudaStream_t)stream;
  if (dtype == COFEM_F64) launch_probe_fill<double>(key, K, D, (double*)out_dev, ld, st);
  else if (dtype == COFEM_F32) launch_probe_fill<float>(key, K, D, (float*)out_dev, ld, st);
  else return COFEM_ERR_INVALID_ARG;
  CKL();
  return COFEM_OK;
}

cofem_status cofem_apply_workspace_bytes(const cofem_op* op, cofem_dtype vec, int32_t ncols,
                                         size_t* bytes) {
  if (!op || !bytes || ncols < 1 || ncols > kMaxCols) return COFEM_ERR_INVALID_ARG;
  if (!op_supports(op, vec)) return COFEM_ERR_UNSUPPORTED;
  *bytes = op_ws_bytes(op, vec, ncols);
  return COFEM_OK;
}

// ||phi_d||^2 with a workspace: the masked DCT's closed form takes one
// adjoint application (its transform workspace for one column) and two
// D-float buffers (the all-ones kept samples, the DCT of the mask)
static size_t col_norms_ws_bytes(const cofem_op* op) {
  if (op->kind != 2) return 0;
  return align256(op_ws_bytes(op, COFEM_F32, 1)) + 2 * align256((size_t)op->dct_D * sizeof(float));
}

cofem_status cofem_col_norms_workspace_bytes(const cofem_op* op, size_t* bytes) {
  if (!op || !bytes) return COFEM_ERR_INVALID_ARG;
  *bytes = col_norms_ws_bytes(op);
  return COFEM_OK;
}

cofem_status cofem_op_col_norms_ws(const cofem_op* op, float* out_dev, void* workspace_dev,
                                   size_t workspace_bytes, void* stream) {
  if (!op || !out_dev) return COFEM_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (op->kind != 2) return mlp_col_norms(op, out_dev, st);
  if (!workspace_dev || ((uintptr_t)workspace_dev & 255) != 0) return COFEM_ERR_INVALID_ARG;
  if (workspace_bytes < col_norms_ws_bytes(op)) return COFEM_ERR_WORKSPACE;
  char* w = (char*)workspace_dev;
  const size_t o1 = align256(op_ws_bytes(op, COFEM_F32, 1));
  const size_t o2 = o1 + align256((size_t)op->dct_D * sizeof(float));
  dct_col_norms(op->dct_D, op->dct_idx, op->dct_N, (float*)(w + o1), (float*)(w + o2), w,
                nullptr, out_dev, st);
  CKL();
  return COFEM_OK;
}

static cofem_status check_block(const cofem_op* op, cofem_dtype vec, int32_t ncols, int64_t ld,
                                int64_t len, void* ws, size_t wsb) {
  if (!op || ncols < 1 || ncols > kMaxCols || ld < len || ld % kLdAlign != 0)
    return COFEM_ERR_INVALID_ARG;
  if (!op_supports(op, vec)) return COFEM_ERR_UNSUPPORTED;
  if (((uintptr_t)ws & 255) != 0) return COFEM_ERR_INVALID_ARG;
  if (wsb < op_ws_bytes(op, vec, ncols)) return COFEM_ERR_WORKSPACE;
  return COFEM_OK;
}

cofem_status cofem_op_apply(const cofem_op* op, cofem_dtype vec, const void* x_dev, int64_t ld,
                            int32_t ncols, const double* alpha_dev, double beta, void* y_dev,
                            void* workspace_dev, size_t workspace_bytes, void* stream) {
  cofem_status rc = check_block(op, vec, ncols, ld, op ? op_D(op) : 0, workspace_dev,
                                workspace_bytes);
  if (rc != COFEM_OK) return rc;
  if (!x_dev || !y_dev || !alpha_dev || !workspace_dev) return COFEM_ERR_INVALID_ARG;
  return op_apply(op, vec, x_dev, ld, ncols, alpha_dev, beta, y_dev, nullptr, nullptr,
                  (char*)workspace_dev, (cudaStream_t)stream);
}

cofem_status cofem_op_apply_timed(const cofem_op* op, cofem_dtype vec, const void* x_dev,
                                  int64_t ld, int32_t ncols, const double* alpha_dev,
                                  double beta, void* y_dev, void* workspace_dev,
                                  size_t workspace_bytes, void* stream, float* kernel_ms,
                                  int32_t max_kernels, int32_t* n_kernels) {
  if (!kernel_ms || !n_kernels || max_kernels < 1 || max_kernels > 16)
    return COFEM_ERR_INVALID_ARG;
  cudaEvent_t ev[17];
  for (int i = 0; i <= max_kernels; ++i) CK(cudaEventCreate(&ev[i]));
  cudaStream_t st = (cudaStream_t)stream;
  cudaEventRecord(ev[0], st);
  apply_ticks_arm(ev + 1, max_kernels);
  cofem_status rc = cofem_op_apply(op, vec, x_dev, ld, ncols, alpha_dev, beta, y_dev,
                                   workspace_dev, workspace_bytes, stream);
  const int n = apply_ticks_disarm();
  if (rc == COFEM_OK) {
    if (cudaEventSynchronize(ev[n]) != cudaSuccess) rc = COFEM_ERR_CUDA;
    for (int i = 0; i < n && rc == COFEM_OK; ++i) cudaEventElapsedTime(&kernel_ms[i], ev[i], ev[i + 1]);
    *n_kernels = n;
  }
  for (int i = 0; i <= max_kernels; ++i) cudaEventDestroy(ev[i]);
  return rc;
}

cofem_status cofem_op_forward(const cofem_op* op, cofem_dtype vec, const void* z_dev, int64_t ldz,
                              int32_t ncols, void* w_dev, int64_t ldw, void* workspace_dev,
                              size_t workspace_bytes, void* stream) {
  cofem_status rc = check_block(op, vec, ncols, ldz, op ? op_D(op) : 0, workspace_dev,
                                workspace_bytes);
  if (rc != COFEM_OK) return rc;
  if (!z_dev || !w_dev || !workspace_dev || ldw < op_N(op) || ldw % kLdAlign)
    return COFEM_ERR_INVALID_ARG;
  return op_forward(op, vec, z_dev, ldz, ncols, w_dev, ldw, (char*)workspace_dev,
                    (cudaStream_t)stream);
}

cofem_status cofem_op_adjoint(const cofem_op* op, cofem_dtype vec, const void* w_dev, int64_t ldw,
                              int32_t ncols, void* z_dev, int64_t ldz, void* workspace_dev,
                              size_t workspace_bytes, void* stream) {
  cofem_status rc = check_block(op, vec, ncols, ldz, op ? op_D(op) : 0, workspace_dev,
                                workspace_bytes);
  if (rc != COFEM_OK) return rc;
  if (!z_dev || !w_dev || !workspace_dev || ldw < op_N(op) || ldw % kLdAlign)
    return COFEM_ERR_INVALID_ARG;
  return op_adjoint(op, vec, w_dev, ldw, ncols, z_dev, ldz, 1.0, (char*)workspace_dev,
                    (cudaStream_t)stream);
}

cofem_status cofem_diag_mstep(uint64_t seed, int64_t t, int32_t K, int64_t D, cofem_dtype vec,
                              const void* x_dev, int64_t ld, double den_floor,
                              double support_threshold, double* mu_dev, double* s_dev,
                              double* alpha_dev, int32_t* counts_dev, void* stream) {
  if (!x_dev || !mu_dev || !s_dev || !alpha_dev || K < 1 || K > 16384 || D < 1 || ld < D ||
      !(den_floor > 0.0))
    return COFEM_ERR_INVALID_ARG;
  CgConf cf;
  memset(&cf, 0, sizeof(cf));
  cf.D = D;
  cf.ld = ld;
  cf.K = K;
  cf.ncols = K + 1;
  cf.T = 1;
  cf.seed = seed;
  cf.den_floor = den_floor;
  cf.support_threshold = support_threshold;
  const uint64_t key = probe_key(seed, t);
  cudaStream_t st = (cudaStream_t)stream;
  if (vec == COFEM_F64)
    launch_diag_mstep<double>(cf, nullptr, key, (const double*)x_dev, mu_dev, s_dev, alpha_dev,
                              counts_dev, nullptr, nullptr, nullptr, nullptr, st);
  else if (vec == COFEM_F32)
    launch_diag_mstep<float>(cf, nullptr, key, (const float*)x_dev, mu_dev, s_dev, alpha_dev,
                             counts_dev, nullptr, nullptr, nullptr, nullptr, st);
  else
    return COFEM_ERR_INVALID_ARG;
  CKL();
  return COFEM_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------
// Internal hooks for entry points defined in other translation units; they
// forward to the same routines cofem_op_apply uses.
namespace cofem {

cofem_status apply_check(const cofem_op* op, cofem_dtype vec, int32_t ncols, int64_t ld) {
  if (!op || ncols < 1 || ncols > kMaxCols || ld < op_D(op) || ld % kLdAlign != 0)
    return COFEM_ERR_INVALID_ARG;
  if (!op_supports(op, vec)) return COFEM_ERR_UNSUPPORTED;
  return COFEM_OK;
}

size_t apply_scratch_bytes(const cofem_op* op, cofem_dtype vec, int32_t ncols) {
  return op_ws_bytes(op, vec, ncols);
}

cofem_status apply_with_scratch(const cofem_op* op, cofem_dtype vec, const void* x, int64_t ld,
                                int32_t ncols, const double* alpha, double beta, void* y,
                                char* scratch, cudaStream_t st) {
  return op_apply(op, vec, x, ld, ncols, alpha, beta, y, nullptr, nullptr, scratch, st);
}

void set_last_error(const char* msg) { g_last_error = msg; }

int op_is_dense(const cofem_op* op) { return op->kind == 0; }
DenseDesc op_dense_desc(const cofem_op* op) { return op->dense; }
int op_conv_desc(const cofem_op* op, int64_t* L, int* C, int* T, const float** h, int* bf16) {
  if (op->kind != 1) return -1;
  *L = op->L;
  *C = op->C;
  *T = op->T;
  *h = op->filters;
  *bf16 = op->conv_tc;
  return 0;
}

}  // namespace cofem

// ------------------------------------------------------------- autotuner
// Times the tensor-core operator application for every pipeline shape
// (CTAs per SM x ring depth) that fits, with CUDA events on the caller's
// stream, and keeps the fastest on the handle.  Inputs are made up in the
// caller's workspace (layout: operator scratch | X | Y | alpha).
namespace cofem {

__global__ void tune_fill_kernel(float* x, int64_t n, double* alpha, int64_t D) {
  pdl_wait();
  pdl_trigger();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] = (float)((mix64((uint64_t)i) >> 40) * (1.0 / 16777216.0) - 0.5);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < D;
       i += (int64_t)gridDim.x * blockDim.x)
    alpha[i] = 1.0;
}

static void tune_layout(const cofem_op* op, int ncols, size_t* ows, size_t* blk, size_t* total) {
  const int64_t ld = round_up(op->dense.D, kLdAlign);
  *ows = align256(op_ws_bytes(op, COFEM_F32, ncols, true));
  *blk = align256((size_t)ncols * ld * sizeof(float));
  *total = *ows + 2 * *blk + align256((size_t)op->dense.D * sizeof(double));
}

}  // namespace cofem

extern "C" size_t cofem_op_dense_autotune_workspace_bytes(const cofem_op* op, int32_t ncols) {
  if (!op || op->kind != 0 || ncols < 1 || ncols > kMaxCols) return 0;
  size_t a, b, t;
  tune_layout(op, ncols, &a, &b, &t);
  return t;
}

extern "C" cofem_status cofem_op_dense_autotune(cofem_op* op, int32_t ncols, void* workspace_dev,
                                                size_t workspace_bytes, void* stream,
                                                int32_t* best_stages, int32_t* best_ctas,
                                                float* best_us) {
  if (!op || op->kind != 0 || !use_tc(op) || ncols < 1 || ncols > kMaxCols || !workspace_dev ||
      ((uintptr_t)workspace_dev & 255))
    return COFEM_ERR_INVALID_ARG;
  size_t ows, blk, total;
  tune_layout(op, ncols, &ows, &blk, &total);
  if (workspace_bytes < total) return COFEM_ERR_WORKSPACE;
  char* ws = (char*)workspace_dev;
  float* X = (float*)(ws + ows);
  float* Y = (float*)(ws + ows + blk);
  double* alpha = (double*)(ws + ows + 2 * blk);
  const int64_t ld = round_up(op->dense.D, kLdAlign);
  cudaStream_t st = (cudaStream_t)stream;
  launch_k(tune_fill_kernel, dim3(1024), dim3(256), 0, st, X, (int64_t)ncols * ld, alpha, op->dense.D);
  CKL();
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const int keep_st = op->dense.tc_stages, keep_cps = op->dense.tc_ctas_per_sm,
            keep_mt = op->dense.tc_row_tiles;
  float best = 1e30f;
  int bst = keep_st, bcps = keep_cps, bmt = keep_mt;
  cofem_status rc = COFEM_OK;
  for (int mt = 1; mt <= 2 && rc == COFEM_OK; ++mt)
  for (int cps = 1; cps <= 4 && rc == COFEM_OK; ++cps) {
    DenseTcPlan full = dense_tc_plan(op->dense.N, op->dense.D, ncols, op->dense.nterms,
                                     num_sms(), cps, 0, op->dense.phi_terms, mt,
                                     op->dense.dtype == COFEM_FP8_E4M3);
    // two tiles per unit need room for four accumulators (else the plan is
    // the one-tile plan, timed already); with all of the tensor memory taken,
    // shapes differ only in stages
    if (mt == 2 && (full.MT != 2 || (cps > 1 && full.tmem_cols > 256))) break;
    for (int stg = 2; stg <= full.stages && rc == COFEM_OK; ++stg) {
      op->dense.tc_row_tiles = mt;
      op->dense.tc_ctas_per_sm = cps;
      op->dense.tc_stages = stg;
      for (int w = 0; w < 2 && rc == COFEM_OK; ++w)
        rc = op_apply(op, COFEM_F32, X, ld, ncols, alpha, 1.0, Y, nullptr, nullptr, ws, st);
      if (rc != COFEM_OK) break;
      const int reps = 5;
      cudaEventRecord(e0, st);
      for (int r = 0; r < reps && rc == COFEM_OK; ++r)
        rc = op_apply(op, COFEM_F32, X, ld, ncols, alpha, 1.0, Y, nullptr, nullptr, ws, st);
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) rc = COFEM_ERR_CUDA;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      const float us = ms * 1000.f / reps;
      if (rc == COFEM_OK && us < best) { best = us; bst = stg; bcps = cps; bmt = mt; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  op->dense.tc_stages = rc == COFEM_OK ? bst : keep_st;
  op->dense.tc_ctas_per_sm = rc == COFEM_OK ? bcps : keep_cps;
  op->dense.tc_row_tiles = rc == COFEM_OK ? bmt : keep_mt;
  if (best_stages) *best_stages = op->dense.tc_stages;
  if (best_ctas) *best_ctas = op->dense.tc_ctas_per_sm;
  if (best_us) *best_us = best;
  return rc;
}

namespace cofem {

}  // namespace cofem
