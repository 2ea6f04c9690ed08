// Shared device/host definitions of libcofem (GB300, sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <utility>

#include "../../include/cofem.h"

namespace cofem {

constexpr int kMaxCols = 64;        // K + 1 <= 64 columns per block
constexpr int kLdAlign = 64;        // leading dimensions are multiples of 64
constexpr int kMaxParts = 2048;     // max partial-sum slots per reduction

// Device-resident control block of one CG solve / one fit.  Lives in the
// workspace; every field is written only by kernels (after a host memset).
struct CgCtl {
  int iter;            // CG iterations done in the current E-step
  int done;            // solve finished (converged or out of iterations)
  int replace;         // true-residual replacement due in this iteration
  int error;           // first cofem_status raised on the device
  long long t;         // EM iteration number of the current E-step (1-based)
  int em_index;        // index of the current E-step in the stats arrays
  int clamps;          // M-step counters of the current EM iteration
  int support;
  int extra_iters;     // learned path: iterations of a preconditioned solve that fell back
  int fallbacks;       // learned path: fallbacks to plain CG so far
  int run;             // the direction update may run (b_j of this iteration are set)
  double normB2;       // ||B||_F^2
  double relres;       // ||R||_F / ||B||_F after the last iteration
  unsigned int counter[8];  // arrival counters of last-block reductions
  unsigned int dir_gen;     // CG update with the direction update: bumped when an iteration is closed
  unsigned long long start_ns;  // device clock (%globaltimer) when the fit's first kernel ran
};

// Per-column CG scalars (double, Sec. 3.2 recurrences).
struct CgScalars {
  double rho[kMaxCols];      // r_j^T r_j
  double rho_new[kMaxCols];
  double gamma[kMaxCols];    // p_j^T A p_j
  double a[kMaxCols];        // step sizes
  double b[kMaxCols];        // direction updates
  double rr_new[kMaxCols];   // preconditioned CG: r_j^T r_j (rho holds r_j^T z_j)
  double bn2[kMaxCols];      // ||B_j||^2 of the solve's right-hand sides
};

// Static problem description passed by value to the CG kernels.
struct CgConf {
  int64_t D;
  int64_t ld;
  int ncols;                 // K + 1
  int K;
  uint64_t seed;
  double tol;
  int max_iters;
  int fixed_iters;
  int replace_every;
  double beta;
  double den_floor;
  double support_threshold;
  int em_iters;
  unsigned long long while_handle;   // cudaGraphConditionalHandle or 0
  unsigned long long if_handle;      // residual-replacement IF node or 0
  unsigned long long inner_handle;   // inner WHILE node (replacement outside the inner loop) or 0
  int gamma_parts;                   // partials of p^T A p written by the operator
  int split_nt;                      // >0: also write P's BF16 terms (tensor-core operator)
  int split_rows;                    // rows of the split buffer (B operand rows)
  void* split_buf;                   // row split_row(j, t), pitch ld, bf16
  const float* minv;                 // preconditioned CG: M^-1 = diag(minv), else null
  unsigned long long fallback_handle;  // IF node: preconditioned solve did not converge
  int fallback_init;                 // this init restarts plain CG after a fallback
  float* alpha32;                    // FP32 copy of alpha kept by the M-step, or null
  int stop_rule;                     // 1: per-column stop (frozen columns have rho_j = 0)
  int T;                             // tasks: columns 0..T-1 are beta Phi^T y_t, then K probes
  int gate_run;                      // CG update: do nothing unless ctl->run (an unrolled copy)
  long long* st_end_ns;              // per EM iteration: device clock at the end of its M-step,
                                     // ns since the fit's first kernel (ctl->start_ns), or null
  unsigned long long gen_wait_ns;    // CG update with the direction update: limit of the
                                     // wait for the closing block (0: 2 s)
};

// Row of the tensor-core B operand that holds BF16 term t of column j when
// each FP32 column is split into nt terms: columns are packed G = 16/nt to a
// group of 16 rows (with nt = 3 the 16th row of each group stays zero).
__host__ __device__ __forceinline__ int split_row(int j, int t, int nt) {
  const int g = 16 / nt;
  return (j / g) * 16 + (j % g) * nt + t;
}

__host__ __device__ inline int64_t round_up(int64_t x, int64_t m) {
  return (x + m - 1) / m * m;
}

// ---------------------------------------------------------------- probes
// SplitMix64 output function (Steele, Lea, Flood, OOPSLA 2014).
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Key of EM iteration t.
__host__ __device__ __forceinline__ uint64_t probe_key(uint64_t seed, long long t) {
  return mix64(mix64(seed) ^ (uint64_t)t);
}

// 64 probe signs of coordinate d, word w (bit k set => p = -1).
__device__ __forceinline__ uint64_t probe_word(uint64_t key, int64_t d, int w) {
  return mix64(key ^ (((uint64_t)d << 8) | (uint64_t)w));
}

// ---------------------------------------------------------- reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Per-thread dot-product accumulators.  FP32 vectors use a compensated FP32
// sum: Knuth's TwoSum keeps the rounding error of every addition and an FMA
// recovers the rounding error of every product, so the pair (s, c) carries
// about twice FP32's precision with FP32 instructions only (FP64 arithmetic
// and f32<->f64 conversions issue at a small fraction of the FP32 rate on
// this GPU).  The value is promoted to FP64 once per thread, and every
// cross-thread reduction is FP64.  FP64 vectors accumulate in FP64.
// Terms of magnitude 1e30 or more (or non-finite) go to an FP64 side sum
// instead, so that squares of large FP32 values cannot overflow.
struct AccF {
  float s = 0.f, c = 0.f;
  double big = 0.0;
  __device__ __forceinline__ void add(float x) {
    if (!(fabsf(x) < 1e30f)) { big += (double)x; return; }
    const float t = s + x;
    const float xv = t - s;
    c += (s - (t - xv)) + (x - xv);
    s = t;
  }
  __device__ __forceinline__ void add_prod(float a, float b) {
    const float p = a * b;
    if (!(fabsf(p) < 1e30f)) { big += (double)a * (double)b; return; }
    c += fmaf(a, b, -p);
    add(p);
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c + big; }
};
struct AccD {
  double s = 0.0;
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ void add_prod(double a, double b) { s += a * b; }
  __device__ __forceinline__ double value() const { return s; }
};
template <typename V> struct AccOf { using T = AccD; };
template <> struct AccOf<float> { using T = AccF; };

// Block-wide sum; result valid in thread 0.  `sh` holds >= 32 doubles.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double r = 0.0;
  if (wid == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    r = lane < nw ? sh[lane] : 0.0;
    r = warp_sum(r);
  }
  return r;
}

// One butterfly step of a compensated FP32 sum: (s, c) += (os, oc).
__device__ __forceinline__ void two_sum_merge(float& s, float& c, float os, float oc) {
  const float t = s + os, bv = t - s;
  c += oc + ((s - (t - bv)) + (os - bv));
  s = t;
}

// Block-wide sums of per-thread accumulators; result valid in thread 0.
// Compensated FP32 accumulators are combined with FP32 TwoSum butterflies
// and promoted to FP64 once; `sh` holds >= 32 doubles.
__device__ __forceinline__ double block_sum(const AccF& a, double* sh) {
  float s = a.s, c = a.c;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    two_sum_merge(s, c, __shfl_xor_sync(0xffffffffu, s, o), __shfl_xor_sync(0xffffffffu, c, o));
  float2* sh2 = reinterpret_cast<float2*>(sh);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh2[wid] = make_float2(s, c);
  __syncthreads();
  double r = 0.0;
  if (wid == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    const float2 v = lane < nw ? sh2[lane] : make_float2(0.f, 0.f);
    s = v.x;
    c = v.y;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
      two_sum_merge(s, c, __shfl_xor_sync(0xffffffffu, s, o), __shfl_xor_sync(0xffffffffu, c, o));
    r = (double)s + (double)c;
  }
  // the FP64 side sums, only when some thread of the block has one
  if (__syncthreads_or(a.big != 0.0)) {
    const double rb = block_sum(a.big, sh);
    r += rb;
  }
  return r;
}
__device__ __forceinline__ double block_sum(const AccD& a, double* sh) { return block_sum(a.s, sh); }

// Records the first device error (later ones are dropped).
__device__ __forceinline__ void raise_error(CgCtl* ctl, int code) {
  atomicCAS(&ctl->error, 0, code);
}

// Last-block arrival: returns true in every thread of the last block to
// arrive on counter `c`; that block must reset the counter.  Whatever the
// last block reads from the other blocks must have been written by their
// thread 0 (its fence orders those writes before the arrival; the other
// threads' stores need no fence and do not wait for one).
__device__ __forceinline__ bool arrive_last(unsigned int* counter) {
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = (atomicAdd(counter, 1u) == gridDim.x * gridDim.y - 1);
    if (last) __threadfence();
  }
  __syncthreads();
  return last;
}

// ------------------------------------------- programmatic dependent launch
// Every kernel waits for its predecessor's results with pdl_wait() before
// touching global memory and lets its dependent launch early with
// pdl_trigger() once its main work is done; launch_k launches with
// programmatic stream serialization, so in a captured graph the next
// kernel's blocks are scheduled while this one drains.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                            cudaStream_t st, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

}  // namespace cofem
