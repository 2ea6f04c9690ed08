// Dense dictionary descriptors and launchers.
#pragma once
#include <type_traits>

#include "kernels.cuh"

namespace cofem {

struct DenseDesc {
  int64_t N, D, ld;        // Phi is N x D row-major, leading dimension ld
  int dtype;               // cofem_dtype of the stored entries
  const void* phi;
  const float* scales;     // FP8 tile scales or nullptr
  int nterms;              // BF16: terms per FP32 vector on tensor cores
                           // (1..3), 0 = CUDA-core path
};

struct DenseSimtPlan {
  int64_t ldw, ld;         // padded N and D
  int S1, S2;              // split-K counts of the two products
  int64_t kps1, kps2;      // K extent of one split
  size_t bytes_wpart, bytes_w, bytes_qpart;
  size_t total() const { return bytes_wpart + bytes_w + bytes_qpart; }
};

DenseSimtPlan dense_simt_plan(int64_t N, int64_t D, int ncols, int vec_bytes, int sms);

// Tensor-core plan (BF16 dictionary, FP32 vectors split into NT BF16 terms).
struct DenseTcPlan {
  int NT, nc, BN;            // terms, output columns, MMA N (B-operand rows)
  uint32_t tmem_cols;        // tensor-memory columns allocated per CTA
  int64_t ld, ldw;           // padded D and N
  int nk1, nk2;              // K blocks (64) of the two products
  int S1, kbps1;             // split-K of the first product
  int stages;                // shared-memory ring depth
  size_t smem;               // dynamic shared memory per CTA
  size_t off_xs, bytes_xs, off_wpart, bytes_wpart, off_ws, bytes_ws, off_cnt, bytes_cnt, total;
};
DenseTcPlan dense_tc_plan(int64_t N, int64_t D, int nc, int NT, int sms);

// Y = beta Phi^T Phi X + alpha . X on tcgen05; returns 0, 1 (tensor map
// encoding failed) or 2 (launch failed).  err: device error word or null.
// flags: kApplyPresplit -- the BF16 terms of X are already in the workspace
// (rows split_row(j, t) of pitch plan.ld at plan.off_xs), written by the CG kernels;
// kApplyZeroCounters -- clear the split-K arrival counters first (needed
// when the workspace does not come from a fit, whose kernels leave them 0).
constexpr unsigned kApplyPresplit = 1u, kApplyZeroCounters = 2u;
int dense_tc_apply(const DenseDesc& op, int NT, const float* X, int64_t ld, int nc, float* Y,
                   double beta, const double* alpha, double* dots, int* nparts, char* ws,
                   int* err, unsigned flags, cudaStream_t st);

template <typename TA, typename V>
void dense_simt_forward(const DenseDesc& op, const V* Z, int64_t ldz, int ncols, V* W,
                        int64_t ldw_out, char* ws, cudaStream_t st);
template <typename TA, typename V>
void dense_simt_adjoint(const DenseDesc& op, const V* W, int64_t ldw, int ncols, V* Y,
                        int64_t ld, double beta, const double* alpha, const V* X,
                        double* dots, int* nparts, char* ws, cudaStream_t st);
template <typename TA, typename V>
void dense_simt_apply(const DenseDesc& op, const V* X, int64_t ld, int ncols, V* Y,
                      double beta, const double* alpha, double* dots, int* nparts, char* ws,
                      cudaStream_t st);

}  // namespace cofem
