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
};

struct DenseSimtPlan {
  int64_t ldw, ld;         // padded N and D
  int S1, S2;              // split-K counts of the two products
  int64_t kps1, kps2;      // K extent of one split
  size_t bytes_wpart, bytes_w, bytes_qpart;
  size_t total() const { return bytes_wpart + bytes_w + bytes_qpart; }
};

DenseSimtPlan dense_simt_plan(int64_t N, int64_t D, int ncols, int vec_bytes, int sms);

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
