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
  int64_t l2_resident_cols;  // tensor-core path: columns d below this are
                             // loaded with an evict-last L2 policy
  const void* packed;        // tensor-core path: tile-major copy of Phi or null
  int tc_ctas_per_sm;        // tensor-core pipeline: resident CTAs per SM (1, 2; 0 = 2)
  int tc_stages;             // shared-memory ring depth (0 = as deep as fits)
  int phi_terms;             // BF16 terms per Phi entry in the packed copy: 1 for a
                             // BF16 dictionary, 2 for an FP32 one (Phi = hi + lo)
  int tc_row_tiles;          // 128-row output tiles per work unit (1, 2; 0 = 1): two
                             // tiles share every B-operand stage
};

// Tile-major ("packed") BF16 layout read by the tensor-core operator: tile
// (mt, kb) holds rows [128 mt, 128 mt + 128) x columns [64 kb, 64 kb + 64) as
// 128 rows of 64 contiguous values (16 KB), tiles ordered kb-fastest, zero
// padded at the edges.  Every TMA box of either product is then one or two
// contiguous DRAM ranges instead of 64-128 rows 64 KB apart.
inline int64_t packed_tiles_m(int64_t N) { return (N + 127) / 128; }
inline int64_t packed_tiles_k(int64_t D) { return (D + 63) / 64; }
inline size_t packed_bytes(int64_t N, int64_t D) {
  return (size_t)packed_tiles_m(N) * packed_tiles_k(D) * 128 * 64 * 2;
}
void dense_pack_bf16(const void* phi, int64_t N, int64_t D, int64_t ld, void* packed,
                     cudaStream_t st);
// FP32 dictionary: two packed images (2 * packed_bytes(N, D) bytes), the
// first holding hi = bf16(Phi), the second lo = bf16(Phi - hi), so that
// hi + lo carries 16 significant bits of every entry.
void dense_pack_f32_terms(const float* phi, int64_t N, int64_t D, int64_t ld, void* packed,
                          cudaStream_t st);
// FP8 E4M3 dictionary: one packed image of packed_bytes(N, D) / 2 bytes, each
// entry's byte at the position of its BF16 value in the BF16 layout.
void dense_pack_fp8(const void* phi, int64_t N, int64_t D, int64_t ld, void* packed,
                    cudaStream_t st);
// FP8 quantisation of an FP32 dictionary: per 128 x 128 tile, scale = the
// smallest power of two with max |phi| / scale <= 448, bytes =
// e4m3(phi / scale) (round to nearest even, saturating); and the CUDA-core
// products of an FP8 dictionary (entries bf16(e4m3 x scale)).
void fp8_quantize_tiles(const float* phi, int64_t N, int64_t D, int64_t ld, uint8_t* out,
                        int64_t ld_out, float* scales, cudaStream_t st);
void fp8_forward(const DenseDesc& op, const float* Z, int64_t ldz, int ncols, float* W,
                 int64_t ldw, cudaStream_t st);
void fp8_adjoint(const DenseDesc& op, const float* W, int64_t ldw, int ncols, float* Z,
                 int64_t ldz, double beta, cudaStream_t st);
void fp8_col_norms(const DenseDesc& op, float* out, cudaStream_t st);


// An FP32 dictionary entry as the tensor-core operator applies it once a
// two-term packed copy is attached: hi + lo with hi = bf16(v), lo =
// bf16(v - hi) (round to nearest even).  hi + lo has at most 17 significant
// bits, so the sum is exact in FP32.  The CUDA-core products of such an
// operator (b = beta Phi^T y, Phi Z, Phi^T W, column norms) read entries
// through this type so that every product of the operator uses the same
// dictionary.
struct F32HiLo {
  float v;
};
__device__ __forceinline__ float hilo_value(float v) {
  const __nv_bfloat16 hi = __float2bfloat16_rn(v);
  const float h = __bfloat162float(hi);
  return h + __bfloat162float(__float2bfloat16_rn(v - h));
}
inline bool dense_applies_hilo(const DenseDesc& d) {
  return d.dtype == COFEM_F32 && d.phi_terms > 1 && d.packed != nullptr;
}

// Runs the bounded-wait self-test; returns the device error word (0 or
// COFEM_ERR_TIMEOUT) or -1 on a CUDA error.
int wait_selftest(int64_t limit_ns, cudaStream_t st);

// Per-kernel event timing of one operator application (diagnostics).
void apply_ticks_arm(cudaEvent_t* events, int cap);
int apply_ticks_disarm();
void apply_tick(cudaStream_t st);

// Batched mode: one CTA per work item of a table built on the host.
struct TcProb {
  int64_t N, D;          // dictionary shape of the problem
  int64_t nkd;           // 64-column tiles of its packed Phi
  int64_t poff;          // element offset of its packed Phi
  int64_t xoff, ld;      // its X / Y block: offset (elements) and leading dimension
  int64_t aoff;          // offset of its alpha (and of its coordinates)
  int64_t boff1;         // column offset of its BF16 terms of X in the split buffer
  int64_t boff2;         // column offset of its BF16 terms of W in Ws
  int64_t wpoff, ldw;    // its split-K partials of W: offset, leading dimension
  int S1;                // splits of its first product
  int dots_base;         // first partial-dot slot of its second product
  double beta;           // its noise precision
};
struct TcItem {
  int prob, tile, split, kb0, kb1;
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
  int MT;                    // 128-row output tiles per work unit
  bool fp8;                  // FP8 dictionary (converter warps, staging area)
  uint32_t acc_cols;         // tensor-memory columns of one accumulator
  uint32_t tmem_cols;        // tensor-memory columns allocated per CTA (two accumulators)
  int grid;                  // resident CTAs of one launch (ctas per SM x SMs)
  int64_t ld, ldw;           // padded D and N
  int nk1, nk2;              // K blocks (64) of the two products
  int S1, kbps1;             // split-K of the first product
  int stages;                // shared-memory ring depth
  size_t smem;               // dynamic shared memory per CTA
  size_t off_xs, bytes_xs, off_wpart, bytes_wpart, off_ws, bytes_ws, total;
};
// PT: BF16 terms per Phi entry (1 or 2); MT: 128-row output tiles per work
// unit (1 or 2); a ring stage holds MT x PT A tiles and one B tile, and a CTA
// allocates 2 x MT accumulators.
// fp8: an FP8 dictionary (one byte per entry in the packed copy): a stage
// also holds the 8 KB of bytes the converter warps expand (MT = PT = 1).
DenseTcPlan dense_tc_plan(int64_t N, int64_t D, int nc, int NT, int sms, int ctas_per_sm = 2,
                          int stages = 0, int PT = 1, int MT = 1, bool fp8 = false);
inline DenseTcPlan dense_tc_plan(const DenseDesc& op, int nc, int sms) {
  return dense_tc_plan(op.N, op.D, nc, op.nterms, sms, op.tc_ctas_per_sm, op.tc_stages,
                       op.phi_terms > 1 ? 2 : 1, op.tc_row_tiles > 1 ? 2 : 1,
                       op.dtype == COFEM_FP8_E4M3);
}

// Y = beta Phi^T Phi X + alpha . X on tcgen05; returns 0, 1 (tensor map
// encoding failed) or 2 (launch failed).  err: device error word or null.
// flags: kApplyPresplit -- the BF16 terms of X are already in the workspace
// (rows split_row(j, t) of pitch plan.ld at plan.off_xs), written by the CG
// kernels.
constexpr unsigned kApplyPresplit = 1u;
// kApplyOpPrepared -- structured operators: per-operator tables in the
// scratch are already built (the masked DCT's mask and twiddles).
constexpr unsigned kApplyOpPrepared = 2u;
// Batched products over a work-item table (see TcItem / TcProb); `grid`
// persistent CTAs (0: one per item) take the items in strides of the grid;
// tmem_cols holds two accumulators.  mode 0:
// split-K partials of W = Phi X (if wterms is set, problems with S1 == 1
// write W's BF16 terms there instead: row 16 (j / G) + NT (j % G) + t,
// G = 16 / NT, column boff2 + n, pitch ldw_terms); mode 1:
// Y = beta Phi^T W + alpha . X with partial dots.  xs / ws: BF16 term
// buffers (BN rows, pitch ldx_total / ldw_total).  Returns 0, 1 (tensor map)
// or 2 (launch).
int dense_tc_batched(int mode, int NT, int nitems, const TcItem* items, const TcProb* probs,
                     const int* done, const void* packed, const __nv_bfloat16* bsrc,
                     int64_t b_cols, int BN, int nc, int stages, uint32_t tmem_cols,
                     size_t smem, float* wpart, const float* X, float* Y, const double* alpha,
                     double* dots, int* err, cudaStream_t st, int grid = 0,
                     __nv_bfloat16* wterms = nullptr, int64_t ldw_terms = 0);

// alpha32: optional FP32 copy of alpha ((float)alpha[d]); saves the per-row
// conversion.  gate: if set, every kernel of the application returns at
// once when *gate == 0 (a step inside a graph that runs only when due).
int dense_tc_apply(const DenseDesc& op, int NT, const float* X, int64_t ld, int nc, float* Y,
                   double beta, const double* alpha, double* dots, int* nparts, char* ws,
                   int* err, unsigned flags, cudaStream_t st, const float* alpha32 = nullptr,
                   const int* gate = nullptr);

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
