// Dense dictionary operator on the 5th-generation tensor cores (tcgen05):
//   A X = beta Phi^T (Phi X) + alpha . X        (Eq. (mat-eq))
// for a BF16 dictionary and FP32 right-hand sides.  An FP32 dictionary runs
// the same kernels with every entry stored as two BF16 terms Phi = hi + lo
// (two packed images, the same 4 bytes per entry as FP32): each ring stage
// then holds both A tiles and the MMA warp accumulates both products.
//
// Each FP32 column x_j is represented exactly enough for FP32 work by NT
// BF16 terms x_j = x_j1 + x_j2 (+ x_j3) (each term the BF16 rounding of the
// remainder).  Products of BF16 values are exact in the FP32 accumulator,
// so NT = 3 reproduces a 24-bit mantissa; term t of column j is stored in row
// split_row(j, t) of a K-major operand (G = 16/NT columns per 16 rows) and
// the terms are summed in the epilogue.
//
//   split   X      -> Xs (BF16, BN rows x ld)
//   GEMM1   W_s    = Phi[:, K-range s] Xs[K-range s]      tcgen05, split-K
//   reduce  W      = sum_s W_s  -> Ws (BF16 terms, BN rows x ldw)
//   GEMM2   Y      = beta Phi^T Ws + alpha . X, plus x_j^T y_j partials
//
// Both GEMMs stream Phi through shared memory with TMA (128-byte swizzle,
// evict-first L2 policy) into a STAGES-deep ring; one thread issues the
// MMAs into a 128 x BN FP32 accumulator in tensor memory; four warps read it
// back with tcgen05.ld.  GEMM1 reads Phi K-major (rows n, d contiguous);
// GEMM2 reads the same bytes MN-major (Phi^T without a transpose copy).
// Every wait is bounded: a timeout sets COFEM_ERR_TIMEOUT and the CTA
// drains its copies, frees its tensor memory and exits.
#include <algorithm>
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "dense.cuh"
#include "tc_ptx.cuh"

namespace cofem {

constexpr int kTcThreads = 192;     // warp 0 TMA, warp 1 MMA/TMEM, warps 2-5 epilogue
constexpr int kTcThreadsFp8 = 448;  // FP8 dictionaries: warps 6-13 convert A tiles to BF16
constexpr int kCvtWarps = (kTcThreadsFp8 - kTcThreads) / 32;
constexpr int kTileM = 128;
constexpr int kTileK = 64;          // 64 bf16 = one 128-byte swizzle row
constexpr uint32_t kATileBytes = kTileM * kTileK * 2;
constexpr uint64_t kWaitLimitNs = 1000000000ull;

constexpr int kMaxStages = 8;
constexpr size_t kSmemPerSm = 227 * 1024;        // usable shared memory per SM

// The NT terms of column j sit in accumulator columns split_row(j, 0..NT-1):
// the epilogue reads 16 accumulator columns at a time, i.e. G = 16/NT
// columns (NT = 3 leaves one of each 16 unused).
template <int NT> struct TermGroup {
  static constexpr int G = 16 / NT, COLS = 16;
};

struct TcArgs {
  int64_t M;            // output rows (N for GEMM1, D for GEMM2)
  int nk_total;         // K blocks of 64
  int kb_per_split;
  int nc;               // output columns
  int units;            // work units (tile x K range), taken by CTAs in strides of gridDim.x
  int units_m;          // output tiles (units = units_m x K splits)
  uint32_t acc_cols;    // tensor-memory columns of one accumulator (two are allocated)
  int BN;               // MMA N (rows of the B operand)
  int stages;           // depth of the shared-memory ring (<= kMaxStages)
  uint32_t tmem_cols;
  int64_t res_d;        // Phi columns d < res_d are loaded evict-last (kept in L2)
  const __nv_bfloat16* packed;   // pre-swizzled tile-major copy of Phi, or null
  int phi_terms;        // 2: Phi = hi + lo, two packed images term_stride apart
                        // (packed copy only); otherwise one
  int64_t term_stride;  // elements from the hi image to the lo image
  int row_tiles;        // 2: a unit is two 128-row output tiles sharing every B stage
                        // (one accumulator each); otherwise one
  int64_t tiles_a;      // packed A tiles along the output rows: 128-row tiles of Phi
                        // (first product), 64-column tiles (second product)
  int fp8;              // FP8 E4M3 dictionary: the packed copy holds one byte per
                        // entry; converter warps turn each A tile into BF16
  const float* scales;  // FP8: scale of every 128 x 128 tile of Phi, row-major
  int64_t scale_cols;   // FP8: tiles per row of the scale table (ceil(D / 128))
  int64_t nkd;          // 64-column tiles of Phi (packed layout)
  // GEMM1: split-K partials (reduced and split by reduce_split_kernel)
  float* wpart;
  int64_t ldw;
  int64_t split_stride;
  // batched GEMM1: problems with one K range write the BF16 terms of W
  // directly (rows as the second product reads them, pitch ldw_terms)
  // instead of FP32 partials; null: always partials
  __nv_bfloat16* wterms;
  int64_t ldw_terms;

  // GEMM2
  float* y;
  const float* x;
  int64_t ld;
  const double* alpha;
  const float* alpha32;  // FP32 copy of alpha (same values as (float)alpha), or null
  double beta;
  double* dots;
  int* err;
  // batched mode (items != null): gridDim.x work items
  const TcItem* items;
  const TcProb* probs;
  const int* done;       // per-problem converged flags: their items exit at once
  const int* gate;       // if set and *gate == 0 the launch does nothing
};

__device__ __forceinline__ void tc_fail(int* err, volatile int* abort) {
  *abort = 1;
  if (err) atomicCAS(err, 0, (int)COFEM_ERR_TIMEOUT);
}

template <int NT>
__device__ __forceinline__ void split_terms(float x, __nv_bfloat16 (&o)[NT]) {
  float r = x;
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    o[t] = __float2bfloat16_rn(r);
    r = r - __bfloat162float(o[t]);
  }
}

// One work unit: a 128-row output tile and a K range of one product (of one
// problem, in the batched mode).
struct TcUnit {
  int64_t m0, M, nkd, ldo, xoff, aoff, woff, sstride, bx0, wo;
  double beta;
  int kb0, kb1, split, dslot;
  bool direct;             // GEMM1 writes BF16 terms of W at column offset wo
  const __nv_bfloat16* pk;
};

template <int MODE>
__device__ __forceinline__ TcUnit tc_unit(const TcArgs& args, int w) {
  TcUnit u;
  u.M = args.M;
  u.nkd = args.nkd;
  u.ldo = MODE == 0 ? args.ldw : args.ld;
  u.xoff = u.aoff = u.woff = u.bx0 = u.wo = 0;
  u.direct = false;
  u.sstride = args.split_stride;
  u.beta = args.beta;
  u.pk = args.packed;
  if (args.items) {
    const TcItem it = args.items[w];
    const TcProb pr = args.probs[it.prob];
    u.m0 = (int64_t)it.tile * kTileM;
    u.kb0 = it.kb0;
    u.kb1 = it.kb1;
    u.split = it.split;
    u.M = MODE == 0 ? pr.N : pr.D;
    u.nkd = pr.nkd;
    u.pk += pr.poff;
    u.ldo = MODE == 0 ? pr.ldw : pr.ld;
    u.xoff = pr.xoff;
    u.aoff = pr.aoff;
    u.woff = pr.wpoff;
    u.sstride = (int64_t)args.nc * pr.ldw;
    u.bx0 = MODE == 0 ? pr.boff1 : pr.boff2;
    u.dslot = pr.dots_base + it.tile;
    u.beta = pr.beta;
    u.direct = MODE == 0 && args.wterms && pr.S1 == 1;
    u.wo = pr.boff2;
  } else {
    const int tile = w % args.units_m, split = w / args.units_m;
    const int mt = args.row_tiles > 1 ? 2 : 1;
    u.m0 = (int64_t)tile * kTileM * mt;
    u.kb0 = split * args.kb_per_split;
    u.kb1 = min(args.nk_total, u.kb0 + args.kb_per_split);
    u.split = split;
    u.dslot = tile * mt;
  }
  return u;
}

// Batched mode: the units of a converged problem are skipped (by every role
// alike: the flags were written by an earlier kernel and do not change).
__device__ __forceinline__ bool unit_skipped(const TcArgs& args, int w) {
  return args.items && args.done && args.done[args.items[w].prob];
}

// Persistent CTAs: CTA b takes the work units b, b + gridDim.x, ...  The
// shared-memory ring runs on across units (one K-block counter for the
// whole CTA), and two tensor-memory accumulators alternate between units so
// that the epilogue of one unit overlaps the main loop of the next.
// Two E4M3 values (low byte first) times `scale`, rounded to BF16 (the
// FP8 -> FP16 conversion is exact; the product is rounded to FP32, then to
// BF16, both to nearest even).
__device__ __forceinline__ uint32_t e4m3x2_to_bf16x2(uint16_t v, float scale) {
  const __half2_raw h = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)v, __NV_E4M3);
  const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&h));
  const __nv_bfloat162 b = __floats2bfloat162_rn(f.x * scale, f.y * scale);
  return *reinterpret_cast<const uint32_t*>(&b);
}

template <int MODE, int NT, bool A8>
__global__ void __launch_bounds__(A8 ? kTcThreadsFp8 : kTcThreads, 1)
dense_tc_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                const TcArgs args) {
  pdl_wait();
  pdl_trigger();
  if (args.gate && *args.gate == 0) return;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t b_bytes = (uint32_t)args.BN * 128u;
  const int PT = args.phi_terms > 1 ? 2 : 1;          // BF16 terms of Phi
  const int MT = args.row_tiles > 1 ? 2 : 1;          // 128-row output tiles per unit
  // a stage holds MT x PT A tiles (tile (mt, pt) at (mt PT + pt) x 16 KB) and one B tile
  const uint32_t a_bytes = (uint32_t)(MT * PT) * kATileBytes;
  // FP8: the bulk copy lands in a staging area after the B tile (half the
  // bytes of the BF16 A tile), which the converter warps expand into A
  const uint32_t a8_bytes = A8 ? kATileBytes / 2 : 0u;
  const uint32_t stage_bytes = a_bytes + b_bytes + a8_bytes;
  const int S = args.stages;
  uint64_t* full = (uint64_t*)(smem + S * stage_bytes);
  uint64_t* empty = full + kMaxStages;
  uint64_t* accfull = empty + kMaxStages;          // [2] accumulator ready
  uint64_t* accempty = accfull + 2;                // [2] accumulator drained
  uint64_t* conv = accempty + 2;                   // [stages] FP8: A converted to BF16
  uint32_t* tmem_slot = (uint32_t*)(conv + kMaxStages);
  volatile int* abort = (volatile int*)(tmem_slot + 1);
  volatile int* bigflag = (volatile int*)(tmem_slot + 2);
  // epilogue partial dots per warp and column: compensated FP32 pairs, and
  // FP64 side sums of out-of-range products (flagged in *bigflag)
  float2* redp = (float2*)(tmem_slot + 4);          // [4][64]
  double* redb = (double*)(redp + 4 * 64);           // [4][64]

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int units = args.units;
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
      tc::mbar_init(&conv[s], kCvtWarps);          // the converter warps
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&accfull[b], 1);
      tc::mbar_init(&accempty[b], 4);              // the four epilogue warps
    }
    *abort = 0;
    *bigflag = 0;
    tc::fence_mbar_init();
    tc::prefetch_tmap(&mapA);
    tc::prefetch_tmap(&mapB);
  }
  if (warp == 1) {
    tc::tmem_alloc(tmem_slot, args.tmem_cols);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      const uint64_t pol_first = tc::policy_evict_first();
      const uint64_t pol_last = tc::policy_evict_last();
      const uint64_t pol_b = pol_last;
      int it = 0;                                  // K blocks issued by this CTA
      for (int w = blockIdx.x; w < units && !*abort; w += gridDim.x) {
        if (unit_skipped(args, w)) continue;
        const TcUnit u = tc_unit<MODE>(args, w);
        const int nk = max(0, u.kb1 - u.kb0);
        for (int i = 0; i < nk; ++i, ++it) {
          const int s = it % S;
          const uint32_t ph = (uint32_t)(it / S) & 1u;
          if (!tc::mbar_wait(&empty[s], ph ^ 1u, abort, kWaitLimitNs)) {
            tc_fail(args.err, abort);
            break;
          }
          uint8_t* sa = smem + s * stage_bytes;
          uint8_t* sb = sa + a_bytes;
          const int kb = u.kb0 + i;
          const int64_t m0 = u.m0;
          if constexpr (A8) {
            // one byte per entry: the same tile layout as the BF16 copy, each
            // byte standing at the position of its BF16 value
            uint8_t* s8 = sb + b_bytes;
            const uint8_t* pk8 = reinterpret_cast<const uint8_t*>(u.pk);
            tc::mbar_arrive_expect_tx(&full[s], a8_bytes + b_bytes);
            const uint64_t pol_a = pol_first;
            if (MODE == 0) {
              tc::bulk_load(s8, pk8 + ((m0 >> 7) * u.nkd + kb) * (int64_t)(kTileM * kTileK),
                            a8_bytes, &full[s], pol_a);
            } else {
              const int64_t c = m0 >> 6;
              const int64_t base = ((int64_t)(kb >> 1) * u.nkd + c) * kTileM + (kb & 1) * 64;
              const uint8_t* src = pk8 + base * kTileK;
              const uint8_t* src2 = c + 1 < u.nkd ? src + kTileM * kTileK : src;
              tc::bulk_load(s8, src, a8_bytes / 2, &full[s], pol_a);
              tc::bulk_load(s8 + a8_bytes / 2, src2, a8_bytes / 2, &full[s], pol_a);
            }
            tc::tma_load_2d(sb, &mapB, &full[s], (int)(u.bx0 + (int64_t)kb * kTileK), 0, pol_b);
            continue;
          }
          tc::mbar_arrive_expect_tx(&full[s], stage_bytes);
          // Phi columns below res_d stay in L2 between the two products and
          // across CG iterations; the rest streams through
          if (MODE == 0) {
            const uint64_t pol_a = (int64_t)kb * kTileK < args.res_d ? pol_last : pol_first;
            if (u.pk) {  // tile (m0 / 128 + mt, kb): one contiguous 16 KB copy per term
              for (int mt = 0; mt < MT; ++mt) {
                // past the last row tile the first tile is copied again: it only
                // feeds output rows >= M, which are not stored
                int64_t rt = (m0 >> 7) + mt;
                if (args.items == nullptr && rt >= args.tiles_a) rt = m0 >> 7;
                const __nv_bfloat16* src = u.pk + (rt * u.nkd + kb) * (kTileM * kTileK);
                uint8_t* dst = sa + (uint32_t)(mt * PT) * kATileBytes;
                tc::bulk_load(dst, src, kATileBytes, &full[s], pol_a);
                if (PT == 2)
                  tc::bulk_load(dst + kATileBytes, src + args.term_stride, kATileBytes, &full[s],
                                pol_a);
              }
            } else if (MT == 2) {
              tc::tma_load_2d(sa, &mapA, &full[s], kb * kTileK, (int)m0, pol_a);
              tc::tma_load_2d(sa + kATileBytes, &mapA, &full[s], kb * kTileK, (int)m0 + kTileM,
                              pol_a);
            } else
              tc::tma_load_2d(sa, &mapA, &full[s], kb * kTileK, (int)m0, pol_a);
          } else {
            const uint64_t pol_a = m0 < args.res_d ? pol_last : pol_first;
            if (u.pk) {
              for (int mt = 0; mt < MT; ++mt) {
                // rows n = 64 kb .. +64 are half (kb & 1) of row tile kb / 2; the
                // two 64-column tiles c and c + 1 give the 128 d's of output tile mt
                int64_t c = (m0 >> 6) + 2 * mt;
                if (args.items == nullptr && c >= u.nkd) c = m0 >> 6;   // rows >= M: not stored
                const int64_t base = ((int64_t)(kb >> 1) * u.nkd + c) * kTileM + (kb & 1) * 64;
                const __nv_bfloat16* src = u.pk + base * kTileK;
                uint8_t* dst = sa + (uint32_t)(mt * PT) * kATileBytes;
                tc::bulk_load(dst, src, kATileBytes / 2, &full[s], pol_a);
                // the next 64-column tile; past the last one (D not a multiple of
                // 128) the same half-tile is copied again: it only feeds output
                // rows d >= D, which are not stored
                const __nv_bfloat16* src2 = c + 1 < u.nkd ? src + kTileM * kTileK : src;
                tc::bulk_load(dst + kATileBytes / 2, src2, kATileBytes / 2, &full[s], pol_a);
                if (PT == 2) {
                  tc::bulk_load(dst + kATileBytes, src + args.term_stride, kATileBytes / 2,
                                &full[s], pol_a);
                  tc::bulk_load(dst + kATileBytes + kATileBytes / 2, src2 + args.term_stride,
                                kATileBytes / 2, &full[s], pol_a);
                }
              }
            } else {
              for (int mt = 0; mt < MT; ++mt) {
                uint8_t* dst = sa + (uint32_t)mt * kATileBytes;
                tc::tma_load_2d(dst, &mapA, &full[s], (int)m0 + kTileM * mt, kb * kTileK, pol_a);
                tc::tma_load_2d(dst + kATileBytes / 2, &mapA, &full[s], (int)m0 + kTileM * mt + 64,
                                kb * kTileK, pol_a);
              }
            }
          }
          tc::tma_load_2d(sb, &mapB, &full[s], (int)(u.bx0 + (int64_t)kb * kTileK), 0, pol_b);
        }
      }
      if (*abort) {
        // drain this CTA's copies still in flight before leaving
        volatile int never = 0;
        for (int i = max(0, it - S); i < it; ++i)
          tc::mbar_wait(&full[i % S], (uint32_t)(i / S) & 1u, &never, kWaitLimitNs);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // A is K-major in the first product, MN-major (Phi^T read in place) in the second
      const uint32_t idesc = tc::idesc_bf16_f32(kTileM, args.BN, MODE == 1 ? 1 : 0, 0);
      int it = 0, lu = -1;
      for (int w = blockIdx.x; w < units && !*abort; w += gridDim.x) {
        if (unit_skipped(args, w)) continue;
        ++lu;
        const TcUnit u = tc_unit<MODE>(args, w);
        const int nk = max(0, u.kb1 - u.kb0);
        const int b = lu & 1;
        // the epilogue must have drained this accumulator (its previous unit)
        if (!tc::mbar_wait(&accempty[b], (uint32_t)((lu >> 1) & 1) ^ 1u, abort, 4 * kWaitLimitNs)) {
          tc_fail(args.err, abort);
          break;
        }
        tc::tc_fence_after();
        const uint32_t acc0 = tmem + (uint32_t)(b * MT) * args.acc_cols;
        for (int i = 0; i < nk; ++i, ++it) {
          const int s = it % S;
          const uint32_t ph = (uint32_t)(it / S) & 1u;
          if (!tc::mbar_wait(&full[s], ph, abort, kWaitLimitNs) ||
              (A8 && !tc::mbar_wait(&conv[s], ph, abort, kWaitLimitNs))) {
            tc_fail(args.err, abort);
            break;
          }
          tc::tc_fence_after();
          const uint32_t a_base = tc::smem_u32(smem + s * stage_bytes);
          const uint32_t b_base = a_base + a_bytes;
          for (int mt = 0; mt < MT; ++mt) {
            const uint32_t acc = acc0 + (uint32_t)mt * args.acc_cols;
            for (int pt = 0; pt < PT; ++pt) {
              const uint32_t at = a_base + (uint32_t)(mt * PT + pt) * kATileBytes;
#pragma unroll
              for (int k = 0; k < kTileK / 16; ++k) {
                uint64_t adesc;
                if (MODE == 0) adesc = tc::smem_desc_sw128(at + k * 32, 16, 1024);
                else adesc = tc::smem_desc_sw128(at + k * 2048, kATileBytes / 2, 1024);
                const uint64_t bdesc = tc::smem_desc_sw128(b_base + k * 32, 16, 1024);
                tc::mma_bf16(acc, adesc, bdesc, idesc, (i > 0 || k > 0 || pt > 0) ? 1u : 0u);
              }
            }
          }
          tc::mma_commit(&empty[s]);
        }
        tc::mma_commit(&accfull[b]);
      }
    }
  } else if (A8 && warp >= kTcThreads / 32) {
    // ------------------------------------------------- FP8 -> BF16 (A tiles)
    // kCvtWarps warps expand each stage's 8 KB of E4M3 bytes into the 16 KB
    // BF16 A tile, times the scale of the 128 x 128 tile of Phi it belongs
    // to; each thread loads all its chunks before converting any (the loads
    // overlap) and stores after
    constexpr int kCvtThreads = kCvtWarps * 32;
    constexpr int kChunks = 512 / kCvtThreads;   // 16-byte chunks per thread and stage
    const int ct = threadIdx.x - kTcThreads;
    int it = 0;
    for (int w = blockIdx.x; w < units && !*abort; w += gridDim.x) {
      if (unit_skipped(args, w)) continue;
      const TcUnit u = tc_unit<MODE>(args, w);
      const int nk = max(0, u.kb1 - u.kb0);
      bool ok = true;
      for (int i = 0; i < nk; ++i, ++it) {
        const int s = it % S;
        const uint32_t ph = (uint32_t)(it / S) & 1u;
        if (!tc::mbar_wait(&full[s], ph, abort, kWaitLimitNs)) {
          tc_fail(args.err, abort);
          ok = false;
          break;
        }
        const int kb = u.kb0 + i;
        const float scale = MODE == 0 ? args.scales[(u.m0 >> 7) * args.scale_cols + (kb >> 1)]
                                      : args.scales[(int64_t)(kb >> 1) * args.scale_cols + (u.m0 >> 7)];
        uint8_t* sa = smem + s * stage_bytes;
        const uint4* s8 = reinterpret_cast<const uint4*>(sa + a_bytes + b_bytes);
        uint4* d16 = reinterpret_cast<uint4*>(sa);
        uint4 v[kChunks];
#pragma unroll
        for (int q = 0; q < kChunks; ++q) v[q] = s8[q * kCvtThreads + ct];
#pragma unroll
        for (int q = 0; q < kChunks; ++q) {
          const int c16 = q * kCvtThreads + ct;    // 16-byte chunk of FP8 bytes
          const uint32_t w4[4] = {v[q].x, v[q].y, v[q].z, v[q].w};
          uint32_t o[8];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            o[2 * k] = e4m3x2_to_bf16x2((uint16_t)(w4[k] & 0xffffu), scale);
            o[2 * k + 1] = e4m3x2_to_bf16x2((uint16_t)(w4[k] >> 16), scale);
          }
          d16[2 * c16] = make_uint4(o[0], o[1], o[2], o[3]);
          d16[2 * c16 + 1] = make_uint4(o[4], o[5], o[6], o[7]);
        }
        tc::fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&conv[s]);
      }
      if (!ok) break;
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int g = warp & 3;                 // tensor-memory lane quarter of this warp
    constexpr int G = TermGroup<NT>::G, COLS = TermGroup<NT>::COLS;
    const int ngroups = (args.nc + G - 1) / G;
    int lu = -1;
    for (int w = blockIdx.x; w < units; w += gridDim.x) {
      if (unit_skipped(args, w)) continue;
      ++lu;
      const TcUnit u = tc_unit<MODE>(args, w);
      const int nk = max(0, u.kb1 - u.kb0);
      const int b = lu & 1;
      // rows of the unit's first output tile (the second tile, if any, follows)
      int64_t row = u.m0 + 32 * g + lane;
      bool live = row < u.M;
      float a32 = 0.f;                     // alpha_row in FP32, converted once per row
      if (MODE == 1 && live)
        a32 = args.alpha32 ? args.alpha32[u.aoff + row]
                           : (args.alpha ? (float)args.alpha[u.aoff + row] : 0.f);
      // second product: x of the next column group is loaded while the
      // current group is processed (one group ahead; the first group while
      // the main loop runs)
      float xnext[G];
      if (MODE == 1) {
#pragma unroll
        for (int jj = 0; jj < G; ++jj)
          xnext[jj] = (live && jj < args.nc) ? args.x[u.xoff + (int64_t)jj * u.ldo + row] : 0.f;
      }
      const bool ok1 = tc::mbar_wait(&accfull[b], (uint32_t)((lu >> 1) & 1), abort,
                                     4 * kWaitLimitNs);
      if (!ok1) tc_fail(args.err, abort);
      // the four epilogue warps take the same decision (named barrier 2)
      uint32_t okall;
      asm volatile(
          "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
          "bar.red.and.pred q, 2, 128, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
          : "=r"(okall)
          : "r"((uint32_t)ok1)
          : "memory");
      if (!okall) break;
      tc::tc_fence_after();
      for (int mt = 0; mt < MT; ++mt) {
      if (mt > 0) {
        row = u.m0 + kTileM * mt + 32 * g + lane;
        live = row < u.M;
        a32 = 0.f;
        if (MODE == 1 && live)
          a32 = args.alpha32 ? args.alpha32[u.aoff + row]
                             : (args.alpha ? (float)args.alpha[u.aoff + row] : 0.f);
        if (MODE == 1) {
#pragma unroll
          for (int jj = 0; jj < G; ++jj)
            xnext[jj] = (live && jj < args.nc) ? args.x[u.xoff + (int64_t)jj * u.ldo + row] : 0.f;
        }
      }
      const uint32_t acc = tmem + (uint32_t)(b * MT + mt) * args.acc_cols;
      for (int gi = 0; gi < ngroups; ++gi) {
        float xcur[G];
        if (MODE == 1) {
#pragma unroll
          for (int jj = 0; jj < G; ++jj) {
            xcur[jj] = xnext[jj];
            const int jn = (gi + 1) * G + jj;
            xnext[jj] = (live && jn < args.nc) ? args.x[u.xoff + (int64_t)jn * u.ldo + row] : 0.f;
          }
        }
        float v[COLS];
#pragma unroll
        for (int c = 0; c < COLS / 16; ++c) {
          float t16[16];
          tc::tmem_ld16(acc + ((uint32_t)(32 * g) << 16) + (uint32_t)(gi * COLS + 16 * c), t16);
#pragma unroll
          for (int q = 0; q < 16; ++q) v[16 * c + q] = t16[q];
        }
        tc::tmem_ld_wait();
        if (nk == 0) {
#pragma unroll
          for (int q = 0; q < COLS; ++q) v[q] = 0.f;
        }
        // x_j^T y_j over the warp's 32 rows (second product): compensated
        // FP32 (product error by FMA, TwoSum butterflies, the G columns of
        // the group interleaved); products of 1e30 or more take an FP64
        // side sum
        float ds[G], dc[G];
        double db[G];
        bool anybig = false;
#pragma unroll
        for (int jj = 0; jj < G; ++jj) {
          const int j = gi * G + jj;
          float sacc = 0.f;
#pragma unroll
          for (int t = NT - 1; t >= 0; --t) sacc += v[jj * NT + t];
          ds[jj] = 0.f;
          dc[jj] = 0.f;
          db[jj] = 0.0;
          if (MODE == 0) {
            if (j < args.nc && live) {
              if (u.direct) {
                __nv_bfloat16 o[NT];
                split_terms<NT>(sacc, o);
#pragma unroll
                for (int t = 0; t < NT; ++t)
                  args.wterms[(int64_t)(gi * 16 + jj * NT + t) * args.ldw_terms + u.wo + row] = o[t];
              } else {
                args.wpart[u.woff + (int64_t)u.split * u.sstride + (int64_t)j * u.ldo + row] = sacc;
              }
            }
          } else if (j < args.nc && live) {
            const float xv = xcur[jj];
            const float yv = fmaf(a32, xv, (float)u.beta * sacc);
            args.y[u.xoff + (int64_t)j * u.ldo + row] = yv;
            const float pp = xv * yv;
            if (fabsf(pp) < 1e30f) {
              ds[jj] = pp;
              dc[jj] = fmaf(xv, yv, -pp);
            } else {
              db[jj] = (double)xv * (double)yv;
              anybig = true;
            }
          }
        }
        if (MODE == 1 && args.dots) {
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int jj = 0; jj < G; ++jj)
              two_sum_merge(ds[jj], dc[jj], __shfl_xor_sync(0xffffffffu, ds[jj], o),
                            __shfl_xor_sync(0xffffffffu, dc[jj], o));
          }
          if (__any_sync(0xffffffffu, anybig)) {
#pragma unroll
            for (int jj = 0; jj < G; ++jj) db[jj] = warp_sum(db[jj]);
            if (lane == 0) *bigflag = 1;
          }
          if (lane == 0) {
#pragma unroll
            for (int jj = 0; jj < G; ++jj)
              if (gi * G + jj < args.nc) {
                redp[(warp - 2) * 64 + gi * G + jj] = make_float2(ds[jj], dc[jj]);
                redb[(warp - 2) * 64 + gi * G + jj] = db[jj];
              }
          }
        }
      }
      if (mt == MT - 1) {
        // this unit's accumulators are drained: the MMA may reuse them
        tc::tc_fence_before();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&accempty[b]);
      }
      if (MODE == 1 && args.dots) {
        asm volatile("bar.sync 1, 128;" ::: "memory");
        if (warp == 2) {
          const bool big = *bigflag != 0;
          for (int j = lane; j < args.nc; j += 32) {
            float ps = redp[j].x, pc = redp[j].y;
#pragma unroll
            for (int q = 1; q < 4; ++q) two_sum_merge(ps, pc, redp[q * 64 + j].x, redp[q * 64 + j].y);
            double t = (double)ps + (double)pc;
            if (big) t += redb[j] + redb[64 + j] + redb[128 + j] + redb[192 + j];
            args.dots[(int64_t)(u.dslot + mt) * kMaxCols + j] = t;
          }
          if (lane == 0) *bigflag = 0;
        }
        // the partials are read before the next tile writes them
        asm volatile("bar.sync 1, 128;" ::: "memory");
      }
      }   // output tiles of the unit
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, args.tmem_cols);
  }
}

// ------------------------------------------------------ split kernels

// Xs[split_row(j, t) * lds + d] = BF16 term t of X[j*ld + d]; rows of no
// (j < nc, t) are zero.  Grid (blocks, ngroups * G): one column slot j per
// blockIdx.y, four consecutive d per thread, one 8-byte store per term.
template <int NT>
__global__ void split_block_kernel(const float* __restrict__ X, int64_t ld, int64_t D,
                                   int64_t lds, int nc, __nv_bfloat16* __restrict__ Xs, const int* gate) {
  pdl_wait();
  pdl_trigger();
  if (gate && *gate == 0) return;
  constexpr int G = TermGroup<NT>::G;
  const int j = blockIdx.y;
  const int gi = j / G, jj = j % G;
  for (int64_t d = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) * 4; d < lds;
       d += (int64_t)gridDim.x * blockDim.x * 4) {
    float r[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) r[i] = (j < nc && d + i < D) ? X[(int64_t)j * ld + d + i] : 0.f;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      __nv_bfloat16 o[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        o[i] = __float2bfloat16_rn(r[i]);
        r[i] -= __bfloat162float(o[i]);
      }
      *reinterpret_cast<uint2*>(Xs + (int64_t)(gi * 16 + jj * NT + t) * lds + d) =
          *reinterpret_cast<uint2*>(o);
    }
    if (jj == G - 1) {     // rows of the group left over by G * NT < 16
      for (int rr = G * NT; rr < 16; ++rr)
        *reinterpret_cast<uint2*>(Xs + (int64_t)(gi * 16 + rr) * lds + d) = make_uint2(0u, 0u);
    }
  }
}

// W[j][n] = sum_s Wpart[s][j][n] (split order) -> BF16 terms of W in rows
// split_row(j, t) of Ws; rows of no (j < nc, t) and n >= N are zero.
// Grid (blocks, ngroups * G): one column slot per blockIdx.y, four
// consecutive n per thread (16-byte loads, 8-byte stores per term).
template <int NT>
__global__ void reduce_split_kernel(const float* __restrict__ Wp, int S, int64_t sstride,
                                    int64_t N, int64_t ldw, int nc,
                                    __nv_bfloat16* __restrict__ Ws, const int* gate) {
  pdl_wait();
  pdl_trigger();
  if (gate && *gate == 0) return;
  constexpr int G = TermGroup<NT>::G;
  const int j = blockIdx.y;
  const int gi = j / G, jj = j % G;
  for (int64_t n = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) * 4; n < ldw;
       n += (int64_t)gridDim.x * blockDim.x * 4) {
    float r[4] = {0.f, 0.f, 0.f, 0.f};
    if (j < nc) {
      for (int s = 0; s < S; ++s) {
        const float4 v = __ldcg(reinterpret_cast<const float4*>(Wp + (int64_t)s * sstride +
                                                                (int64_t)j * ldw + n));
        r[0] += v.x; r[1] += v.y; r[2] += v.z; r[3] += v.w;
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (n + i >= N) r[i] = 0.f;
    }
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      __nv_bfloat16 o[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        o[i] = __float2bfloat16_rn(r[i]);
        r[i] -= __bfloat162float(o[i]);
      }
      *reinterpret_cast<uint2*>(Ws + (int64_t)(gi * 16 + jj * NT + t) * ldw + n) =
          *reinterpret_cast<uint2*>(o);
    }
    if (jj == G - 1) {
      for (int rr = G * NT; rr < 16; ++rr)
        *reinterpret_cast<uint2*>(Ws + (int64_t)(gi * 16 + rr) * ldw + n) = make_uint2(0u, 0u);
    }
  }
}

// Tile (mt, kb) = Phi[128 mt + r][64 kb + c], r < 128, c < 64, stored as the
// 128-byte-swizzled shared-memory image the MMA reads: row r at r * 64
// values, its 16-byte chunk q (values 8q .. 8q+7) at chunk position
// q ^ (r mod 8).  Zero outside N x D.  One thread per 16-byte chunk.
__global__ void pack_kernel(const __nv_bfloat16* __restrict__ phi, int64_t N, int64_t D,
                            int64_t ld, int64_t nkd, int64_t total8,
                            __nv_bfloat16* __restrict__ packed) {
  pdl_wait();
  pdl_trigger();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total8;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = i * 8;                 // destination element of the chunk
    const int64_t row = e >> 6;              // packed row index
    const int c0 = (int)((((e & 63) >> 3) ^ (row & 7)) << 3);   // source column
    const int r = (int)(row & 127);
    const int64_t tile = row >> 7;
    const int64_t kb = tile % nkd, mt = tile / nkd;
    const int64_t n = mt * 128 + r, d0 = kb * 64 + c0;
    __nv_bfloat16 v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q)
      v[q] = (n < N && d0 + q < D) ? phi[n * ld + d0 + q] : __float2bfloat16_rn(0.f);
    *reinterpret_cast<uint4*>(packed + e) = *reinterpret_cast<uint4*>(v);
  }
}

// FP32 dictionary: the same tile layout, written twice -- image 0 holds
// hi = bf16(Phi), image 1 (total8 * 8 elements later) lo = bf16(Phi - hi).
__global__ void pack_f32_terms_kernel(const float* __restrict__ phi, int64_t N, int64_t D,
                                      int64_t ld, int64_t nkd, int64_t total8,
                                      __nv_bfloat16* __restrict__ packed) {
  pdl_wait();
  pdl_trigger();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total8;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = i * 8;
    const int64_t row = e >> 6;
    const int c0 = (int)((((e & 63) >> 3) ^ (row & 7)) << 3);
    const int r = (int)(row & 127);
    const int64_t tile = row >> 7;
    const int64_t kb = tile % nkd, mt = tile / nkd;
    const int64_t n = mt * 128 + r, d0 = kb * 64 + c0;
    __nv_bfloat16 hi[8], lo[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float v = (n < N && d0 + q < D) ? phi[n * ld + d0 + q] : 0.f;
      hi[q] = __float2bfloat16_rn(v);
      lo[q] = __float2bfloat16_rn(v - __bfloat162float(hi[q]));
    }
    *reinterpret_cast<uint4*>(packed + e) = *reinterpret_cast<uint4*>(hi);
    *reinterpret_cast<uint4*>(packed + total8 * 8 + e) = *reinterpret_cast<uint4*>(lo);
  }
}

void dense_pack_f32_terms(const float* phi, int64_t N, int64_t D, int64_t ld, void* packed,
                          cudaStream_t st) {
  const int64_t total8 = (int64_t)(packed_bytes(N, D) / 16);
  const int64_t blocks = (total8 + 255) / 256;
  launch_k(pack_f32_terms_kernel, dim3((unsigned)(blocks < 65535 ? blocks : 65535)), dim3(256), 0,
           st, phi, N, D, ld, packed_tiles_k(D), total8, (__nv_bfloat16*)packed);
}

// FP8 dictionary (one byte per entry, row-major with leading dimension ld):
// the same tile layout, one byte at the position of each BF16 value.
__global__ void pack_fp8_kernel(const uint8_t* __restrict__ phi, int64_t N, int64_t D,
                                int64_t ld, int64_t nkd, int64_t total8,
                                uint8_t* __restrict__ packed) {
  pdl_wait();
  pdl_trigger();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total8;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = i * 8;
    const int64_t row = e >> 6;
    const int c0 = (int)((((e & 63) >> 3) ^ (row & 7)) << 3);
    const int r = (int)(row & 127);
    const int64_t tile = row >> 7;
    const int64_t kb = tile % nkd, mt = tile / nkd;
    const int64_t n = mt * 128 + r, d0 = kb * 64 + c0;
    uint8_t v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = (n < N && d0 + q < D) ? phi[n * ld + d0 + q] : (uint8_t)0;
    *reinterpret_cast<uint2*>(packed + e) = *reinterpret_cast<uint2*>(v);
  }
}

void dense_pack_fp8(const void* phi, int64_t N, int64_t D, int64_t ld, void* packed,
                    cudaStream_t st) {
  const int64_t total8 = (int64_t)(packed_bytes(N, D) / 16);
  const int64_t blocks = (total8 + 255) / 256;
  launch_k(pack_fp8_kernel, dim3((unsigned)(blocks < 65535 ? blocks : 65535)), dim3(256), 0, st,
           (const uint8_t*)phi, N, D, ld, packed_tiles_k(D), total8, (uint8_t*)packed);
}

void dense_pack_bf16(const void* phi, int64_t N, int64_t D, int64_t ld, void* packed,
                     cudaStream_t st) {
  const int64_t total8 = (int64_t)(packed_bytes(N, D) / 16);
  const int64_t blocks = (total8 + 255) / 256;
  launch_k(pack_kernel, dim3((unsigned)(blocks < 65535 ? blocks : 65535)), dim3(256), 0, st, (const __nv_bfloat16*)phi, N, D, ld, packed_tiles_k(D), total8, (__nv_bfloat16*)packed);
}

// Bounded-wait self-test: one thread waits on phase 0 of an mbarrier that
// nothing arrives on, with the kernels' own wait routine.
__device__ int g_wait_selftest_err;
__global__ void wait_selftest_kernel(uint64_t limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x != 0) return;
  abort_flag = 0;
  tc::mbar_init(&bar, 1);
  tc::fence_mbar_init();
  if (!tc::mbar_wait(&bar, 0u, &abort_flag, limit_ns))
    atomicCAS(&g_wait_selftest_err, 0, (int)COFEM_ERR_TIMEOUT);
}

int wait_selftest(int64_t limit_ns, cudaStream_t st) {
  const int zero = 0;
  if (cudaMemcpyToSymbolAsync(g_wait_selftest_err, &zero, sizeof(int), 0,
                              cudaMemcpyHostToDevice, st) != cudaSuccess)
    return -1;
  wait_selftest_kernel<<<1, 32, 0, st>>>((uint64_t)limit_ns);
  if (cudaGetLastError() != cudaSuccess) return -1;
  int out = 0;
  if (cudaMemcpyFromSymbolAsync(&out, g_wait_selftest_err, sizeof(int), 0,
                                cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return -1;
  if (cudaStreamSynchronize(st) != cudaSuccess) return -1;
  return out;
}

// ----------------------------------------------------------- host side

// Optional per-kernel timing of one operator application (cofem_op_apply_timed):
// when armed, every launch site records an event after its kernel.
static thread_local cudaEvent_t* g_tick_events = nullptr;
static thread_local int g_tick_count = 0, g_tick_cap = 0;
void apply_ticks_arm(cudaEvent_t* events, int cap) {
  g_tick_events = events;
  g_tick_cap = cap;
  g_tick_count = 0;
}
int apply_ticks_disarm() {
  const int n = g_tick_count;
  g_tick_events = nullptr;
  g_tick_cap = 0;
  g_tick_count = 0;
  return n;
}
void apply_tick(cudaStream_t st) {
  if (g_tick_events && g_tick_count < g_tick_cap) cudaEventRecord(g_tick_events[g_tick_count++], st);
}

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

// 2-D bf16 map: inner extent `inner` (elements), `outer` rows, row pitch
// `pitch` elements, box {64, box_rows}, 128-byte swizzle, zero fill.
static bool make_map(CUtensorMap* m, const void* base, uint64_t inner, uint64_t outer,
                     uint64_t pitch, uint32_t box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {pitch * 2};
  cuuint32_t box[2] = {64, box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides,
                  box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

static int term_group(int NT) { return 16 / NT; }

DenseTcPlan dense_tc_plan(int64_t N, int64_t D, int nc, int NT, int sms, int ctas_per_sm,
                          int stages, int PT, int MT, bool fp8) {
  DenseTcPlan p;
  if (ctas_per_sm < 1 || ctas_per_sm > 4) ctas_per_sm = 2;
  MT = MT > 1 && !fp8 ? 2 : 1;
  if (fp8) PT = 1;
  p.fp8 = fp8;
  p.NT = NT;
  p.nc = nc;
  const int ngroups = (nc + term_group(NT) - 1) / term_group(NT);
  p.BN = ngroups * 16;
  uint32_t tc = 32;
  while (tc < (uint32_t)p.BN) tc <<= 1;
  p.acc_cols = tc;
  // the tensor memory holds 512 columns: two sets of MT accumulators must fit
  // (BN > 128, i.e. 256-column accumulators, leaves room for one tile per unit)
  if (2 * MT * tc > 512) MT = 1;
  p.MT = MT;
  p.tmem_cols = 2 * MT * tc;             // two sets of MT accumulators (persistent CTAs)
  p.ld = round_up(D, kLdAlign);
  p.ldw = round_up(N, kLdAlign);
  const int mt1 = (int)((N + kTileM * MT - 1) / (kTileM * MT));   // units along N
  p.nk1 = (int)((D + kTileK - 1) / kTileK);
  p.nk2 = (int)((N + kTileK - 1) / kTileK);
  int per_sm = 512 / (int)p.tmem_cols < ctas_per_sm ? 512 / (int)p.tmem_cols : ctas_per_sm;
  if (per_sm < 1) per_sm = 1;
  // split-K of the first product: the CTAs (at most per_sm * sms, one wave)
  // take mt1 x S1 units in turn.  The most K blocks any CTA streams is
  // ceil(mt1 S1 / grid) ceil(nk1 / S1); take the fewest splits (fewer
  // partial sums to write and reduce) within 10 % of the best balance.
  const int grid = per_sm * sms;
  auto per_cta = [&](int s1, int* kbps_out, int* s1_out) {
    const int kbps = (p.nk1 + s1 - 1) / s1;
    const int s1r = (p.nk1 + kbps - 1) / kbps;            // splits actually used
    *kbps_out = kbps;
    *s1_out = s1r;
    return (((int64_t)mt1 * s1r + grid - 1) / grid) * kbps;
  };
  int64_t best = -1;
  for (int s1 = 1; s1 <= 32 && s1 <= p.nk1; ++s1) {
    int kb, sr;
    const int64_t w = per_cta(s1, &kb, &sr);
    if (best < 0 || w < best) best = w;
  }
  for (int s1 = 1; s1 <= 32 && s1 <= p.nk1; ++s1) {
    int kb, sr;
    if (per_cta(s1, &kb, &sr) * 10 <= best * 11) { p.S1 = sr; p.kbps1 = kb; break; }
  }
  const size_t fixed = 1024 + 3 * kMaxStages * 8 + 32 + 64 + 4 * 64 * 8 * 2 + 64;
  const size_t stage = (size_t)((PT > 1 ? 2 : 1) * MT) * kATileBytes + (size_t)p.BN * 128 +
                       (fp8 ? kATileBytes / 2 : 0);
  // each resident CTA also costs 1 KB of reserved shared memory
  const size_t budget = kSmemPerSm / per_sm - 1024;
  int st = (int)((budget - fixed) / stage);
  if (st > kMaxStages) st = kMaxStages;
  if (stages > 0 && stages < st) st = stages;
  if (st < 2) st = 2;
  p.stages = st;
  p.smem = st * stage + fixed;
  // accumulators that fill the tensor memory leave room for one CTA per SM:
  // ask for more than half of the shared memory as well, so that a second
  // CTA never lands on the SM and waits in its tensor-memory allocation
  if (p.tmem_cols > 256 && p.smem < kSmemPerSm / 2 + 1024) p.smem = kSmemPerSm / 2 + 1024;
  p.grid = grid;
  p.off_xs = 0;
  p.bytes_xs = round_up((int64_t)p.BN * p.ld * 2, 256);
  p.off_wpart = p.bytes_xs;
  p.bytes_wpart = round_up((int64_t)p.S1 * nc * p.ldw * 4, 256);
  p.off_ws = p.off_wpart + p.bytes_wpart;
  p.bytes_ws = round_up((int64_t)p.BN * p.ldw * 2, 256);
  p.total = p.off_ws + p.bytes_ws;
  return p;
}

template <int MODE, int NT>
static cudaError_t launch_tc(dim3 grid, size_t smem, const CUtensorMap& a, const CUtensorMap& b,
                             const TcArgs& args, cudaStream_t st) {
  if (args.fp8) {
    if constexpr (NT == 3) {
      auto k = dense_tc_kernel<MODE, NT, true>;
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      launch_k(k, dim3(grid), dim3(kTcThreadsFp8), smem, st, a, b, args);
      return cudaGetLastError();
    } else {
      return cudaErrorInvalidValue;          // FP8 dictionaries take three vector terms
    }
  }
  auto k = dense_tc_kernel<MODE, NT, false>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  launch_k(k, dim3(grid), dim3(kTcThreads), smem, st, a, b, args);
  return cudaGetLastError();
}

template <int NT>
static int dense_tc_apply_t(const DenseDesc& op, const float* X, int64_t ld, int nc, float* Y,
                            double beta, const double* alpha, double* dots, int* nparts,
                            char* ws, int* err, unsigned flags, cudaStream_t st,
                            const float* alpha32, const int* gate) {
  const int sms = num_sms();
  const bool fp8 = op.dtype == COFEM_FP8_E4M3;
  const int PT = op.phi_terms > 1 && op.packed ? 2 : 1;
  DenseTcPlan p = dense_tc_plan(op.N, op.D, nc, NT, sms, op.tc_ctas_per_sm, op.tc_stages, PT,
                                op.tc_row_tiles > 1 ? 2 : 1, fp8);
  const int MT = p.MT;                   // the plan falls back to one tile when TMEM is short
  if (fp8 && !op.packed) return 1;       // FP8 dictionaries run from the packed copy only
  const bool presplit = (flags & kApplyPresplit) != 0;
  __nv_bfloat16* Xs = (__nv_bfloat16*)(ws + p.off_xs);
  float* Wp = (float*)(ws + p.off_wpart);
  __nv_bfloat16* Ws = (__nv_bfloat16*)(ws + p.off_ws);
  // split X (leading dim ld) into BF16 terms Xs (pitch p.ld): GEMM1's operand
  // (skipped when the caller's kernels already wrote Xs)
  if (!presplit) {
    const int64_t need4 = (p.ld / 4 + 255) / 256;
    dim3 g((unsigned)(need4 < 64 ? need4 : 64), (p.BN / 16) * TermGroup<NT>::G);
    launch_k(split_block_kernel<NT>, dim3(g), dim3(256), 0, st, X, ld, op.D, p.ld, nc, Xs, gate);
    apply_tick(st);
  }
  CUtensorMap mPhi1, mXs, mPhi2, mWs;
  const int64_t nkd = packed_tiles_k(op.D);
  if (op.packed) {
    const uint64_t rows = (uint64_t)packed_tiles_m(op.N) * nkd * kTileM;
    if (!make_map(&mPhi1, op.packed, 64, rows, 64, kTileM)) return 1;
    if (!make_map(&mPhi2, op.packed, 64, rows, 64, 64)) return 1;
  } else {
    if (!make_map(&mPhi1, op.phi, op.D, op.N, op.ld, kTileM)) return 1;
    if (!make_map(&mPhi2, op.phi, op.D, op.N, op.ld, 64)) return 1;
  }
  if (!make_map(&mXs, Xs, op.D, p.BN, p.ld, p.BN)) return 1;
  if (!make_map(&mWs, Ws, op.N, p.BN, p.ldw, p.BN)) return 1;

  TcArgs a1 = {};
  a1.M = op.N;
  a1.nk_total = p.nk1;
  a1.kb_per_split = p.kbps1;
  a1.nc = nc;
  a1.BN = p.BN;
  a1.stages = p.stages;
  a1.tmem_cols = p.tmem_cols;
  a1.res_d = op.l2_resident_cols;
  a1.packed = (const __nv_bfloat16*)op.packed;
  a1.phi_terms = PT;
  a1.term_stride = (int64_t)(packed_bytes(op.N, op.D) / 2);
  a1.nkd = nkd;
  a1.wpart = Wp;
  a1.ldw = p.ldw;
  a1.split_stride = (int64_t)nc * p.ldw;
  a1.err = err;
  a1.gate = gate;
  a1.row_tiles = MT;
  a1.tiles_a = packed_tiles_m(op.N);
  a1.fp8 = fp8;
  a1.scales = op.scales;
  a1.scale_cols = (op.D + 127) / 128;
  a1.units_m = (int)((op.N + kTileM * MT - 1) / (kTileM * MT));
  a1.units = a1.units_m * p.S1;
  a1.acc_cols = p.acc_cols;
  dim3 g1((unsigned)std::min(a1.units, p.grid), 1);
  if (launch_tc<0, NT>(g1, p.smem, mPhi1, mXs, a1, st) != cudaSuccess) return 2;
  apply_tick(st);
  {
    const int64_t need4 = (p.ldw / 4 + 127) / 128;
    dim3 g((unsigned)(need4 < 64 ? need4 : 64), (p.BN / 16) * TermGroup<NT>::G);
    launch_k(reduce_split_kernel<NT>, dim3(g), dim3(128), 0, st, Wp, p.S1, a1.split_stride, op.N, p.ldw, nc, Ws, gate);
    apply_tick(st);
  }


  TcArgs a2 = {};
  a2.M = op.D;
  a2.nk_total = p.nk2;
  a2.kb_per_split = p.nk2;
  a2.nc = nc;
  a2.BN = p.BN;
  a2.stages = p.stages;
  a2.tmem_cols = p.tmem_cols;
  a2.res_d = op.l2_resident_cols;
  a2.packed = (const __nv_bfloat16*)op.packed;
  a2.phi_terms = PT;
  a2.term_stride = a1.term_stride;
  a2.nkd = nkd;
  a2.y = Y;
  a2.x = X;
  a2.ld = ld;
  a2.alpha = alpha;
  a2.alpha32 = alpha32;
  a2.beta = beta;
  a2.dots = dots;
  a2.err = err;
  a2.gate = gate;
  a2.row_tiles = MT;
  a2.tiles_a = nkd;
  a2.fp8 = fp8;
  a2.scales = op.scales;
  a2.scale_cols = (op.D + 127) / 128;
  a2.units_m = (int)((op.D + kTileM * MT - 1) / (kTileM * MT));
  a2.units = a2.units_m;
  a2.acc_cols = p.acc_cols;
  dim3 g2((unsigned)std::min(a2.units, p.grid), 1);
  if (launch_tc<1, NT>(g2, p.smem, mPhi2, mWs, a2, st) != cudaSuccess) return 2;
  apply_tick(st);
  if (nparts) *nparts = dots ? a2.units * MT : 0;
  return 0;
}

int dense_tc_batched(int mode, int NT, int nitems, const TcItem* items, const TcProb* probs,
                     const int* done, const void* packed, const __nv_bfloat16* bsrc,
                     int64_t b_cols, int BN, int nc, int stages, uint32_t tmem_cols,
                     size_t smem, float* wpart, const float* X, float* Y, const double* alpha,
                     double* dots, int* err, cudaStream_t st, int grid,
                     __nv_bfloat16* wterms, int64_t ldw_terms) {
  CUtensorMap mA, mB;
  // mapA is unused in the batched mode (Phi comes from the packed copy);
  // any valid map will do
  if (!make_map(&mA, bsrc, (uint64_t)b_cols, (uint64_t)BN, (uint64_t)b_cols, 64)) return 1;
  if (!make_map(&mB, bsrc, (uint64_t)b_cols, (uint64_t)BN, (uint64_t)b_cols, (uint32_t)BN)) return 1;
  TcArgs a = {};
  a.nc = nc;
  a.BN = BN;
  a.stages = stages;
  a.tmem_cols = tmem_cols;
  a.acc_cols = tmem_cols / 2;               // two accumulators
  a.units = nitems;
  a.units_m = 1;
  a.packed = (const __nv_bfloat16*)packed;
  a.wpart = wpart;
  a.wterms = mode == 0 ? wterms : nullptr;
  a.ldw_terms = ldw_terms;
  a.x = X;
  a.y = Y;
  a.alpha = alpha;
  a.alpha32 = nullptr;
  a.dots = dots;
  a.err = err;
  a.items = items;
  a.probs = probs;
  a.done = done;
  dim3 g((unsigned)(grid > 0 && grid < nitems ? grid : nitems), 1);
  cudaError_t e;
  switch ((mode << 2) | NT) {
    case 1: e = launch_tc<0, 1>(g, smem, mA, mB, a, st); break;
    case 2: e = launch_tc<0, 2>(g, smem, mA, mB, a, st); break;
    case 3: e = launch_tc<0, 3>(g, smem, mA, mB, a, st); break;
    case 5: e = launch_tc<1, 1>(g, smem, mA, mB, a, st); break;
    case 6: e = launch_tc<1, 2>(g, smem, mA, mB, a, st); break;
    default: e = launch_tc<1, 3>(g, smem, mA, mB, a, st); break;
  }
  return e == cudaSuccess ? 0 : 2;
}

int dense_tc_apply(const DenseDesc& op, int NT, const float* X, int64_t ld, int nc, float* Y,
                   double beta, const double* alpha, double* dots, int* nparts, char* ws,
                   int* err, unsigned flags, cudaStream_t st, const float* alpha32,
                   const int* gate) {
  switch (NT) {
    case 1: return dense_tc_apply_t<1>(op, X, ld, nc, Y, beta, alpha, dots, nparts, ws, err, flags, st,
                                           alpha32, gate);
    case 2: return dense_tc_apply_t<2>(op, X, ld, nc, Y, beta, alpha, dots, nparts, ws, err, flags, st,
                                           alpha32, gate);
    default: return dense_tc_apply_t<3>(op, X, ld, nc, Y, beta, alpha, dots, nparts, ws, err, flags, st,
                                           alpha32, gate);
  }
}

}  // namespace cofem
