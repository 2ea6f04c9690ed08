// Dense dictionary operator on the 5th-generation tensor cores (tcgen05):
//   A X = beta Phi^T (Phi X) + alpha . X        (Eq. (mat-eq))
// for a BF16 dictionary and FP32 right-hand sides.
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
#include <cuda.h>
#include <cudaTypedefs.h>

#include "dense.cuh"
#include "tc_ptx.cuh"

namespace cofem {

constexpr int kTcThreads = 192;     // warp 0 TMA, warp 1 MMA/TMEM, warps 2-5 epilogue
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
  int BN;               // MMA N (rows of the B operand)
  int stages;           // depth of the shared-memory ring (<= kMaxStages)
  uint32_t tmem_cols;
  int64_t res_d;        // Phi columns d < res_d are loaded evict-last (kept in L2)
  const __nv_bfloat16* packed;   // pre-swizzled tile-major copy of Phi, or null
  int64_t nkd;          // 64-column tiles of Phi (packed layout)
  // GEMM1: split-K partials (reduced and split by reduce_split_kernel)
  float* wpart;
  int64_t ldw;
  int64_t split_stride;

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

template <int MODE, int NT>
__global__ void __launch_bounds__(kTcThreads, 1)
dense_tc_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                const TcArgs args) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t b_bytes = (uint32_t)args.BN * 128u;
  const uint32_t stage_bytes = kATileBytes + b_bytes;
  const int S = args.stages;
  uint64_t* full = (uint64_t*)(smem + S * stage_bytes);
  uint64_t* empty = full + kMaxStages;
  uint64_t* accbar = empty + kMaxStages;
  uint32_t* tmem_slot = (uint32_t*)(accbar + 1);
  volatile int* abort = (volatile int*)(tmem_slot + 1);
  // epilogue partial dots per warp and column: compensated FP32 pairs, and
  // FP64 side sums of out-of-range products (flagged in *bigflag)
  float2* redp = (float2*)(tmem_slot + 4);          // [4][64]
  double* redb = (double*)(redp + 4 * 64);           // [4][64]
  volatile int* bigflag = (volatile int*)(tmem_slot + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // geometry of this CTA's work (one problem, or one item of a batch)
  int64_t m0, M = args.M, nkd = args.nkd, ldo = MODE == 0 ? args.ldw : args.ld;
  int64_t xoff = 0, aoff = 0, woff = 0, sstride = args.split_stride, bx0 = 0;
  double beta = args.beta;
  int kb0, kb1, split, dslot;
  const __nv_bfloat16* pk = args.packed;
  if (args.items) {
    const TcItem it = args.items[blockIdx.x];
    if (args.done && args.done[it.prob]) return;        // converged: nothing to do
    const TcProb pr = args.probs[it.prob];
    m0 = (int64_t)it.tile * kTileM;
    kb0 = it.kb0;
    kb1 = it.kb1;
    split = it.split;
    M = MODE == 0 ? pr.N : pr.D;
    nkd = pr.nkd;
    pk += pr.poff;
    ldo = MODE == 0 ? pr.ldw : pr.ld;
    xoff = pr.xoff;
    aoff = pr.aoff;
    woff = pr.wpoff;
    sstride = (int64_t)args.nc * pr.ldw;
    bx0 = MODE == 0 ? pr.boff1 : pr.boff2;
    dslot = pr.dots_base + it.tile;
    beta = pr.beta;
  } else {
    m0 = (int64_t)blockIdx.x * kTileM;
    kb0 = blockIdx.y * args.kb_per_split;
    kb1 = min(args.nk_total, kb0 + args.kb_per_split);
    split = blockIdx.y;
    dslot = blockIdx.x;
  }
  const int nk = max(0, kb1 - kb0);

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    tc::mbar_init(accbar, 1);
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
      int issued = 0;
      for (int i = 0; i < nk; ++i) {
        const int s = i % S;
        const uint32_t ph = (uint32_t)(i / S) & 1u;
        if (!tc::mbar_wait(&empty[s], ph ^ 1u, abort, kWaitLimitNs)) {
          tc_fail(args.err, abort);
          break;
        }
        uint8_t* sa = smem + s * stage_bytes;
        uint8_t* sb = sa + kATileBytes;
        tc::mbar_arrive_expect_tx(&full[s], stage_bytes);
        const int kb = kb0 + i;
        // Phi columns below res_d stay in L2 between the two products and
        // across CG iterations; the rest streams through
        if (MODE == 0) {
          const uint64_t pol_a = (int64_t)kb * kTileK < args.res_d ? pol_last : pol_first;
          if (pk)   // tile (m0 / 128, kb): one contiguous 16 KB copy
            tc::bulk_load(sa, pk + ((m0 >> 7) * nkd + kb) * (kTileM * kTileK), kATileBytes,
                          &full[s], pol_a);
          else
            tc::tma_load_2d(sa, &mapA, &full[s], kb * kTileK, (int)m0, pol_a);
        } else {
          const uint64_t pol_a = m0 < args.res_d ? pol_last : pol_first;
          if (pk) {
            // rows n = 64 kb .. +64 are half (kb & 1) of row tile kb / 2; the
            // two 64-column tiles m0/64 and m0/64 + 1 give the 128 d's
            const int64_t base = ((int64_t)(kb >> 1) * nkd + (m0 >> 6)) * kTileM + (kb & 1) * 64;
            const __nv_bfloat16* src = pk + base * kTileK;
            tc::bulk_load(sa, src, kATileBytes / 2, &full[s], pol_a);
            // the next 64-column tile; past the last one (D not a multiple of
            // 128) the same half-tile is copied again: it only feeds output
            // rows d >= D, which are not stored
            const __nv_bfloat16* src2 = (m0 >> 6) + 1 < nkd ? src + kTileM * kTileK : src;
            tc::bulk_load(sa + kATileBytes / 2, src2, kATileBytes / 2, &full[s], pol_a);
          } else {
            tc::tma_load_2d(sa, &mapA, &full[s], (int)m0, kb * kTileK, pol_a);
            tc::tma_load_2d(sa + kATileBytes / 2, &mapA, &full[s], (int)m0 + 64, kb * kTileK, pol_a);
          }
        }
        tc::tma_load_2d(sb, &mapB, &full[s], (int)(bx0 + (int64_t)kb * kTileK), 0, pol_b);
        ++issued;
      }
      if (*abort) {
        // drain this CTA's copies still in flight before leaving
        volatile int never = 0;
        for (int i = max(0, issued - S); i < issued; ++i)
          tc::mbar_wait(&full[i % S], (uint32_t)(i / S) & 1u, &never, kWaitLimitNs);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // A is K-major in the first product, MN-major (Phi^T read in place) in the second
      const uint32_t idesc = tc::idesc_bf16_f32(kTileM, args.BN, MODE == 1 ? 1 : 0, 0);
      for (int i = 0; i < nk; ++i) {
        const int s = i % S;
        const uint32_t ph = (uint32_t)(i / S) & 1u;
        if (!tc::mbar_wait(&full[s], ph, abort, kWaitLimitNs)) {
          tc_fail(args.err, abort);
          break;
        }
        tc::tc_fence_after();
        const uint32_t a_base = tc::smem_u32(smem + s * stage_bytes);
        const uint32_t b_base = a_base + kATileBytes;
#pragma unroll
        for (int k = 0; k < kTileK / 16; ++k) {
          uint64_t adesc;
          if (MODE == 0) adesc = tc::smem_desc_sw128(a_base + k * 32, 16, 1024);
          else adesc = tc::smem_desc_sw128(a_base + k * 2048, kATileBytes / 2, 1024);
          const uint64_t bdesc = tc::smem_desc_sw128(b_base + k * 32, 16, 1024);
          tc::mma_bf16(tmem, adesc, bdesc, idesc, (i > 0 || k > 0) ? 1u : 0u);
        }
        tc::mma_commit(&empty[s]);
      }
      tc::mma_commit(accbar);
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int g = warp & 3;                 // tensor-memory lane quarter of this warp
    const int64_t row = m0 + 32 * g + lane;
    constexpr int G = TermGroup<NT>::G, COLS = TermGroup<NT>::COLS;
    constexpr int MG = (kMaxCols + G - 1) / G;      // most column groups
    const int ngroups = (args.nc + G - 1) / G;
    const bool live = row < M;
    float a32 = 0.f;                     // alpha_row in FP32, converted once per row
    if (MODE == 1 && live)
      a32 = args.alpha32 ? args.alpha32[aoff + row]
                         : (args.alpha ? (float)args.alpha[aoff + row] : 0.f);
    const bool ok = tc::mbar_wait(accbar, 0, abort, 4 * kWaitLimitNs);
    if (!ok) tc_fail(args.err, abort);
    tc::tc_fence_after();
#pragma unroll
    for (int gi = 0; gi < MG; ++gi) {
      if (gi >= ngroups) break;
      float v[COLS];
#pragma unroll
      for (int c = 0; c < COLS / 16; ++c) {
        float t16[16];
        tc::tmem_ld16(tmem + ((uint32_t)(32 * g) << 16) + (uint32_t)(gi * COLS + 16 * c), t16);
#pragma unroll
        for (int q = 0; q < 16; ++q) v[16 * c + q] = t16[q];
      }
      tc::tmem_ld_wait();
      if (nk == 0 || !ok) {
#pragma unroll
        for (int q = 0; q < COLS; ++q) v[q] = 0.f;
      }
      // x_j^T y_j over the warp's 32 rows (second product): compensated
      // FP32 (product error by FMA, TwoSum butterflies, the G columns of the
      // group interleaved), FP64 once per warp and column; products of 1e30
      // or more take an FP64 side sum
      float ds[G], dc[G];
      double db[G];
      bool anybig = false;
#pragma unroll
      for (int jj = 0; jj < G; ++jj) {
        const int j = gi * G + jj;
        float acc = 0.f;
#pragma unroll
        for (int t = NT - 1; t >= 0; --t) acc += v[jj * NT + t];
        ds[jj] = 0.f;
        dc[jj] = 0.f;
        db[jj] = 0.0;
        if (MODE == 0) {
          if (j < args.nc && live)
            args.wpart[woff + (int64_t)split * sstride + (int64_t)j * ldo + row] = acc;
        } else if (j < args.nc && live) {
          const float xv = args.x[xoff + (int64_t)j * ldo + row];
          const float yv = fmaf(a32, xv, (float)beta * acc);
          args.y[xoff + (int64_t)j * ldo + row] = yv;
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
    if (MODE == 1 && args.dots) {
      asm volatile("bar.sync 1, 128;" ::: "memory");
      if (warp == 2) {
        const bool big = *bigflag != 0;
        for (int j = lane; j < args.nc; j += 32) {
          float ps = redp[j].x, pc = redp[j].y;
#pragma unroll
          for (int w = 1; w < 4; ++w) two_sum_merge(ps, pc, redp[w * 64 + j].x, redp[w * 64 + j].y);
          double t = (double)ps + (double)pc;
          if (big) t += redb[j] + redb[64 + j] + redb[128 + j] + redb[192 + j];
          args.dots[(int64_t)dslot * kMaxCols + j] = t;
        }
      }
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
                                   int64_t lds, int nc, __nv_bfloat16* __restrict__ Xs) {
  pdl_wait();
  pdl_trigger();
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
                                    __nv_bfloat16* __restrict__ Ws) {
  pdl_wait();
  pdl_trigger();
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
                          int stages) {
  DenseTcPlan p;
  if (ctas_per_sm < 1 || ctas_per_sm > 4) ctas_per_sm = 2;
  p.NT = NT;
  p.nc = nc;
  const int ngroups = (nc + term_group(NT) - 1) / term_group(NT);
  p.BN = ngroups * 16;
  uint32_t tc = 32;
  while (tc < (uint32_t)p.BN) tc <<= 1;
  p.tmem_cols = tc;
  p.ld = round_up(D, kLdAlign);
  p.ldw = round_up(N, kLdAlign);
  const int mt1 = (int)((N + kTileM - 1) / kTileM);
  p.nk1 = (int)((D + kTileK - 1) / kTileK);
  p.nk2 = (int)((N + kTileK - 1) / kTileK);
  int per_sm = 512 / (int)p.tmem_cols < ctas_per_sm ? 512 / (int)p.tmem_cols : ctas_per_sm;
  if (per_sm < 1) per_sm = 1;
  // one wave: at most per_sm * sms CTAs in the split-K product
  int want = (per_sm * sms) / mt1;
  if (want < 1) want = 1;
  if (want > p.nk1) want = p.nk1;
  p.kbps1 = (p.nk1 + want - 1) / want;
  p.S1 = (p.nk1 + p.kbps1 - 1) / p.kbps1;
  const size_t fixed = 1024 + 2 * kMaxStages * 8 + 64 + 4 * 64 * 8 * 2 + 64;
  const size_t stage = kATileBytes + (size_t)p.BN * 128;
  // each resident CTA also costs 1 KB of reserved shared memory
  const size_t budget = kSmemPerSm / per_sm - 1024;
  int st = (int)((budget - fixed) / stage);
  if (st > kMaxStages) st = kMaxStages;
  if (stages > 0 && stages < st) st = stages;
  if (st < 2) st = 2;
  p.stages = st;
  p.smem = st * stage + fixed;
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
  auto k = dense_tc_kernel<MODE, NT>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  launch_k(k, dim3(grid), dim3(kTcThreads), smem, st, a, b, args);
  return cudaGetLastError();
}

template <int NT>
static int dense_tc_apply_t(const DenseDesc& op, const float* X, int64_t ld, int nc, float* Y,
                            double beta, const double* alpha, double* dots, int* nparts,
                            char* ws, int* err, unsigned flags, cudaStream_t st,
                            const float* alpha32) {
  const int sms = num_sms();
  DenseTcPlan p = dense_tc_plan(op.N, op.D, nc, NT, sms, op.tc_ctas_per_sm, op.tc_stages);
  const bool presplit = (flags & kApplyPresplit) != 0;
  __nv_bfloat16* Xs = (__nv_bfloat16*)(ws + p.off_xs);
  float* Wp = (float*)(ws + p.off_wpart);
  __nv_bfloat16* Ws = (__nv_bfloat16*)(ws + p.off_ws);
  // split X (leading dim ld) into BF16 terms Xs (pitch p.ld): GEMM1's operand
  // (skipped when the caller's kernels already wrote Xs)
  if (!presplit) {
    const int64_t need4 = (p.ld / 4 + 255) / 256;
    dim3 g((unsigned)(need4 < 64 ? need4 : 64), (p.BN / 16) * TermGroup<NT>::G);
    launch_k(split_block_kernel<NT>, dim3(g), dim3(256), 0, st, X, ld, op.D, p.ld, nc, Xs);
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
  a1.nkd = nkd;
  a1.wpart = Wp;
  a1.ldw = p.ldw;
  a1.split_stride = (int64_t)nc * p.ldw;
  a1.err = err;
  dim3 g1((unsigned)((op.N + kTileM - 1) / kTileM), p.S1);
  if (launch_tc<0, NT>(g1, p.smem, mPhi1, mXs, a1, st) != cudaSuccess) return 2;
  apply_tick(st);
  {
    const int64_t need4 = (p.ldw / 4 + 127) / 128;
    dim3 g((unsigned)(need4 < 64 ? need4 : 64), (p.BN / 16) * TermGroup<NT>::G);
    launch_k(reduce_split_kernel<NT>, dim3(g), dim3(128), 0, st, Wp, p.S1, a1.split_stride, op.N, p.ldw, nc, Ws);
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
  a2.nkd = nkd;
  a2.y = Y;
  a2.x = X;
  a2.ld = ld;
  a2.alpha = alpha;
  a2.alpha32 = alpha32;
  a2.beta = beta;
  a2.dots = dots;
  a2.err = err;
  dim3 g2((unsigned)((op.D + kTileM - 1) / kTileM), 1);
  if (launch_tc<1, NT>(g2, p.smem, mPhi2, mWs, a2, st) != cudaSuccess) return 2;
  apply_tick(st);
  if (nparts) *nparts = dots ? (int)g2.x : 0;
  return 0;
}

int dense_tc_batched(int mode, int NT, int nitems, const TcItem* items, const TcProb* probs,
                     const int* done, const void* packed, const __nv_bfloat16* bsrc,
                     int64_t b_cols, int BN, int nc, int stages, uint32_t tmem_cols,
                     size_t smem, float* wpart, const float* X, float* Y, const double* alpha,
                     double* dots, int* err, cudaStream_t st) {
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
  a.packed = (const __nv_bfloat16*)packed;
  a.wpart = wpart;
  a.x = X;
  a.y = Y;
  a.alpha = alpha;
  a.alpha32 = nullptr;
  a.dots = dots;
  a.err = err;
  a.items = items;
  a.probs = probs;
  a.done = done;
  dim3 g((unsigned)nitems, 1);
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
                   int* err, unsigned flags, cudaStream_t st, const float* alpha32) {
  switch (NT) {
    case 1: return dense_tc_apply_t<1>(op, X, ld, nc, Y, beta, alpha, dots, nparts, ws, err, flags, st,
                                           alpha32);
    case 2: return dense_tc_apply_t<2>(op, X, ld, nc, Y, beta, alpha, dots, nparts, ws, err, flags, st,
                                           alpha32);
    default: return dense_tc_apply_t<3>(op, X, ld, nc, Y, beta, alpha, dots, nparts, ws, err, flags, st,
                                           alpha32);
  }
}

}  // namespace cofem
