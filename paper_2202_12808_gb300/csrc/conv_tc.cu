// Circular convolutional dictionary on the 5th-generation tensor cores
// (tcgen05), BF16 filters and FP32 vectors.  Both products of the E-step
// operator A X = beta Phi^T Phi X + alpha . X (Eq. (mat-eq)) with the
// convolutional Phi of Sec. 3.2 are written as GEMMs over blocks of 128
// outputs.  With a tile of 64 blocks (8192 outputs) starting at P0 and
// P_b = P0 + 128 b (all indices mod L):
//
//   forward  (Phi z)[P_b + i]     = sum_c sum_{s<192} F_c[i][s] z_c[P_b - 64 + s],
//            F_c[i][s] = h[c][i + 64 - s]      (zero unless 0 <= i + 64 - s < T)
//   adjoint  (Phi^T w)_c[P_b + i] = sum_{s<192} G_c[i][s] w[P_b + s],
//            G_c[i][s] = h[c][s - i]           (zero unless 0 <= s - i < T)
//
// The Toeplitz matrices F_c, G_c are the A operand (M = 128 outputs of a
// block; K = the 192 window offsets, three 64-wide atoms in the 128-byte-
// swizzled K-major layout), built once per fit (or per stand-alone
// application) in global memory as the images the MMA reads and streamed by
// bulk copies.  The data windows are the B operand: 64 blocks for each BF16
// term of the data, x = x1 + x2 + x3 with x1 = x truncated to BF16, x2 =
// (x - x1) truncated, x3 = x - x1 - x2 (each subtraction exact; x3 has at
// most 8 significant bits, so the three terms hold x exactly and the
// products are exact in the FP32 accumulator).  The terms are stacked along
// N (row 64 t + b of a 192-row B operand), so one MMA per K step reads the
// filter tile once for all three (shared-memory operand traffic, not the
// tensor pipe, bounds a 128 x 64 MMA) and the epilogue adds columns b,
// 64 + b and 128 + b.  All windows of a tile lie in one run of 8256 samples
// (the tile plus 64 on the left for the forward product, on the right for
// the adjoint): a bulk copy stages that run raw (FP32) in shared memory and
// producer warps (eight in the forward, four in the adjoint) split it into
// the B tiles.  One thread issues the MMAs into 128 x 192 FP32 accumulators
// in tensor memory, lane = output i of a block, column = (term, block)
// (forward: one per tile, double-buffered; adjoint: one per channel, two
// slots), so the epilogue warps' loads and stores of 32 consecutive outputs
// are single 128-byte lines.  The adjoint's epilogue applies beta, adds
// alpha . x and accumulates the x_j^T y_j partial of the tile.
//
// Compared with the direct form (2 T C L flops per column), the block
// Toeplitz form does 192 / T times the multiply-adds (3x at T = 64) on three
// data terms, on units more than 20x faster than the FP32 CUDA cores, so the
// tensor pipe is not what bounds them: the forward (C L floats read and L
// written per column) is bound by shared-memory traffic, the producers'
// rewrite of the windows into term tiles and the MMA's operand reads; the
// adjoint (L + 2 C L read: w, x, alpha; C L written) by its epilogue's loads
// of x and alpha.
//
// Every wait is bounded: a timeout sets COFEM_ERR_TIMEOUT in the error word
// and the CTA drains its copies, frees its tensor memory and exits.
#include "kernels.cuh"
#include "tc_ptx.cuh"

namespace cofem {
void apply_tick(cudaStream_t st);

namespace {

constexpr int kCtM = 128;                           // outputs per block (MMA M)
constexpr int kCtN = 64;                            // blocks per tile (MMA N)
constexpr int kCtTile = kCtM * kCtN;                // 8192 outputs per tile
constexpr int kCtWin = kCtTile + 64;                // staged samples per tile
constexpr int kCtAtoms = 3;                         // K = 192 window offsets
constexpr uint32_t kCtRawBytes = 33 * 1024;         // >= kCtWin * 4, 1024-aligned
constexpr uint32_t kCtATile = kCtM * 128;           // 16 KB: 128 rows x 64 BF16
constexpr uint32_t kCtBTile = kCtN * 128;           // 8 KB: 64 rows x 64 BF16
constexpr int kCtTerms = 3;
constexpr int kCtAccCols = kCtTerms * kCtN;         // 192 accumulator columns
constexpr int kCtSlots = 2;                         // adjoint: channel accumulators
constexpr uint64_t kCtWaitNs = 1000000000ull;
constexpr int kCtProdWarps = 8;                     // forward producers

// forward: warp 0 raw loader, 1 MMA, 2-5 epilogue, 6-13 producers, 14 filter loader
constexpr int kFwdProd = 6, kFwdFilt = 14;
constexpr int kCtFwdThreads = 15 * 32;
constexpr int kFwdStages = 3;                       // (channel, atom) stages
constexpr uint32_t kFwdStageBytes = kCtATile + kCtTerms * kCtBTile;   // 40 KB
constexpr uint32_t kFwdRaw = 0;
constexpr uint32_t kFwdStage = kFwdRaw + 2 * kCtRawBytes;
constexpr uint32_t kFwdBar = kFwdStage + kFwdStages * kFwdStageBytes;
constexpr size_t kFwdSmem = kFwdBar + 256 + 1024;

// adjoint: warp 0 raw loader, 1 MMA, 2-17 epilogue, 18-21 producers, 22 filter loader
constexpr int kAdjEpiWarps = 16;
constexpr int kAdjProdWarps = 4;
constexpr int kAdjEpi = 2, kAdjProd = 18, kAdjFilt = 22;
constexpr int kCtAdjThreads = 23 * 32;
constexpr int kAdjRing = 4;                          // filter tiles in flight
constexpr uint32_t kAdjRaw = 0;
constexpr uint32_t kAdjData = kAdjRaw + kCtRawBytes;                 // [atom][term] B tiles
constexpr uint32_t kAdjFiltTiles = kAdjData + kCtAtoms * kCtTerms * kCtBTile;
constexpr uint32_t kAdjBar = kAdjFiltTiles + kAdjRing * kCtATile;
constexpr size_t kAdjSmem = kAdjBar + 512 + 1024;
static_assert(kFwdSmem <= 227 * 1024 && kAdjSmem <= 227 * 1024, "shared memory");
static_assert(kCtWin * 4 <= (int)kCtRawBytes, "raw stage");

__device__ __forceinline__ void ct_fail(int* err, volatile int* abort) {
  *abort = 1;
  if (err) atomicCAS(err, 0, (int)COFEM_ERR_TIMEOUT);
}

// The warps of one role take the same decision (named barrier `id` over
// `n` threads): true only if every thread passed `ok`.
__device__ __forceinline__ bool all_ok(bool ok, int id, int n) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
      "bar.red.and.pred q, %2, %3, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)ok), "r"(id), "r"(n)
      : "memory");
  return r != 0;
}

// The BF16 bits of the upper halves of two FP32 values, a in the low half.
__device__ __forceinline__ uint32_t upper_pair(float a, float b) {
  return __byte_perm(__float_as_uint(a), __float_as_uint(b), 0x7632);
}
__device__ __forceinline__ float trunc16(float x) {
  return __uint_as_float(__float_as_uint(x) & 0xFFFF0000u);
}

// Producer step: the three BF16 term tiles of one 64-wide K atom a from the
// raw window, B_t[b][k] = term t of raw[128 b + 64 a + k], b < 64.  Task =
// (row b, quarter q of its 64 values): one 16-byte shared load, three
// 8-byte stores at the swizzled position of chunk q/2 (half q & 1).
template <int NPROD>
__device__ __forceinline__ void build_atom(const float* raw, int a, uint8_t* b0, int ptid) {
#pragma unroll 2
  for (int task = ptid; task < kCtN * 16; task += NPROD) {
    const int row = task >> 4, q = task & 15;
    const float4 v = *reinterpret_cast<const float4*>(raw + 128 * row + 64 * a + 4 * q);
    const uint32_t off = (uint32_t)row * 128u + ((uint32_t)((q >> 1) ^ (row & 7)) << 4) +
                         ((uint32_t)(q & 1) << 3);
    const float h0 = trunc16(v.x), h1 = trunc16(v.y), h2 = trunc16(v.z), h3 = trunc16(v.w);
    const float r0 = v.x - h0, r1 = v.y - h1, r2 = v.z - h2, r3 = v.w - h3;
    const float m0 = trunc16(r0), m1 = trunc16(r1), m2 = trunc16(r2), m3 = trunc16(r3);
    const float l0 = r0 - m0, l1 = r1 - m1, l2 = r2 - m2, l3 = r3 - m3;
    *reinterpret_cast<uint2*>(b0 + off) = make_uint2(upper_pair(h0, h1), upper_pair(h2, h3));
    *reinterpret_cast<uint2*>(b0 + kCtBTile + off) =
        make_uint2(upper_pair(m0, m1), upper_pair(m2, m3));
    *reinterpret_cast<uint2*>(b0 + 2 * kCtBTile + off) =
        make_uint2(upper_pair(l0, l1), upper_pair(l2, l3));
  }
}

// Adjoint accumulator slot of channel c is c mod kCtSlots; its use number
// (for the barrier parity) after `lu` earlier tiles of this CTA, each using
// the slot once per channel c' < C with c' = c mod kCtSlots
__device__ __forceinline__ int slot_use(int lu, int c, int C) {
  const int sl = c % kCtSlots;
  return lu * ((C - 1 - sl) / kCtSlots + 1) + c / kCtSlots;
}

__device__ __forceinline__ int64_t wrap(int64_t i, int64_t L) {
  i %= L;
  return i < 0 ? i + L : i;
}

struct CtArgs {
  int C;
  int64_t L;
  int ncols;
  int units;                      // ncols x tiles
  const float* x;                 // forward: Z (ldx); adjoint: W (ldx)
  int64_t ldx;
  float* y;                       // forward: W; adjoint: Y (ldy)
  int64_t ldy;
  const __nv_bfloat16* img;       // Toeplitz tiles, (c, atom) at (3 c + atom) x 8192 elements
  // adjoint epilogue
  double beta;
  const double* alpha;
  const float* alpha32;
  const float* xd;                // x for alpha . x and the dots (pitch ldy)
  double* dots;
  int* err;
};

// ------------------------------------------------------------- forward
__global__ void __launch_bounds__(kCtFwdThreads, 1) conv_tc_forward_kernel(CtArgs g) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* rfull = (uint64_t*)(smem + kFwdBar);   // [2] raw window landed
  uint64_t* rempty = rfull + 2;                    // [2] raw window read (producers)
  uint64_t* dfull = rempty + 2;                    // [stages] data terms written
  uint64_t* ffull = dfull + kFwdStages;            // [stages] filter tile landed
  uint64_t* sempty = ffull + kFwdStages;           // [stages] consumed (MMA)
  uint64_t* accfull = sempty + kFwdStages;         // [2]
  uint64_t* accempty = accfull + 2;                // [2]
  uint32_t* tmem_slot = (uint32_t*)(accempty + 2);
  volatile int* abort = (volatile int*)(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t L = g.L;
  if (threadIdx.x == 0) {
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(&rfull[i], 1);
      tc::mbar_init(&rempty[i], kCtProdWarps);
      tc::mbar_init(&accfull[i], 1);
      tc::mbar_init(&accempty[i], 4);
    }
    for (int i = 0; i < kFwdStages; ++i) {
      tc::mbar_init(&dfull[i], kCtProdWarps);
      tc::mbar_init(&ffull[i], 1);
      tc::mbar_init(&sempty[i], 1);
    }
    *abort = 0;
    tc::fence_mbar_init();
  }
  if (warp == 1) {
    tc::tmem_alloc(tmem_slot, 512);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------- raw loader
    if (lane == 0) {
      const uint64_t pol = tc::policy_evict_first();
      int rc = 0;
      bool ok = true;
      for (int u = blockIdx.x; ok && u < g.units && !*abort; u += gridDim.x) {
        const int q = u / g.ncols, j = u % g.ncols;
        const int64_t P0 = (int64_t)q * kCtTile;
        const int64_t len = L - P0 < kCtTile ? L - P0 : kCtTile;
        for (int c = 0; c < g.C; ++c, ++rc) {
          const int rs = rc & 1;
          if (!tc::mbar_wait(&rempty[rs], (uint32_t)((rc >> 1) & 1) ^ 1u, abort, 4 * kCtWaitNs)) {
            ok = false;
            break;
          }
          const float* xc = g.x + (int64_t)j * g.ldx + (int64_t)c * L;
          uint8_t* raw = smem + kFwdRaw + rs * kCtRawBytes;
          tc::mbar_arrive_expect_tx(&rfull[rs], 256u + (uint32_t)len * 4u);
          tc::bulk_load(raw, xc + wrap(P0 - 64, L), 256u, &rfull[rs], pol);
          tc::bulk_load(raw + 256, xc + P0, (uint32_t)len * 4u, &rfull[rs], pol);
        }
      }
      if (!ok) ct_fail(g.err, abort);
      if (*abort) {
        volatile int never = 0;
        for (int i = rc - 2 > 0 ? rc - 2 : 0; i < rc; ++i)
          tc::mbar_wait(&rfull[i & 1], (uint32_t)((i >> 1) & 1), &never, kCtWaitNs);
      }
    }
  } else if (warp == kFwdFilt) {
    // ---------------------------------------------------- filter loader
    if (lane == 0) {
      const uint64_t pol = tc::policy_evict_last();
      int sc = 0;
      bool ok = true;
      for (int u = blockIdx.x; ok && u < g.units && !*abort; u += gridDim.x) {
        for (int c = 0; ok && c < g.C; ++c)
          for (int a = 0; a < kCtAtoms; ++a, ++sc) {
            const int ss = sc % kFwdStages;
            if (!tc::mbar_wait(&sempty[ss], (uint32_t)((sc / kFwdStages) & 1) ^ 1u, abort,
                               4 * kCtWaitNs)) {
              ok = false;
              break;
            }
            tc::mbar_arrive_expect_tx(&ffull[ss], kCtATile);
            tc::bulk_load(smem + kFwdStage + ss * kFwdStageBytes,
                          g.img + (int64_t)(kCtAtoms * c + a) * (kCtM * 64), kCtATile, &ffull[ss],
                          pol);
          }
      }
      if (!ok) ct_fail(g.err, abort);
      if (*abort) {
        volatile int never = 0;
        for (int i = sc - kFwdStages > 0 ? sc - kFwdStages : 0; i < sc; ++i)
          tc::mbar_wait(&ffull[i % kFwdStages], (uint32_t)((i / kFwdStages) & 1), &never,
                        kCtWaitNs);
      }
    }
  } else if (warp == 1) {
    // --------------------------------------------------------------- MMA
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_bf16_f32(kCtM, kCtAccCols, 0, 0);
      int sc = 0, lu = 0;
      bool ok = true;
      for (int u = blockIdx.x; ok && u < g.units && !*abort; u += gridDim.x, ++lu) {
        const int b = lu & 1;
        if (!tc::mbar_wait(&accempty[b], (uint32_t)((lu >> 1) & 1) ^ 1u, abort, 4 * kCtWaitNs)) {
          ok = false;
          break;
        }
        tc::tc_fence_after();
        const uint32_t acc = tmem + (uint32_t)(b * 256);
        for (int c = 0; ok && c < g.C; ++c)
          for (int a = 0; a < kCtAtoms; ++a, ++sc) {
            const int ss = sc % kFwdStages;
            const uint32_t ph = (uint32_t)((sc / kFwdStages) & 1);
            if (!tc::mbar_wait(&ffull[ss], ph, abort, kCtWaitNs) ||
                !tc::mbar_wait(&dfull[ss], ph, abort, kCtWaitNs)) {
              ok = false;
              break;
            }
            tc::tc_fence_after();
            const uint32_t a0 = tc::smem_u32(smem + kFwdStage + ss * kFwdStageBytes);
            const uint32_t b0 = a0 + kCtATile;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const uint64_t ad = tc::smem_desc_sw128(a0 + k * 32, 16, 1024);
              const uint64_t bd = tc::smem_desc_sw128(b0 + k * 32, 16, 1024);
              tc::mma_bf16(acc, ad, bd, idesc, (c | a | k) != 0 ? 1u : 0u);
            }
            tc::mma_commit(&sempty[ss]);
          }
        if (!ok) break;
        tc::mma_commit(&accfull[b]);
      }
      if (!ok) ct_fail(g.err, abort);
    }
  } else if (warp < kFwdProd) {
    // ---------------------------------------------------------- epilogue
    const int gq = warp & 3;                 // tensor-memory lane quarter
    const int i = 32 * gq + lane;            // output within a block
    int lu = 0;
    for (int u = blockIdx.x; u < g.units; u += gridDim.x, ++lu) {
      const int q = u / g.ncols, j = u % g.ncols;
      const int b = lu & 1;
      const bool ok = tc::mbar_wait(&accfull[b], (uint32_t)((lu >> 1) & 1), abort, 4 * kCtWaitNs);
      if (!ok) ct_fail(g.err, abort);
      if (!all_ok(ok, 2, 128)) break;
      tc::tc_fence_after();
      // column 64 t + bb holds term t of block bb: the three are added
      float v[kCtN];
      const uint32_t tbase = tmem + ((uint32_t)(32 * gq) << 16) + (uint32_t)(b * 256);
#pragma unroll
      for (int ch = 0; ch < kCtN / 16; ++ch) {
        float t0[16], t1[16], t2[16];
        tc::tmem_ld16(tbase + (uint32_t)(16 * ch), t0);
        tc::tmem_ld16(tbase + (uint32_t)(kCtN + 16 * ch), t1);
        tc::tmem_ld16(tbase + (uint32_t)(2 * kCtN + 16 * ch), t2);
        tc::tmem_ld_wait();
#pragma unroll
        for (int e = 0; e < 16; ++e) v[16 * ch + e] = t0[e] + (t1[e] + t2[e]);
      }
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&accempty[b]);
      // column = block: the warp's 32 lanes store 32 consecutive outputs
      const int64_t p0 = (int64_t)q * kCtTile + i;
      float* yb = g.y + (int64_t)j * g.ldy + p0;
      const int64_t rem = L - p0;                 // blocks bb < nv hold outputs < L
      const int nv = rem <= 0 ? 0 : (int)((rem + kCtM - 1) / kCtM);
#pragma unroll
      for (int bb = 0; bb < kCtN; ++bb)
        if (bb < nv) yb[kCtM * bb] = v[bb];
    }
  } else {
    // ---------------------------------------------------------- producers
    const int ptid = threadIdx.x - kFwdProd * 32;
    int rc = 0, sc = 0;
    bool ok = true;
    for (int u = blockIdx.x; ok && u < g.units && !*abort; u += gridDim.x) {
      for (int c = 0; ok && c < g.C; ++c, ++rc) {
        const int rs = rc & 1;
        if (!tc::mbar_wait(&rfull[rs], (uint32_t)((rc >> 1) & 1), abort, 4 * kCtWaitNs)) {
          ok = false;
          break;
        }
        const float* raw = (const float*)(smem + kFwdRaw + rs * kCtRawBytes);
        for (int a = 0; a < kCtAtoms; ++a, ++sc) {
          const int ss = sc % kFwdStages;
          if (!tc::mbar_wait(&sempty[ss], (uint32_t)((sc / kFwdStages) & 1) ^ 1u, abort,
                             4 * kCtWaitNs)) {
            ok = false;
            break;
          }
          build_atom<kCtProdWarps * 32>(raw, a, smem + kFwdStage + ss * kFwdStageBytes + kCtATile,
                                        ptid);
          tc::fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) tc::mbar_arrive(&dfull[ss]);
        }
        if (!ok) break;
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&rempty[rs]);
      }
    }
    if (!ok) ct_fail(g.err, abort);
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, 512);
  }
}

// ------------------------------------------------------------- adjoint
__global__ void __launch_bounds__(kCtAdjThreads, 1) conv_tc_adjoint_kernel(CtArgs g) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* wfull = (uint64_t*)(smem + kAdjBar);   // raw w window landed
  uint64_t* wempty = wfull + 1;                    // raw window read (producers)
  uint64_t* dfull = wempty + 1;                    // data term tiles written
  uint64_t* dempty = dfull + 1;                    // data tiles consumed (MMA, whole tile)
  uint64_t* ffull = dempty + 1;                    // [ring] filter tiles landed
  uint64_t* fempty = ffull + kAdjRing;             // [ring]
  uint64_t* sfull = fempty + kAdjRing;             // [slots] channel accumulator ready
  uint64_t* sempty = sfull + kCtSlots;             // [slots] drained (epilogue)
  uint32_t* tmem_slot = (uint32_t*)(sempty + kCtSlots);
  volatile int* abort = (volatile int*)(tmem_slot + 1);
  float2* reds = (float2*)(tmem_slot + 4);         // [epilogue warps]
  double* redb = (double*)(reds + kAdjEpiWarps);   // [epilogue warps]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t L = g.L;
  if (threadIdx.x == 0) {
    tc::mbar_init(wfull, 1);
    tc::mbar_init(wempty, kAdjProdWarps);
    tc::mbar_init(dfull, kAdjProdWarps);
    tc::mbar_init(dempty, 1);
    for (int i = 0; i < kAdjRing; ++i) {
      tc::mbar_init(&ffull[i], 1);
      tc::mbar_init(&fempty[i], 1);
    }
    for (int i = 0; i < kCtSlots; ++i) {
      tc::mbar_init(&sfull[i], 1);
      tc::mbar_init(&sempty[i], kAdjEpiWarps);
    }
    *abort = 0;
    tc::fence_mbar_init();
  }
  if (warp == 1) {
    tc::tmem_alloc(tmem_slot, 512);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------- raw loader
    if (lane == 0) {
      const uint64_t pol = tc::policy_evict_first();
      int lu = 0;
      bool ok = true;
      for (int u = blockIdx.x; u < g.units && !*abort; u += gridDim.x, ++lu) {
        const int q = u / g.ncols, j = u % g.ncols;
        const int64_t P0 = (int64_t)q * kCtTile;
        const int64_t len = L - P0 < kCtTile ? L - P0 : kCtTile;
        if (!tc::mbar_wait(wempty, (uint32_t)(lu & 1) ^ 1u, abort, 4 * kCtWaitNs)) {
          ok = false;
          break;
        }
        const float* wj = g.x + (int64_t)j * g.ldx;
        tc::mbar_arrive_expect_tx(wfull, (uint32_t)len * 4u + 256u);
        tc::bulk_load(smem + kAdjRaw, wj + P0, (uint32_t)len * 4u, wfull, pol);
        tc::bulk_load(smem + kAdjRaw + (uint32_t)len * 4u, wj + wrap(P0 + len, L), 256u, wfull,
                      pol);
      }
      if (!ok) ct_fail(g.err, abort);
      if (*abort && lu > 0) {
        volatile int never = 0;
        tc::mbar_wait(wfull, (uint32_t)((lu - 1) & 1), &never, kCtWaitNs);
      }
    }
  } else if (warp == kAdjFilt) {
    // ---------------------------------------------------- filter loader
    if (lane == 0) {
      const uint64_t pol = tc::policy_evict_last();
      int fc = 0;
      bool ok = true;
      for (int u = blockIdx.x; ok && u < g.units && !*abort; u += gridDim.x)
        for (int c = 0; ok && c < g.C; ++c)
          for (int a = 0; a < kCtAtoms; ++a, ++fc) {
            const int fs = fc % kAdjRing;
            if (!tc::mbar_wait(&fempty[fs], (uint32_t)((fc / kAdjRing) & 1) ^ 1u, abort,
                               4 * kCtWaitNs)) {
              ok = false;
              break;
            }
            tc::mbar_arrive_expect_tx(&ffull[fs], kCtATile);
            tc::bulk_load(smem + kAdjFiltTiles + fs * kCtATile,
                          g.img + (int64_t)(kCtAtoms * c + a) * (kCtM * 64), kCtATile, &ffull[fs],
                          pol);
          }
      if (!ok) ct_fail(g.err, abort);
      if (*abort) {
        volatile int never = 0;
        for (int i = fc - kAdjRing > 0 ? fc - kAdjRing : 0; i < fc; ++i)
          tc::mbar_wait(&ffull[i % kAdjRing], (uint32_t)((i / kAdjRing) & 1), &never, kCtWaitNs);
      }
    }
  } else if (warp == 1) {
    // --------------------------------------------------------------- MMA
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_bf16_f32(kCtM, kCtAccCols, 0, 0);
      int lu = 0, fc = 0;
      bool ok = true;
      const uint32_t d0 = tc::smem_u32(smem + kAdjData);
      for (int u = blockIdx.x; ok && u < g.units && !*abort; u += gridDim.x, ++lu) {
        if (!tc::mbar_wait(dfull, (uint32_t)(lu & 1), abort, 4 * kCtWaitNs)) {
          ok = false;
          break;
        }
        tc::tc_fence_after();
        for (int c = 0; ok && c < g.C; ++c) {
          const int sl = c % kCtSlots;
          if (!tc::mbar_wait(&sempty[sl], (uint32_t)(slot_use(lu, c, g.C) & 1) ^ 1u, abort,
                             4 * kCtWaitNs)) {
            ok = false;
            break;
          }
          tc::tc_fence_after();
          const uint32_t acc = tmem + (uint32_t)(sl * 256);
          for (int a = 0; a < kCtAtoms; ++a, ++fc) {
            const int fs = fc % kAdjRing;
            if (!tc::mbar_wait(&ffull[fs], (uint32_t)((fc / kAdjRing) & 1), abort, kCtWaitNs)) {
              ok = false;
              break;
            }
            tc::tc_fence_after();
            const uint32_t a0 = tc::smem_u32(smem + kAdjFiltTiles + fs * kCtATile);
            // the 192-row B operand of atom a: its three term tiles, contiguous
            const uint32_t b0 = d0 + (uint32_t)(a * kCtTerms) * kCtBTile;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const uint64_t ad = tc::smem_desc_sw128(a0 + k * 32, 16, 1024);
              const uint64_t bd = tc::smem_desc_sw128(b0 + k * 32, 16, 1024);
              tc::mma_bf16(acc, ad, bd, idesc, (a | k) != 0 ? 1u : 0u);
            }
            tc::mma_commit(&fempty[fs]);
          }
          if (!ok) break;
          tc::mma_commit(&sfull[sl]);
        }
        if (!ok) break;
        tc::mma_commit(dempty);
      }
      if (!ok) ct_fail(g.err, abort);
    }
  } else if (warp < kAdjProd) {
    // ---------------------------------------------------------- epilogue
    // warps 2..17: lane quarter warp & 3 (outputs i of a block), blocks
    // 16 hh .. 16 hh + 15 (hh = (warp - 2) / 4)
    const int gq = warp & 3, hh = (warp - kAdjEpi) >> 2, ew = warp - kAdjEpi;
    const int i = 32 * gq + lane;
    const float beta = (float)g.beta;
    const bool diag = g.alpha32 != nullptr || g.alpha != nullptr;
    int lu = 0;
    for (int u = blockIdx.x; u < g.units; u += gridDim.x, ++lu) {
      const int q = u / g.ncols, j = u % g.ncols;
      // this thread's outputs p0 + 128 bb, bb < 16 (block 16 hh + bb); those
      // with bb < nv lie below L
      const int64_t p0 = (int64_t)q * kCtTile + (int64_t)kCtM * 16 * hh + i;
      const int64_t rem = L - p0;
      const int nv = rem <= 0 ? 0 : (rem >= 16 * kCtM ? 16 : (int)((rem + kCtM - 1) / kCtM));
      AccF dot;
      float sbig = 0.f;
      bool failed = false;
      for (int c = 0; c < g.C; ++c) {
        const int sl = c % kCtSlots;
        // x and alpha of this channel's 16 outputs, loaded before the wait
        const float* xb = g.xd + (int64_t)j * g.ldy + (int64_t)c * L + p0;
        float xr[16], ar[16];
        if (diag) {
          if (g.alpha32) {
            const float* ab = g.alpha32 + (int64_t)c * L + p0;
#pragma unroll
            for (int bb = 0; bb < 16; ++bb) {
              xr[bb] = bb < nv ? xb[kCtM * bb] : 0.f;
              ar[bb] = bb < nv ? ab[kCtM * bb] : 0.f;
            }
          } else {
            const double* ab = g.alpha + (int64_t)c * L + p0;
#pragma unroll
            for (int bb = 0; bb < 16; ++bb) {
              xr[bb] = bb < nv ? xb[kCtM * bb] : 0.f;
              ar[bb] = bb < nv ? (float)ab[kCtM * bb] : 0.f;
            }
          }
        }
        if (!failed &&
            !tc::mbar_wait(&sfull[sl], (uint32_t)(slot_use(lu, c, g.C) & 1), abort, 4 * kCtWaitNs)) {
          ct_fail(g.err, abort);
          failed = true;
        }
        if (failed) continue;
        tc::tc_fence_after();
        // column 64 t + b of the slot holds term t of block b
        const uint32_t tb = tmem + ((uint32_t)(32 * gq) << 16) + (uint32_t)(sl * 256 + 16 * hh);
        // terms 2 and 1 first (the small ones), then term 0: 32 registers
        float ts[16], tt[16];
        tc::tmem_ld16(tb + kCtN, ts);
        tc::tmem_ld16(tb + 2 * kCtN, tt);
        tc::tmem_ld_wait();
#pragma unroll
        for (int e = 0; e < 16; ++e) ts[e] += tt[e];
        tc::tmem_ld16(tb, tt);
        tc::tmem_ld_wait();
        tc::tc_fence_before();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&sempty[sl]);
        float* yb = g.y + (int64_t)j * g.ldy + (int64_t)c * L + p0;
        // x_j^T y_j: compensated FP32 (product error by FMA, TwoSum); a
        // product of 1e30 or more goes, scaled by 2^-64, to a plain FP32 side
        // sum instead (no FP64 per element: it runs at 1/64 of FP32 here)
#pragma unroll
        for (int bb = 0; bb < 16; ++bb) {
          if (bb < nv) {
            const float acc = tt[bb] + ts[bb];
            float o;
            if (diag) {
              o = fmaf(ar[bb], xr[bb], beta * acc);
              const float pp = xr[bb] * o;
              const bool fin = fabsf(pp) < 1e30f;
              sbig += fin ? 0.f : (xr[bb] * 0x1p-64f) * o;
              dot.c += fin ? fmaf(xr[bb], o, -pp) : 0.f;
              const float x = fin ? pp : 0.f;
              const float t = dot.s + x, xv = t - dot.s;
              dot.c += (dot.s - (t - xv)) + (x - xv);
              dot.s = t;
            } else {
              o = beta * acc;
            }
            yb[kCtM * bb] = o;
          }
        }
      }
      dot.big = (double)sbig * 0x1p64;
      // the epilogue warps agree once per tile (a failed wait ends them all)
      if (!all_ok(!failed, 2, 32 * kAdjEpiWarps)) break;
      if (g.dots) {
        // x_j^T y_j over the tile: compensated FP32 within each warp, the
        // warps merged in a fixed order, FP64 side sums of huge products
        float s = dot.s, cpart = dot.c;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
          two_sum_merge(s, cpart, __shfl_xor_sync(0xffffffffu, s, o),
                        __shfl_xor_sync(0xffffffffu, cpart, o));
        const double big = warp_sum(dot.big);
        if (lane == 0) {
          reds[ew] = make_float2(s, cpart);
          redb[ew] = big;
        }
        asm volatile("bar.sync 1, %0;" ::"r"(32 * kAdjEpiWarps) : "memory");
        if (ew == 0 && lane == 0) {
          float ps = reds[0].x, pc = reds[0].y;
          double pb2 = redb[0];
          for (int w = 1; w < kAdjEpiWarps; ++w) {
            two_sum_merge(ps, pc, reds[w].x, reds[w].y);
            pb2 += redb[w];
          }
          g.dots[(int64_t)q * kMaxCols + j] = (double)ps + (double)pc + pb2;
        }
        asm volatile("bar.sync 1, %0;" ::"r"(32 * kAdjEpiWarps) : "memory");
      }
    }
  } else if (warp < kAdjFilt) {
    // ---------------------------------------------------------- producers
    const int ptid = threadIdx.x - kAdjProd * 32;
    int lu = 0;
    for (int u = blockIdx.x; u < g.units && !*abort; u += gridDim.x, ++lu) {
      if (!tc::mbar_wait(wfull, (uint32_t)(lu & 1), abort, 4 * kCtWaitNs) ||
          !tc::mbar_wait(dempty, (uint32_t)(lu & 1) ^ 1u, abort, 4 * kCtWaitNs)) {
        ct_fail(g.err, abort);
        break;
      }
      const float* raw = (const float*)(smem + kAdjRaw);
      for (int a = 0; a < kCtAtoms; ++a)
        build_atom<kAdjProdWarps * 32>(raw, a, smem + kAdjData + (uint32_t)(a * kCtTerms) * kCtBTile,
                                       ptid);
      tc::fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) {
        tc::mbar_arrive(dfull);
        tc::mbar_arrive(wempty);
      }
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, 512);
  }
}

// Rounded filters and Toeplitz images: h64[c][t] = bf16(h[c][t]) (zero for
// t >= T); image 0 (forward) tile (c, a) row i holds F_c[i][64 a + k], image
// 1 (adjoint) G_c[i][64 a + k], k < 64, i < 128, as the 128-byte-swizzled
// shared-memory image (row i at i * 64 values, 16-byte chunk q at position
// q ^ (i mod 8)).  One thread per tap or per 16-byte chunk.
__global__ void conv_tc_prep_kernel(const float* __restrict__ h, int C, int T,
                                    float* __restrict__ h64, __nv_bfloat16* __restrict__ img) {
  pdl_wait();
  pdl_trigger();
  const int ntap = C * 64;
  const int per_img = C * kCtAtoms * kCtM * 8;   // chunks of one image
  for (int task = blockIdx.x * blockDim.x + threadIdx.x; task < ntap + 2 * per_img;
       task += gridDim.x * blockDim.x) {
    if (task < ntap) {
      const int c = task >> 6, t = task & 63;
      h64[task] = t < T ? __bfloat162float(__float2bfloat16_rn(h[c * T + t])) : 0.f;
      continue;
    }
    const int e = task - ntap;
    const int im = e / per_img, r = e % per_img;
    const int pos = r & 7, row = (r >> 3) & (kCtM - 1);
    const int tile = r >> 10;                     // 3 c + a
    const int c = tile / kCtAtoms, a = tile % kCtAtoms;
    const int qsrc = pos ^ (row & 7);
    uint32_t w[4];
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) {
      float f[2];
#pragma unroll
      for (int h2 = 0; h2 < 2; ++h2) {
        const int s = 64 * a + 8 * qsrc + 2 * k2 + h2;
        const int tap = im == 0 ? row + 64 - s : s - row;
        f[h2] = (tap >= 0 && tap < T) ? h[c * T + tap] : 0.f;
      }
      const __nv_bfloat16 b0 = __float2bfloat16_rn(f[0]), b1 = __float2bfloat16_rn(f[1]);
      w[k2] = (uint32_t)__bfloat16_as_ushort(b0) | ((uint32_t)__bfloat16_as_ushort(b1) << 16);
    }
    __nv_bfloat16* dst = img + (int64_t)im * C * kCtAtoms * (kCtM * 64) +
                         ((int64_t)tile * kCtM + row) * 64 + 8 * pos;
    *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

}  // namespace

size_t conv_tc_image_bytes(int C) { return (size_t)2 * C * kCtAtoms * kCtATile; }

void conv_tc_prepare(const float* h, int C, int T, float* h64, __nv_bfloat16* img,
                     cudaStream_t st) {
  const int n = C * 64 + 2 * C * kCtAtoms * kCtM * 8;
  launch_k(conv_tc_prep_kernel, dim3((unsigned)((n + 255) / 256)), dim3(256), 0, st, h, C, T, h64,
           img);
  apply_tick(st);
}

static int conv_tc_grid(int units) {
  const int sms = num_sms();
  return units < sms ? units : sms;
}

void conv_tc_forward(int C, int64_t L, const float* Z, int64_t ldz, int ncols, float* W,
                     int64_t ldw, const __nv_bfloat16* img, int* err, cudaStream_t st) {
  cudaFuncSetAttribute(conv_tc_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)kFwdSmem);
  CtArgs a = {};
  a.C = C;
  a.L = L;
  a.ncols = ncols;
  a.units = ncols * (int)((L + kCtTile - 1) / kCtTile);
  a.x = Z;
  a.ldx = ldz;
  a.y = W;
  a.ldy = ldw;
  a.img = img;
  a.err = err;
  launch_k(conv_tc_forward_kernel, dim3((unsigned)conv_tc_grid(a.units)), dim3(kCtFwdThreads),
           kFwdSmem, st, a);
  apply_tick(st);
}

int conv_tc_adjoint(int C, int64_t L, const float* W, int64_t ldw, int ncols, float* Y,
                    int64_t ld, double beta, const double* alpha, const float* alpha32,
                    const float* X, double* dots, const __nv_bfloat16* img, int* err,
                    cudaStream_t st) {
  cudaFuncSetAttribute(conv_tc_adjoint_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)kAdjSmem);
  const int nq = (int)((L + kCtTile - 1) / kCtTile);
  CtArgs a = {};
  a.C = C;
  a.L = L;
  a.ncols = ncols;
  a.units = ncols * nq;
  a.x = W;
  a.ldx = ldw;
  a.y = Y;
  a.ldy = ld;
  a.img = img + (size_t)C * kCtAtoms * (kCtM * 64);
  a.beta = beta;
  a.alpha = alpha;
  a.alpha32 = alpha32;
  a.xd = X;
  a.dots = dots;
  a.err = err;
  launch_k(conv_tc_adjoint_kernel, dim3((unsigned)conv_tc_grid(a.units)), dim3(kCtAdjThreads),
           kAdjSmem, st, a);
  apply_tick(st);
  return nq;
}

}  // namespace cofem
