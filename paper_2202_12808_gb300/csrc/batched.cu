// Many independent SBL problems of uneven size in one fit (cofem_fit_batched):
// Algorithm 1 run for every problem at once, each problem with its own
// column-wise CG recurrences (Sec. 3.2), its own stop test and its own
// probes, on BF16 dictionaries through the tensor-core operator.
//
// Layout: the problems' vectors are concatenated (problem i's block of K+1
// columns at xoff_i with leading dimension ld_i); their dictionaries are
// packed (tile-major, pre-swizzled) one after another.  The two products of
// every operator application are grouped GEMMs over a host-built table of
// work items (problem, row tile, K range), longest first; the items of a
// problem whose CG has converged exit at once (per-problem done mask).  The
// vector kernels run over a (chunk, column, problem) grid and reduce per
// problem in a fixed order.  One CUDA graph per EM iteration: a WHILE node
// repeats the CG iteration until every problem is done.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "dense.cuh"

namespace cofem {

constexpr int kBSub = 4;                // 16-byte chunks per thread
constexpr int kBChunk = 1024 * kBSub;   // vector elements per block (256 threads x 4 x kBSub)

struct BVec {                           // one problem, as the vector kernels see it
  int64_t D, ld, xoff, aoff, boff1;
  uint64_t seed;
  int nch;                              // chunks of kBChunk elements
  int dots_base, ndots;                 // its slots of the operator's partial dots
};

struct BState {                         // one problem's CG state (device)
  int iter, done, error, pad;
  int clamps, support;
  unsigned int counter[4];
  double normB2, relres;
  double b0norm2;                       // ||b||^2 of column 0 (probe columns: D)
  double rho[kMaxCols], rho_new[kMaxCols], b[kMaxCols];
  // learned start: the solve is preconditioned (rho holds r_j^T z_j, z = M^-1 r,
  // rr_new the r_j^T r_j of the stop test); iterations of a preconditioned
  // solve that fell back, fallbacks so far
  double rr_new[kMaxCols];
  int pcg, extra_iters, fallbacks, pad2;
};

struct BCtl {
  long long t;
  int em_index;
  int error;
  int fallbacks;                        // learned start: fallbacks to plain CG, all problems
  int pad;
};

struct BConf {
  int nprob, nc, K;
  double tol;
  int max_iters, fixed_iters;
  double den_floor, support_threshold;
  int em_iters;
  unsigned long long while_handle;
  int nch_max;                           // partial-sum slots per problem
  int stop_rule;                         // 1: per-column stop (frozen columns have rho_j = 0)
  int split_nt;
  int64_t split_ld;                      // pitch of the BF16 split buffer
  __nv_bfloat16* split_buf;
  const float* minv;                     // learned start: M^-1 per coordinate (aoff + d), else null
  unsigned long long while2_handle;      // learned start: the plain-CG rerun loop
  long long t_first;                     // learned start: EM iteration of the fit's first E-step
  int only_undone;                       // binit: re-initialise only problems with done == 0
};

__device__ __forceinline__ void bset_cond(unsigned long long h, unsigned v) {
  if (h) cudaGraphSetConditional((cudaGraphConditionalHandle)h, v);
}

__device__ __forceinline__ void bsplit4(const BConf& cf, const BVec& pv, int j, int64_t d,
                                        const float (&v)[4]) {
  float r[4] = {v[0], v[1], v[2], v[3]};
  for (int t = 0; t < cf.split_nt; ++t) {
    __nv_bfloat16 o[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      o[i] = __float2bfloat16_rn(r[i]);
      r[i] -= __bfloat162float(o[i]);
    }
    *reinterpret_cast<uint2*>(cf.split_buf + (int64_t)split_row(j, t, cf.split_nt) * cf.split_ld +
                              pv.boff1 + d) = *reinterpret_cast<uint2*>(o);
  }
}

__device__ __forceinline__ float bprobe(uint64_t key, int64_t d, int k) {
  const uint64_t h = probe_word(key, d, k >> 6);
  return ((h >> (k & 63)) & 1ull) ? -1.f : 1.f;
}

// per-problem last-block arrival on st.counter[c] among `expected` blocks
// As arrive_last: what the last block reads was written by each block's
// thread 0, which fences before arriving.
__device__ __forceinline__ bool barrive_last(unsigned int* counter, unsigned expected) {
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(counter, 1u) == expected - 1;
    if (last) __threadfence();
  }
  __syncthreads();
  return last;
}

// All threads of the problem's last block (blockDim >= nc): b_j by thread j,
// the residual total by the first warp (fixed order), the stop test (joint,
// or per column as in the single-problem solver).
__device__ void bfinalize(const BConf& cf, BState* st, int64_t D) {
  __shared__ double tot_sh;
  __syncthreads();
  const int j = threadIdx.x;
  if (j < 32) {
    double t = 0.0;
    for (int c = j; c < cf.nc; c += 32) t += st->pcg ? st->rr_new[c] : st->rho_new[c];
    t = warp_sum(t);
    if (j == 0) tot_sh = t;
  }
  int live = 0;
  if (j < cf.nc) {
    const double r0 = st->rho[j], r1 = st->rho_new[j];
    if (cf.stop_rule == 1) {
      const double bn2 = j == 0 ? st->b0norm2 : (double)D;
      live = r0 > 0.0 && !(sqrt(r1) < cf.tol * sqrt(bn2));
      st->b[j] = live ? r1 / r0 : 0.0;
      st->rho[j] = live ? r1 : 0.0;
    } else {
      st->b[j] = r0 > 0.0 ? r1 / r0 : 0.0;
      st->rho[j] = r1;
    }
  }
  const int nlive = __syncthreads_count(live);
  if (j == 0) {
    const double relres = sqrt(tot_sh) / sqrt(st->normB2);
    st->relres = relres;
    int done;
    if (cf.fixed_iters > 0) done = st->iter >= cf.fixed_iters;
    else if (cf.stop_rule == 1) done = nlive == 0 || st->iter >= cf.max_iters;
    else done = relres < cf.tol || st->iter >= cf.max_iters;
    if (!isfinite(relres)) { st->error = COFEM_ERR_NONFINITE; done = 1; }
    st->done = done;
  }
}

// X = 0, R = P = B (b and the problem's probes), P's BF16 terms; rho, ||B||.
__global__ void binit_kernel(BConf cf, const BVec* pvs, BState* sts, int* done, const BCtl* ctl,
                             float* X, float* R, float* P, const float* bv, double* part) {
  pdl_wait();
  pdl_trigger();
  __shared__ double sh[32];
  const int pi = blockIdx.z, j = blockIdx.y, c = blockIdx.x;
  const BVec pv = pvs[pi];
  if (c >= pv.nch) return;
  if (cf.only_undone && done[pi]) return;   // rerun only the problems that fell back
  BState* st = sts + pi;
  const uint64_t key = probe_key(pv.seed, ctl->t);
  float* x = X + pv.xoff + (int64_t)j * pv.ld;
  float* r = R + pv.xoff + (int64_t)j * pv.ld;
  float* p = P + pv.xoff + (int64_t)j * pv.ld;
  AccF acc;
#pragma unroll
  for (int u = 0; u < kBSub; ++u) {
    const int64_t d = (int64_t)c * kBChunk + u * 1024 + threadIdx.x * 4;
    if (d < pv.ld) {
      float v[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        float w = 0.f;
        if (d + i < pv.D) {
          if (j == 0) { w = bv[pv.aoff + d + i]; acc.add_prod(w, w); }
          else w = bprobe(key, d + i, j - 1);
        }
        v[i] = w;
        x[d + i] = 0.f;
        r[d + i] = w;
        p[d + i] = w;
      }
      if (cf.split_nt > 0) bsplit4(cf, pv, j, d, v);
    }
  }
  if (j == 0) {
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) part[((int64_t)pi * cf.nch_max + c) * kMaxCols] = s;
  }
  if (barrive_last(&st->counter[0], (unsigned)(pv.nch * cf.nc))) {
    if (threadIdx.x == 0) {
      double b2 = 0.0;
      for (int i = 0; i < pv.nch; ++i) b2 += part[((int64_t)pi * cf.nch_max + i) * kMaxCols];
      st->rho[0] = b2;
      for (int jj = 1; jj < cf.nc; ++jj) st->rho[jj] = (double)pv.D;
      st->normB2 = b2 + (double)cf.K * (double)pv.D;
      st->b0norm2 = b2;
      if (cf.stop_rule == 1 && !(b2 > 0.0)) st->rho[0] = 0.0;   // b = 0: x = 0, frozen
      st->relres = 1.0;
      st->iter = 0;
      st->pcg = 0;
      if (!cf.only_undone) st->extra_iters = 0;
      st->clamps = 0;
      st->support = 0;
      int dn = 0;
      if (!(st->normB2 > 0.0)) dn = 1;
      if (!isfinite(st->normB2)) { st->error = COFEM_ERR_NONFINITE; dn = 1; }
      st->done = dn;
      done[pi] = dn;
      st->counter[0] = 0;
    }
  }
}

// Learned start, after Q = A X0: R = B - Q, Z = M^-1 R, P = Z (and P's BF16
// terms); rho_j = r_j^T z_j, rr_j = r_j^T r_j; ||B||; the stop test on
// ||R||_F / ||B||_F.  Grid and reductions as in binit_kernel.
__global__ void binit_warm_kernel(BConf cf, const BVec* pvs, BState* sts, int* done,
                                  const BCtl* ctl, float* R, float* P, const float* Q,
                                  const float* bv, double* part, double* part2, double* partb) {
  pdl_wait();
  pdl_trigger();
  __shared__ double sh[32];
  const int pi = blockIdx.z, j = blockIdx.y, c = blockIdx.x;
  const BVec pv = pvs[pi];
  if (c >= pv.nch) return;
  BState* st = sts + pi;
  const uint64_t key = probe_key(pv.seed, ctl->t);
  float* r = R + pv.xoff + (int64_t)j * pv.ld;
  float* p = P + pv.xoff + (int64_t)j * pv.ld;
  const float* q = Q + pv.xoff + (int64_t)j * pv.ld;
  AccF az, ar, ab;
#pragma unroll
  for (int u = 0; u < kBSub; ++u) {
    const int64_t d = (int64_t)c * kBChunk + u * 1024 + threadIdx.x * 4;
    if (d < pv.ld) {
      float v[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        float bw = 0.f, rv = 0.f, zv = 0.f;
        if (d + i < pv.D) {
          if (j == 0) { bw = bv[pv.aoff + d + i]; ab.add_prod(bw, bw); }
          else bw = bprobe(key, d + i, j - 1);
          rv = bw - q[d + i];
          zv = rv * cf.minv[pv.aoff + d + i];
        }
        r[d + i] = rv;
        p[d + i] = zv;
        v[i] = zv;
        az.add_prod(rv, zv);
        ar.add_prod(rv, rv);
      }
      if (cf.split_nt > 0) bsplit4(cf, pv, j, d, v);
    }
  }
  const double sz = block_sum(az, sh);
  const double sr = block_sum(ar, sh);
  const double sb = j == 0 ? block_sum(ab, sh) : 0.0;
  const int64_t slot = ((int64_t)pi * cf.nch_max + c) * kMaxCols;
  if (threadIdx.x == 0) {
    part[slot + j] = sz;
    part2[slot + j] = sr;
    if (j == 0) partb[(int64_t)pi * cf.nch_max + c] = sb;
    __threadfence();
  }
  if (barrive_last(&st->counter[0], (unsigned)(pv.nch * cf.nc))) {
    if (threadIdx.x < cf.nc) {
      double tz = 0.0, tr = 0.0;
      for (int i = 0; i < pv.nch; ++i) {
        tz += part[((int64_t)pi * cf.nch_max + i) * kMaxCols + threadIdx.x];
        tr += part2[((int64_t)pi * cf.nch_max + i) * kMaxCols + threadIdx.x];
      }
      st->rho[threadIdx.x] = tz;
      st->rr_new[threadIdx.x] = tr;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double b2 = 0.0, r2 = 0.0;
      for (int i = 0; i < pv.nch; ++i) b2 += partb[(int64_t)pi * cf.nch_max + i];
      for (int jj = 0; jj < cf.nc; ++jj) r2 += st->rr_new[jj];
      st->normB2 = b2 + (double)cf.K * (double)pv.D;
      st->b0norm2 = b2;
      st->relres = st->normB2 > 0.0 ? sqrt(r2) / sqrt(st->normB2) : 0.0;
      st->iter = 0;
      st->pcg = 1;
      st->extra_iters = 0;
      st->clamps = 0;
      st->support = 0;
      int dn = !(st->normB2 > 0.0) || (cf.fixed_iters == 0 && st->relres < cf.tol);
      if (!isfinite(st->normB2) || !isfinite(st->relres)) { st->error = COFEM_ERR_NONFINITE; dn = 1; }
      st->done = dn;
      done[pi] = dn;
      st->counter[0] = 0;
    }
  }
}

// Learned start, after the preconditioned solves: a problem whose solve ran
// into the cap without meeting the tolerance (not at the fit's first E-step,
// where the solve is plain CG) is rerun as plain CG from zero; its
// iterations so far are kept in extra_iters.  done[i] = 0 marks the reruns;
// the rerun loop's condition is whether any problem fell back.
__global__ void bfallback_kernel(BConf cf, BState* sts, int* done, BCtl* ctl) {
  pdl_wait();
  pdl_trigger();
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  const bool first = ctl->t == cf.t_first;
  for (int i = threadIdx.x; i < cf.nprob; i += blockDim.x) {
    BState* st = sts + i;
    const bool fb = !first && cf.fixed_iters == 0 && st->pcg && !st->error &&
                    !(st->relres < cf.tol);
    if (fb) {
      st->extra_iters = st->iter;
      st->fallbacks += 1;
      atomicAdd(&ctl->fallbacks, 1);
      any = 1;
    }
    done[i] = fb ? 0 : 1;
  }
  __syncthreads();
  if (threadIdx.x == 0) bset_cond(cf.while2_handle, any ? 1u : 0u);
}

// a_j = rho_j / gamma_j of every unconverged problem and column, gamma_j =
// p_j^T A p_j summed from the second product's partial dots; one warp per
// (problem, column): blocks of kStepWarps warps, grid (problems, column
// groups).  A breakdown (gamma <= 0 with rho > 0) sets the problem's error.
constexpr int kStepWarps = 8;
__global__ void bstep_kernel(BConf cf, const BVec* pvs, BState* sts, const int* done,
                             const double* dots, float* astep) {
  pdl_wait();
  pdl_trigger();
  const int pi = blockIdx.x, lane = threadIdx.x & 31;
  const int j = blockIdx.y * kStepWarps + (threadIdx.x >> 5);
  if (j >= cf.nc || done[pi]) return;
  const BVec pv = pvs[pi];
  BState* st = sts + pi;
  double g = 0.0;
  for (int i0 = lane; i0 < pv.ndots; i0 += 64) {
    const double g0 = dots[(int64_t)(pv.dots_base + i0) * kMaxCols + j];
    const double g1 = i0 + 32 < pv.ndots ? dots[(int64_t)(pv.dots_base + i0 + 32) * kMaxCols + j] : 0.0;
    g += g0 + g1;
  }
  g = warp_sum(g);
  if (lane == 0) {
    const double rho = st->rho[j];
    double a = 0.0;
    if (rho > 0.0) {
      if (!(g > 0.0)) st->error = isfinite(g) ? COFEM_ERR_BREAKDOWN : COFEM_ERR_NONFINITE;
      else a = rho / g;
    }
    astep[(int64_t)pi * kMaxCols + j] = (float)a;
  }
}

// x += a p, r -= a q (a from bstep_kernel), rho_new partials; last block:
// stop test.  Grid (chunks, 1, problems): a block takes one chunk of a
// problem through all its columns (per-block latency paid once, not once
// per column); per column, each warp folds its compensated partial with
// shuffles, and the warps' partials are combined in warp order at the end.
__global__ void bupdate_kernel(BConf cf, const BVec* pvs, BState* sts, int* done, float* X,
                               float* R, const float* P, const float* Q, const float* astep,
                               double* part, double* part2) {
  pdl_wait();
  pdl_trigger();
  constexpr int kWarps = 256 / 32;
  __shared__ float2 red2[kWarps][kMaxCols];      // per warp and column: (sum, compensation)
  __shared__ double redb[kWarps][kMaxCols];      // FP64 side sums of out-of-range products
  __shared__ float2 rrd2[kWarps][kMaxCols];      // preconditioned solves: r^T r as well
  __shared__ double rrdb[kWarps][kMaxCols];
  const int pi = blockIdx.z, c = blockIdx.x;
  const BVec pv = pvs[pi];
  if (c >= pv.nch || done[pi]) return;
  BState* st = sts + pi;
  const bool pcg = cf.minv && st->pcg;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int j = 0; j < cf.nc; ++j) {
    const int64_t o0 = pv.xoff + (int64_t)j * pv.ld;
    float4 xv[kBSub], rv[kBSub], pp[kBSub], qq[kBSub];
#pragma unroll
    for (int u = 0; u < kBSub; ++u) {
      const int64_t d = (int64_t)c * kBChunk + u * 1024 + threadIdx.x * 4;
      if (d < pv.ld) {
        xv[u] = *reinterpret_cast<const float4*>(X + o0 + d);
        rv[u] = *reinterpret_cast<const float4*>(R + o0 + d);
        pp[u] = *reinterpret_cast<const float4*>(P + o0 + d);
        qq[u] = *reinterpret_cast<const float4*>(Q + o0 + d);
      }
    }
    const float a = astep[(int64_t)pi * kMaxCols + j];
    AccF acc, acc2;                    // rho_new (r^T r, or r^T z when preconditioned); r^T r
#pragma unroll
    for (int u = 0; u < kBSub; ++u) {
      const int64_t d = (int64_t)c * kBChunk + u * 1024 + threadIdx.x * 4;
      if (d < pv.ld) {
        float4 x4 = xv[u], r4 = rv[u];
        x4.x = fmaf(a, pp[u].x, x4.x); x4.y = fmaf(a, pp[u].y, x4.y);
        x4.z = fmaf(a, pp[u].z, x4.z); x4.w = fmaf(a, pp[u].w, x4.w);
        r4.x = fmaf(-a, qq[u].x, r4.x); r4.y = fmaf(-a, qq[u].y, r4.y);
        r4.z = fmaf(-a, qq[u].z, r4.z); r4.w = fmaf(-a, qq[u].w, r4.w);
        if (pcg) {
          const float rr[4] = {r4.x, r4.y, r4.z, r4.w};
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const float mv = d + i < pv.D ? cf.minv[pv.aoff + d + i] : 0.f;
            acc.add_prod(rr[i], rr[i] * mv);
            acc2.add_prod(rr[i], rr[i]);
          }
        } else {
          acc.add_prod(r4.x, r4.x);
          acc.add_prod(r4.y, r4.y);
          acc.add_prod(r4.z, r4.z);
          acc.add_prod(r4.w, r4.w);
        }
        *reinterpret_cast<float4*>(X + o0 + d) = x4;
        *reinterpret_cast<float4*>(R + o0 + d) = r4;
      }
    }
    float sv = acc.s, cv = acc.c;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
      two_sum_merge(sv, cv, __shfl_xor_sync(0xffffffffu, sv, o), __shfl_xor_sync(0xffffffffu, cv, o));
    const double bg = warp_sum(acc.big);
    if (lane == 0) {
      red2[wid][j] = make_float2(sv, cv);
      redb[wid][j] = bg;
    }
    if (pcg) {
      float s2 = acc2.s, c2 = acc2.c;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
        two_sum_merge(s2, c2, __shfl_xor_sync(0xffffffffu, s2, o),
                      __shfl_xor_sync(0xffffffffu, c2, o));
      const double b2 = warp_sum(acc2.big);
      if (lane == 0) {
        rrd2[wid][j] = make_float2(s2, c2);
        rrdb[wid][j] = b2;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x < cf.nc) {
    const int j = threadIdx.x;
    float sv = red2[0][j].x, cv = red2[0][j].y;
    double bg = redb[0][j];
    for (int w = 1; w < kWarps; ++w) {
      two_sum_merge(sv, cv, red2[w][j].x, red2[w][j].y);
      bg += redb[w][j];
    }
    part[((int64_t)pi * cf.nch_max + c) * kMaxCols + j] = ((double)sv + (double)cv) + bg;
    if (pcg) {
      float s2 = rrd2[0][j].x, c2 = rrd2[0][j].y;
      double b2 = rrdb[0][j];
      for (int w = 1; w < kWarps; ++w) {
        two_sum_merge(s2, c2, rrd2[w][j].x, rrd2[w][j].y);
        b2 += rrdb[w][j];
      }
      part2[((int64_t)pi * cf.nch_max + c) * kMaxCols + j] = ((double)s2 + (double)c2) + b2;
    }
    __threadfence();                   // the last block reads these partials
  }
  if (barrive_last(&st->counter[1], (unsigned)pv.nch)) {
    if (threadIdx.x < cf.nc) {
      double t = 0.0, t2 = 0.0;
      for (int i = 0; i < pv.nch; ++i) {
        t += part[((int64_t)pi * cf.nch_max + i) * kMaxCols + threadIdx.x];
        if (pcg) t2 += part2[((int64_t)pi * cf.nch_max + i) * kMaxCols + threadIdx.x];
      }
      st->rho_new[threadIdx.x] = t;
      if (pcg) st->rr_new[threadIdx.x] = t2;
    }
    if (threadIdx.x == 0) {
      st->iter += 1;
      st->counter[1] = 0;
    }
    bfinalize(cf, st, pv.D);
    if (threadIdx.x == 0) done[pi] = st->done;
  }
}

// WHILE condition: some problem still iterating.
__global__ void bcond_kernel(BConf cf, const int* done) {
  pdl_wait();
  pdl_trigger();
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < cf.nprob; i += blockDim.x)
    if (!done[i]) any = 1;
  __syncthreads();
  if (threadIdx.x == 0) bset_cond(cf.while_handle, any ? 1u : 0u);
}

// p = r + b p and P's BF16 terms.
__global__ void bdirection_kernel(BConf cf, const BVec* pvs, const BState* sts, const int* done,
                                  const float* R, float* P) {
  pdl_wait();
  pdl_trigger();
  const int pi = blockIdx.z, j = blockIdx.y, c = blockIdx.x;
  const BVec pv = pvs[pi];
  if (c >= pv.nch || done[pi]) return;
  const float b = (float)sts[pi].b[j];
  const bool pcg = cf.minv && sts[pi].pcg;
  const int64_t o0 = pv.xoff + (int64_t)j * pv.ld;
  float4 rv[kBSub], pp[kBSub];
#pragma unroll
  for (int u = 0; u < kBSub; ++u) {
    const int64_t d = (int64_t)c * kBChunk + u * 1024 + threadIdx.x * 4;
    if (d < pv.ld) {
      rv[u] = *reinterpret_cast<const float4*>(R + o0 + d);
      pp[u] = *reinterpret_cast<const float4*>(P + o0 + d);
    }
  }
#pragma unroll
  for (int u = 0; u < kBSub; ++u) {
    const int64_t d = (int64_t)c * kBChunk + u * 1024 + threadIdx.x * 4;
    if (d < pv.ld) {
      float4 p4 = pp[u], z4 = rv[u];
      if (pcg) {             // z = M^-1 r (zero past D)
        z4.x *= d + 0 < pv.D ? cf.minv[pv.aoff + d + 0] : 0.f;
        z4.y *= d + 1 < pv.D ? cf.minv[pv.aoff + d + 1] : 0.f;
        z4.z *= d + 2 < pv.D ? cf.minv[pv.aoff + d + 2] : 0.f;
        z4.w *= d + 3 < pv.D ? cf.minv[pv.aoff + d + 3] : 0.f;
      }
      p4.x = fmaf(b, p4.x, z4.x); p4.y = fmaf(b, p4.y, z4.y);
      p4.z = fmaf(b, p4.z, z4.z); p4.w = fmaf(b, p4.w, z4.w);
      *reinterpret_cast<float4*>(P + o0 + d) = p4;
      if (cf.split_nt > 0) {
        const float v[4] = {p4.x, p4.y, p4.z, p4.w};
        bsplit4(cf, pv, j, d, v);
      }
    }
  }
}

// W = sum_s W_s (split order) -> BF16 terms in Ws; grid (chunks, slots, problems).
template <int NT>
__global__ void breduce_kernel(const TcProb* probs, const int* done, int nc, const float* Wp,
                               __nv_bfloat16* Ws, int64_t ldw_total) {
  pdl_wait();
  pdl_trigger();
  constexpr int G = 16 / NT;
  const int pi = blockIdx.z, j = blockIdx.y;
  const TcProb pr = probs[pi];
  if (done[pi] || pr.S1 == 1) return;   // one K range: the product wrote the terms
  const int gi = j / G, jj = j % G;
  const int64_t n = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
  if (n >= pr.ldw) return;
  float r[4] = {0.f, 0.f, 0.f, 0.f};
  if (j < nc) {
    for (int s = 0; s < pr.S1; ++s) {
      const float4 v = __ldcg(reinterpret_cast<const float4*>(
          Wp + pr.wpoff + (int64_t)s * nc * pr.ldw + (int64_t)j * pr.ldw + n));
      r[0] += v.x; r[1] += v.y; r[2] += v.z; r[3] += v.w;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (n + i >= pr.N) r[i] = 0.f;
  }
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    __nv_bfloat16 o[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      o[i] = __float2bfloat16_rn(r[i]);
      r[i] -= __bfloat162float(o[i]);
    }
    *reinterpret_cast<uint2*>(Ws + (int64_t)(gi * 16 + jj * NT + t) * ldw_total + pr.boff2 + n) =
        *reinterpret_cast<uint2*>(o);
  }
  if (jj == G - 1)
    for (int rr = G * NT; rr < 16; ++rr)
      *reinterpret_cast<uint2*>(Ws + (int64_t)(gi * 16 + rr) * ldw_total + pr.boff2 + n) =
          make_uint2(0u, 0u);
}

// mu, s, alpha of every problem (Eq. (diag-estimate), M-step); counters.
__global__ void bdiag_kernel(BConf cf, const BVec* pvs, BState* sts, const BCtl* ctl,
                             const float* X, double* mu, double* s, double* alpha) {
  pdl_wait();
  pdl_trigger();
  __shared__ double sh[32];
  const int pi = blockIdx.z, c = blockIdx.x;
  const BVec pv = pvs[pi];
  if (c >= pv.nch) return;
  const uint64_t key = probe_key(pv.seed, ctl->t);
  int clamps = 0, support = 0, bad = 0;
  for (int64_t d = (int64_t)c * kBChunk + threadIdx.x; d < min(pv.D, (int64_t)(c + 1) * kBChunk);
       d += blockDim.x) {
    const double m = (double)X[pv.xoff + d];
    double acc = 0.0;
    for (int k = 0; k < cf.K; ++k) {
      const double xv = (double)X[pv.xoff + (int64_t)(k + 1) * pv.ld + d];
      acc += bprobe(key, d, k) < 0.f ? -xv : xv;
    }
    const double sd = acc * (1.0 / (double)cf.K);     // as in the single-problem M-step
    const double den = m * m + sd;
    if (den < cf.den_floor) ++clamps;
    const double al = __drcp_rn(fmax(den, cf.den_floor));
    if (!isfinite(m) || !isfinite(sd)) bad = 1;
    if (al < cf.support_threshold) ++support;
    mu[pv.aoff + d] = m;
    s[pv.aoff + d] = sd;
    alpha[pv.aoff + d] = al;
  }
  const double cs = block_sum((double)clamps, sh);
  const double ss = block_sum((double)support, sh);
  const double bs = block_sum((double)bad, sh);
  if (threadIdx.x == 0) {
    if (cs > 0) atomicAdd(&sts[pi].clamps, (int)cs);
    if (ss > 0) atomicAdd(&sts[pi].support, (int)ss);
    if (bs > 0) sts[pi].error = COFEM_ERR_NONFINITE;
  }
}

// per-problem statistics of this EM iteration; t += 1
__global__ void bfinish_kernel(BConf cf, BState* sts, BCtl* ctl, int32_t* st_iters,
                               double* st_relres, int32_t* st_clamps, int32_t* st_support) {
  pdl_wait();
  pdl_trigger();
  const int e = ctl->em_index;
  for (int i = threadIdx.x; i < cf.nprob; i += blockDim.x) {
    if (e < cf.em_iters) {
      st_iters[(int64_t)i * cf.em_iters + e] = sts[i].iter + sts[i].extra_iters;
      st_relres[(int64_t)i * cf.em_iters + e] = sts[i].relres;
      st_clamps[(int64_t)i * cf.em_iters + e] = sts[i].clamps;
      st_support[(int64_t)i * cf.em_iters + e] = sts[i].support;
    }
    if (sts[i].error) atomicCAS(&ctl->error, 0, sts[i].error);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    ctl->em_index = e + 1;
    ctl->t += 1;
  }
}

__global__ void bctl_init_kernel(BCtl* ctl, long long t0) {
  pdl_wait();
  pdl_trigger();
  ctl->t = t0;
  ctl->em_index = 0;
  ctl->error = 0;
  ctl->fallbacks = 0;
}

__global__ void bfill_kernel(double* x, int64_t n, double v) {
  pdl_wait();
  pdl_trigger();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] = v;
}

// ============================================================= host side

static size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

struct BLayout {
  // per-problem geometry
  std::vector<BVec> vec;
  std::vector<TcProb> tcp;
  std::vector<TcItem> items1, items2;
  int nch_max = 0, ndots = 0, BN = 0, NT = 3, stages = 3, grid = 0;
  bool any_split = false;                 // some problem's first product is split over K
  uint32_t tmem_cols = 0;                 // two accumulators
  size_t smem = 0;
  int64_t ldx_total = 0, ldw_total = 0, dtot = 0, ldw_max = 0;
  // workspace offsets
  size_t o_packed, o_X, o_R, o_P, o_Q, o_b, o_xs, o_ws, o_wpart, o_dots, o_part, o_astep, o_state, o_done,
      o_ctl, o_vec, o_tcp, o_it1, o_it2, o_st_it, o_st_rr, o_st_cl, o_st_sp, o_simt, total;
  // learned start: M^-1 and ||phi_d||^2 per coordinate, second and norm partials,
  // the warm-start kernel's problem table
  size_t o_minv = 0, o_pn2 = 0, o_part2 = 0, o_partb = 0, o_wprob = 0;
  std::vector<BWarmProb> wprob;
  int64_t ld_max = 0;
};

// K blocks (64 columns of Phi) of one first-product work item at most: up to
// D = 8192 a problem's first product is one K range per tile, whose
// epilogue writes the BF16 terms of W itself (no split-K reduction); the
// items, sorted longest first, still balance over the persistent CTAs.
constexpr int kB1MaxKb = 128;

static cofem_status blayout(int n, const cofem_problem* pr, const cofem_params* p, BLayout* L) {
  const int nc = p->K + 1;
  L->NT = 3;
  const int G = 16 / L->NT;
  L->BN = ((nc + G - 1) / G) * 16;
  // pipeline shape: two CTAs per SM until the autotuner (btune) has run
  DenseTcPlan plan = dense_tc_plan(2048, 8192, nc, L->NT, num_sms(), 2, 0);
  L->tmem_cols = plan.tmem_cols;
  L->stages = plan.stages;
  L->smem = plan.smem;
  L->grid = plan.grid;
  int64_t xoff = 0, aoff = 0, b1 = 0, b2 = 0, wpoff = 0, poff = 0;
  size_t simt = 0;
  int dots = 0;
  for (int i = 0; i < n; ++i) {
    const int64_t N = pr[i].N, D = pr[i].D;
    if (N < 1 || D < 1 || !pr[i].phi_dev || !pr[i].y_dev || pr[i].ld < D || pr[i].ld % 64 ||
        !(pr[i].beta > 0.0) || ((uintptr_t)pr[i].phi_dev & 255))
      return COFEM_ERR_INVALID_ARG;
    const int64_t ld = round_up(D, kLdAlign), ldw = round_up(N, kLdAlign);
    BVec v;
    v.D = D; v.ld = ld; v.xoff = xoff; v.aoff = aoff; v.boff1 = b1; v.seed = pr[i].seed;
    v.nch = (int)((ld + kBChunk - 1) / kBChunk);
    v.dots_base = dots;
    v.ndots = (int)((D + 127) / 128);
    TcProb t;
    t.N = N; t.D = D; t.nkd = packed_tiles_k(D); t.poff = poff; t.xoff = xoff; t.ld = ld;
    t.aoff = aoff; t.boff1 = b1; t.boff2 = b2; t.wpoff = wpoff; t.ldw = ldw;
    const int nk1 = (int)((D + 63) / 64);
    t.S1 = (nk1 + kB1MaxKb - 1) / kB1MaxKb;
    const int kbps = (nk1 + t.S1 - 1) / t.S1;
    t.dots_base = dots;
    t.beta = pr[i].beta;
    for (int mt = 0; mt < (int)((N + 127) / 128); ++mt)
      for (int sp = 0; sp < t.S1; ++sp)
        L->items1.push_back({i, mt, sp, sp * kbps, std::min(nk1, (sp + 1) * kbps)});
    const int nk2 = (int)((N + 63) / 64);
    for (int mt = 0; mt < v.ndots; ++mt) L->items2.push_back({i, mt, 0, 0, nk2});
    L->vec.push_back(v);
    L->tcp.push_back(t);
    L->wprob.push_back({D, ld, xoff, aoff, b1, pr[i].seed, pr[i].beta});
    L->ld_max = std::max(L->ld_max, ld);
    xoff += (int64_t)nc * ld;
    aoff += D;
    b1 += ld;
    b2 += ldw;
    if (t.S1 > 1) {
      wpoff += (int64_t)t.S1 * nc * ldw;
      L->any_split = true;
    }
    poff += (int64_t)(packed_bytes(N, D) / 2);
    dots += v.ndots;
    L->nch_max = std::max(L->nch_max, v.nch);
    L->ldw_max = std::max(L->ldw_max, ldw);
    DenseSimtPlan sp = dense_simt_plan(N, D, 1, 4, num_sms());
    simt = std::max(simt, sp.total());
  }
  // longest items first
  std::stable_sort(L->items1.begin(), L->items1.end(),
                   [](const TcItem& a, const TcItem& b) { return a.kb1 - a.kb0 > b.kb1 - b.kb0; });
  std::stable_sort(L->items2.begin(), L->items2.end(),
                   [](const TcItem& a, const TcItem& b) { return a.kb1 > b.kb1; });
  L->ndots = dots;
  L->ldx_total = b1;
  L->ldw_total = b2;
  L->dtot = aoff;
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t r = o; o += a256(bytes); return r; };
  L->o_packed = take((size_t)poff * 2);
  L->o_X = take((size_t)xoff * 4);
  L->o_R = take((size_t)xoff * 4);
  L->o_P = take((size_t)xoff * 4);
  L->o_Q = take((size_t)xoff * 4);
  L->o_b = take((size_t)aoff * 4);
  L->o_xs = take((size_t)L->BN * b1 * 2);
  L->o_ws = take((size_t)L->BN * b2 * 2);
  L->o_wpart = take((size_t)wpoff * 4);
  L->o_dots = take((size_t)dots * kMaxCols * 8);
  L->o_part = take((size_t)n * L->nch_max * kMaxCols * 8);
  L->o_astep = take((size_t)n * kMaxCols * 4);
  L->o_state = take((size_t)n * sizeof(BState));
  L->o_done = take((size_t)n * 4);
  L->o_ctl = take(sizeof(BCtl));
  L->o_vec = take((size_t)n * sizeof(BVec));
  L->o_tcp = take((size_t)n * sizeof(TcProb));
  L->o_it1 = take(L->items1.size() * sizeof(TcItem));
  L->o_it2 = take(L->items2.size() * sizeof(TcItem));
  const int ne = std::max(1, p->em_iters);
  L->o_st_it = take((size_t)n * ne * 4);
  L->o_st_rr = take((size_t)n * ne * 8);
  L->o_st_cl = take((size_t)n * ne * 4);
  L->o_st_sp = take((size_t)n * ne * 4);
  L->o_simt = take(simt);
  if (p->mlp) {
    L->o_minv = take((size_t)aoff * 4);
    L->o_pn2 = take((size_t)aoff * 4);
    L->o_part2 = take((size_t)n * L->nch_max * kMaxCols * 8);
    L->o_partb = take((size_t)n * L->nch_max * 8);
    L->o_wprob = take((size_t)n * sizeof(BWarmProb));
  }
  L->total = o;
  return COFEM_OK;
}

static cofem_status bcheck(int n, const cofem_problem* pr, const cofem_params* p) {
  if (n < 1 || !pr || !p) return COFEM_ERR_INVALID_ARG;
  if (p->K < 1 || p->K + 1 > kMaxCols || p->em_iters < 0 || p->cg_max_iters < 1) return COFEM_ERR_INVALID_ARG;
  if (p->vec_dtype != COFEM_F32) return COFEM_ERR_UNSUPPORTED;
  if (p->resid_replace_every != 0) return COFEM_ERR_UNSUPPORTED;
  if (!(p->den_floor > 0.0) || p->t_offset < 0) return COFEM_ERR_INVALID_ARG;
  if (p->stop_rule != 0 && p->stop_rule != 1) return COFEM_ERR_INVALID_ARG;
  if (p->tasks > 1) return COFEM_ERR_UNSUPPORTED;
  if (p->mlp && p->stop_rule == 1) return COFEM_ERR_UNSUPPORTED;
  if (p->solver != 0) return p->solver == 1 ? COFEM_ERR_UNSUPPORTED : COFEM_ERR_INVALID_ARG;
  return COFEM_OK;
}

}  // namespace cofem

// ------------------------------------------------------------------ fit
namespace cofem {

namespace {
struct BStreams {
  cudaStream_t s[3] = {nullptr, nullptr, nullptr};
  ~BStreams() {
    for (auto x : s)
      if (x) cudaStreamDestroy(x);
  }
};
}  // namespace

#define BCK(x)                                      \
  do {                                              \
    if ((x) != cudaSuccess) return COFEM_ERR_CUDA;  \
  } while (0)

static cofem_status batched_graph(int n, const cofem_params* p, const BLayout& L, char* ws,
                                  double* mu, double* s, double* alpha, cudaGraphExec_t* exec) {
  const int nc = p->K + 1;
  BStreams ss;
  for (auto& x : ss.s) BCK(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
  float* X = (float*)(ws + L.o_X);
  float* R = (float*)(ws + L.o_R);
  float* P = (float*)(ws + L.o_P);
  float* Q = (float*)(ws + L.o_Q);
  const float* bv = (const float*)(ws + L.o_b);
  __nv_bfloat16* xs = (__nv_bfloat16*)(ws + L.o_xs);
  __nv_bfloat16* wsb = (__nv_bfloat16*)(ws + L.o_ws);
  float* wpart = (float*)(ws + L.o_wpart);
  double* dots = (double*)(ws + L.o_dots);
  double* part = (double*)(ws + L.o_part);
  BState* sts = (BState*)(ws + L.o_state);
  int* done = (int*)(ws + L.o_done);
  BCtl* ctl = (BCtl*)(ws + L.o_ctl);
  const BVec* pvs = (const BVec*)(ws + L.o_vec);
  const TcProb* tcp = (const TcProb*)(ws + L.o_tcp);
  const TcItem* it1 = (const TcItem*)(ws + L.o_it1);
  const TcItem* it2 = (const TcItem*)(ws + L.o_it2);

  BConf cf;
  memset(&cf, 0, sizeof(cf));
  cf.nprob = n;
  cf.nc = nc;
  cf.K = p->K;
  cf.tol = p->cg_tol;
  cf.max_iters = p->cg_max_iters;
  cf.fixed_iters = p->fixed_cg_iters;
  cf.stop_rule = p->fixed_cg_iters > 0 ? 0 : p->stop_rule;
  cf.den_floor = p->den_floor;
  cf.support_threshold = p->support_threshold;
  cf.em_iters = p->em_iters;
  cf.nch_max = L.nch_max;
  cf.split_nt = L.NT;
  cf.split_ld = L.ldx_total;
  cf.split_buf = xs;

  const bool learned = p->mlp != nullptr;
  if (learned) {
    cf.minv = (const float*)(ws + L.o_minv);
    cf.t_first = p->t_offset + 1;
  }
  float* astep = (float*)(ws + L.o_astep);
  int* err = &ctl->error;
  const int G = 16 / L.NT;
  const dim3 rg((unsigned)((L.ldw_max / 4 + 127) / 128), (L.BN / 16) * G, n);
  const dim3 vg(L.nch_max, nc, n);

  // first product (split-K partials, or W's terms directly), reduction, second
  // product of every unconverged problem's block Xin -> Y (with partial dots)
  auto apply = [&](cudaStream_t bs, const float* Xin, float* Y, double* dts) -> cofem_status {
    if (dense_tc_batched(0, L.NT, (int)L.items1.size(), it1, tcp, done, ws + L.o_packed, xs,
                         L.ldx_total, L.BN, nc, L.stages, L.tmem_cols, L.smem, wpart, nullptr,
                         nullptr, nullptr, nullptr, err, bs, L.grid, wsb, L.ldw_total) != 0)
      return COFEM_ERR_CUDA;
    if (L.any_split) {
      if (L.NT == 3)
        BCK(launch_k(breduce_kernel<3>, rg, dim3(128), 0, bs, tcp, (const int*)done, nc,
                     (const float*)wpart, wsb, L.ldw_total));
      else if (L.NT == 2)
        BCK(launch_k(breduce_kernel<2>, rg, dim3(128), 0, bs, tcp, (const int*)done, nc,
                     (const float*)wpart, wsb, L.ldw_total));
      else
        BCK(launch_k(breduce_kernel<1>, rg, dim3(128), 0, bs, tcp, (const int*)done, nc,
                     (const float*)wpart, wsb, L.ldw_total));
    }
    if (dense_tc_batched(1, L.NT, (int)L.items2.size(), it2, tcp, done, ws + L.o_packed, wsb,
                         L.ldw_total, L.BN, nc, L.stages, L.tmem_cols, L.smem, nullptr, Xin, Y,
                         alpha, dts, err, bs, L.grid) != 0)
      return COFEM_ERR_CUDA;
    return COFEM_OK;
  };
  // a WHILE loop of CG iterations (its condition set by the kernel before it)
  auto add_loop = [&](cudaStream_t outer, cudaStream_t bs, cudaGraphConditionalHandle h,
                      const BConf& c) -> cofem_status {
    cudaStreamCaptureStatus st2;
    cudaGraph_t gg = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    BCK(cudaStreamGetCaptureInfo(outer, &st2, nullptr, &gg, &deps, nullptr, &ndeps));
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    BCK(cudaGraphAddNode(&node, gg, deps, nullptr, ndeps, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    BCK(cudaStreamUpdateCaptureDependencies(outer, &node, nullptr, 1,
                                            cudaStreamSetCaptureDependencies));
    BCK(cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    cofem_status rc = apply(bs, P, Q, dots);
    if (rc != COFEM_OK) return rc;
    BCK(launch_k(bstep_kernel, dim3(n, (nc + kStepWarps - 1) / kStepWarps), dim3(32 * kStepWarps),
                 0, bs, c, pvs, sts, (const int*)done, (const double*)dots, astep));
    const dim3 cg1(L.nch_max, 1, n);           // a block per chunk, all columns
    BCK(launch_k(bupdate_kernel, cg1, dim3(256), 0, bs, c, pvs, sts, done, X, R, (const float*)P,
                 (const float*)Q, (const float*)astep, part,
                 learned ? (double*)(ws + L.o_part2) : nullptr));
    BCK(launch_k(bcond_kernel, dim3(1), dim3(256), 0, bs, c, (const int*)done));
    BCK(launch_k(bdirection_kernel, vg, dim3(256), 0, bs, c, pvs, (const BState*)sts,
                 (const int*)done, (const float*)R, P));
    cudaGraph_t tmp;
    BCK(cudaStreamEndCapture(bs, &tmp));
    return COFEM_OK;
  };

  cudaStream_t cs = ss.s[0];
  BCK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
  cudaStreamCaptureStatus status;
  cudaGraph_t g = nullptr;
  BCK(cudaStreamGetCaptureInfo(cs, &status, nullptr, &g, nullptr, nullptr, nullptr));
  cudaGraphConditionalHandle hw;
  BCK(cudaGraphConditionalHandleCreate(&hw, g, 0, cudaGraphCondAssignDefault));
  cf.while_handle = (unsigned long long)hw;
  cudaGraphConditionalHandle hw2 = 0;
  if (learned) {
    BCK(cudaGraphConditionalHandleCreate(&hw2, g, 0, cudaGraphCondAssignDefault));
    cf.while2_handle = (unsigned long long)hw2;
    // warm start X0, M^-1 (plain start at the fit's first E-step), Q = A X0,
    // preconditioned start
    launch_batched_warm_start(n, p->K, L.ld_max, (const BWarmProb*)(ws + L.o_wprob), &ctl->t,
                              cf.t_first, (const __nv_bfloat16*)p->mlp, alpha,
                              (const float*)(ws + L.o_pn2), mu, s, X, (float*)(ws + L.o_minv),
                              done, L.NT, xs, L.ldx_total, cs);
    BCK(cudaGetLastError());
    cofem_status rc = apply(cs, X, Q, nullptr);
    if (rc != COFEM_OK) return rc;
    BCK(launch_k(binit_warm_kernel, vg, dim3(256), 0, cs, cf, pvs, sts, done, (const BCtl*)ctl,
                 R, P, (const float*)Q, bv, part, (double*)(ws + L.o_part2),
                 (double*)(ws + L.o_partb)));
  } else {
    BCK(launch_k(binit_kernel, vg, dim3(256), 0, cs, cf, pvs, sts, done, (const BCtl*)ctl, X, R,
                 P, bv, part));
  }
  BCK(launch_k(bcond_kernel, dim3(1), dim3(256), 0, cs, cf, (const int*)done));
  {
    cofem_status rc = add_loop(cs, ss.s[1], hw, cf);
    if (rc != COFEM_OK) return rc;
  }
  if (learned) {
    // problems whose preconditioned solve missed the tolerance: plain CG
    // from zero (their done flags cleared, the others' set)
    BCK(launch_k(bfallback_kernel, dim3(1), dim3(256), 0, cs, cf, sts, done, ctl));
    BConf cf2 = cf;
    cf2.only_undone = 1;
    cf2.while_handle = (unsigned long long)hw2;
    BCK(launch_k(binit_kernel, vg, dim3(256), 0, cs, cf2, pvs, sts, done, (const BCtl*)ctl, X,
                 R, P, bv, part));
    BCK(launch_k(bcond_kernel, dim3(1), dim3(256), 0, cs, cf2, (const int*)done));
    cofem_status rc = add_loop(cs, ss.s[2], hw2, cf2);
    if (rc != COFEM_OK) return rc;
  }
  BCK(launch_k(bdiag_kernel, dim3(L.nch_max, 1, n), dim3(256), 0, cs, cf, pvs, sts,
               (const BCtl*)ctl, (const float*)X, mu, s, alpha));
  BCK(launch_k(bfinish_kernel, dim3(1), dim3(256), 0, cs, cf, sts, ctl,
               (int32_t*)(ws + L.o_st_it), (double*)(ws + L.o_st_rr), (int32_t*)(ws + L.o_st_cl),
               (int32_t*)(ws + L.o_st_sp)));
  cudaGraph_t graph;
  BCK(cudaStreamEndCapture(cs, &graph));
  cudaError_t e = cudaGraphInstantiate(exec, graph, 0);
  cudaGraphDestroy(graph);
  return e == cudaSuccess ? COFEM_OK : COFEM_ERR_CUDA;
}

}  // namespace cofem

using namespace cofem;

extern "C" cofem_status cofem_batched_workspace_bytes(int32_t n, const cofem_problem* problems,
                                                      const cofem_params* p, size_t* bytes) {
  cofem_status rc = bcheck(n, problems, p);
  if (rc != COFEM_OK) return rc;
  if (!bytes) return COFEM_ERR_INVALID_ARG;
  BLayout L;
  rc = blayout(n, problems, p, &L);
  if (rc != COFEM_OK) return rc;
  *bytes = L.total;
  return COFEM_OK;
}

// Autotuner of the grouped products: times both products (the real item
// tables and dictionaries of this fit, nothing converged yet) for every
// pipeline shape that fits (1 or 2 CTAs per SM, 2 .. max stages) and keeps
// the fastest.  Writes only workspace regions the fit overwrites.
static cofem_status btune(int nc, BLayout* L, char* ws, const double* alpha, cudaStream_t st) {
  const TcProb* tcp = (const TcProb*)(ws + L->o_tcp);
  const TcItem* it1 = (const TcItem*)(ws + L->o_it1);
  const TcItem* it2 = (const TcItem*)(ws + L->o_it2);
  const int* done = (const int*)(ws + L->o_done);
  float* P = (float*)(ws + L->o_P);
  float* Q = (float*)(ws + L->o_Q);
  cudaEvent_t e0, e1;
  BCK(cudaEventCreate(&e0));
  BCK(cudaEventCreate(&e1));
  float best = 1e30f;
  BLayout keep = *L;
  int bst = L->stages, bgrid = L->grid;
  size_t bsmem = L->smem;
  cofem_status rc = COFEM_OK;
  for (int cps = 1; cps <= 2 && rc == COFEM_OK; ++cps) {
    const DenseTcPlan full = dense_tc_plan(2048, 8192, nc, L->NT, num_sms(), cps, 0);
    for (int stg = 2; stg <= full.stages && rc == COFEM_OK; ++stg) {
      const DenseTcPlan q = dense_tc_plan(2048, 8192, nc, L->NT, num_sms(), cps, stg);
      auto run = [&]() {
        int r = dense_tc_batched(0, L->NT, (int)L->items1.size(), it1, tcp, done,
                                 ws + L->o_packed, (const __nv_bfloat16*)(ws + L->o_xs),
                                 L->ldx_total, L->BN, nc, q.stages, q.tmem_cols, q.smem,
                                 (float*)(ws + L->o_wpart), nullptr, nullptr, nullptr, nullptr,
                                 nullptr, st, q.grid, (__nv_bfloat16*)(ws + L->o_ws),
                                 L->ldw_total);
        if (r == 0)
          r = dense_tc_batched(1, L->NT, (int)L->items2.size(), it2, tcp, done,
                               ws + L->o_packed, (const __nv_bfloat16*)(ws + L->o_ws),
                               L->ldw_total, L->BN, nc, q.stages, q.tmem_cols, q.smem, nullptr,
                               P, Q, alpha, (double*)(ws + L->o_dots), nullptr, st, q.grid);
        return r;
      };
      if (run() != 0) { rc = COFEM_ERR_CUDA; break; }
      cudaEventRecord(e0, st);
      for (int r = 0; r < 2 && rc == COFEM_OK; ++r)
        if (run() != 0) rc = COFEM_ERR_CUDA;
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) rc = COFEM_ERR_CUDA;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rc == COFEM_OK && ms < best) {
        best = ms;
        bst = q.stages;
        bgrid = q.grid;
        bsmem = q.smem;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != COFEM_OK) {
    *L = keep;
    return rc;
  }
  L->stages = bst;
  L->grid = bgrid;
  L->smem = bsmem;
  return COFEM_OK;
}

extern "C" cofem_status cofem_fit_batched(int32_t n, const cofem_problem* problems,
                                          const cofem_params* p, void* workspace_dev,
                                          size_t workspace_bytes, double* mu_dev, double* s_dev,
                                          double* alpha_dev, cofem_stats* stats, void* stream) {
  cofem_status rc = bcheck(n, problems, p);
  if (rc != COFEM_OK) return rc;
  if (!workspace_dev || !mu_dev || !s_dev || !alpha_dev || ((uintptr_t)workspace_dev & 255))
    return COFEM_ERR_INVALID_ARG;
  BLayout L;
  rc = blayout(n, problems, p, &L);
  if (rc != COFEM_OK) return rc;
  if (workspace_bytes < L.total) return COFEM_ERR_WORKSPACE;
  char* ws = (char*)workspace_dev;
  cudaStream_t st = (cudaStream_t)stream;
  // zero all but the packed dictionaries (overwritten below)
  BCK(cudaMemsetAsync(ws + L.o_X, 0, L.total - L.o_X, st));
  BCK(cudaMemcpyAsync(ws + L.o_vec, L.vec.data(), n * sizeof(BVec), cudaMemcpyHostToDevice, st));
  BCK(cudaMemcpyAsync(ws + L.o_tcp, L.tcp.data(), n * sizeof(TcProb), cudaMemcpyHostToDevice, st));
  BCK(cudaMemcpyAsync(ws + L.o_it1, L.items1.data(), L.items1.size() * sizeof(TcItem),
                      cudaMemcpyHostToDevice, st));
  BCK(cudaMemcpyAsync(ws + L.o_it2, L.items2.data(), L.items2.size() * sizeof(TcItem),
                      cudaMemcpyHostToDevice, st));
  if (p->mlp) {
    BCK(cudaMemcpyAsync(ws + L.o_wprob, L.wprob.data(), n * sizeof(BWarmProb),
                        cudaMemcpyHostToDevice, st));
    // ||phi_d||^2 of every problem's dictionary (the network's features)
    for (int i = 0; i < n; ++i)
      launch_col_norms_bf16(problems[i].phi_dev, problems[i].N, problems[i].D, problems[i].ld,
                            (float*)(ws + L.o_pn2) + L.vec[i].aoff, st);
    BCK(cudaGetLastError());
  }
  BCK(launch_k(bctl_init_kernel, dim3(1), dim3(1), 0, st, (BCtl*)(ws + L.o_ctl),
               (long long)(p->t_offset + 1)));
  if (p->t_offset == 0)
    BCK(launch_k(bfill_kernel, dim3(1024), dim3(256), 0, st, alpha_dev, L.dtot, p->alpha_init));
  for (int i = 0; i < n; ++i) {
    const cofem_problem& q = problems[i];
    // packed dictionary, and b = beta Phi^T y (once per fit)
    dense_pack_bf16(q.phi_dev, q.N, q.D, q.ld, ws + L.o_packed + L.tcp[i].poff * 2, st);
    DenseDesc dd = {};
    dd.N = q.N;
    dd.D = q.D;
    dd.ld = q.ld;
    dd.dtype = COFEM_BF16;
    dd.phi = q.phi_dev;
    dense_simt_adjoint<__nv_bfloat16, float>(dd, (const float*)q.y_dev, q.N, 1,
                                             (float*)(ws + L.o_b) + L.vec[i].aoff,
                                             L.vec[i].ld, q.beta, nullptr, nullptr, nullptr,
                                             nullptr, ws + L.o_simt, st);
  }
  BCK(cudaGetLastError());
  if (p->em_iters > 0) {
    rc = btune(p->K + 1, &L, ws, alpha_dev, st);
    if (rc != COFEM_OK) return rc;
    cudaGraphExec_t exec = nullptr;
    rc = batched_graph(n, p, L, ws, mu_dev, s_dev, alpha_dev, &exec);
    if (rc != COFEM_OK) {
      if (exec) cudaGraphExecDestroy(exec);
      return rc;
    }
    for (int t = 0; t < p->em_iters; ++t)
      if (cudaGraphLaunch(exec, st) != cudaSuccess) {
        cudaGraphExecDestroy(exec);
        return COFEM_ERR_CUDA;
      }
    const cudaError_t e = cudaStreamSynchronize(st);
    cudaGraphExecDestroy(exec);
    if (e != cudaSuccess) return COFEM_ERR_CUDA;
  } else {
    BCK(cudaStreamSynchronize(st));
  }
  BCtl hctl;
  BCK(cudaMemcpy(&hctl, ws + L.o_ctl, sizeof(hctl), cudaMemcpyDeviceToHost));
  set_last_fit_fallbacks(p->mlp ? hctl.fallbacks : 0);
  if (stats && p->em_iters > 0) {
    const size_t m = (size_t)n * p->em_iters;
    if (stats->cg_iters) BCK(cudaMemcpy(stats->cg_iters, ws + L.o_st_it, 4 * m, cudaMemcpyDeviceToHost));
    if (stats->relres) BCK(cudaMemcpy(stats->relres, ws + L.o_st_rr, 8 * m, cudaMemcpyDeviceToHost));
    if (stats->clamps) BCK(cudaMemcpy(stats->clamps, ws + L.o_st_cl, 4 * m, cudaMemcpyDeviceToHost));
    if (stats->support) BCK(cudaMemcpy(stats->support, ws + L.o_st_sp, 4 * m, cudaMemcpyDeviceToHost));
  }
  return hctl.error ? (cofem_status)hctl.error : COFEM_OK;
}
