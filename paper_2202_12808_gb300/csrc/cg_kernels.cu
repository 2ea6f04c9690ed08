// Column-wise conjugate gradients on A X = B (Sec. 3.2) and the fused
// probe / diagonal-estimate / M-step kernel (Sec. 3.1, Eq. (diag-estimate),
// Eq. (mstep), Algorithm 1).
//
// Vectors are blocks of `ncols` columns of leading dimension `ld` (a
// multiple of 64); entries d in [D, ld) are kept at zero, so the streaming
// kernels run over [0, ld) with 16-byte vector accesses.  Column 0 is the
// mean system, columns 1..K the probes.  Every per-column dot product is
// accumulated in double, reduced per block by warp shuffles, then summed
// over blocks in a fixed order by the last block to arrive (deterministic).
#include <cstring>

#include "kernels.cuh"

namespace cofem {

constexpr int kUpdChunks = 4;     // 16-byte chunks per thread and pass in the CG update

template <typename V> struct Vec16;
template <> struct Vec16<float> { using T = float4; static constexpr int W = 4; };
template <> struct Vec16<double> { using T = double2; static constexpr int W = 2; };

template <typename V>
__device__ __forceinline__ void vload(const V* p, V (&v)[16 / sizeof(V)]) {
  using T = typename Vec16<V>::T;
  T t = *reinterpret_cast<const T*>(p);
  if constexpr (sizeof(V) == 4) { v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w; }
  else { v[0] = t.x; v[1] = t.y; }
}
template <typename V>
__device__ __forceinline__ void vstore(V* p, const V (&v)[16 / sizeof(V)]) {
  using T = typename Vec16<V>::T;
  T t;
  if constexpr (sizeof(V) == 4) { t.x = v[0]; t.y = v[1]; t.z = v[2]; t.w = v[3]; }
  else { t.x = v[0]; t.y = v[1]; }
  *reinterpret_cast<T*>(p) = t;
}

__device__ __forceinline__ void set_cond(unsigned long long h, unsigned v) {
  if (h) cudaGraphSetConditional((cudaGraphConditionalHandle)h, v);
}

// BF16 terms of one FP32 value (each the rounding of the remainder).
__device__ __forceinline__ void write_split(const CgConf& cf, int j, int64_t d, float v) {
  __nv_bfloat16* buf = reinterpret_cast<__nv_bfloat16*>(cf.split_buf);
  float r = v;
  for (int t = 0; t < cf.split_nt; ++t) {
    const __nv_bfloat16 o = __float2bfloat16_rn(r);
    r -= __bfloat162float(o);
    buf[(int64_t)split_row(j, t, cf.split_nt) * cf.ld + d] = o;
  }
}
__device__ __forceinline__ void write_split(const CgConf& cf, int j, int64_t d, double v) {}

// Same for 4 consecutive values (d a multiple of 4): one 8-byte store per term.
__device__ __forceinline__ void write_split4(const CgConf& cf, int j, int64_t d,
                                             const float (&v)[4]) {
  __nv_bfloat16* buf = reinterpret_cast<__nv_bfloat16*>(cf.split_buf);
  float r[4] = {v[0], v[1], v[2], v[3]};
  for (int t = 0; t < cf.split_nt; ++t) {
    __nv_bfloat16 o[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      o[i] = __float2bfloat16_rn(r[i]);
      r[i] -= __bfloat162float(o[i]);
    }
    __nv_bfloat162 lo = __halves2bfloat162(o[0], o[1]), hi = __halves2bfloat162(o[2], o[3]);
    uint2 pk;
    pk.x = *reinterpret_cast<uint32_t*>(&lo);
    pk.y = *reinterpret_cast<uint32_t*>(&hi);
    *reinterpret_cast<uint2*>(buf + (int64_t)split_row(j, t, cf.split_nt) * cf.ld + d) = pk;
  }
}
__device__ __forceinline__ void write_split4(const CgConf&, int, int64_t, const double (&)[2]) {}

// out[j] = sum over i < nparts of part[i * kMaxCols + j], j < ncols
// (blockDim >= ncols): thread j loads its column's partials eight at a time
// and adds them as a fixed binary tree (deterministic, few dependent FP64
// additions: FP64 latency is long on this GPU).
__device__ __forceinline__ void column_sums(const double* part, int nparts, int ncols,
                                            double* out) {
  const int j = threadIdx.x;
  if (j < ncols) {
    double acc = 0.0;
    for (int i0 = 0; i0 < nparts; i0 += 8) {
      double v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        v[u] = i0 + u < nparts ? part[(int64_t)(i0 + u) * kMaxCols + j] : 0.0;
      acc += ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]));
    }
    out[j] = acc;
  }
}

// Closes one CG iteration (called by the last block, all threads; blockDim
// >= ncols): the residual norms rho_new are final.  Stop test, direction
// coefficients b_j (thread j), the residual total by the first warp.
__device__ void cg_finalize(const CgConf& cf, CgCtl* ctl, CgScalars* sc) {
  __shared__ double tot_sh;
  __syncthreads();
  const int j = threadIdx.x;
  if (j < 32) {
    double t = 0.0;
    for (int c = j; c < cf.ncols; c += 32) t += cf.minv ? sc->rr_new[c] : sc->rho_new[c];
    t = warp_sum(t);
    if (j == 0) tot_sh = t;
  }
  int live = 0;
  if (j < cf.ncols) {
    const double r0 = sc->rho[j], r1 = sc->rho_new[j];
    if (cf.stop_rule == 1) {
      // per-column rule: column j is frozen once ||r_j|| < tol ||b_j||; a
      // frozen column keeps rho_j = 0, so a_j = b_j = 0 from then on
      live = r0 > 0.0 && !(sqrt(r1) < cf.tol * sqrt(sc->bn2[j]));
      sc->b[j] = live ? r1 / r0 : 0.0;
      sc->rho[j] = live ? r1 : 0.0;
    } else {
      sc->b[j] = r0 > 0.0 ? r1 / r0 : 0.0;
      sc->rho[j] = r1;
    }
  }
  const int nlive = __syncthreads_count(live);
  if (j == 0) {
    const double relres = sqrt(tot_sh) / sqrt(ctl->normB2);
    ctl->relres = relres;
    const int it = ctl->iter;
    int done;
    if (cf.fixed_iters > 0) done = it >= cf.fixed_iters;
    else if (cf.stop_rule == 1) done = nlive == 0 || it >= cf.max_iters;
    else done = (relres < cf.tol) || (it >= cf.max_iters);
    if (!isfinite(relres)) { raise_error(ctl, COFEM_ERR_NONFINITE); done = 1; }
    // a block of this launch that gave up its wait has ended the loops: do
    // not restart them (a timeout raised after this read still ends them at
    // the next update launch, which checks the error word first)
    if (*(volatile int*)&ctl->error == (int)COFEM_ERR_TIMEOUT) done = 1;
    ctl->done = done;
    ctl->run = !done;
    set_cond(cf.while_handle, done ? 0u : 1u);
    set_cond(cf.inner_handle, done ? 0u : 1u);
    if (done && cf.fallback_handle)
      set_cond(cf.fallback_handle, (cf.fixed_iters == 0 && !(relres < cf.tol)) ? 1u : 0u);
  }
}

// ---------------------------------------------------------------- probes

template <typename V>
__global__ void probe_fill_kernel(uint64_t key, int K, int64_t D, V* out, int64_t ld) {
  pdl_wait();
  pdl_trigger();
  const int k = blockIdx.y;
  for (int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; d < ld;
       d += (int64_t)gridDim.x * blockDim.x) {
    V v = V(0);
    if (d < D) {
      const uint64_t h = probe_word(key, d, k >> 6);
      v = ((h >> (k & 63)) & 1ull) ? V(-1) : V(1);
    }
    out[(int64_t)k * ld + d] = v;
  }
}

// ------------------------------------------------------------- CG start
// X = 0, R = P = B = [b_1..b_T | p_1..p_K] (b_t = beta Phi^T y_t, T tasks);
// rho_j = ||B_j||^2 (= D for a probe).
template <typename V>
__global__ void cg_init_kernel(CgConf cf, CgCtl* ctl, CgScalars* sc, V* X, V* R, V* P,
                               const V* bvec, double* part) {
  pdl_wait();
  pdl_trigger();
  __shared__ double sh[32];
  const int j = blockIdx.y;
  const uint64_t key = probe_key(cf.seed, ctl->t);
  typename AccOf<V>::T acc;
  V* x = X + (int64_t)j * cf.ld;
  V* r = R + (int64_t)j * cf.ld;
  V* p = P + (int64_t)j * cf.ld;
  for (int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; d < cf.ld;
       d += (int64_t)gridDim.x * blockDim.x) {
    V v = V(0);
    if (d < cf.D) {
      if (j < cf.T) {
        v = bvec[(int64_t)j * cf.ld + d];
        acc.add_prod(v, v);
      } else {
        const int k = j - cf.T;
        const uint64_t h = probe_word(key, d, k >> 6);
        v = ((h >> (k & 63)) & 1ull) ? V(-1) : V(1);
      }
    }
    x[d] = V(0);
    r[d] = v;
    p[d] = v;
    if (cf.split_nt > 0) write_split(cf, j, d, v);
  }
  if (j < cf.T) {
    const double s = block_sum(acc, sh);
    if (threadIdx.x == 0) part[(int64_t)blockIdx.x * kMaxCols + j] = s;
  }
  if (arrive_last(&ctl->counter[0])) {
    // ||b_t||^2 per task (thread t, blocks in order); a probe has ||p||^2 = D
    if (threadIdx.x < cf.ncols) {
      const int jj = threadIdx.x;
      double b2 = (double)cf.D;
      if (jj < cf.T) {
        b2 = 0.0;
        for (int i = 0; i < (int)gridDim.x; ++i) b2 += part[(int64_t)i * kMaxCols + jj];
      }
      sc->rho[jj] = b2;
      sc->bn2[jj] = b2;
      // per-column rule: every column starts at ||r_j|| / ||b_j|| = 1, so
      // the joint start test below covers it; a zero task column (b_t = 0)
      // is solved by x = 0 and frozen at once
      if (cf.stop_rule == 1 && !(b2 > 0.0)) sc->rho[jj] = 0.0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double b2 = 0.0;
      for (int t = 0; t < cf.T; ++t) b2 += sc->bn2[t];
      const double n2 = b2 + (double)cf.K * (double)cf.D;
      ctl->normB2 = n2;
      ctl->relres = n2 > 0.0 ? 1.0 : 0.0;
      if (cf.fallback_init) {
        ctl->extra_iters = ctl->iter;
        ctl->fallbacks += 1;
      }
      ctl->iter = 0;
      ctl->replace = 0;
      ctl->clamps = 0;
      ctl->support = 0;
      int done = 0;
      if (!(n2 > 0.0)) done = 1;                       // B = 0: X = 0 solves it
      else if (cf.fixed_iters == 0 && 1.0 < cf.tol) done = 1;
      if (!isfinite(n2)) { raise_error(ctl, COFEM_ERR_NONFINITE); done = 1; }
      ctl->done = done;
      ctl->run = 0;
      set_cond(cf.while_handle, done ? 0u : 1u);
      ctl->counter[0] = 0;
    }
  }
}

// ------------------------------------------ preconditioned start from X0
// Q = A X0 given; R = B - Q, Z = M^-1 R, P = Z; rho_j = r_j^T z_j; the stop
// test uses ||R||_F / ||B||_F.  ctl->iter = 0.
template <typename V>
__global__ void cg_init_warm_kernel(CgConf cf, CgCtl* ctl, CgScalars* sc, const V* X, V* R,
                                    V* P, const V* Q, const V* bvec, double* pz, double* pr,
                                    double* pb) {
  pdl_wait();
  pdl_trigger();
  __shared__ double sh[32];
  const int j = blockIdx.y;
  const uint64_t key = probe_key(cf.seed, ctl->t);
  typename AccOf<V>::T az, ar, ab;
  V* r = R + (int64_t)j * cf.ld;
  V* p = P + (int64_t)j * cf.ld;
  const V* q = Q + (int64_t)j * cf.ld;
  for (int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; d < cf.ld;
       d += (int64_t)gridDim.x * blockDim.x) {
    V bv = V(0);
    if (d < cf.D) {
      if (j == 0) bv = bvec[d];
      else {
        const int k = j - 1;
        const uint64_t h = probe_word(key, d, k >> 6);
        bv = ((h >> (k & 63)) & 1ull) ? V(-1) : V(1);
      }
    }
    const V rv = d < cf.D ? bv - q[d] : V(0);
    const V zv = rv * (V)cf.minv[d];
    r[d] = rv;
    p[d] = zv;
    if (cf.split_nt > 0) write_split(cf, j, d, zv);
    az.add_prod(rv, zv);
    ar.add_prod(rv, rv);
    if (j == 0) ab.add_prod(bv, bv);
  }
  const double sz = block_sum(az, sh);
  const double sr = block_sum(ar, sh);
  const double sb = block_sum(ab, sh);
  if (threadIdx.x == 0) {
    pz[(int64_t)blockIdx.x * kMaxCols + j] = sz;
    pr[(int64_t)blockIdx.x * kMaxCols + j] = sr;
    if (j == 0) pb[blockIdx.x] = sb;
  }
  if (arrive_last(&ctl->counter[0])) {
    column_sums(pz, gridDim.x, cf.ncols, sc->rho);
    column_sums(pr, gridDim.x, cf.ncols, sc->rr_new);
    __syncthreads();
    if (threadIdx.x == 0) {
      double b2 = 0.0, r2 = 0.0;
      for (int i = 0; i < (int)gridDim.x; ++i) b2 += pb[i];
      for (int jj = 0; jj < cf.ncols; ++jj) r2 += sc->rr_new[jj];
      const double n2 = b2 + (double)cf.K * (double)cf.D;
      ctl->normB2 = n2;
      const double relres = n2 > 0.0 ? sqrt(r2) / sqrt(n2) : 0.0;
      ctl->relres = relres;
      ctl->iter = 0;
      ctl->extra_iters = 0;
      ctl->replace = 0;
      ctl->clamps = 0;
      ctl->support = 0;
      int done = !(n2 > 0.0) || relres < cf.tol;
      if (!isfinite(n2) || !isfinite(relres)) { raise_error(ctl, COFEM_ERR_NONFINITE); done = 1; }
      ctl->done = done;
      set_cond(cf.while_handle, done ? 0u : 1u);
      set_cond(cf.fallback_handle, 0u);
      ctl->counter[0] = 0;
    }
  }
}

// Waits (thread 0) until *gen differs from g0; false after limit_ns.
__device__ __forceinline__ bool wait_gen(const unsigned int* gen, unsigned int g0,
                                         uint64_t limit_ns) {
  const volatile unsigned int* g = gen;
  uint64_t t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  while (*g == g0) {
    __nanosleep(32);
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 > limit_ns) return false;
  }
  return true;
}

constexpr uint64_t kGenWaitNs = 2000000000ull;

// --------------------------------------- x += a p, r -= a q, rho_new = r^T r
// a_j = rho_j / gamma_j with gamma_j the fixed-order sum of the operator's
// per-block partials of p_j^T A p_j (every block computes the same value).
//
// DIR: the same launch also applies the direction update p = r + b p (or
// p = M^-1 r + b p): the last block closes the iteration as usual (b_j, the
// stop test, ctl->run), then releases the other blocks, which wait for it
// (bounded) and update p from the r and p values they still hold.  The
// host launches this form only when the whole grid fits on the GPU at once
// (occupancy), so that every block the wait depends on is resident.
template <typename V, bool DIR>
__global__ void cg_update_kernel(CgConf cf, CgCtl* ctl, CgScalars* sc, V* X, V* R,
                                 V* P, const V* Q, const double* gparts, double* part,
                                 double* part2) {
  pdl_wait();
  pdl_trigger();
  __shared__ double sh[32];
  __shared__ double a_sh;
  __shared__ int go_sh;
  // second copy of an unrolled loop body: the first copy may have ended the
  // solve or handed over to the residual replacement
  if (cf.gate_run && *(volatile int*)&ctl->run == 0) return;
  unsigned int g0 = 0;
  if (DIR) {
    if (*(volatile int*)&ctl->error == (int)COFEM_ERR_TIMEOUT) {
      // an earlier wait gave up: end the solve instead of iterating on
      if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
        ctl->done = 1;
        ctl->run = 0;
        set_cond(cf.while_handle, 0u);
        set_cond(cf.inner_handle, 0u);
      }
      return;
    }
    // read before this block arrives, so before the last block can bump it
    if (threadIdx.x == 0) g0 = *(volatile unsigned int*)&ctl->dir_gen;
  }
  constexpr int W = 16 / sizeof(V);
  // chunks of W values per thread and pass: the fused form keeps the last
  // pass's r and p in registers for the direction update; the plain form
  // takes fewer per pass (fewer registers, more resident blocks)
  constexpr int U = DIR ? kUpdChunks : 2;
  const int j = blockIdx.y;
  V* x = X + (int64_t)j * cf.ld;
  V* r = R + (int64_t)j * cf.ld;
  const V* p = P + (int64_t)j * cf.ld;
  const V* q = Q + (int64_t)j * cf.ld;
  // chunk u of a pass starts at base + u * ts; the first pass's loads are
  // issued before a_j is known, so that they overlap the reduction of the
  // operator's partials below, and every pass loads before it stores
  const int64_t d0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) * W;
  const int64_t ts = (int64_t)gridDim.x * blockDim.x * W;
  V xv[U][W], rv[U][W], pv[U][W], qv[U][W];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int64_t d = d0 + u * ts;
    if (d < cf.ld) {
      vload(x + d, xv[u]); vload(r + d, rv[u]); vload(p + d, pv[u]); vload(q + d, qv[u]);
    }
  }
  if (threadIdx.x < 32) {
    // gamma_j = p_j^T A p_j: the operator's partials, eight per lane as a
    // fixed tree, then a butterfly
    double g = 0.0;
    for (int i0 = threadIdx.x; i0 < cf.gamma_parts; i0 += 256) {
      double v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int i = i0 + 32 * u;
        v[u] = i < cf.gamma_parts ? gparts[(int64_t)i * kMaxCols + j] : 0.0;
      }
      g += ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]));
    }
    g = warp_sum(g);
    if (threadIdx.x == 0) {
      const double rho = sc->rho[j];
      double a = 0.0;
      if (rho > 0.0) {
        if (!(g > 0.0)) {
          if (blockIdx.x == 0)
            raise_error(ctl, isfinite(g) ? COFEM_ERR_BREAKDOWN : COFEM_ERR_NONFINITE);
        } else {
          a = rho / g;
        }
      }
      a_sh = a;
      if (blockIdx.x == 0) { sc->gamma[j] = g; sc->a[j] = a; }
    }
  }
  __syncthreads();
  const V a = (V)a_sh;
  typename AccOf<V>::T acc, accz;
  for (int64_t base = d0; base < cf.ld; base += U * ts) {
    if (base != d0) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t d = base + u * ts;
        if (d < cf.ld) {
          vload(x + d, xv[u]); vload(r + d, rv[u]); vload(p + d, pv[u]); vload(q + d, qv[u]);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t d = base + u * ts;
      if (d < cf.ld) {
#pragma unroll
        for (int i = 0; i < W; ++i) {
          xv[u][i] = fma(a, pv[u][i], xv[u][i]);
          rv[u][i] = fma(-a, qv[u][i], rv[u][i]);
          acc.add_prod(rv[u][i], rv[u][i]);
          if (cf.minv) accz.add_prod(rv[u][i] * (V)cf.minv[d + i], rv[u][i]);
        }
        vstore(x + d, xv[u]); vstore(r + d, rv[u]);
      }
    }
  }
  const double s = block_sum(acc, sh);
  if (threadIdx.x == 0) part[(int64_t)blockIdx.x * kMaxCols + j] = s;
  if (cf.minv) {
    const double sz = block_sum(accz, sh);
    if (threadIdx.x == 0) part2[(int64_t)blockIdx.x * kMaxCols + j] = sz;
  }
  const bool last = arrive_last(&ctl->counter[1]);
  if (last) {
    if (cf.minv) {
      column_sums(part, gridDim.x, cf.ncols, sc->rr_new);
      column_sums(part2, gridDim.x, cf.ncols, sc->rho_new);
    } else {
      column_sums(part, gridDim.x, cf.ncols, sc->rho_new);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      ctl->iter += 1;
      ctl->counter[1] = 0;
      const int rep = cf.replace_every > 0 && (ctl->iter % cf.replace_every) == 0;
      ctl->replace = rep;
      set_cond(cf.if_handle, rep ? 1u : 0u);
      if (rep) {
        // the true residual and the stop test come first: no direction update
        // yet, and the inner loop (if any) hands over to the replacement
        ctl->run = 0;
        set_cond(cf.inner_handle, 0u);
      }
    }
    __syncthreads();
    if (!ctl->replace) cg_finalize(cf, ctl, sc);
  }
  if constexpr (DIR) {
    __syncthreads();
    if (threadIdx.x == 0) {
      int go = 1;
      if (last) {
        // b_j, rho_j and ctl->run are written (this block, before the barrier)
        __threadfence();
        atomicAdd(&ctl->dir_gen, 1u);
      } else {
        go = wait_gen(&ctl->dir_gen, g0, cf.gen_wait_ns ? cf.gen_wait_ns : kGenWaitNs);
        if (!go) {
          raise_error(ctl, COFEM_ERR_TIMEOUT);
          set_cond(cf.while_handle, 0u);
          set_cond(cf.inner_handle, 0u);
        }
        __threadfence();
      }
      go_sh = go && *(volatile int*)&ctl->run;
    }
    __syncthreads();
    if (!go_sh) return;
    const V b = (V)__ldcg(&sc->b[j]);
    V* pw = P + (int64_t)j * cf.ld;
    for (int64_t base = d0; base < cf.ld; base += U * ts) {
      // the registers hold r (updated) and p of the loop's last pass
      const bool held = base + U * ts >= cf.ld;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t d = base + u * ts;
        if (d < cf.ld) {
          V rr[W], pp[W];
          if (held) {
#pragma unroll
            for (int i = 0; i < W; ++i) { rr[i] = rv[u][i]; pp[i] = pv[u][i]; }
          } else {
            vload(r + d, rr);
            vload(pw + d, pp);
          }
          if (cf.minv) {
#pragma unroll
            for (int i = 0; i < W; ++i) rr[i] = rr[i] * (V)cf.minv[d + i];
          }
#pragma unroll
          for (int i = 0; i < W; ++i) pp[i] = fma(b, pp[i], rr[i]);
          vstore(pw + d, pp);
          if (cf.split_nt > 0) write_split4(cf, j, d, pp);
        }
      }
    }
  }
}

// ------------------------------ residual replacement: r = B - Q (Q = A x)
template <typename V>
__global__ void cg_true_resid_kernel(CgConf cf, CgCtl* ctl, CgScalars* sc, V* R,
                                     const V* Q, const V* bvec, double* part, double* part2) {
  pdl_wait();
  pdl_trigger();
  __shared__ double sh[32];
  if (!ctl->replace) return;
  const int j = blockIdx.y;
  const uint64_t key = probe_key(cf.seed, ctl->t);
  V* r = R + (int64_t)j * cf.ld;
  const V* q = Q + (int64_t)j * cf.ld;
  typename AccOf<V>::T acc, accz;
  for (int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; d < cf.D;
       d += (int64_t)gridDim.x * blockDim.x) {
    V bv;
    if (j < cf.T) bv = bvec[(int64_t)j * cf.ld + d];
    else {
      const int k = j - cf.T;
      const uint64_t h = probe_word(key, d, k >> 6);
      bv = ((h >> (k & 63)) & 1ull) ? V(-1) : V(1);
    }
    const V rv = bv - q[d];
    r[d] = rv;
    acc.add_prod(rv, rv);
    if (cf.minv) accz.add_prod(rv * (V)cf.minv[d], rv);
  }
  const double s = block_sum(acc, sh);
  if (threadIdx.x == 0) part[(int64_t)blockIdx.x * kMaxCols + j] = s;
  if (cf.minv) {
    const double sz = block_sum(accz, sh);
    if (threadIdx.x == 0) part2[(int64_t)blockIdx.x * kMaxCols + j] = sz;
  }
  if (arrive_last(&ctl->counter[2])) {
    if (cf.minv) {
      column_sums(part, gridDim.x, cf.ncols, sc->rr_new);
      column_sums(part2, gridDim.x, cf.ncols, sc->rho_new);
    } else {
      column_sums(part, gridDim.x, cf.ncols, sc->rho_new);
    }
    if (threadIdx.x == 0) { ctl->counter[2] = 0; ctl->replace = 0; }
    cg_finalize(cf, ctl, sc);
  }
}

// ------------------------------------------------------ p = r + b p
template <typename V>
__global__ void cg_direction_kernel(CgConf cf, const CgCtl* ctl, const CgScalars* sc,
                                    const V* R, V* P) {
  pdl_wait();
  pdl_trigger();
  constexpr int W = 16 / sizeof(V);
  if (!ctl->run) return;
  const int j = blockIdx.y;
  const V b = (V)sc->b[j];
  const V* r = R + (int64_t)j * cf.ld;
  V* p = P + (int64_t)j * cf.ld;
  for (int64_t d = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) * W; d < cf.ld;
       d += (int64_t)gridDim.x * blockDim.x * W) {
    V rv[W], pv[W];
    vload(r + d, rv); vload(p + d, pv);
    if (cf.minv) {
#pragma unroll
      for (int i = 0; i < W; ++i) rv[i] = rv[i] * (V)cf.minv[d + i];
    }
#pragma unroll
    for (int i = 0; i < W; ++i) pv[i] = fma(b, pv[i], rv[i]);
    vstore(p + d, pv);
    if (cf.split_nt > 0) write_split4(cf, j, d, pv);
  }
}

// ------------------------------------ diagonal estimate + M-step (fused)
// mu_d = x_0d, s_d = (1/K) sum_k p_kd x_kd, alpha_d = 1/max(mu^2 + s, floor).
// In fit mode (ctl != nullptr) the key comes from ctl->t, the counters go to
// ctl and the last block records the E-step's statistics and advances t.
template <typename V>
__global__ void diag_mstep_kernel(CgConf cf, CgCtl* ctl, uint64_t key_in, const V* X,
                                  double* mu, double* s, double* alpha, int32_t* counts,
                                  int32_t* st_iters, double* st_relres, int32_t* st_clamps,
                                  int32_t* st_support) {
  pdl_wait();
  pdl_trigger();
  const uint64_t key = ctl ? probe_key(cf.seed, ctl->t) : key_in;
  const int K = cf.K;
  const double inv_k = 1.0 / (double)K;
  int clamps = 0, support = 0, bad = 0;
  for (int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; d < cf.D;
       d += (int64_t)gridDim.x * blockDim.x) {
    // mu_t = column t of X; the M-step uses the mean of mu_t^2 over the
    // tasks (one task: mu^2)
    double m = (double)X[d], m2 = m * m;
    for (int t = 1; t < cf.T; ++t) {
      const double mt = (double)X[(int64_t)t * cf.ld + d];
      m2 += mt * mt;
      mu[(int64_t)t * cf.D + d] = mt;
      if (!isfinite(mt)) bad = 1;
    }
    if (cf.T > 1) m2 /= (double)cf.T;
    typename AccOf<V>::T acc;          // sum_k p_kd x_kd (compensated for FP32 X)
    for (int w = 0; w * 64 < K; ++w) {
      const uint64_t h = probe_word(key, d, w);
      const int kend = min(K, (w + 1) * 64);
      for (int k = w * 64; k < kend; ++k) {
        const V xv = X[(int64_t)(k + cf.T) * cf.ld + d];
        acc.add(((h >> (k & 63)) & 1ull) ? -xv : xv);
      }
    }
    // s_d = sum / K and alpha_d = 1 / max(mu^2 + s, floor); FP64 runs at a
    // small fraction of the FP32 rate on this GPU, so the per-coordinate FP64
    // work is kept short: a multiplication by 1/K (exact for K a power of
    // two, else within an ulp of the quotient) and the correctly rounded
    // reciprocal intrinsic (the same IEEE value as 1.0 / x)
    const double sd = acc.value() * inv_k;
    const double den = m2 + sd;
    if (den < cf.den_floor) ++clamps;
    const double al = __drcp_rn(fmax(den, cf.den_floor));
    if (!isfinite(m) || !isfinite(sd)) bad = 1;
    if (al < cf.support_threshold) ++support;
    mu[d] = m;
    s[d] = sd;
    alpha[d] = al;
    if (cf.alpha32) cf.alpha32[d] = (float)al;
  }
  // the counters: integer warp sums, one atomic per warp
  const int cs = __reduce_add_sync(0xffffffffu, clamps);
  const int ss = __reduce_add_sync(0xffffffffu, support);
  const int bs = __reduce_or_sync(0xffffffffu, bad);
  int* cc = ctl ? &ctl->clamps : counts;
  int* sp = ctl ? &ctl->support : (counts ? counts + 1 : nullptr);
  if ((threadIdx.x & 31) == 0) {
    if (cc && cs > 0) atomicAdd(cc, cs);
    if (sp && ss > 0) atomicAdd(sp, ss);
    if (bs && ctl) raise_error(ctl, COFEM_ERR_NONFINITE);
  }
  if (ctl && arrive_last(&ctl->counter[3])) {
    if (threadIdx.x == 0) {
      const int e = ctl->em_index;
      if (e < cf.em_iters) {
        st_iters[e] = ctl->iter + ctl->extra_iters;
        st_relres[e] = ctl->relres;
        st_clamps[e] = ctl->clamps;
        st_support[e] = ctl->support;
        if (cf.st_end_ns) {
          unsigned long long now;
          asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
          cf.st_end_ns[e] = (long long)(now - ctl->start_ns);
        }
      }
      ctl->em_index = e + 1;
      ctl->t += 1;
      ctl->counter[3] = 0;
    }
  }
}

// --------------------------------------------------- small helpers

template <typename V>
__global__ void scale_kernel(V* x, int64_t n, double beta) {
  pdl_wait();
  pdl_trigger();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] = (V)((double)x[i] * beta);
}

// ------------------------------------------------------------ launchers

static int vec_blocks(int64_t ld, int W, int ncols, int sms) {
  int64_t need = (ld / W + 255) / 256;
  int64_t cap = (int64_t)8 * sms / (ncols > 0 ? ncols : 1);
  if (cap < 1) cap = 1;
  int64_t b = need < cap ? need : cap;
  if (b > kMaxParts) b = kMaxParts;
  return (int)(b < 1 ? 1 : b);
}

template <typename V>
void launch_probe_fill(uint64_t key, int K, int64_t D, V* out, int64_t ld, cudaStream_t st) {
  const int sms = num_sms();
  dim3 g(vec_blocks(ld, 1, K, sms), K);
  launch_k(probe_fill_kernel<V>, dim3(g), dim3(256), 0, st, key, K, D, out, ld);
}

template <typename V>
void launch_cg_init(const CgConf& cf, CgCtl* ctl, CgScalars* sc, V* X, V* R, V* P,
                    const V* bvec, double* part, cudaStream_t st) {
  dim3 g(vec_blocks(cf.ld, 1, cf.ncols, num_sms()), cf.ncols);
  launch_k(cg_init_kernel<V>, dim3(g), dim3(256), 0, st, cf, ctl, sc, X, R, P, bvec, part);
}

template <typename V>
bool launch_cg_update(const CgConf& cf, CgCtl* ctl, CgScalars* sc, V* X, V* R, V* P,
                      const V* Q, const double* gparts, double* part, double* part2,
                      cudaStream_t st, bool with_direction) {
  const int sms = num_sms();
  dim3 g(vec_blocks(cf.ld, kUpdChunks * 16 / sizeof(V), cf.ncols, sms), cf.ncols);
  if (with_direction) {
    // the fused form waits on every block of its grid: only when all fit at once
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cg_update_kernel<V, true>, 256,
                                                      0) != cudaSuccess)
      per_sm = 0;
    if ((int64_t)g.x * g.y <= (int64_t)per_sm * sms) {
      launch_k(cg_update_kernel<V, true>, dim3(g), dim3(256), 0, st, cf, ctl, sc, X, R, P, Q,
               gparts, part, part2);
      return true;
    }
    cudaGetLastError();
  }
  launch_k(cg_update_kernel<V, false>, dim3(g), dim3(256), 0, st, cf, ctl, sc, X, R, P, Q, gparts,
           part, part2);
  return false;
}

template <typename V>
void launch_cg_init_warm(const CgConf& cf, CgCtl* ctl, CgScalars* sc, const V* X, V* R, V* P,
                         const V* Q, const V* bvec, double* pz, double* pr, double* pb,
                         cudaStream_t st) {
  dim3 g(vec_blocks(cf.ld, 1, cf.ncols, num_sms()), cf.ncols);
  launch_k(cg_init_warm_kernel<V>, dim3(g), dim3(256), 0, st, cf, ctl, sc, X, R, P, Q, bvec, pz,
           pr, pb);
}

template <typename V>
void launch_cg_true_resid(const CgConf& cf, CgCtl* ctl, CgScalars* sc, V* R, const V* Q,
                          const V* bvec, double* part, double* part2, cudaStream_t st) {
  dim3 g(vec_blocks(cf.ld, 1, cf.ncols, num_sms()), cf.ncols);
  launch_k(cg_true_resid_kernel<V>, dim3(g), dim3(256), 0, st, cf, ctl, sc, R, Q, bvec, part,
           part2);
}

template <typename V>
void launch_cg_direction(const CgConf& cf, const CgCtl* ctl, const CgScalars* sc,
                         const V* R, V* P, cudaStream_t st) {
  dim3 g(vec_blocks(cf.ld, 16 / sizeof(V), cf.ncols, num_sms()), cf.ncols);
  launch_k(cg_direction_kernel<V>, dim3(g), dim3(256), 0, st, cf, ctl, sc, R, P);
}

template <typename V>
void launch_diag_mstep(const CgConf& cf, CgCtl* ctl, uint64_t key, const V* X, double* mu,
                       double* s, double* alpha, int32_t* counts, int32_t* st_iters,
                       double* st_relres, int32_t* st_clamps, int32_t* st_support,
                       cudaStream_t st) {
  int blocks = vec_blocks(cf.ld, 1, 1, num_sms());
  launch_k(diag_mstep_kernel<V>, dim3(blocks), dim3(256), 0, st, cf, ctl, key, X, mu, s, alpha, counts,
                                               st_iters, st_relres, st_clamps, st_support);
}

template <typename V>
void launch_scale(V* x, int64_t n, double beta, cudaStream_t st) {
  int blocks = (int)((n + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  launch_k(scale_kernel<V>, dim3(blocks), dim3(256), 0, st, x, n, beta);
}

#define COFEM_INST(V)                                                                   \
  template void launch_probe_fill<V>(uint64_t, int, int64_t, V*, int64_t, cudaStream_t); \
  template void launch_cg_init<V>(const CgConf&, CgCtl*, CgScalars*, V*, V*, V*,         \
                                  const V*, double*, cudaStream_t);                     \
  template bool launch_cg_update<V>(const CgConf&, CgCtl*, CgScalars*, V*, V*, V*,       \
                                    const V*, const double*, double*, double*,          \
                                    cudaStream_t, bool);                                \
  template void launch_cg_init_warm<V>(const CgConf&, CgCtl*, CgScalars*, const V*, V*,  \
                                       V*, const V*, const V*, double*, double*,        \
                                       double*, cudaStream_t);                          \
  template void launch_cg_true_resid<V>(const CgConf&, CgCtl*, CgScalars*, V*, const V*, \
                                        const V*, double*, double*, cudaStream_t);      \
  template void launch_cg_direction<V>(const CgConf&, const CgCtl*, const CgScalars*,    \
                                       const V*, V*, cudaStream_t);                     \
  template void launch_diag_mstep<V>(const CgConf&, CgCtl*, uint64_t, const V*, double*, \
                                     double*, double*, int32_t*, int32_t*, double*,     \
                                     int32_t*, int32_t*, cudaStream_t);                 \
  template void launch_scale<V>(V*, int64_t, double, cudaStream_t);
COFEM_INST(float)
COFEM_INST(double)


// Self-test of the fused update's bounded wait: one launch of the update with
// the direction update over 2 columns of 4096 values (8 blocks, all resident)
// whose arrival counter starts far past the grid size, so that no block is
// the last one and every other block's wait for the closing block runs out
// after limit_ns.  Workspace: control, scalars, partials, four blocks.
size_t cg_update_selftest_bytes() {
  return 4096 + sizeof(CgCtl) + sizeof(CgScalars) + 3 * 8 * kMaxCols * sizeof(double) +
         4 * 2 * 4096 * sizeof(float);
}

int cg_update_selftest(int64_t limit_ns, char* ws, cudaStream_t st) {
  char* o = (char*)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
  CgCtl* ctl = (CgCtl*)o;
  o += (sizeof(CgCtl) + 255) & ~(size_t)255;
  CgScalars* sc = (CgScalars*)o;
  o += (sizeof(CgScalars) + 255) & ~(size_t)255;
  double* gparts = (double*)o;
  double* part = gparts + 8 * kMaxCols;
  double* part2 = part + 8 * kMaxCols;
  float* X = (float*)(part2 + 8 * kMaxCols);
  float* R = X + 2 * 4096;
  float* P = R + 2 * 4096;
  float* Q = P + 2 * 4096;
  if (cudaMemsetAsync(ws, 0, cg_update_selftest_bytes(), st) != cudaSuccess) return -1;
  const unsigned int far = 1u << 30;
  if (cudaMemcpyAsync(&ctl->counter[1], &far, sizeof(far), cudaMemcpyHostToDevice, st) !=
      cudaSuccess)
    return -1;
  CgConf cf;
  memset(&cf, 0, sizeof(cf));
  cf.D = 4096;
  cf.ld = 4096;
  cf.ncols = 2;
  cf.K = 1;
  cf.T = 1;
  cf.tol = 1e-6;
  cf.max_iters = 10;
  cf.gen_wait_ns = (unsigned long long)limit_ns;
  cg_update_kernel<float, true><<<dim3(4, 2), dim3(256), 0, st>>>(cf, ctl, sc, X, R, P, Q,
                                                                  gparts, part, part2);
  if (cudaGetLastError() != cudaSuccess) return -1;
  int err = 0;
  if (cudaMemcpyAsync(&err, &ctl->error, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return -1;
  if (cudaStreamSynchronize(st) != cudaSuccess) return -1;
  return err;
}


// Timing of the CG vector kernels outside a fit graph (diagnostics): a
// synthetic state of ncols columns of D FP32 values (every column with
// rho_j = 1 and gamma_j = 1), then `reps` launches each of the CG update
// (with the direction update fused where its grid is resident, as in the
// fit, and P's three BF16 terms written), the separate direction update, and
// the diagonal estimate + M-step, each timed with CUDA events on `st`.
// ms[0..2] = mean milliseconds per launch, ms[3] = 1 if the update's launch
// held the direction update (its grid resident at once), else 0; returns 0,
// or -1 on a CUDA error.
static int64_t cgb_ld(int64_t D) { return round_up(D, kLdAlign); }
static int cgb_bn(int ncols) { return 16 * ((ncols + 4) / 5); }
size_t cg_kernels_bench_bytes(int64_t D, int ncols) {
  const int64_t ld = cgb_ld(D);
  return 4096 + sizeof(CgCtl) + sizeof(CgScalars) + 3 * (size_t)kMaxParts * kMaxCols * 8 +
         4 * (size_t)ncols * ld * 4 + (size_t)cgb_bn(ncols) * ld * 2 + 3 * (size_t)ld * 8 +
         (size_t)ld * 4 + 8 * 256;
}

__global__ void cgb_fill_kernel(float* v, int64_t n, uint32_t salt) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t h = mix64((uint64_t)i * 0x9E3779B97F4A7C15ull ^ salt);
    v[i] = (float)((double)(h >> 40) / (double)(1ull << 24) - 0.5);
  }
}

__global__ void cgb_reset_kernel(CgCtl* ctl, CgScalars* sc, double* gparts, int ncols) {
  const int j = threadIdx.x;
  if (j < ncols) {
    sc->rho[j] = 1.0;
    gparts[j] = 1.0;
  }
  if (j == 0) {
    ctl->normB2 = 1.0;
    ctl->error = 0;
    ctl->run = 1;
  }
}

int cg_kernels_bench(int64_t D, int ncols, int reps, char* ws, cudaStream_t st, float* ms) {
  const int64_t ld = cgb_ld(D);
  auto al = [](char* p) { return (char*)(((uintptr_t)p + 255) & ~(uintptr_t)255); };
  char* o = al(ws);
  CgCtl* ctl = (CgCtl*)o;                    o = al(o + sizeof(CgCtl));
  CgScalars* sc = (CgScalars*)o;             o = al(o + sizeof(CgScalars));
  double* gparts = (double*)o;               o = al(o + (size_t)kMaxParts * kMaxCols * 8);
  double* part = (double*)o;                 o = al(o + (size_t)kMaxParts * kMaxCols * 8);
  double* part2 = (double*)o;                o = al(o + (size_t)kMaxParts * kMaxCols * 8);
  float* X = (float*)o;                      o = al(o + (size_t)ncols * ld * 4);
  float* R = (float*)o;                      o = al(o + (size_t)ncols * ld * 4);
  float* P = (float*)o;                      o = al(o + (size_t)ncols * ld * 4);
  float* Q = (float*)o;                      o = al(o + (size_t)ncols * ld * 4);
  __nv_bfloat16* xs = (__nv_bfloat16*)o;     o = al(o + (size_t)cgb_bn(ncols) * ld * 2);
  double* mu = (double*)o;                   o = al(o + (size_t)ld * 8);
  double* s = (double*)o;                    o = al(o + (size_t)ld * 8);
  double* alpha = (double*)o;                o = al(o + (size_t)ld * 8);
  float* alpha32 = (float*)o;
  if (cudaMemsetAsync(ws, 0, cg_kernels_bench_bytes(D, ncols), st) != cudaSuccess) return -1;
  cgb_fill_kernel<<<1024, 256, 0, st>>>(X, 4 * (int64_t)ncols * ld, 7u);
  CgConf cf;
  memset(&cf, 0, sizeof(cf));
  cf.D = D;
  cf.ld = ld;
  cf.ncols = ncols;
  cf.K = ncols - 1;
  cf.T = 1;
  cf.seed = 1;
  cf.tol = 0.0;
  cf.max_iters = 1 << 30;
  cf.den_floor = 1e-12;
  cf.support_threshold = 1e6;
  cf.gamma_parts = 1;
  cf.split_nt = 3;
  cf.split_rows = cgb_bn(ncols);
  cf.split_buf = xs;
  cf.alpha32 = alpha32;
  cudaEvent_t ev[2];
  if (cudaEventCreate(&ev[0]) != cudaSuccess || cudaEventCreate(&ev[1]) != cudaSuccess) return -1;
  bool fused = false;
  for (int k = 0; k < 3; ++k) {
    float tot = 0.f;
    for (int r = 0; r < reps + 1; ++r) {
      cgb_reset_kernel<<<1, 64, 0, st>>>(ctl, sc, gparts, ncols);
      cudaEventRecord(ev[0], st);
      if (k == 0)
        fused = launch_cg_update<float>(cf, ctl, sc, X, R, P, Q, gparts, part, part2, st, true);
      else if (k == 1) launch_cg_direction<float>(cf, ctl, sc, R, P, st);
      else launch_diag_mstep<float>(cf, nullptr, probe_key(cf.seed, 1), X, mu, s, alpha, nullptr,
                                    nullptr, nullptr, nullptr, nullptr, st);
      cudaEventRecord(ev[1], st);
      if (cudaEventSynchronize(ev[1]) != cudaSuccess) return -1;
      float m = 0.f;
      cudaEventElapsedTime(&m, ev[0], ev[1]);
      if (r > 0) tot += m;                   // the first launch warms up
    }
    ms[k] = tot / (float)reps;
  }
  ms[3] = fused ? 1.f : 0.f;
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace cofem
