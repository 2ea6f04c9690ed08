// Masked-DCT dictionary (the structured Phi of Sec. 4.2): Phi = M C^T with C
// the orthonormal DCT-II matrix of size D (C^T = C^-1 its inverse, DCT-III)
// and M the N x D row selection of an undersampling mask:
//   Phi z      = (C^T z)[idx]                    inverse DCT, keep N samples
//   Phi^T w    = C scatter_idx(w)                zero-fill, forward DCT
//   Phi^T Phi x = C (m . (C^T x))                m = 0/1 mask of the kept samples
// so one operator application of the E-step, A X = beta Phi^T Phi X + alpha . X
// (Eq. (mat-eq)), is an inverse DCT, a mask, and a forward DCT per column:
// tau_D = O(D log D) (Sec. 3.2).
//
// DCTs by a complex FFT of half the length, M = D/2 (Makhoul's mapping,
// IEEE TASSP 1980, with the real sequence packed two to a complex value):
//   DCT-II:  v_m = x_{2m} (m < M), v_m = x_{2D-1-2m} (m >= M);
//            z_n = v_{2n} + i v_{2n+1}; Z = FFT_M(z);
//            E_k = (Z_k + conj Z_{M-k}) / 2, O_k = (Z_k - conj Z_{M-k}) / 2i,
//            V_k = E_k + e^{-2 pi i k / D} O_k, V_{k+M} = E_k - e^{-2 pi i k / D} O_k;
//            X_k = s_k Re(e^{-i pi k / 2D} V_k),  s_0 = sqrt(1/D), s_k = sqrt(2/D)
//   DCT-III: V_k = e^{i pi k / 2D} (X_k / s_k - i X_{D-k} / s_{D-k}) (X_D := 0);
//            Z'_k = (V_k + V_{k+M}) + i e^{2 pi i k / D} (V_k - V_{k+M});
//            z = IFFT_M(Z') / D; v_{2n} = Re z_n, v_{2n+1} = Im z_n;
//            x_{2m} = v_m, x_{2m+1} = v_{D-1-m}
// and the FFT of length M = M1 M2 by the four-step decomposition: pass 1 runs
// M2 transforms of length M1 over the stride-M2 subsequences and multiplies by
// e^{-+2 pi i n2 k1 / M}, pass 2 runs M1 transforms of length M2 over the
// rows; the DCT pre- and post-processing is fused into the loads of pass 1 and
// the stores of pass 2.  The forward DCT's post-processing pairs output k
// with M - k, which pass 2 finds in its own block: a block holds transforms
// k1 and M1 - k1 together (0 and M1/2 are their own partners).  Each block
// holds G transforms (G Lf = kFftElems complex values) in shared memory and
// runs a Stockham (self-sorting) mixed-radix FFT on them: radix-8 stages,
// then one radix-4 or radix-2 stage, each thread reading its butterflies'
// inputs into registers, all threads synchronising, then writing the outputs
// (natural order in and out, a per-block twiddle table).
#include "kernels.cuh"

namespace cofem {
void apply_tick(cudaStream_t st);
}

namespace cofem {

constexpr int kFftElems = 2048;    // complex values per block
// shared-memory index of complex value i: one pad every 8 values, so that
// the stride-8 writes of a radix-8 stage spread over the banks
__device__ __forceinline__ int pad(int i) { return i + (i >> 3); }
constexpr int kFftSmem = kFftElems + kFftElems / 8;
constexpr int kFftThreads = 256;
constexpr int kFftMaxLg = 11;      // transforms of up to 2048 points per pass (D <= 2^22)

enum DctMode { kIdct1 = 0, kIdct2 = 1, kDct1 = 2, kDct2 = 3 };

struct DctArgs {
  int64_t D;
  int lg1, lg2;            // M = D/2 = M1 M2, M1 = 2^lg1 (pass 1 length), M2 = 2^lg2 (pass 2)
  const float* xin;        // real input: X (IDCT1) or T (DCT1)
  int64_t ldx;
  float2* cbuf;            // complex intermediate, ncols x M, pitch M
  float* tout;             // IDCT2: real output (time domain), pitch ldt
  int64_t ldt;
  const float* mask;       // IDCT2: 0/1 per sample, or null (keep all)
  float* yout;             // DCT2 output, pitch ldy
  int64_t ldy;
  double beta;             // DCT2: output scale
  const double* alpha;     // DCT2: + alpha . x (x = xdiag) when alpha or alpha32 is set
  const float* alpha32;
  const float* xdiag;
  int64_t ldxd;
  double* dots;            // DCT2: per-block partials of x_j^T y_j, [block][kMaxCols]
  const float2* tabM;      // e^{i pi n / 2D}, n < D (DCT pre-/post-twiddles)
  const float2* tabW;      // e^{-2 pi i q / M}, q < M2 (low part of the four-step twiddle)
  const float2* tabR;      // e^{-2 pi i k / D}, k < M (even/odd recombination)
};

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// e^{i pi t} for t = num / den (num, den integers, den a power of two)
__device__ __forceinline__ float2 cis_pi(float t) {
  float s, c;
  sincospif(t, &s, &c);
  return make_float2(c, s);
}

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// (sgn i) z
__device__ __forceinline__ float2 mul_i(float2 z, float sgn) { return make_float2(-sgn * z.y, sgn * z.x); }

// In-register DFTs of length 2, 4, 8 with root e^{sgn 2 pi i / R}.
template <int LR>
__device__ __forceinline__ void dft_reg(float2 (&v)[1 << LR], float sgn) {
  if (LR == 1) {
    const float2 a = v[0];
    v[0] = cadd(a, v[1]);
    v[1] = csub(a, v[1]);
  } else if (LR == 2) {
    const float2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
    const float2 s13 = cadd(v[1], v[3]), d13 = mul_i(csub(v[1], v[3]), sgn);
    v[0] = cadd(s02, s13);
    v[2] = csub(s02, s13);
    v[1] = cadd(d02, d13);
    v[3] = csub(d02, d13);
  } else {
    // radix 2 x 4: X_k = E_k + w^k O_k, X_{k+4} = E_k - w^k O_k, w = e^{sgn i pi / 4}
    float2 e[4] = {v[0], v[2], v[4], v[6]}, o[4] = {v[1], v[3], v[5], v[7]};
    dft_reg<2>(e, sgn);
    dft_reg<2>(o, sgn);
    const float h = 0.70710678118654752f;
    const float2 t1 = make_float2(h * (o[1].x - sgn * o[1].y), h * (o[1].y + sgn * o[1].x));
    const float2 t2 = mul_i(o[2], sgn);
    const float2 t3 = make_float2(h * (-o[3].x - sgn * o[3].y), h * (-o[3].y + sgn * o[3].x));
    v[0] = cadd(e[0], o[0]);
    v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], t1);
    v[5] = csub(e[1], t1);
    v[2] = cadd(e[2], t2);
    v[6] = csub(e[2], t2);
    v[3] = cadd(e[3], t3);
    v[7] = csub(e[3], t3);
  }
}

// e^{sgn 2 pi i m / Lf} from the half table tw[m] (m < Lf/2), m < Lf
__device__ __forceinline__ float2 twiddle(const float2* tw, int m, int half) {
  const float2 w = tw[m & (half - 1)];
  return m < half ? w : make_float2(-w.x, -w.y);
}

// One Stockham stage of radix R = 2^LR over G transforms of length 2^lg in
// s[pad(...)], Ns = product of the radices of the earlier stages: butterfly
// j of a transform reads elements j + r Lf/R, twiddles them by
// e^{sgn 2 pi i (j mod Ns) r / (Ns R)}, and writes element
// (j - j mod Ns) R + (j mod Ns) + r Ns.
template <int LR>
__device__ __forceinline__ void fft_stage(float2* s, const float2* tw, int lg, int G, int lgNs,
                                          float sgn) {
  constexpr int R = 1 << LR;
  constexpr int TPT = kFftElems / kFftThreads / R;      // butterflies per thread
  const int Lf = 1 << lg, nb = Lf >> LR, ntask = G * nb;
  const int Ns = 1 << lgNs;
  float2 v[TPT][R];
  int dst[TPT];
#pragma unroll
  for (int q = 0; q < TPT; ++q) {
    const int b = threadIdx.x + q * kFftThreads;
    dst[q] = -1;
    if (b < ntask) {
      const int t = b >> (lg - LR), j = b & (nb - 1);
      const int base = t << lg;
      const int jm = j & (Ns - 1);
      const int unit = jm << (lg - lgNs - LR);       // Lf (j mod Ns) / (Ns R)
#pragma unroll
      for (int r = 0; r < R; ++r) v[q][r] = s[pad(base + j + r * nb)];
#pragma unroll
      for (int r = 1; r < R; ++r) v[q][r] = cmul(v[q][r], twiddle(tw, (unit * r) & (Lf - 1), Lf >> 1));
      dft_reg<LR>(v[q], sgn);
      dst[q] = base + ((j - jm) << LR) + jm;
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < TPT; ++q)
    if (dst[q] >= 0) {
#pragma unroll
      for (int r = 0; r < R; ++r) s[pad(dst[q] + (r << lgNs))] = v[q][r];
    }
  __syncthreads();
}

// G transforms of length 2^lg in natural order in s[pad(t << lg ...)]:
// radix-8 stages, then one radix-4 or radix-2 stage; natural order out.
__device__ void fft_stages(float2* s, const float2* tw, int lg, int G, float sgn) {
  int lgNs = 0;
  while (lg - lgNs >= 3) {
    fft_stage<3>(s, tw, lg, G, lgNs, sgn);
    lgNs += 3;
  }
  if (lg - lgNs == 2) fft_stage<2>(s, tw, lg, G, lgNs, sgn);
  else if (lg - lgNs == 1) fft_stage<1>(s, tw, lg, G, lgNs, sgn);
}


// grid (transform groups, ncols), kFftThreads threads.
template <int MODE>
__global__ void __launch_bounds__(kFftThreads, 3)
dct_pass_kernel(DctArgs a) {
  pdl_wait();
  pdl_trigger();
  __shared__ float2 s[kFftSmem];
  __shared__ float2 tw[1 << (kFftMaxLg - 1)];
  __shared__ double red[32];
  constexpr bool pass1 = MODE == kIdct1 || MODE == kDct1;
  constexpr bool inverse = MODE == kIdct1 || MODE == kIdct2;
  constexpr int kPer = kFftElems / kFftThreads;   // elements per thread
  const int j = blockIdx.y;
  const int D = (int)a.D;                          // <= 2^22
  const int M = D >> 1;
  const int M1 = 1 << a.lg1;
  const int lg = pass1 ? a.lg1 : a.lg2;           // length of this pass's transforms
  const int Lf = 1 << lg;
  const int ntr = pass1 ? (1 << a.lg2) : M1;      // transforms in the pass
  const int G = min(kFftElems >> lg, ntr);
  const int lgG = __ffs(G) - 1;                    // G is a power of two
  const int nel = G << lg;                         // elements of this block
  const float sgn = inverse ? 1.f : -1.f;
  for (int i = threadIdx.x; i < (Lf >> 1); i += blockDim.x)
    tw[i] = cis_pi(sgn * 2.f * (float)i / (float)Lf);
  const float sD = sqrtf(1.f / (float)D), sK = sqrtf(2.f / (float)D);
  const float rsD = 1.f / sD, rsK = 1.f / sK;
  float2* cb = a.cbuf + (int64_t)j * M;
  // pass 2: local transform tt is k1 = pi (tt < G/2) or its partner M1 - pi
  // (tt >= G/2), pi = blockIdx.x G/2 + tt mod G/2; pair 0 holds k1 = 0 and
  // k1 = M1/2, each its own partner
  const int hG = G >> 1;
  auto k1_of = [&](int tt) {
    const int pi = blockIdx.x * hG + (tt & (hG - 1));
    return tt < hG ? pi : (pi == 0 ? (M1 >> 1) : M1 - pi);
  };
  const int t0 = blockIdx.x * G;                   // pass 1: first transform n2

  // ---- load: all of a thread's global loads first, then the shared stores
  float2 v[kPer];
  if (pass1) {
    // element n1 of transform n2 is z_n, n = M2 n1 + n2; consecutive threads
    // take consecutive n2
    const float* xj = a.xin + (int64_t)j * a.ldx;
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int i = threadIdx.x + q * kFftThreads;
      v[q] = make_float2(0.f, 0.f);
      if (i < nel) {
        const int n = ((i >> lgG) << a.lg2) + t0 + (i & (G - 1));
        if (MODE == kIdct1) {
          // V_n and V_{n+M} from X_n, X_{D-n}, X_{n+M}, X_{M-n}
          const float x0 = xj[n] * (n == 0 ? rsD : rsK);
          const float x0r = n == 0 ? 0.f : xj[D - n] * rsK;
          const float x1 = xj[n + M] * rsK;
          const float x1r = xj[M - n] * rsK;
          const float2 va = cmul(a.tabM[n], make_float2(x0, -x0r));
          const float2 vb = cmul(a.tabM[n + M], make_float2(x1, -x1r));
          const float2 rr = a.tabR[n];                // e^{-2 pi i n / D}; conjugated
          const float2 dv = csub(va, vb);
          const float2 t = cmul(make_float2(rr.x, -rr.y), dv);
          v[q] = cadd(cadd(va, vb), make_float2(-t.y, t.x));   // + i e^{2 pi i n/D} (V_n - V_{n+M})
        } else {
          // z_n = v_{2n} + i v_{2n+1}, v_m = T[2m] (m < M), T[2D-1-2m] (m >= M)
          const int m0 = 2 * n, m1 = 2 * n + 1;
          v[q] = make_float2(xj[m0 < M ? 2 * m0 : 2 * D - 1 - 2 * m0],
                             xj[m1 < M ? 2 * m1 : 2 * D - 1 - 2 * m1]);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int i = threadIdx.x + q * kFftThreads;
      if (i < nel) s[pad(((i & (G - 1)) << lg) + (i >> lgG))] = v[q];
    }
  } else {
    // transform k1 is the contiguous row cb[M2 k1 ...]
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int i = threadIdx.x + q * kFftThreads;
      if (i < nel) v[q] = cb[(k1_of(i >> lg) << a.lg2) + (i & (Lf - 1))];
    }
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int i = threadIdx.x + q * kFftThreads;
      if (i < nel) s[pad(i)] = v[q];
    }
  }
  __syncthreads();
  fft_stages(s, tw, lg, G, sgn);

  // ---- store
  if (pass1) {
    // twiddle e^{sgn 2 pi i n2 k1 / M} = e^{sgn 2 pi i qh / M1} e^{sgn 2 pi i ql / M}
    // with n2 k1 = qh M2 + ql (the first factor is this pass's own table),
    // then cb[M2 k1 + n2]
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int i = threadIdx.x + q * kFftThreads;
      if (i < nel) {
        const int tt = i & (G - 1), f = i >> lgG;
        const int n2 = t0 + tt;
        const int r = n2 * f;                      // < M
        const float2 lo = a.tabW[r & ((1 << a.lg2) - 1)];
        const float2 w = cmul(twiddle(tw, r >> a.lg2, Lf >> 1),
                              inverse ? make_float2(lo.x, -lo.y) : lo);
        cb[(f << a.lg2) + n2] = cmul(w, s[pad((tt << lg) + f)]);
      }
    }
  } else {
    AccF dot;
    const bool diag = MODE == kDct2 && (a.alpha32 != nullptr || a.alpha != nullptr);
    // frequency k2 of transform k1 is k = k1 + M1 k2 < M; consecutive
    // threads take consecutive local transforms
    const int M2 = 1 << a.lg2;
#pragma unroll 4
    for (int q = 0; q < kPer; ++q) {
      const int i = threadIdx.x + q * kFftThreads;
      if (i < nel) {
        const int tt = i & (G - 1), f = i >> lgG;
        const int k1 = k1_of(tt);
        const int k = k1 + (f << a.lg1);
        const float2 zk = s[pad((tt << lg) + f)];
        if (MODE == kIdct2) {
          // v_{2k} = Re z_k / D, v_{2k+1} = Im z_k / D, then x_{2m} = v_m,
          // x_{2m+1} = v_{D-1-m}
          const float invD = 1.f / (float)D;
          const int m0 = 2 * k, m1 = 2 * k + 1;
          const int y0 = m0 < M ? 2 * m0 : 2 * (D - 1 - m0) + 1;
          const int y1 = m1 < M ? 2 * m1 : 2 * (D - 1 - m1) + 1;
          const float g0 = a.mask ? a.mask[y0] : 1.f, g1 = a.mask ? a.mask[y1] : 1.f;
          a.tout[(int64_t)j * a.ldt + y0] = g0 * zk.x * invD;
          a.tout[(int64_t)j * a.ldt + y1] = g1 * zk.y * invD;
        } else {
          // partner M - k: (0, M2 - k2) for k1 = 0, else (M1 - k1, M2 - 1 - k2),
          // in local transform tt (pair 0) or tt ^ G/2
          const int pt = (blockIdx.x == 0 && (tt & (hG - 1)) == 0) ? tt : (tt ^ hG);
          const int pf = k1 == 0 ? ((M2 - f) & (M2 - 1)) : (M2 - 1 - f);
          const float2 zp0 = s[pad((pt << lg) + pf)];
          const float2 zp = make_float2(zp0.x, -zp0.y);               // conj Z_{M-k}
          const float2 e = make_float2(0.5f * (zk.x + zp.x), 0.5f * (zk.y + zp.y));
          const float2 dd = make_float2(0.5f * (zk.x - zp.x), 0.5f * (zk.y - zp.y));
          const float2 o = cmul(a.tabR[k], make_float2(dd.y, -dd.x));  // e^{-2 pi i k/D} (Z - conj Z')/2i
          const float2 va = cadd(e, o), vb = csub(e, o);               // V_k, V_{k+M}
          const float2 wa = a.tabM[k], wb = a.tabM[k + M];             // conjugated below
          const float oa = (k == 0 ? sD : sK) * (wa.x * va.x + wa.y * va.y);
          const float ob = sK * (wb.x * vb.x + wb.y * vb.y);
          float outa = (float)a.beta * oa, outb = (float)a.beta * ob;
          if (diag) {
            const float xa = a.xdiag[(int64_t)j * a.ldxd + k];
            const float xb = a.xdiag[(int64_t)j * a.ldxd + k + M];
            const float ala = a.alpha32 ? a.alpha32[k] : (float)a.alpha[k];
            const float alb = a.alpha32 ? a.alpha32[k + M] : (float)a.alpha[k + M];
            outa = fmaf(ala, xa, outa);
            outb = fmaf(alb, xb, outb);
            dot.add_prod(xa, outa);
            dot.add_prod(xb, outb);
          }
          a.yout[(int64_t)j * a.ldy + k] = outa;
          a.yout[(int64_t)j * a.ldy + k + M] = outb;
        }
      }
    }
    if (MODE == kDct2 && a.dots) {
      const double sdot = block_sum(dot, red);
      if (threadIdx.x == 0) a.dots[(int64_t)blockIdx.x * kMaxCols + j] = sdot;
    }
  }
}

// tabM[n] = e^{i pi n / 2D} (n < D), tabW[q] = e^{-2 pi i q / M} (q < M2),
// tabR[k] = e^{-2 pi i k / D} (k < M)
__global__ void dct_twiddle_kernel(int64_t D, int M2, float2* tabM, float2* tabW, float2* tabR) {
  pdl_wait();
  pdl_trigger();
  const int64_t M = D / 2;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < D;
       n += (int64_t)gridDim.x * blockDim.x) {
    tabM[n] = cis_pi((float)n / (float)(2 * D));
    if (n < M2) tabW[n] = cis_pi(-2.f * (float)n / (float)M);
    if (n < M) tabR[n] = cis_pi(-2.f * (float)n / (float)D);
  }
}

// 0/1 mask of the kept samples (dst must be zeroed); idx must be strictly
// increasing in [0, D): a violation sets *err and is skipped.
__global__ void dct_mask_kernel(const int32_t* idx, int64_t N, int64_t D, float* mask,
                                int* err) {
  pdl_wait();
  pdl_trigger();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = idx[i];
    const bool ok = v >= 0 && v < D && (i == 0 || idx[i - 1] < v);
    if (!ok) {
      if (err) atomicCAS(err, 0, (int)COFEM_ERR_INVALID_ARG);
      continue;
    }
    mask[v] = 1.f;
  }
}

// T[j][idx[i]] = W[j][i] (T zeroed before)
__global__ void dct_scatter_kernel(const int32_t* idx, int64_t N, int64_t D, const float* W,
                                   int64_t ldw, float* T, int64_t ldt, int* err) {
  pdl_wait();
  pdl_trigger();
  const int j = blockIdx.y;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = idx[i];
    if (v < 0 || v >= D) {
      if (err) atomicCAS(err, 0, (int)COFEM_ERR_INVALID_ARG);
      continue;
    }
    T[(int64_t)j * ldt + v] = W[(int64_t)j * ldw + i];
  }
}

// W[j][i] = T[j][idx[i]]
__global__ void dct_gather_kernel(const int32_t* idx, int64_t N, int64_t D, const float* T,
                                  int64_t ldt, float* W, int64_t ldw, int* err) {
  pdl_wait();
  pdl_trigger();
  const int j = blockIdx.y;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = idx[i];
    float w = 0.f;
    if (v >= 0 && v < D) w = T[(int64_t)j * ldt + v];
    else if (err) atomicCAS(err, 0, (int)COFEM_ERR_INVALID_ARG);
    W[(int64_t)j * ldw + i] = w;
  }
}

// ------------------------------------------------------------ launchers

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static int ilog2(int64_t D) {
  int p = 0;
  while (((int64_t)1 << p) < D) ++p;
  return p;
}

bool dct_size_ok(int64_t D) {
  const int p = ilog2(D);
  return D >= 16 && ((int64_t)1 << p) == D && p <= 2 * kFftMaxLg;
}

// workspace: complex buffer (ncols x D/2), real T (ncols x D), mask (D),
// twiddle tables tabM (D complex), tabW (D/2) and tabR (D/2)
static size_t cbuf_bytes(int64_t D, int ncols) { return align256((size_t)ncols * (D / 2) * sizeof(float2)); }
static size_t tout_bytes(int64_t D, int ncols) { return align256((size_t)ncols * D * sizeof(float)); }
size_t dct_ws_bytes(int64_t D, int ncols) {
  return cbuf_bytes(D, ncols) + tout_bytes(D, ncols) + align256((size_t)D * sizeof(float)) +
         align256((size_t)D * sizeof(float2)) + 2 * align256((size_t)(D / 2) * sizeof(float2));
}

// Carves the workspace; fills the twiddle tables (one small launch) unless
// `tables` is false (they are already there).
static DctArgs dct_args(int64_t D, char* ws, int ncols, cudaStream_t st, bool tables = true) {
  DctArgs a = {};
  a.D = D;
  const int p = ilog2(D) - 1;                      // M = D/2 = 2^p
  a.lg2 = p / 2;                                   // M2 <= M1: pass 2 holds >= 2 transforms
  a.lg1 = p - a.lg2;
  a.cbuf = (float2*)ws;
  a.tout = (float*)(ws + cbuf_bytes(D, ncols));
  a.ldt = D;
  char* t = ws + cbuf_bytes(D, ncols) + tout_bytes(D, ncols) + align256((size_t)D * sizeof(float));
  float2* tabM = (float2*)t;
  float2* tabW = (float2*)(t + align256((size_t)D * sizeof(float2)));
  float2* tabR = (float2*)(t + align256((size_t)D * sizeof(float2)) +
                           align256((size_t)(D / 2) * sizeof(float2)));
  if (tables)
    launch_k(dct_twiddle_kernel, dim3((unsigned)std::min<int64_t>((D + 255) / 256, 1024)),
             dim3(256), 0, st, D, 1 << a.lg2, tabM, tabW, tabR);
  a.tabM = tabM;
  a.tabW = tabW;
  a.tabR = tabR;
  return a;
}
static float* dct_mask_buf(int64_t D, char* ws, int ncols) {
  return (float*)(ws + cbuf_bytes(D, ncols) + tout_bytes(D, ncols));
}

template <int MODE>
static void dct_launch(const DctArgs& a, int ncols, cudaStream_t st) {
  const bool pass1 = MODE == kIdct1 || MODE == kDct1;
  const int lg = pass1 ? a.lg1 : a.lg2;
  const int ntr = pass1 ? (1 << a.lg2) : (1 << a.lg1);
  const int G = std::min(kFftElems >> lg, ntr);
  launch_k(dct_pass_kernel<MODE>, dim3((unsigned)(ntr / G), (unsigned)ncols), dim3(kFftThreads),
           0, st, a);
}
static int dct_parts(const DctArgs& a) {
  const int G = std::min(kFftElems >> a.lg2, 1 << a.lg1);
  return (1 << a.lg1) / G;
}

// The mask and the twiddle tables in the workspace (dct_apply with
// prepared = true reuses them).
void dct_prepare(int64_t D, const int32_t* idx, int64_t N, int ncols, char* ws, int* err,
                 cudaStream_t st) {
  dct_args(D, ws, ncols, st, true);
  float* mask = dct_mask_buf(D, ws, ncols);
  cudaMemsetAsync(mask, 0, (size_t)D * sizeof(float), st);
  launch_k(dct_mask_kernel, dim3((unsigned)std::min<int64_t>((N + 255) / 256, 4096)), dim3(256),
           0, st, idx, N, D, mask, err);
}

// Y = beta C (m . C^T X) + alpha . X, dots partials of x_j^T y_j
int dct_apply(int64_t D, const int32_t* idx, int64_t N, const float* X, int64_t ld, int ncols,
              float* Y, double beta, const double* alpha, const float* alpha32, double* dots,
              char* ws, int* err, cudaStream_t st, bool prepared) {
  if (!prepared) dct_prepare(D, idx, N, ncols, ws, err, st);
  DctArgs a = dct_args(D, ws, ncols, st, false);
  float* mask = dct_mask_buf(D, ws, ncols);
  apply_tick(st);
  a.xin = X;
  a.ldx = ld;
  a.mask = mask;
  dct_launch<kIdct1>(a, ncols, st);
  apply_tick(st);
  dct_launch<kIdct2>(a, ncols, st);
  apply_tick(st);
  a.xin = a.tout;
  a.ldx = a.ldt;
  dct_launch<kDct1>(a, ncols, st);
  apply_tick(st);
  a.yout = Y;
  a.ldy = ld;
  a.beta = beta;
  a.alpha = alpha;
  a.alpha32 = alpha32;
  a.xdiag = X;
  a.ldxd = ld;
  a.dots = dots;
  dct_launch<kDct2>(a, ncols, st);
  apply_tick(st);
  return dct_parts(a);
}

// W = Phi Z: inverse DCT, keep the N masked samples
void dct_forward(int64_t D, const int32_t* idx, int64_t N, const float* Z, int64_t ldz, int ncols,
                 float* W, int64_t ldw, char* ws, int* err, cudaStream_t st) {
  DctArgs a = dct_args(D, ws, ncols, st);
  a.xin = Z;
  a.ldx = ldz;
  a.mask = nullptr;
  dct_launch<kIdct1>(a, ncols, st);
  dct_launch<kIdct2>(a, ncols, st);
  launch_k(dct_gather_kernel, dim3((unsigned)std::min<int64_t>((N + 255) / 256, 4096), ncols),
           dim3(256), 0, st, idx, N, D, (const float*)a.tout, a.ldt, W, ldw, err);
}

// ||phi_d||^2 of the masked dictionary (the learned start's feature and
// Jacobi scale).  phi_d is row d of C restricted to the kept samples, so with
// cos^2 t = (1 + cos 2t) / 2,
//   ||phi_d||^2 = sum_{n kept} C_dn^2 = (s_d^2 / 2) (N + T_d),
//   T_d = sum_{n kept} cos(pi 2d (2n + 1) / 2D),
// and T_d comes from X = C m, the orthonormal DCT-II of the 0/1 mask m:
// T_d = X_{2d} / s_{2d} for 2d < D, 0 for 2d = D, and -X_{2D-2d} / s_{2D-2d}
// for 2d > D (cos(pi (2n + 1) - t) = -cos t).
__global__ void dct_col_norms_kernel(int64_t D, int64_t N, const float* X, float* out) {
  pdl_wait();
  pdl_trigger();
  const double inv_d = 1.0 / (double)D;
  for (int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; d < D;
       d += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = 2 * d;
    double t = 0.0;
    if (k < D) t = (double)X[k] / sqrt((k == 0 ? 1.0 : 2.0) * inv_d);
    else if (k > D) t = -(double)X[2 * D - k] / sqrt(2.0 * inv_d);
    const double sd2 = (d == 0 ? 1.0 : 2.0) * inv_d;
    out[d] = (float)(0.5 * sd2 * ((double)N + t));
  }
}

__global__ void dct_fill_ones_kernel(float* v, int64_t n) {
  pdl_wait();
  pdl_trigger();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    v[i] = 1.f;
}

void dct_col_norms(int64_t D, const int32_t* idx, int64_t N, float* ones_buf, float* x_buf,
                   char* ws, int* err, float* out, cudaStream_t st) {
  launch_k(dct_fill_ones_kernel, dim3((unsigned)std::min<int64_t>((N + 255) / 256, 4096)),
           dim3(256), 0, st, ones_buf, N);
  dct_adjoint(D, idx, N, ones_buf, N, 1, x_buf, D, 1.0, ws, err, st);
  launch_k(dct_col_norms_kernel, dim3((unsigned)std::min<int64_t>((D + 255) / 256, 4096)),
           dim3(256), 0, st, D, N, (const float*)x_buf, out);
}

// Z = beta Phi^T W: zero-fill the unkept samples, forward DCT
void dct_adjoint(int64_t D, const int32_t* idx, int64_t N, const float* W, int64_t ldw, int ncols,
                 float* Z, int64_t ldz, double beta, char* ws, int* err, cudaStream_t st) {
  DctArgs a = dct_args(D, ws, ncols, st);
  cudaMemsetAsync(a.tout, 0, (size_t)ncols * D * sizeof(float), st);
  launch_k(dct_scatter_kernel, dim3((unsigned)std::min<int64_t>((N + 255) / 256, 4096), ncols),
           dim3(256), 0, st, idx, N, D, W, ldw, a.tout, a.ldt, err);
  a.xin = a.tout;
  a.ldx = a.ldt;
  dct_launch<kDct1>(a, ncols, st);
  a.yout = Z;
  a.ldy = ldz;
  a.beta = beta;
  dct_launch<kDct2>(a, ncols, st);
}

}  // namespace cofem
