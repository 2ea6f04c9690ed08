// Circular convolutional dictionary (a structured Phi of Sec. 3.2, whose
// application costs O(C T L) instead of O(N D)):
//   (Phi z)[n]     = sum_c sum_{t<T} h[c][t] z_c[(n - t) mod L]        forward
//   (Phi^T w)_c[m] = sum_{t<T} h[c][t] w[(m + t) mod L]               adjoint
// with N = L and D = C L, coordinate d = c L + m.  The operator of the
// E-step, A X = beta Phi^T Phi X + alpha . X (Eq. (mat-eq)), is one forward
// and one adjoint launch; the adjoint's epilogue applies beta, adds
// alpha . x and accumulates the x_j^T (A x)_j partials of the CG step.
//
// Both kernels stage a tile of TILE = 256 * R outputs (R = 16) plus a T-1
// halo of the input column in shared memory (wrapping circularly; the
// forward kernel copies the next channel's tile with cp.async while it
// computes the current one), and every thread produces R consecutive outputs
// from register windows of 31 staged values, one window per 16 filter taps
// (taps read as float4): 31 shared loads per 256 FMAs.  The shared tile is
// skewed by one word every 16 (index i -> i + i/16) so that threads reading
// at stride R hit distinct banks.  The grid runs the columns of a tile side
// by side so alpha stays in L2.
#include "kernels.cuh"

namespace cofem {
void apply_tick(cudaStream_t st);
}

namespace cofem {

constexpr int kConvThreads = 256;
constexpr int kConvR = 16;                           // outputs per thread
constexpr int kConvTile = kConvThreads * kConvR;    // 4096 outputs per block
constexpr int kConvMaxT = 64;
constexpr int kTapChunk = 16;                        // filter taps per register window
static_assert(kTapChunk == kConvR, "the window indexing assumes a chunk of R taps");

__host__ __device__ constexpr int skew(int i) { return i + (i >> 4); }
constexpr int kStageWords = skew(kConvTile + kConvMaxT) + 8;   // one staged tile

// w[i] = tile[skew(x0 + i)], i < 31, for x0 a multiple of 16: the skew
// adds x0/16 to every index and one more to i >= 16, so one base pointer
// and constant offsets replace the per-load arithmetic.  Thread t's window
// starts at 16 t + const, i.e. at word 17 t + const: distinct banks.
__device__ __forceinline__ void load_window(const float* tile, int x0,
                                            float (&w)[2 * kTapChunk - 1]) {
  const float* lo = tile + skew(x0);
  const float* hi = lo + 1;
#pragma unroll
  for (int i = 0; i < kTapChunk; ++i) w[i] = lo[i];
#pragma unroll
  for (int i = kTapChunk; i < 2 * kTapChunk - 1; ++i) w[i] = hi[i];
}

// 4-byte asynchronous global -> shared copies (cp.async), grouped per channel.
__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// W[j][n] = sum_c sum_t h[c][t] Z[j][c*L + (n - t) mod L]
// grid (ncols, L / TILE): the columns of one tile run side by side.
template <int T>
__global__ void __launch_bounds__(kConvThreads, 2)
conv_forward_kernel(const float* __restrict__ h, int C, int64_t L, const float* __restrict__ Z,
                    int64_t ldz, float* __restrict__ W, int64_t ldw) {
  pdl_wait();
  pdl_trigger();
  // two staged tiles: channel c + 1 is copied (cp.async) while channel c
  // is computed
  __shared__ float zs2[2][kStageWords];
  const int j = blockIdx.x;
  const int64_t n0 = (int64_t)blockIdx.y * kConvTile;
  const int tid = threadIdx.x;
  float acc[kConvR];
#pragma unroll
  for (int r = 0; r < kConvR; ++r) acc[r] = 0.f;
  const int span = kConvTile + T - 1;
  const bool wrap1 = L >= span;              // one add or subtract of L suffices
  const int base = (T - 1) + tid * kConvR;   // zs index of output n0 + tid*R at tap 0
  auto stage = [&](int c, float* buf) {
    const float* zc = Z + (int64_t)j * ldz + (int64_t)c * L;
    for (int i = tid; i < span; i += kConvThreads) {
      int64_t n = n0 - (T - 1) + i;
      if (wrap1) n = n < 0 ? n + L : (n >= L ? n - L : n);
      else n = ((n % L) + L) % L;            // L shorter than the staged span
      cp_async4(buf + skew(i), zc + n);
    }
    cp_async_commit();
  };
  stage(0, zs2[0]);
  for (int c = 0; c < C; ++c) {
    if (c + 1 < C) stage(c + 1, zs2[(c + 1) & 1]);
    else cp_async_commit();                  // an empty group keeps the count uniform
    cp_async_wait1();                        // this thread's copies of channel c landed
    __syncthreads();                         // everyone's
    const float* zs = zs2[c & 1];
    // taps t0 .. t0+15: output r at tap t0 + q reads w[r - q + 15], a
    // window of 31 staged values loaded once per chunk (static indices)
#pragma unroll 1
    for (int t0 = 0; t0 < T; t0 += kTapChunk) {
      float w[2 * kTapChunk - 1];
      load_window(zs, base - t0 - (kTapChunk - 1), w);
      float hr[kTapChunk];
      const float4* h4 = reinterpret_cast<const float4*>(h + c * T + t0);
#pragma unroll
      for (int q4 = 0; q4 < kTapChunk / 4; ++q4) {
        const float4 v = __ldg(h4 + q4);
        hr[4 * q4] = v.x; hr[4 * q4 + 1] = v.y; hr[4 * q4 + 2] = v.z; hr[4 * q4 + 3] = v.w;
      }
#pragma unroll
      for (int q = 0; q < kTapChunk; ++q) {
#pragma unroll
        for (int r = 0; r < kConvR; ++r) acc[r] = fmaf(hr[q], w[r - q + kTapChunk - 1], acc[r]);
      }
    }
    __syncthreads();                         // this tile is read before it is refilled
  }
  float* wj = W + (int64_t)j * ldw + n0 + tid * kConvR;
  if (n0 + tid * kConvR + kConvR <= L) {
#pragma unroll
    for (int q = 0; q < kConvR / 4; ++q)
      reinterpret_cast<float4*>(wj)[q] =
          make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
  }
}

// Y[j][c*L + m] = beta * sum_t h[c][t] W[j][(m + t) mod L] (+ alpha . X),
// dots[tile][j] = sum over the block of X . Y.      grid (ncols, L / TILE)
template <int T>
__global__ void __launch_bounds__(kConvThreads, 3)
conv_adjoint_kernel(const float* __restrict__ h, int C, int64_t L, const float* __restrict__ W,
                    int64_t ldw, float* __restrict__ Y, int64_t ld, double beta,
                    const double* __restrict__ alpha, const float* __restrict__ alpha32,
                    const float* __restrict__ X, double* dots) {
  pdl_wait();
  pdl_trigger();
  __shared__ float ws[skew(kConvTile + kConvMaxT) + 8];
  __shared__ double red[32];
  const int j = blockIdx.x;
  const int64_t m0 = (int64_t)blockIdx.y * kConvTile;
  const int tid = threadIdx.x;
  const int span = kConvTile + T - 1;
  const float* wj = W + (int64_t)j * ldw;
  // the column's tile is staged by cp.async (no load -> store round trip
  // through registers per element)
  for (int i = tid; i < span; i += kConvThreads) {
    int64_t n = m0 + i;
    n = L >= span ? (n >= L ? n - L : n) : n % L;
    cp_async4(ws + skew(i), wj + n);
  }
  cp_async_commit();
  cp_async_wait0();
  __syncthreads();
  const int base = tid * kConvR;
  const bool live = m0 + base + kConvR <= L;
  AccF dot;
  float sbig = 0.f;        // products of 1e30 or more, scaled by 2^-64 (FP32, not FP64)
  const bool diag = alpha32 != nullptr || alpha != nullptr;
  const float beta32 = (float)beta;
  for (int c = 0; c < C; ++c) {
    float acc[kConvR];
#pragma unroll
    for (int r = 0; r < kConvR; ++r) acc[r] = 0.f;
    // the epilogue's x and alpha are loaded first: their latency overlaps
    // the channel's FMAs
    const int64_t d = (int64_t)c * L + m0 + base;
    float xr[kConvR], ar[kConvR];
    if (live && diag) {
      const float4* x4 = reinterpret_cast<const float4*>(X + (int64_t)j * ld + d);
#pragma unroll
      for (int q = 0; q < kConvR / 4; ++q) {
        const float4 v = x4[q];
        xr[4 * q] = v.x; xr[4 * q + 1] = v.y; xr[4 * q + 2] = v.z; xr[4 * q + 3] = v.w;
      }
      if (alpha32) {
        const float4* a4 = reinterpret_cast<const float4*>(alpha32 + d);
#pragma unroll
        for (int q = 0; q < kConvR / 4; ++q) {
          const float4 v = a4[q];
          ar[4 * q] = v.x; ar[4 * q + 1] = v.y; ar[4 * q + 2] = v.z; ar[4 * q + 3] = v.w;
        }
      } else {
#pragma unroll
        for (int e = 0; e < kConvR; ++e) ar[e] = (float)alpha[d + e];
      }
    }
    // taps t0 .. t0+15: output r at tap t0 + q reads w[r + q], a window of
    // 31 staged values loaded once per chunk (static indices)
#pragma unroll 1
    for (int t0 = 0; t0 < T; t0 += kTapChunk) {
      float w[2 * kTapChunk - 1];
      load_window(ws, base + t0, w);
      float hr[kTapChunk];
      const float4* h4 = reinterpret_cast<const float4*>(h + c * T + t0);
#pragma unroll
      for (int q4 = 0; q4 < kTapChunk / 4; ++q4) {
        const float4 v = __ldg(h4 + q4);
        hr[4 * q4] = v.x; hr[4 * q4 + 1] = v.y; hr[4 * q4 + 2] = v.z; hr[4 * q4 + 3] = v.w;
      }
#pragma unroll
      for (int q = 0; q < kTapChunk; ++q) {
#pragma unroll
        for (int r = 0; r < kConvR; ++r) acc[r] = fmaf(hr[q], w[r + q], acc[r]);
      }
    }
    if (live) {
      float* yj = Y + (int64_t)j * ld + d;
#pragma unroll
      for (int q = 0; q < kConvR / 4; ++q) {
        float out[4];
        if (diag) {
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const float xv = xr[4 * q + e];
            out[e] = fmaf(ar[4 * q + e], xv, beta32 * acc[4 * q + e]);
            // compensated FP32 x^T y (product error by FMA, TwoSum)
            const float pp = xv * out[e];
            const bool fin = fabsf(pp) < 1e30f;
            sbig += fin ? 0.f : (xv * 0x1p-64f) * out[e];
            dot.c += fin ? fmaf(xv, out[e], -pp) : 0.f;
            const float x = fin ? pp : 0.f;
            const float t = dot.s + x, tv = t - dot.s;
            dot.c += (dot.s - (t - tv)) + (x - tv);
            dot.s = t;
          }
        } else {
#pragma unroll
          for (int e = 0; e < 4; ++e) out[e] = beta32 * acc[4 * q + e];
        }
        reinterpret_cast<float4*>(yj)[q] = make_float4(out[0], out[1], out[2], out[3]);
      }
    }
  }
  if (dots) {
    dot.big = (double)sbig * 0x1p64;
    const double s = block_sum(dot, red);
    if (tid == 0) dots[(int64_t)blockIdx.y * kMaxCols + j] = s;
  }
}

// ------------------------------------------------------------ launchers
// T is instantiated for 64 taps (the dictionaries of the large workload)
// and for every T <= 64 through the generic 64-tap kernel with zero taps
// appended by the caller (the operator pads h to 64 taps).

void conv_forward(const float* h64, int C, int64_t L, const float* Z, int64_t ldz, int ncols,
                  float* W, int64_t ldw, cudaStream_t st) {
  dim3 g(ncols, (unsigned)((L + kConvTile - 1) / kConvTile));
  launch_k(conv_forward_kernel<kConvMaxT>, dim3(g), dim3(kConvThreads), 0, st, h64, C, L, Z, ldz, W, ldw);
  apply_tick(st);
}

int conv_adjoint(const float* h64, int C, int64_t L, const float* W, int64_t ldw, int ncols,
                 float* Y, int64_t ld, double beta, const double* alpha, const float* X,
                 double* dots, cudaStream_t st, const float* alpha32) {
  dim3 g(ncols, (unsigned)((L + kConvTile - 1) / kConvTile));
  launch_k(conv_adjoint_kernel<kConvMaxT>, dim3(g), dim3(kConvThreads), 0, st, h64, C, L, W, ldw, Y, ld, beta,
                                                            alpha, alpha32, X, dots);
  apply_tick(st);
  return (int)g.y;
}

__global__ void pad_filters_kernel(const float* h, int C, int T, float* h64) {
  pdl_wait();
  pdl_trigger();
  for (int i = threadIdx.x + blockIdx.x * blockDim.x; i < C * kConvMaxT;
       i += blockDim.x * gridDim.x) {
    const int c = i / kConvMaxT, t = i % kConvMaxT;
    h64[i] = t < T ? h[c * T + t] : 0.f;
  }
}

// FP32 copy of alpha for an application without one: each value converted
// once (the adjoint epilogues then read 4 bytes per coordinate and convert
// nothing; a conversion per coordinate and column runs on the FP64 pipe)
__global__ void alpha_f32_kernel(const double* a, int64_t n, float* out) {
  pdl_wait();
  pdl_trigger();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)a[i];
}

void conv_alpha_f32(const double* alpha, int64_t n, float* out, cudaStream_t st) {
  const int64_t b = (n + 255) / 256;
  launch_k(alpha_f32_kernel, dim3((unsigned)(b < 4096 ? b : 4096)), dim3(256), 0, st, alpha, n,
           out);
  apply_tick(st);
}

void conv_pad_filters(const float* h, int C, int T, float* h64, cudaStream_t st) {
  launch_k(pad_filters_kernel, dim3((C * kConvMaxT + 255) / 256), dim3(256), 0, st, h, C, T, h64);
}

}  // namespace cofem
