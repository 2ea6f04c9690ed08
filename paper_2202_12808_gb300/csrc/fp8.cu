// FP8 E4M3 dictionaries with a scale per 128 x 128 tile (the precision
// option of the dense operator): quantisation of an FP32 dictionary and the
// CUDA-core products that run once per fit (beta Phi^T y, the stand-alone
// forward / adjoint, column norms).  The operator of the CG loop runs on the
// tensor cores (dense_tc.cu), whose converter warps expand the same bytes.
//
// Every product applies the entry bf16(e4m3(q) x scale): the FP8 value is
// exact in FP32, the product with the tile's scale is rounded to FP32 and
// then to BF16, both to nearest even, exactly as the tensor-core path's
// converter does, so that all products of a handle use one dictionary.
#include <cuda_fp8.h>

#include "dense.cuh"

namespace cofem {

__device__ __forceinline__ float fp8_entry(const uint8_t* q, const float* scales, int64_t sc,
                                           int64_t ld, int64_t n, int64_t d) {
  const __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)q[n * ld + d], __NV_E4M3);
  const float v = __half2float(*reinterpret_cast<const __half*>(&h));
  return __bfloat162float(__float2bfloat16_rn(v * scales[(n >> 7) * sc + (d >> 7)]));
}

// One block per 128 x 128 tile: the tile's largest magnitude, its scale (the
// smallest power of two s with max |phi| / s <= 448, 1 for an all-zero
// tile), then the bytes e4m3(phi / s) (exact division, rounding to nearest
// even, saturating).
__global__ void fp8_quantize_kernel(const float* __restrict__ phi, int64_t N, int64_t D,
                                    int64_t ld, uint8_t* __restrict__ out, int64_t ldo,
                                    float* __restrict__ scales) {
  pdl_wait();
  pdl_trigger();
  __shared__ float red[32];
  __shared__ float sc_sh;
  const int64_t tm = blockIdx.y, tn = blockIdx.x;
  const int64_t sc_cols = (D + 127) / 128;
  float amax = 0.f;
  for (int i = threadIdx.x; i < 128 * 128; i += blockDim.x) {
    const int64_t n = tm * 128 + i / 128, d = tn * 128 + i % 128;
    if (n < N && d < D) amax = fmaxf(amax, fabsf(phi[n * ld + d]));
  }
  for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = amax;
  __syncthreads();
  if (threadIdx.x == 0) {
    float m = 0.f;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) m = fmaxf(m, red[w]);
    float s = 1.f;
    if (m > 0.f) {
      int e = 0;
      const float f = frexpf(m / 448.f, &e);      // m / 448 = f 2^e, f in [0.5, 1)
      s = ldexpf(1.f, f == 0.5f ? e - 1 : e);
    }
    sc_sh = s;
    scales[tm * sc_cols + tn] = s;
  }
  __syncthreads();
  const float inv = 1.f / sc_sh;                   // a power of two: exact
  for (int i = threadIdx.x; i < 128 * 128; i += blockDim.x) {
    const int64_t n = tm * 128 + i / 128, d = tn * 128 + i % 128;
    if (n < N && d < D)
      out[n * ldo + d] = (uint8_t)__nv_cvt_float_to_fp8(phi[n * ld + d] * inv, __NV_SATFINITE,
                                                         __NV_E4M3);
  }
}

void fp8_quantize_tiles(const float* phi, int64_t N, int64_t D, int64_t ld, uint8_t* out,
                        int64_t ld_out, float* scales, cudaStream_t st) {
  const dim3 g((unsigned)((D + 127) / 128), (unsigned)((N + 127) / 128));
  launch_k(fp8_quantize_kernel, g, dim3(256), 0, st, phi, N, D, ld, out, ld_out, scales);
}

// W[j][n] = sum_d Phi(n, d) Z[j][d]: a block per row n, eight columns per
// pass, FP32 accumulation, block reduction in a fixed order.
__global__ void fp8_forward_kernel(const uint8_t* __restrict__ q, const float* __restrict__ scales,
                                   int64_t N, int64_t D, int64_t ld, const float* __restrict__ Z,
                                   int64_t ldz, int ncols, float* __restrict__ W, int64_t ldw) {
  pdl_wait();
  pdl_trigger();
  __shared__ float red[8][32];
  const int64_t n = blockIdx.x;
  const int64_t sc = (D + 127) / 128;
  for (int j0 = 0; j0 < ncols; j0 += 8) {
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int64_t d = threadIdx.x; d < D; d += blockDim.x) {
      const float a = fp8_entry(q, scales, sc, ld, n, d);
#pragma unroll
      for (int c = 0; c < 8; ++c)
        if (j0 + c < ncols) acc[c] = fmaf(a, Z[(int64_t)(j0 + c) * ldz + d], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      float v = acc[c];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if ((threadIdx.x & 31) == 0) red[c][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < 8 && j0 + (int)threadIdx.x < ncols) {
      float t = 0.f;
      for (int w = 0; w < (int)blockDim.x / 32; ++w) t += red[threadIdx.x][w];
      W[(int64_t)(j0 + threadIdx.x) * ldw + n] = t;
    }
    __syncthreads();
  }
}

// Z[j][d] = beta sum_n Phi(n, d) W[j][n]: a thread per coordinate d (rows
// of Phi read coalesced), eight columns per block (blockIdx.y).
__global__ void fp8_adjoint_kernel(const uint8_t* __restrict__ q, const float* __restrict__ scales,
                                   int64_t N, int64_t D, int64_t ld, const float* __restrict__ W,
                                   int64_t ldw, int ncols, float* __restrict__ Z, int64_t ldz,
                                   double beta) {
  pdl_wait();
  pdl_trigger();
  const int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int j0 = blockIdx.y * 8;
  const int64_t sc = (D + 127) / 128;
  if (d >= D) return;
  float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int64_t n = 0; n < N; ++n) {
    const float a = fp8_entry(q, scales, sc, ld, n, d);
#pragma unroll
    for (int c = 0; c < 8; ++c)
      if (j0 + c < ncols) acc[c] = fmaf(a, W[(int64_t)(j0 + c) * ldw + n], acc[c]);
  }
#pragma unroll
  for (int c = 0; c < 8; ++c)
    if (j0 + c < ncols) Z[(int64_t)(j0 + c) * ldz + d] = (float)(beta * (double)acc[c]);
}

__global__ void fp8_col_norms_kernel(const uint8_t* __restrict__ q, const float* __restrict__ scales,
                                     int64_t N, int64_t D, int64_t ld, float* __restrict__ out) {
  pdl_wait();
  pdl_trigger();
  const int64_t sc = (D + 127) / 128;
  for (int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; d < D;
       d += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int64_t n = 0; n < N; ++n) {
      const double v = fp8_entry(q, scales, sc, ld, n, d);
      acc += v * v;
    }
    out[d] = (float)acc;
  }
}

void fp8_forward(const DenseDesc& op, const float* Z, int64_t ldz, int ncols, float* W,
                 int64_t ldw, cudaStream_t st) {
  launch_k(fp8_forward_kernel, dim3((unsigned)op.N), dim3(256), 0, st, (const uint8_t*)op.phi,
           op.scales, op.N, op.D, op.ld, Z, ldz, ncols, W, ldw);
}

void fp8_adjoint(const DenseDesc& op, const float* W, int64_t ldw, int ncols, float* Z,
                 int64_t ldz, double beta, cudaStream_t st) {
  const dim3 g((unsigned)((op.D + 255) / 256), (unsigned)((ncols + 7) / 8));
  launch_k(fp8_adjoint_kernel, g, dim3(256), 0, st, (const uint8_t*)op.phi, op.scales, op.N, op.D,
           op.ld, W, ldw, ncols, Z, ldz, beta);
}

void fp8_col_norms(const DenseDesc& op, float* out, cudaStream_t st) {
  const int64_t b = (op.D + 255) / 256;
  launch_k(fp8_col_norms_kernel, dim3((unsigned)(b < 4096 ? b : 4096)), dim3(256), 0, st,
           (const uint8_t*)op.phi, op.scales, op.N, op.D, op.ld, out);
}

}  // namespace cofem
