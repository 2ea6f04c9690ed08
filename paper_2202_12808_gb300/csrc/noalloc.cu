// cofem_op_apply_noalloc: the operator application A X of cofem_op_apply,
// for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc (or hand out a workspace) at the time
// they apply the operator: a plugin running inside a host application that
// owns every byte of the device memory pool and forbids allocation after
// start-up, or a latency-critical loop where an allocation would synchronise
// the device.  For them this entry point takes its scratch from one array
// compiled into the library, so the caller passes only inputs and outputs.
//
// The array is a file-scope __device__ array of kNoAllocScratchBytes.  Every
// GPU that loads the library holds it until the process exits.  All calls on
// a device share it and it keeps whatever the last call left there: the
// kernels write every scratch entry they later read, so nothing needs to
// start at zero, but two calls whose work overlaps on the GPU (different
// streams, or host threads without ordering) race on it and give wrong
// results.  Host code cannot use the array's name as a device address: the
// first call on each device looks the address up with cudaGetSymbolAddress
// (with that device current) and caches it; make that first call before any
// stream capture.  The cache lives as long as the process: a
// cudaDeviceReset of the device would leave it stale, so no call may follow
// a reset.
#include <cstdio>
#include <mutex>

#include "kernels.cuh"

namespace cofem {
cofem_status apply_check(const cofem_op* op, cofem_dtype vec, int32_t ncols, int64_t ld);
size_t apply_scratch_bytes(const cofem_op* op, cofem_dtype vec, int32_t ncols);
cofem_status apply_with_scratch(const cofem_op* op, cofem_dtype vec, const void* x, int64_t ld,
                                int32_t ncols, const double* alpha, double beta, void* y,
                                char* scratch, cudaStream_t st);
void set_last_error(const char* msg);
}  // namespace cofem

static constexpr size_t kNoAllocScratchBytes = (size_t)16 << 20;   // 16 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[128] = {nullptr};

// Device address of the scratch array on the current device (looked up once).
static cofem_status noalloc_scratch(char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) {
    cofem::set_last_error("cofem_op_apply_noalloc: no current CUDA device");
    return COFEM_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      char buf[256];
      snprintf(buf, sizeof(buf), "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
      cofem::set_last_error(buf);
      return COFEM_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = p;
  }
  *out = (char*)g_noalloc_ptr[dev];
  return COFEM_OK;
}

extern "C" size_t cofem_noalloc_scratch_capacity(void) { return kNoAllocScratchBytes; }

extern "C" cofem_status cofem_op_apply_noalloc(const cofem_op* op, cofem_dtype vec,
                                               const void* x_dev, int64_t ld, int32_t ncols,
                                               const double* alpha_dev, double beta,
                                               void* y_dev, void* stream) {
  cofem_status rc = cofem::apply_check(op, vec, ncols, ld);
  if (rc != COFEM_OK) return rc;
  if (!x_dev || !y_dev || !alpha_dev) return COFEM_ERR_INVALID_ARG;
  const size_t need = cofem::apply_scratch_bytes(op, vec, ncols);
  if (need > kNoAllocScratchBytes) {
    char buf[256];
    snprintf(buf, sizeof(buf),
             "cofem_op_apply_noalloc: this operator and column count need %zu bytes of scratch; "
             "the library's static scratch holds %zu",
             need, kNoAllocScratchBytes);
    cofem::set_last_error(buf);
    return COFEM_ERR_WORKSPACE;
  }
  char* scratch = nullptr;
  rc = noalloc_scratch(&scratch);
  if (rc != COFEM_OK) return rc;
  return cofem::apply_with_scratch(op, vec, x_dev, ld, ncols, alpha_dev, beta, y_dev, scratch,
                                   (cudaStream_t)stream);
}
