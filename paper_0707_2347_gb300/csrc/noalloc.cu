// An entry point for callers that cannot allocate device memory.
//
// swmm_muladd_noalloc runs the same plans as swmm_muladd, but takes the
// schedule's temporaries and the tensor-core operand staging from a static
// device array instead of the stream-ordered pool.  The array is a
// file-scope __device__ variable, so every device that loads this library
// holds it for the life of the process.  Host code only ever sees a
// host-side stand-in for the array's name; the real device address is
// obtained once per device with cudaGetSymbolAddress, with that device
// current, the first time the entry point runs on it.
#include <cstdint>
#include <mutex>

#include "swmm.h"
#include "swmm_internal.h"

namespace swmm {
int muladd_with_scratch(swmm_t h, int64_t m, int64_t k, int64_t n, const void *alpha, const void *A, int64_t lda,
                        const void *B, int64_t ldb, const void *beta, void *C, int64_t ldc, const swmm_opts *opts,
                        void *scratch, int64_t scratch_bytes);
int handle_device(swmm_t h);
}  // namespace swmm

namespace {

constexpr int64_t kStaticScratchBytes = SWMM_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kStaticScratchBytes];

std::mutex g_lock;
void *g_addr[kMaxDevices] = {nullptr};

// Device address of g_scratch on `dev` (made current for the query).
cudaError_t scratch_address(int dev, void **out) {
  std::lock_guard<std::mutex> guard(g_lock);
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  if (!g_addr[dev]) {
    int prev = 0;
    cudaError_t e = cudaGetDevice(&prev);
    if (e != cudaSuccess) return e;
    if (prev != dev && (e = cudaSetDevice(dev)) != cudaSuccess) return e;
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (prev != dev) cudaSetDevice(prev);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int swmm_muladd_noalloc(swmm_t h, int64_t m, int64_t k, int64_t n, const void *alpha, const void *A,
                                   int64_t lda, const void *B, int64_t ldb, const void *beta, void *C, int64_t ldc,
                                   const swmm_opts *opts) {
  if (!h) return SWMM_EINVAL;
  void *scratch = nullptr;
  if (scratch_address(swmm::handle_device(h), &scratch) != cudaSuccess) {
    cudaGetLastError();
    return SWMM_ECUDA;
  }
  return swmm::muladd_with_scratch(h, m, k, n, alpha, A, lda, B, ldb, beta, C, ldc, opts, scratch,
                                   kStaticScratchBytes);
}
