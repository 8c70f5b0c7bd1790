// Randomised residual probe of a product C = alpha A B + beta C_in.
//
// For a random vector x the probe forms r = C x - alpha A (B x) - beta C_in x
// with three matrix-vector products (Freivalds' check).  Over Z/pZ the
// arithmetic is exact: a wrong C gives r = 0 with probability at most 1/p
// per vector.  In FP32 mode the products run in FP64 (the only place the
// library computes in FP64; the product itself never does), so r measures
// the error of C against the exact product applied to x.
//
// matvec_kernel: one warp per matrix row, 16-byte loads along the row when
// the view allows them, an HBM-bound stream over the matrix.  Mod p: the
// elements are reduced to [0, p) (Barrett, m = floor(2^32 / p)), products are
// below 2^32 and each lane sums at most 2^26 of them in 64 bits.
#include <algorithm>
#include <cstdint>

#include "swmm_internal.h"

namespace swmm {
namespace {

constexpr int kRowsPerBlock = 8;

__device__ __forceinline__ uint32_t bred(uint32_t v, uint32_t p, uint32_t m) {
  const uint32_t q = __umulhi(v, m);
  const uint32_t r = v - q * p;
  return min(r, r - p);
}

template <bool MODP, bool VEC>
__global__ void matvec_kernel(const char *M, int64_t rows, int64_t cols, int64_t ld, const void *xv, void *yv,
                              uint32_t p, uint32_t bm) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * kRowsPerBlock;
  for (int64_t r = (int64_t)blockIdx.x * kRowsPerBlock + (threadIdx.x >> 5); r < rows; r += nwarps) {
    const char *row = M + r * ld * 4;
    uint64_t accu = 0;
    double accf = 0.0;
    int64_t j0 = 0;
    if (VEC) {
      const int64_t c4 = cols / 4;
      for (int64_t q = lane; q < c4; q += 32) {
        const uint4 w = *reinterpret_cast<const uint4 *>(row + q * 16);
        const uint32_t e[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          if (MODP)
            accu += (uint64_t)bred(e[i], p, bm) * static_cast<const uint32_t *>(xv)[4 * q + i];
          else
            accf = fma((double)__uint_as_float(e[i]), static_cast<const double *>(xv)[4 * q + i], accf);
        }
      }
      j0 = c4 * 4;
    }
    for (int64_t j = j0 + lane; j < cols; j += 32) {
      const uint32_t e = reinterpret_cast<const uint32_t *>(row)[j];
      if (MODP)
        accu += (uint64_t)bred(e, p, bm) * static_cast<const uint32_t *>(xv)[j];
      else
        accf = fma((double)__uint_as_float(e), static_cast<const double *>(xv)[j], accf);
    }
    if (MODP) {
      accu %= p;  // keep the warp sum far from 2^64
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) accu += __shfl_xor_sync(0xffffffffu, accu, o);
      if (lane == 0) static_cast<uint32_t *>(yv)[r] = (uint32_t)(accu % p);
    } else {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) accf += __shfl_xor_sync(0xffffffffu, accf, o);
      if (lane == 0) static_cast<double *>(yv)[r] = accf;
    }
  }
}

// r = v - alpha u - beta y0 (y0 may be null: beta term absent)
template <bool MODP>
__global__ void residual_kernel(int64_t m, const void *v, const void *u, const void *y0, void *r, uint32_t au,
                                uint32_t bu, double af, double bf, uint32_t p) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    if (MODP) {
      const uint64_t vi = static_cast<const uint32_t *>(v)[i] % p;
      const uint64_t ui = (uint64_t)au * (static_cast<const uint32_t *>(u)[i] % p) % p;
      const uint64_t yi = y0 ? (uint64_t)bu * (static_cast<const uint32_t *>(y0)[i] % p) % p : 0;
      static_cast<uint32_t *>(r)[i] = (uint32_t)((vi + 2 * (uint64_t)p - ui - yi) % p);
    } else {
      double x = static_cast<const double *>(v)[i] - af * static_cast<const double *>(u)[i];
      if (y0) x -= bf * static_cast<const double *>(y0)[i];
      static_cast<double *>(r)[i] = x;
    }
  }
}

}  // namespace

cudaError_t launch_matvec(const void *M, int64_t rows, int64_t cols, int64_t ld, const void *x, void *y, uint32_t p,
                          bool modp, int num_sms, cudaStream_t s) {
  if (rows <= 0) return cudaSuccess;
  const bool vec = ((uintptr_t)M % 16 == 0) && (ld % 4 == 0);
  const int64_t want = (rows + kRowsPerBlock - 1) / kRowsPerBlock;
  const int grid = (int)std::min<int64_t>(want, (int64_t)num_sms * 8);
  const uint32_t bm = modp ? (uint32_t)(0x100000000ull / p) : 0;
  const char *Mc = static_cast<const char *>(M);
  if (modp) {
    if (vec)
      matvec_kernel<true, true><<<grid, 32 * kRowsPerBlock, 0, s>>>(Mc, rows, cols, ld, x, y, p, bm);
    else
      matvec_kernel<true, false><<<grid, 32 * kRowsPerBlock, 0, s>>>(Mc, rows, cols, ld, x, y, p, bm);
  } else {
    if (vec)
      matvec_kernel<false, true><<<grid, 32 * kRowsPerBlock, 0, s>>>(Mc, rows, cols, ld, x, y, p, bm);
    else
      matvec_kernel<false, false><<<grid, 32 * kRowsPerBlock, 0, s>>>(Mc, rows, cols, ld, x, y, p, bm);
  }
  return cudaGetLastError();
}

cudaError_t launch_residual(int64_t m, const void *v, const void *u, const void *y0, void *r, uint32_t au,
                            uint32_t bu, double af, double bf, uint32_t p, bool modp, int num_sms, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  const int grid = (int)std::min<int64_t>((m + 255) / 256, (int64_t)num_sms * 4);
  if (modp)
    residual_kernel<true><<<grid, 256, 0, s>>>(m, v, u, y0, r, au, bu, af, bf, p);
  else
    residual_kernel<false><<<grid, 256, 0, s>>>(m, v, u, y0, r, au, bu, af, bf, p);
  return cudaGetLastError();
}

}  // namespace swmm
