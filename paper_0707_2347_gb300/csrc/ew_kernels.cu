// Elementwise kernels of the schedules: the block additions of Tables 1-9
// (the 8 pre-additions S1..S4, T1..T4 of Section 2, the post-additions
// U1..U7, and the schedule-specific Z1, Z2, Z3, W1 rows), plus the
// prologue/epilogue passes of a fused Winograd level.
//
// All are HBM-bound streams over strided 2-D blocks: one thread handles four
// consecutive elements with 16-byte loads/stores when the views allow it
// (base 16-byte aligned, ld and cols multiples of 4), else one element.
// Inputs mod p may be any representative below 2^32 (a fused Winograd level
// leaves unreduced sums in its destination): every input is first reduced
// with a Barrett step using m = floor(2^32 / p); outputs are canonical in
// [0, p).
#include <cstdint>

#include "swmm_internal.h"

namespace swmm {
namespace {

struct V {
  char *ptr;
  int64_t ld;
  int esz;  // 4: 32-bit elements; 2: 16-bit values in [0, p)
};

// four consecutive elements from column c of row r (16-byte / 8-byte loads)
__device__ __forceinline__ uint4 ld4(const V &v, int64_t r, int64_t c) {
  if (v.esz == 4) return *reinterpret_cast<const uint4 *>(v.ptr + 4 * (r * v.ld + c));
  const uint2 h = *reinterpret_cast<const uint2 *>(v.ptr + 2 * (r * v.ld + c));
  return make_uint4(h.x & 0xFFFFu, h.x >> 16, h.y & 0xFFFFu, h.y >> 16);
}
__device__ __forceinline__ void st4(const V &v, int64_t r, int64_t c, uint4 o) {
  if (v.esz == 4) {
    *reinterpret_cast<uint4 *>(v.ptr + 4 * (r * v.ld + c)) = o;
  } else {
    *reinterpret_cast<uint2 *>(v.ptr + 2 * (r * v.ld + c)) = make_uint2(o.x | (o.y << 16), o.z | (o.w << 16));
  }
}
__device__ __forceinline__ uint32_t ld1(const V &v, int64_t r, int64_t c) {
  if (v.esz == 4) return *reinterpret_cast<const uint32_t *>(v.ptr + 4 * (r * v.ld + c));
  return *reinterpret_cast<const uint16_t *>(v.ptr + 2 * (r * v.ld + c));
}
__device__ __forceinline__ void st1(const V &v, int64_t r, int64_t c, uint32_t x) {
  if (v.esz == 4)
    *reinterpret_cast<uint32_t *>(v.ptr + 4 * (r * v.ld + c)) = x;
  else
    *reinterpret_cast<uint16_t *>(v.ptr + 2 * (r * v.ld + c)) = (uint16_t)x;
}

__device__ __forceinline__ uint32_t red2p(uint32_t r, uint32_t p) {
  // r in [0, 2p) -> [0, p): the wrapped r - p is huge when r < p
  return min(r, r - p);
}

__device__ __forceinline__ uint32_t mulmod(uint32_t u, uint32_t x, uint32_t p, uint32_t m) {
  uint32_t prod = u * x;  // u, x < p < 2^16
  uint32_t q = __umulhi(prod, m);
  return red2p(prod - q * p, p);
}

// any 32-bit representative -> [0, p)
__device__ __forceinline__ uint32_t bred(uint32_t x, uint32_t p, uint32_t m) {
  uint32_t q = __umulhi(x, m);
  return red2p(x - q * p, p);
}

// coefficient classes: 0 = +1, 1 = -1, 2 = general u
template <int K1, int K2>
__device__ __forceinline__ uint32_t comb(uint32_t a, uint32_t b, uint32_t u1, uint32_t u2, uint32_t p,
                                         uint32_t m) {
  a = bred(a, p, m);
  b = bred(b, p, m);
  uint32_t x = (K1 == 0) ? a : (K1 == 1 ? (p - a) : mulmod(u1, a, p, m));
  uint32_t y = (K2 == 0) ? b : (K2 == 1 ? (p - b) : mulmod(u2, b, p, m));
  // x in [0, p], y in [0, p]: x + y < 2p + 1; p - 0 = p is reduced too
  uint32_t r = x + y;
  r = red2p(r, p);
  return red2p(r, p);
}

template <int K1, int K2, bool VEC>
__global__ void add_modp_kernel(V d, V s1, V s2, int64_t rows, int64_t cols, uint32_t u1, uint32_t u2,
                                uint32_t p, uint32_t m) {
  const int64_t cw = VEC ? cols / 4 : cols;
  const int64_t total = rows * cw;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = i / cw, c = i - r * cw;
    if (VEC) {
      const uint4 a = ld4(s1, r, 4 * c);
      const uint4 b = ld4(s2, r, 4 * c);
      uint4 o;
      o.x = comb<K1, K2>(a.x, b.x, u1, u2, p, m);
      o.y = comb<K1, K2>(a.y, b.y, u1, u2, p, m);
      o.z = comb<K1, K2>(a.z, b.z, u1, u2, p, m);
      o.w = comb<K1, K2>(a.w, b.w, u1, u2, p, m);
      st4(d, r, 4 * c, o);
    } else {
      st1(d, r, c, comb<K1, K2>(ld1(s1, r, c), ld1(s2, r, c), u1, u2, p, m));
    }
  }
}

template <bool VEC>
__global__ void add_f32_kernel(V d, V s1, V s2, int64_t rows, int64_t cols, float c1, float c2) {
  const int64_t cw = VEC ? cols / 4 : cols;
  const int64_t total = rows * cw;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = i / cw, c = i - r * cw;
    if (VEC) {
      const float4 a = *reinterpret_cast<const float4 *>(s1.ptr + 4 * (r * s1.ld + 4 * c));
      const float4 b = *reinterpret_cast<const float4 *>(s2.ptr + 4 * (r * s2.ld + 4 * c));
      float4 o;
      o.x = c1 * a.x + c2 * b.x;
      o.y = c1 * a.y + c2 * b.y;
      o.z = c1 * a.z + c2 * b.z;
      o.w = c1 * a.w + c2 * b.w;
      *reinterpret_cast<float4 *>(d.ptr + 4 * (r * d.ld + 4 * c)) = o;
    } else {
      float a = *reinterpret_cast<const float *>(s1.ptr + 4 * (r * s1.ld + c));
      float b = *reinterpret_cast<const float *>(s2.ptr + 4 * (r * s2.ld + c));
      *reinterpret_cast<float *>(d.ptr + 4 * (r * d.ld + c)) = c1 * a + c2 * b;
    }
  }
}

// mode 2: float *= coef (coef 0 writes 0); mode 3: int mod p *= coef;
// mode 4: int mod p reduced to [0, p)
template <int MODE, bool VEC>
__global__ void convert_kernel(V d, int64_t rows, int64_t cols, uint32_t coef, float fcoef, uint32_t p,
                               uint32_t m) {
  const int64_t cw = VEC ? cols / 4 : cols;
  const int64_t total = rows * cw;
  auto f = [&](uint32_t x) -> uint32_t {
    if (MODE == 2) {
      return __float_as_uint(fcoef == 0.f ? 0.f : fcoef * __uint_as_float(x));
    } else if (MODE == 3) {
      return coef == 0 ? 0u : mulmod(coef, bred(x, p, m), p, m);
    } else {
      return bred(x, p, m);
    }
  };
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = i / cw, c = i - r * cw;
    if (VEC) {
      uint4 *ptr = reinterpret_cast<uint4 *>(d.ptr + 4 * (r * d.ld + 4 * c));
      uint4 a = *ptr;
      a.x = f(a.x);
      a.y = f(a.y);
      a.z = f(a.z);
      a.w = f(a.w);
      *ptr = a;
    } else {
      uint32_t *ptr = reinterpret_cast<uint32_t *>(d.ptr + 4 * (r * d.ld + c));
      *ptr = f(*ptr);
    }
  }
}

// four elements per access: 16 (32-bit) or 8 (16-bit) aligned bytes
bool vec_ok(const View &v) {
  return ((uintptr_t)v.ptr % (4 * v.esz) == 0) && (v.ld % 4 == 0) && (v.cols % 4 == 0);
}

void grid_for(int64_t work, int &blocks, int &threads) {
  threads = 256;
  int64_t b = (work + threads - 1) / threads;
  // enough CTAs to fill 152 SMs several times; the loops are grid-stride
  const int64_t cap = 152 * 16;
  blocks = (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

V mk(const View &v) { return V{v.ptr, v.ld, v.esz}; }

// d <- s element by element, between 32-bit and 16-bit storage (a 16-bit
// destination receives the value reduced to [0, p))
__global__ void copy_kernel(V d, V s, int64_t rows, int64_t cols, uint32_t p, uint32_t m) {
  const int64_t total = rows * cols;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / cols, c = i - r * cols;
    const uint32_t x = ld1(s, r, c);
    st1(d, r, c, d.esz == 2 ? bred(x, p, m) : x);
  }
}

template <int K1, int K2>
cudaError_t add_dispatch_vec(View d, View s1, View s2, uint32_t u1, uint32_t u2, uint32_t p, cudaStream_t s) {
  uint32_t m = (uint32_t)(0x100000000ull / p);
  bool vec = vec_ok(d) && vec_ok(s1) && vec_ok(s2);
  int b, t;
  grid_for(vec ? d.rows * d.cols / 4 : d.rows * d.cols, b, t);
  if (vec)
    add_modp_kernel<K1, K2, true><<<b, t, 0, s>>>(mk(d), mk(s1), mk(s2), d.rows, d.cols, u1, u2, p, m);
  else
    add_modp_kernel<K1, K2, false><<<b, t, 0, s>>>(mk(d), mk(s1), mk(s2), d.rows, d.cols, u1, u2, p, m);
  return cudaGetLastError();
}

int klass(uint32_t u, uint32_t p) { return u == 1 ? 0 : (u == p - 1 ? 1 : 2); }

}  // namespace

cudaError_t launch_add(View d, View s1, View s2, int64_t c1, int64_t c2, uint32_t p, int fp32,
                       cudaStream_t s) {
  if (d.rows == 0 || d.cols == 0) return cudaSuccess;
  if (fp32) return launch_add_f(d, s1, s2, (float)c1, (float)c2, s);
  uint32_t u1 = (uint32_t)(((c1 % (int64_t)p) + p) % p);
  uint32_t u2 = (uint32_t)(((c2 % (int64_t)p) + p) % p);
  int k1 = klass(u1, p), k2 = klass(u2, p);
#define SWMM_ADD_CASE(A, B) \
  if (k1 == A && k2 == B) return add_dispatch_vec<A, B>(d, s1, s2, u1, u2, p, s);
  SWMM_ADD_CASE(0, 0)
  SWMM_ADD_CASE(0, 1)
  SWMM_ADD_CASE(1, 0)
  SWMM_ADD_CASE(1, 1)
  SWMM_ADD_CASE(0, 2)
  SWMM_ADD_CASE(2, 0)
  SWMM_ADD_CASE(1, 2)
  SWMM_ADD_CASE(2, 1)
  SWMM_ADD_CASE(2, 2)
#undef SWMM_ADD_CASE
  return cudaErrorInvalidValue;
}

cudaError_t launch_add_f(View d, View s1, View s2, float c1, float c2, cudaStream_t s) {
  if (d.rows == 0 || d.cols == 0) return cudaSuccess;
  bool vec = vec_ok(d) && vec_ok(s1) && vec_ok(s2);
  int b, t;
  grid_for(vec ? d.rows * d.cols / 4 : d.rows * d.cols, b, t);
  if (vec)
    add_f32_kernel<true><<<b, t, 0, s>>>(mk(d), mk(s1), mk(s2), d.rows, d.cols, c1, c2);
  else
    add_f32_kernel<false><<<b, t, 0, s>>>(mk(d), mk(s1), mk(s2), d.rows, d.cols, c1, c2);
  return cudaGetLastError();
}

template <int MODE>
static cudaError_t conv(View d, uint32_t coef, float fcoef, uint32_t p, cudaStream_t s) {
  if (d.rows == 0 || d.cols == 0) return cudaSuccess;
  uint32_t m = p ? (uint32_t)(0x100000000ull / p) : 0;
  bool vec = vec_ok(d);
  int b, t;
  grid_for(vec ? d.rows * d.cols / 4 : d.rows * d.cols, b, t);
  if (vec)
    convert_kernel<MODE, true><<<b, t, 0, s>>>(mk(d), d.rows, d.cols, coef, fcoef, p, m);
  else
    convert_kernel<MODE, false><<<b, t, 0, s>>>(mk(d), d.rows, d.cols, coef, fcoef, p, m);
  return cudaGetLastError();
}

cudaError_t launch_scale_f(View d, float coef, cudaStream_t s) { return conv<2>(d, 0, coef, 0, s); }
cudaError_t launch_scale_modp(View d, uint32_t coef, uint32_t p, cudaStream_t s) {
  return conv<3>(d, coef % p, 0.f, p, s);
}
cudaError_t launch_canon_modp(View d, uint32_t p, cudaStream_t s) { return conv<4>(d, 0, 0.f, p, s); }
cudaError_t launch_zero(View d, cudaStream_t s) {
  if (d.rows == 0 || d.cols == 0) return cudaSuccess;
  return cudaMemset2DAsync(d.ptr, d.ld * d.esz, 0, d.cols * d.esz, d.rows, s);
}

cudaError_t launch_copy(View d, View src, uint32_t p, cudaStream_t s) {
  if (d.rows == 0 || d.cols == 0) return cudaSuccess;
  if (d.esz == src.esz)
    return cudaMemcpy2DAsync(d.ptr, d.ld * d.esz, src.ptr, src.ld * src.esz, d.cols * d.esz, d.rows,
                             cudaMemcpyDeviceToDevice, s);
  if (p == 0) return cudaErrorInvalidValue;  // 16-bit storage is mod p only
  int b, t;
  grid_for(d.rows * d.cols, b, t);
  copy_kernel<<<b, t, 0, s>>>(mk(d), mk(src), d.rows, d.cols, p, (uint32_t)(0x100000000ull / p));
  return cudaGetLastError();
}

}  // namespace swmm
