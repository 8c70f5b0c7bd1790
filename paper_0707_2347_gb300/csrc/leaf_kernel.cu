// Leaf products of the Strassen-Winograd recursion on the sm_103a tensor
// cores (tcgen05 MMA, accumulators in tensor memory, operands staged by TMA).
//
// pack_* : operand staging.  One launch reads the four quadrants of a
//   Winograd level's operand once and writes the seven signed combinations
//   the level multiplies (A11, A12, S4, A22, S1, S2, S3 or B11, B21, B22,
//   T4, T1, T2, T3, Section 2), already in the tensor-core number format, so
//   the pre-additions never exist as int32/float blocks in HBM.  Exact
//   arithmetic over Z/pZ on the floating-point tensor pipe (sm_103a has no
//   integer tcgen05 MMA): each entry is brought to a centred representative
//   and split into fp16 limbs of magnitude <= 128 (one limb when p <= 256,
//   x = 256 h + l when p < 2^16); fp16 holds these integers exactly.  FP32
//   mode scales each operand by a power of two (from its max |x|, amax_*)
//   and splits x s into fp16 hi + lo.
//
// gemm_* : persistent warp-specialised GEMM over up to seven products (one
//   fused Winograd level, or one classical leaf).  Warp 0 issues TMA loads
//   of 128-byte-swizzled K-major tiles into a shared-memory ring, warp 1
//   allocates tensor memory and issues tcgen05.mma from one thread, warps
//   2-9 drain the accumulators.  Limb products are <= 2^14 in magnitude, so
//   an fp32 accumulator summing at most 1024 of them stays below 2^24 and is
//   exact; longer K is reduced mod p in place in tensor memory every 960 K.
//   The epilogue recombines 2^16 hh + 2^8 (hl + lh) + ll mod p with exact
//   fp32 operations (FP32 mode: hi hi + hi lo + lo hi, unscaled), applies
//   alpha / beta, and either stores (one target) or adds its signed
//   contribution into up to four targets with TMA reductions (the
//   post-additions U1..U7 of a fused level).
// Every mbarrier wait is bounded (globaltimer); on expiry the kernel sets the
// error word and unwinds, freeing its tensor memory.
#include <cstdint>
#include <cuda_fp16.h>

#include "swmm_internal.h"

namespace swmm {
namespace dev {

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// ---------------------------------------------------------- conversions
// x in [0, p) -> u = c + 32896 with c = x (mod p), c in [-32896, 32895]
__device__ __forceinline__ uint32_t centre16(uint32_t x, uint32_t p) {
  uint32_t t = x + 32896u;
  return __viaddmin_u32(t, 0u - p, t);  // the wrapped t - p is huge unless x >= p - 32896
}
// x in [0, p), p <= 256 -> u = c + 128 with c = x (mod p), c in [-128, 127]
__device__ __forceinline__ uint32_t centre8(uint32_t x, uint32_t p) {
  uint32_t t = x + 128u;
  return __viaddmin_u32(t, 0u - p, t);
}
__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
  uint32_t d;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
  return d;
}
// two offset values v in [0, 256] in the 16-bit halves -> fp16x2 of v - 128:
// 0x6400 | v is the fp16 of 1024 + v, and 1024 + v - 1152 is exact.
__device__ __forceinline__ uint32_t offset_to_h2(uint32_t packed) {
  uint32_t h = packed | 0x64006400u;
  __half2 r = __hsub2(*reinterpret_cast<__half2 *>(&h), __halves2half2(__ushort_as_half(0x6480), __ushort_as_half(0x6480)));
  return *reinterpret_cast<uint32_t *>(&r);
}
// x in [0, 4p] -> [0, p)
__device__ __forceinline__ uint32_t red4p(uint32_t x, uint32_t p) {
  x = min(x, x - 2 * p);  // [0, 2p]
  x = min(x, x - p);      // [0, p]
  return min(x, x - p);
}

// N (even) combined values -> N/2 words of plane 0 and of plane 1
template <int MODE, int N>
__device__ __forceinline__ void convert_n(const uint32_t (&x)[N], uint32_t p, float fs, uint32_t (&w0)[N / 2],
                                          uint32_t (&w1)[N / 2]) {
#pragma unroll
  for (int j = 0; j < N / 2; ++j) {
    if (MODE == MODE_MODP2) {
      uint32_t u0 = centre16(x[2 * j], p), u1 = centre16(x[2 * j + 1], p);
      w0[j] = offset_to_h2(prmt(u0, u1, 0x6521u));               // h + 128 = u >> 8
      w1[j] = offset_to_h2(prmt(u0, u1, 0x4400u) & 0x00FF00FFu);  // l + 128 = u & 255
    } else if (MODE == MODE_MODP1) {
      uint32_t u0 = centre8(x[2 * j], p), u1 = centre8(x[2 * j + 1], p);
      w0[j] = offset_to_h2(prmt(u0, u1, 0x4400u) & 0x00FF00FFu);
      w1[j] = 0;
    } else {
      // scaled value v = x fs (|v| < 2^14): hi = fp16(v), lo = fp16(v - hi);
      // hi + lo carries 22 significant bits of v
      const float a = __uint_as_float(x[2 * j]) * fs, b = __uint_as_float(x[2 * j + 1]) * fs;
      const __half2 hi = __floats2half2_rn(a, b);
      const float2 hf = __half22float2(hi);
      const __half2 lo = __floats2half2_rn(a - hf.x, b - hf.y);
      w0[j] = *reinterpret_cast<const uint32_t *>(&hi);
      w1[j] = *reinterpret_cast<const uint32_t *>(&lo);
    }
  }
}

// 8 combined values -> plane 0 and plane 1 (16 bytes each)
template <int MODE>
__device__ __forceinline__ void convert8(const uint32_t (&x)[8], uint32_t p, float fs, uint4 &o0, uint4 &o1) {
  uint32_t w0[4], w1[4];
  convert_n<MODE, 8>(x, p, fs, w0, w1);
  o0 = make_uint4(w0[0], w0[1], w0[2], w0[3]);
  o1 = make_uint4(w1[0], w1[1], w1[2], w1[3]);
}

// 2 combined values -> plane 0 and plane 1 (4 bytes each)
template <int MODE>
__device__ __forceinline__ void emit2(const uint32_t (&x)[2], uint32_t p, float fs, uint16_t *dst, int64_t plane) {
  uint32_t w0[1], w1[1];
  convert_n<MODE, 2>(x, p, fs, w0, w1);
  *reinterpret_cast<uint32_t *>(dst) = w0[0];
  if (MODE != MODE_MODP1) *reinterpret_cast<uint32_t *>(dst + plane) = w1[0];
}

// 4 combined values -> plane 0 and plane 1 (8 bytes each)
template <int MODE>
__device__ __forceinline__ void emit4(const uint32_t (&x)[4], uint32_t p, float fs, uint16_t *dst, int64_t plane) {
  uint32_t w0[2], w1[2];
  convert_n<MODE, 4>(x, p, fs, w0, w1);
  *reinterpret_cast<uint2 *>(dst) = make_uint2(w0[0], w0[1]);
  if (MODE != MODE_MODP1) *reinterpret_cast<uint2 *>(dst + plane) = make_uint2(w1[0], w1[1]);
}

// Bring a raw source value to the representative the combinations use:
// mod p any 32-bit representative -> [0, p) (Barrett, m = floor(2^32 / p));
// FP32 unchanged.
template <int MODE>
__device__ __forceinline__ uint32_t source_value(uint32_t x, uint32_t p, uint32_t m) {
  if (MODE == MODE_FP32) return x;
  uint32_t r = x - __umulhi(x, m) * p;
  return min(r, r - p);
}

// signed combination sum_q coef[o][q] * v[q] of reduced source values
template <int MODE>
__device__ __forceinline__ uint32_t combine(const PackArgs &a, int o, const uint32_t *v, uint32_t p) {
  if (MODE == MODE_FP32) {
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < kMaxSrc; ++q) {
      const int c = a.coef[o][q];
      if (c > 0) s += __uint_as_float(v[q]);
      if (c < 0) s -= __uint_as_float(v[q]);
    }
    return __float_as_uint(s);
  } else {
    uint32_t s = 0;
#pragma unroll
    for (int q = 0; q < kMaxSrc; ++q) {
      const int c = a.coef[o][q];
      if (c > 0) s += v[q];
      if (c < 0) s += p - v[q];
    }
    return red4p(s, p);
  }
}

// write output o of one 8-element unit: plane 0 and plane 1
template <int MODE>
__device__ __forceinline__ void emit_unit(const PackArgs &a, int o, const uint32_t (&v)[kMaxSrc][8], uint16_t *dst,
                                          int64_t plane, float fs) {
  uint32_t x[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    uint32_t w[kMaxSrc];
#pragma unroll
    for (int q = 0; q < kMaxSrc; ++q) w[q] = v[q][e];
    x[e] = combine<MODE>(a, o, w, a.p);
  }
  uint4 o0, o1;
  convert8<MODE>(x, a.p, fs, o0, o1);
  *reinterpret_cast<uint4 *>(dst) = o0;
  if (MODE != MODE_MODP1) *reinterpret_cast<uint4 *>(dst + plane) = o1;
}

// one 8-element unit of already combined values -> plane 0 and plane 1
template <int MODE>
__device__ __forceinline__ void emit8(const uint32_t (&x)[8], uint32_t p, float fs, uint16_t *dst, int64_t plane) {
  uint4 o0, o1;
  convert8<MODE>(x, p, fs, o0, o1);
  *reinterpret_cast<uint4 *>(dst) = o0;
  if (MODE != MODE_MODP1) *reinterpret_cast<uint4 *>(dst + plane) = o1;
}

// x - y of two reduced values (mod p: both in [0, p), result in [0, p))
template <int MODE>
__device__ __forceinline__ uint32_t lin_sub(uint32_t x, uint32_t y, uint32_t p) {
  if (MODE == MODE_FP32) return __float_as_uint(__uint_as_float(x) - __uint_as_float(y));
  const uint32_t r = x + p - y;
  return min(r, r - p);
}
template <int MODE>
__device__ __forceinline__ uint32_t lin_add(uint32_t x, uint32_t y, uint32_t p) {
  if (MODE == MODE_FP32) return __float_as_uint(__uint_as_float(x) + __uint_as_float(y));
  const uint32_t r = x + y;
  return min(r, r - p);
}

// every output of one unit (sources already reduced); v[q] = quadrant q of
// (X11, X12, X21, X22) for the Winograd sets
template <int MODE, int SET>
__device__ __forceinline__ void emit_all(const PackArgs &a, const uint32_t (&v)[kMaxSrc][8], int64_t off,
                                         int64_t plane, float fs) {
  const uint32_t p = a.p;
  if (SET == PACK_WINOGRAD_A) {
    uint32_t s1[8], s2[8], t[8];
    emit8<MODE>(v[0], p, fs, a.out[0] + off, plane);  // A11
    emit8<MODE>(v[1], p, fs, a.out[1] + off, plane);  // A12
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      s1[e] = lin_add<MODE>(v[2][e], v[3][e], p);  // S1 = A21 + A22
      s2[e] = lin_sub<MODE>(s1[e], v[0][e], p);    // S2 = S1 - A11
      t[e] = lin_sub<MODE>(v[1][e], s2[e], p);     // S4 = A12 - S2
    }
    emit8<MODE>(t, p, fs, a.out[2] + off, plane);
    emit8<MODE>(v[3], p, fs, a.out[3] + off, plane);  // A22
    emit8<MODE>(s1, p, fs, a.out[4] + off, plane);
    emit8<MODE>(s2, p, fs, a.out[5] + off, plane);
#pragma unroll
    for (int e = 0; e < 8; ++e) t[e] = lin_sub<MODE>(v[0][e], v[2][e], p);  // S3 = A11 - A21
    emit8<MODE>(t, p, fs, a.out[6] + off, plane);
  } else if (SET == PACK_WINOGRAD_B) {
    uint32_t t1[8], t2[8], t[8];
    emit8<MODE>(v[0], p, fs, a.out[0] + off, plane);  // B11
    emit8<MODE>(v[2], p, fs, a.out[1] + off, plane);  // B21
    emit8<MODE>(v[3], p, fs, a.out[2] + off, plane);  // B22
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      t1[e] = lin_sub<MODE>(v[1][e], v[0][e], p);  // T1 = B12 - B11
      t2[e] = lin_sub<MODE>(v[3][e], t1[e], p);    // T2 = B22 - T1
      t[e] = lin_sub<MODE>(t2[e], v[2][e], p);     // T4 = T2 - B21
    }
    emit8<MODE>(t, p, fs, a.out[3] + off, plane);
    emit8<MODE>(t1, p, fs, a.out[4] + off, plane);
    emit8<MODE>(t2, p, fs, a.out[5] + off, plane);
#pragma unroll
    for (int e = 0; e < 8; ++e) t[e] = lin_sub<MODE>(v[3][e], v[1][e], p);  // T3 = B22 - B12
    emit8<MODE>(t, p, fs, a.out[6] + off, plane);
  } else {
    for (int o = 0; o < a.nout; ++o) emit_unit<MODE>(a, o, v, a.out[o] + off, plane, fs);
  }
}

// n consecutive elements (n = 8, 4 or 2) of row r from column c of one block of
// 32-bit (esz 4) or 16-bit (esz 2) elements; 0 outside rows x cols; vector
// loads when aligned
template <int N>
__device__ __forceinline__ void load_row(const char *blk, int64_t ld, int r, int c, int rows, int cols, uint32_t *w,
                                         int esz) {
  const char *base = blk + esz * ((int64_t)r * ld + c);
  if (esz == 2) {
    if (r < rows && c + N <= cols && ((uintptr_t)base & (2 * N - 1)) == 0) {
      uint32_t h[N / 2];
      if constexpr (N == 8) {
        const uint4 x = *reinterpret_cast<const uint4 *>(base);
        h[0] = x.x;
        h[1] = x.y;
        h[2] = x.z;
        h[3] = x.w;
      } else if constexpr (N == 4) {
        const uint2 x = *reinterpret_cast<const uint2 *>(base);
        h[0] = x.x;
        h[1] = x.y;
      } else {
        h[0] = *reinterpret_cast<const uint32_t *>(base);
      }
#pragma unroll
      for (int i = 0; i < N / 2; ++i) {
        w[2 * i] = h[i] & 0xFFFFu;
        w[2 * i + 1] = h[i] >> 16;
      }
    } else {
#pragma unroll
      for (int e = 0; e < N; ++e)
        w[e] = (r < rows && c + e < cols) ? (uint32_t) reinterpret_cast<const uint16_t *>(base)[e] : 0u;
    }
    return;
  }
  if (N == 2 && r < rows && c + N <= cols && ((uintptr_t)base & 7) == 0) {
    const uint2 x = *reinterpret_cast<const uint2 *>(base);
    w[0] = x.x;
    w[1] = x.y;
  } else if (N >= 4 && r < rows && c + N <= cols && ((uintptr_t)base & 15) == 0) {
#pragma unroll
    for (int i = 0; i < N / 4; ++i) {
      const uint4 x = *reinterpret_cast<const uint4 *>(base + 16 * i);
      w[4 * i] = x.x;
      w[4 * i + 1] = x.y;
      w[4 * i + 2] = x.z;
      w[4 * i + 3] = x.w;
    }
  } else {
#pragma unroll
    for (int e = 0; e < N; ++e) w[e] = (r < rows && c + e < cols) ? reinterpret_cast<const uint32_t *>(base)[e] : 0u;
  }
}

// source q at (r, c..c+N): sum_t tsign[t] * term t, every term reduced first
template <int MODE, int N>
__device__ __forceinline__ void load_source(const PackArgs &a, int q, int r, int c, uint32_t *v) {
  load_row<N>(a.src[q][0], a.ld[q][0], r, c, a.rows, a.cols, v, a.tesz[0]);
#pragma unroll
  for (int e = 0; e < N; ++e) v[e] = source_value<MODE>(v[e], a.p, a.barrett);
  if (a.nterm == 1 && a.tsign[0] > 0) return;  // one plain block (every launch but symbolic sums)
  if (a.tsign[0] < 0) {
#pragma unroll
    for (int e = 0; e < N; ++e) v[e] = lin_sub<MODE>(MODE == MODE_FP32 ? __float_as_uint(0.f) : 0u, v[e], a.p);
  }
  for (int t = 1; t < a.nterm; ++t) {
    uint32_t w[N];
    load_row<N>(a.src[q][t], a.ld[q][t], r, c, a.rows, a.cols, w, a.tesz[t]);
#pragma unroll
    for (int e = 0; e < N; ++e) {
      const uint32_t x = source_value<MODE>(w[e], a.p, a.barrett);
      v[e] = a.tsign[t] > 0 ? lin_add<MODE>(v[e], x, a.p) : lin_sub<MODE>(v[e], x, a.p);
    }
  }
}

// ------------------------------------------------------------------ pack
// plain layout: thread = 8 consecutive columns of one row; every source
// value is loaded and reduced once, then combined for each output.
template <int MODE, int SET>
__device__ __forceinline__ void pack_row_unit(const PackArgs &a, int64_t u, int64_t plane, float fs) {
  const int r = (int)(u / (a.pcol_pad / 8));
  const int c0 = (int)(u - (int64_t)r * (a.pcol_pad / 8)) * 8;
  uint32_t v[kMaxSrc][8];
#pragma unroll
  for (int q = 0; q < kMaxSrc; ++q) {
    if (q < a.nsrc) {
      load_source<MODE, 8>(a, q, r, c0, v[q]);
    } else {
#pragma unroll
      for (int e = 0; e < 8; ++e) v[q][e] = 0;
    }
  }
  emit_all<MODE, SET>(a, v, (int64_t)r * a.pcol_pad + c0, plane, fs);
}

template <int MODE, int SET>
__device__ __forceinline__ void pack_rows_body(const PackArgs &a, int block, int nblocks) {
  const int64_t units = (int64_t)a.prow_pad * (a.pcol_pad / 8);
  const int64_t plane = (int64_t)a.prow_pad * a.pcol_pad;
  const float fs = MODE == MODE_FP32 ? fp16_scale(*a.amax, a.terms) : 1.f;
  for (int64_t u = block * (int64_t)blockDim.x + threadIdx.x; u < units; u += (int64_t)nblocks * blockDim.x)
    pack_row_unit<MODE, SET>(a, u, plane, fs);
}

// transposed layout: a CTA stages a 32 (source rows) x 64 (source cols) tile
// of every source in shared memory (reduced once), then each thread reads
// its 8 source rows of one source column and writes packed row = column.
template <int MODE, int SET>
__device__ __forceinline__ void pack_cols_body(const PackArgs &a, uint32_t (&tile)[kMaxSrc][32][65], int bx, int by) {
  const int r0 = by * 32;  // source rows = packed columns (K)
  const int c0 = bx * 64;  // source cols = packed rows (N)
  const int t = threadIdx.x;
  const int64_t plane = (int64_t)a.prow_pad * a.pcol_pad;
  const float fs = MODE == MODE_FP32 ? fp16_scale(*a.amax, a.terms) : 1.f;
  for (int q = 0; q < a.nsrc; ++q) {
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int vi = t + 256 * i;
      const int rr = vi >> 4, cc = (vi & 15) * 4;
      uint32_t w[4];
      load_source<MODE, 4>(a, q, r0 + rr, c0 + cc, w);
#pragma unroll
      for (int e = 0; e < 4; ++e) tile[q][rr][cc + e] = w[e];
    }
  }
  __syncthreads();
  const int pc = t >> 2, pr8 = (t & 3) * 8;
  uint32_t v[kMaxSrc][8];
#pragma unroll
  for (int q = 0; q < kMaxSrc; ++q) {
#pragma unroll
    for (int e = 0; e < 8; ++e) v[q][e] = q < a.nsrc ? tile[q][pr8 + e][pc] : 0u;
  }
  emit_all<MODE, SET>(a, v, (int64_t)(c0 + pc) * a.pcol_pad + r0 + pr8, plane, fs);
}

// both operands of a product (or of a fused level) in one launch: blocks
// [0, na) pack a (plain layout), the rest pack b (transposed), tile by tile
template <int MODE, int SA, int SB>
__global__ void __launch_bounds__(256) pack_pair_kernel(const __grid_constant__ PackArgs a,
                                                        const __grid_constant__ PackArgs b, int na, int tiles_x) {
  __shared__ uint32_t tile[kMaxSrc][32][65];
  if ((int)blockIdx.x < na) {
    pack_rows_body<MODE, SA>(a, blockIdx.x, na);
  } else {
    const int i = (int)blockIdx.x - na;
    pack_cols_body<MODE, SB>(b, tile, i % tiles_x, i / tiles_x);
  }
}

// ------------------------------------------------------------ level pack
// Every fused level under one table level in one pass (PackLevel).  Level
// j's operand quadrant q is sum_Q coef[j][Q] * (sub-block q of operand
// quadrant Q), so each of the 16 sub-blocks is read from DRAM once per
// position, held on chip, and all levels' 49 operands are formed from it.

// level j's four Winograd sources at one position from the 16 sub-block
// values w[Q][q][e] (reduced)
template <int MODE, int N>
__device__ __forceinline__ void level_sources(const PackLevel &L, int side, int j, const uint32_t (&w)[4][4][N],
                                              uint32_t (&v)[4][N]) {
  const uint32_t p = L.p;
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int e = 0; e < N; ++e) v[q][e] = MODE == MODE_FP32 ? __float_as_uint(0.f) : 0u;
#pragma unroll
  for (int Q = 0; Q < 4; ++Q) {
    const int c = L.coef[side][j][Q];
    if (c == 0) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int e = 0; e < N; ++e) v[q][e] = c > 0 ? lin_add<MODE>(v[q][e], w[Q][q][e], p) : lin_sub<MODE>(v[q][e], w[Q][q][e], p);
  }
}

// the seven Winograd outputs of one side from the four sources v (quadrants
// X11, X12, X21, X22), N elements each, output i at out + i * ostride + off
template <int MODE, int N, int SIDE>
__device__ __forceinline__ void level_emit(const uint32_t (&v)[4][N], uint32_t p, float fs, uint16_t *out,
                                           int64_t ostride, int64_t off, int64_t plane) {
  uint32_t x[N], y[N], z[N];
  auto put = [&](int i, const uint32_t (&t)[N]) {
    if constexpr (N == 8) emit8<MODE>(t, p, fs, out + i * ostride + off, plane);
    else if constexpr (N == 4) emit4<MODE>(t, p, fs, out + i * ostride + off, plane);
    else emit2<MODE>(t, p, fs, out + i * ostride + off, plane);
  };
  if (SIDE == 0) {
    put(0, v[0]);  // A11
    put(1, v[1]);  // A12
    put(3, v[3]);  // A22
#pragma unroll
    for (int e = 0; e < N; ++e) {
      x[e] = lin_add<MODE>(v[2][e], v[3][e], p);  // S1 = A21 + A22
      y[e] = lin_sub<MODE>(x[e], v[0][e], p);     // S2 = S1 - A11
      z[e] = lin_sub<MODE>(v[1][e], y[e], p);     // S4 = A12 - S2
    }
    put(4, x);
    put(5, y);
    put(2, z);
#pragma unroll
    for (int e = 0; e < N; ++e) z[e] = lin_sub<MODE>(v[0][e], v[2][e], p);  // S3 = A11 - A21
    put(6, z);
  } else {
    put(0, v[0]);  // B11
    put(1, v[2]);  // B21
    put(2, v[3]);  // B22
#pragma unroll
    for (int e = 0; e < N; ++e) {
      x[e] = lin_sub<MODE>(v[1][e], v[0][e], p);  // T1 = B12 - B11
      y[e] = lin_sub<MODE>(v[3][e], x[e], p);     // T2 = B22 - T1
      z[e] = lin_sub<MODE>(y[e], v[2][e], p);     // T4 = T2 - B21
    }
    put(4, x);
    put(5, y);
    put(3, z);
#pragma unroll
    for (int e = 0; e < N; ++e) z[e] = lin_sub<MODE>(v[3][e], v[1][e], p);  // T3 = B22 - B12
    put(6, z);
  }
}

// L2 prefetch of the 4 elements at (r, c) of every sub-block of one side
// (in-bounds positions only), so that the next tile's loads, issued after
// this tile's stores, find their lines in L2
__device__ __forceinline__ void level_prefetch(const PackLevel &L, int side, int r, int c) {
  if (r >= L.rows[side] || c >= L.cols[side]) return;
#pragma unroll
  for (int Q = 0; Q < 4; ++Q)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const char *a = L.src[side][Q][q] + (int64_t)L.esz[side][Q] * ((int64_t)r * L.ld[side][Q] + c);
      asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
    }
}

// plain side (A): a thread takes kLvlRowN consecutive columns of one row of
// every sub-block (16 kLvlRowN values in registers), then writes every
// level's outputs.  Two columns a thread halve the registers and double the
// resident warps, but measured slower (277 against 235 us at 8192^2 depth
// 2); three quarters of the pass's bytes are stores, which then go out in
// half-width instructions.
constexpr int kLvlRowN = 4;
template <int MODE>
__global__ void __launch_bounds__(256) level_rows_kernel(const __grid_constant__ PackLevel L) {
  constexpr int N = kLvlRowN;
  const int rows = L.rows[0], cols = L.cols[0], pc = L.pcol_pad[0];
  const int64_t units = (int64_t)L.prow_pad[0] * (pc / N);
  const int64_t plane = (int64_t)L.prow_pad[0] * pc;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < units; u += stride) {
    const int r = (int)(u / (pc / N));
    const int c0 = (int)(u - (int64_t)r * (pc / N)) * N;
    uint32_t w[4][4][N];
#pragma unroll
    for (int Q = 0; Q < 4; ++Q)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        load_row<N>(L.src[0][Q][q], L.ld[0][Q], r, c0, rows, cols, w[Q][q], L.esz[0][Q]);
#pragma unroll
        for (int e = 0; e < N; ++e) w[Q][q][e] = source_value<MODE>(w[Q][q][e], L.p, L.barrett);
      }
    for (int j = 0; j < L.n; ++j) {
      uint32_t v[4][N];
      level_sources<MODE, N>(L, 0, j, w, v);
      const float fs = MODE == MODE_FP32 ? fp16_scale(L.amax[0], L.terms[0][j]) : 1.f;
      level_emit<MODE, N, 0>(v, L.p, fs, L.out[0][j], L.ostride[0], (int64_t)r * pc + c0, plane);
    }
  }
}

// transposed side (B): a block of kLvlColThreads stages a 64 (source rows)
// x 16 (source cols) tile of every sub-block in shared memory; a thread then
// takes 2 source rows of one source column (packed row = that column; 32
// threads write 128 contiguous bytes of it) and writes every level's
// outputs.  Persistent over the tiles, with an L2 prefetch of the next one.
constexpr int kLvlTileK = 64, kLvlTileN = 16, kLvlColThreads = 512;
template <int MODE>
__global__ void __launch_bounds__(kLvlColThreads, 2)
    level_cols_kernel(const __grid_constant__ PackLevel L, int tiles_x, int tiles) {
  extern __shared__ uint32_t lvl_tile[];  // [16][kLvlTileK][kLvlTileN + 1]
  constexpr int W = kLvlTileN + 1;
  const int rows = L.rows[1], cols = L.cols[1], pc = L.pcol_pad[1];
  const int64_t plane = (int64_t)L.prow_pad[1] * pc;
  const int t = threadIdx.x, rr = t >> 3, cc = (t & 7) * 2;  // load: 64 rows x 8 pairs
  const int pcol = t >> 5, pr2 = (t & 31) * 2;                // emit: 16 columns x 32 row pairs
  for (int i = blockIdx.x; i < tiles; i += gridDim.x) {
    const int bx = i % tiles_x, by = i / tiles_x;
    const int r0 = by * kLvlTileK, c0 = bx * kLvlTileN;
    if (i > (int)blockIdx.x) __syncthreads();  // the previous tile's reads are done
#pragma unroll
    for (int Q = 0; Q < 4; ++Q)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        uint32_t x[2];
        load_row<2>(L.src[1][Q][q], L.ld[1][Q], r0 + rr, c0 + cc, rows, cols, x, L.esz[1][Q]);
#pragma unroll
        for (int e = 0; e < 2; ++e)
          lvl_tile[((Q * 4 + q) * kLvlTileK + rr) * W + cc + e] = source_value<MODE>(x[e], L.p, L.barrett);
      }
    __syncthreads();
    if (i + (int)gridDim.x < tiles) {  // the next tile's lines, while this one is written
      const int in = i + gridDim.x;
      level_prefetch(L, 1, (in / tiles_x) * kLvlTileK + rr, (in % tiles_x) * kLvlTileN + cc);
    }
    uint32_t w[4][4][2];
#pragma unroll
    for (int Q = 0; Q < 4; ++Q)
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int e = 0; e < 2; ++e) w[Q][q][e] = lvl_tile[((Q * 4 + q) * kLvlTileK + pr2 + e) * W + pcol];
    for (int j = 0; j < L.n; ++j) {
      uint32_t v[4][2];
      level_sources<MODE, 2>(L, 1, j, w, v);
      const float fs = MODE == MODE_FP32 ? fp16_scale(L.amax[1], L.terms[1][j]) : 1.f;
      level_emit<MODE, 2, 1>(v, L.p, fs, L.out[1][j], L.ostride[1], (int64_t)(c0 + pcol) * pc + r0 + pr2, plane);
    }
  }
}

// FP32 mode: max |x| over the sources of each side (blockIdx.y), one row per
// block iteration, 16-byte loads when the view allows them; the block
// maximum is atomically maxed into amax[side] as float bits (non-negative
// floats order like their bit patterns).  NaN is ignored, inf propagates.
__global__ void __launch_bounds__(256) amax_kernel(const __grid_constant__ AmaxArgs a) {
  const int side = blockIdx.y;
  const int64_t rows = a.rows[side], cols = a.cols[side];
  float m = 0.f;
  for (int q = 0; q < a.nsrc[side]; ++q) {
    const char *base = a.src[side][q];
    const int64_t ld = a.ld[side][q];
    const bool vec = ((uintptr_t)base % 16 == 0) && (ld % 4 == 0) && (cols % 4 == 0);
    for (int64_t r = blockIdx.x; r < rows; r += gridDim.x) {
      const float *row = reinterpret_cast<const float *>(base) + r * ld;
      if (vec) {
        for (int64_t c = 4 * (int64_t)threadIdx.x; c < cols; c += 4 * (int64_t)blockDim.x) {
          const float4 v = *reinterpret_cast<const float4 *>(row + c);
          m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
        }
      } else {
        for (int64_t c = threadIdx.x; c < cols; c += blockDim.x) m = fmaxf(m, fabsf(row[c]));
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ float wm[8];
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < 8 ? wm[threadIdx.x] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0 && m > 0.f) atomicMax(a.amax + side, __float_as_uint(m));
  }
}

// ------------------------------------------------------------ GEMM glue
constexpr int kThreads = 320;                 // producer, MMA, 8 epilogue warps
constexpr int kEpiThreads = 256;
constexpr int kChunkKB = 960 / kBK;           // k-blocks between in-place reductions (960 K)
constexpr int kNoDrainKB = 1024 / kBK;        // up to 1024 K no reduction is needed
constexpr int kStageScale = 64 / kBK;         // stages per 64 K of operands
constexpr int kPlaneBytes = kBM * kBK * 2;    // one A limb plane of a stage
constexpr int kEpiBytes = 2 * kBM * 32 * 4;   // 32 KB: 128 rows x 64 columns, 2 boxes of 32

template <int MODE>
struct Cfg;
template <>
struct Cfg<MODE_MODP1> {
  static constexpr int BN = 256, A_PLANES = 1, STAGES = 4 * kStageScale, ACC_BUFS = 2, BUF_COLS = 256;
};
template <>
struct Cfg<MODE_MODP2> {
  static constexpr int BN = kModp2BN, A_PLANES = 2, STAGES = (kModp2BN == 64 ? 4 : 3) * kStageScale;
  static constexpr int ACC_BUFS = kModp2BN == 64 ? 2 : 1, BUF_COLS = 4 * kModp2BN;
};
template <>
struct Cfg<MODE_FP32> {
  static constexpr int BN = 128, A_PLANES = 2, STAGES = 3 * kStageScale, ACC_BUFS = 2, BUF_COLS = 256;
};
template <int MODE>
__host__ __device__ constexpr int b_rows() {  // B rows per stage: one plane (p <= 256) or [hi | lo]
  return MODE == MODE_MODP1 ? Cfg<MODE>::BN : 2 * Cfg<MODE>::BN;
}
template <int MODE>
__host__ __device__ constexpr int stage_bytes() {
  return Cfg<MODE>::A_PLANES * kPlaneBytes + b_rows<MODE>() * kBK * 2;
}
template <int MODE>
__host__ __device__ constexpr int smem_bytes() {
  return Cfg<MODE>::STAGES * stage_bytes<MODE>() + kEpiBytes + 1024 + 256;
}
static_assert(smem_bytes<MODE_MODP1>() <= 232448 && smem_bytes<MODE_MODP2>() <= 232448 &&
                  smem_bytes<MODE_FP32>() <= 232448,
              "shared memory per CTA");

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t *b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t gtime() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

struct Ctl {
  volatile int abort;
  uint32_t tmem_base;
  uint64_t wait_ns;  // bound of every wait
};

// Wait for phase `parity` of barrier b.  Gives up when another warp of the
// CTA has aborted, or after ctl->wait_ns (then it aborts the CTA and records
// SWMM_ETIMEOUT in the error word).
__device__ __forceinline__ bool wait_bar(uint64_t *b, uint32_t parity, Ctl *ctl, int *err) {
  if (mbar_try(b, parity)) return true;
  const uint64_t t0 = gtime();
  for (uint32_t it = 0;; ++it) {
    if (mbar_try(b, parity)) return true;
    if ((it & 63) == 63) {
      if (ctl->abort) return false;
      if (gtime() - t0 > ctl->wait_ns) {
        ctl->abort = 1;
        if (err) atomicExch(err, kErrTimeout);
        return false;
      }
    }
  }
}
// Wait for work this CTA already issued (TMA loads, MMAs) to land before it
// exits, whether or not the CTA has aborted; bounded by ctl->wait_ns too.
__device__ __forceinline__ void wait_done(uint64_t *b, uint32_t parity, Ctl *ctl, int *err) {
  if (mbar_try(b, parity)) return;
  const uint64_t t0 = gtime();
  for (uint32_t it = 0;; ++it) {
    if (mbar_try(b, parity)) return;
    if ((it & 63) == 63 && gtime() - t0 > ctl->wait_ns) {
      ctl->abort = 1;
      if (err) atomicExch(err, kErrTimeout);
      return;
    }
  }
}

__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kEpiThreads) : "memory"); }
// Epilogue barrier that also agrees on the abort flag: true on every
// epilogue thread when no thread saw it set, false on every thread
// otherwise, so all of them take the same path to the next barrier.
__device__ __forceinline__ bool epi_agree(const Ctl *ctl) {
  uint32_t ok;
  const uint32_t mine = ctl->abort ? 0u : 1u;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}"
      : "=r"(ok)
      : "r"(mine), "n"(kEpiThreads)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_commit(uint64_t *b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(b))
               : "memory");
}
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void tma_load(uint32_t dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_store(const CUtensorMap *map, int x, int y, uint32_t src) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];" ::"l"(map), "r"(x),
               "r"(y), "r"(src)
               : "memory");
}
__device__ __forceinline__ void tma_reduce_add(const CUtensorMap *map, int x, int y, uint32_t src) {
  asm volatile("cp.reduce.async.bulk.tensor.2d.global.shared::cta.add.tile.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                   map),
               "r"(x), "r"(y), "r"(src)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float *v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
          taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
      "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
      "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
      "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
      "r"(__float_as_uint(v[15]))
      : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// After tcgen05.wait::ld: ties 16 loaded registers to the wait so that no
// arithmetic on them is scheduled before it.
__device__ __forceinline__ void reg_fence16(float (&v)[16]) {
  asm volatile(""
               : "+f"(v[0]), "+f"(v[1]), "+f"(v[2]), "+f"(v[3]), "+f"(v[4]), "+f"(v[5]), "+f"(v[6]), "+f"(v[7]),
                 "+f"(v[8]), "+f"(v[9]), "+f"(v[10]), "+f"(v[11]), "+f"(v[12]), "+f"(v[13]), "+f"(v[14]),
                 "+f"(v[15]));
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ uint4 lds128(uint32_t a) {
  uint4 v;
  asm volatile("ld.shared.v4.b32 {%0,%1,%2,%3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
  return v;
}
__device__ __forceinline__ uint32_t lds32(uint32_t a) {
  uint32_t v;
  asm volatile("ld.shared.b32 %0, [%1];" : "=r"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ void sts128(uint32_t a, uint4 v) {
  asm volatile("st.shared.v4.b32 [%0], {%1,%2,%3,%4};" ::"r"(a), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w) : "memory");
}

// Shared-memory matrix descriptor: K-major operand whose rows are kBK fp16
// values (kBK * 2 bytes, swizzled over that width), 8-row core groups
// 8 * kBK * 2 bytes apart (stride byte offset), descriptor version 1.
// Swizzle field: 2 = 128-byte, 4 = 64-byte.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  constexpr uint64_t kRowBytes = kBK * 2;
  uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;                          // leading byte offset (unused for this layout)
  d |= (uint64_t)((8 * kRowBytes) >> 4) << 32;     // stride byte offset
  d |= (uint64_t)1 << 46;                          // version
  d |= (uint64_t)(kRowBytes == 128 ? 2 : 4) << 61;  // swizzle
  return d;
}
// Instruction descriptor, kind::f16: D fp32, A/B fp16 (fmt 0; 1 would be bf16),
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_f16(int ab_fmt, int M, int N) {
  return (1u << 4) | ((uint32_t)ab_fmt << 7) | ((uint32_t)ab_fmt << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

struct TileInfo {
  int pi, m0, n0;
};
template <int BN>
__device__ __forceinline__ TileInfo decode(const GemmParams &P, int g) {
  int pi = 0;
  while (pi + 1 < P.nprod && g >= P.prod[pi + 1].tile_begin) ++pi;
  const Product &pr = P.prod[pi];
  const int local = g - pr.tile_begin;
  const int G = 16;  // tile rows visited together (L2 reuse of B' columns)
  const int per_group = G * pr.tiles_n;
  const int gid = local / per_group;
  const int first = gid * G;
  const int gs = min(pr.tiles_m - first, G);
  const int r = local - gid * per_group;
  TileInfo t;
  t.pi = pi;
  t.m0 = (first + r % gs) * kBM;
  t.n0 = (r / gs) * BN;
  return t;
}

// --------------------------------------------------------- epilogue math
struct Epi {
  uint32_t p, m;
  float pf, inv_p;
  float fsc;  // FP32 mode: alpha / (s_A s_B), undoing the operand scales
  // mod p, reductions with alpha = +-1: the contribution sign (+1 / -1) folded
  // into a lazy representative p +- r in [p/2, 3p/2]; 0: canonical value,
  // then alpha and the sign
  int lsg;
  __device__ __forceinline__ uint32_t out(float r) const {  // r = fr(...) in [-p/2, p/2]
    if (lsg == 0) return canon(r);
    const float x = lsg > 0 ? pf + r : pf - r;
    return __float_as_uint(x + 12582912.0f) - 0x4B400000u;
  }
  __device__ __forceinline__ float fr(float f) const {  // centred residue, exact |f| <= 2^24
    const float MAGIC = 12582912.0f;                     // 1.5 * 2^23: rint via addition
    float q = __fmaf_rn(f, inv_p, MAGIC) - MAGIC;
    return __fmaf_rn(q, -pf, f);
  }
  __device__ __forceinline__ uint32_t canon(float r) const {  // r in (-p, p) -> [0, p)
    r = r < 0.f ? r + pf : r;
    return __float_as_uint(r + 12582912.0f) - 0x4B400000u;
  }
  __device__ __forceinline__ uint32_t mulmod(uint32_t u, uint32_t x) const {  // u, x < p
    uint32_t prod = u * x;
    uint32_t q = __umulhi(prod, m);
    uint32_t r = prod - q * p;
    return min(r, r - p);
  }
  __device__ __forceinline__ uint32_t red(uint32_t x) const {  // any x -> [0, p)
    uint32_t q = __umulhi(x, m);
    uint32_t r = x - q * p;
    return min(r, r - p);
  }
};

// 2^16 hh + 2^8 (hl + lh) + ll mod p for 16 columns, every intermediate an
// exact fp32 integer; q = {hh, hl, lh, ll}
__device__ __forceinline__ void modp2_recombine(const Epi &E, const float (&q)[4][16], uint32_t *v) {
#pragma unroll
  for (int e = 0; e < 16; ++e) {
    const float s = E.fr(E.fr(q[1][e]) + E.fr(q[2][e]));
    const float t1 = E.fr(__fmaf_rn(256.f, E.fr(q[0][e]), s));
    v[e] = E.out(E.fr(__fmaf_rn(256.f, t1, E.fr(q[3][e]))));
  }
}

// alpha and the sign of a reduction target on 16 mod-p results (nothing
// left to do when they were folded into lazy representatives)
__device__ __forceinline__ void modp_finish(const Product &pr, const Epi &E, int sign, uint32_t *v) {
  if (E.lsg != 0) return;
#pragma unroll
  for (int e = 0; e < 16; ++e) {
    uint32_t x = v[e];
    if (pr.alpha_u != 1) x = E.mulmod(pr.alpha_u, x);
    if (pr.epilogue == EPI_REDUCE && sign < 0) x = x == 0 ? 0u : E.p - x;
    v[e] = x;
  }
}

// p < 2^16, one accumulator buffer, released in two halves: columns
// [0, 2 BN) hold hh | hl and [2 BN, 4 BN) hold lh | ll.  First every
// X = 2^8 fr(hh) + fr(hl) of the thread's 64 columns is formed (|X| <
// 2^23 + 2^15) and the first half released (the next tile's A_h products
// may start), then v = fr(2^8 fr(X + fr(lh)) + fr(ll)) = 2^16 hh + 2^8 (hl +
// lh) + ll mod p and the second half released.  Every intermediate is an
// exact fp32 integer (below 2^24).
__device__ __forceinline__ void modp2_drain_split(const Product &pr, const Epi &E, uint32_t d, int hsel, int sign,
                                                  uint32_t (&vals)[2][32], uint64_t *half0, uint64_t *half1) {
  // Eight groups of 16 columns (four of hh | hl, then four of lh | ll), read
  // out of tensor memory with the next group's loads in flight while the
  // current one is combined, so only the first load's latency is exposed.
  float X[4][16];
  float a[2][16], b[2][16];
  auto issue = [&](int g, int s) {
    const int col = (g & 2) * 32 + hsel * 32 + (g & 1) * 16 + (g < 4 ? 0 : 2 * kModp2BN);
    tmem_ld16(d + col, a[s]);
    tmem_ld16(d + kModp2BN + col, b[s]);
  };
  issue(0, 0);
  tmem_wait_ld();
  reg_fence16(a[0]);
  reg_fence16(b[0]);
#pragma unroll
  for (int g = 0; g < 8; ++g) {
    const int s = g & 1;
    if (g + 1 < 8) issue(g + 1, s ^ 1);
    if (g < 4) {
#pragma unroll
      for (int e = 0; e < 16; ++e) X[g][e] = __fmaf_rn(256.f, E.fr(a[s][e]), E.fr(b[s][e]));
      if (g == 3) {  // hh | hl read out: the next tile's A_h products may start
        tc_fence_before();
        mbar_arrive(half0);
      }
    } else {
      uint32_t *v = vals[(g - 4) >> 1] + (g & 1) * 16;
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const float y = E.fr(X[g - 4][e] + E.fr(a[s][e]));
        v[e] = E.out(E.fr(__fmaf_rn(256.f, y, E.fr(b[s][e]))));
      }
      modp_finish(pr, E, sign, v);
    }
    if (g + 1 < 8) {
      tmem_wait_ld();
      reg_fence16(a[s ^ 1]);
      reg_fence16(b[s ^ 1]);
    }
  }
  tc_fence_before();
  mbar_arrive(half1);
}

// Values of 16 consecutive columns of one row before any beta term: mod p
// results (alpha applied; REDUCE: the signed contribution p - v for a
// negative target) or floats (FP32: alpha applied, sign folded for REDUCE).
template <int MODE>
__device__ __forceinline__ void tile_values(const Product &pr, const Epi &E, uint32_t d, int col, int sign,
                                            uint32_t *v) {
  if (MODE == MODE_MODP2) {
    float q[4][16];
    tmem_ld16(d + col, q[0]);
    tmem_ld16(d + kModp2BN + col, q[1]);
    tmem_ld16(d + 2 * kModp2BN + col, q[2]);
    tmem_ld16(d + 3 * kModp2BN + col, q[3]);
    tmem_wait_ld();
#pragma unroll
    for (int i = 0; i < 4; ++i) reg_fence16(q[i]);
    modp2_recombine(E, q, v);
  } else if (MODE == MODE_MODP1) {
    float a[16];
    tmem_ld16(d + col, a);
    tmem_wait_ld();
    reg_fence16(a);
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] = E.out(E.fr(a[e]));
  } else {
    float a[16], b[16];
    tmem_ld16(d + col, a);
    tmem_ld16(d + 128 + col, b);
    tmem_wait_ld();
    reg_fence16(a);
    reg_fence16(b);
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      float f = E.fsc * (a[e] + b[e]);
      if (pr.epilogue == EPI_REDUCE && sign < 0) f = -f;
      v[e] = __float_as_uint(f);
    }
    return;
  }
  modp_finish(pr, E, sign, v);
}

// value + beta * c for a STORE with beta (c may be any representative mod p)
template <int MODE>
__device__ __forceinline__ uint32_t add_beta(const Product &pr, const Epi &E, uint32_t v, uint32_t c) {
  if (MODE == MODE_FP32) return __float_as_uint(__uint_as_float(v) + pr.beta_f * __uint_as_float(c));
  const uint32_t w = v + E.mulmod(pr.beta_u, E.red(c));
  return min(w, w - E.p);
}

// ------------------------------------------------------------- the GEMM
template <int MODE>
__global__ void __launch_bounds__(kThreads, 1) gemm_kernel(const __grid_constant__ GemmParams P) {
  using C = Cfg<MODE>;
  constexpr int BN = C::BN;
  constexpr int SB = stage_bytes<MODE>();
  constexpr bool modp = MODE != MODE_FP32;
  // p < 2^16 with one accumulator buffer: released in two halves
  constexpr bool SPLIT = MODE == MODE_MODP2 && C::ACC_BUFS == 1;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char *ebuf = smem + C::STAGES * SB;  // epilogue tile, 4 swizzled boxes
  uint64_t *bars = reinterpret_cast<uint64_t *>(ebuf + kEpiBytes);
  uint64_t *full = bars;                      // [STAGES]
  uint64_t *empty = bars + C::STAGES;         // [STAGES]
  uint64_t *acc_full = bars + 2 * C::STAGES;  // [2]
  uint64_t *acc_empty = acc_full + 2;         // [2]
  uint64_t *drain_full = acc_empty + 2;
  uint64_t *drain_empty = drain_full + 1;
  uint64_t *final_bar = drain_empty + 1;
  uint64_t *cbar = final_bar + 1;       // beta source tile loaded
  uint64_t *stall_bar = cbar + 1;       // test hook: nothing ever arrives here
  Ctl *ctl = reinterpret_cast<Ctl *>(stall_bar + 1);

  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;

  if (tid == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], kEpiThreads);
    }
    mbar_init(drain_full, 1);
    mbar_init(drain_empty, kEpiThreads);
    mbar_init(final_bar, 1);
    mbar_init(cbar, 1);
    mbar_init(stall_bar, 1);
    ctl->abort = 0;
    ctl->wait_ns = P.wait_ns;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&ctl->tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = ctl->tmem_base;

  if (warp == 0) {
    // =============================== TMA producer ===============================
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      uint32_t issued = 0, last_phase = 0;  // per stage: a load was issued; its phase parity
      // test hook: a wait that nothing completes runs out (SWMM_ETIMEOUT)
      const bool stalled = P.test_stall && !wait_bar(stall_bar, 0, ctl, P.err);
      for (int g = blockIdx.x; g < P.total_tiles && !stalled; g += gridDim.x) {
        const TileInfo ti = decode<BN>(P, g);
        const Product &pr = P.prod[ti.pi];
        const int nkb = pr.Kpad / kBK;
        bool bad = false;
        for (int kb = 0; kb < nkb; ++kb) {
          if (!wait_bar(&empty[stage], phase ^ 1, ctl, P.err)) {
            bad = true;
            break;
          }
          const uint32_t sA = smem_u32(smem + stage * SB);
          const uint32_t sB = sA + C::A_PLANES * kPlaneBytes;
          mbar_expect_tx(&full[stage], SB);
          issued |= 1u << stage;
          last_phase = (last_phase & ~(1u << stage)) | (phase << stage);
          const int k0 = kb * kBK;
          tma_load(sA, &pr.ta, k0, ti.m0, &full[stage]);
          if (C::A_PLANES == 2) tma_load(sA + kPlaneBytes, &pr.ta, k0, pr.a_plane_rows + ti.m0, &full[stage]);
          if (MODE == MODE_MODP1) {
            tma_load(sB, &pr.tb, k0, ti.n0, &full[stage]);  // 256-row box
          } else {
            tma_load(sB, &pr.tb, k0, ti.n0, &full[stage]);
            tma_load(sB + C::BN * kBK * 2, &pr.tb, k0, pr.b_plane_rows + ti.n0, &full[stage]);
          }
          if (++stage == C::STAGES) {
            stage = 0;
            phase ^= 1;
          }
        }
        if (bad) break;
      }
      // no load may still be writing shared memory when the CTA exits (after
      // an abort some were never consumed)
      for (int st = 0; st < C::STAGES; ++st)
        if (issued >> st & 1) wait_done(&full[st], last_phase >> st & 1, ctl, P.err);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ================================ MMA issuer ================================
    if (lane == 0) {
      const uint32_t fmt = 0;  // fp16 operands in every mode
      const uint32_t id256 = idesc_f16(fmt, kBM, 256);
      const uint32_t id128 = idesc_f16(fmt, kBM, 128);
      const uint32_t idB2 = idesc_f16(fmt, kBM, 2 * BN);  // N = [hi | lo] rows of B
      int stage = 0;
      uint32_t phase = 0, tcount = 0, dcount = 0;
      for (int g = blockIdx.x; g < P.total_tiles; g += gridDim.x, ++tcount) {
        const TileInfo ti = decode<BN>(P, g);
        const Product &pr = P.prod[ti.pi];
        const int nkb = pr.Kpad / kBK;
        const int buf = C::ACC_BUFS == 2 ? (int)(tcount & 1) : 0;
        const uint32_t use = C::ACC_BUFS == 2 ? (tcount >> 1) : tcount;
        if (!wait_bar(&acc_empty[buf], (use & 1) ^ 1, ctl, P.err)) break;
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(buf * C::BUF_COLS);
        bool bad = false;
        int kb = 0;
        if (SPLIT) {
          // The first half (hh | hl) is free: issue the A_h products of the
          // k-blocks already staged, then wait for the second half (lh | ll)
          // and issue their A_l products, releasing the stages.
          const int pre = nkb < C::STAGES ? nkb : C::STAGES;
          const int stage0 = stage;
          const uint32_t phase0 = phase;
          for (int j = 0; j < pre && !bad; ++j) {
            if (!wait_bar(&full[stage], phase, ctl, P.err)) {
              bad = true;
              break;
            }
            tc_fence_after();
            const uint32_t sA = smem_u32(smem + stage * SB);
            const uint32_t sB = sA + C::A_PLANES * kPlaneBytes;
#pragma unroll
            for (int k = 0; k < kBK / 16; ++k)
              tc_mma(d, sdesc(sA + 32 * k), sdesc(sB + 32 * k), idB2, (j > 0 || k > 0) ? 1u : 0u);
            if (++stage == C::STAGES) {
              stage = 0;
              phase ^= 1;
            }
          }
          if (!bad && !wait_bar(&acc_empty[1], (use & 1) ^ 1, ctl, P.err)) bad = true;
          if (bad) break;
          tc_fence_after();
          stage = stage0;
          phase = phase0;
          for (int j = 0; j < pre; ++j) {
            const uint32_t sA = smem_u32(smem + stage * SB);
            const uint32_t sB = sA + C::A_PLANES * kPlaneBytes;
#pragma unroll
            for (int k = 0; k < kBK / 16; ++k)
              tc_mma(d + 2 * BN, sdesc(sA + kPlaneBytes + 32 * k), sdesc(sB + 32 * k), idB2,
                     (j > 0 || k > 0) ? 1u : 0u);
            tc_commit(&empty[stage]);
            if (++stage == C::STAGES) {
              stage = 0;
              phase ^= 1;
            }
          }
          kb = pre;
        }
        for (; kb < nkb; ++kb) {
          if (!wait_bar(&full[stage], phase, ctl, P.err)) {
            bad = true;
            break;
          }
          tc_fence_after();
          const uint32_t sA = smem_u32(smem + stage * SB);
          const uint32_t sB = sA + C::A_PLANES * kPlaneBytes;
#pragma unroll
          for (int k = 0; k < kBK / 16; ++k) {
            const uint32_t acc = (kb > 0 || k > 0) ? 1u : 0u;
            const uint64_t a0 = sdesc(sA + 32 * k);
            const uint64_t bd = sdesc(sB + 32 * k);
            if (MODE == MODE_MODP1) {
              tc_mma(d, a0, bd, id256, acc);
            } else if (MODE == MODE_MODP2) {
              const uint64_t a1 = sdesc(sA + kPlaneBytes + 32 * k);
              tc_mma(d, a0, bd, idB2, acc);           // [hh | hl]
              tc_mma(d + 2 * BN, a1, bd, idB2, acc);  // [lh | ll]
            } else {
              const uint64_t a1 = sdesc(sA + kPlaneBytes + 32 * k);
              tc_mma(d, a0, bd, id256, acc);       // [hi*hi | hi*lo]
              tc_mma(d + 128, a1, bd, id128, 1u);  // lo*hi onto the hi*lo half
            }
          }
          tc_commit(&empty[stage]);
          if (++stage == C::STAGES) {
            stage = 0;
            phase ^= 1;
          }
          if (modp && nkb > kNoDrainKB && (kb + 1) % kChunkKB == 0 && kb + 1 < nkb) {
            // keep every fp32 partial sum below 2^24: reduce mod p in place
            tc_commit(drain_full);
            if (!wait_bar(drain_empty, dcount & 1, ctl, P.err)) {
              bad = true;
              break;
            }
            ++dcount;
            tc_fence_after();
          }
        }
        if (bad) break;
        tc_commit(&acc_full[buf]);
      }
      tc_commit(final_bar);  // no MMA may still run when the allocation is freed
      wait_done(final_bar, 0, ctl, P.err);
    }
    __syncwarp();
  } else {
    // ================================= epilogue =================================
    // Warp w in 2..9 reads tensor-memory lanes 32 (w % 4) .. +31.  The tile is
    // written in 64-column chunks through a 32 KB staging buffer (two boxes of
    // 32 columns); in each chunk warp w owns box (w - 2) / 4.
    const int et = tid - 64;
    const int q4 = warp & 3;
    const int hsel = (warp - 2) >> 2;
    const int row = q4 * 32 + lane;
    const bool issuer = et == 0;
    const uint32_t lane_addr = (uint32_t)((q4 * 32) << 16);
    const uint32_t eb = smem_u32(ebuf);
    Epi E;
    E.p = P.p;
    E.m = P.barrett;
    E.pf = (float)P.p;
    E.inv_p = P.inv_p;
    E.fsc = 0.f;
    E.lsg = 0;
    uint32_t tcount = 0, dcount = 0, cphase = 0;
    for (int g = blockIdx.x; g < P.total_tiles; g += gridDim.x, ++tcount) {
      const TileInfo ti = decode<BN>(P, g);
      const Product &pr = P.prod[ti.pi];
      const int nkb = pr.Kpad / kBK;
      const int buf = C::ACC_BUFS == 2 ? (int)(tcount & 1) : 0;
      const uint32_t use = C::ACC_BUFS == 2 ? (tcount >> 1) : tcount;
      const uint32_t d = tmem + lane_addr + (uint32_t)(buf * C::BUF_COLS);
      if (MODE == MODE_FP32)
        E.fsc = pr.alpha_f / (fp16_scale(pr.amax[0], pr.terms_a) * fp16_scale(pr.amax[1], pr.terms_b));
      if (modp) {
        const bool unit = pr.alpha_u == 1 || pr.alpha_u == P.p - 1;
        E.lsg = (pr.epilogue == EPI_REDUCE && unit) ? (((pr.t[0].sign < 0) != (pr.alpha_u != 1)) ? -1 : 1) : 0;
      }
      const bool tma = pr.tma_epi != 0;
      const bool with_beta = pr.epilogue == EPI_STORE && pr.use_beta;
      const int sign = pr.t[0].sign;
      bool bad = false;
      if (modp && nkb > kNoDrainKB) {
        const int ndrain = (nkb - 1) / kChunkKB;
        for (int q = 0; q < ndrain; ++q, ++dcount) {
          wait_bar(drain_full, dcount & 1, ctl, P.err);
          if (!epi_agree(ctl)) {  // every epilogue thread takes the same exit
            bad = true;
            break;
          }
          tc_fence_after();
          constexpr int cols = MODE == MODE_MODP2 ? 4 * BN : 256;
          for (int c = hsel * (cols / 2); c < (hsel + 1) * (cols / 2); c += 32) {
            float v[32];
            tmem_ld16(d + c, v);
            tmem_ld16(d + c + 16, v + 16);
            tmem_wait_ld();
#pragma unroll
            for (int e = 0; e < 32; ++e) v[e] = E.fr(v[e]);
            tmem_st16(d + c, v);
            tmem_st16(d + c + 16, v + 16);
          }
          tmem_wait_st();
          tc_fence_before();
          mbar_arrive(drain_empty);
        }
        if (bad) break;
      }
      wait_bar(&acc_full[buf], use & 1, ctl, P.err);
      if (!epi_agree(ctl)) break;
      tc_fence_after();
      constexpr int NCH = BN / 64;
      // With a single accumulator buffer the next tile's MMAs wait for this
      // drain, so every chunk is read out of tensor memory before the first
      // store (HOLD = NCH); with two buffers the chunks are read and stored
      // one after the other.
      constexpr int HOLD = C::ACC_BUFS == 1 ? NCH : 1;
      uint32_t vals[HOLD][32];
      if (HOLD > 1) {
        if (SPLIT) {
          // the two halves of the accumulator are released one after the other
          modp2_drain_split(pr, E, d, hsel, sign, *reinterpret_cast<uint32_t(*)[2][32]>(vals), &acc_empty[0],
                            &acc_empty[1]);
        } else {
#pragma unroll
          for (int ch = 0; ch < HOLD; ++ch) {
            tile_values<MODE>(pr, E, d, ch * 64 + hsel * 32, sign, vals[ch]);
            tile_values<MODE>(pr, E, d, ch * 64 + hsel * 32 + 16, sign, vals[ch] + 16);
          }
          tc_fence_before();
          mbar_arrive(&acc_empty[buf]);  // accumulators free for the next tile
        }
      }
#pragma unroll
      for (int ch = 0; ch < NCH; ++ch) {
        const int tc0 = ch * 64 + hsel * 32;  // tile column of this thread's first value
        uint32_t *v = vals[HOLD > 1 ? ch : 0];
        if (HOLD == 1) {
          tile_values<MODE>(pr, E, d, tc0, sign, v);
          tile_values<MODE>(pr, E, d, tc0 + 16, sign, v + 16);
          if (ch == NCH - 1) {
            tc_fence_before();
            mbar_arrive(&acc_empty[buf]);  // accumulators free for the next tile
          }
        }
        if (tma) {
          if (issuer) {
            bulk_wait_read0();  // the previous chunk's TMA has read the buffer
            if (with_beta) {
              int boxes = 0;
              for (int b = 0; b < 2; ++b) boxes += ti.n0 + ch * 64 + 32 * b < pr.N;
              mbar_expect_tx(cbar, boxes * 16384);
              for (int b = 0; b < 2; ++b)
                if (ti.n0 + ch * 64 + 32 * b < pr.N)
                  tma_load(eb + b * 16384, &pr.tmap[0], ti.n0 + ch * 64 + 32 * b, ti.m0, cbar);
            }
          }
          epi_sync();
          if (with_beta) {
            wait_done(cbar, cphase, ctl, P.err);  // the load lands even after an abort
            cphase ^= 1;
          }
          const uint32_t rowbase = eb + hsel * 16384 + row * 128;
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const uint32_t a = rowbase + ((j ^ (row & 7)) << 4);
            uint4 w = make_uint4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
            if (with_beta) {
              const uint4 c = lds128(a);
              w.x = add_beta<MODE>(pr, E, w.x, c.x);
              w.y = add_beta<MODE>(pr, E, w.y, c.y);
              w.z = add_beta<MODE>(pr, E, w.z, c.z);
              w.w = add_beta<MODE>(pr, E, w.w, c.w);
            }
            sts128(a, w);
          }
          fence_proxy_async();
          if (!epi_agree(ctl)) {
            bad = true;
            break;
          }
          if (issuer) {
            for (int b = 0; b < 2; ++b) {
              const int x = ti.n0 + ch * 64 + 32 * b;
              if (x >= pr.N) break;
              if (pr.epilogue == EPI_STORE) {
                tma_store(&pr.tmap[0], x, ti.m0, eb + b * 16384);
              } else {
                for (int t = 0; t < pr.ntargets; ++t) tma_reduce_add(&pr.tmap[t], x, ti.m0, eb + b * 16384);
              }
            }
            bulk_commit();
          }
        } else {
          // Targets TMA cannot address (row pitch or base not 16-byte
          // aligned): the chunk goes through the staging buffer so that each
          // warp then writes whole row segments (32 consecutive columns per
          // instruction) with plain stores or reductions.
          if (issuer) bulk_wait_read0();  // an earlier TMA tile has read the buffer
          epi_sync();
          {
            const uint32_t rowbase = eb + hsel * 16384 + row * 128;
#pragma unroll
            for (int j = 0; j < 8; ++j)
              sts128(rowbase + ((j ^ (row & 7)) << 4), make_uint4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]));
          }
          epi_sync();
          const int wi = et >> 5;
          for (int rr = wi; rr < kBM; rr += kEpiThreads / 32) {
            const int g_r = ti.m0 + rr;
            if (g_r >= pr.M) break;
#pragma unroll
            for (int h2 = 0; h2 < 2; ++h2) {
              const int c = h2 * 32 + lane;
              const int g_c = ti.n0 + ch * 64 + c;
              if (g_c >= pr.N) continue;
              const uint32_t x =
                  lds32(eb + h2 * 16384 + rr * 128 + ((((c & 31) >> 2) ^ (rr & 7)) << 4) + (c & 3) * 4);
              if (pr.epilogue == EPI_STORE) {
                uint32_t *dst = reinterpret_cast<uint32_t *>((char *)pr.t[0].ptr) + (int64_t)g_r * pr.t[0].ld + g_c;
                *dst = with_beta ? add_beta<MODE>(pr, E, x, *dst) : x;
              } else {
                for (int t = 0; t < pr.ntargets; ++t) {
                  if (modp)
                    atomicAdd(reinterpret_cast<unsigned int *>((char *)pr.t[t].ptr) + (int64_t)g_r * pr.t[t].ld + g_c,
                              x);
                  else
                    atomicAdd(reinterpret_cast<float *>((char *)pr.t[t].ptr) + (int64_t)g_r * pr.t[t].ld + g_c,
                              __uint_as_float(x));
                }
              }
            }
          }
        }
      }
      if (bad) break;
    }
    if (issuer) bulk_wait0();
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
  }
}

// ------------------------------------------------------------ SIMT leaf
__global__ void leaf_simt_kernel(const __grid_constant__ SimtArgs A, const __grid_constant__ GemmParams P, int mode) {
  const int r = blockIdx.y * 16 + threadIdx.y;
  const int c = blockIdx.x * 16 + threadIdx.x;
  if (r >= A.M || c >= A.N) return;
  const uint64_t p = P.p;
  uint64_t acc = 0;
  double facc = 0.0;
  for (int k = 0; k < A.K; ++k) {
    if (mode != MODE_FP32) {
      int64_t a = 0, b = 0;
      for (int t = 0; t < A.na; ++t) {
        int64_t v = *((const int32_t *)A.a[t] + (int64_t)r * A.lda[t] + k);
        a += A.sa[t] > 0 ? v : -v;
      }
      for (int t = 0; t < A.nb; ++t) {
        int64_t v = *((const int32_t *)A.b[t] + (int64_t)k * A.ldb[t] + c);
        b += A.sb[t] > 0 ? v : -v;
      }
      a = ((a % (int64_t)p) + (int64_t)p) % (int64_t)p;
      b = ((b % (int64_t)p) + (int64_t)p) % (int64_t)p;
      acc = (acc + (uint64_t)a * (uint64_t)b) % p;
    } else {
      float a = 0.f, b = 0.f;
      for (int t = 0; t < A.na; ++t) {
        float v = *((const float *)A.a[t] + (int64_t)r * A.lda[t] + k);
        a += A.sa[t] > 0 ? v : -v;
      }
      for (int t = 0; t < A.nb; ++t) {
        float v = *((const float *)A.b[t] + (int64_t)k * A.ldb[t] + c);
        b += A.sb[t] > 0 ? v : -v;
      }
      facc += (double)a * (double)b;
    }
  }
  if (mode != MODE_FP32) {
    uint64_t v = (acc * P.alpha_u) % p;
    if (P.epilogue == EPI_STORE) {
      uint32_t *dst = (uint32_t *)A.t[0].ptr + (int64_t)r * A.t[0].ld + c;
      if (P.use_beta) v = (v + (uint64_t)P.beta_u * ((*dst) % p)) % p;
      *dst = (uint32_t)v;
    } else {
      for (int t = 0; t < A.ntargets; ++t) {
        unsigned int *dst = (unsigned int *)A.t[t].ptr + (int64_t)r * A.t[t].ld + c;
        uint64_t w = A.t[t].sign > 0 ? v : (p - v) % p;
        atomicAdd(dst, (unsigned int)w);
      }
    }
  } else {
    float v = P.alpha_f * (float)facc;
    if (P.epilogue == EPI_STORE) {
      float *dst = (float *)A.t[0].ptr + (int64_t)r * A.t[0].ld + c;
      if (P.use_beta) v += P.beta_f * (*dst);
      *dst = v;
    } else {
      for (int t = 0; t < A.ntargets; ++t) {
        float *dst = (float *)A.t[t].ptr + (int64_t)r * A.t[t].ld + c;
        atomicAdd(dst, (float)A.t[t].sign * v);
      }
    }
  }
}

}  // namespace dev

// ================================================================= host side
template <int MODE, int SA, int SB>
static cudaError_t pair_sets(const PackArgs &a, const PackArgs &b, cudaStream_t s) {
  const int64_t units = (int64_t)a.prow_pad * (a.pcol_pad / 8);
  const int64_t want = (units + 255) / 256;
  const int na = (int)(want > 152 * 16 ? 152 * 16 : want);
  const int tiles_x = b.prow_pad / 64, tiles = tiles_x * (b.pcol_pad / 32);
  if (na + tiles <= 0) return cudaSuccess;
  dev::pack_pair_kernel<MODE, SA, SB><<<na + tiles, 256, 0, s>>>(a, b, na, tiles_x);
  return cudaGetLastError();
}
template <int MODE>
static cudaError_t pair_mode(const PackArgs &a, const PackArgs &b, cudaStream_t s) {
  const bool quads = a.nsrc == 4 && a.nout == 7 && b.nsrc == 4 && b.nout == 7;
  if (a.set == PACK_WINOGRAD_A && b.set == PACK_WINOGRAD_B && quads)
    return pair_sets<MODE, PACK_WINOGRAD_A, PACK_WINOGRAD_B>(a, b, s);
  if (a.set != PACK_GENERIC || b.set != PACK_GENERIC) return cudaErrorInvalidValue;
  return pair_sets<MODE, PACK_GENERIC, PACK_GENERIC>(a, b, s);
}

cudaError_t launch_pack_pair(const PackArgs &a, const PackArgs &b, int mode, cudaStream_t s) {
  if (a.transpose || !b.transpose || a.prow_pad == 0 || a.pcol_pad == 0 || b.prow_pad == 0 || b.pcol_pad == 0)
    return cudaErrorInvalidValue;
  switch (mode) {
    case MODE_MODP1: return pair_mode<MODE_MODP1>(a, b, s);
    case MODE_MODP2: return pair_mode<MODE_MODP2>(a, b, s);
    case MODE_FP32: return pair_mode<MODE_FP32>(a, b, s);
  }
  return cudaErrorInvalidValue;
}

template <int MODE>
static cudaError_t level_mode(const PackLevel &L, int side, cudaStream_t s) {
  if (side == 0) {
    const int64_t units = (int64_t)L.prow_pad[0] * (L.pcol_pad[0] / dev::kLvlRowN);
    const int64_t want = (units + 255) / 256;
    const int na = (int)(want > 152 * 8 ? 152 * 8 : want);
    if (na > 0) dev::level_rows_kernel<MODE><<<na, 256, 0, s>>>(L);
    return cudaGetLastError();
  }
  constexpr int smem = 16 * dev::kLvlTileK * (dev::kLvlTileN + 1) * 4;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(dev::level_cols_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int tiles_x = L.prow_pad[1] / dev::kLvlTileN, tiles = tiles_x * (L.pcol_pad[1] / dev::kLvlTileK);
  const int grid = tiles < 152 * 2 ? tiles : 152 * 2;  // two resident blocks per SM
  if (tiles > 0) dev::level_cols_kernel<MODE><<<grid, dev::kLvlColThreads, smem, s>>>(L, tiles_x, tiles);
  return cudaGetLastError();
}

cudaError_t launch_pack_level(const PackLevel &L, int side, int mode, cudaStream_t s) {
  if (L.n < 1 || L.n > kMaxOut || side < 0 || side > 1) return cudaErrorInvalidValue;
  const int planes = mode == MODE_MODP1 ? 1 : 2;
  for (int side = 0; side < 2; ++side) {
    if (L.prow_pad[side] <= 0 || L.pcol_pad[side] <= 0 || L.prow_pad[side] % 64 || L.pcol_pad[side] % 64 ||
        L.rows[side] < 0 || L.cols[side] < 0 ||
        L.ostride[side] < planes * (int64_t)L.prow_pad[side] * L.pcol_pad[side])
      return cudaErrorInvalidValue;
    for (int Q = 0; Q < 4; ++Q)
      if (L.esz[side][Q] != 4 && L.esz[side][Q] != 2) return cudaErrorInvalidValue;
  }
  if (L.prow_pad[0] < L.rows[0] || L.pcol_pad[0] < L.cols[0] || L.prow_pad[1] < L.cols[1] ||
      L.pcol_pad[1] < L.rows[1])
    return cudaErrorInvalidValue;
  switch (mode) {
    case MODE_MODP1: return level_mode<MODE_MODP1>(L, side, s);
    case MODE_MODP2: return level_mode<MODE_MODP2>(L, side, s);
    case MODE_FP32: return level_mode<MODE_FP32>(L, side, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_amax(const AmaxArgs &a, cudaStream_t s) {
  const int64_t rows = a.rows[0] > a.rows[1] ? a.rows[0] : a.rows[1];
  if (rows <= 0) return cudaSuccess;
  dim3 grid((unsigned)(rows < 152 * 4 ? rows : 152 * 4), 2);
  dev::amax_kernel<<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}


template <int MODE>
static cudaError_t gemm_mode(const GemmParams &P, int num_sms, cudaStream_t s) {
  constexpr int smem = dev::smem_bytes<MODE>();
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(dev::gemm_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  int grid = P.total_tiles < num_sms ? P.total_tiles : num_sms;
  if (grid <= 0) return cudaSuccess;
  dev::gemm_kernel<MODE><<<grid, dev::kThreads, smem, s>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_gemm_tc(const GemmParams &P, int mode, int num_sms, cudaStream_t s) {
  switch (mode) {
    case MODE_MODP1: return gemm_mode<MODE_MODP1>(P, num_sms, s);
    case MODE_MODP2: return gemm_mode<MODE_MODP2>(P, num_sms, s);
    case MODE_FP32: return gemm_mode<MODE_FP32>(P, num_sms, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_leaf_simt(const SimtArgs &A, const GemmParams &P, int mode, cudaStream_t s) {
  if (A.M == 0 || A.N == 0) return cudaSuccess;
  dim3 block(16, 16);
  dim3 grid((A.N + 15) / 16, (A.M + 15) / 16);
  dev::leaf_simt_kernel<<<grid, block, 0, s>>>(A, P, mode);
  return cudaGetLastError();
}

}  // namespace swmm
