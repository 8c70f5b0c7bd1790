// Internal interfaces shared by the host executor and the CUDA kernels.
#pragma once

#include <cmath>
#include <cstdint>
#include <cstring>
#include <cuda.h>
#include <cuda_runtime.h>

namespace swmm {

constexpr int kErrTimeout = 5;  // matches SWMM_ETIMEOUT

// A strided 2-D block of 32-bit elements (int32 mod p or float), or of
// 16-bit elements (esz = 2: values in [0, p) of a schedule temporary over
// Z/pZ with p < 2^16).
struct View {
  char *ptr = nullptr;
  int64_t rows = 0, cols = 0, ld = 0;  // ld in elements
  char *base = nullptr;                // root of the matrix the view was cut from (null: ptr)
  int esz = 4;                         // bytes per element
  char *at(int64_t r, int64_t c) const { return ptr + esz * (r * ld + c); }
  View sub(int64_t r0, int64_t c0, int64_t nr, int64_t nc) const {
    View v;
    v.base = base ? base : ptr;
    v.ptr = at(r0, c0);
    v.rows = nr;
    v.cols = nc;
    v.ld = ld;
    v.esz = esz;
    return v;
  }
  // the same rows as 16-bit elements: same row pitch in bytes, each row's
  // values in the first half of its bytes (so a view carved from a larger
  // block stays inside that block)
  View narrow() const {
    View v = *this;
    if (esz == 4) {
      v.esz = 2;
      v.ld = 2 * ld;
    }
    return v;
  }
  // quadrant (i, j) in {0,1}^2 of an even-sized block (Section 2 split)
  View quad(int i, int j) const { return sub(i * (rows / 2), j * (cols / 2), rows / 2, cols / 2); }
};

// Leaf arithmetic: one fp16 limb (p <= 256), two fp16 limbs (p < 2^16), or
// fp16 hi/lo of a scaled float (FP32 mode).
enum Mode : int { MODE_MODP1 = 0, MODE_MODP2 = 1, MODE_FP32 = 2 };

// Output columns of a leaf tile for p < 2^16.  Its four limb products need
// 4 x BN tensor-memory columns: BN = 128 fills the 512 columns with one
// accumulator (the next tile's MMAs wait for the epilogue to read it out);
// BN = 64 leaves room for two, but its N = 128 MMAs and twice the A-tile
// reloads ran the classical product at 1263 instead of 1788 TFLOP/s.
constexpr int kModp2BN = 128;

inline int planes_of(int mode) { return mode == MODE_MODP1 ? 1 : 2; }
inline int bn_of(int mode) { return mode == MODE_MODP1 ? 256 : (mode == MODE_MODP2 ? kModp2BN : 128); }
constexpr int kBM = 128;  // leaf tile rows
// Leaf k-block: 64 fp16 values = one 128-byte row (128-byte swizzle).  32
// (64-byte rows, twice the stages in the same shared memory) was measured
// slower: 1643 against 1760 TFLOP/s on the classical product.
constexpr int kBK = 64;

// ------------------------------------------------------------------ packing
// Operand staging for the tensor cores.  A pack launch reads up to four
// source blocks Q_0..Q_3 (rows x cols, int32 mod p or float) and writes up
// to seven outputs; output o is sum_s coef[o][s] * Q_s, converted to limb
// planes of 16-bit values.  Plain layout: plane-major, then rows_pad rows of
// cols_pad halves (K contiguous).  Transposed layout (B operands): the
// packed row index is the source column.  Entries outside rows x cols are 0.
// Each source may itself be a signed sum of up to kMaxTerm blocks (a
// pre-addition of the level above): Q_s = sum_t tsign[t] * src[s][t].
constexpr int kMaxSrc = 4;
constexpr int kMaxOut = 7;
constexpr int kMaxTerm = 4;
struct PackArgs {
  const char *src[kMaxSrc][kMaxTerm];
  int64_t ld[kMaxSrc][kMaxTerm];
  int8_t tsign[kMaxTerm];
  int8_t tesz[kMaxTerm];  // bytes per element of each term's blocks: 4, or 2 (16-bit mod p values)
  int32_t nterm;  // >= 1
  int32_t nsrc;
  uint16_t *out[kMaxOut];
  int8_t coef[kMaxOut][kMaxSrc];
  int32_t nout;
  int32_t rows, cols;          // source extent
  int32_t prow_pad, pcol_pad;  // packed extent (packed rows x packed cols)
  int32_t transpose;
  uint32_t p;
  uint32_t barrett;  // floor(2^32 / p)
  int32_t set;       // PACK_GENERIC: coef; PACK_WINOGRAD_A / _B: the Section 2 sums
  // FP32 mode: max |source| (float bits, written on the device by
  // launch_amax) and the largest sum of |coef| over the outputs; the pack
  // scales every value by fp16_scale(*amax, terms) before splitting it.
  const uint32_t *amax;
  int32_t terms;
};
// Output sets of a pack launch.  The Winograd sets take the four quadrants
// (X11, X12, X21, X22) and write, in order, A11, A12, S4, A22, S1, S2, S3
// (A side) or B11, B21, B22, T4, T1, T2, T3 (B side), forming the chains
// S2 = S1 - A11, S4 = A12 - S2 and T2 = B22 - T1, T4 = T2 - B21 once.
enum PackSet : int { PACK_GENERIC = 0, PACK_WINOGRAD_A = 1, PACK_WINOGRAD_B = 2 };
// a (plain layout) and b (transposed: packed row = source column) in one launch
cudaError_t launch_pack_pair(const PackArgs &a, const PackArgs &b, int mode, cudaStream_t s);
// The packs of the n fused levels under one table level in one pass.  Side
// 0 is the A side (plain layout), side 1 the B side (transposed).  src[s][Q]
// [q] is sub-block q (X11, X12, X21, X22) of operand quadrant Q of side s;
// level j's operand is sum_Q coef[s][j][Q] * quadrant Q, and its seven
// Winograd outputs (Section 2's sums; the order of the Winograd pack sets)
// are at out[s][j] + i * ostride[s] halves.  rows x cols is a sub-block's
// extent, prow_pad x pcol_pad an output's packed extent (multiples of 64).
// launch_pack_level forms one side's outputs (the two sides may run at
// once).
struct PackLevel {
  const char *src[2][4][4];
  int64_t ld[2][4];
  int8_t esz[2][4];  // 4, or 2 (16-bit mod p values)
  int8_t coef[2][kMaxOut][4];
  uint16_t *out[2][kMaxOut];
  int64_t ostride[2];
  int32_t rows[2], cols[2], prow_pad[2], pcol_pad[2];
  // FP32 mode: amax[s] bounds every entry of side s, terms[s][j] the sum of
  // |coefficients| of level j's operands (the scale fp16_scale uses)
  const uint32_t *amax;
  int32_t terms[2][kMaxOut];
  uint32_t p, barrett;
  int32_t n;
};
cudaError_t launch_pack_level(const PackLevel &L, int side, int mode, cudaStream_t s);

// ---------------------------------------------------------------- leaf GEMM
// One product of a grouped leaf launch: P = A' x B' from packed operands.
// Epilogue STORE: T0 <- alpha * P + beta * T0 (only target 0).
// Epilogue REDUCE: for each target t, T_t += sign_t * alpha * P (mod p: the
// canonical contribution, p - v for a negative sign, added as an unsigned
// integer, so targets hold representatives that are reduced later).
constexpr int kMaxTargets = 4;
constexpr int kMaxProducts = 21;  // 7 per fused level (3 merged), or up to 21 classical leaves

struct Target {
  void *ptr;
  int64_t ld;
  int32_t sign;
  int32_t vec_ok;  // 16-byte aligned rows
};

struct Product {
  CUtensorMap ta;  // packed A': 2-D (K_pad halves) x (planes * M_pad rows)
  CUtensorMap tb;  // packed B': 2-D (K_pad halves) x (planes * N_pad rows)
  CUtensorMap tmap[kMaxTargets];  // targets (fp32 words, 32 x 128 boxes, 128-byte swizzle)
  int32_t tma_epi;                // every target addressable by TMA: staged epilogue
  Target t[kMaxTargets];
  int32_t ntargets;
  int32_t M, N, Kpad;
  int32_t a_plane_rows, b_plane_rows;  // M_pad, N_pad
  int32_t tiles_m, tiles_n;
  int32_t tile_begin;  // first global tile index of this product
  // FP32 mode: the A-side and B-side amax words and term counts of this
  // product's packs, to undo their scales in the epilogue
  const uint32_t *amax;  // [2]: A side, B side
  int32_t terms_a, terms_b;
  // scalars and epilogue of this product (one launch may hold products of
  // different calls): STORE t0 <- alpha P (+ beta t0 when use_beta), or
  // REDUCE every target += sign alpha P
  int32_t epilogue, use_beta;
  uint32_t alpha_u, beta_u;
  float alpha_f, beta_f;
};

enum Epilogue : int { EPI_STORE = 0, EPI_REDUCE = 1 };

// The scalar and epilogue fields here serve the SIMT diagnostic leaf; the
// tensor-core kernel reads the per-product copies.
struct GemmParams {
  Product prod[kMaxProducts];
  int32_t nprod;
  int32_t total_tiles;
  int32_t epilogue;
  uint32_t p;        // modulus (mod p modes)
  uint32_t alpha_u;  // alpha mod p
  uint32_t beta_u;   // beta mod p (STORE)
  float alpha_f, beta_f;
  uint32_t barrett;  // floor(2^32 / p)
  float inv_p;       // 1/p rounded to float
  int32_t use_beta;  // STORE: read T0 and add beta * T0
  int *err;          // device error word (bounded waits)
  uint64_t wait_ns;  // bound of every mbarrier wait (globaltimer ns)
  int32_t test_stall;  // test hook: the producer first waits on a barrier nothing arrives at
};
static_assert(sizeof(GemmParams) <= 32764, "kernel parameter space");

// FP32 mode operand scale: a power of two s with |x s| < 2^14 for every
// value the pack writes (|x| <= terms * amax), so that hi = fp16(x s) and
// lo = fp16(x s - hi) stay in fp16's normal range; 1 for a zero or
// non-finite bound.
__host__ __device__ inline float fp16_scale(uint32_t amax_bits, int terms) {
  float a;
  memcpy(&a, &amax_bits, 4);
  const float bound = a * (float)terms;
  if (!(bound > 0.f) || !(bound < 3.0e38f)) return 1.f;
  int e;
  frexpf(bound, &e);  // bound < 2^e
  return ldexpf(1.f, 14 - e);
}

// max |x| over up to 4 views per side (side 0: A, side 1: B), atomically
// maxed into amax[side] (float bits; the words must be zeroed first)
struct AmaxArgs {
  const char *src[2][kMaxTerm];
  int64_t ld[2][kMaxTerm];
  int64_t rows[2], cols[2];
  int32_t nsrc[2];
  uint32_t *amax;
};
cudaError_t launch_amax(const AmaxArgs &a, cudaStream_t s);

// Encode a 2-D tensor map over a packed buffer (rows x kpad halves).
bool make_tmap(CUtensorMap *map, const void *base, int64_t rows, int64_t kpad, int box_rows);
// Encode a 2-D tensor map over a target block of 32-bit words (rows x cols,
// leading dimension ld); false when TMA cannot address it (alignment).
bool make_target_tmap(CUtensorMap *map, const void *base, int64_t rows, int64_t cols, int64_t ld, bool fp32);

cudaError_t launch_gemm_tc(const GemmParams &P, int mode, int num_sms, cudaStream_t s);

// SIMT reference leaf on raw (unpacked) operands, for diagnostics: one
// product, operands as signed sums of up to four views.
struct SimtArgs {
  const char *a[4];
  int64_t lda[4];
  int32_t sa[4], na;
  const char *b[4];
  int64_t ldb[4];
  int32_t sb[4], nb;
  Target t[kMaxTargets];
  int32_t ntargets;
  int32_t M, N, K;
};
cudaError_t launch_leaf_simt(const SimtArgs &A, const GemmParams &P, int mode, cudaStream_t s);

// -------------------------------------------------------------- elementwise
// dst <- c1 * s1 + c2 * s2 over an r x c block; coefficients are reduced
// mod p (mod p mode) or used as floats.  dst may equal s1 or s2 exactly.
cudaError_t launch_add(View dst, View s1, View s2, int64_t c1, int64_t c2, uint32_t p, int fp32,
                       cudaStream_t s);
cudaError_t launch_add_f(View dst, View s1, View s2, float c1, float c2, cudaStream_t s);
// FP32: dst <- coef * dst (coef 0 writes zeros)
cudaError_t launch_scale_f(View dst, float coef, cudaStream_t s);
// mod p: dst <- coef * dst mod p, canonical (int32 in place; coef 0 writes 0)
cudaError_t launch_scale_modp(View dst, uint32_t coef, uint32_t p, cudaStream_t s);
// mod p: dst <- dst mod p (any representative below 2^32 -> [0, p))
cudaError_t launch_canon_modp(View dst, uint32_t p, cudaStream_t s);
// dst <- 0
cudaError_t launch_zero(View dst, cudaStream_t s);
// dst <- src
cudaError_t launch_copy(View dst, View src, uint32_t p, cudaStream_t s);

// ------------------------------------------------------- residual probe
// y = M x for a row-major rows x cols matrix (mod p: int32 elements, uint32
// x and y in [0, p); FP32 mode: float elements, double x and y).
cudaError_t launch_matvec(const void *M, int64_t rows, int64_t cols, int64_t ld, const void *x, void *y, uint32_t p,
                          bool modp, int num_sms, cudaStream_t s);
// r = v - alpha u - beta y0 elementwise over m entries (y0 may be null)
cudaError_t launch_residual(int64_t m, const void *v, const void *u, const void *y0, void *r, uint32_t au,
                            uint32_t bu, double af, double bf, uint32_t p, bool modp, int num_sms, cudaStream_t s);

}  // namespace swmm
