// Recursive executor: walks the paper's schedule tables and lowers each row
// to kernel launches in row order, on one stream or, under a Flow, on
// capture streams ordered by the memory each launch touches.
#pragma once

#include <cstdint>
#include <string>

#include <vector>

#include "flow.h"
#include "schedules.h"
#include "swmm_internal.h"

namespace swmm {

struct Scalar {
  uint32_t u = 0;  // mod p value in [0, p)
  float f = 0.f;   // FP32 mode value
};

// An operand given as a signed sum of up to kMaxTerm blocks of one shape:
// a pre-addition of the level above that is formed while the fused level
// packs its operands, instead of being written to a temporary.
struct Lin {
  int n = 0;
  View v[kMaxTerm];
  int8_t s[kMaxTerm] = {0, 0, 0, 0};
  static Lin of(const View &x) {
    Lin l;
    l.n = 1;
    l.v[0] = x;
    l.s[0] = 1;
    return l;
  }
  const View &shape() const { return v[0]; }
};

// One classical product of a grouped leaf launch: D <- alpha L R (+ beta D).
struct LeafJob {
  View L, R, D;
};

// Where a recursion level takes its temporaries X, Y, Z from.
struct Arena {
  bool carve = false;  // true: quadrants of `region` (Algorithm 2 carves C22)
  View region;
};

// Event pair around leaf GEMM launches (SWMM_FLAG_TIMING).
struct TimingHook {
  virtual void begin(cudaStream_t s) = 0;
  virtual void end(cudaStream_t s, double tensor_flops) = 0;
  virtual ~TimingHook() {}
};

struct Exec {
  // configuration
  int mode = MODE_MODP2;
  uint32_t p = 0;
  bool fp32 = false;
  bool fused = true;
  bool simt = false;
  bool dry = true;  // planning pass: count and size, launch nothing
  cudaStream_t stream = nullptr;
  int num_sms = 152;
  int *err = nullptr;
  uint64_t wait_ns = 4000000000ull;  // bound of the GEMM's device-side waits
  int *stall_left = nullptr;         // test hook: GEMM launches still to stall (handle counter)
  TimingHook *timing = nullptr;
  // the handle's own schedule (K_CUSTOM), if any
  const KindInfo *custom = nullptr;
  const KindInfo &info(Kind k) const { return k == K_CUSTOM ? *custom : kind_info(k); }

  // workspace for temporaries (bump allocator, bytes); ws_limit >= 0 is the
  // size of the area given to a real run (a temporary past it fails the
  // call instead of writing beyond the area)
  char *ws = nullptr;
  int64_t ws_top = 0, ws_peak = 0, ws_limit = -1;
  // tensor-core operand staging (bytes): stage_slots areas of stage_need
  // bytes used in turn by successive leaf launches (two under a Flow, so
  // the next leaf's operands are packed while the current one multiplies)
  char *stage = nullptr;
  int64_t stage_need = 0, stage_limit = -1;  // stage_limit >= 0: bytes of the area at `stage`
  // > 0: operand staging bound (SWMM_FLAG_LOWMEM); products of a fused level
  // or of a leaf group are staged and multiplied in groups that fit it
  int64_t stage_budget = 0;
  int stage_slots = 1;
  int stage_turn = 0;
  // table levels that packed the operands of all their fused levels in one
  // pass (each stages one area; two areas in turn when there are several,
  // so one level's pack need not wait for the previous level's products)
  int level_packs = 0;
  bool level_pack_ok = true;  // the call may pack table levels in one pass
  // dataflow ordering over capture streams (null: every launch on `stream`)
  Flow *flow = nullptr;
  // Deferred leaf GEMM launches: products of leaf groups and fused levels
  // wait in `pend` and independent ones share one launch (merge = true), so
  // the fixed cost of a launch is paid once for several small levels.  The
  // pending launch is issued before any operation that touches its memory.
  bool merge = false;
  struct Pending {
    GemmParams P;
    int n = 0, tiles = 0;
    double flops = 0.0;
    bool additive = true;  // every product only reduce-adds into its targets
    std::vector<Rect> rd, wr;
  };
  Pending pend;
  bool flushing = false;
  void flush();

  // statistics
  int64_t tmp_elems = 0, tmp_peak_elems = 0;
  int64_t add_elems = 0, leaf_flops = 0, leaf_launches = 0, ew_launches = 0, leaf_products = 0;
  int64_t pack_bytes = 0;        // bytes the operand packs read and write
  int64_t level_pack_bytes = 0;  // the part of pack_bytes moved by one-pass level packs

  // Blocks holding unreduced representatives mod p (destinations of a fused
  // level's reduce-adds) that no later operation has brought back to
  // [0, p); only these need the final canonical pass.
  std::vector<View> lazy_views;
  void mark_lazy(const View &v);
  void mark_canonical(const View &v);  // every element of v is now in [0, p)

  cudaError_t cuda_err = cudaSuccess;
  std::string fail;  // first failure description

  bool ok() const { return cuda_err == cudaSuccess && fail.empty(); }

  // D <- alpha L R (+ beta D when acc) by schedule `k` with `depth` levels.
  void call(Kind k, Scalar alpha, bool acc, Scalar beta, View L, View R, View D, int depth, const Arena &ar);
  // classical leaf product (one tensor-core launch)
  void leaf(Scalar alpha, bool acc, Scalar beta, View L, View R, View D);
  // classical products of independent problems in one grouped launch
  void leaf_group(Scalar alpha, bool acc, Scalar beta, const LeafJob *jobs, int njobs);
  // Algorithm 2 (IPMM)
  void ipmm(View L, View R, View D, int depth, int64_t cutoff, Kind acc_kind);
  // Algorithm 1 (IP0vMM): D <- alpha L R for n < m, n <= k, n | m, n | k
  void ip0vmm(Scalar alpha, View L, View R, View D, int depth);
  // Section 7.2: D <- alpha L R + beta D by t x t blocks of D
  void tblock(Scalar alpha, Scalar beta, View L, View R, View D, int t, int depth, Kind acc_kind);
  // Host <-> device copies of a block and the canonical pass of a block, as
  // ordered operations (under a Flow they wait only for the launches that
  // touch the block; `token` chains copies of one direction in issue order)
  void copy_in(View dv, const char *host, int64_t hld, const Rect &token);
  void copy_out(char *host, int64_t hld, View dv, const Rect &token);
  void canon(View v);

 private:
  // operands of a fused level formed by its table level's one pack: this
  // level's staging (its A operands, then its B operands) and the staging
  // base that holds the FP32 amax words
  struct Prepacked {
    char *base;
    char *stg;
  };
  void fused_level(Scalar alpha, bool acc, Scalar beta, const Lin &L, const Lin &R, View D,
                   const Prepacked *pre = nullptr);
  void level_bytes(const View &L, const View &R, int64_t &abytes, int64_t &bbytes) const;
  void pack_args(const Lin &LL, const Lin &RL, int g0, int gn, char *stg, const uint32_t *amax, PackArgs &pa,
                 PackArgs &pb) const;
  // would call() with these sizes and depth run a fused level?
  bool fuses(int64_t m, int64_t k, int64_t n, int depth) const;
  void peel(Kind k, Scalar alpha, bool acc, Scalar beta, View L, View R, View D, int depth, const Arena &ar);
  void table(Kind k, Scalar alpha, bool acc, Scalar beta, View L, View R, View D, int depth, const Arena &ar);
  void add(View d, View s1, View s2, Scalar c1, Scalar c2);
  // stream for a launch reading rd and writing wr; op_end() after issuing it
  cudaStream_t op_begin(const std::vector<Rect> &rd, const std::vector<Rect> &wr, bool dma = false);
  void op_end();
  char *next_stage();
  void queue_gemm(const GemmParams *P, const std::vector<Rect> &rd, const std::vector<Rect> &wr, bool additive,
                  double flops, int nprod);
  void fp32_amax(uint32_t *amax, const View *a, int na, const View *b, int nb);
  void scale(View d, bool keep, Scalar beta);  // d <- beta d, or 0
  void check(cudaError_t e, const char *what);
  View alloc_tmp(int64_t rows, int64_t cols);
  Scalar one() const;
  int limb_products() const;
  Scalar neg(Scalar s) const;
};

}  // namespace swmm
