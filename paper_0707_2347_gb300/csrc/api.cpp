// C ABI of the library (include/swmm.h): argument validation, planning,
// workspace management, CUDA-graph capture and dispatch to the executor.
#include "swmm.h"
#include "swmm_search.h"

#include <algorithm>
#include <array>
#include <cstddef>
#include <cstdio>
#include <tuple>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "executor.h"

namespace swmm {

// ------------------------------------------------------------ tensor maps
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// 2-D map over `rows` rows of `kpad` 16-bit values; boxes of kBK x box_rows
// land in shared memory with the swizzle (64-byte rows: 64-byte swizzle)
// the MMA descriptors use.
bool make_tmap(CUtensorMap *map, const void *base, int64_t rows, int64_t kpad, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)kpad, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)kpad * 2};
  cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, const_cast<void *>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, kBK * 2 == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool make_target_tmap(CUtensorMap *map, const void *base, int64_t rows, int64_t cols, int64_t ld, bool fp32) {
  EncodeTiledFn fn = encode_fn();
  // TMA stores write whole 16-byte chunks at the inner boundary: a width that
  // is not a multiple of 4 words would clobber the neighbouring columns, so
  // such targets take the epilogue's direct path.
  if (!fn || ((uintptr_t)base % 16) != 0 || (ld % 4) != 0 || rows <= 0 || cols <= 0 || (cols % 4) != 0) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
  cuuint32_t box[2] = {32, (cuuint32_t)kBM};
  cuuint32_t estr[2] = {1, 1};
  // the element type matters for TMA reduce-add: float sums or unsigned
  // integer sums of mod p contributions
  CUresult r = fn(map, fp32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT32, 2,
                  const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// Event pairs around leaf GEMM launches (SWMM_FLAG_TIMING).
constexpr uint64_t kDefaultWaitNs = 4000000000ull;  // 4 s

struct EventTimer : TimingHook {
  std::vector<cudaEvent_t> ev;  // pairs: 2i = begin, 2i + 1 = end
  std::vector<double> flops;
  size_t used = 0;  // pairs recorded since the last reset
  void begin(cudaStream_t s) override {
    if (2 * used + 2 > ev.size()) {
      cudaEvent_t a, b;
      cudaEventCreate(&a);
      cudaEventCreate(&b);
      ev.push_back(a);
      ev.push_back(b);
      flops.push_back(0.0);
    }
    record(ev[2 * used], s);
  }
  // Inside a stream capture an external record becomes an event node of the
  // graph, so each replay refreshes the timestamps; outside, a plain record.
  static void record(cudaEvent_t e, cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cs);
    if (cs == cudaStreamCaptureStatusActive)
      cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
    else
      cudaEventRecord(e, s);
  }
  void end(cudaStream_t s, double f) override {
    record(ev[2 * used + 1], s);
    flops[used] = f;
    ++used;
  }
  ~EventTimer() override {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  }
};

// A captured call: its instantiated graph, the statistics of the capture and
// the leaf-timing events recorded in it (their times refresh on each replay).
struct GraphEntry {
  std::string key;
  cudaGraphExec_t exec = nullptr;
  swmm_stats stats;
  EventTimer timer;
  std::vector<int32_t> chosen;  // batched calls: (sched, depth) per problem
  GraphEntry() { std::memset(&stats, 0, sizeof(stats)); }
  ~GraphEntry() {
    if (exec) cudaGraphExecDestroy(exec);
  }
};

}  // namespace swmm

using namespace swmm;

struct swmm_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int num_sms = 152;
  int *d_err = nullptr;
  // swmm_test_hook: bound of the device-side waits, GEMM launches still to
  // stall, device allocations still to fail
  uint64_t wait_ns = kDefaultWaitNs;
  int stall_left = 0;
  int fail_allocs = 0;
  int64_t lowmem_bytes = SWMM_LOWMEM_STAGE_BYTES;  // staging bound of SWMM_FLAG_LOWMEM calls
  swmm_stats stats;
  std::string last_error;
  EventTimer timer;
  EventTimer *last_timer = &timer;
  // CUDA graph cache (SWMM_FLAG_GRAPH)
  std::vector<std::unique_ptr<GraphEntry>> graphs;
  cudaStream_t cap = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  // dataflow capture: side streams and an event per launch of a captured call
  cudaStream_t flow_streams[kFlowStreams - 1] = {};
  std::vector<cudaEvent_t> flow_events;
  // swmm_muladd_host: device copies of the operands (grown on demand) and
  // two host bytes whose addresses order the copies of each direction
  char *io_buf = nullptr;
  size_t io_bytes = 0;
  char io_token[2] = {0, 0};
  // the handle's own schedule (SWMM_CUSTOM, swmm_set_schedule)
  CustomSchedule custom;
  KindInfo custom_info{"custom", nullptr, false, true};
  bool has_custom = false;
  // autotuner decisions: (m, k, n, mode, p) -> (sched, depth, est_us, elems)
  std::vector<std::pair<std::array<int64_t, 5>, std::tuple<int32_t, int32_t, double, int64_t>>> tuned;
  // measured decisions of batched calls with SWMM_FLAG_TUNE: (m, k, n, mode, p) -> (sched, depth)
  std::vector<std::pair<std::array<int64_t, 5>, std::pair<int32_t, int32_t>>> measured;
  ~swmm_ctx() {
    graphs.clear();
    for (cudaStream_t s : flow_streams)
      if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : flow_events) cudaEventDestroy(e);
    if (io_buf) cudaFree(io_buf);
    if (cap) cudaStreamDestroy(cap);
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_out) cudaEventDestroy(ev_out);
  }
};

namespace {

// swmm_test_hook(SWMM_HOOK_FAIL_ALLOCS): true when this allocation is to fail
bool injected_alloc_failure(swmm_t h) {
  if (h->fail_allocs <= 0) return false;
  --h->fail_allocs;
  return true;
}

int fail(swmm_t h, int code, const std::string &msg) {
  if (h) h->last_error = msg;
  return code;
}

struct Req {
  int entry;  // 0 mul, 1 muladd, 2 inplace
  int64_t m, k, n;
  const void *A, *B;
  void *C;
  int64_t lda, ldb, ldc;
  const void *alpha, *beta;
};

Kind kind_of(int sched) {
  switch (sched) {
    case SWMM_T1_DHSS: return K_T1;
    case SWMM_T2_HLJJTT: return K_T2;
    case SWMM_T3_IP: return K_IP;
    case SWMM_T4_OVL: return K_OVL;
    case SWMM_T4M_OVL: return K_OVLM;
    case SWMM_T5_OVR: return K_OVR;
    case SWMM_T6_ACLR: return K_ACLR;
    case SWMM_T7_ACCR: return K_ACCR;
    case SWMM_T8_ACR: return K_ACR;
    case SWMM_T9_ACC: return K_ACC;
    case SWMM_CUSTOM: return K_CUSTOM;
  }
  return NKIND;
}

// Temporaries per level the paper gives for each schedule (Section 3,
// Section 5, Section 6), summed over `levels` levels: the Lemma 1 series.
int64_t paper_elems(int sched, int64_t m, int64_t k, int64_t n, int levels, int custom_temps = 0) {
  int64_t s = 0;
  for (int i = 0; i < levels; ++i) {
    m /= 2;
    k /= 2;
    n /= 2;
    switch (sched) {
      case SWMM_T1_DHSS: s += m * std::max(k, n) + k * n; break;  // Eq. (1)
      case SWMM_T2_HLJJTT: s += m * k + k * n + m * n; break;    // Eq. (2)
      case SWMM_T4_OVL:
      case SWMM_T4M_OVL:
      case SWMM_T5_OVR: s += n * n; break;  // Sec. 5.1
      case SWMM_T6_ACLR:
      case SWMM_T7_ACCR:
      case SWMM_T9_ACC: s += 2 * n * n; break;                  // Eq. (3), Sec. 6
      case SWMM_T8_ACR: s += std::max(m, k) * n + m * k; break;  // Sec. 5.3
      case SWMM_CUSTOM: s += custom_temps * n * n; break;        // its own temporaries
      default: break;                                           // IP, IPMM, classical: 0
    }
  }
  return s;
}

// number of Winograd levels the recursion performs (odd dimensions are
// peeled, so each level halves the even core)
int levels_possible(int64_t m, int64_t k, int64_t n, int depth) {
  int d = 0;
  while (d < depth && m >= 2 && k >= 2 && n >= 2) {
    m /= 2;
    k /= 2;
    n /= 2;
    ++d;
  }
  return d;
}

bool overlaps(const void *a, int64_t ar, int64_t ac, int64_t lda, const void *b, int64_t br, int64_t bc,
              int64_t ldb) {
  if (ar == 0 || ac == 0 || br == 0 || bc == 0) return false;
  const char *a0 = (const char *)a, *a1 = a0 + 4 * ((ar - 1) * lda + ac);
  const char *b0 = (const char *)b, *b1 = b0 + 4 * ((br - 1) * ldb + bc);
  return a0 < b1 && b0 < a1;
}

struct Scratch {
  char *base;
  int64_t bytes;
};

// operand staging per slot up to which leaf launches are merged
constexpr int64_t kMergeStageBytes = 96ll << 20;
// base of the temporaries in a planning pass (a placeholder above any device
// address; the pass never dereferences it)
char *const kPlanWorkspace = reinterpret_cast<char *>(uintptr_t(4) << 44);

void reset_counts(Exec &x) {
  x.ws_top = x.ws_peak = x.stage_need = 0;
  x.tmp_elems = x.tmp_peak_elems = 0;
  x.add_elems = x.leaf_flops = x.leaf_launches = x.ew_launches = x.leaf_products = 0;
  x.pack_bytes = x.level_pack_bytes = 0;
  x.level_packs = 0;
  x.lazy_views.clear();
  x.stage_turn = 0;
}

// A validated, planned call.
struct Plan {
  Req q;
  swmm_opts o;
  Exec x;  // the dry run: sizes and counts
  View L, R, D;
  Scalar alpha, beta;
  bool accum = false, ne = false;
  int sched = 0, depth = 0, lv = 0;
  int64_t cutoff = 1024;
  Kind ipmm_acc = K_T2;  // accumulation kind of IPMM and of the Section 7.2 blocks
  int tblock = 2;
  int64_t paper = 0;
  std::vector<LeafJob> jobs;  // a grouped launch of classical problems (batched calls)
  // host operands (swmm_muladd_host): L, R, D are the handle's device copies
  bool host_io = false;
  const char *hA = nullptr, *hB = nullptr;
  char *hC = nullptr;
  int64_t hlda = 0, hldb = 0, hldc = 0;
};

// The 2 x 2 blocks of A, B and C in the order the top level's table first
// reads them (A, B, C in order for the other drivers), so that copies to
// the device arrive in the order the work needs them.
std::vector<Loc> first_use(swmm_t h, int sched) {
  std::vector<Loc> order;
  auto add = [&](Loc l) {
    if (l <= C22 && std::find(order.begin(), order.end(), l) == order.end()) order.push_back(l);
  };
  const Kind k = kind_of(sched);
  if (k != NKIND) {
    for (const Row &row : k == K_CUSTOM ? h->custom.rows : *kind_info(k).table) {
      if (row.op == OP_MUL) {
        add(row.s1);
        add(row.s2);
        if (row.acc) add(row.dst);
      } else {
        add(row.s1);
        if (row.op == OP_ADD) add(row.s2);
      }
    }
  }
  for (int l = A11; l <= C22; ++l) add((Loc)l);
  return order;
}

// 2 x 2 split of a block that also covers odd sizes
View block_of(const View &v, int i, int j) {
  const int64_t r0 = i ? v.rows / 2 : 0, c0 = j ? v.cols / 2 : 0;
  const int64_t nr = i ? v.rows - v.rows / 2 : v.rows / 2, nc = j ? v.cols - v.cols / 2 : v.cols / 2;
  return v.sub(r0, c0, nr, nc);
}

void execute(const Plan &P, Exec &e) {
  if (!P.ne) return;
  if (!P.jobs.empty())
    e.leaf_group(P.alpha, P.accum, P.beta, P.jobs.data(), (int)P.jobs.size());
  else if (P.sched == SWMM_IPMM)
    e.ipmm(P.L, P.R, P.D, P.depth, P.cutoff, P.ipmm_acc);
  else if (P.sched == SWMM_IP0VMM)
    e.ip0vmm(P.alpha, P.L, P.R, P.D, P.depth);
  else if (P.sched == SWMM_TBLOCK)
    e.tblock(P.alpha, P.beta, P.L, P.R, P.D, P.tblock, P.depth, P.ipmm_acc);
  else if (P.sched == SWMM_CLASSICAL)
    e.leaf(P.alpha, P.accum, P.beta, P.L, P.R, P.D);
  else
    e.call(kind_of(P.sched), P.alpha, P.accum, P.beta, P.L, P.R, P.D, P.depth, Arena{});
}

// level_packs: table levels may pack their fused levels in one pass (off
// for calls on a caller's static scratch, which must fit the smaller
// per-level staging)
int make_plan(swmm_t h, const Req &q, const swmm_opts *o, bool check_ptrs, Plan &P, bool level_packs = true) {
  if (!o) return fail(h, SWMM_EINVAL, "opts is NULL");
  if (o->mode != SWMM_MODP && o->mode != SWMM_FP32) return fail(h, SWMM_EINVAL, "unknown mode");
  if (o->mode == SWMM_MODP && (o->p <= 2 || o->p >= 65536)) return fail(h, SWMM_EINVAL, "p must satisfy 2 < p < 65536");
  if (q.m < 0 || q.k < 0 || q.n < 0) return fail(h, SWMM_EINVAL, "negative dimension");
  if (q.m > (1 << 30) || q.k > (1 << 30) || q.n > (1 << 30)) return fail(h, SWMM_EINVAL, "dimension too large");
  if (o->depth < 0 || o->depth > 30) return fail(h, SWMM_EINVAL, "depth out of range");
  const int sched = o->sched;
  const bool accum = q.entry == 1 || (q.entry == 2 && q.beta != nullptr);
  // schedule / entry point consistency (overwrite contracts, Sections 3, 5)
  bool okk = false;
  if (q.entry == 0) okk = sched == SWMM_CLASSICAL || sched == SWMM_T1_DHSS || sched == SWMM_IPMM;
  if (q.entry == 1)
    okk = sched == SWMM_CLASSICAL || sched == SWMM_T2_HLJJTT || sched == SWMM_T9_ACC || sched == SWMM_TBLOCK;
  if (q.entry == 2 && !accum)
    okk = sched == SWMM_T3_IP || sched == SWMM_T4_OVL || sched == SWMM_T4M_OVL || sched == SWMM_T5_OVR ||
          sched == SWMM_IP0VMM;
  if (q.entry == 2 && accum) okk = sched == SWMM_T6_ACLR || sched == SWMM_T7_ACCR || sched == SWMM_T8_ACR;
  if (sched == SWMM_CUSTOM) {
    if (!h->has_custom) return fail(h, SWMM_EINVAL, "no schedule set on this handle (swmm_set_schedule)");
    // the entry point that matches the schedule's contract
    const bool ro = h->custom.preserve == 0xffu;
    okk = h->custom.accumulate == accum && (q.entry == 2 ? !ro : ro && q.entry == (accum ? 1 : 0));
  }
  if (!okk) return fail(h, SWMM_EINVAL, "schedule not valid for this entry point");
  const bool ne = q.m > 0 && q.n > 0;
  if (check_ptrs) {
    if (ne && !q.C) return fail(h, SWMM_EINVAL, "C is NULL");
    if (ne && q.k > 0 && (!q.A || !q.B)) return fail(h, SWMM_EINVAL, "A or B is NULL");
    if (q.lda < std::max<int64_t>(q.k, 1) || q.ldb < std::max<int64_t>(q.n, 1) || q.ldc < std::max<int64_t>(q.n, 1))
      return fail(h, SWMM_EINVAL, "leading dimension smaller than the number of columns");
    if (((uintptr_t)q.A | (uintptr_t)q.B | (uintptr_t)q.C) & 3) return fail(h, SWMM_EINVAL, "pointers must be 4-byte aligned");
    if (overlaps(q.A, q.m, q.k, q.lda, q.C, q.m, q.n, q.ldc) || overlaps(q.B, q.k, q.n, q.ldb, q.C, q.m, q.n, q.ldc))
      return fail(h, SWMM_EINVAL, "A or B overlaps C");
    if (q.entry == 2 && overlaps(q.A, q.m, q.k, q.lda, q.B, q.k, q.n, q.ldb))
      return fail(h, SWMM_EINVAL, "A and B overlap (the schedule overwrites them)");
  }
  const int depth = sched == SWMM_CLASSICAL ? 0 : o->depth;
  const int tb = o->tblock > 0 ? o->tblock : 2;
  if (sched == SWMM_TBLOCK) {
    if (tb < 2 || tb > 64) return fail(h, SWMM_EINVAL, "tblock must be in [2, 64] (Section 7.2)");
    if (q.m % tb || q.k % tb || q.n % tb)
      return fail(h, SWMM_EINVAL, "Section 7.2 blocking needs m, k and n multiples of t");
    if (o->ipmm_acc == SWMM_T9_ACC && !(q.m == q.k && q.k == q.n))
      return fail(h, SWMM_EINVAL, "Section 7.2 with Table 9 blocks needs square operands");
  }
  const int lv = sched == SWMM_TBLOCK ? levels_possible(q.m / tb, q.k / tb, q.n / tb, depth)
                                      : levels_possible(q.m, q.k, q.n, depth);
  if (sched != SWMM_CLASSICAL && sched != SWMM_IPMM && sched != SWMM_IP0VMM && sched != SWMM_TBLOCK && lv > 0) {
    const KindInfo &K = sched == SWMM_CUSTOM ? h->custom_info : kind_info(kind_of(sched));
    if (K.square && !(q.m == q.k && q.k == q.n))
      return fail(h, SWMM_EINVAL, std::string(K.name) + " needs square operands (Section 5.3)");
    if (sched == SWMM_T3_IP && !(q.k == q.n && q.n <= q.m))
      return fail(h, SWMM_EINVAL, "IP needs k = n <= m (Section 5.3)");
  }
  if (sched == SWMM_IPMM && q.m != q.n) return fail(h, SWMM_EINVAL, "IPMM needs m = n (Algorithm 2)");
  if (sched == SWMM_IP0VMM && ne &&
      !(q.n < q.m && q.n <= q.k && q.n > 0 && q.m % q.n == 0 && q.k % q.n == 0))
    return fail(h, SWMM_EINVAL, "IP0vMM needs n < m, n <= k, n dividing m and k (Algorithm 1)");

  P.q = q;
  P.o = *o;
  P.accum = accum;
  P.ne = ne;
  P.sched = sched;
  P.depth = depth;
  P.lv = lv;
  Exec &x = P.x;
  x.fp32 = o->mode == SWMM_FP32;
  x.p = x.fp32 ? 0 : o->p;
  x.mode = x.fp32 ? MODE_FP32 : (o->p <= 256 ? MODE_MODP1 : MODE_MODP2);
  x.fused = !(o->flags & SWMM_FLAG_UNFUSED);
  x.simt = (o->flags & SWMM_FLAG_SIMT_LEAF) != 0;
  x.num_sms = h->num_sms;
  x.stage_budget = (o->flags & SWMM_FLAG_LOWMEM) ? h->lowmem_bytes : 0;
  x.wait_ns = h->wait_ns;
  x.level_pack_ok = level_packs;
  x.stall_left = &h->stall_left;
  x.err = h->d_err;
  x.custom = h->has_custom ? &h->custom_info : nullptr;
  if (x.fp32) {
    P.alpha.f = q.alpha ? *(const float *)q.alpha : 1.f;
    P.beta.f = q.beta ? *(const float *)q.beta : 0.f;
  } else {
    P.alpha.u = q.alpha ? *(const uint32_t *)q.alpha % x.p : 1u;
    P.beta.u = q.beta ? *(const uint32_t *)q.beta % x.p : 0u;
  }
  P.L.ptr = (char *)q.A;
  P.L.rows = q.m;
  P.L.cols = q.k;
  P.L.ld = q.lda;
  P.R.ptr = (char *)q.B;
  P.R.rows = q.k;
  P.R.cols = q.n;
  P.R.ld = q.ldb;
  P.D.ptr = (char *)q.C;
  P.D.rows = q.m;
  P.D.cols = q.n;
  P.D.ld = q.ldc;
  P.cutoff = o->ipmm_cutoff > 0 ? o->ipmm_cutoff : 1024;
  P.ipmm_acc = o->ipmm_acc == SWMM_T9_ACC ? K_ACC : K_T2;
  P.tblock = tb;
  // planning pass: sizes and counts, no launches.  Temporaries get
  // placeholder addresses above every real one (never dereferenced), so the
  // pass sees the same overlaps between blocks as the run.
  x.dry = true;
  x.ws = kPlanWorkspace;
  execute(P, x);
  x.flush();
  if (!x.fail.empty()) return fail(h, SWMM_EINVAL, x.fail);
  // small leaf launches share launches (four staging slots in turn; leaf
  // launches of prepacked levels need no slot of their own)
  if (x.stage_need > 0 && (x.stage_need <= kMergeStageBytes || x.level_packs) && !x.simt && x.leaf_launches > 1 &&
      x.stage_budget == 0) {
    reset_counts(x);
    x.merge = true;
    x.stage_slots = 4;
    execute(P, x);
    x.flush();
    if (!x.fail.empty()) return fail(h, SWMM_EINVAL, x.fail);
  }
  x.ws = nullptr;
  // levels that materialise temporaries: all but a fused last one
  const int tmp_levels = (x.fused && lv > 0 && sched != SWMM_IPMM) ? lv - 1 : lv;
  if (sched == SWMM_TBLOCK)  // one block call's temporaries (Section 7.2)
    P.paper = paper_elems(o->ipmm_acc == SWMM_T9_ACC ? SWMM_T9_ACC : SWMM_T2_HLJJTT, q.m / tb, q.k / tb, q.n / tb,
                          tmp_levels);
  else
    P.paper = paper_elems(sched, q.m, q.k, q.n, tmp_levels, h->custom.temps);
  return SWMM_OK;
}

// The lazy blocks of an executor that overlap `d` (clipped to d when they
// are views of the same root; whole otherwise).
std::vector<View> lazy_in(const Exec &r, const View &d) {
  std::vector<View> out;
  const Rect rd = rect_of(d);
  for (const View &x : r.lazy_views) {
    const Rect rx = rect_of(x);
    if (!overlaps(rx, rd)) continue;
    if (rx.base == rd.base && rx.ld == rd.ld && rx.ld > 0) {
      const int64_t r0 = std::max(rx.r0, rd.r0), c0 = std::max(rx.c0, rd.c0);
      const int64_t r1 = std::min(rx.r0 + rx.rows, rd.r0 + rd.rows), c1 = std::min(rx.c0 + rx.cols, rd.c0 + rd.cols);
      out.push_back(d.sub(r0 - rd.r0, c0 - rd.c0, r1 - r0, c1 - c0));
    } else {
      out.push_back(x);
    }
  }
  return out;
}

// Canonical pass over the lazy parts of block b (host-operand copies back).
void canon_lazy(Exec &r, const View &b) {
  for (const View &v : lazy_in(r, b)) r.canon(v);
}

// Staging areas a run of plan x uses in turn: one area per table level
// packed in one pass (two when there are several), four for merged leaf
// launches, two for fused levels under the dataflow capture, else one.
int stage_slots_for(const Exec &x, bool merge, bool use_flow) {
  if (x.level_packs) return x.level_packs > 1 ? 2 : 1;
  if (merge) return 4;
  return use_flow && x.stage_budget == 0 ? 2 : 1;
}

// Issue a planned call on `stream`: workspace, kernels, final canonical
// pass, release.  Adds its counters to `st`.
int enqueue(swmm_t h, const Plan &P, cudaStream_t stream, TimingHook *timing, const Scratch *ext, swmm_stats &st,
            bool use_flow = false) {
  const Exec &x = P.x;
  Exec r = x;
  r.merge = x.merge && !ext;
  r.stage_slots = stage_slots_for(x, r.merge, use_flow);
  const int64_t stage_bytes = r.stage_slots * ((x.stage_need + 1023) / 1024 * 1024);
  r.dry = false;
  r.lazy_views.clear();
  r.stream = stream;
  r.timing = timing;
  r.ws_top = r.ws_peak = 0;
  r.tmp_elems = r.tmp_peak_elems = 0;
  r.add_elems = r.leaf_flops = r.leaf_launches = r.ew_launches = r.leaf_products = 0;
  r.pack_bytes = r.level_pack_bytes = 0;
  r.level_packs = 0;  // counted again by the run (the plan's count chose the staging areas)
  r.stage_need = x.stage_need;
  if (ext) {
    // caller-provided scratch: carve, never allocate
    const int64_t ws_bytes = (x.ws_peak + 1023) / 1024 * 1024;
    if (ws_bytes + stage_bytes > ext->bytes)
      return fail(h, SWMM_EINVAL,
                  "plan needs " + std::to_string(ws_bytes + stage_bytes) + " bytes of scratch, more than the " +
                      std::to_string(ext->bytes) + "-byte static scratch");
    r.ws = x.ws_peak > 0 ? ext->base : nullptr;
    r.stage = x.stage_need > 0 ? ext->base + ws_bytes : nullptr;
    r.ws_limit = ws_bytes;
    r.stage_limit = stage_bytes;
  } else {
    r.ws_limit = x.ws_peak;
    r.stage_limit = stage_bytes;
    if (x.ws_peak > 0 &&
        (injected_alloc_failure(h) || cudaMallocAsync((void **)&r.ws, x.ws_peak, stream) != cudaSuccess)) {
      cudaGetLastError();
      return fail(h, SWMM_ENOMEM, "workspace allocation failed");
    }
    if (x.stage_need > 0 &&
        (injected_alloc_failure(h) || cudaMallocAsync((void **)&r.stage, stage_bytes, stream) != cudaSuccess)) {
      cudaGetLastError();
      if (r.ws) cudaFreeAsync(r.ws, stream);
      return fail(h, SWMM_ENOMEM, "staging allocation failed");
    }
  }
  // host operands: the blocks go to the device in the order the table reads
  // them, and C's blocks come back as soon as they are final
  const Rect tok_in = rect_bytes(&h->io_token[0], 1), tok_out = rect_bytes(&h->io_token[1], 1);
  auto host_in = [&]() {
    if (!P.host_io) return;
    for (Loc l : first_use(h, P.sched)) {
      const int q = (l - A11) % 4, i = q / 2, j = q % 2;
      const View &dv = l <= A22 ? P.L : (l <= B22 ? P.R : P.D);
      const char *hp = l <= A22 ? P.hA : (l <= B22 ? P.hB : P.hC);
      const int64_t hld = l <= A22 ? P.hlda : (l <= B22 ? P.hldb : P.hldc);
      const View b = block_of(dv, i, j);
      const int64_t r0 = i ? dv.rows / 2 : 0, c0 = j ? dv.cols / 2 : 0;
      r.copy_in(b, hp + 4 * (r0 * hld + c0), hld, tok_in);
    }
  };
  auto host_out = [&]() {
    if (!P.host_io) return;
    for (int q = 0; q < 4; ++q) {
      const int i = q / 2, j = q % 2;
      const View b = block_of(P.D, i, j);
      canon_lazy(r, b);
      const int64_t r0 = i ? P.D.rows / 2 : 0, c0 = j ? P.D.cols / 2 : 0;
      r.copy_out(P.hC + 4 * (r0 * P.hldc + c0), P.hldc, b, tok_out);
    }
  };
  if (use_flow) {
    Flow flow(stream, h->flow_streams, h->flow_events);
    r.flow = &flow;
    host_in();
    execute(P, r);
    r.flush();
    host_out();
    flow.join();
    r.flow = nullptr;
    if (flow.error() != cudaSuccess && r.cuda_err == cudaSuccess) {
      r.cuda_err = flow.error();
      r.fail = std::string("dataflow ordering: ") + cudaGetErrorString(flow.error());
    }
  } else {
    host_in();
    execute(P, r);
    r.flush();
    host_out();
  }
  if (r.ok()) {
    // blocks of C whose last writer was a fused level's reduce-add hold
    // unreduced representatives: one canonicalising pass over each
    for (const View &v : lazy_in(r, P.D)) {
      ++r.ew_launches;
      cudaError_t e = launch_canon_modp(v, r.p, stream);
      if (e != cudaSuccess) {
        r.cuda_err = e;
        r.fail = std::string("canonical pass: ") + cudaGetErrorString(e);
        break;
      }
    }
  }
  if (!ext && r.ws) cudaFreeAsync(r.ws, stream);
  if (!ext && r.stage) cudaFreeAsync(r.stage, stream);
  st.workspace_bytes = std::max<int64_t>(st.workspace_bytes, x.ws_peak);
  st.plan_extra_elems = std::max<int64_t>(st.plan_extra_elems, x.tmp_peak_elems);
  st.paper_extra_elems = std::max<int64_t>(st.paper_extra_elems, P.paper);
  st.staging_bytes = std::max<int64_t>(st.staging_bytes, x.stage_need > 0 ? stage_bytes : 0);
  st.add_elems += r.add_elems;
  st.leaf_flops += r.leaf_flops;
  st.leaf_launches += r.leaf_launches;
  st.ew_launches += r.ew_launches;
  st.leaf_products += r.leaf_products;
  st.pack_bytes += r.pack_bytes;
  st.level_packs += r.level_packs;
  if (r.cuda_err != cudaSuccess) return fail(h, SWMM_ECUDA, r.fail);
  if (!r.fail.empty()) return fail(h, SWMM_EINVAL, r.fail);
  return SWMM_OK;
}

void key_append(std::string &k, const void *p, size_t n) { k.append((const char *)p, n); }

GraphEntry *find_graph(swmm_t h, const std::string &key) {
  for (auto &e : h->graphs)
    if (e->key == key) return e.get();
  return nullptr;
}

int launch_graph(swmm_t h, GraphEntry *g) {
  if (cudaEventRecord(h->ev_in, h->stream) != cudaSuccess || cudaStreamWaitEvent(h->cap, h->ev_in, 0) != cudaSuccess ||
      cudaGraphLaunch(g->exec, h->cap) != cudaSuccess || cudaEventRecord(h->ev_out, h->cap) != cudaSuccess ||
      cudaStreamWaitEvent(h->stream, h->ev_out, 0) != cudaSuccess) {
    cudaError_t e = cudaGetLastError();
    return fail(h, SWMM_ECUDA, std::string("graph launch failed: ") + cudaGetErrorString(e));
  }
  h->stats = g->stats;
  h->last_timer = &g->timer;
  return SWMM_OK;
}

// Run a list of plans, directly or through a cached CUDA graph under `key`
// (callers look the key up before planning, so a replay skips planning).
int run_plans(swmm_t h, const std::vector<Plan> &plans, uint32_t flags, const Scratch *ext,
              const std::string &key = std::string(), GraphEntry **entry = nullptr) {
  const bool timing = (flags & SWMM_FLAG_TIMING) != 0 && !ext;
  swmm_stats st;
  std::memset(&st, 0, sizeof(st));
  if (!(flags & SWMM_FLAG_GRAPH) || ext) {
    h->last_timer = &h->timer;
    if (ext) h->timer.used = 0;  // static-scratch calls record no leaf timing
    for (const Plan &P : plans) {
      int rc = enqueue(h, P, h->stream, timing ? &h->timer : nullptr, ext, st);
      if (rc != SWMM_OK) return rc;
    }
    h->stats = st;
    return SWMM_OK;
  }
  GraphEntry *g = find_graph(h, key);
  if (!g) {
    if (!h->cap) {
      if (cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return fail(h, SWMM_ECUDA, "graph stream creation failed");
      }
    }
    const bool use_flow = !(flags & SWMM_FLAG_SERIAL);
    if (use_flow) {
      // side streams and enough events for the largest plan, made before
      // the capture starts
      size_t need = 2;
      for (const Plan &P : plans)
        need = std::max<size_t>(need, (size_t)(8 * P.x.leaf_launches + 2 * P.x.leaf_products +
                                               2 * P.x.ew_launches + 48));
      for (cudaStream_t &s : h->flow_streams)
        if (!s && cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
          cudaGetLastError();
          return fail(h, SWMM_ECUDA, "flow stream creation failed");
        }
      while (h->flow_events.size() < need) {
        cudaEvent_t e;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
          cudaGetLastError();
          return fail(h, SWMM_ECUDA, "flow event creation failed");
        }
        h->flow_events.push_back(e);
      }
    }
    std::unique_ptr<GraphEntry> ne(new GraphEntry());
    ne->key = key;
    if (cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      return fail(h, SWMM_ECUDA, "stream capture failed to start");
    }
    int rc = SWMM_OK;
    for (const Plan &P : plans) {
      rc = enqueue(h, P, h->cap, timing ? &ne->timer : nullptr, nullptr, ne->stats, use_flow);
      if (rc != SWMM_OK) break;
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->cap, &graph);
    if (rc != SWMM_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (e != cudaSuccess || cudaGraphInstantiate(&ne->exec, graph, 0) != cudaSuccess) {
      cudaGetLastError();
      if (graph) cudaGraphDestroy(graph);
      return fail(h, SWMM_ECUDA, "graph capture or instantiation failed");
    }
    cudaGraphDestroy(graph);
    if (h->graphs.size() >= 32) h->graphs.erase(h->graphs.begin());
    g = ne.get();
    h->graphs.push_back(std::move(ne));
  }
  if (entry) *entry = g;
  return launch_graph(h, g);
}

// Graph-cache key of a call from its raw arguments (everything baked into
// the captured kernels: sizes, pointers, leading dimensions, options, scalar
// values).
std::string call_key(const Req &q, const swmm_opts *o) {
  std::string k;
  key_append(k, &q.entry, sizeof(q.entry));
  int64_t dims[6] = {q.m, q.k, q.n, q.lda, q.ldb, q.ldc};
  key_append(k, dims, sizeof(dims));
  const void *ptrs[3] = {q.A, q.B, q.C};
  key_append(k, ptrs, sizeof(ptrs));
  key_append(k, o, sizeof(*o));
  uint32_t sc[3] = {q.alpha ? *(const uint32_t *)q.alpha : 0u, q.beta ? *(const uint32_t *)q.beta : 0u,
                    (uint32_t)(q.alpha != nullptr) | ((uint32_t)(q.beta != nullptr) << 1)};
  key_append(k, sc, sizeof(sc));
  return k;
}

int run(swmm_t h, const Req &q, const swmm_opts *o, const Scratch *ext = nullptr) {
  if (!h) return SWMM_EINVAL;
  h->last_error.clear();
  if (!o) return fail(h, SWMM_EINVAL, "opts is NULL");
  std::string key;
  if ((o->flags & SWMM_FLAG_GRAPH) && !ext) {
    key = call_key(q, o);
    if (GraphEntry *g = find_graph(h, key)) return launch_graph(h, g);
  }
  std::vector<Plan> plans(1);
  int rc = make_plan(h, q, o, true, plans[0], ext == nullptr);
  if (rc != SWMM_OK) return rc;
  return run_plans(h, plans, o->flags, ext, key);
}

// Classical problems with the same arithmetic (mode, modulus, scalars)
// become plans with grouped leaf launches of up to kMaxProducts products
// (operand staging of a group capped at 2 GiB), grouped by decreasing inner
// dimension; the problems are independent, so any order gives the same
// results.
std::vector<Plan> group_classical(std::vector<Plan> &each) {
  constexpr int64_t kGroupStageBytes = 2ll << 30;
  auto groupable = [](const Plan &P) {
    return P.sched == SWMM_CLASSICAL && P.ne && P.q.k > 0 && !P.x.simt && P.jobs.empty();
  };
  auto same = [](const Plan &a, const Plan &b) {
    return a.x.mode == b.x.mode && a.x.p == b.x.p && a.accum == b.accum && a.alpha.u == b.alpha.u &&
           a.beta.u == b.beta.u && a.alpha.f == b.alpha.f && a.beta.f == b.beta.f;
  };
  std::vector<Plan> out;
  out.reserve(each.size());
  std::vector<std::vector<size_t>> kinds;  // indices of groupable plans per arithmetic
  for (size_t i = 0; i < each.size(); ++i) {
    if (!groupable(each[i])) {
      out.push_back(std::move(each[i]));
      continue;
    }
    size_t c = 0;
    while (c < kinds.size() && !same(each[kinds[c][0]], each[i])) ++c;
    if (c == kinds.size()) kinds.emplace_back();
    kinds[c].push_back(i);
  }
  for (std::vector<size_t> &idx : kinds) {
    // problems of similar inner dimension share a launch (similar tile times)
    std::stable_sort(idx.begin(), idx.end(), [&](size_t x, size_t y) { return each[x].q.k > each[y].q.k; });
    for (size_t a = 0; a < idx.size();) {
      size_t b = a + 1;
      int64_t bytes = each[idx[a]].x.stage_need;
      while (b < idx.size() && b - a < (size_t)kMaxProducts && bytes + each[idx[b]].x.stage_need <= kGroupStageBytes)
        bytes += each[idx[b++]].x.stage_need;
      Plan G = each[idx[a]];
      if (b - a > 1) {
        for (size_t t = a; t < b; ++t) G.jobs.push_back(LeafJob{each[idx[t]].L, each[idx[t]].R, each[idx[t]].D});
        // longest inner dimension first: the persistent launch deals tiles
        // out in order, so the tiles that take longest start first
        std::stable_sort(G.jobs.begin(), G.jobs.end(),
                         [](const LeafJob &x, const LeafJob &y) { return x.L.cols > y.L.cols; });
        // plan the group: sizes and counts of the grouped launch
        Exec &x = G.x;
        reset_counts(x);
        x.merge = false;
        x.stage_slots = 1;
        x.dry = true;
        x.ws = kPlanWorkspace;
        execute(G, x);
        x.flush();
        x.ws = nullptr;
      }
      out.push_back(std::move(G));
      a = b;
    }
  }
  return out;
}

// ---------------------------------------------------------------- autotuner
// Cost model of a planned call on one GB300 (microseconds): tensor work at a
// rate that falls with small leaf products, HBM-bound passes, and a fixed
// cost per launch.  Additions and per-level packs move about 5.5 TB/s; the
// one-pass level packs, whose stores are three quarters of their bytes,
// about 4.2 TB/s (measured: 8.7 GB in 1.99 ms at 16384^2 depth 2, 0.55 GB
// in 0.134 ms per level-2 table at 8192^2 depth 3).
double model_us(const Plan &P) {
  const Exec &x = P.x;
  const double limbs = x.mode == MODE_MODP1 ? 1.0 : (x.mode == MODE_MODP2 ? 4.0 : 3.0);
  const double flops = (double)x.leaf_flops * limbs;
  const double per_product = x.leaf_products ? (double)x.leaf_flops / (double)x.leaf_products : 0.0;
  const double tiles = per_product / (2.0 * 128.0 * 128.0 * 1024.0);  // 128 x 128 x 1024 tile units
  const double eff = 0.95 * tiles / (tiles + 6.0) + 0.05;
  // limb flop/us at the sustained tensor peak: 1.75e9 for the mod-p limbs,
  // 1.45e9 for FP32 mode's hi/lo products (16384^3 classical: 1737 against
  // 1443 TFLOP/s measured, the latter with its amax passes)
  const double rate = (x.mode == MODE_FP32 ? 1.45e9 : 1.75e9) * eff;
  const double bytes = (double)x.add_elems * 12.0 + (double)(x.pack_bytes - x.level_pack_bytes);
  const double launches = (double)(x.leaf_launches + x.ew_launches);
  return flops / rate + bytes / 5.5e6 + (double)x.level_pack_bytes / 4.2e6 + launches * 2.5;
}

// A call without operands, for planning only: placeholder addresses, never
// dereferenced, disjoint from each other and from the planning pass's
// temporaries, so the plan sees the same overlaps as a call with real
// operands (packed leading dimensions).
Req placeholder_req(int entry, int64_t m, int64_t k, int64_t n, const void *alpha, const void *beta) {
  const void *fa = reinterpret_cast<const void *>(uintptr_t(1) << 44);
  const void *fb = reinterpret_cast<const void *>(uintptr_t(2) << 44);
  void *fc = reinterpret_cast<void *>(uintptr_t(3) << 44);
  return Req{entry, m, k, n, fa, fb, fc, std::max<int64_t>(k, 1), std::max<int64_t>(n, 1), std::max<int64_t>(n, 1),
             alpha, beta};
}

// The counts of a planned call, as an eager run would report them (no
// final canonical pass; the staging of an eager call).
void plan_counts(const Plan &P, swmm_stats *out) {
  const Exec &x = P.x;
  std::memset(out, 0, sizeof(*out));
  out->workspace_bytes = x.ws_peak;
  out->plan_extra_elems = x.tmp_peak_elems;
  out->paper_extra_elems = P.paper;
  out->add_elems = x.add_elems;
  out->leaf_flops = x.leaf_flops;
  out->leaf_launches = x.leaf_launches;
  out->ew_launches = x.ew_launches;
  out->leaf_products = x.leaf_products;
  out->staging_bytes = x.stage_need > 0 ? stage_slots_for(x, x.merge, false) * ((x.stage_need + 1023) / 1024 * 1024) : 0;
  out->pack_bytes = x.pack_bytes;
  out->level_packs = x.level_packs;
}

// The dry run of a call with no operands: the entry point the schedule's
// contract implies, unit scalars.
int plan_only(swmm_t h, int64_t m, int64_t k, int64_t n, const swmm_opts *opts, Plan &P) {
  if (!opts) return fail(h, SWMM_EINVAL, "opts is NULL");
  const int s = opts->sched;
  bool acc_inplace = s == SWMM_T6_ACLR || s == SWMM_T7_ACCR || s == SWMM_T8_ACR;
  int entry = 0;
  if (s == SWMM_T2_HLJJTT || s == SWMM_T9_ACC || s == SWMM_TBLOCK) entry = 1;
  if (s == SWMM_T3_IP || s == SWMM_T4_OVL || s == SWMM_T4M_OVL || s == SWMM_T5_OVR || s == SWMM_IP0VMM ||
      acc_inplace)
    entry = 2;
  if (s == SWMM_CUSTOM && h->has_custom) {
    const bool ro = h->custom.preserve == 0xffu;
    entry = ro ? (h->custom.accumulate ? 1 : 0) : 2;
    acc_inplace = !ro && h->custom.accumulate;
  }
  static const uint32_t one = 1;
  static const float onef = 1.f;
  const void *u = opts->mode == SWMM_FP32 ? (const void *)&onef : (const void *)&one;
  return make_plan(h, placeholder_req(entry, m, k, n, u, acc_inplace || entry == 1 ? u : nullptr), opts, false, P);
}

// The handle's own schedule: checked in the pebble game, lowered to rows.
int set_schedule(swmm_t h, const swmm_search_spec *spec, const swmm_search_row *rows, int32_t nrows) {
  if (!spec || !rows) return fail(h, SWMM_EINVAL, "spec or rows is NULL");
  CustomSchedule cs;
  std::string err;
  if (!lower_schedule(*spec, rows, nrows, &cs, &err)) return fail(h, SWMM_EINVAL, "schedule rejected: " + err);
  if (!h->graphs.empty()) {
    // captured calls hold the previous schedule: let them finish, drop them
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e == cudaSuccess && h->cap) e = cudaStreamSynchronize(h->cap);
    if (e != cudaSuccess) return fail(h, SWMM_ECUDA, cudaGetErrorString(e));
    h->graphs.clear();
  }
  h->custom = std::move(cs);
  h->custom_info = KindInfo{"custom", &h->custom.rows, h->custom.accumulate, true};
  h->has_custom = true;
  return SWMM_OK;
}

}  // namespace

namespace swmm {
int handle_device(swmm_t h) { return h ? h->device : -1; }

int muladd_with_scratch(swmm_t h, int64_t m, int64_t k, int64_t n, const void *alpha, const void *A, int64_t lda,
                        const void *B, int64_t ldb, const void *beta, void *C, int64_t ldc, const swmm_opts *opts,
                        void *scratch, int64_t scratch_bytes) {
  if (!alpha || !beta) return fail(h, SWMM_EINVAL, "alpha and beta are required");
  Req q{1, m, k, n, A, B, C, lda, ldb, ldc, alpha, beta};
  Scratch s{(char *)scratch, scratch_bytes};
  return run(h, q, opts, &s);
}
}  // namespace swmm

extern "C" {

int swmm_create(swmm_t *out, int device, void *stream) {
  if (!out) return SWMM_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return SWMM_ECUDA;
  }
  swmm_t h = new swmm_ctx();
  h->device = device;
  h->stream = (cudaStream_t)stream;
  if (cudaSetDevice(device) != cudaSuccess ||
      cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaMalloc((void **)&h->d_err, sizeof(int)) != cudaSuccess ||
      cudaMemset(h->d_err, 0, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return SWMM_ECUDA;
  }
  std::memset(&h->stats, 0, sizeof(h->stats));
  *out = h;
  return SWMM_OK;
}

int swmm_destroy(swmm_t h) {
  if (!h) return SWMM_EINVAL;
  if (h->d_err) cudaFree(h->d_err);
  delete h;
  return SWMM_OK;
}

int swmm_set_stream(swmm_t h, void *stream) {
  if (!h) return SWMM_EINVAL;
  h->stream = (cudaStream_t)stream;
  return SWMM_OK;
}

int swmm_mul(swmm_t h, int64_t m, int64_t k, int64_t n, const void *A, int64_t lda, const void *B, int64_t ldb,
             void *C, int64_t ldc, const swmm_opts *opts) {
  Req q{0, m, k, n, A, B, C, lda, ldb, ldc, nullptr, nullptr};
  return run(h, q, opts);
}

int swmm_muladd(swmm_t h, int64_t m, int64_t k, int64_t n, const void *alpha, const void *A, int64_t lda,
                const void *B, int64_t ldb, const void *beta, void *C, int64_t ldc, const swmm_opts *opts) {
  if (!alpha || !beta) return fail(h, SWMM_EINVAL, "alpha and beta are required");
  Req q{1, m, k, n, A, B, C, lda, ldb, ldc, alpha, beta};
  return run(h, q, opts);
}

int swmm_muladd_host(swmm_t h, int64_t m, int64_t k, int64_t n, const void *alpha, const void *A, int64_t lda,
                     const void *B, int64_t ldb, const void *beta, void *C, int64_t ldc, const swmm_opts *opts) {
  if (!h) return SWMM_EINVAL;
  h->last_error.clear();
  if (!alpha || !beta) return fail(h, SWMM_EINVAL, "alpha and beta are required");
  if (!opts) return fail(h, SWMM_EINVAL, "opts is NULL");
  if (m < 0 || k < 0 || n < 0) return fail(h, SWMM_EINVAL, "negative dimension");
  if (m > (1 << 30) || k > (1 << 30) || n > (1 << 30)) return fail(h, SWMM_EINVAL, "dimension too large");
  if (m == 0 || n == 0) return SWMM_OK;
  if (!C || (k > 0 && (!A || !B))) return fail(h, SWMM_EINVAL, "NULL pointer");
  if (lda < std::max<int64_t>(k, 1) || ldb < std::max<int64_t>(n, 1) || ldc < std::max<int64_t>(n, 1))
    return fail(h, SWMM_EINVAL, "leading dimension smaller than the number of columns");
  // device copies: leading dimensions rounded to 16 bytes, blocks 256-byte aligned
  const int64_t dla = (k + 3) / 4 * 4, dlb = (n + 3) / 4 * 4, dlc = dlb;
  auto r256 = [](int64_t b) { return (b + 255) / 256 * 256; };
  const int64_t bA = r256(4 * m * dla), bB = r256(4 * k * dlb), bC = r256(4 * m * dlc);
  const size_t need = (size_t)(bA + bB + bC);
  if (need > h->io_bytes) {
    // the cached graphs refer to the old copies: drop them
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e == cudaSuccess && h->cap) e = cudaStreamSynchronize(h->cap);
    if (e != cudaSuccess) return fail(h, SWMM_ECUDA, cudaGetErrorString(e));
    h->graphs.clear();
    if (h->io_buf) cudaFree(h->io_buf);
    h->io_buf = nullptr;
    h->io_bytes = 0;
    if (injected_alloc_failure(h) || cudaMalloc((void **)&h->io_buf, need) != cudaSuccess) {
      cudaGetLastError();
      h->io_buf = nullptr;
      return fail(h, SWMM_ENOMEM, "device copies of the operands");
    }
    h->io_bytes = need;
  }
  char *dA = h->io_buf, *dB = h->io_buf + bA, *dC = h->io_buf + bA + bB;
  Req q{1, m, k, n, dA, dB, dC, dla, dlb, dlc, alpha, beta};
  std::string key;
  if (opts->flags & SWMM_FLAG_GRAPH) {
    key = call_key(q, opts);
    key.append("host");
    const void *hp[4] = {A, B, C, h->io_buf};
    key_append(key, hp, sizeof(hp));
    const int64_t hl[3] = {lda, ldb, ldc};
    key_append(key, hl, sizeof(hl));
    if (GraphEntry *g = find_graph(h, key)) return launch_graph(h, g);
  }
  std::vector<Plan> plans(1);
  int rc = make_plan(h, q, opts, true, plans[0]);
  if (rc != SWMM_OK) return rc;
  Plan &P = plans[0];
  P.host_io = true;
  P.hA = static_cast<const char *>(A);
  P.hB = static_cast<const char *>(B);
  P.hC = static_cast<char *>(C);
  P.hlda = lda;
  P.hldb = ldb;
  P.hldc = ldc;
  return run_plans(h, plans, opts->flags, nullptr, key);
}

int swmm_mul_inplace(swmm_t h, int64_t m, int64_t k, int64_t n, void *A, int64_t lda, void *B, int64_t ldb, void *C,
                     int64_t ldc, const void *alpha, const void *beta, const swmm_opts *opts) {
  Req q{2, m, k, n, A, B, C, lda, ldb, ldc, alpha, beta};
  return run(h, q, opts);
}

int swmm_workspace_elems(swmm_t h, int64_t m, int64_t k, int64_t n, const swmm_opts *opts, int64_t *paper_out,
                         int64_t *plan_out) {
  swmm_ctx planner;  // planning needs no device: a NULL handle is accepted
  if (!h) h = &planner;
  h->last_error.clear();
  Plan P;
  const int rc = plan_only(h, m, k, n, opts, P);
  if (rc != SWMM_OK) return rc;
  if (paper_out) *paper_out = P.paper;
  if (plan_out) *plan_out = P.x.tmp_peak_elems;
  return SWMM_OK;
}

int swmm_plan_stats(swmm_t h, int64_t m, int64_t k, int64_t n, const swmm_opts *opts, swmm_stats *out) {
  swmm_ctx planner;  // planning needs no device: a NULL handle is accepted
  if (!h) h = &planner;
  h->last_error.clear();
  if (!out) return fail(h, SWMM_EINVAL, "out is NULL");
  Plan P;
  const int rc = plan_only(h, m, k, n, opts, P);
  if (rc != SWMM_OK) return rc;
  plan_counts(P, out);
  return SWMM_OK;
}

int swmm_schedule_stats(const swmm_search_spec *spec, const swmm_search_row *rows, int32_t nrows, int64_t m,
                        int64_t k, int64_t n, const swmm_opts *opts, swmm_stats *out) {
  swmm_ctx planner;  // no device
  int rc = set_schedule(&planner, spec, rows, nrows);
  if (rc != SWMM_OK) return rc;
  if (!opts || opts->sched != SWMM_CUSTOM || !out) return SWMM_EINVAL;
  Plan P;
  rc = plan_only(&planner, m, k, n, opts, P);
  if (rc != SWMM_OK) return rc;
  plan_counts(P, out);
  return SWMM_OK;
}


int swmm_autotune(swmm_t h, int64_t m, int64_t k, int64_t n, int32_t mode, uint32_t p, int32_t *sched,
                  int32_t *depth, double *est_us, int64_t *extra_elems) {
  swmm_ctx planner;
  if (!h) h = &planner;
  h->last_error.clear();
  const std::array<int64_t, 5> tk{m, k, n, mode, mode == SWMM_FP32 ? 0 : (int64_t)p};
  for (auto &e : h->tuned) {
    if (e.first == tk) {
      if (sched) *sched = std::get<0>(e.second);
      if (depth) *depth = std::get<1>(e.second);
      if (est_us) *est_us = std::get<2>(e.second);
      if (extra_elems) *extra_elems = std::get<3>(e.second);
      return SWMM_OK;
    }
  }
  static const uint32_t one = 1;
  static const float onef = 1.f;
  const void *sc = mode == SWMM_FP32 ? (const void *)&onef : (const void *)&one;
  double best = 1e300;
  int bs = SWMM_CLASSICAL, bd = 0;
  int64_t be = 0;
  const int cands[3] = {SWMM_CLASSICAL, SWMM_T2_HLJJTT, SWMM_T9_ACC};
  for (int c : cands) {
    for (int d = (c == SWMM_CLASSICAL ? 0 : 1); d <= (c == SWMM_CLASSICAL ? 0 : 3); ++d) {
      if (c == SWMM_T9_ACC && !(m == k && k == n)) continue;
      swmm_opts o;
      std::memset(&o, 0, sizeof(o));
      o.mode = mode;
      o.p = p;
      o.sched = c;
      o.depth = d;
      Plan P;
      if (make_plan(h, placeholder_req(1, m, k, n, sc, sc), &o, false, P) != SWMM_OK) continue;
      const double t = model_us(P);
      if (t < best) {
        best = t;
        bs = c;
        bd = d;
        be = P.x.tmp_peak_elems;
      }
    }
  }
  if (best >= 1e300) return fail(h, SWMM_EINVAL, "no valid plan");
  if (h != &planner && h->tuned.size() < 4096) h->tuned.push_back({tk, std::make_tuple(bs, bd, best, be)});
  if (sched) *sched = bs;
  if (depth) *depth = bd;
  if (est_us) *est_us = best;
  if (extra_elems) *extra_elems = be;
  h->last_error.clear();
  return SWMM_OK;
}

// SWMM_FLAG_TUNE: problems below this size (2 m k n) take the model's choice;
// a Winograd level cannot pay for its packs there (measured: Table 2 depth 1
// against the classical product, 1.00x at 4096^3 over Z/65521).
constexpr double kTuneMinFlops = 2.0 * 3072.0 * 3072.0 * 3072.0;

// The measured choice for one batched problem (SWMM_FLAG_TUNE): the classical
// product and one Winograd level (Table 2, or Table 9 for square problems),
// each run on a scratch copy of C on the handle's stream, once to warm up and
// twice timed with events; the faster wins and is kept per shape and mode.
int measure_pick(swmm_t h, const swmm_problem &pb, int32_t *s, int32_t *d) {
  const std::array<int64_t, 5> key{pb.m, pb.k, pb.n, pb.mode, pb.mode == SWMM_FP32 ? 0 : (int64_t)pb.p};
  for (auto &e : h->measured)
    if (e.first == key) {
      *s = e.second.first;
      *d = e.second.second;
      return SWMM_OK;
    }
  char *scr = nullptr;
  const int64_t bytes = 4 * pb.m * pb.n;
  if (injected_alloc_failure(h) || cudaMallocAsync((void **)&scr, bytes, h->stream) != cudaSuccess) {
    cudaGetLastError();
    return fail(h, SWMM_ENOMEM, "tuning scratch");
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = SWMM_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = SWMM_ECUDA;
  const void *al = pb.mode == SWMM_FP32 ? (const void *)&pb.alpha_f : (const void *)&pb.alpha_u;
  const void *be = pb.mode == SWMM_FP32 ? (const void *)&pb.beta_f : (const void *)&pb.beta_u;
  const int cands[3][2] = {{SWMM_CLASSICAL, 0}, {SWMM_T2_HLJJTT, 1}, {SWMM_T9_ACC, 1}};
  const bool square = pb.m == pb.k && pb.k == pb.n;
  float best = 1e30f;
  int bs = SWMM_CLASSICAL, bd = 0;
  for (int c = 0; c < 3 && rc == SWMM_OK; ++c) {
    if (cands[c][0] == SWMM_T9_ACC && !square) continue;
    if (cands[c][0] == SWMM_T2_HLJJTT && square) continue;  // Table 9 takes the square ones
    swmm_opts o;
    std::memset(&o, 0, sizeof(o));
    o.mode = pb.mode;
    o.p = pb.p;
    o.sched = cands[c][0];
    o.depth = cands[c][1];
    Req q{1, pb.m, pb.k, pb.n, pb.A, pb.B, scr, pb.lda, pb.ldb, pb.n, al, be};
    if (cudaMemcpy2DAsync(scr, 4 * pb.n, pb.C, 4 * pb.ldc, 4 * pb.n, pb.m, cudaMemcpyDeviceToDevice, h->stream) !=
        cudaSuccess) {
      rc = SWMM_ECUDA;
      break;
    }
    rc = run(h, q, &o);
    if (rc != SWMM_OK) break;
    if (cudaEventRecord(e0, h->stream) != cudaSuccess) rc = SWMM_ECUDA;
    for (int r = 0; r < 2 && rc == SWMM_OK; ++r) rc = run(h, q, &o);
    if (rc != SWMM_OK) break;
    float ms = 0.f;
    if (cudaEventRecord(e1, h->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      rc = SWMM_ECUDA;
      break;
    }
    if (ms < best) {
      best = ms;
      bs = cands[c][0];
      bd = cands[c][1];
    }
  }
  cudaFreeAsync(scr, h->stream);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (rc == SWMM_ECUDA) {
    cudaError_t e = cudaGetLastError();
    return fail(h, SWMM_ECUDA, std::string("tuning run: ") + cudaGetErrorString(e));
  }
  if (rc != SWMM_OK) return rc;
  if (h->measured.size() < 4096) h->measured.push_back({key, {bs, bd}});
  *s = bs;
  *d = bd;
  return SWMM_OK;
}

int swmm_muladd_batched(swmm_t h, int count, swmm_problem *probs, uint32_t flags) {
  if (!h) return SWMM_EINVAL;
  h->last_error.clear();
  if (count < 0 || (count > 0 && !probs)) return fail(h, SWMM_EINVAL, "bad problem list");
  std::string key;
  if (flags & SWMM_FLAG_GRAPH) {
    key.assign("batch");
    key_append(key, &flags, sizeof(flags));
    for (int i = 0; i < count; ++i) key_append(key, &probs[i], offsetof(swmm_problem, chosen_sched));
    if (GraphEntry *g = find_graph(h, key)) {
      for (int i = 0; i < count && 2 * i + 1 < (int)g->chosen.size(); ++i) {
        probs[i].chosen_sched = g->chosen[2 * i];
        probs[i].chosen_depth = g->chosen[2 * i + 1];
      }
      return launch_graph(h, g);
    }
  }
  std::vector<Plan> each(count);
  for (int i = 0; i < count; ++i) {
    swmm_problem &pb = probs[i];
    int32_t s = pb.sched, d = pb.depth;
    if (s == SWMM_AUTO) {
      // a malformed problem keeps the model's choice and fails in make_plan below
      const bool sane = pb.A && pb.B && pb.C && pb.m > 0 && pb.k > 0 && pb.n > 0 && pb.lda >= pb.k &&
                        pb.ldb >= pb.n && pb.ldc >= pb.n;
      const bool big = sane && 2.0 * (double)pb.m * (double)pb.k * (double)pb.n >= kTuneMinFlops;
      int rc = (flags & SWMM_FLAG_TUNE) && big ? measure_pick(h, pb, &s, &d)
                                              : swmm_autotune(h, pb.m, pb.k, pb.n, pb.mode, pb.p, &s, &d, nullptr,
                                                              nullptr);
      if (rc != SWMM_OK) return rc;
    }
    pb.chosen_sched = s;
    pb.chosen_depth = d;
    swmm_opts o;
    std::memset(&o, 0, sizeof(o));
    o.mode = pb.mode;
    o.p = pb.p;
    o.sched = s;
    o.depth = d;
    o.flags = flags & (SWMM_FLAG_UNFUSED | SWMM_FLAG_SIMT_LEAF);
    const void *al = pb.mode == SWMM_FP32 ? (const void *)&pb.alpha_f : (const void *)&pb.alpha_u;
    const void *be = pb.mode == SWMM_FP32 ? (const void *)&pb.beta_f : (const void *)&pb.beta_u;
    Req q{1, pb.m, pb.k, pb.n, pb.A, pb.B, pb.C, pb.lda, pb.ldb, pb.ldc, al, be};
    int rc = make_plan(h, q, &o, true, each[i]);
    if (rc != SWMM_OK) return fail(h, rc, "problem " + std::to_string(i) + ": " + h->last_error);
  }
  const std::vector<Plan> plans = group_classical(each);
  GraphEntry *g = nullptr;
  int rc = run_plans(h, plans, flags, nullptr, key, &g);
  if (rc == SWMM_OK && g) {
    g->chosen.clear();
    for (int i = 0; i < count; ++i) {
      g->chosen.push_back(probs[i].chosen_sched);
      g->chosen.push_back(probs[i].chosen_depth);
    }
  }
  return rc;
}

int swmm_leaf_timing(swmm_t h, int reset, double *gemm_ms, int64_t *launches, double *tensor_flops) {
  if (!h) return SWMM_EINVAL;
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return fail(h, SWMM_ECUDA, cudaGetErrorString(e));
  EventTimer &t = *h->last_timer;
  double ms = 0.0, fl = 0.0;
  for (size_t i = 0; i < t.used; ++i) {
    float v = 0.f;
    if (cudaEventElapsedTime(&v, t.ev[2 * i], t.ev[2 * i + 1]) != cudaSuccess)
      return fail(h, SWMM_ECUDA, "event timing failed");
    ms += v;
    fl += t.flops[i];
  }
  if (gemm_ms) *gemm_ms = ms;
  if (launches) *launches = (int64_t)t.used;
  if (tensor_flops) *tensor_flops = fl;
  if (reset && h->last_timer == &h->timer) h->timer.used = 0;
  return SWMM_OK;
}

int swmm_matvec(swmm_t h, int64_t rows, int64_t cols, const void *M, int64_t ldm, const void *x, void *y,
                const swmm_opts *opts) {
  if (!h) return SWMM_EINVAL;
  if (!opts) return fail(h, SWMM_EINVAL, "opts is NULL");
  const bool modp = opts->mode == SWMM_MODP;
  if (!modp && opts->mode != SWMM_FP32) return fail(h, SWMM_EINVAL, "unknown mode");
  if (modp && (opts->p <= 2 || opts->p >= 65536)) return fail(h, SWMM_EINVAL, "p must satisfy 2 < p < 65536");
  if (rows < 0 || cols < 0) return fail(h, SWMM_EINVAL, "negative dimension");
  if (rows > (1 << 30) || cols > (1 << 30)) return fail(h, SWMM_EINVAL, "dimension too large");
  if (rows == 0) return SWMM_OK;
  if (!y || (cols > 0 && (!M || !x))) return fail(h, SWMM_EINVAL, "NULL pointer");
  if (ldm < cols || ldm < 1) return fail(h, SWMM_EINVAL, "leading dimension smaller than the number of columns");
  const uintptr_t xa = modp ? 3 : 7;
  if (((uintptr_t)M & 3) || ((uintptr_t)x & xa) || ((uintptr_t)y & xa))
    return fail(h, SWMM_EINVAL, "misaligned pointer");
  cudaError_t e = launch_matvec(M, rows, cols, ldm, x, y, opts->p, modp, h->num_sms, h->stream);
  if (e != cudaSuccess) return fail(h, SWMM_ECUDA, cudaGetErrorString(e));
  return SWMM_OK;
}

int swmm_residual(swmm_t h, int64_t m, int64_t k, int64_t n, const void *alpha, const void *A, int64_t lda,
                  const void *B, int64_t ldb, const void *beta, const void *y0, const void *C, int64_t ldc,
                  const void *x, void *r, const swmm_opts *opts) {
  if (!h) return SWMM_EINVAL;
  if (!opts) return fail(h, SWMM_EINVAL, "opts is NULL");
  if (!alpha || !beta) return fail(h, SWMM_EINVAL, "alpha and beta are required");
  const bool modp = opts->mode == SWMM_MODP;
  if (!modp && opts->mode != SWMM_FP32) return fail(h, SWMM_EINVAL, "unknown mode");
  if (modp && (opts->p <= 2 || opts->p >= 65536)) return fail(h, SWMM_EINVAL, "p must satisfy 2 < p < 65536");
  if (m < 0 || k < 0 || n < 0) return fail(h, SWMM_EINVAL, "negative dimension");
  if (m == 0) return SWMM_OK;
  if (!r || !C || (n > 0 && !x) || (k > 0 && (!A || !B))) return fail(h, SWMM_EINVAL, "NULL pointer");
  uint32_t au = 0, bu = 0;
  double af = 0.0, bf = 0.0;
  bool with_beta;
  if (modp) {
    au = *static_cast<const uint32_t *>(alpha) % opts->p;
    bu = *static_cast<const uint32_t *>(beta) % opts->p;
    with_beta = bu != 0;
  } else {
    af = *static_cast<const float *>(alpha);
    bf = *static_cast<const float *>(beta);
    with_beta = bf != 0.0;
  }
  if (with_beta && !y0) return fail(h, SWMM_EINVAL, "y0 = C_in x is required when beta != 0");
  const uintptr_t va = modp ? 3 : 7;
  if (((uintptr_t)r & va) || ((uintptr_t)y0 & va) || ((uintptr_t)x & va))
    return fail(h, SWMM_EINVAL, "misaligned pointer");
  const size_t es = modp ? 4 : 8;
  char *tmp = nullptr;
  const size_t bytes = (size_t)(k + 2 * m) * es;
  cudaError_t e = injected_alloc_failure(h) ? cudaErrorMemoryAllocation
                                             : cudaMallocAsync((void **)&tmp, bytes, h->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(h, SWMM_ENOMEM, "probe temporaries");
  }
  void *t = tmp, *u = tmp + k * es, *v = tmp + (k + m) * es;
  int rc = SWMM_OK;
  // t = B x, u = A t, v = C x, r = v - alpha u - beta y0
  if (k > 0) rc = swmm_matvec(h, k, n, B, ldb, x, t, opts);
  if (rc == SWMM_OK) rc = swmm_matvec(h, m, k, A, k > 0 ? lda : 1, t, u, opts);
  if (rc == SWMM_OK) rc = swmm_matvec(h, m, n, C, n > 0 ? ldc : 1, x, v, opts);
  if (rc == SWMM_OK) {
    e = launch_residual(m, v, u, with_beta ? y0 : nullptr, r, au, bu, af, bf, opts->p, modp, h->num_sms, h->stream);
    if (e != cudaSuccess) rc = fail(h, SWMM_ECUDA, cudaGetErrorString(e));
  }
  cudaFreeAsync(tmp, h->stream);
  return rc;
}

int swmm_get_stats(swmm_t h, swmm_stats *out) {
  if (!h || !out) return SWMM_EINVAL;
  *out = h->stats;
  return SWMM_OK;
}

int swmm_sync(swmm_t h) {
  if (!h) return SWMM_EINVAL;
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return fail(h, SWMM_ECUDA, cudaGetErrorString(e));
  int v = 0;
  if (cudaMemcpy(&v, h->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(h, SWMM_ECUDA, "reading the error word failed");
  if (v) {
    cudaMemset(h->d_err, 0, sizeof(int));
    return fail(h, SWMM_ETIMEOUT, "a kernel's bounded wait expired");
  }
  return SWMM_OK;
}

int swmm_memory_use(swmm_t h, int reset, int64_t *out) {
  if (!h || !out) return SWMM_EINVAL;
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess && h->cap) e = cudaStreamSynchronize(h->cap);
  cudaMemPool_t pool = nullptr;
  if (e == cudaSuccess) e = cudaDeviceGetDefaultMemPool(&pool, h->device);
  cuuint64_t v[4] = {0, 0, 0, 0};
  if (e == cudaSuccess) e = cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &v[0]);
  if (e == cudaSuccess) e = cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &v[1]);
  if (e == cudaSuccess) e = cudaDeviceGetGraphMemAttribute(h->device, cudaGraphMemAttrUsedMemCurrent, &v[2]);
  if (e == cudaSuccess) e = cudaDeviceGetGraphMemAttribute(h->device, cudaGraphMemAttrUsedMemHigh, &v[3]);
  if (e == cudaSuccess && reset) {
    cuuint64_t zero = 0;
    e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &zero);
    if (e == cudaSuccess) e = cudaDeviceSetGraphMemAttribute(h->device, cudaGraphMemAttrUsedMemHigh, &zero);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(h, SWMM_ECUDA, std::string("memory pool query: ") + cudaGetErrorString(e));
  }
  for (int i = 0; i < 4; ++i) out[i] = (int64_t)v[i];
  return SWMM_OK;
}

int swmm_test_hook(swmm_t h, int32_t hook, int64_t value) {
  if (!h) return SWMM_EINVAL;
  switch (hook) {
    case SWMM_HOOK_WAIT_NS:
      h->wait_ns = value > 0 ? (uint64_t)value : kDefaultWaitNs;
      return SWMM_OK;
    case SWMM_HOOK_STALL_GEMMS:
      h->stall_left = value > 0 ? (int)std::min<int64_t>(value, 1 << 30) : 0;
      return SWMM_OK;
    case SWMM_HOOK_FAIL_ALLOCS:
      h->fail_allocs = value > 0 ? (int)std::min<int64_t>(value, 1 << 30) : 0;
      return SWMM_OK;
    case SWMM_HOOK_LOWMEM_BYTES:
      h->lowmem_bytes = value > 0 ? value : SWMM_LOWMEM_STAGE_BYTES;
      return SWMM_OK;
  }
  return fail(h, SWMM_EINVAL, "unknown test hook");
}

const char *swmm_strerror(int code) {
  switch (code) {
    case SWMM_OK: return "ok";
    case SWMM_EINVAL: return "invalid argument";
    case SWMM_ENOMEM: return "out of device memory";
    case SWMM_EUNSUPPORTED: return "unsupported";
    case SWMM_ECUDA: return "CUDA error";
    case SWMM_ETIMEOUT: return "device wait timed out";
  }
  return "unknown error";
}

const char *swmm_last_error(swmm_t h) { return h ? h->last_error.c_str() : "invalid handle"; }

int swmm_set_schedule(swmm_t h, const swmm_search_spec *spec, const swmm_search_row *rows, int32_t nrows) {
  if (!h) return SWMM_EINVAL;
  h->last_error.clear();
  return set_schedule(h, spec, rows, nrows);
}

int swmm_schedule_workspace(const swmm_search_spec *spec, const swmm_search_row *rows, int32_t nrows, int64_t m,
                            int64_t k, int64_t n, const swmm_opts *opts, int64_t *paper_elems, int64_t *plan_elems,
                            double *model_us_out) {
  swmm_ctx planner;  // no device
  int rc = set_schedule(&planner, spec, rows, nrows);
  if (rc != SWMM_OK) return rc;
  if (!opts || opts->sched != SWMM_CUSTOM) return SWMM_EINVAL;
  Plan P;
  rc = plan_only(&planner, m, k, n, opts, P);
  if (rc != SWMM_OK) return rc;
  if (paper_elems) *paper_elems = P.paper;
  if (plan_elems) *plan_elems = P.x.tmp_peak_elems;
  if (model_us_out) *model_us_out = model_us(P);
  return SWMM_OK;
}

}  // extern "C"
