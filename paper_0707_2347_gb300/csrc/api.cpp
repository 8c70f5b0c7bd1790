// C ABI of the library (include/swmm.h): argument validation, workspace
// management and dispatch to the schedule executor.
#include "swmm.h"

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>

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

// 2-D map over `rows` rows of `kpad` 16-bit values; boxes of 64 x box_rows
// land in shared memory with the 128-byte swizzle the MMA descriptors use.
bool make_tmap(CUtensorMap *map, const void *base, int64_t rows, int64_t kpad, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)kpad, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)kpad * 2};
  cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, const_cast<void *>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool make_target_tmap(CUtensorMap *map, const void *base, int64_t rows, int64_t cols, int64_t ld, bool fp32) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || ((uintptr_t)base % 16) != 0 || (ld % 4) != 0 || rows <= 0 || cols <= 0) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
  cuuint32_t box[2] = {32, (cuuint32_t)kBM};
  cuuint32_t estr[2] = {1, 1};
  // the element type matters for TMA reduce-add: float sums or unsigned
  // integer sums of mod p contributions
  CUresult r = fn(map, fp32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT32, 2,
                  const_cast<void *>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace swmm

using namespace swmm;

#include <vector>

struct EventTimer : swmm::TimingHook {
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
    cudaEventRecord(ev[2 * used], s);
  }
  void end(cudaStream_t s, double f) override {
    cudaEventRecord(ev[2 * used + 1], s);
    flops[used] = f;
    ++used;
  }
  ~EventTimer() override {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  }
};

struct swmm_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int num_sms = 152;
  int *d_err = nullptr;
  swmm_stats stats;
  std::string last_error;
  EventTimer timer;
};

namespace {

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
  }
  return NKIND;
}

// Temporaries per level the paper gives for each schedule (Section 3,
// Section 5, Section 6), summed over `levels` levels: the Lemma 1 series.
int64_t paper_elems(int sched, int64_t m, int64_t k, int64_t n, int levels) {
  int64_t s = 0;
  for (int i = 0; i < levels; ++i) {
    m /= 2;
    k /= 2;
    n /= 2;
    switch (sched) {
      case SWMM_T1_DHSS: s += m * std::max(k, n) + k * n; break;        // Eq. (1)
      case SWMM_T2_HLJJTT: s += m * k + k * n + m * n; break;          // Eq. (2)
      case SWMM_T4_OVL:
      case SWMM_T4M_OVL:
      case SWMM_T5_OVR: s += n * n; break;                             // Sec. 5.1
      case SWMM_T6_ACLR:
      case SWMM_T7_ACCR:
      case SWMM_T9_ACC: s += 2 * n * n; break;                         // Eq. (3), Sec. 6
      case SWMM_T8_ACR: s += std::max(m, k) * n + m * k; break;         // Sec. 5.3
      default: break;                                                  // IP, IPMM, classical: 0
    }
  }
  return s;
}

// number of Winograd levels the recursion actually performs
int levels_possible(int64_t m, int64_t k, int64_t n, int depth) {
  int d = 0;
  while (d < depth && m >= 2 && k >= 2 && n >= 2 && m % 2 == 0 && k % 2 == 0 && n % 2 == 0) {
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

int run(swmm_t h, const Req &q, const swmm_opts *o, bool dry_only, int64_t *paper_out, int64_t *plan_out,
        const Scratch *ext = nullptr) {
  if (!h) return SWMM_EINVAL;
  h->last_error.clear();
  if (!o) return fail(h, SWMM_EINVAL, "opts is NULL");
  if (o->mode != SWMM_MODP && o->mode != SWMM_FP32) return fail(h, SWMM_EINVAL, "unknown mode");
  if (o->mode == SWMM_MODP && (o->p <= 2 || o->p >= 65536)) return fail(h, SWMM_EINVAL, "p must satisfy 2 < p < 65536");
  if (q.m < 0 || q.k < 0 || q.n < 0) return fail(h, SWMM_EINVAL, "negative dimension");
  if (q.m > (1 << 30) || q.k > (1 << 30) || q.n > (1 << 30)) return fail(h, SWMM_EINVAL, "dimension too large");
  if (o->depth < 0 || o->depth > 30) return fail(h, SWMM_EINVAL, "depth out of range");
  const int sched = o->sched;
  const bool accum_req = q.entry == 1 || (q.entry == 2 && q.beta != nullptr);
  // schedule / entry point consistency (overwrite contracts, Sections 3, 5)
  bool okk = false;
  if (q.entry == 0) okk = sched == SWMM_CLASSICAL || sched == SWMM_T1_DHSS || sched == SWMM_IPMM;
  if (q.entry == 1) okk = sched == SWMM_CLASSICAL || sched == SWMM_T2_HLJJTT || sched == SWMM_T9_ACC;
  if (q.entry == 2 && !accum_req)
    okk = sched == SWMM_T3_IP || sched == SWMM_T4_OVL || sched == SWMM_T4M_OVL || sched == SWMM_T5_OVR;
  if (q.entry == 2 && accum_req) okk = sched == SWMM_T6_ACLR || sched == SWMM_T7_ACCR || sched == SWMM_T8_ACR;
  if (!okk) return fail(h, SWMM_EINVAL, "schedule not valid for this entry point");
  const bool ne = q.m > 0 && q.n > 0;
  if (!dry_only) {
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
  const int lv = levels_possible(q.m, q.k, q.n, depth);
  if (sched != SWMM_CLASSICAL && sched != SWMM_IPMM && lv > 0) {
    const KindInfo &K = kind_info(kind_of(sched));
    if (K.square && !(q.m == q.k && q.k == q.n))
      return fail(h, SWMM_EINVAL, std::string(K.name) + " needs square operands (Section 5.3)");
    if (sched == SWMM_T3_IP && !(q.k == q.n && q.n <= q.m))
      return fail(h, SWMM_EINVAL, "IP needs k = n <= m (Section 5.3)");
  }
  if (sched == SWMM_IPMM && q.m != q.n) return fail(h, SWMM_EINVAL, "IPMM needs m = n (Algorithm 2)");

  Exec x;
  x.fp32 = o->mode == SWMM_FP32;
  x.p = x.fp32 ? 0 : o->p;
  x.mode = x.fp32 ? MODE_FP32 : (o->p <= 256 ? MODE_MODP1 : MODE_MODP2);
  x.fused = !(o->flags & SWMM_FLAG_UNFUSED);
  x.simt = (o->flags & SWMM_FLAG_SIMT_LEAF) != 0;
  x.stream = h->stream;
  x.num_sms = h->num_sms;
  x.err = h->d_err;
  x.timing = (o->flags & SWMM_FLAG_TIMING) && !ext ? &h->timer : nullptr;
  Scalar alpha, beta;
  if (x.fp32) {
    alpha.f = q.alpha ? *(const float *)q.alpha : 1.f;
    beta.f = q.beta ? *(const float *)q.beta : 0.f;
  } else {
    alpha.u = q.alpha ? *(const uint32_t *)q.alpha % x.p : 1u;
    beta.u = q.beta ? *(const uint32_t *)q.beta % x.p : 0u;
  }
  View L, R, D;
  L.ptr = (char *)q.A;
  L.rows = q.m;
  L.cols = q.k;
  L.ld = q.lda;
  R.ptr = (char *)q.B;
  R.rows = q.k;
  R.cols = q.n;
  R.ld = q.ldb;
  D.ptr = (char *)q.C;
  D.rows = q.m;
  D.cols = q.n;
  D.ld = q.ldc;
  const int64_t cutoff = o->ipmm_cutoff > 0 ? o->ipmm_cutoff : 1024;
  const Kind ipmm_acc = o->ipmm_acc == SWMM_T9_ACC ? K_ACC : K_T2;

  auto execute = [&](Exec &e) {
    if (!ne) return;
    if (sched == SWMM_IPMM)
      e.ipmm(L, R, D, depth, cutoff, ipmm_acc);
    else if (sched == SWMM_CLASSICAL)
      e.leaf(alpha, accum_req, beta, L, R, D);
    else
      e.call(kind_of(sched), alpha, accum_req, beta, L, R, D, depth, Arena{});
  };
  // planning pass: sizes and counts, no launches
  x.dry = true;
  execute(x);
  if (!x.fail.empty()) return fail(h, SWMM_EINVAL, x.fail);
  // levels that materialise temporaries: all but a fused last one
  const int tmp_levels = (x.fused && lv > 0 && sched != SWMM_IPMM) ? lv - 1 : lv;
  const int64_t paper = paper_elems(sched, q.m, q.k, q.n, tmp_levels);
  if (paper_out) *paper_out = paper;
  if (plan_out) *plan_out = x.tmp_peak_elems;
  if (dry_only) return SWMM_OK;

  Exec r = x;
  r.dry = false;
  r.lazy = false;
  r.ws_top = r.ws_peak = 0;
  r.tmp_elems = r.tmp_peak_elems = 0;
  r.add_elems = r.leaf_flops = r.leaf_launches = r.ew_launches = r.leaf_products = 0;
  r.stage_need = x.stage_need;
  if (ext) {
    // caller-provided scratch: carve, never allocate
    const int64_t ws_bytes = (x.ws_peak + 1023) / 1024 * 1024;
    if (ws_bytes + x.stage_need > ext->bytes)
      return fail(h, SWMM_EINVAL,
                  "plan needs " + std::to_string(ws_bytes + x.stage_need) + " bytes of scratch, more than the " +
                      std::to_string(ext->bytes) + "-byte static scratch");
    r.ws = x.ws_peak > 0 ? ext->base : nullptr;
    r.stage = x.stage_need > 0 ? ext->base + ws_bytes : nullptr;
  } else if (x.ws_peak > 0) {
    if (cudaMallocAsync((void **)&r.ws, x.ws_peak, h->stream) != cudaSuccess) {
      cudaGetLastError();
      return fail(h, SWMM_ENOMEM, "workspace allocation failed");
    }
  }
  if (!ext && x.stage_need > 0) {
    if (cudaMallocAsync((void **)&r.stage, x.stage_need, h->stream) != cudaSuccess) {
      cudaGetLastError();
      if (r.ws) cudaFreeAsync(r.ws, h->stream);
      return fail(h, SWMM_ENOMEM, "staging allocation failed");
    }
  }
  execute(r);
  if (r.lazy && r.ok()) {
    // fused levels leave unreduced representatives: one canonicalising pass
    ++r.ew_launches;
    cudaError_t e = launch_canon_modp(D, r.p, h->stream);
    if (e != cudaSuccess) {
      r.cuda_err = e;
      r.fail = std::string("canonical pass: ") + cudaGetErrorString(e);
    }
  }
  if (!ext && r.ws) cudaFreeAsync(r.ws, h->stream);
  if (!ext && r.stage) cudaFreeAsync(r.stage, h->stream);
  std::memset(&h->stats, 0, sizeof(h->stats));
  h->stats.workspace_bytes = x.ws_peak;
  h->stats.plan_extra_elems = x.tmp_peak_elems;
  h->stats.paper_extra_elems = paper;
  h->stats.add_elems = r.add_elems;
  h->stats.leaf_flops = r.leaf_flops;
  h->stats.leaf_launches = r.leaf_launches;
  h->stats.ew_launches = r.ew_launches;
  h->stats.leaf_products = r.leaf_products;
  h->stats.staging_bytes = x.stage_need;
  if (r.cuda_err != cudaSuccess) return fail(h, SWMM_ECUDA, r.fail);
  if (!r.fail.empty()) return fail(h, SWMM_EINVAL, r.fail);
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
  return run(h, q, opts, false, nullptr, nullptr, &s);
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
  return run(h, q, opts, false, nullptr, nullptr);
}

int swmm_muladd(swmm_t h, int64_t m, int64_t k, int64_t n, const void *alpha, const void *A, int64_t lda,
                const void *B, int64_t ldb, const void *beta, void *C, int64_t ldc, const swmm_opts *opts) {
  if (!alpha || !beta) return fail(h, SWMM_EINVAL, "alpha and beta are required");
  Req q{1, m, k, n, A, B, C, lda, ldb, ldc, alpha, beta};
  return run(h, q, opts, false, nullptr, nullptr);
}

int swmm_mul_inplace(swmm_t h, int64_t m, int64_t k, int64_t n, void *A, int64_t lda, void *B, int64_t ldb, void *C,
                     int64_t ldc, const void *alpha, const void *beta, const swmm_opts *opts) {
  Req q{2, m, k, n, A, B, C, lda, ldb, ldc, alpha, beta};
  return run(h, q, opts, false, nullptr, nullptr);
}

int swmm_workspace_elems(swmm_t h, int64_t m, int64_t k, int64_t n, const swmm_opts *opts, int64_t *paper_elems,
                         int64_t *plan_elems) {
  swmm_ctx planner;  // planning needs no device: a NULL handle is accepted
  if (!h) h = &planner;
  if (!opts) return fail(h, SWMM_EINVAL, "opts is NULL");
  const int s = opts->sched;
  const bool acc_inplace = s == SWMM_T6_ACLR || s == SWMM_T7_ACCR || s == SWMM_T8_ACR;
  int entry = 0;
  if (s == SWMM_T2_HLJJTT || s == SWMM_T9_ACC) entry = 1;
  if (s == SWMM_T3_IP || s == SWMM_T4_OVL || s == SWMM_T4M_OVL || s == SWMM_T5_OVR || acc_inplace) entry = 2;
  static const uint32_t one = 1;
  Req q{entry, m, k, n, nullptr, nullptr, nullptr, k, n, n, &one, acc_inplace || entry == 1 ? &one : nullptr};
  return run(h, q, opts, true, paper_elems, plan_elems);
}

int swmm_leaf_timing(swmm_t h, int reset, double *gemm_ms, int64_t *launches, double *tensor_flops) {
  if (!h) return SWMM_EINVAL;
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return fail(h, SWMM_ECUDA, cudaGetErrorString(e));
  double ms = 0.0, fl = 0.0;
  for (size_t i = 0; i < h->timer.used; ++i) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, h->timer.ev[2 * i], h->timer.ev[2 * i + 1]) != cudaSuccess)
      return fail(h, SWMM_ECUDA, "event timing failed");
    ms += t;
    fl += h->timer.flops[i];
  }
  if (gemm_ms) *gemm_ms = ms;
  if (launches) *launches = (int64_t)h->timer.used;
  if (tensor_flops) *tensor_flops = fl;
  if (reset) h->timer.used = 0;
  return SWMM_OK;
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

}  // extern "C"
