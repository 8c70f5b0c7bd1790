// Recursive executor of the schedules (Tables 1-9, Algorithm 2).
//
// A call D <- alpha L R (+ beta D) of kind k with depth d:
//   * d == 0, or a dimension odd or < 2: one classical leaf product;
//   * d == 1 with fusion on: the whole last Winograd level (Section 2) in one
//     grouped tensor-core launch: seven products whose operands are the
//     signed quadrant sums S1..S4 / T1..T4 formed while packing, and whose
//     results are added into the four quadrants of D (the post-additions
//     U1..U7) -- no temporary of this level is materialised;
//   * otherwise: the rows of table k, in order, each ADD/COPY row one
//     elementwise launch and each MUL row a recursive call of depth d - 1.
// Temporaries of a level come from the handle's workspace (a bump allocator,
// so the peak is exactly the sum over the live levels, Lemma 1) or, inside
// Algorithm 2, are carved from C22.
#include "executor.h"

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cstdio>
#include <cstring>

namespace swmm {

namespace {
int64_t rup(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// NVTX range over the issue of one table level / fused level / driver (the
// launches it enqueues; visible to profilers, free when none is attached)
struct Range {
  bool on;
  Range(bool active, const char *what, int64_t m, int64_t k, int64_t n, int depth) : on(active) {
    if (!on) return;
    char buf[96];
    snprintf(buf, sizeof(buf), "%s %lldx%lldx%lld d%d", what, (long long)m, (long long)k, (long long)n, depth);
    nvtxRangePushA(buf);
  }
  ~Range() {
    if (on) nvtxRangePop();
  }
};
bool aligned16(const void *p, int64_t ld) { return ((uintptr_t)p % 16 == 0) && (ld % 4 == 0); }

// One Winograd level as a fused level computes it (Section 2's sums).
// Operand coefficients over (X11, X12, X21, X22), product i in row i:
const int8_t acoef[7][4] = {
    {1, 0, 0, 0},    // A11
    {0, 1, 0, 0},    // A12
    {1, 1, -1, -1},  // S4 = A12 - A21 - A22 + A11
    {0, 0, 0, 1},    // A22
    {0, 0, 1, 1},    // S1 = A21 + A22
    {-1, 0, 1, 1},   // S2 = A21 + A22 - A11
    {1, 0, -1, 0},   // S3 = A11 - A21
};
const int8_t bcoef[7][4] = {
    {1, 0, 0, 0},    // B11
    {0, 0, 1, 0},    // B21
    {0, 0, 0, 1},    // B22
    {1, -1, -1, 1},  // T4 = B22 - B12 + B11 - B21
    {-1, 1, 0, 0},   // T1 = B12 - B11
    {1, -1, 0, 1},   // T2 = B22 - B12 + B11
    {0, -1, 0, 1},   // T3 = B22 - B12
};
// targets: quadrant index (0 = C11, 1 = C12, 2 = C21, 3 = C22) and sign
const int8_t tgt[7][4] = {
    {1, 1, 1, 1}, {1, 0, 0, 0}, {0, 1, 0, 0}, {0, 0, -1, 0}, {0, 1, 0, 1}, {0, 1, 1, 1}, {0, 0, 1, 1},
};
// Order of the products in a launch: most targets first (P1, P6, P5, P7,
// then P2, P3, P4), so the reduce-adds of a launch's last wave, which no
// longer overlap any multiplication, are single-target ones.
const int ord[7] = {0, 5, 4, 6, 1, 2, 3};
}  // namespace

// tensor-core products per leaf product: 1 limb (p <= 256), 2 x 2 limbs,
// or hi*hi + hi*lo + lo*hi in FP32 mode
int Exec::limb_products() const { return mode == MODE_MODP1 ? 1 : (mode == MODE_MODP2 ? 4 : 3); }

Scalar Exec::one() const {
  Scalar s;
  s.u = 1;
  s.f = 1.f;
  return s;
}
Scalar Exec::neg(Scalar s) const {
  Scalar r;
  r.u = s.u == 0 ? 0 : p - s.u;
  r.f = -s.f;
  return r;
}

void Exec::check(cudaError_t e, const char *what) {
  if (e != cudaSuccess && cuda_err == cudaSuccess) {
    cuda_err = e;
    fail = std::string(what) + ": " + cudaGetErrorString(e);
  }
}

View Exec::alloc_tmp(int64_t rows, int64_t cols) {
  View v;
  v.rows = rows;
  v.cols = cols;
  v.ld = cols;
  v.ptr = ws ? ws + ws_top : nullptr;
  if (!dry && ws_limit >= 0 && ws_top + rows * cols * 4 > ws_limit) {
    // the planning pass sized the area: a real run must never need more
    if (fail.empty()) fail = "temporaries exceed the planned workspace";
    v.ptr = nullptr;
  }
  ws_top += rup(rows * cols * 4, 256);
  ws_peak = std::max(ws_peak, ws_top);
  tmp_elems += rows * cols;
  tmp_peak_elems = std::max(tmp_peak_elems, tmp_elems);
  return v;
}

// every element of `in` lies in `out` (exact for views of one root and
// leading dimension; false otherwise)
static bool contains(const Rect &out, const Rect &in) {
  return out.base == in.base && out.ld == in.ld && out.ld > 0 && in.r0 >= out.r0 && in.c0 >= out.c0 &&
         in.r0 + in.rows <= out.r0 + out.rows && in.c0 + in.cols <= out.c0 + out.cols;
}

void Exec::mark_lazy(const View &v) {
  if (fp32 || v.rows == 0 || v.cols == 0) return;
  const Rect r = rect_of(v);
  for (const View &x : lazy_views)
    if (contains(rect_of(x), r)) return;
  lazy_views.push_back(v);
}

void Exec::mark_canonical(const View &v) {
  if (lazy_views.empty()) return;
  const Rect r = rect_of(v);
  lazy_views.erase(std::remove_if(lazy_views.begin(), lazy_views.end(),
                                  [&](const View &x) { return contains(r, rect_of(x)); }),
                   lazy_views.end());
}

static bool any_overlap(const std::vector<Rect> &a, const std::vector<Rect> &b) {
  for (const Rect &x : a)
    for (const Rect &y : b)
      if (overlaps(x, y)) return true;
  return false;
}

cudaStream_t Exec::op_begin(const std::vector<Rect> &rd, const std::vector<Rect> &wr, bool dma) {
  // a deferred GEMM launch goes out before anything that touches its memory
  if (pend.n > 0 && !flushing &&
      (any_overlap(rd, pend.wr) || any_overlap(wr, pend.rd) || any_overlap(wr, pend.wr)))
    flush();
  if (!flow) return stream;
  return flow->begin(rd.data(), (int)rd.size(), wr.data(), (int)wr.size(), dma);
}

void Exec::op_end() {
  if (flow) flow->end();
}

// Queue the products of one leaf group or fused level (P: its parameters,
// null in a dry run) for a GEMM launch; they join the pending launch unless
// it is full or they depend on it (reduce-adds into a common target commute
// and may share it).
void Exec::queue_gemm(const GemmParams *P, const std::vector<Rect> &rd, const std::vector<Rect> &wr, bool additive,
                      double flops, int nprod) {
  if (pend.n > 0) {
    const bool fits = pend.n + nprod <= kMaxProducts;
    const bool dep = any_overlap(rd, pend.wr) || any_overlap(wr, pend.rd) ||
                     (any_overlap(wr, pend.wr) && !(additive && pend.additive));
    if (!fits || dep) flush();
  }
  if (pend.n == 0) {
    if (P) pend.P = *P;
    pend.tiles = 0;
    pend.flops = 0.0;
    pend.additive = true;
    pend.rd.clear();
    pend.wr.clear();
  }
  if (P) {
    for (int i = 0; i < nprod; ++i) {
      Product &q = pend.P.prod[pend.n + i];
      q = P->prod[i];
      q.tile_begin = pend.tiles;
      pend.tiles += q.tiles_m * q.tiles_n;
    }
  }
  pend.n += nprod;
  pend.flops += flops;
  pend.additive = pend.additive && additive;
  pend.rd.insert(pend.rd.end(), rd.begin(), rd.end());
  pend.wr.insert(pend.wr.end(), wr.begin(), wr.end());
  if (!merge) flush();
}

void Exec::flush() {
  if (pend.n == 0) return;
  ++leaf_launches;
  if (!dry) {
    pend.P.nprod = pend.n;
    pend.P.total_tiles = pend.tiles;
    pend.P.wait_ns = wait_ns;
    pend.P.test_stall = 0;
    if (stall_left && *stall_left > 0) {
      --*stall_left;
      pend.P.test_stall = 1;
    }
    flushing = true;
    cudaStream_t st = op_begin(pend.rd, pend.wr);
    flushing = false;
    if (timing) timing->begin(st);
    check(launch_gemm_tc(pend.P, mode, num_sms, st), "leaf gemm");
    if (timing) timing->end(st, pend.flops);
    op_end();
  }
  pend.n = 0;
  pend.tiles = 0;
  pend.flops = 0.0;
  pend.rd.clear();
  pend.wr.clear();
}

char *Exec::next_stage() {
  const int64_t slot = rup(stage_need, 1024);
  const int64_t off = (stage_turn++ % stage_slots) * slot;
  if (stage_limit >= 0 && off + stage_need > stage_limit) {
    // the planning pass sized the area: a real run must never need more
    if (fail.empty()) fail = "operand staging exceeds the planned area";
    return nullptr;
  }
  return stage + off;
}

// FP32 mode: zero the two amax words at the head of a staging slot, then
// max |x| over the A-side and the B-side sources of the coming packs.
void Exec::fp32_amax(uint32_t *amax, const View *a, int na, const View *b, int nb) {
  const Rect rh = rect_bytes(amax, 2 * sizeof(uint32_t));
  cudaStream_t st = op_begin({}, {rh});
  check(cudaMemsetAsync(amax, 0, 2 * sizeof(uint32_t), st), "amax reset");
  op_end();
  AmaxArgs g;
  std::memset(&g, 0, sizeof(g));
  std::vector<Rect> rd;
  for (int q = 0; q < na; ++q) {
    g.src[0][q] = a[q].ptr;
    g.ld[0][q] = a[q].ld;
    rd.push_back(rect_of(a[q]));
  }
  for (int q = 0; q < nb; ++q) {
    g.src[1][q] = b[q].ptr;
    g.ld[1][q] = b[q].ld;
    rd.push_back(rect_of(b[q]));
  }
  g.nsrc[0] = na;
  g.nsrc[1] = nb;
  g.rows[0] = na ? a[0].rows : 0;
  g.cols[0] = na ? a[0].cols : 0;
  g.rows[1] = nb ? b[0].rows : 0;
  g.cols[1] = nb ? b[0].cols : 0;
  g.amax = amax;
  st = op_begin(rd, {rh});
  check(launch_amax(g, st), "amax");
  op_end();
}

void Exec::add(View d, View s1, View s2, Scalar c1, Scalar c2) {
  add_elems += d.rows * d.cols;
  ++ew_launches;
  mark_canonical(d);
  if (dry) return;
  cudaStream_t st = op_begin({rect_of(s1), rect_of(s2)}, {rect_of(d)});
  if (fp32)
    check(launch_add_f(d, s1, s2, c1.f, c2.f, st), "add");
  else
    check(launch_add(d, s1, s2, c1.u, c2.u, p, 0, st), "add");
  op_end();
}

void Exec::scale(View d, bool keep, Scalar beta) {
  ++ew_launches;
  mark_canonical(d);
  if (dry) return;
  cudaStream_t st = op_begin({}, {rect_of(d)});
  if (fp32)
    check(launch_scale_f(d, keep ? beta.f : 0.f, st), "scale");
  else
    check(launch_scale_modp(d, keep ? beta.u : 0u, p, st), "scale");
  op_end();
}

// ----------------------------------------------------------------- leaves
static void fill_common(GemmParams &P, const Exec &x, Scalar alpha, bool acc, Scalar beta, int epi) {
  std::memset(&P, 0, sizeof(P));
  P.epilogue = epi;
  P.p = x.p ? x.p : 1;
  P.alpha_u = alpha.u;
  P.beta_u = beta.u;
  P.alpha_f = alpha.f;
  P.beta_f = beta.f;
  P.barrett = x.p ? (uint32_t)(0x100000000ull / x.p) : 0;
  P.inv_p = x.p ? 1.0f / (float)x.p : 0.f;
  P.use_beta = acc ? 1 : 0;
  P.err = x.err;
}

static void set_scalars(Product &pr, Scalar alpha, bool acc, Scalar beta, int epi) {
  pr.epilogue = epi;
  pr.use_beta = acc ? 1 : 0;
  pr.alpha_u = alpha.u;
  pr.beta_u = beta.u;
  pr.alpha_f = alpha.f;
  pr.beta_f = beta.f;
}

void Exec::leaf(Scalar alpha, bool acc, Scalar beta, View L, View R, View D) {
  const int64_t m = L.rows, k = L.cols, n = R.cols;
  if (m == 0 || n == 0) return;
  if (k == 0) {  // empty inner dimension: D <- beta D (or 0)
    scale(D, acc, beta);
    return;
  }
  if (!simt) {
    const int pl = planes_of(mode);
    const int64_t per_k = pl * (rup(m, kBM) + rup(n, bn_of(mode))) * 2;  // staging bytes per unit of k
    const int64_t hdr = fp32 ? 1024 : 0;
    if (stage_budget > 0 && k > kBK && hdr + per_k * rup(k, kBK) > stage_budget) {
      // under a staging bound: K-slabs whose operands fit it, each after the
      // first accumulating into D (D <- alpha L_j R_j + D)
      const int64_t ks = std::max<int64_t>(kBK, (stage_budget - hdr) / per_k / kBK * kBK);
      for (int64_t k0 = 0; k0 < k; k0 += ks) {
        const int64_t kk = std::min(ks, k - k0);
        const LeafJob job{L.sub(0, k0, m, kk), R.sub(k0, 0, kk, n), D};
        leaf_group(alpha, k0 == 0 ? acc : true, k0 == 0 ? beta : one(), &job, 1);
      }
      return;
    }
    const LeafJob job{L, R, D};
    leaf_group(alpha, acc, beta, &job, 1);
    return;
  }
  leaf_flops += 2 * m * n * k;
  ++leaf_products;
  ++leaf_launches;
  if (dry) return;
  GemmParams P;
  fill_common(P, *this, alpha, acc, beta, EPI_STORE);
  SimtArgs S;
  std::memset(&S, 0, sizeof(S));
  S.a[0] = L.ptr;
  S.lda[0] = L.ld;
  S.sa[0] = 1;
  S.na = 1;
  S.b[0] = R.ptr;
  S.ldb[0] = R.ld;
  S.sb[0] = 1;
  S.nb = 1;
  S.t[0].ptr = D.ptr;
  S.t[0].ld = D.ld;
  S.t[0].sign = 1;
  S.ntargets = 1;
  S.M = (int)m;
  S.N = (int)n;
  S.K = (int)k;
  mark_canonical(D);
  cudaStream_t st = op_begin({rect_of(L), rect_of(R)}, {rect_of(D)});
  check(launch_leaf_simt(S, P, mode, st), "simt leaf");
  op_end();
}

// Classical leaf products of independent problems (same mode, modulus and
// scalars, every dimension > 0) in one persistent grouped GEMM launch: each
// product's operands are packed into its own part of one staging slot, and
// the launch's tiles cover every product, so problems too small to fill the
// GPU on their own fill it together.
void Exec::leaf_group(Scalar alpha, bool acc, Scalar beta, const LeafJob *jobs, int njobs) {
  if (njobs <= 0) return;
  if (njobs > kMaxProducts) {
    if (fail.empty()) fail = "too many products in one grouped launch";
    return;
  }
  const int pl = planes_of(mode), bn = bn_of(mode);
  const int64_t hdr = fp32 ? 1024 : 0;  // FP32 mode: the operands' amax words
  if (stage_budget > 0 && njobs > 1) {
    // under a staging bound: launches of consecutive problems whose staging
    // fits it (a problem larger than the bound is staged alone)
    int64_t bytes[kMaxProducts], total = 0;
    for (int i = 0; i < njobs; ++i) {
      const int64_t m = jobs[i].L.rows, k = jobs[i].L.cols, n = jobs[i].R.cols;
      bytes[i] = hdr + rup(pl * rup(m, kBM) * rup(k, kBK) * 2, 1024) + rup(pl * rup(n, bn) * rup(k, kBK) * 2, 1024);
      total += bytes[i];
    }
    if (total > stage_budget) {
      const int64_t keep = stage_budget;
      stage_budget = 0;
      int first = 0;
      int64_t sum = 0;
      for (int i = 0; i < njobs; ++i) {
        if (i > first && sum + bytes[i] > keep) {
          leaf_group(alpha, acc, beta, jobs + first, i - first);
          first = i;
          sum = 0;
        }
        sum += bytes[i];
      }
      leaf_group(alpha, acc, beta, jobs + first, njobs - first);
      stage_budget = keep;
      return;
    }
  }
  int64_t Mp[kMaxProducts], Np[kMaxProducts], Kp[kMaxProducts], ab[kMaxProducts], bb[kMaxProducts],
      off[kMaxProducts];
  int64_t total = 0;
  double tflops = 0.0;
  for (int i = 0; i < njobs; ++i) {
    const int64_t m = jobs[i].L.rows, k = jobs[i].L.cols, n = jobs[i].R.cols;
    Mp[i] = rup(m, kBM);
    Np[i] = rup(n, bn);
    Kp[i] = rup(k, kBK);
    ab[i] = rup(pl * Mp[i] * Kp[i] * 2, 1024);
    bb[i] = rup(pl * Np[i] * Kp[i] * 2, 1024);
    off[i] = total;
    total += hdr + ab[i] + bb[i];
    pack_bytes += (int64_t)jobs[i].L.esz * m * k + (int64_t)jobs[i].R.esz * k * n + ab[i] + bb[i];
    leaf_flops += 2 * m * n * k;
    ++leaf_products;
    tflops += 2.0 * m * n * k * limb_products();
  }
  stage_need = std::max(stage_need, total);
  ew_launches += njobs * (fp32 ? 2 : 1);
  if (dry) {
    queue_gemm(nullptr, {}, {}, false, tflops, njobs);
    return;
  }
  char *base = next_stage();
  if (!base) return;
  GemmParams P;
  fill_common(P, *this, alpha, acc, beta, EPI_STORE);
  std::vector<Rect> grd, gwr;
  int tiles = 0;
  for (int i = 0; i < njobs; ++i) {
    const View &L = jobs[i].L, &R = jobs[i].R, &D = jobs[i].D;
    const int64_t m = L.rows, k = L.cols, n = R.cols;
    char *stg = base + off[i];
    uint32_t *amax = fp32 ? reinterpret_cast<uint32_t *>(stg) : nullptr;
    uint16_t *Ap = reinterpret_cast<uint16_t *>(stg + hdr);
    uint16_t *Bp = reinterpret_cast<uint16_t *>(stg + hdr + ab[i]);
    const Rect ra = rect_bytes(Ap, ab[i]), rb = rect_bytes(Bp, bb[i]), rh = rect_bytes(stg, 8);
    if (fp32) fp32_amax(amax, &L, 1, &R, 1);
    PackArgs pa;
    std::memset(&pa, 0, sizeof(pa));
    pa.src[0][0] = L.ptr;
    pa.ld[0][0] = L.ld;
    pa.tsign[0] = 1;
    pa.tesz[0] = (int8_t)L.esz;
    pa.nterm = 1;
    pa.nsrc = 1;
    pa.out[0] = Ap;
    pa.coef[0][0] = 1;
    pa.nout = 1;
    pa.rows = (int)m;
    pa.cols = (int)k;
    pa.prow_pad = (int)Mp[i];
    pa.pcol_pad = (int)Kp[i];
    pa.transpose = 0;
    pa.p = p;
    pa.barrett = p ? (uint32_t)(0x100000000ull / p) : 0;
    pa.amax = amax;
    pa.terms = 1;
    PackArgs pb = pa;
    pb.src[0][0] = R.ptr;
    pb.ld[0][0] = R.ld;
    pb.tesz[0] = (int8_t)R.esz;
    pb.out[0] = Bp;
    pb.rows = (int)k;
    pb.cols = (int)n;
    pb.prow_pad = (int)Np[i];
    pb.pcol_pad = (int)Kp[i];
    pb.transpose = 1;
    pb.amax = amax ? amax + 1 : nullptr;
    cudaStream_t st = op_begin({rect_of(L), rect_of(R), rh}, {ra, rb});
    check(launch_pack_pair(pa, pb, mode, st), "pack");
    op_end();
    Product &pr = P.prod[i];
    if (!make_tmap(&pr.ta, Ap, pl * Mp[i], Kp[i], kBM) || !make_tmap(&pr.tb, Bp, pl * Np[i], Kp[i], bn)) {
      if (fail.empty()) fail = "tensor map encoding failed";
      return;
    }
    pr.t[0].ptr = D.ptr;
    pr.t[0].ld = D.ld;
    pr.t[0].sign = 1;
    pr.t[0].vec_ok = aligned16(D.ptr, D.ld);
    pr.ntargets = 1;
    pr.tma_epi = make_target_tmap(&pr.tmap[0], D.ptr, m, n, D.ld, fp32) ? 1 : 0;
    pr.M = (int)m;
    pr.N = (int)n;
    pr.Kpad = (int)Kp[i];
    pr.a_plane_rows = (int)Mp[i];
    pr.b_plane_rows = (int)Np[i];
    pr.tiles_m = (int)(Mp[i] / kBM);
    pr.tiles_n = (int)(Np[i] / bn);
    pr.tile_begin = tiles;
    pr.amax = amax;
    pr.terms_a = pr.terms_b = 1;
    set_scalars(pr, alpha, acc, beta, EPI_STORE);
    tiles += pr.tiles_m * pr.tiles_n;
    grd.push_back(ra);
    grd.push_back(rb);
    grd.push_back(rh);
    gwr.push_back(rect_of(D));
    mark_canonical(D);
  }
  P.nprod = njobs;
  P.total_tiles = tiles;
  queue_gemm(&P, grd, gwr, false, tflops, njobs);
}

// One whole Winograd level (Section 2) with fused pre- and post-additions.
// Products and where their signed, alpha-scaled results go:
//   P1 = A11 B11 -> +C11 +C12 +C21 +C22     P5 = S1 T1 -> +C12 +C22
//   P2 = A12 B21 -> +C11                     P6 = S2 T2 -> +C12 +C21 +C22
//   P3 = S4 B22  -> +C12                     P7 = S3 T3 -> +C21 +C22
//   P4 = A22 T4  -> -C21
// with S1 = A21 + A22, S2 = S1 - A11, S3 = A11 - A21, S4 = A12 - S2 and
// T1 = B12 - B11, T2 = B22 - T1, T3 = B22 - B12, T4 = T2 - B21, i.e.
// C11 = U1, C12 = U5, C21 = U6, C22 = U7.
bool Exec::fuses(int64_t m, int64_t k, int64_t n, int depth) const {
  return fused && depth == 1 && m >= 2 && k >= 2 && n >= 2 && m % 2 == 0 && k % 2 == 0 && n % 2 == 0;
}

// Staged sizes of one product of a fused level over L (m x k) and R (k x n).
void Exec::level_bytes(const View &L, const View &R, int64_t &abytes, int64_t &bbytes) const {
  const int pl = planes_of(mode), bn = bn_of(mode);
  const int64_t Mp = rup(L.rows / 2, kBM), Np = rup(R.cols / 2, bn), Kp = rup(L.cols / 2, kBK);
  abytes = rup(pl * Mp * Kp * 2, 1024);
  bbytes = rup(pl * Np * Kp * 2, 1024);
}

// Pack arguments of products [g0, g0 + gn) (in launch order) of the fused
// level over LL x RL, outputs at stg (the gn A operands, then the gn B
// operands).  The sources are the quadrants the group's operands use (all
// four for a whole level), each the signed sum of that quadrant of every
// term.  A whole level forms the chains S2 = S1 - A11, S4 = A12 - S2 and
// T2 = B22 - T1, T4 = T2 - B21 once per element, output i holding product
// i; a group's generic pack writes its products in launch order.
void Exec::pack_args(const Lin &LL, const Lin &RL, int g0, int gn, char *stg, const uint32_t *amax, PackArgs &pa,
                     PackArgs &pb) const {
  const View &L = LL.shape(), &R = RL.shape();
  const int64_t hm = L.rows / 2, hk = L.cols / 2, hn = R.cols / 2;
  const int64_t Mp = rup(hm, kBM), Np = rup(hn, bn_of(mode)), Kp = rup(hk, kBK);
  int64_t abytes, bbytes;
  level_bytes(L, R, abytes, bbytes);
  std::memset(&pa, 0, sizeof(pa));
  std::memset(&pb, 0, sizeof(pb));
  auto sources = [&](const Lin &LIN, const int8_t (*cf)[4], PackArgs &pk) {
    int map[4], ns = 0;
    for (int q = 0; q < 4; ++q) {
      bool used = false;
      for (int i = g0; i < g0 + gn; ++i) used = used || cf[ord[i]][q] != 0;
      map[q] = used ? ns++ : -1;
      if (!used) continue;
      for (int t = 0; t < LIN.n; ++t) {
        const View qd = LIN.v[t].quad(q / 2, q % 2);
        pk.src[map[q]][t] = qd.ptr;
        pk.ld[map[q]][t] = qd.ld;
      }
    }
    for (int t = 0; t < LIN.n; ++t) {
      pk.tsign[t] = LIN.s[t];
      pk.tesz[t] = (int8_t)LIN.v[t].esz;
    }
    pk.nterm = LIN.n;
    pk.nsrc = ns;
    pk.nout = gn;
    for (int j = 0; j < gn; ++j)
      for (int q = 0; q < 4; ++q)
        if (map[q] >= 0) pk.coef[j][map[q]] = cf[ord[g0 + j]][q];
  };
  sources(LL, acoef, pa);
  sources(RL, bcoef, pb);
  pa.set = gn == 7 ? PACK_WINOGRAD_A : PACK_GENERIC;
  pb.set = gn == 7 ? PACK_WINOGRAD_B : PACK_GENERIC;
  for (int j = 0; j < gn; ++j) {
    pa.out[j] = reinterpret_cast<uint16_t *>(stg + j * abytes);
    pb.out[j] = reinterpret_cast<uint16_t *>(stg + gn * abytes + j * bbytes);
  }
  pa.rows = (int)hm;
  pa.cols = (int)hk;
  pa.prow_pad = (int)Mp;
  pa.pcol_pad = (int)Kp;
  pa.transpose = 0;
  pa.p = p;
  pa.barrett = p ? (uint32_t)(0x100000000ull / p) : 0;
  pb.barrett = pa.barrett;
  pb.rows = (int)hk;
  pb.cols = (int)hn;
  pb.prow_pad = (int)Np;
  pb.pcol_pad = (int)Kp;
  pb.transpose = 1;
  pb.p = p;
  // |S4|, |T4| <= 4 max|source|, a source <= nterm max|term entry|
  pa.amax = amax;
  pb.amax = amax ? amax + 1 : nullptr;
  pa.terms = 4 * LL.n;
  pb.terms = 4 * RL.n;
}

void Exec::fused_level(Scalar alpha, bool acc, Scalar beta, const Lin &LL, const Lin &RL, View D,
                       const Prepacked *pre) {
  const View &L = LL.shape(), &R = RL.shape();
  const Range nv(!dry, "fused level", L.rows, L.cols, R.cols, 1);
  const int64_t hm = L.rows / 2, hk = L.cols / 2, hn = R.cols / 2;
  View Dq[4] = {D.quad(0, 0), D.quad(0, 1), D.quad(1, 0), D.quad(1, 1)};
  leaf_flops += 7 * 2 * hm * hn * hk;
  leaf_products += 7;
  // prologue: D <- beta D; nothing when beta = 1, zeros for C <- alpha AB.
  // The products are then added as unreduced representatives (mod p), so D
  // stays lazy until a consumer or the final pass reduces it.
  mark_lazy(D);
  const bool keep = acc && (fp32 ? beta.f == 1.f : beta.u == 1u);
  if (!keep) {
    ++ew_launches;
    if (!dry) {
      cudaStream_t st = op_begin({}, {rect_of(D)});
      if (!acc)
        check(launch_zero(D, st), "fused prologue");
      else if (fp32)
        check(launch_scale_f(D, beta.f, st), "fused prologue");
      else
        check(launch_scale_modp(D, beta.u, p, st), "fused prologue");
      op_end();
    }
  }
  GemmParams P;
  fill_common(P, *this, alpha, false, beta, EPI_REDUCE);
  if (simt) {
    ++leaf_launches;
    if (!dry) {
      if (LL.n != 1 || RL.n != 1 || LL.s[0] != 1 || RL.s[0] != 1) {
        if (fail.empty()) fail = "SIMT fused level needs materialised operands";
        return;
      }
      const View Lq[4] = {L.quad(0, 0), L.quad(0, 1), L.quad(1, 0), L.quad(1, 1)};
      const View Rq[4] = {R.quad(0, 0), R.quad(0, 1), R.quad(1, 0), R.quad(1, 1)};
      for (int i = 0; i < 7; ++i) {
        SimtArgs S;
        std::memset(&S, 0, sizeof(S));
        for (int q = 0; q < 4; ++q) {
          if (acoef[i][q]) {
            S.a[S.na] = Lq[q].ptr;
            S.lda[S.na] = Lq[q].ld;
            S.sa[S.na++] = acoef[i][q];
          }
          if (bcoef[i][q]) {
            S.b[S.nb] = Rq[q].ptr;
            S.ldb[S.nb] = Rq[q].ld;
            S.sb[S.nb++] = bcoef[i][q];
          }
          if (tgt[i][q]) {
            S.t[S.ntargets].ptr = Dq[q].ptr;
            S.t[S.ntargets].ld = Dq[q].ld;
            S.t[S.ntargets++].sign = tgt[i][q];
          }
        }
        S.M = (int)hm;
        S.N = (int)hn;
        S.K = (int)hk;
        cudaStream_t st = op_begin({rect_of(L), rect_of(R)}, {rect_of(D)});
        check(launch_leaf_simt(S, P, mode, st), "simt fused leaf");
        op_end();
      }
    }
  } else {
    const int pl = planes_of(mode), bn = bn_of(mode);
    const int64_t Mp = rup(hm, kBM), Np = rup(hn, bn), Kp = rup(hk, kBK);
    const int64_t abytes = rup(pl * Mp * Kp * 2, 1024), bbytes = rup(pl * Np * Kp * 2, 1024);
    const int64_t hdr = fp32 ? 1024 : 0;  // FP32 mode: the operands' amax words
    // Products staged and multiplied together: all seven (one pack forms
    // every operand of the level from one read of the quadrants), or, under
    // a staging budget, groups of consecutive products whose operands fit it
    // (each group's pack reads only the quadrants its operands use).
    int group = 7;
    if (stage_budget > 0 && !pre)
      group = (int)std::max<int64_t>(1, std::min<int64_t>(7, (stage_budget - hdr) / (abytes + bbytes)));
    const int ngroups = (7 + group - 1) / group;
    // prepacked (`pre`): the table level's one pack formed this level's
    // operands at pre->stg (FP32 amax words at pre->base), and counted them
    if (!pre) {
      stage_need = std::max(stage_need, hdr + group * (abytes + bbytes));
      ew_launches += ngroups * (fp32 ? 2 : 1);
    }
    for (int g0 = 0; g0 < 7 && !pre; g0 += group) {  // each group reads the quadrants its operands use
      int qa = 0, qb = 0;
      for (int q = 0; q < 4; ++q) {
        bool ua = false, ub = false;
        for (int i = g0; i < std::min(7, g0 + group); ++i) {
          ua = ua || acoef[ord[i]][q] != 0;
          ub = ub || bcoef[ord[i]][q] != 0;
        }
        qa += ua;
        qb += ub;
      }
      for (int t = 0; t < LL.n; ++t) pack_bytes += (int64_t)qa * LL.v[t].esz * hm * hk;
      for (int t = 0; t < RL.n; ++t) pack_bytes += (int64_t)qb * RL.v[t].esz * hk * hn;
      pack_bytes += std::min(group, 7 - g0) * (abytes + bbytes);
    }
    const double pflops = 2.0 * hm * hn * hk * limb_products();
    if (dry) {
      for (int g0 = 0; g0 < 7; g0 += group) queue_gemm(nullptr, {}, {}, true, std::min(group, 7 - g0) * pflops,
                                                       std::min(group, 7 - g0));
      return;
    }
    // the quadrants of every term of an operand, as pack sources
    std::vector<Rect> rdA, rdB;
    for (int t = 0; t < LL.n; ++t) rdA.push_back(rect_of(LL.v[t]));
    for (int t = 0; t < RL.n; ++t) rdB.push_back(rect_of(RL.v[t]));
    for (int g0 = 0; g0 < 7; g0 += group) {
      const int gn = std::min(group, 7 - g0);
      char *base = pre ? pre->base : next_stage();
      if (!base) return;
      uint32_t *amax = fp32 ? reinterpret_cast<uint32_t *>(base) : nullptr;
      char *stg = pre ? pre->stg : base + hdr;
      const Rect ra = rect_bytes(stg, gn * abytes), rb = rect_bytes(stg + gn * abytes, gn * bbytes);
      const Rect rh = rect_bytes(base, 8);
      if (fp32 && !pre) fp32_amax(amax, LL.v, LL.n, RL.v, RL.n);
      PackArgs pa, pb;
      pack_args(LL, RL, g0, gn, stg, amax, pa, pb);
      if (!pre) {
        std::vector<Rect> rdAB{rh};
        rdAB.insert(rdAB.end(), rdA.begin(), rdA.end());
        rdAB.insert(rdAB.end(), rdB.begin(), rdB.end());
        cudaStream_t st = op_begin(rdAB, {ra, rb});
        check(launch_pack_pair(pa, pb, mode, st), "fused pack");
        op_end();
      }
      int tiles = 0;
      for (int j = 0; j < gn; ++j) {
        const int i = ord[g0 + j];              // the product in launch slot j
        const int o = gn == 7 ? i : j;          // its pack output
        Product &pr = P.prod[j];
        if (!make_tmap(&pr.ta, pa.out[o], pl * Mp, Kp, kBM) || !make_tmap(&pr.tb, pb.out[o], pl * Np, Kp, bn)) {
          if (fail.empty()) fail = "tensor map encoding failed";
          return;
        }
        pr.ntargets = 0;
        for (int q = 0; q < 4; ++q) {
          if (!tgt[i][q]) continue;
          Target &T = pr.t[pr.ntargets++];
          T.ptr = Dq[q].ptr;
          T.ld = Dq[q].ld;
          T.sign = tgt[i][q];
          T.vec_ok = aligned16(Dq[q].ptr, Dq[q].ld);
        }
        pr.tma_epi = 1;
        for (int t = 0; t < pr.ntargets; ++t)
          if (!make_target_tmap(&pr.tmap[t], pr.t[t].ptr, hm, hn, pr.t[t].ld, fp32)) pr.tma_epi = 0;
        pr.M = (int)hm;
        pr.N = (int)hn;
        pr.Kpad = (int)Kp;
        pr.a_plane_rows = (int)Mp;
        pr.b_plane_rows = (int)Np;
        pr.tiles_m = (int)(Mp / kBM);
        pr.tiles_n = (int)(Np / bn);
        pr.tile_begin = tiles;
        pr.amax = amax;
        pr.terms_a = pa.terms;
        pr.terms_b = pb.terms;
        set_scalars(pr, alpha, false, beta, EPI_REDUCE);
        tiles += pr.tiles_m * pr.tiles_n;
      }
      P.nprod = gn;
      P.total_tiles = tiles;
      queue_gemm(&P, {ra, rb, rh}, {rect_of(D)}, true, gn * pflops, gn);
    }
  }
}

// ------------------------------------------------------------- recursion
void Exec::call(Kind k, Scalar alpha, bool acc, Scalar beta, View L, View R, View D, int depth, const Arena &ar) {
  if (!ok()) return;
  const int64_t m = L.rows, kk = L.cols, n = R.cols;
  if (depth <= 0 || m < 2 || kk < 2 || n < 2) {
    leaf(alpha, acc, beta, L, R, D);
    return;
  }
  if (m % 2 || kk % 2 || n % 2) {
    peel(k, alpha, acc, beta, L, R, D, depth, ar);
    return;
  }
  if (fused && depth == 1) {
    fused_level(alpha, acc, beta, Lin::of(L), Lin::of(R), D);
    return;
  }
  table(k, alpha, acc, beta, L, R, D, depth, ar);
}

// Dynamic peeling of odd dimensions (the paper leaves "peeling or padding"
// open, Sections 7.1 and 8): with m' = m - m%2, k' = k - k%2, n' = n - n%2,
//   C[m', :]    <- alpha A[m', :] B            (+ beta C[m', :])   last row
//   C[:m', n']  <- alpha A[:m', :] B[:, n']    (+ beta C[:m', n'])  last column
//   C[:m', :n'] <- the schedule on the even core A[:m', :k'] B[:k', :n']
//   C[:m', :n'] += alpha A[:m', k'] B[k', :n']                   rank-1 for odd k
// The row and column products run first because an overwriting schedule
// may destroy the core of A and B; the rank-1 term only reads the peeled
// column of A and row of B, which no schedule on the core touches.
void Exec::peel(Kind k, Scalar alpha, bool acc, Scalar beta, View L, View R, View D, int depth, const Arena &ar) {
  const int64_t m = L.rows, kk = L.cols, n = R.cols;
  const int64_t m2 = m - m % 2, k2 = kk - kk % 2, n2 = n - n % 2;
  if (m2 < m) leaf(alpha, acc, beta, L.sub(m2, 0, 1, kk), R, D.sub(m2, 0, 1, n));
  if (n2 < n) leaf(alpha, acc, beta, L.sub(0, 0, m2, kk), R.sub(0, n2, kk, 1), D.sub(0, n2, m2, 1));
  call(k, alpha, acc, beta, L.sub(0, 0, m2, k2), R.sub(0, 0, k2, n2), D.sub(0, 0, m2, n2), depth, ar);
  if (k2 < kk) leaf(alpha, true, one(), L.sub(0, k2, m2, 1), R.sub(k2, 0, 1, n2), D.sub(0, 0, m2, n2));
}

void Exec::table(Kind k, Scalar alpha, bool acc, Scalar beta, View L, View R, View D, int depth,
                 const Arena &ar) {
  const KindInfo &K = info(k);
  const Range nv(!dry, K.name, L.rows, L.cols, R.cols, depth);
  const int64_t hm = L.rows / 2, hk = L.cols / 2, hn = R.cols / 2;
  auto dims = [&](Shape s, int64_t &r, int64_t &c) {
    r = s == SH_B ? hk : hm;
    c = s == SH_A ? hk : hn;
  };
  // bounding box of every temporary over the values the table stores there
  int64_t tr[3] = {0, 0, 0}, tc[3] = {0, 0, 0};
  for (const Row &row : *K.table) {
    if (row.dst >= LX && row.dst <= LZ) {
      int64_t r, c;
      dims(row.op == OP_MUL ? SH_C : row.shape, r, c);
      const int t = row.dst - LX;
      tr[t] = std::max(tr[t], r);
      tc[t] = std::max(tc[t], c);
    }
  }
  View tmp[3];
  Arena sub = ar;
  const int64_t mark_top = ws_top, mark_elems = tmp_elems;
  if (ar.carve) {
    const View &g = ar.region;
    View qd[3] = {g.quad(0, 0), g.quad(0, 1), g.quad(1, 0)};
    int used = 0;
    for (int t = 0; t < 3; ++t) {
      if (!tr[t]) continue;
      if (tr[t] > qd[used].rows || tc[t] > qd[used].cols) {
        if (fail.empty()) fail = "temporary does not fit in the carved scratch block";
        return;
      }
      tmp[t] = qd[used++].sub(0, 0, tr[t], tc[t]);
    }
    sub.carve = true;
    sub.region = g.quad(1, 1);
  } else {
    for (int t = 0; t < 3; ++t)
      if (tr[t]) tmp[t] = alloc_tmp(tr[t], tc[t]);
  }
  View loc[NLOC];
  const View Lq[4] = {L.quad(0, 0), L.quad(0, 1), L.quad(1, 0), L.quad(1, 1)};
  const View Rq[4] = {R.quad(0, 0), R.quad(0, 1), R.quad(1, 0), R.quad(1, 1)};
  const View Dq[4] = {D.quad(0, 0), D.quad(0, 1), D.quad(1, 0), D.quad(1, 1)};
  for (int q = 0; q < 4; ++q) {
    loc[A11 + q] = Lq[q];
    loc[B11 + q] = Rq[q];
    loc[C11 + q] = Dq[q];
  }
  loc[LX] = tmp[0];
  loc[LY] = tmp[1];
  loc[LZ] = tmp[2];
  // 16-bit temporaries.  Over Z/pZ (p < 2^16) a value a row writes into a
  // temporary and that is an operand of a product (an S or T value, never
  // a C-shaped one) is stored as 16-bit [0, p) in the temporary's storage,
  // halving its traffic.  Only where every product of this level is a fused
  // level: a table call below could overwrite its operand blocks with
  // C-shaped values (Tables 3-8), which need 32 bits.
  const bool narrow_ok = !fp32 && !simt && fuses(hm, hk, hn, depth - 1);
  bool nar[NLOC] = {};  // the value a temporary holds is stored as 16-bit
  auto at_as = [&](Loc l, Shape s, bool narrow) -> View {
    int64_t r, c;
    dims(s, r, c);
    const View &v = loc[l];
    if (r > v.rows || c > v.cols) {
      if (fail.empty()) fail = std::string(K.name) + ": value does not fit its location (shape precondition)";
      return v;
    }
    return narrow ? v.narrow().sub(0, 0, r, c) : v.sub(0, 0, r, c);
  };
  auto at = [&](Loc l, Shape s) -> View { return at_as(l, s, nar[l]); };
  // representation of a new value of shape s written into l
  auto narrow_for = [&](Loc l, Shape s) { return narrow_ok && (l == LX || l == LY || l == LZ) && s != SH_C; };
  auto coef = [&](Coef c) -> Scalar {
    switch (c) {
      case CF_ONE: return one();
      case CF_NEG: return neg(one());
      case CF_ALPHA: return alpha;
      case CF_NALPHA: return neg(alpha);
      case CF_BETA: return beta;
      case CF_NBETA: return neg(beta);
    }
    return one();
  };
  // Pre-additions kept symbolic.  When every product of this level is a
  // fused level, a row that writes a signed sum of operand quadrants into a
  // temporary, or into a block of C (searched schedules park S and T values
  // there while C is dead), only records the sum (a Lin); the fused level
  // forms it while packing.  A recorded sum is written out before any other
  // kind of row reads its location, and before any row writes a block it
  // refers to, so every value the table reads is the one its rows define;
  // a sum still recorded in C when the table ends is written out.  Only for
  // quadrants above kVirtMinBytes: smaller blocks stay in L2 between an
  // addition and its reader, and re-reading several terms in the pack then
  // costs more than the addition saves.
  // With one pack for the whole level (below) every sub-block is read once,
  // so the sums are kept symbolic down to kLevelPackMinBytes quadrants.
  constexpr int64_t kVirtMinBytes = 32ll << 20, kLevelPackMinBytes = 4ll << 20;
  const bool fuses_below = !simt && fuses(hm, hk, hn, depth - 1);
  bool virt = fuses_below && 4 * hm * hk >= kVirtMinBytes && 4 * hk * hn >= kVirtMinBytes;
  const bool level_pack_size = fuses_below && 4 * hm * hk >= kLevelPackMinBytes && 4 * hk * hn >= kLevelPackMinBytes;
  Lin sym[NLOC];
  View symdst[NLOC];
  bool has[NLOC] = {};
  bool dirty[NLOC] = {};  // written by a row (not a recorded sum) in this call
  auto is_tmp = [](Loc l) { return l == LX || l == LY || l == LZ; };
  auto sym_dst = [&](Loc l) { return is_tmp(l) || (l >= C11 && l <= C22); };  // may hold a recorded sum
  auto operand_loc = [](Loc l) { return l >= A11 && l <= B22; };
  auto operand_quad = [](Loc l, Shape sh) {
    return (sh == SH_A && l >= A11 && l <= A22) || (sh == SH_B && l >= B11 && l <= B22);
  };
  auto sgn = [&](int v) { return v > 0 ? one() : neg(one()); };
  auto materialize = [&](Loc l) {
    if (!has[l]) return;
    has[l] = false;
    dirty[l] = true;
    const Lin &v = sym[l];
    const View &d = symdst[l];
    if (v.n == 1) {
      add(d, v.v[0], v.v[0], sgn(v.s[0]), Scalar{});
      return;
    }
    add(d, v.v[0], v.v[1], sgn(v.s[0]), sgn(v.s[1]));
    for (int t = 2; t < v.n; ++t) add(d, d, v.v[t], one(), sgn(v.s[t]));
  };
  auto before_write = [&](const View &w) {
    const Rect rw = rect_of(w);
    for (int li = 0; li < NLOC; ++li) {
      const Loc l = (Loc)li;
      if (!has[l]) continue;
      for (int t = 0; t < sym[l].n; ++t)
        if (overlaps(rect_of(sym[l].v[t]), rw)) {
          materialize(l);
          break;
        }
    }
  };
  auto same = [](const View &x, const View &y) {
    return x.ptr == y.ptr && x.ld == y.ld && x.rows == y.rows && x.cols == y.cols && x.esz == y.esz;
  };
  // c1 x + c2 y as a Lin of at most kMaxTerm unit-coefficient terms
  auto compose = [&](const Lin &x, int c1, const Lin &y, int c2, Lin &r) {
    r = Lin();
    int acc[2 * kMaxTerm];
    View vs[2 * kMaxTerm];
    int n = 0;
    auto put = [&](const Lin &z, int c) {
      for (int t = 0; t < z.n; ++t) {
        int j = 0;
        while (j < n && !same(vs[j], z.v[t])) ++j;
        if (j == n) {
          vs[n] = z.v[t];
          acc[n++] = 0;
        }
        acc[j] += c * z.s[t];
      }
    };
    put(x, c1);
    put(y, c2);
    for (int j = 0; j < n; ++j) {
      if (acc[j] == 0) continue;
      if (acc[j] != 1 && acc[j] != -1) return false;
      if (r.n == kMaxTerm) return false;
      r.v[r.n] = vs[j];
      r.s[r.n++] = (int8_t)acc[j];
    }
    return r.n > 0;
  };
  // One pack for every fused level of this table level.  When each product
  // row's operands are signed sums of operand quadrants that no row
  // overwrites (found by replaying the rows' symbolic sums, issuing
  // nothing), the seven levels' 49 operands per side are formed in one
  // pass that reads each sub-block of A and B once, instead of one pack per
  // level re-reading the quadrants of every term (Table 9 reads 14 per
  // side).  It stages all 49 operand pairs at once.
  constexpr int64_t kLevelPackMaxBytes = 32ll << 30;
  Prepacked pre[7] = {};
  bool prepacked = false;
  Lin pla[7], plb[7];
  if (level_pack_size && stage_budget == 0 && level_pack_ok) {
    int nmul = 0;
    bool okp = true;
    bool hs[NLOC] = {}, dirty[NLOC] = {};
    Lin ss[NLOC];
    // an operand quadrant is a term only while it holds its input value
    auto operand = [&](Loc l, Shape sh, Lin &out) {
      if (hs[l]) {
        out = ss[l];
        return true;
      }
      if (!operand_quad(l, sh) || dirty[l]) return false;
      out = Lin::of(at(l, sh));
      return true;
    };
    // a row writes location l (shape sh): a recorded sum with a term there
    // would have to be written out first
    auto written = [&](Loc l, Shape sh) {
      dirty[l] = true;
      hs[l] = false;
      const Rect rw = rect_of(at(l, sh));
      for (int li = 0; li < NLOC; ++li)
        for (int t = 0; hs[li] && t < ss[li].n; ++t)
          if (overlaps(rect_of(ss[li].v[t]), rw)) okp = false;
    };
    for (const Row &row : *K.table) {
      if (!okp) break;
      if (row.op == OP_ADD) {
        const bool unit = (row.c1 == CF_ONE || row.c1 == CF_NEG) && (row.c2 == CF_ONE || row.c2 == CF_NEG);
        Lin x, y, r;
        if (unit && (sym_dst(row.dst) || operand_loc(row.dst)) && row.shape != SH_C && operand(row.s1, row.shape, x) &&
            operand(row.s2, row.shape, y) && compose(x, row.c1 == CF_ONE ? 1 : -1, y, row.c2 == CF_ONE ? 1 : -1, r)) {
          ss[row.dst] = r;
          hs[row.dst] = true;
          continue;
        }
        okp = !hs[row.s1] && !hs[row.s2];  // a recorded sum would be written out
        written(row.dst, row.shape);
      } else if (row.op == OP_COPY) {
        okp = !hs[row.s1];
        written(row.dst, row.shape);
      } else {
        okp = nmul < 7 && operand(row.s1, SH_A, pla[nmul]) && operand(row.s2, SH_B, plb[nmul]);
        ++nmul;
        if (okp) written(row.dst, SH_C);
      }
    }
    // each level's operand over the four operand quadrants of its side
    int8_t qc[2][7][4] = {};
    for (int j = 0; j < nmul && okp; ++j)
      for (int side = 0; side < 2 && okp; ++side) {
        const Lin &lj = side ? plb[j] : pla[j];
        const View *quads = side ? Rq : Lq;
        for (int t = 0; t < lj.n && okp; ++t) {
          int Q = 0;
          while (Q < 4 && !same(lj.v[t], quads[Q])) ++Q;
          okp = Q < 4 && qc[side][j][Q] == 0;
          if (okp) qc[side][j][Q] = lj.s[t];
        }
      }
    int64_t abytes = 0, bbytes = 0;
    if (okp && nmul == 7) level_bytes(pla[0].shape(), plb[0].shape(), abytes, bbytes);
    const int64_t hdr = fp32 ? 1024 : 0, per = 7 * (abytes + bbytes);
    if (okp && nmul == 7 && hdr + 7 * per <= kLevelPackMaxBytes) {
      prepacked = true;
      virt = true;
      ++level_packs;
      stage_need = std::max(stage_need, hdr + 7 * per);
      ew_launches += fp32 ? 3 : 2;
      pack_bytes += 4 * (L.rows * L.cols + R.rows * R.cols) + 7 * per;
      level_pack_bytes += 4 * (L.rows * L.cols + R.rows * R.cols) + 7 * per;
      if (!dry) {
        char *base = next_stage();
        if (!base) return;
        uint32_t *amax = fp32 ? reinterpret_cast<uint32_t *>(base) : nullptr;
        if (fp32) fp32_amax(amax, Lq, 4, Rq, 4);
        PackLevel PL;
        std::memset(&PL, 0, sizeof(PL));
        PL.n = 7;
        for (int side = 0; side < 2; ++side)
          for (int Q = 0; Q < 4; ++Q) {
            const View &qd = side ? Rq[Q] : Lq[Q];
            for (int q = 0; q < 4; ++q) PL.src[side][Q][q] = qd.quad(q / 2, q % 2).ptr;
            PL.ld[side][Q] = qd.ld;
            PL.esz[side][Q] = (int8_t)qd.esz;
          }
        for (int j = 0; j < 7; ++j) {
          pre[j].base = base;
          pre[j].stg = base + hdr + j * per;
          PackArgs pa, pb;  // extents, scale terms and output places of level j
          pack_args(pla[j], plb[j], 0, 7, pre[j].stg, amax, pa, pb);
          PL.out[0][j] = pa.out[0];
          PL.out[1][j] = pb.out[0];
          PL.terms[0][j] = pa.terms;
          PL.terms[1][j] = pb.terms;
          for (int side = 0; side < 2; ++side)
            for (int Q = 0; Q < 4; ++Q) PL.coef[side][j][Q] = qc[side][j][Q];
          if (j == 0) {
            PL.rows[0] = pa.rows;
            PL.cols[0] = pa.cols;
            PL.prow_pad[0] = pa.prow_pad;
            PL.pcol_pad[0] = pa.pcol_pad;
            PL.rows[1] = pb.rows;
            PL.cols[1] = pb.cols;
            PL.prow_pad[1] = pb.prow_pad;
            PL.pcol_pad[1] = pb.pcol_pad;
            PL.p = pa.p;
            PL.barrett = pa.barrett;
          }
        }
        PL.ostride[0] = abytes / 2;
        PL.ostride[1] = bbytes / 2;
        PL.amax = amax;
        // the two sides write disjoint parts of every level's staging, so
        // the dataflow capture can run them at once
        for (int side = 0; side < 2; ++side) {
          std::vector<Rect> wr;
          for (int j = 0; j < 7; ++j)
            wr.push_back(side ? rect_bytes(pre[j].stg + 7 * abytes, 7 * bbytes) : rect_bytes(pre[j].stg, 7 * abytes));
          cudaStream_t st = op_begin({side ? rect_of(R) : rect_of(L), rect_bytes(base, 8)}, wr);
          check(launch_pack_level(PL, side, mode, st), "level pack");
          op_end();
        }
      }
    }
  }
  // With one pass packing the level, operand quadrants are read before any
  // row runs: a quadrant a row has written (dirty) is no longer a term, and
  // sums may be recorded in operand quadrants too (in-place tables park
  // them there; the blocks keep their input values).
  auto quad_term = [&](Loc l, Shape sh) { return operand_quad(l, sh) && !(prepacked && dirty[l]); };
  int jmul = 0;
  auto same_lin = [&](const Lin &x, const Lin &y) {
    if (x.n != y.n) return false;
    for (int t = 0; t < x.n; ++t)
      if (!same(x.v[t], y.v[t]) || x.s[t] != y.s[t]) return false;
    return true;
  };
  for (const Row &row : *K.table) {
    if (!ok()) return;
    if (row.op == OP_ADD) {
      const View a = at(row.s1, row.shape), b = at(row.s2, row.shape);
      const bool nd = narrow_for(row.dst, row.shape);
      const View d = at_as(row.dst, row.shape, nd);
      nar[row.dst] = nd;
      bool recorded = false;
      const bool unit = (row.c1 == CF_ONE || row.c1 == CF_NEG) && (row.c2 == CF_ONE || row.c2 == CF_NEG);
      if (virt && unit && (sym_dst(row.dst) || (prepacked && operand_loc(row.dst))) && row.shape != SH_C &&
          (has[row.s1] || quad_term(row.s1, row.shape)) && (has[row.s2] || quad_term(row.s2, row.shape))) {
        Lin r;
        const Lin x = has[row.s1] ? sym[row.s1] : Lin::of(a), y = has[row.s2] ? sym[row.s2] : Lin::of(b);
        if (compose(x, row.c1 == CF_ONE ? 1 : -1, y, row.c2 == CF_ONE ? 1 : -1, r)) {
          sym[row.dst] = r;
          symdst[row.dst] = d;
          has[row.dst] = true;
          recorded = true;
        }
      }
      if (!recorded) {
        materialize(row.s1);
        materialize(row.s2);
        before_write(d);
        has[row.dst] = false;
        dirty[row.dst] = true;
        add(d, a, b, coef(row.c1), coef(row.c2));
      }
    } else if (row.op == OP_COPY) {
      const View src = at(row.s1, row.shape);
      const bool nd = narrow_for(row.dst, row.shape);
      View d = at_as(row.dst, row.shape, nd);
      nar[row.dst] = nd;
      materialize(row.s1);
      before_write(d);
      has[row.dst] = false;
      dirty[row.dst] = true;
      ++ew_launches;
      add_elems += d.rows * d.cols;
      {  // a copy keeps the source's representatives
        bool src_lazy = false;
        for (const View &x : lazy_views)
          if (overlaps(rect_of(x), rect_of(src))) src_lazy = true;
        if (src_lazy)
          mark_lazy(d);
        else
          mark_canonical(d);
      }
      if (!dry) {
        cudaStream_t st = op_begin({rect_of(src)}, {rect_of(d)});
        check(launch_copy(d, src, p, st), "copy");
        op_end();
      }
    } else {
      const KindInfo &S = info(row.kind);
      const View a = at(row.s1, SH_A), b = at(row.s2, SH_B);
      nar[row.dst] = false;  // a product is C-shaped: 32-bit
      const View d = at(row.dst, SH_C);
      const Scalar al = coef(row.c1), be = row.acc ? coef(row.cacc) : Scalar{};
      before_write(d);
      dirty[row.dst] = true;
      if (virt) {
        // a fused level reads its operands (symbolic or not) and writes d
        const Lin la = has[row.s1] ? sym[row.s1] : Lin::of(a), lb = has[row.s2] ? sym[row.s2] : Lin::of(b);
        has[row.dst] = false;
        if (prepacked && (jmul >= 7 || !same_lin(la, pla[jmul]) || !same_lin(lb, plb[jmul]))) {
          if (fail.empty()) fail = "level pack: operands differ from the replay";
          return;
        }
        fused_level(al, S.accumulate, be, la, lb, d, prepacked ? &pre[jmul++] : nullptr);
      } else {
        has[row.dst] = false;
        call(row.kind, al, S.accumulate, be, a, b, d, depth - 1, sub);
      }
    }
  }
  // Temporaries are dead here; a sum still recorded in C is written out,
  // and so is one recorded in an operand block that a row wrote earlier
  // (the block holds neither its input nor the value the rows define,
  // which a table that restores the block relies on).  An operand block
  // never written keeps its input value.
  for (int li = C11; li <= C22 && ok(); ++li) materialize((Loc)li);
  for (int li = A11; li <= B22 && ok(); ++li)
    if (dirty[li]) materialize((Loc)li);
  if (!ar.carve) {
    ws_top = mark_top;
    tmp_elems = mark_elems;
  }
}

// Algorithm 2: C11, C12, C21 by n/2 x n/2 Winograd products over the 2k/n
// block columns (Table 1 first, then the accumulating schedule), all
// temporaries carved from C22; then C22 recursively; classical base case.
void Exec::ipmm(View L, View R, View D, int depth, int64_t cutoff, Kind acc_kind) {
  if (!ok()) return;
  const Range nv(!dry, "IPMM", L.rows, L.cols, R.cols, depth);
  const int64_t n = D.rows, k = L.cols;
  if (n <= cutoff || n % 2 || n < 2 || k % (n / 2)) {
    leaf(one(), false, Scalar{}, L, R, D);
    return;
  }
  const int64_t h = n / 2, nb = k / h;
  int d = 0;
  for (int64_t s = h; d < depth && s % 2 == 0 && s >= 2; s /= 2) ++d;
  Arena ar;
  ar.carve = true;
  ar.region = D.quad(1, 1);
  const View Cq[3] = {D.quad(0, 0), D.quad(0, 1), D.quad(1, 0)};
  const int ai[3] = {0, 0, 1}, bj[3] = {0, 1, 0};
  for (int i = 0; i < nb; ++i) {
    for (int c = 0; c < 3; ++c) {
      View Ab = L.sub(ai[c] * h, i * h, h, h);
      View Bb = R.sub(i * h, bj[c] * h, h, h);
      if (i == 0)
        call(K_T1, one(), false, Scalar{}, Ab, Bb, Cq[c], d, ar);
      else
        call(acc_kind, one(), true, one(), Ab, Bb, Cq[c], d, ar);
    }
  }
  ipmm(L.sub(h, 0, h, k), R.sub(0, h, k, h), D.quad(1, 1), depth, cutoff, acc_kind);
}

// Algorithm 1 (IP0vMM, Section 5.3): C (m x n) is split into n x n row
// blocks C_1..C_m0, A into n x n blocks A_ij, B into n x n row blocks B_j.
//   C_1 <- alpha A_11 B_1                    Table 1, temporaries in C_2
//   C_i <- alpha A_i1 B_1        i >= 2      Table 4 (overwrites A_i1),
//   C_i <- alpha A_ij B_j + C_i  j >= 2      Table 2,
// the last two with every temporary carved from A_11, which is dead once
// C_1 is formed.  A is overwritten; B is read-only; no extra memory.
void Exec::ip0vmm(Scalar alpha, View L, View R, View D, int depth) {
  if (!ok()) return;
  const Range nv(!dry, "IP0vMM", L.rows, L.cols, R.cols, depth);
  const int64_t m = L.rows, k = L.cols, n = R.cols;
  const int64_t m0 = m / n, k0 = k / n;
  int d = 0;
  for (int64_t s = n; d < depth && s % 2 == 0 && s >= 2; s /= 2) ++d;
  Arena first;
  first.carve = true;
  first.region = D.sub(n, 0, n, n);
  call(K_T1, alpha, false, Scalar{}, L.sub(0, 0, n, n), R.sub(0, 0, n, n), D.sub(0, 0, n, n), d, first);
  Arena rest;
  rest.carve = true;
  rest.region = L.sub(0, 0, n, n);
  for (int64_t i = 1; i < m0; ++i)
    call(K_OVL, alpha, false, Scalar{}, L.sub(i * n, 0, n, n), R.sub(0, 0, n, n), D.sub(i * n, 0, n, n), d, rest);
  for (int64_t j = 1; j < k0; ++j)
    for (int64_t i = 0; i < m0; ++i)
      call(K_T2, alpha, true, one(), L.sub(i * n, j * n, n, n), R.sub(j * n, 0, n, n), D.sub(i * n, 0, n, n), d,
           rest);
}

// Section 7.2: D (m x n) in t x t blocks D_ij of (m/t) x (n/t); each is
//   D_ij <- alpha A_i1 B_1j + beta D_ij,  then  D_ij <- alpha A_il B_lj + D_ij
// for l = 2..t, every call by the accumulating schedule acc_kind (Table 2,
// or Table 9) at `depth` levels.  The calls run one after the other, so the
// temporaries of one block call are all the extra memory: (n/t)^2 with
// Table 2, 2 (n/t)^2 / 3 with Table 9.
void Exec::tblock(Scalar alpha, Scalar beta, View L, View R, View D, int t, int depth, Kind acc_kind) {
  if (!ok()) return;
  const Range nv(!dry, "t-blocks", L.rows, L.cols, R.cols, depth);
  const int64_t mt = L.rows / t, kt = L.cols / t, nt = R.cols / t;
  for (int i = 0; i < t; ++i)
    for (int j = 0; j < t; ++j)
      for (int l = 0; l < t; ++l)
        call(acc_kind, alpha, true, l == 0 ? beta : one(), L.sub(i * mt, l * kt, mt, kt), R.sub(l * kt, j * nt, kt, nt),
             D.sub(i * mt, j * nt, mt, nt), depth, Arena{});
}

void Exec::copy_in(View dv, const char *host, int64_t hld, const Rect &token) {
  if (dry || dv.rows == 0 || dv.cols == 0) return;
  cudaStream_t st = op_begin({token}, {rect_of(dv), token}, true);
  check(cudaMemcpy2DAsync(dv.ptr, 4 * dv.ld, host, 4 * hld, 4 * dv.cols, dv.rows, cudaMemcpyHostToDevice, st),
        "copy to device");
  op_end();
}

void Exec::copy_out(char *host, int64_t hld, View dv, const Rect &token) {
  if (dry || dv.rows == 0 || dv.cols == 0) return;
  cudaStream_t st = op_begin({rect_of(dv), token}, {token}, true);
  check(cudaMemcpy2DAsync(host, 4 * hld, dv.ptr, 4 * dv.ld, 4 * dv.cols, dv.rows, cudaMemcpyDeviceToHost, st),
        "copy to host");
  op_end();
}

void Exec::canon(View v) {
  ++ew_launches;
  mark_canonical(v);
  if (dry || v.rows == 0 || v.cols == 0) return;
  cudaStream_t st = op_begin({}, {rect_of(v)});
  check(launch_canon_modp(v, p, st), "canonical pass");
  op_end();
}

}  // namespace swmm
