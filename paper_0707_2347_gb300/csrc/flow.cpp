// Dataflow ordering of launches over capture streams (see flow.h).
#include "flow.h"

#include <algorithm>

namespace swmm {

Rect rect_of(const View &v) {
  Rect r;
  r.base = v.base ? v.base : v.ptr;
  // 16-bit views get their own leading dimension (twice the 32-bit one), so
  // against 32-bit views of the same root only their byte spans are compared
  r.ld = v.esz == 4 ? v.ld : -v.ld;
  const int64_t off = (int64_t)(v.ptr - r.base) / v.esz;
  r.r0 = v.ld > 0 ? off / v.ld : 0;
  r.c0 = v.ld > 0 ? off % v.ld : off;
  r.rows = v.rows;
  r.cols = v.cols;
  r.lo = (uintptr_t)v.ptr;
  r.hi = (v.rows > 0 && v.cols > 0) ? r.lo + v.esz * (uintptr_t)((v.rows - 1) * v.ld + v.cols) : r.lo;
  return r;
}

Rect rect_bytes(const void *p, int64_t bytes) {
  Rect r;
  r.base = static_cast<const char *>(p);
  r.ld = 0;  // not a 2-D view: address spans only
  r.lo = (uintptr_t)p;
  r.hi = r.lo + (uintptr_t)std::max<int64_t>(bytes, 0);
  return r;
}

bool overlaps(const Rect &a, const Rect &b) {
  if (a.lo >= a.hi || b.lo >= b.hi) return false;
  if (a.hi <= b.lo || b.hi <= a.lo) return false;
  if (a.base == b.base && a.ld == b.ld && a.ld != 0)
    return a.r0 < b.r0 + b.rows && b.r0 < a.r0 + a.rows && a.c0 < b.c0 + b.cols && b.c0 < a.c0 + a.cols;
  return true;
}

Flow::Flow(cudaStream_t origin, const cudaStream_t *extra, const std::vector<cudaEvent_t> &events) : ev_(events) {
  st_[0] = origin;
  for (int s = 1; s < kFlowStreams; ++s) st_[s] = extra[s - 1];
  for (int s = 0; s < kFlowStreams; ++s) {
    forked_[s] = s == 0;
    for (int t = 0; t < kFlowStreams; ++t) vc_[s][t] = 0;
  }
  // the other streams start after everything the origin holds (allocations)
  if (ev_.empty())
    err_ = cudaErrorInvalidValue;
  else
    check(cudaEventRecord(ev_[0], origin));
}

void Flow::check(cudaError_t e) {
  if (e != cudaSuccess && err_ == cudaSuccess) err_ = e;
}

bool Flow::conflict(const Op &o, const Rect *rd, int nrd, const Rect *wr, int nwr) const {
  for (const Rect &w : o.wr) {
    for (int i = 0; i < nrd; ++i)
      if (overlaps(w, rd[i])) return true;
    for (int i = 0; i < nwr; ++i)
      if (overlaps(w, wr[i])) return true;
  }
  for (const Rect &r : o.rd)
    for (int i = 0; i < nwr; ++i)
      if (overlaps(r, wr[i])) return true;
  return false;
}

cudaStream_t Flow::begin(const Rect *rd, int nrd, const Rect *wr, int nwr, bool dma) {
  const int j = (int)ops_.size();
  if (err_ != cudaSuccess || j + 1 >= (int)ev_.size()) {
    if (err_ == cudaSuccess) err_ = cudaErrorInvalidValue;  // event pool too small
    return st_[0];
  }
  std::vector<int> deps;  // latest first
  for (int i = j - 1; i >= 0; --i)
    if (conflict(ops_[i], rd, nrd, wr, nwr)) deps.push_back(i);
  int s;
  const int d0 = deps.empty() ? -1 : deps[0];
  if (dma) {
    s = 0;
  } else if (d0 >= 0 && vc_[ops_[d0].s][ops_[d0].s] == d0 + 1) {
    s = ops_[d0].s;  // the latest conflicting launch ends its stream: follow it
  } else {
    // no predecessor, or later unrelated launches sit behind it on its
    // stream: the kernel stream whose tail is oldest (an event orders it
    // after d0)
    s = 1;
    int best = vc_[1][1];
    for (int t = 2; t < kFlowStreams; ++t)
      if (vc_[t][t] < best) {
        best = vc_[t][t];
        s = t;
      }
  }
  if (!forked_[s]) {
    check(cudaStreamWaitEvent(st_[s], ev_[0], 0));
    forked_[s] = true;
  }
  Op op;
  op.rd.assign(rd, rd + nrd);
  op.wr.assign(wr, wr + nwr);
  op.s = s;
  for (int t = 0; t < kFlowStreams; ++t) op.vc[t] = vc_[s][t];
  for (int i : deps) {
    const Op &d = ops_[i];
    if (op.vc[d.s] >= i + 1) continue;  // already ordered before by an earlier wait
    check(cudaStreamWaitEvent(st_[s], ev_[i + 1], 0));
    ++waits_;
    for (int t = 0; t < kFlowStreams; ++t) op.vc[t] = std::max(op.vc[t], d.vc[t]);
  }
  op.vc[s] = j + 1;
  ops_.push_back(std::move(op));
  open_ = true;
  return st_[s];
}

void Flow::end() {
  if (!open_) return;
  open_ = false;
  const int j = (int)ops_.size() - 1;
  const Op &op = ops_[j];
  check(cudaEventRecord(ev_[j + 1], st_[op.s]));
  for (int t = 0; t < kFlowStreams; ++t) vc_[op.s][t] = op.vc[t];
}

void Flow::join() {
  for (int s = 1; s < kFlowStreams; ++s) {
    const int last = vc_[s][s];  // 1 + index of the stream's last launch
    if (!forked_[s] || last == 0) continue;
    // an explicit edge from every side stream's tail, even when implied, so
    // that the capture sees each branch joined
    check(cudaStreamWaitEvent(st_[0], ev_[last], 0));
    ++waits_;
    for (int t = 0; t < kFlowStreams; ++t) vc_[0][t] = std::max(vc_[0][t], vc_[s][t]);
  }
}

}  // namespace swmm
