// Dataflow ordering of one call's kernel launches over a few CUDA streams.
//
// The schedule tables are sequences of rows, but many consecutive rows touch
// disjoint blocks: the A-side and B-side pre-additions, products into
// different quadrants of C, the staging of the next leaf's operands while
// the current leaf multiplies.  While a call is captured into a CUDA graph,
// every launch declares the rectangles of memory it reads and writes; it is
// placed on one of kFlowStreams capture streams and waits (through events,
// which become graph edges) only for the earlier launches it conflicts with:
// read after write, write after read, write after write on overlapping
// memory.  Program order is kept wherever it matters, so the result is the
// one the rows compute in order; the GPU may overlap bandwidth-bound passes
// with tensor-core leaves.
//
// Vector clocks per stream keep the waits minimal: a launch skips a wait
// that an earlier wait on its stream already implies.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "swmm_internal.h"

namespace swmm {

// A rectangle of 4-byte elements of one allocation, and its address span.
struct Rect {
  const char *base = nullptr;  // root pointer of the allocation the view came from
  int64_t ld = 0, r0 = 0, c0 = 0, rows = 0, cols = 0;
  uintptr_t lo = 0, hi = 0;  // [lo, hi): bytes spanned
};
Rect rect_of(const View &v);
Rect rect_bytes(const void *p, int64_t bytes);
// Exact for two rectangles of the same root and leading dimension,
// conservative (address spans) otherwise.
bool overlaps(const Rect &a, const Rect &b);

constexpr int kFlowStreams = 4;

class Flow {
 public:
  // origin: the capturing stream (all launches are ordered after what it
  // holds so far); extra: kFlowStreams - 1 streams owned by the caller;
  // events: a pool of at least (launches + 1) events created beforehand.
  Flow(cudaStream_t origin, const cudaStream_t *extra, const std::vector<cudaEvent_t> &events);
  // Stream for the next launch, after the waits its conflicts need.  Copies
  // between host and device (dma) go to the origin stream, which kernels
  // use only to follow a predecessor that ends it, so that no kernel waits
  // behind copies it does not need.
  cudaStream_t begin(const Rect *rd, int nrd, const Rect *wr, int nwr, bool dma = false);
  // The launch announced by begin() has been issued.
  void end();
  // The origin stream waits for every launch issued so far.
  void join();
  cudaError_t error() const { return err_; }
  int64_t waits() const { return waits_; }
  int64_t launches() const { return (int64_t)ops_.size(); }

 private:
  struct Op {
    std::vector<Rect> rd, wr;
    int s = 0;
    int vc[kFlowStreams] = {0, 0, 0, 0};  // 1 + index of the latest op per stream ordered before (or = this one)
  };
  bool conflict(const Op &o, const Rect *rd, int nrd, const Rect *wr, int nwr) const;
  void check(cudaError_t e);

  cudaStream_t st_[kFlowStreams];
  bool forked_[kFlowStreams];
  int vc_[kFlowStreams][kFlowStreams];  // clock of each stream's tail
  const std::vector<cudaEvent_t> &ev_;
  std::vector<Op> ops_;
  cudaError_t err_ = cudaSuccess;
  int64_t waits_ = 0;
  bool open_ = false;
};

}  // namespace swmm
