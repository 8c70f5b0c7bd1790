// Host checks of the dependency rectangles that order captured launches
// (flow.h): views of one root with one leading dimension are compared
// exactly, anything else conservatively by address span.
#include <cstdio>
#include <cstdlib>

#include "flow.h"

using swmm::overlaps;
using swmm::Rect;
using swmm::rect_bytes;
using swmm::rect_of;
using swmm::View;

static int failures = 0;
#define EXPECT(cond)                                                \
  do {                                                              \
    if (!(cond)) {                                                  \
      std::printf("FAILED line %d: %s\n", __LINE__, #cond);      \
      ++failures;                                                   \
    }                                                               \
  } while (0)

int main() {
  static char buf[1 << 22];
  View M;  // an 8 x 8 matrix of 4-byte elements, leading dimension 10
  M.ptr = buf;
  M.rows = 8;
  M.cols = 8;
  M.ld = 10;
  const View q[4] = {M.quad(0, 0), M.quad(0, 1), M.quad(1, 0), M.quad(1, 1)};
  // quadrants interleave in memory but never share an element
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) EXPECT(overlaps(rect_of(q[i]), rect_of(q[j])) == (i == j));
  // a quadrant of a quadrant lies in its parent only
  const View qq = q[3].quad(1, 0);
  EXPECT(overlaps(rect_of(qq), rect_of(q[3])));
  EXPECT(!overlaps(rect_of(qq), rect_of(q[2])));
  EXPECT(!overlaps(rect_of(qq), rect_of(q[1])));
  // the exact coordinates of a sub-view
  const Rect r = rect_of(M.sub(3, 5, 2, 2));
  EXPECT(r.r0 == 3 && r.c0 == 5 && r.rows == 2 && r.cols == 2 && r.base == buf);
  // one row against one column
  EXPECT(overlaps(rect_of(M.sub(7, 0, 1, 8)), rect_of(M.sub(0, 7, 8, 1))));
  EXPECT(!overlaps(rect_of(M.sub(7, 0, 1, 7)), rect_of(M.sub(0, 7, 7, 1))));
  // empty views touch nothing
  EXPECT(!overlaps(rect_of(M.sub(2, 2, 0, 3)), rect_of(M)));
  // another leading dimension over the same bytes: address spans decide
  View T;
  T.ptr = buf + 4 * 10;  // starts at row 1 of M
  T.rows = 2;
  T.cols = 20;
  T.ld = 20;
  EXPECT(overlaps(rect_of(T), rect_of(q[0])));
  View far = T;
  far.ptr = buf + (1 << 21);
  EXPECT(!overlaps(rect_of(far), rect_of(M)));
  // byte ranges (operand staging)
  EXPECT(overlaps(rect_bytes(buf, 64), rect_bytes(buf + 60, 8)));
  EXPECT(!overlaps(rect_bytes(buf, 64), rect_bytes(buf + 64, 8)));
  EXPECT(overlaps(rect_bytes(buf, 40), rect_of(M)));
  EXPECT(!overlaps(rect_bytes(buf + 4 * 80, 16), rect_of(M)));
  if (failures == 0) std::printf("ok\n");
  return failures == 0 ? 0 : 1;
}
