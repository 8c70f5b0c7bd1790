// Schedule tables of the paper as data, and the recursive executor that
// lowers them to kernel launches.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "swmm_internal.h"
#include "swmm_search.h"

namespace swmm {

// Storage locations named in the tables' "loc." column.
enum Loc : int8_t {
  A11, A12, A21, A22, B11, B12, B21, B22, C11, C12, C21, C22, LX, LY, LZ, NLOC
};

// Kinds of (recursive) calls: the tables themselves plus the classical leaf.
enum Kind : int8_t {
  K_T1,    // Table 1  (Douglas et al.)       C <- aAB
  K_T2,    // Table 2  (Huss-Lederman et al.) C <- aAB + bC
  K_IP,    // Table 3                           C <- aAB, overwrites A, B
  K_OVL,   // Table 4                           C <- aAB, overwrites A
  K_OVLM,  // Section 5.1 variant of Table 4, overwrites A11, A21
  K_OVR,   // Table 5                           C <- aAB, overwrites B
  K_ACLR,  // Table 6                           C <- aAB + bC, overwrites A, B
  K_ACCR,  // Table 7                           C <- aAB + bC, overwrites B
  K_ACR,   // Table 8                           C <- aAB + bC, overwrites B12, B21
  K_ACC,   // Table 9                           C <- aAB + bC, read-only
  NKIND,
  K_CUSTOM  // a schedule given to the handle (swmm_set_schedule), not a table
};

// Coefficients appearing in the tables.
enum Coef : int8_t { CF_ONE, CF_NEG, CF_ALPHA, CF_NALPHA, CF_BETA, CF_NBETA };

// Shape class of a value: A-shaped (S), B-shaped (T) or C-shaped (P, U, Z, W).
enum Shape : int8_t { SH_A, SH_B, SH_C };

enum RowOp : int8_t { OP_ADD, OP_MUL, OP_COPY };

struct Row {
  RowOp op;
  Loc dst;
  Shape shape;   // of the value written (ADD / COPY)
  Loc s1, s2;    // ADD: operands; MUL: left, right; COPY: s1
  Coef c1, c2;   // ADD coefficients; MUL: c1 = alpha coefficient
  Kind kind;     // MUL: kind of the recursive call
  bool acc;      // MUL: accumulates into dst
  Coef cacc;     // MUL: coefficient of the value held by dst
};

struct KindInfo {
  const char *name;
  const std::vector<Row> *table;
  bool accumulate;
  bool square;
};

const KindInfo &kind_info(Kind k);  // k < NKIND

// A one-level schedule in the rows of include/swmm_search.h, checked by
// replaying it in the pebble game and lowered to executor rows (recursive
// calls of the schedule itself become K_CUSTOM).  False, with the reason
// in *err, when a row is not a legal move or the results do not end in
// place.
struct CustomSchedule {
  std::vector<Row> rows;
  bool accumulate = false;
  uint32_t preserve = 0;  // bit b: block b (A11..B22) is kept
  int temps = 0;          // temporaries the rows use
};
bool lower_schedule(const swmm_search_spec &spec, const swmm_search_row *rows, int nrows, CustomSchedule *out,
                    std::string *err);

}  // namespace swmm
