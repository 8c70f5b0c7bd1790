/*
 * swmm_search.h - pebble-game search for the memory schedules of one
 * Winograd level (Section 4 of Boyer, Dumas, Pernet and Zhou, ISSAC 2009).
 *
 * Section 4 finds schedules such as Tables 3-5 by an exhaustive search over
 * a pebble game played on the value graph of Winograd's algorithm (Section
 * 2): a pebble is a block of memory; a value is computed when a pebble is
 * put on it (in a fresh block, or in place over an operand that is no longer
 * needed), freed when nothing needs it any more, or duplicated.  Section
 * 5.1 then states two results of that search: no in-place product C <- AB
 * overwrites fewer than four input blocks, and none overwrites only one of
 * A and B without a temporary.
 *
 * This entry point plays that game for one level of the recursion (square
 * blocks unless the spec gives the operands' relative sizes), with the
 * locations the tables use: the quadrants A11 ... C22 of
 * the caller's matrices and up to three temporaries X, Y, Z.  Values are
 * vectors over the operand blocks, the seven products P1 ... P7 and the
 * blocks of the input C; a row may compute any candidate value that is one
 * of
 *   - a block addition  w = u + c v       (c in {1, -1, beta, -beta}),
 *   - a product         w = P_i            (operands: the Section 2 sums),
 *   - an accumulation   w = +-P_i + c v    (a recursive call of an
 *                                          accumulating kind onto v),
 *   - a copy of a value into another block,
 * from the candidate values listed by swmm_search_node_name (the Section 2
 * values and, for C <- alpha AB + beta C, the intermediate values of Tables
 * 2 and 6-9).  A product is a recursive call of one of the allowed kinds:
 * the kind's contract says which operand blocks it overwrites (they hold
 * garbage afterwards), whether it accumulates, and the destination never
 * aliases an operand.  Each of the seven products is computed once.
 *
 * The search is a depth-first enumeration of the game's states (block
 * contents, values computed, products used, input blocks overwritten) with
 * a visited set and admissible bounds (rows and block additions still
 * needed, blocks that will be overwritten), so a negative answer with
 * `exhausted` set is a proof that no schedule within the spec's limits
 * exists in this model.
 *
 * No GPU is used; the library may be loaded on a host without one.
 */
#ifndef SWMM_SEARCH_H
#define SWMM_SEARCH_H

#include <stdint.h>

#include "swmm.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Locations (the tables' "loc." column). */
#define SWMM_LOC_A11 0  /* A11 A12 A21 A22 = 0..3, B11 .. B22 = 4..7, */
#define SWMM_LOC_B11 4  /* C11 .. C22 = 8..11, X Y Z = 12..14          */
#define SWMM_LOC_C11 8
#define SWMM_LOC_X 12
#define SWMM_NLOC 15

/* Row operations of a found schedule. */
#define SWMM_ROW_ADD 0  /* dst <- s1 + coef * s2 */
#define SWMM_ROW_MUL 1  /* dst <- sign * alpha * s1 * s2 (+ coef * dst if accumulate) */
#define SWMM_ROW_COPY 2 /* dst <- s1 */

/* Coefficients. */
#define SWMM_COEF_ONE 0
#define SWMM_COEF_NEG 1
#define SWMM_COEF_BETA 2
#define SWMM_COEF_NBETA 3

/* Kind of a recursive call: a schedule code of swmm.h (SWMM_T1_DHSS ...
 * SWMM_T9_ACC, SWMM_T4M_OVL) or the schedule being searched for. */
#define SWMM_SEARCH_SELF 31

typedef struct {
  int32_t accumulate;   /* 0: C <- alpha AB (C holds nothing on entry);
                           1: C <- alpha AB + beta C */
  uint32_t preserve;    /* bit b (b = location 0..7): that block of A or B
                           must hold its input value when the level ends
                           (it may be overwritten in between only if a copy
                           restores it); other input blocks may be
                           overwritten */
  int32_t temps;        /* temporaries X, Y, Z available, 0..3 */
  uint32_t kinds;       /* bit s: recursive calls may use the contract of
                           schedule code s of swmm.h (1..9, 11) or, for bit
                           SWMM_SEARCH_SELF, of the schedule searched for
                           (which overwrites the left operand when a block of
                           A is not preserved, the right one when a block of
                           B is not, and accumulates as `accumulate` says) */
  int32_t max_written;  /* at most this many of the 8 blocks of A and B may
                           be written or overwritten by a call; -1: any */
  int32_t max_copies;   /* copy rows allowed (Section 4 rule 4), >= 0; a
                           copy goes into a free block */
  int32_t recompute;    /* 1: an operand sum (S1..S4, T1..T4) may be formed
                           again (Table 9 forms T1 and T2 twice); 0: each
                           value once.  Values of C are formed once. */
  int32_t max_rows;     /* longest schedule searched, <= SWMM_SEARCH_MAX_ROWS */
  int32_t max_adds;     /* at most this many block additions (each one pass
                           over HBM at an upper level), <= 255; -1: any
                           (0 allows none) */
  int64_t max_states;   /* give up after visiting this many states (<= 0:
                           2^26) */
  uint64_t exclude;     /* bit v: candidate value v (swmm_search_node_name)
                           is never formed, to search a smaller graph */
  int32_t m, k, n;      /* relative sizes of the operands (A m x k, B k x n,
                           C m x n; Section 5.3): a value goes only into a
                           block it fits (temporaries hold any), the square
                           tables (4-7, 9) are not called unless m = k = n,
                           Table 3 only when k = n <= m.  0, 0, 0: square */
  int32_t order;        /* SWMM_ORDER_*: which values the search tries to
                           form first.  The answer to "does a schedule
                           exist" does not depend on it; which schedule is
                           found first and how fast does */
} swmm_search_spec;

#define SWMM_ORDER_ASCENDING 0  /* candidate list order (operand sums first) */
#define SWMM_ORDER_DESCENDING 1 /* results and sums of products first */
#define SWMM_ORDER_PORTFOLIO 2  /* both in turn, budgets growing fourfold
                                   (2^16, 2^16, 2^18, 2^18, ... states) */

#define SWMM_SEARCH_MAX_ROWS 64

typedef struct {
  int32_t op;         /* SWMM_ROW_* */
  int32_t dst;        /* location written */
  int32_t s1, s2;     /* ADD: operand locations; MUL: left and right
                         operand locations; COPY: s1 is the source */
  int32_t coef;       /* ADD: coefficient of s2; MUL with accumulate: of the
                         value dst held; SWMM_COEF_* */
  int32_t accumulate; /* MUL: 1 if dst's previous value is accumulated */
  int32_t sign;       /* MUL: +1 or -1 (applied to alpha) */
  int32_t kind;       /* MUL: kind of the recursive call */
  int32_t node;       /* value written (swmm_search_node_name) */
} swmm_search_row;

typedef struct {
  int32_t found;      /* 1: rows hold a schedule meeting the spec */
  int32_t exhausted;  /* 1: every state was visited: with found == 0, no
                         schedule of at most max_rows rows (and max_adds
                         additions) exists in this model */
  int32_t nrows;      /* rows written */
  int32_t written;    /* input blocks the schedule writes or overwrites */
  int32_t temps_used; /* temporaries the schedule writes */
  int64_t states;     /* states visited */
} swmm_search_result;

/* Search for a schedule meeting `spec`.  rows: host array of max_rows_out
 * entries (the schedule, in order, when found).  Returns SWMM_OK (whether
 * or not a schedule was found: see res), SWMM_EINVAL for a bad spec or a
 * NULL pointer, SWMM_ENOMEM when the visited set cannot grow. */
int swmm_schedule_search(const swmm_search_spec *spec, swmm_search_row *rows, int32_t max_rows_out,
                         swmm_search_result *res);

/* Play the rows of a given schedule (op, dst, s1, s2, coef, accumulate,
 * sign, kind; node is ignored) under the rules above and the contract of
 * `spec`: each row must be a legal move (operands present, the value it
 * forms a candidate, a product one of the seven with the Section 2 operands
 * and not computed before, the call's kind allowed, its destination not an
 * operand), and at the end the results and the preserved blocks must be in
 * place.  Writes each row's value into rows[i].node.  res->found is 1 when
 * the schedule is legal and complete; res->nrows is the index of the first
 * illegal row (nrows when every row is legal); written and temps_used count
 * the blocks it writes.  Returns SWMM_OK, or SWMM_EINVAL for a bad spec or
 * pointer. */
int swmm_schedule_check(const swmm_search_spec *spec, swmm_search_row *rows, int32_t nrows,
                        swmm_search_result *res);

/* Give handle h a schedule of its own: `rows` (nrows of them) are checked
 * as swmm_schedule_check does under `spec` and kept by the handle; calls
 * with opts->sched == SWMM_CUSTOM then run them at every Winograd level,
 * with rows whose kind is SWMM_SEARCH_SELF recursing into the same
 * schedule and other kinds into the paper's tables (the last level is the
 * fused tensor-core level, as for the tables).  The operands must be
 * square; the entry point follows the contract (see SWMM_CUSTOM).  Blocks
 * of A and B the spec does not preserve may come back overwritten.  Cached
 * graphs of earlier calls are dropped (after the handle's streams finish
 * the work already issued; SWMM_ECUDA if that wait fails).  Returns SWMM_OK, or SWMM_EINVAL
 * (reason in swmm_last_error) for an illegal or incomplete schedule. */
int swmm_set_schedule(swmm_t h, const swmm_search_spec *spec, const swmm_search_row *rows, int32_t nrows);

/* Plan a call of schedule `rows` without a handle or a device: what
 * swmm_workspace_elems reports for it (paper_elems: the schedule's own
 * temporaries over the levels that keep them; plan_elems: the planner's
 * peak), and the time the autotuner's model gives the plan (model_us, from
 * the plan's leaf flops, block-addition and staging bytes and launches; a
 * ranking aid, not a measurement).  opts->sched must be SWMM_CUSTOM.  Any
 * output pointer may be NULL. */
int swmm_schedule_workspace(const swmm_search_spec *spec, const swmm_search_row *rows, int32_t nrows, int64_t m,
                            int64_t k, int64_t n, const swmm_opts *opts, int64_t *paper_elems,
                            int64_t *plan_elems, double *model_us);

/* The plan's counts for a call of schedule `rows`, as swmm_plan_stats gives
 * them for the printed schedules (temporaries, staging, additions,
 * launches, pack bytes, one-pass level packs); no handle, no device.
 * opts->sched must be SWMM_CUSTOM. */
int swmm_schedule_stats(const swmm_search_spec *spec, const swmm_search_row *rows, int32_t nrows, int64_t m,
                        int64_t k, int64_t n, const swmm_opts *opts, swmm_stats *out);

/* The rows of the paper's table `sched` (SWMM_T1_DHSS ... SWMM_T9_ACC,
 * SWMM_T4M_OVL) as the library runs them, in the form swmm_schedule_check
 * and swmm_set_schedule take (node = -1; a recursive call of the table
 * itself has the table's own code as kind), so that a table can be
 * replayed, or changed (another kind for some rows) and run as the
 * handle's schedule.  *nrows receives the table's row count.  Returns
 * SWMM_OK, or SWMM_EINVAL for an unknown code or when max_rows is smaller
 * than the table. */
int swmm_table_rows(int32_t sched, swmm_search_row *rows, int32_t max_rows, int32_t *nrows);

/* Name of candidate value `node` of the graph for `accumulate` (0 or 1):
 * "A11" ... "B22" and "C11" ... "C22" for the inputs, "S1" ... "T4", "P1" ...
 * "P7", "U1" ... "U7" for the Section 2 values (U1, U5, U6, U7 are the
 * results, plus beta times the input C when accumulating), other sums
 * written out ("P5+bC12-bC21").  NULL when out of range. */
const char *swmm_search_node_name(int32_t accumulate, int32_t node);

/* Number of candidate values of the graph for `accumulate`. */
int32_t swmm_search_node_count(int32_t accumulate);

#ifdef __cplusplus
}
#endif

#endif
