/*
 * swmm.h - memory-efficient Strassen-Winograd matrix multiplication on GB300.
 *
 * C ABI of the library.  It implements the schedules of Boyer, Dumas, Pernet
 * and Zhou, "Memory efficient scheduling of Strassen-Winograd's matrix
 * multiplication algorithm" (ISSAC 2009):
 *
 *   Section 2  : Winograd's 2x2 block algorithm (8 pre-additions, 7
 *                products, 7 post-additions).
 *   Table 1    : C <- AB with two temporaries (Douglas et al.).
 *   Table 2    : C <- alpha AB + beta C with three temporaries
 *                (Huss-Lederman et al.).
 *   Tables 3-5 : C <- AB overwriting A and B (IP), A (OvL) or B (OvR).
 *   Tables 6-8 : C <- alpha AB + beta C overwriting A and B (AcLR), B (AccR),
 *                B12 and B21 (AcR, rectangular).
 *   Table 9    : C <- alpha AB + beta C, read-only inputs, two temporaries
 *                (Acc, Section 6).
 *   Alg. 2     : IPMM, C <- AB with read-only inputs and no extra memory
 *                (Section 7.1); temporaries are carved from C22.
 *
 * Conventions (every entry point):
 *   - Matrices are row-major.  lda, ldb, ldc are leading dimensions in
 *     elements, >= the number of columns.
 *   - A, B, C are DEVICE pointers owned by the caller.  Mode SWMM_MODP:
 *     int32 elements holding values in [0, p); outputs are canonical in
 *     [0, p).  Mode SWMM_FP32: float elements.
 *   - alpha and beta point to HOST scalars: uint32_t (reduced mod p by the
 *     library) in SWMM_MODP mode, float in SWMM_FP32 mode.
 *   - Calls are asynchronous on the handle's stream.  Workspace (the
 *     schedules' temporaries X, Y, Z) is allocated stream-ordered from the
 *     device's default memory pool for the duration of a call, sized exactly
 *     to the plan's peak; its size is reported by swmm_get_stats.
 *   - Argument errors are detected before any launch and return SWMM_EINVAL
 *     (see swmm_last_error for the reason); a CUDA failure returns
 *     SWMM_ECUDA.  Device-side waits are bounded: a kernel that gives up
 *     records SWMM_ETIMEOUT, reported by swmm_sync.
 *   - A and B must not overlap C.  A and B may overlap each other only for
 *     the read-only schedules.
 *   - Execution order: the rows of a table are issued in order; the leaf
 *     products of independent fused levels (those touching different
 *     blocks, or only adding into a common one) may share one grouped
 *     launch when their operand staging is small (at most 96 MiB per level),
 *     and on quadrants above 32 MiB the pre-additions that only feed a fused
 *     level are formed while its operands are packed.  Results are those of
 *     the rows in order; over Z/pZ they are bit-identical.
 */
#ifndef SWMM_H
#define SWMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define SWMM_OK 0
#define SWMM_EINVAL 1
#define SWMM_ENOMEM 2
#define SWMM_EUNSUPPORTED 3
#define SWMM_ECUDA 4
#define SWMM_ETIMEOUT 5

/* arithmetic modes */
#define SWMM_MODP 0 /* exact arithmetic over Z/pZ, 2 < p < 2^16 */
#define SWMM_FP32 1 /* float32 storage (Section 2 algorithm over the reals;
                       accuracy mode): each leaf operand is scaled by a
                       power of two from its max |x| and split into fp16
                       hi + lo (22 significant bits); hi*hi + hi*lo + lo*hi
                       are accumulated in fp32 and the scales undone */

/* schedules (the table numbers of the paper) */
#define SWMM_CLASSICAL 0 /* one classical product, no Winograd level */
#define SWMM_T1_DHSS 1   /* Table 1, C <- AB, read-only inputs */
#define SWMM_T2_HLJJTT 2 /* Table 2, C <- aAB + bC, read-only inputs */
#define SWMM_T3_IP 3     /* Table 3, C <- AB, overwrites A and B */
#define SWMM_T4_OVL 4    /* Table 4, C <- AB, overwrites A */
#define SWMM_T5_OVR 5    /* Table 5, C <- AB, overwrites B */
#define SWMM_T6_ACLR 6   /* Table 6, C <- aAB + bC, overwrites A and B */
#define SWMM_T7_ACCR 7   /* Table 7, C <- aAB + bC, overwrites B */
#define SWMM_T8_ACR 8    /* Table 8, C <- aAB + bC, overwrites B12, B21 */
#define SWMM_T9_ACC 9    /* Table 9, C <- aAB + bC, read-only inputs */
#define SWMM_IPMM 10     /* Algorithm 2, C <- AB, read-only, no extra memory */
#define SWMM_T4M_OVL 11  /* Section 5.1 variant of Table 4: overwrites A11, A21 */
#define SWMM_IP0VMM 12   /* Algorithm 1, C <- aAB for n < m, n <= k, n dividing
                            m and k; overwrites A, no extra memory */
#define SWMM_TBLOCK 13   /* Section 7.2, C <- aAB + bC, read-only inputs: C in
                            t x t blocks, each the sum of t products with
                            accumulation by Table 2 (or Table 9); the
                            temporaries of one block call at a time */
#define SWMM_CUSTOM 14   /* the handle's own one-level schedule (swmm_set_schedule in
                            swmm_search.h), square operands; its entry point
                            follows its contract: swmm_mul (read-only C <- aAB),
                            swmm_muladd (read-only C <- aAB + bC) or
                            swmm_mul_inplace (it overwrites a block of A or B) */
#define SWMM_AUTO (-1)   /* batched calls: the autotuner picks schedule and depth */

/* flags */
#define SWMM_FLAG_UNFUSED 1u   /* run the table at every level down to
                                  classical leaves (the literal schedule);
                                  default fuses the last Winograd level
                                  into one grouped leaf launch */
#define SWMM_FLAG_SIMT_LEAF 2u /* leaves on a plain CUDA-core kernel instead
                                  of the tcgen05 kernel (diagnostics) */
#define SWMM_FLAG_TIMING 4u    /* record a CUDA event pair around every leaf
                                  GEMM launch (read with swmm_leaf_timing) */
#define SWMM_FLAG_GRAPH 8u     /* capture the call's launches in a CUDA graph
                                  on first use and replay it for identical
                                  calls (same sizes, pointers, options and
                                  scalars); the graph runs on an internal
                                  stream ordered after and before the handle's
                                  stream by events.  The captured launches
                                  are ordered by the memory they touch: a
                                  launch waits only for earlier launches
                                  whose blocks it reads or writes, so
                                  independent rows of a schedule may overlap
                                  (operand staging then uses at least two
                                  areas in turn) */
#define SWMM_FLAG_SERIAL 16u   /* with SWMM_FLAG_GRAPH: capture every launch
                                  in row order on one stream */
#define SWMM_FLAG_LOWMEM 32u   /* bound the tensor-core operand staging to
                                  SWMM_LOWMEM_STAGE_BYTES: one staging area,
                                  leaf launches not merged, and a fused level
                                  (or a group of classical problems) staged
                                  and multiplied in groups of products that
                                  fit the bound; a single product whose
                                  operands exceed it is staged whole.  Slower
                                  (more, smaller launches), never different
                                  results */
#define SWMM_LOWMEM_STAGE_BYTES (64ll << 20)
#define SWMM_FLAG_TUNE 64u     /* swmm_muladd_batched: problems with SWMM_AUTO
                                  and 2 m k n >= 2 * 3072^3 get the measured
                                  choice instead of the model's: the classical
                                  product and one Winograd level (Table 2, or
                                  Table 9 if square) are each run on a scratch
                                  copy of C (device memory for one C, taken
                                  from and returned to the stream-ordered
                                  pool) and timed on the GPU the first time a
                                  shape and mode is seen; the handle keeps the
                                  result.  The first call with new shapes
                                  waits for those runs */

typedef struct swmm_ctx *swmm_t;

typedef struct {
  int32_t mode;        /* SWMM_MODP or SWMM_FP32 */
  uint32_t p;          /* modulus for SWMM_MODP: 2 < p < 65536 */
  int32_t sched;       /* SWMM_CLASSICAL ... SWMM_IP0VMM */
  int32_t depth;       /* Winograd recursion levels (0 = classical) */
  uint32_t flags;      /* SWMM_FLAG_* */
  int32_t ipmm_cutoff; /* IPMM: classical base case once the C block is
                          <= this size (0 = 1024) */
  int32_t ipmm_acc;    /* accumulation schedule of IPMM and SWMM_TBLOCK:
                          SWMM_T2_HLJJTT (default, 0) or SWMM_T9_ACC
                          (Sections 7.1 and 7.2) */
  int32_t tblock;      /* SWMM_TBLOCK: t >= 2 blocks per dimension (0 = 2);
                          m, k and n must be multiples of t */
} swmm_opts;

typedef struct {
  int64_t workspace_bytes;    /* device bytes allocated for temporaries */
  int64_t plan_extra_elems;   /* peak temporary elements of the plan run */
  int64_t paper_extra_elems;  /* the paper's count at the same depth for the
                                 levels that materialise temporaries */
  int64_t add_elems;          /* element operations of addition passes */
  int64_t leaf_flops;         /* 2 m n k summed over leaf products */
  int64_t leaf_launches;      /* leaf GEMM kernel launches */
  int64_t ew_launches;        /* elementwise kernel launches */
  int64_t leaf_products;      /* leaf products computed */
  int64_t staging_bytes;      /* device bytes of tensor-core operand staging
                                 (packed limb planes of the leaf operands;
                                 not part of the schedules' temporaries) */
  int64_t pack_bytes;         /* bytes the operand packs read and write */
  int64_t level_packs;        /* table levels whose fused levels' operands
                                 were formed in one pass */
  int64_t reserved[5];
} swmm_stats;

/* Create a handle bound to CUDA device `device` and stream `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *h receives the
 * handle; destroy it with swmm_destroy. */
int swmm_create(swmm_t *h, int device, void *cuda_stream);
int swmm_destroy(swmm_t h);
int swmm_set_stream(swmm_t h, void *cuda_stream);

/* C <- A B (m x k times k x n).  A and B are read-only: allowed schedules
 * SWMM_CLASSICAL, SWMM_T1_DHSS, SWMM_IPMM (Table 1, Algorithm 2).
 * IPMM needs m = n and k a multiple of n/2 at every level (Section 7.1);
 * other shapes return SWMM_EINVAL. */
int swmm_mul(swmm_t h, int64_t m, int64_t k, int64_t n,
             const void *A, int64_t lda, const void *B, int64_t ldb,
             void *C, int64_t ldc, const swmm_opts *opts);

/* One problem of a batched call (C <- alpha A B + beta C, read-only A, B). */
typedef struct {
  int64_t m, k, n;
  const void *A;
  int64_t lda;
  const void *B;
  int64_t ldb;
  void *C;
  int64_t ldc;
  int32_t mode;          /* SWMM_MODP or SWMM_FP32 */
  uint32_t p;            /* modulus (SWMM_MODP) */
  uint32_t alpha_u, beta_u; /* scalars (SWMM_MODP) */
  float alpha_f, beta_f;    /* scalars (SWMM_FP32) */
  int32_t sched;         /* SWMM_AUTO, SWMM_CLASSICAL, SWMM_T2_HLJJTT or SWMM_T9_ACC */
  int32_t depth;         /* used when sched != SWMM_AUTO */
  int32_t chosen_sched;  /* out: the schedule that ran */
  int32_t chosen_depth;  /* out: the depth that ran */
} swmm_problem;

/* C <- alpha A B + beta C with read-only A and B: SWMM_CLASSICAL,
 * SWMM_T2_HLJJTT (Table 2), SWMM_T9_ACC (Table 9, square), SWMM_TBLOCK
 * (Section 7.2; m, k, n multiples of opts->tblock, square blocks when the
 * base schedule is Table 9). */
int swmm_muladd(swmm_t h, int64_t m, int64_t k, int64_t n, const void *alpha,
                const void *A, int64_t lda, const void *B, int64_t ldb,
                const void *beta, void *C, int64_t ldc, const swmm_opts *opts);

/* C <- alpha A B + beta C with A, B and C in HOST memory (the paper has no
 * counterpart: the operands of a product that does not start on the GPU).
 * The handle copies A, B and C into device buffers it keeps (grown on demand,
 * freed by swmm_destroy), runs the same schedules as swmm_muladd, and copies
 * C back.  The copies go block by block (the 2 x 2 blocks of A, B and C) in
 * the order the top level's table first reads them, and C's blocks return as
 * soon as each is final; with SWMM_FLAG_GRAPH the product starts before the
 * last copy ends.  Page-locked host memory lets the copies overlap the work;
 * pageable memory works but copies synchronously.  A, B, C: host pointers,
 * row-major, leading dimensions in elements.  Asynchronous on the handle's
 * stream: C holds the result after swmm_sync.  Errors as swmm_muladd, plus
 * SWMM_ENOMEM when the device copies cannot be allocated. */
int swmm_muladd_host(swmm_t h, int64_t m, int64_t k, int64_t n, const void *alpha,
                     const void *A, int64_t lda, const void *B, int64_t ldb,
                     const void *beta, void *C, int64_t ldc, const swmm_opts *opts);

/* The same operation as swmm_muladd for callers that cannot allocate device
 * memory (the paper has no counterpart: it is a deployment variant).  Code
 * running where cudaMalloc/cudaMallocAsync are unavailable or forbidden --
 * inside a memory budget owned by another allocator, in a real-time path
 * that must not reach the CUDA driver's allocator, or in a process whose pools
 * are reserved -- gets the schedule's temporaries and the tensor-core
 * operand staging from one static device array of
 * SWMM_NOALLOC_SCRATCH_BYTES bytes that every GPU which loads the library
 * holds until the process exits.  Plans that need more scratch fail with
 * SWMM_EINVAL (swmm_last_error gives the sizes).  Nothing is allocated and
 * no scratch content needs to start at zero.  The first call on a device
 * looks the array's device address up (cudaGetSymbolAddress); make that
 * first call before any stream capture.  All calls share the array: calls
 * whose work overlaps on the GPU (different streams, or several handles)
 * race on it and must be serialised by the caller.  These calls always run
 * eagerly in row order on the handle's stream: SWMM_FLAG_GRAPH,
 * SWMM_FLAG_SERIAL and SWMM_FLAG_TIMING are ignored, leaf launches are not
 * merged, and swmm_leaf_timing reports no launches after such a call. */
#define SWMM_NOALLOC_SCRATCH_BYTES (32ll << 20)
int swmm_muladd_noalloc(swmm_t h, int64_t m, int64_t k, int64_t n, const void *alpha,
                        const void *A, int64_t lda, const void *B, int64_t ldb,
                        const void *beta, void *C, int64_t ldc, const swmm_opts *opts);

/* Schedules that may overwrite their inputs (Sections 5.1-5.3).
 * beta == NULL: C <- alpha A B with SWMM_T3_IP (k = n <= m), SWMM_T4_OVL,
 * SWMM_T4M_OVL, SWMM_T5_OVR (square), or SWMM_IP0VMM (Algorithm 1: A is
 * m x k, B is k x n with n < m, n <= k, n dividing m and k; C is split
 * into n x n row blocks C_1..C_m/n; C_1 <- A_11 B_1 by Table 1 with C_2 as
 * scratch, then A_11 is the scratch of C_i <- A_i1 B_1 by Table 4 and of
 * C_i <- A_ij B_j + C_i by Table 2).  beta != NULL: C <- alpha A B + beta C
 * with SWMM_T6_ACLR, SWMM_T7_ACCR (square), SWMM_T8_ACR (any even shape).
 * On return the overwritten operand blocks hold unspecified values:
 *   IP, AcLR: all of A and B;  OvL, IP0vMM: A;  OvLM: A11, A21;
 *   OvR, AccR: B;  AcR: B12, B21.  Every other block is left bit-identical. */
int swmm_mul_inplace(swmm_t h, int64_t m, int64_t k, int64_t n,
                     void *A, int64_t lda, void *B, int64_t ldb,
                     void *C, int64_t ldc, const void *alpha, const void *beta,
                     const swmm_opts *opts);

/* Many independent products of uneven shapes in one call.  Each problem
 * runs the plan its `sched` names (SWMM_AUTO: the autotuner's choice, see
 * swmm_autotune); odd dimensions are peeled at every Winograd level.  With
 * SWMM_FLAG_GRAPH the whole batch is captured once into one CUDA graph and
 * replayed by identical later calls.  The C blocks of different problems
 * must not overlap. */
int swmm_muladd_batched(swmm_t h, int count, swmm_problem *probs, uint32_t flags);

/* The autotuner: for C <- A B + C of size (m, k, n) in `mode`, evaluate the
 * classical product, Table 2 and (square) Table 9 at depths 1-3 with the
 * planner and a cost model of this GPU (tensor rate by leaf size, HBM-bound
 * passes, launch cost), and return the fastest (*sched, *depth), its
 * modelled time (*est_us) and its peak temporary elements (*extra_elems).
 * No device work; h may be NULL. */
int swmm_autotune(swmm_t h, int64_t m, int64_t k, int64_t n, int32_t mode, uint32_t p,
                  int32_t *sched, int32_t *depth, double *est_us, int64_t *extra_elems);

/* Peak temporary elements the plan for (m, k, n, opts) uses
 * (*plan_elems) and the paper's count for the same levels (*paper_elems;
 * Lemma 1 sums, Section 3).  No device work; h may be NULL. */
int swmm_workspace_elems(swmm_t h, int64_t m, int64_t k, int64_t n,
                         const swmm_opts *opts, int64_t *paper_elems,
                         int64_t *plan_elems);

/* The counts of the plan for (m, k, n, opts) as an eager call would run it,
 * in *out (the fields of swmm_stats; staging_bytes for an eager call, whose
 * fused levels share one staging area unless launches are merged): the
 * planning pass of the library, with no operands and no device work.  The
 * entry point is the one the schedule's contract implies (as
 * swmm_workspace_elems), with unit scalars; the final canonical pass over
 * blocks of C last written by reduce-adds, which only a real call knows,
 * is not counted.  h may be NULL. */
int swmm_plan_stats(swmm_t h, int64_t m, int64_t k, int64_t n, const swmm_opts *opts, swmm_stats *out);

/* Leaf GEMM timing recorded by calls made with SWMM_FLAG_TIMING since the
 * last reset.  Waits for the handle's stream, then returns the summed
 * event-measured duration of those launches (*gemm_ms), their number
 * (*launches) and the tensor-pipe flops they executed (*tensor_flops:
 * 2 m n k per product times the limb products per product: 1 for p <= 256,
 * 4 for larger p, 3 in SWMM_FP32 mode).  reset != 0 clears the record
 * afterwards.  Any output pointer may be NULL. */
int swmm_leaf_timing(swmm_t h, int reset, double *gemm_ms, int64_t *launches,
                     double *tensor_flops);

/* Randomised residual probe of a product (Freivalds' check).  The paper
 * has no counterpart: it verifies the result of any entry point above
 * without an O(n^3) reference product.
 *
 * swmm_matvec: y = M x for a row-major rows x cols matrix M with leading
 * dimension ldm.  SWMM_MODP: M holds int32 values (reduced mod p as read),
 * x and y are uint32 in [0, p), and the sum is exact.  SWMM_FP32: M holds
 * float, x and y are double, and the sum is formed in FP64.  M, x and y are
 * DEVICE pointers (y: rows entries); only opts->mode and opts->p are read.
 * Asynchronous on the handle's stream.
 *
 * swmm_residual: r = C x - alpha A (B x) - beta y0, where C is the result of
 * an earlier C <- alpha A B + beta C_in (or C <- alpha A B with beta = 0) and
 * y0 = C_in x was formed with swmm_matvec before that call (y0 may be NULL
 * when beta is 0).  x has n entries, y0 and r have m entries; all are
 * DEVICE pointers of swmm_matvec's element type.  alpha and beta point to
 * HOST scalars as for swmm_muladd.  Over Z/pZ a wrong C gives r == 0 with
 * probability at most 1/p for a uniformly random x.  In SWMM_FP32 mode r is
 * the FP64 residual of the float result; FP64 is used in this probe only,
 * never in the products.  Temporaries (k + 2m entries) are taken from and
 * returned to the stream-ordered pool within the call.
 * Errors: SWMM_EINVAL for bad sizes, NULL or misaligned pointers (x, y, r,
 * y0 must be 4-byte aligned mod p, 8-byte aligned in FP32 mode), or a
 * missing y0 with beta != 0; SWMM_ENOMEM; SWMM_ECUDA. */
int swmm_matvec(swmm_t h, int64_t rows, int64_t cols, const void *M,
                int64_t ldm, const void *x, void *y, const swmm_opts *opts);
int swmm_residual(swmm_t h, int64_t m, int64_t k, int64_t n,
                  const void *alpha, const void *A, int64_t lda,
                  const void *B, int64_t ldb, const void *beta,
                  const void *y0, const void *C, int64_t ldc, const void *x,
                  void *r, const swmm_opts *opts);

/* Measured device memory of the library's calls (the paper counts extra
 * memory in Table 10; this is the same quantity in bytes, as the device saw
 * it).  Waits for the handle's streams, then writes out[0] = bytes of the
 * device's default memory pool in use now (workspace and staging of eager
 * calls come from it), out[1] = its high-water mark since the last reset,
 * out[2] = bytes of graph memory in use now (the same for calls captured
 * with SWMM_FLAG_GRAPH; graphs a handle keeps may hold some), out[3] = its
 * high-water mark.  reset != 0 then sets both marks back to the current
 * use, so the peak extra memory of the calls that follow is
 * max(out[1] - out[0], out[3] - out[2]) read after them against the values
 * read at the reset.  Both are per device: other users of the default pool
 * or of graph memory on the device count too. */
int swmm_memory_use(swmm_t h, int reset, int64_t *out);

/* Statistics of the last completed call on this handle. */
int swmm_get_stats(swmm_t h, swmm_stats *out);

/* Wait for the handle's stream and report device-side errors
 * (SWMM_ETIMEOUT if a kernel's bounded wait gave up). */
int swmm_sync(swmm_t h);

/* Failure injection for tests of the error paths (the paper has no
 * counterpart).  Failures are made on the host or by a device wait that is
 * bounded: nothing faults, traps or hangs the GPU.
 *   SWMM_HOOK_WAIT_NS      every mbarrier wait of the leaf GEMM kernel
 *                          gives up after `value` ns (value <= 0: the
 *                          default, 4 s); on expiry the kernel drains the
 *                          copies and products it issued, frees its tensor
 *                          memory and returns, and swmm_sync reports
 *                          SWMM_ETIMEOUT.
 *   SWMM_HOOK_STALL_GEMMS  the next `value` leaf GEMM launches first wait
 *                          on a barrier that nothing arrives at, so that
 *                          wait runs out (their results are undefined).
 *   SWMM_HOOK_FAIL_ALLOCS  the next `value` device allocations of the
 *                          handle's calls fail: the call returns
 *                          SWMM_ENOMEM before any launch.
 *   SWMM_HOOK_LOWMEM_BYTES the staging bound of SWMM_FLAG_LOWMEM calls on
 *                          this handle (value <= 0: SWMM_LOWMEM_STAGE_BYTES),
 *                          so that small products exercise the grouping.
 * Settings apply to calls made afterwards on this handle; graphs captured
 * earlier (SWMM_FLAG_GRAPH) keep what they captured.  Returns SWMM_EINVAL
 * for an unknown hook. */
#define SWMM_HOOK_WAIT_NS 1
#define SWMM_HOOK_STALL_GEMMS 2
#define SWMM_HOOK_FAIL_ALLOCS 3
#define SWMM_HOOK_LOWMEM_BYTES 4
int swmm_test_hook(swmm_t h, int32_t hook, int64_t value);

const char *swmm_strerror(int code);
/* Text of the last error on this handle (empty if none). */
const char *swmm_last_error(swmm_t h);

#ifdef __cplusplus
}
#endif
#endif /* SWMM_H */
