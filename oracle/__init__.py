"""CPU oracle for memory-efficient Strassen-Winograd schedules.

TEST INFRASTRUCTURE ONLY.  Only `tests/`, `__graft_entry__.smoke()` and the
CPU-baseline leg of `bench.py` may import this package.  The product path
(the C-ABI library and its Python binding) never imports, links or calls it,
and this package never imports the product package.

Parts:
  ring        the two coefficient rings the paper's algorithm runs over
              (Z/pZ with exact integers, and FP64 reals).
  classical   the plain definition C <- alpha*A*B + beta*C (Section 2 and
              Section 3.2 problem statements).
  schedules   a literal, row-by-row interpreter of Tables 1-9 with liveness,
              clobber, aliasing, restoration and temporary-memory tracking.
  ipmm        Algorithm 2 (IPMM) and Algorithm 1 (IP0vMM) drivers.
  counts      recurrences and closed forms of Section 3 and Theorem 1-3.
  probes      Freivalds residual probe and floating-point error metrics.
"""
