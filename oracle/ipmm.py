"""Algorithm 2 (IPMM, Section 7.1) and Algorithm 1 (IP0vMM, Section 5.3).

IPMM computes C <- A B for A n x k, B k x n (k >= n, both powers of two)
without overwriting A or B and without any extra memory: the three
quadrants C11, C12, C21 are built from n/2 x n/2 Winograd products (Table 1
for the first block column, then Table 2, or Table 9, accumulations over
the remaining 2k/n - 1 block columns), all temporaries carved from C22, and
C22 is then computed by the same algorithm on A's bottom rows and B's right
columns.  The recursion stops at a classical base case.

IP0vMM computes C <- A B for n < min(m, k), overwriting A and B.  The index
ranges of the printed algorithm are garbled; they are read as: C is split
into m0 = m/n row blocks C_1..C_m0; C_1 <- A_11 B_1 by Table 1 with C_2 as
scratch; then A_11 is scratch for C_i <- A_i1 B_1 (Table 4, i = 2..m0) and
for C_i <- A_ij B_j + C_i (Table 2, j = 2..k0, i = 1..m0).

Test infrastructure only (see oracle/__init__.py).
"""
from __future__ import annotations

import numpy as np

from .schedules import CarveArena, Interpreter, ScheduleError


def ipmm(ring, A, B, *, depth: int, cutoff: int = 1, acc_kind: str = "T2", seed: int = 7):
    """Return (C, stats).  `depth` = Winograd levels of each Table 1 / Table 2
    sub-call (capped by the block size); the IPMM recursion on C22 stops when
    the block is <= cutoff or odd, where a classical product finishes it."""
    A = np.array(A, dtype=ring.dtype, copy=True)
    B = np.array(B, dtype=ring.dtype, copy=True)
    A0, B0 = A.copy(), B.copy()
    n, k = A.shape
    if B.shape != (k, n):
        raise ValueError("IPMM needs A n x k and B k x n")
    C = ring.poison(np.random.default_rng(seed), (n, n)).astype(ring.dtype)
    it = Interpreter(ring, seed=seed)
    _ipmm_rec(it, A, B, C, depth, cutoff, acc_kind)
    if not (np.array_equal(A, A0, equal_nan=True) and np.array_equal(B, B0, equal_nan=True)):
        raise ScheduleError("IPMM modified a read-only input")
    return ring.canon(C), it.stats


def _levels(size: int, depth: int) -> int:
    d = 0
    while d < depth and size % 2 == 0 and size >= 2:
        size //= 2
        d += 1
    return d


def _ipmm_rec(it, A, B, C, depth, cutoff, acc_kind):
    n, k = A.shape
    if n <= cutoff or n % 2 or k % (n // 2):
        it.leaf(1, None, A, B, C)
        return
    h = n // 2
    nb = k // h  # = 2k/n block columns of A, block rows of B
    blk = lambda M, i, j: M[i * h:(i + 1) * h, j * h:(j + 1) * h]
    scratch = C[h:, h:]
    d = _levels(h, depth)
    one = it.ring.scalar(1)
    for (ci, cj), (ai, bj) in (((0, 0), (0, 0)), ((0, 1), (0, 1)), ((1, 0), (1, 0))):
        it.call("T1", one, None, blk(A, ai, 0), blk(B, 0, bj), blk(C, ci, cj), d,
                CarveArena(scratch, it.ring, it.stats, it.rng))
    for i in range(1, nb):
        for (ci, cj), (ai, bj) in (((0, 0), (0, 0)), ((0, 1), (0, 1)), ((1, 0), (1, 0))):
            it.call(acc_kind, one, one, blk(A, ai, i), blk(B, i, bj), blk(C, ci, cj), d,
                    CarveArena(scratch, it.ring, it.stats, it.rng))
    _ipmm_rec(it, A[h:, :], B[:, h:], scratch, depth, cutoff, acc_kind)


def ip0vmm(ring, A, B, *, depth: int, seed: int = 9):
    """Return (C, A_after, B_after, stats) for Algorithm 1 (n < min(m, k))."""
    A = np.array(A, dtype=ring.dtype, copy=True)
    B = np.array(B, dtype=ring.dtype, copy=True)
    m, k = A.shape
    n = B.shape[1]
    if not (n < m and n <= k and m % n == 0 and k % n == 0):
        raise ValueError("IP0vMM needs n < m, n <= k, n dividing m and k")
    m0, k0 = m // n, k // n
    C = ring.poison(np.random.default_rng(seed), (m, n)).astype(ring.dtype)
    it = Interpreter(ring, seed=seed)
    Ab = lambda i, j: A[i * n:(i + 1) * n, j * n:(j + 1) * n]
    Bb = lambda j: B[j * n:(j + 1) * n, :]
    Cb = lambda i: C[i * n:(i + 1) * n, :]
    d = _levels(n, depth)
    one = ring.scalar(1)
    it.call("T1", one, None, Ab(0, 0), Bb(0), Cb(0), d, CarveArena(Cb(1), ring, it.stats, it.rng))
    scratch = Ab(0, 0)  # A_11 is dead from here on
    for i in range(1, m0):
        it.call("OvL", one, None, Ab(i, 0), Bb(0), Cb(i), d, CarveArena(scratch, ring, it.stats, it.rng))
    for j in range(1, k0):
        for i in range(m0):
            it.call("T2", one, one, Ab(i, j), Bb(j), Cb(i), d, CarveArena(scratch, ring, it.stats, it.rng))
    return ring.canon(C), A, B, it.stats
