"""Classical product: the plain definition every schedule must reproduce.

Section 2 defines C = A x B for an m x k matrix A and a k x n matrix B;
Section 3.2 defines the accumulating operation C <- alpha*A*B + beta*C.
Over Z/pZ the result is unique, so the definition itself is the oracle:
every Strassen-Winograd schedule must reach exactly these values.

Test infrastructure only (see oracle/__init__.py).
"""
from __future__ import annotations

import numpy as np


def mul_modp(A, B, p: int) -> np.ndarray:
    """(A B) mod p, canonical int64 in [0, p).  A: m x k, B: k x n."""
    A = np.asarray(A, dtype=np.int64) % p
    B = np.asarray(B, dtype=np.int64) % p
    if A.shape[1] != B.shape[0]:
        raise ValueError("inner dimensions differ")
    if A.shape[1] == 0:
        return np.zeros((A.shape[0], B.shape[1]), dtype=np.int64)
    # each product < p^2 < 2^32: an int64 sum of k < 2^31 of them is exact
    return np.mod(A @ B, p)


def muladd_modp(alpha, A, B, beta, C, p: int) -> np.ndarray:
    """(alpha A B + beta C) mod p (Section 3.2 operation)."""
    AB = mul_modp(A, B, p)
    C = np.asarray(C, dtype=np.int64) % p
    return np.mod((int(alpha) % p) * AB + (int(beta) % p) * C, p)


def rows_muladd_modp(rows, alpha, A, B, beta, C, p: int) -> np.ndarray:
    """Selected rows of (alpha A B + beta C) mod p, computed one row block at a
    time so the full product is never formed (spot checks at large n)."""
    rows = np.asarray(rows, dtype=np.int64)
    Ar = np.asarray(A[rows, :], dtype=np.int64)
    Cr = None if C is None else np.asarray(C[rows, :], dtype=np.int64)
    AB = mul_modp(Ar, B, p)
    if Cr is None:
        return np.mod((int(alpha) % p) * AB, p)
    return np.mod((int(alpha) % p) * AB + (int(beta) % p) * (Cr % p), p)


def mul_f64(A, B) -> np.ndarray:
    """A B in float64."""
    return np.asarray(A, dtype=np.float64) @ np.asarray(B, dtype=np.float64)


def muladd_f64(alpha, A, B, beta, C) -> np.ndarray:
    """alpha A B + beta C in float64."""
    return float(alpha) * mul_f64(A, B) + float(beta) * np.asarray(C, dtype=np.float64)


def rows_muladd_f64(rows, alpha, A, B, beta, C) -> np.ndarray:
    rows = np.asarray(rows, dtype=np.int64)
    r = float(alpha) * mul_f64(A[rows, :], B)
    if C is not None:
        r = r + float(beta) * np.asarray(C[rows, :], dtype=np.float64)
    return r


def triple_loop_modp(A, B, p: int) -> list:
    """Pure-Python triple loop, independent of numpy's matmul.  Tiny inputs
    only: it pins mul_modp to the textbook definition sum_l a_il b_lj."""
    m, k = len(A), len(A[0]) if len(A) else 0
    n = len(B[0]) if len(B) else 0
    out = [[0] * n for _ in range(m)]
    for i in range(m):
        for j in range(n):
            s = 0
            for l in range(k):
                s += int(A[i][l]) * int(B[l][j])
            out[i][j] = s % p
    return out
