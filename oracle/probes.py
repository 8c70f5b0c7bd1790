"""Checks usable at sizes where the full classical product is too slow.

  * freivalds_modp: exact randomized residual (alpha A (B x) + beta C_in x -
    C_out x) mod p for random x; a wrong C_out passes one vector with
    probability at most 1/p.
  * residual_f64: the same residual in float64 for the FP mode.
  * fp_error: max |C - C64| / (||A||max ||B||max) and the Frobenius variant;
    the paper does not fix a norm (it excludes stability, Section 1), so the
    max-norm form used for fast matrix multiplication error bounds is taken.

Test infrastructure only (see oracle/__init__.py).
"""
from __future__ import annotations

import numpy as np


def freivalds_modp(alpha, A, B, beta, C_in, C_out, p: int, vectors: int = 2, seed: int = 99) -> bool:
    rng = np.random.default_rng(seed)
    A = np.asarray(A, dtype=np.int64) % p
    B = np.asarray(B, dtype=np.int64) % p
    Co = np.asarray(C_out, dtype=np.int64) % p
    for _ in range(vectors):
        x = rng.integers(0, p, size=(B.shape[1],), dtype=np.int64)
        Bx = (B @ x) % p
        lhs = (int(alpha) % p) * ((A @ Bx) % p)
        if C_in is not None and beta is not None:
            lhs = lhs + (int(beta) % p) * ((np.asarray(C_in, dtype=np.int64) % p) @ x % p)
        r = (lhs - (Co @ x) % p) % p
        if np.any(r != 0):
            return False
    return True


def residual_f64(alpha, A, B, beta, C_in, C_out, vectors: int = 2, seed: int = 98) -> float:
    """max over probe vectors of ||alpha A(Bx) + beta C_in x - C_out x||_inf /
    (||A||max ||B||max ||x||_1)."""
    rng = np.random.default_rng(seed)
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    Co = np.asarray(C_out, dtype=np.float64)
    scale = np.abs(A).max() * np.abs(B).max()
    worst = 0.0
    for _ in range(vectors):
        x = rng.standard_normal(B.shape[1])
        lhs = alpha * (A @ (B @ x))
        if C_in is not None and beta:
            lhs = lhs + beta * (np.asarray(C_in, dtype=np.float64) @ x)
        r = np.abs(lhs - Co @ x).max() / (scale * np.abs(x).sum())
        worst = max(worst, r)
    return worst


def fp_error(C, C64, A, B) -> dict:
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    D = np.asarray(C, dtype=np.float64) - np.asarray(C64, dtype=np.float64)
    na, nb = np.abs(A).max(), np.abs(B).max()
    return {
        "max_rel": float(np.abs(D).max() / (na * nb)),
        "fro_rel": float(np.linalg.norm(D) / (np.linalg.norm(A) * np.linalg.norm(B))),
    }


def fp_bound(n: int) -> float:
    """FP32-mode tolerance: 1e-5 * n^0.6 (relative to ||A|| ||B||)."""
    return 1e-5 * n ** 0.6
