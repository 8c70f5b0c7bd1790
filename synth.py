"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds no arithmetic of the method: it only draws matrices.  Both
the CPU oracle and the GPU path receive the same arrays from here, so a
disagreement between them can never come from the inputs.

Workload recipe (stands in for the paper's experiments, which used random
dense matrices, Section 8 / Table 11):
  * Z/pZ mode: entries uniform in [0, p-1], int32, row-major.
  * FP32 mode: entries N(0, 1), float32, row-major.
  * batched mode: shapes (m, k, n) uniform integers in [lo, hi].
Seeds: A=1, B=2, C=3, batch shapes=4; a matrix is identified by
(seed, tag) so different matrices of one problem never share a stream.
"""
from __future__ import annotations

import numpy as np

SEED_A, SEED_B, SEED_C, SEED_SHAPES, SEED_X = 1, 2, 3, 4, 5  # SEED_X: probe vectors


def _rng(seed: int, tag: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), int(tag)])))


def modp_matrix(seed: int, rows: int, cols: int, p: int, tag: int = 0) -> np.ndarray:
    """rows x cols int32 matrix with entries uniform in [0, p-1]."""
    if rows == 0 or cols == 0:
        return np.zeros((rows, cols), dtype=np.int32)
    return _rng(seed, tag).integers(0, p, size=(rows, cols), dtype=np.int32)


def normal_matrix(seed: int, rows: int, cols: int, tag: int = 0) -> np.ndarray:
    """rows x cols float32 matrix with N(0,1) entries."""
    if rows == 0 or cols == 0:
        return np.zeros((rows, cols), dtype=np.float32)
    return _rng(seed, tag).standard_normal(size=(rows, cols), dtype=np.float32)


def adversarial_modp(rows: int, cols: int, p: int, pattern: str) -> np.ndarray:
    """Worst cases for exact leaf accumulation.

    'max'      every entry p-1 (centred value -1, the smallest magnitude)
    'half'     every entry (p-1)//2 (largest positive centred value)
    'halfneg'  every entry (p+1)//2 (largest negative centred value)
    'alt'      checkerboard of (p-1)//2 and (p+1)//2
    """
    h = (p - 1) // 2
    if pattern == "max":
        return np.full((rows, cols), p - 1, dtype=np.int32)
    if pattern == "half":
        return np.full((rows, cols), h, dtype=np.int32)
    if pattern == "halfneg":
        return np.full((rows, cols), h + 1, dtype=np.int32)
    if pattern == "alt":
        i = np.add.outer(np.arange(rows), np.arange(cols)) & 1
        return np.where(i == 0, h, h + 1).astype(np.int32)
    raise ValueError(pattern)


def batch_shapes(count: int, lo: int, hi: int, seed: int = SEED_SHAPES) -> list[tuple[int, int, int]]:
    """`count` shapes (m, k, n), each dimension uniform in [lo, hi]."""
    r = _rng(seed, 0).integers(lo, hi + 1, size=(count, 3))
    return [tuple(int(v) for v in row) for row in r]
