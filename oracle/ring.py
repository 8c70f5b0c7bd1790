"""Coefficient rings used by the oracle.

Winograd's algorithm only uses +, - and x, so it runs over any ring
(Section 2; the introduction names finite fields and floating point).
The oracle implements two:
  * ModP: Z/pZ, values stored as canonical int64 in [0, p).
  * Real: float64.

Test infrastructure only (see oracle/__init__.py).
"""
from __future__ import annotations

import numpy as np


class ModP:
    """Z/pZ with canonical representatives in [0, p)."""

    exact = True

    def __init__(self, p: int):
        if p < 2:
            raise ValueError("p must be >= 2")
        self.p = int(p)
        self.dtype = np.int64

    def __repr__(self):
        return f"ModP({self.p})"

    def scalar(self, s) -> int:
        return int(s) % self.p

    def canon(self, x: np.ndarray) -> np.ndarray:
        return np.mod(np.asarray(x, dtype=np.int64), self.p)

    def lincomb(self, terms) -> np.ndarray:
        """sum of coef * array, reduced mod p.  terms: [(coef, array)]."""
        acc = None
        for c, a in terms:
            t = (self.scalar(c) * np.asarray(a, dtype=np.int64)) % self.p
            acc = t if acc is None else (acc + t) % self.p
        return acc

    def matmul(self, a: np.ndarray, b: np.ndarray) -> np.ndarray:
        # entries < 2^16 so each product < 2^32; an int64 sum of fewer than
        # 2^31 such products cannot overflow.
        a = np.asarray(a, dtype=np.int64)
        b = np.asarray(b, dtype=np.int64)
        assert a.shape[1] < (1 << 31)
        return np.mod(a @ b, self.p)

    def poison(self, rng: np.random.Generator, shape) -> np.ndarray:
        return rng.integers(0, self.p, size=shape, dtype=np.int64)

    def zeros(self, shape) -> np.ndarray:
        return np.zeros(shape, dtype=np.int64)

    def equal(self, x, y) -> bool:
        return np.array_equal(self.canon(x), self.canon(y))


class Real:
    """float64 arithmetic."""

    exact = False

    def __init__(self):
        self.dtype = np.float64

    def __repr__(self):
        return "Real()"

    def scalar(self, s) -> float:
        return float(s)

    def canon(self, x: np.ndarray) -> np.ndarray:
        return np.asarray(x, dtype=np.float64)

    def lincomb(self, terms) -> np.ndarray:
        acc = None
        for c, a in terms:
            t = float(c) * np.asarray(a, dtype=np.float64)
            acc = t if acc is None else acc + t
        return acc

    def matmul(self, a, b) -> np.ndarray:
        return np.asarray(a, dtype=np.float64) @ np.asarray(b, dtype=np.float64)

    def poison(self, rng: np.random.Generator, shape) -> np.ndarray:
        # NaN propagates through every later use of a dead value.
        return np.full(shape, np.nan)

    def zeros(self, shape) -> np.ndarray:
        return np.zeros(shape, dtype=np.float64)

    def equal(self, x, y) -> bool:
        return np.array_equal(np.asarray(x), np.asarray(y))
