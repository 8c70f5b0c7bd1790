"""Pins of the classical oracle to definitions independent of numpy matmul."""
import numpy as np
import pytest

from oracle import classical, probes, ring


@pytest.mark.parametrize("p", [2, 3, 251, 65521])
@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 3, 4), (5, 1, 3), (7, 6, 5)])
def test_mul_modp_matches_triple_loop(p, shape):
    m, k, n = shape
    rng = np.random.default_rng(m * 100 + k * 10 + n + p)
    A = rng.integers(0, p, (m, k))
    B = rng.integers(0, p, (k, n))
    ref = classical.triple_loop_modp(A.tolist(), B.tolist(), p)
    assert classical.mul_modp(A, B, p).tolist() == ref


def test_mul_modp_closed_forms():
    p = 65521
    n = 37
    I = np.eye(n, dtype=np.int64)
    rng = np.random.default_rng(3)
    A = rng.integers(0, p, (n, n))
    assert np.array_equal(classical.mul_modp(A, I, p), A)
    assert np.array_equal(classical.mul_modp(I, A, p), A)
    # all-(p-1) times all-(p-1): each entry is k (p-1)^2 = k mod p
    k = 50
    J = np.full((n, k), p - 1)
    K = np.full((k, n), p - 1)
    assert np.all(classical.mul_modp(J, K, p) == k % p)
    # permutation matrix permutes rows
    perm = rng.permutation(n)
    P = np.zeros((n, n), dtype=np.int64)
    P[np.arange(n), perm] = 1
    assert np.array_equal(classical.mul_modp(P, A, p), A[perm])


def test_muladd_modp_definition():
    p = 251
    rng = np.random.default_rng(5)
    A, B, C = (rng.integers(0, p, s) for s in [(4, 6), (6, 3), (4, 3)])
    tl = np.array(classical.triple_loop_modp(A.tolist(), B.tolist(), p))
    ref = (7 * tl + 11 * C) % p
    assert np.array_equal(classical.muladd_modp(7, A, B, 11, C, p), ref)
    rows = [0, 3]
    assert np.array_equal(classical.rows_muladd_modp(rows, 7, A, B, 11, C, p), ref[rows])


def test_mul_modp_empty_inner_dimension():
    A = np.zeros((3, 0), dtype=np.int64)
    B = np.zeros((0, 2), dtype=np.int64)
    assert np.array_equal(classical.mul_modp(A, B, 7), np.zeros((3, 2)))


def test_f64_matches_loop():
    rng = np.random.default_rng(6)
    A = rng.standard_normal((3, 4))
    B = rng.standard_normal((4, 2))
    ref = [[sum(A[i, l] * B[l, j] for l in range(4)) for j in range(2)] for i in range(3)]
    assert np.allclose(classical.mul_f64(A, B), ref, rtol=1e-14, atol=1e-14)


def test_freivalds_accepts_and_rejects():
    p = 65521
    rng = np.random.default_rng(8)
    A, B, C = (rng.integers(0, p, (20, 20)) for _ in range(3))
    out = classical.muladd_modp(3, A, B, 5, C, p)
    assert probes.freivalds_modp(3, A, B, 5, C, out, p)
    bad = out.copy()
    bad[7, 11] = (bad[7, 11] + 1) % p
    assert not probes.freivalds_modp(3, A, B, 5, C, bad, p)


def test_fp_error_metric_scale():
    A = np.full((2, 2), 2.0)
    B = np.full((2, 2), 3.0)
    C = np.zeros((2, 2))
    C64 = np.zeros((2, 2))
    C64[0, 0] = 0.6
    assert probes.fp_error(C, C64, A, B)["max_rel"] == pytest.approx(0.1)


def test_ring_modp_canon():
    R = ring.ModP(7)
    assert R.canon(np.array([-1, 7, 15])).tolist() == [6, 0, 1]
    assert R.lincomb([(-1, np.array([3])), (2, np.array([5]))]).tolist() == [0]
