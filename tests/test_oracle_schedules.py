"""Pins of the schedule interpreter: every table reaches the plain definition,
reads only live values, keeps its declared read-only inputs, and uses the
temporary memory and operation counts the paper states."""
import itertools
import os
from fractions import Fraction as F

import numpy as np
import pytest

from oracle import classical, counts, ring, schedules as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
ALL = list(S.KINDS)


def _ref(kind, A, B, C, alpha, beta, R):
    if isinstance(R, ring.ModP):
        if S.KINDS[kind].accumulate:
            return classical.muladd_modp(alpha, A, B, beta, C, R.p)
        return classical.muladd_modp(alpha, A, B, 0, C, R.p)
    if S.KINDS[kind].accumulate:
        return classical.muladd_f64(alpha, A, B, beta, C)
    return alpha * classical.mul_f64(A, B)


@pytest.mark.parametrize("kind", ALL)
@pytest.mark.parametrize("p", [251, 65521])
@pytest.mark.parametrize("n,depth", [(2, 1), (4, 1), (4, 2), (8, 3), (16, 2), (32, 3), (12, 2), (6, 3)])
def test_schedule_equals_definition_modp(kind, p, n, depth):
    R = ring.ModP(p)
    rng = np.random.default_rng(n * 7 + depth)
    A, B, C = (rng.integers(0, p, (n, n)) for _ in range(3))
    alpha, beta = int(rng.integers(0, p)), int(rng.integers(0, p))
    out, _, _, st = S.run(kind, R, A, B, C, alpha=alpha, beta=beta, depth=depth)
    assert np.array_equal(out, _ref(kind, A, B, C, alpha, beta, R))


@pytest.mark.parametrize("kind", ALL)
def test_schedule_real_ring(kind):
    R = ring.Real()
    rng = np.random.default_rng(11)
    A, B, C = (rng.standard_normal((16, 16)) for _ in range(3))
    out, _, _, _ = S.run(kind, R, A, B, C, alpha=0.75, beta=-1.5, depth=3)
    assert np.allclose(out, _ref(kind, A, B, C, 0.75, -1.5, R), rtol=1e-11, atol=1e-11)


@pytest.mark.parametrize("kind,shape", [
    ("T1", (8, 4, 16)), ("T1", (16, 8, 4)), ("T1", (4, 16, 8)),
    ("T2", (8, 4, 16)), ("T2", (4, 16, 8)),
    ("AcR", (8, 16, 4)), ("AcR", (16, 4, 8)), ("AcR", (4, 8, 16)),
    ("IP", (16, 8, 8)), ("IP", (32, 8, 8)),
])
def test_rectangular(kind, shape):
    m, k, n = shape
    p = 65521
    R = ring.ModP(p)
    rng = np.random.default_rng(m + k + n)
    A, B, C = rng.integers(0, p, (m, k)), rng.integers(0, p, (k, n)), rng.integers(0, p, (m, n))
    out, _, _, _ = S.run(kind, R, A, B, C, alpha=2, beta=3, depth=2)
    assert np.array_equal(out, _ref(kind, A, B, C, 2, 3, R))


def test_in_place_precondition_k_le_min_mn():
    # Section 5.3: the in-place schedule needs k = n <= m (or the transpose);
    # with k > n the S blocks do not fit in the C quadrants.
    R = ring.ModP(7)
    A = np.ones((8, 16), dtype=np.int64)
    B = np.ones((16, 8), dtype=np.int64)
    with pytest.raises(S.ScheduleError):
        S.run("IP", R, A, B, depth=1)


@pytest.mark.parametrize("kind", ALL)
def test_exhaustive_z2_n2(kind):
    """All 2^12 (A,B,C) triples over Z/2Z (2^8 for C <- AB kinds), one level."""
    R = ring.ModP(2)
    acc = S.KINDS[kind].accumulate
    nbits = 12 if acc else 8
    for bits in range(1 << nbits):
        v = [(bits >> i) & 1 for i in range(nbits)]
        A = np.array(v[0:4]).reshape(2, 2)
        B = np.array(v[4:8]).reshape(2, 2)
        C = np.array(v[8:12]).reshape(2, 2) if acc else np.zeros((2, 2), dtype=np.int64)
        out, _, _, _ = S.run(kind, R, A, B, C, alpha=1, beta=1, depth=1, poison=False)
        ref = (A @ B + (C if acc else 0)) % 2
        assert np.array_equal(out, ref), (kind, bits)


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                rows.append(line.split())
    return rows


def test_memory_matches_table10():
    for kind, ntmp, coef in _golden("table10.txt"):
        c = F(coef)
        for n in (2, 4, 8, 16, 32):
            R = ring.ModP(65521)
            rng = np.random.default_rng(n)
            A, B, C = (rng.integers(0, 65521, (n, n)) for _ in range(3))
            _, _, _, st = S.run(kind, R, A, B, C, depth=20, poison=False)
            assert F(st.peak_tmp) == c * (n * n - 1), (kind, n)
        assert counts.BLOCKS_PER_LEVEL[kind] == int(ntmp)


@pytest.mark.parametrize("kind", ALL)
@pytest.mark.parametrize("n,depth", [(64, 1), (64, 2), (64, 3), (32, 4)])
def test_memory_truncated_depth(kind, n, depth):
    R = ring.ModP(251)
    rng = np.random.default_rng(1)
    A, B, C = (rng.integers(0, 251, (n, n)) for _ in range(3))
    _, _, _, st = S.run(kind, R, A, B, C, depth=depth, poison=False)
    assert st.peak_tmp == counts.mem_depth(kind, n, depth)


@pytest.mark.parametrize("m,k,n", [(8, 4, 16), (16, 8, 4), (4, 16, 8), (32, 8, 16), (8, 8, 8)])
def test_rectangular_memory_lemma1(m, k, n):
    R = ring.ModP(251)
    rng = np.random.default_rng(2)
    A, B, C = rng.integers(0, 251, (m, k)), rng.integers(0, 251, (k, n)), rng.integers(0, 251, (m, n))
    _, _, _, st1 = S.run("T1", R, A, B, depth=20, poison=False)
    assert F(st1.peak_tmp) == counts.E1(m, k, n)
    _, _, _, st2 = S.run("T2", R, A, B, C, depth=20, poison=False)
    assert F(st2.peak_tmp) == counts.E2(m, k, n)


def test_arithmetic_matches_theorem3_golden():
    for kind, n, W in _golden("theorem3_arith.txt"):
        n, W = int(n), int(W)
        R = ring.ModP(65521)
        rng = np.random.default_rng(n)
        A, B, C = (rng.integers(0, 65521, (n, n)) for _ in range(3))
        _, _, _, st = S.run(kind, R, A, B, C, depth=20, poison=False)
        assert st.ops == W, (kind, n, st.ops)


@pytest.mark.parametrize("n", [2, 4, 8, 16, 32])
def test_arithmetic_all_kinds(n):
    expect = {"T1": counts.W1_closed, "IP": counts.W1_closed, "OvL": counts.W1_closed,
              "OvLM": counts.W1_closed, "OvR": counts.W1_closed, "T2": counts.W2_closed,
              "AcLR": counts.W6_closed, "AccR": counts.W7_closed, "Acc": counts.W9_rec,
              "AcR": counts.W8_rec}
    for kind, f in expect.items():
        R = ring.ModP(65521)
        rng = np.random.default_rng(n)
        A, B, C = (rng.integers(0, 65521, (n, n)) for _ in range(3))
        _, _, _, st = S.run(kind, R, A, B, C, depth=20, poison=False)
        assert st.ops == f(n), kind


def test_seven_products_fifteen_additions_per_level():
    # Section 2: one Winograd level is 8 pre-additions, 7 products and 7
    # post-additions; Table 1 at one level does 15 block additions.
    R = ring.ModP(251)
    rng = np.random.default_rng(4)
    n = 8
    A, B = rng.integers(0, 251, (n, n)), rng.integers(0, 251, (n, n))
    _, _, _, st = S.run("T1", R, A, B, depth=1)
    assert st.leaves == 7
    assert st.adds == 15 * (n // 2) ** 2
    assert st.calls["T1"] == 8
    adds = {"T1": 15, "T2": 14, "IP": 15, "OvL": 15, "OvR": 15, "AcLR": 17, "AccR": 17, "Acc": 17, "AcR": 16}
    for kind, a in adds.items():
        C = rng.integers(0, 251, (n, n))
        _, _, _, st = S.run(kind, R, A, B, C, depth=1)
        assert st.adds == a * (n // 2) ** 2, kind
        assert st.leaves == 7, kind


def test_total_allocations():
    rec = {"T1": counts.A1_rec, "T2": counts.A2_rec, "OvL": counts.A4_rec, "OvR": counts.A4_rec,
           "AcLR": counts.A6_rec, "AccR": counts.A7_rec, "Acc": counts.A9_rec, "IP": lambda n: 0}
    for kind, f in rec.items():
        for n in (2, 4, 8, 16):
            R = ring.ModP(251)
            rng = np.random.default_rng(n)
            A, B, C = (rng.integers(0, 251, (n, n)) for _ in range(3))
            _, _, _, st = S.run(kind, R, A, B, C, depth=20, poison=False)
            assert st.total_alloc == f(n), (kind, n)


PRESERVE = {
    "T1": ("A", "B"), "T2": ("A", "B"), "Acc": ("A", "B"), "OvL": ("B",), "OvR": ("A",),
    "AccR": ("A",), "IP": (), "AcLR": (),
}


@pytest.mark.parametrize("kind", list(PRESERVE))
def test_restoration(kind):
    p = 65521
    R = ring.ModP(p)
    rng = np.random.default_rng(9)
    n = 32
    A, B, C = (rng.integers(0, p, (n, n)) for _ in range(3))
    _, A2, B2, _ = S.run(kind, R, A, B, C, depth=3)
    keep = PRESERVE[kind]
    if "A" in keep:
        assert np.array_equal(A2, A)
    else:
        assert not np.array_equal(A2, A)
    if "B" in keep:
        assert np.array_equal(B2, B)
    else:
        assert not np.array_equal(B2, B)


def test_restoration_modified_ovl_and_acr():
    p = 65521
    R = ring.ModP(p)
    rng = np.random.default_rng(10)
    n = 32
    A, B, C = (rng.integers(0, p, (n, n)) for _ in range(3))
    h = n // 2
    _, A2, B2, _ = S.run("OvLM", R, A, B, depth=3)
    assert np.array_equal(B2, B)
    assert np.array_equal(A2[:h, h:], A[:h, h:]) and np.array_equal(A2[h:, h:], A[h:, h:])
    assert not np.array_equal(A2[:h, :h], A[:h, :h])
    _, A2, B2, _ = S.run("AcR", R, A, B, C, depth=3)
    assert np.array_equal(A2, A)
    assert np.array_equal(B2[:h, :h], B[:h, :h]) and np.array_equal(B2[h:, h:], B[h:, h:])


# ---------------------------------------------------------------- planted
# mistakes: a wrong sign, a wrong location or a reordered row must be caught
def _mutants():
    t1 = list(S.TABLE1)
    yield "sign", [S.ADD("X", "S3", [(1, "A11"), (1, "A21")])] + t1[1:]
    r = list(t1)
    r[11] = S.MUL("C12", "P1", "T1", "a", "A11", "B11")  # P1 on top of P6
    yield "location", r
    r = list(t1)
    r[3], r[6] = r[6], r[3]  # S2 before S1 exists
    yield "order", r
    r = list(t1)
    r[21] = S.ADD("C11", "U1", [(1, "P1"), (1, "P4")])  # wrong operand (dead)
    yield "dead", r
    t9 = list(S.TABLE9)
    t9[18] = S.MUL("C21", "U3", "AcLR", "a", "S3", "T3", ("b", "U2"))  # beta instead of 1
    yield "t9coef", t9
    t3 = list(S.TABLE3)
    t3[7] = S.ADD("B11", "T2", [(1, "B22"), (-1, "T3")])  # T3 was clobbered by row 5
    yield "clobbered", t3


@pytest.mark.parametrize("label,table", list(_mutants()), ids=[m[0] for m in _mutants()])
def test_planted_mistakes_are_caught(label, table, monkeypatch):
    base = {"sign": "T1", "location": "T1", "order": "T1", "dead": "T1", "t9coef": "Acc", "clobbered": "IP"}[label]
    K = S.KINDS[base]
    monkeypatch.setitem(S.KINDS, base, S.Kind(table, K.accumulate, K.clobber, K.preserve, K.square))
    p = 65521
    R = ring.ModP(p)
    rng = np.random.default_rng(12)
    n = 8
    A, B, C = (rng.integers(0, p, (n, n)) for _ in range(3))
    try:
        out, _, _, _ = S.run(base, R, A, B, C, alpha=3, beta=5, depth=2)
    except S.ScheduleError:
        return
    assert not np.array_equal(out, _ref(base, A, B, C, 3, 5, R))


def test_counts_document_misprints():
    # Table 9's printed closed form does not solve its recurrence (n = 2: 14 vs 30)
    assert counts.W9_rec(2) == 30 and counts.W9_printed(2) != 30
    for n in (2, 4, 8, 16, 1024):
        assert counts.W9_rec(n) == counts.W9_solution(n)
        assert counts.W7_rec(n, 17) == counts.W7_closed(n)
    # Theorem 3 prints 16 additions for Table 7; only 17 gives the closed form
    assert counts.W7_rec(4, 16) != counts.W7_closed(4)
