"""Literal interpreter of the paper's memory schedules (Tables 1-9).

Each table is transcribed below as the list of its rows, in the printed
order, with the location column kept verbatim.  The interpreter executes
the rows on numpy views of the caller's matrices, so a row that writes into
"A21" really overwrites that quadrant of the caller's A, and a recursive call
really receives quadrant views of its operands.

While it runs it enforces the rules the tables rely on:
  * liveness: every operand a row names must be the value currently held by
    the location the schedule put it in (a value dies when its location is
    overwritten, or when a recursive call that may overwrite it returns);
  * clobbering: after a recursive call of a kind that may overwrite its
    inputs (IP, OvL, OvR, AcLR, AccR, AcR; Sections 5.1-5.3) the caller fills
    those inputs with garbage, so a schedule that relies on them fails;
  * aliasing: a product never writes over one of its own operands, and an
    addition writes either to a fresh location or exactly in place;
  * restoration: inputs a kind declares read-only are compared bit for bit
    before and after every call of that kind;
  * memory: temporaries X, Y, Z are allocated per recursion level and their
    element counts tracked (current, peak, and total allocations, Section 3
    and Theorem 3);
  * operation counts: scalar additions of the block additions, and the
    scalar operations of the classical leaves (C <- AB costs m n (2k - 1),
    C <- AB + C costs 2 m n k, so a 1x1 leaf costs 1 or 2 as in W(1)).

Row notation:
  ADD(loc, name, [(coef, value), ...])     loc <- sum coef * value
  MUL(loc, name, kind, acoef, left, right, acc)
        loc <- acoef * kind(left x right) [+ bcoef * value]   acc=(bcoef, value)
  COPY(loc, name, value)                   loc <- value
Coefficients: 1, -1, 'a' (the call's alpha), '-a', 'b' (the call's beta), '-b'.

Readings of garbled or ambiguous passages (all checked by the tests):
  * Table 6 prints row numbers 5 and 17 twice; the rows are taken in printed
    order (24 rows).
  * Table 9 row 19 "U3 = P7 + U2 = alpha AcLR(S3 T3 + U2)" is an AcLR call with
    alpha and accumulation coefficient +1 on C21 (which holds U2); row 24
    "U6 = U3 - P4 = -alpha AccR(A22 T4 - U3)" is an AccR call with -alpha and
    coefficient +1 on C21 (which holds U3).
  * Table 9 is run on square blocks: its rows 19 and 24 call the square-only
    schedules of Tables 6 and 7 (Section 5.3 states Tables 4-7 need equal
    sizes).
  * The modified OvL schedule of Section 5.1 inserts 18bis after row 18 and
    19bis after row 19, and replaces row 21 by an OvR call.

Test infrastructure only (see oracle/__init__.py).
"""
from __future__ import annotations

from collections import Counter
from dataclasses import dataclass, field

import numpy as np


# ----------------------------------------------------------------------------
# row constructors
# ----------------------------------------------------------------------------
def ADD(loc, name, terms):
    return ("add", loc, name, tuple(terms))


def MUL(loc, name, kind, acoef, left, right, acc=None):
    return ("mul", loc, name, kind, acoef, left, right, acc)


def COPY(loc, name, src):
    return ("copy", loc, name, src)


# ----------------------------------------------------------------------------
# Table 1 (Douglas et al.): C <- A B, two temporaries X, Y  (Section 3.1)
# ----------------------------------------------------------------------------
TABLE1 = [
    ADD("X", "S3", [(1, "A11"), (-1, "A21")]),
    ADD("Y", "T3", [(1, "B22"), (-1, "B12")]),
    MUL("C21", "P7", "T1", "a", "S3", "T3"),
    ADD("X", "S1", [(1, "A21"), (1, "A22")]),
    ADD("Y", "T1", [(1, "B12"), (-1, "B11")]),
    MUL("C22", "P5", "T1", "a", "S1", "T1"),
    ADD("X", "S2", [(1, "S1"), (-1, "A11")]),
    ADD("Y", "T2", [(1, "B22"), (-1, "T1")]),
    MUL("C12", "P6", "T1", "a", "S2", "T2"),
    ADD("X", "S4", [(1, "A12"), (-1, "S2")]),
    MUL("C11", "P3", "T1", "a", "S4", "B22"),
    MUL("X", "P1", "T1", "a", "A11", "B11"),
    ADD("C12", "U2", [(1, "P1"), (1, "P6")]),
    ADD("C21", "U3", [(1, "U2"), (1, "P7")]),
    ADD("C12", "U4", [(1, "U2"), (1, "P5")]),
    ADD("C22", "U7", [(1, "U3"), (1, "P5")]),
    ADD("C12", "U5", [(1, "U4"), (1, "P3")]),
    ADD("Y", "T4", [(1, "T2"), (-1, "B21")]),
    MUL("C11", "P4", "T1", "a", "A22", "T4"),
    ADD("C21", "U6", [(1, "U3"), (-1, "P4")]),
    MUL("C11", "P2", "T1", "a", "A12", "B21"),
    ADD("C11", "U1", [(1, "P1"), (1, "P2")]),
]

# ----------------------------------------------------------------------------
# Table 2 (Huss-Lederman et al.): C <- alpha A B + beta C, temporaries X,Y,Z
# ----------------------------------------------------------------------------
TABLE2 = [
    ADD("X", "S1", [(1, "A21"), (1, "A22")]),
    ADD("Y", "T1", [(1, "B12"), (-1, "B11")]),
    MUL("Z", "P5", "T1", "a", "S1", "T1"),
    ADD("C22", "C22b", [(1, "P5"), ("b", "C22")]),
    ADD("C12", "C12b", [(1, "P5"), ("b", "C12")]),
    ADD("X", "S2", [(1, "S1"), (-1, "A11")]),
    ADD("Y", "T2", [(1, "B22"), (-1, "T1")]),
    MUL("Z", "P1", "T1", "a", "A11", "B11"),
    ADD("C11", "C11b", [(1, "P1"), ("b", "C11")]),
    MUL("Z", "U2", "T2", "a", "S2", "T2", (1, "P1")),
    MUL("C11", "U1", "T2", "a", "A12", "B21", (1, "C11b")),
    ADD("X", "S4", [(1, "A12"), (-1, "S2")]),
    ADD("Y", "T4", [(1, "T2"), (-1, "B21")]),
    MUL("C12", "C12c", "T2", "a", "S4", "B22", (1, "C12b")),
    ADD("C12", "U5", [(1, "U2"), (1, "C12c")]),
    MUL("C21", "P4b", "T2", "a", "A22", "T4", ("-b", "C21")),
    ADD("X", "S3", [(1, "A11"), (-1, "A21")]),
    ADD("Y", "T3", [(1, "B22"), (-1, "B12")]),
    MUL("Z", "U3", "T2", "a", "S3", "T3", (1, "U2")),
    ADD("C22", "U7", [(1, "U3"), (1, "C22b")]),
    ADD("C21", "U6", [(1, "U3"), (-1, "P4b")]),
]

# ----------------------------------------------------------------------------
# Table 3 (IP): C <- A B in place, overwrites A and B, no temporary (Sec. 5.1)
# ----------------------------------------------------------------------------
TABLE3 = [
    ADD("C11", "S3", [(1, "A11"), (-1, "A21")]),
    ADD("A21", "S1", [(1, "A21"), (1, "A22")]),
    ADD("C22", "T1", [(1, "B12"), (-1, "B11")]),
    ADD("B12", "T3", [(1, "B22"), (-1, "B12")]),
    MUL("C21", "P7", "IP", "a", "S3", "T3"),
    ADD("C12", "S2", [(1, "S1"), (-1, "A11")]),
    MUL("C11", "P1", "IP", "a", "A11", "B11"),
    ADD("B11", "T2", [(1, "B22"), (-1, "T1")]),
    MUL("A11", "P5", "IP", "a", "S1", "T1"),
    ADD("C22", "T4", [(1, "T2"), (-1, "B21")]),
    MUL("A21", "P4", "IP", "a", "A22", "T4"),
    ADD("A22", "S4", [(1, "A12"), (-1, "S2")]),
    MUL("C22", "P6", "IP", "a", "S2", "T2"),
    ADD("C22", "U2", [(1, "P1"), (1, "P6")]),
    MUL("C12", "P2", "IP", "a", "A12", "B21"),
    ADD("C11", "U1", [(1, "P1"), (1, "P2")]),
    ADD("C12", "U4", [(1, "U2"), (1, "P5")]),
    ADD("C22", "U3", [(1, "U2"), (1, "P7")]),
    ADD("C21", "U6", [(1, "U3"), (-1, "P4")]),
    ADD("C22", "U7", [(1, "U3"), (1, "P5")]),
    MUL("A12", "P3", "IP", "a", "S4", "B22"),
    ADD("C12", "U5", [(1, "U4"), (1, "P3")]),
]

# ----------------------------------------------------------------------------
# Table 4 (OvL): C <- A B overwriting A, one temporary X (Section 5.1)
# ----------------------------------------------------------------------------
TABLE4 = [
    ADD("C22", "S3", [(1, "A11"), (-1, "A21")]),
    ADD("A21", "S1", [(1, "A21"), (1, "A22")]),
    ADD("C12", "S2", [(1, "S1"), (-1, "A11")]),
    ADD("C21", "T1", [(1, "B12"), (-1, "B11")]),
    MUL("C11", "P1", "OvL", "a", "A11", "B11"),
    ADD("A11", "T3", [(1, "B22"), (-1, "B12")]),
    MUL("X", "P7", "IP", "a", "S3", "T3"),
    ADD("A11", "T2", [(1, "B22"), (-1, "T1")]),
    MUL("C22", "P5", "IP", "a", "S1", "T1"),
    ADD("C21", "S4", [(1, "A12"), (-1, "S2")]),
    MUL("A21", "P3", "OvL", "a", "S4", "B22"),
    MUL("C21", "P6", "OvL", "a", "S2", "T2"),
    ADD("A11", "T4", [(1, "T2"), (-1, "B21")]),
    ADD("C21", "U2", [(1, "P1"), (1, "P6")]),
    ADD("C12", "U4", [(1, "U2"), (1, "P5")]),
    ADD("C21", "U3", [(1, "U2"), (1, "P7")]),
    ADD("C22", "U7", [(1, "U3"), (1, "P5")]),
    ADD("C12", "U5", [(1, "U4"), (1, "P3")]),
    MUL("X", "P2", "OvL", "a", "A12", "B21"),
    ADD("C11", "U1", [(1, "P1"), (1, "P2")]),
    MUL("A21", "P4", "IP", "a", "A22", "T4"),
    ADD("C21", "U6", [(1, "U3"), (-1, "P4")]),
]

# Section 5.1 variant of Table 4 that overwrites only A11 and A21: a copy of
# A12 is parked in A21 (18bis) before the OvL call of row 19 destroys A12,
# restored right after (19bis), and row 21 calls OvR instead of IP.
TABLE4M = [
    ADD("C22", "S3", [(1, "A11"), (-1, "A21")]),
    ADD("A21", "S1", [(1, "A21"), (1, "A22")]),
    ADD("C12", "S2", [(1, "S1"), (-1, "A11")]),
    ADD("C21", "T1", [(1, "B12"), (-1, "B11")]),
    MUL("C11", "P1", "OvLM", "a", "A11", "B11"),
    ADD("A11", "T3", [(1, "B22"), (-1, "B12")]),
    MUL("X", "P7", "IP", "a", "S3", "T3"),
    ADD("A11", "T2", [(1, "B22"), (-1, "T1")]),
    MUL("C22", "P5", "IP", "a", "S1", "T1"),
    ADD("C21", "S4", [(1, "A12"), (-1, "S2")]),
    MUL("A21", "P3", "OvLM", "a", "S4", "B22"),
    MUL("C21", "P6", "OvLM", "a", "S2", "T2"),
    ADD("A11", "T4", [(1, "T2"), (-1, "B21")]),
    ADD("C21", "U2", [(1, "P1"), (1, "P6")]),
    ADD("C12", "U4", [(1, "U2"), (1, "P5")]),
    ADD("C21", "U3", [(1, "U2"), (1, "P7")]),
    ADD("C22", "U7", [(1, "U3"), (1, "P5")]),
    ADD("C12", "U5", [(1, "U4"), (1, "P3")]),
    COPY("A21", "A12c", "A12"),                       # 18bis
    MUL("X", "P2", "OvLM", "a", "A12", "B21"),
    COPY("A12", "A12", "A12c"),                       # 19bis
    ADD("C11", "U1", [(1, "P1"), (1, "P2")]),
    MUL("A21", "P4", "OvR", "a", "A22", "T4"),        # row 21 with OvR
    ADD("C21", "U6", [(1, "U3"), (-1, "P4")]),
]

# ----------------------------------------------------------------------------
# Table 5 (OvR): C <- A B overwriting B, one temporary X (Section 5.1)
# ----------------------------------------------------------------------------
TABLE5 = [
    ADD("C22", "S3", [(1, "A11"), (-1, "A21")]),
    ADD("C21", "S1", [(1, "A21"), (1, "A22")]),
    ADD("C12", "T1", [(1, "B12"), (-1, "B11")]),
    MUL("C11", "P1", "OvR", "a", "A11", "B11"),
    ADD("B11", "S2", [(1, "S1"), (-1, "A11")]),
    ADD("B12", "T3", [(1, "B22"), (-1, "B12")]),
    MUL("X", "P7", "IP", "a", "S3", "T3"),
    ADD("B12", "T2", [(1, "B22"), (-1, "T1")]),
    MUL("C22", "P5", "IP", "a", "S1", "T1"),
    ADD("C12", "T4", [(1, "T2"), (-1, "B21")]),
    MUL("C21", "P6", "OvR", "a", "S2", "T2"),
    MUL("B12", "P4", "OvR", "a", "A22", "T4"),
    ADD("B11", "S4", [(1, "A12"), (-1, "S2")]),
    ADD("C21", "U2", [(1, "P1"), (1, "P6")]),
    ADD("C12", "U4", [(1, "U2"), (1, "P5")]),
    ADD("C21", "U3", [(1, "U2"), (1, "P7")]),
    ADD("C22", "U7", [(1, "U3"), (1, "P5")]),
    ADD("C21", "U6", [(1, "U3"), (-1, "P4")]),
    MUL("B12", "P3", "IP", "a", "S4", "B22"),
    ADD("C12", "U5", [(1, "U4"), (1, "P3")]),
    MUL("B12", "P2", "OvR", "a", "A12", "B21"),
    ADD("C11", "U1", [(1, "P1"), (1, "P2")]),
]

# ----------------------------------------------------------------------------
# Table 6 (AcLR): C <- alpha A B + beta C overwriting A and B, temps X, Y
# ----------------------------------------------------------------------------
TABLE6 = [
    ADD("C22", "Z1", [(1, "C22"), (-1, "C12")]),
    ADD("X", "S1", [(1, "A21"), (1, "A22")]),
    ADD("Y", "T1", [(1, "B12"), (-1, "B11")]),
    ADD("C21", "Z2", [(1, "C21"), (-1, "Z1")]),
    ADD("B12", "T3", [(1, "B22"), (-1, "B12")]),
    ADD("A21", "S3", [(1, "A11"), (-1, "A21")]),
    MUL("C22", "P7b", "AcLR", "a", "S3", "T3", ("b", "Z1")),
    ADD("A21", "S2", [(1, "S1"), (-1, "A11")]),
    ADD("B12", "T2", [(1, "B22"), (-1, "T1")]),
    MUL("C12", "P5b", "AcLR", "a", "S1", "T1", ("b", "C12")),
    MUL("Y", "P1", "IP", "a", "A11", "B11"),
    ADD("X", "T4", [(1, "T2"), (-1, "B21")]),
    MUL("C21", "P4b", "AcLR", "a", "A22", "T4", ("-b", "Z2")),
    ADD("A22", "S4", [(1, "A12"), (-1, "S2")]),
    MUL("X", "P6", "IP", "a", "S2", "T2"),
    MUL("C11", "P2b", "AcLR", "a", "A12", "B21", ("b", "C11")),
    ADD("C11", "U1", [(1, "P1"), (1, "P2b")]),
    ADD("X", "U2", [(1, "P1"), (1, "P6")]),
    ADD("C22", "U3", [(1, "U2"), (1, "P7b")]),
    ADD("X", "U4", [(1, "U2"), (1, "P5b")]),
    ADD("C21", "U6", [(1, "U3"), (-1, "P4b")]),
    ADD("C22", "U7", [(1, "U3"), (1, "P5b")]),
    MUL("C12", "P3", "IP", "a", "S4", "B22"),
    ADD("C12", "U5", [(1, "U4"), (1, "P3")]),
]

# ----------------------------------------------------------------------------
# Table 7 (AccR): C <- alpha A B + beta C overwriting B, temps X, Y
# ----------------------------------------------------------------------------
TABLE7 = [
    ADD("C22", "Z1", [(1, "C22"), (-1, "C12")]),
    ADD("X", "T1", [(1, "B12"), (-1, "B11")]),
    ADD("C21", "Z2", [(1, "C21"), (-1, "Z1")]),
    ADD("B12", "T3", [(1, "B22"), (-1, "B12")]),
    ADD("Y", "S3", [(1, "A11"), (-1, "A21")]),
    MUL("C22", "P7b", "AccR", "a", "S3", "T3", ("b", "Z1")),
    ADD("Y", "S1", [(1, "A21"), (1, "A22")]),
    ADD("B12", "T2", [(1, "B22"), (-1, "T1")]),
    MUL("C12", "P5b", "AccR", "a", "S1", "T1", ("b", "C12")),
    ADD("X", "T4", [(1, "T2"), (-1, "B21")]),
    MUL("C21", "P4b", "AccR", "a", "A22", "T4", ("-b", "Z2")),
    MUL("X", "P1", "OvR", "a", "A11", "B11"),
    MUL("C11", "P2b", "AccR", "a", "A12", "B21", ("b", "C11")),
    ADD("Y", "S2", [(1, "S1"), (-1, "A11")]),
    MUL("B21", "P6", "OvR", "a", "S2", "T2"),
    ADD("Y", "S4", [(1, "A12"), (-1, "S2")]),
    ADD("B21", "U2", [(1, "P1"), (1, "P6")]),
    ADD("C22", "U3", [(1, "U2"), (1, "P7b")]),
    ADD("B21", "U4", [(1, "U2"), (1, "P5b")]),
    ADD("C21", "U6", [(1, "U3"), (-1, "P4b")]),
    ADD("C11", "U1", [(1, "P1"), (1, "P2b")]),
    ADD("C22", "U7", [(1, "U3"), (1, "P5b")]),
    MUL("C12", "P3", "IP", "a", "S4", "B22"),
    ADD("C12", "U5", [(1, "U4"), (1, "P3")]),
]

# ----------------------------------------------------------------------------
# Table 8 (AcR): rectangular C <- alpha A B + beta C overwriting B12, B21
# ----------------------------------------------------------------------------
TABLE8 = [
    ADD("C22", "Z1", [(1, "C22"), (-1, "C12")]),
    ADD("X", "T1", [(1, "B12"), (-1, "B11")]),
    ADD("C21", "Z2", [(1, "C21"), (-1, "Z1")]),
    ADD("B12", "T3", [(1, "B22"), (-1, "B12")]),
    ADD("Y", "S3", [(1, "A11"), (-1, "A21")]),
    MUL("C22", "P7b", "AcR", "a", "S3", "T3", ("b", "Z1")),
    ADD("Y", "S1", [(1, "A21"), (1, "A22")]),
    ADD("B12", "T2", [(1, "B22"), (-1, "T1")]),
    MUL("C12", "P5b", "AcR", "a", "S1", "T1", ("b", "C12")),
    ADD("X", "T4", [(1, "T2"), (-1, "B21")]),
    MUL("C21", "P4b", "AcR", "a", "A22", "T4", ("-b", "Z2")),
    MUL("X", "P1", "T1", "a", "A11", "B11"),
    MUL("C11", "P2b", "AcR", "a", "A12", "B21", ("b", "C11")),
    ADD("C11", "U1", [(1, "P1"), (1, "P2b")]),
    ADD("Y", "S2", [(1, "S1"), (-1, "A11")]),
    MUL("X", "U2", "AcR", "a", "S2", "T2", (1, "P1")),
    ADD("C22", "U3", [(1, "U2"), (1, "P7b")]),
    ADD("C21", "U6", [(1, "U3"), (-1, "P4b")]),
    ADD("C22", "U7", [(1, "U3"), (1, "P5b")]),
    ADD("X", "U4", [(1, "U2"), (1, "P5b")]),
    ADD("Y", "S4", [(1, "A12"), (-1, "S2")]),
    MUL("C12", "P3", "T1", "a", "S4", "B22"),
    ADD("C12", "U5", [(1, "U4"), (1, "P3")]),
]

# ----------------------------------------------------------------------------
# Table 9 (Acc): C <- alpha A B + beta C, read-only A and B, temps X, Y (Sec 6)
# ----------------------------------------------------------------------------
TABLE9 = [
    ADD("C22", "Z1", [(1, "C22"), (-1, "C12")]),
    ADD("C12", "Z3", [(1, "C12"), (-1, "C21")]),
    ADD("X", "S1", [(1, "A21"), (1, "A22")]),
    ADD("Y", "T1", [(1, "B12"), (-1, "B11")]),
    MUL("C12", "P5b", "Acc", "a", "S1", "T1", ("b", "Z3")),
    ADD("X", "S2", [(1, "S1"), (-1, "A11")]),
    ADD("Y", "T2", [(1, "B22"), (-1, "T1")]),
    MUL("C21", "P6b", "Acc", "a", "S2", "T2", ("b", "C21")),
    ADD("X", "S4", [(1, "A12"), (-1, "S2")]),
    ADD("C22", "W1", [(1, "P5b"), ("b", "Z1")]),
    MUL("C12", "P3c", "Acc", "a", "S4", "B22", (1, "P5b")),
    MUL("X", "P1", "T1", "a", "A11", "B11"),
    ADD("C21", "U2", [(1, "P6b"), (1, "P1")]),
    MUL("C11", "P2b", "Acc", "a", "A12", "B21", ("b", "C11")),
    ADD("C11", "U1", [(1, "P1"), (1, "P2b")]),
    ADD("C12", "U5", [(1, "U2"), (1, "P3c")]),
    ADD("X", "S3", [(1, "A11"), (-1, "A21")]),
    ADD("Y", "T3", [(1, "B22"), (-1, "B12")]),
    MUL("C21", "U3", "AcLR", "a", "S3", "T3", (1, "U2")),
    ADD("C22", "U7", [(1, "U3"), (1, "W1")]),
    ADD("Y", "T1p", [(1, "B12"), (-1, "B11")]),
    ADD("Y", "T2p", [(1, "B22"), (-1, "T1p")]),
    ADD("Y", "T4", [(1, "T2p"), (-1, "B21")]),
    MUL("C21", "U6", "AccR", "-a", "A22", "T4", (1, "U3")),
]


@dataclass(frozen=True)
class Kind:
    table: list
    accumulate: bool          # C <- alpha AB + beta C  (else C <- alpha AB)
    clobber: frozenset        # operand blocks the kind may overwrite
    preserve: frozenset       # operand blocks it must leave bit-identical
    square: bool              # the table needs m = k = n (Section 5.3)


_ALL_L = frozenset({"L11", "L12", "L21", "L22"})
_ALL_R = frozenset({"R11", "R12", "R21", "R22"})

KINDS = {
    "T1": Kind(TABLE1, False, frozenset(), _ALL_L | _ALL_R, False),
    "T2": Kind(TABLE2, True, frozenset(), _ALL_L | _ALL_R, False),
    "IP": Kind(TABLE3, False, _ALL_L | _ALL_R, frozenset(), False),
    "OvL": Kind(TABLE4, False, _ALL_L, _ALL_R, True),
    "OvLM": Kind(TABLE4M, False, frozenset({"L11", "L21"}), _ALL_R | {"L12", "L22"}, True),
    "OvR": Kind(TABLE5, False, _ALL_R, _ALL_L, True),
    "AcLR": Kind(TABLE6, True, _ALL_L | _ALL_R, frozenset(), True),
    "AccR": Kind(TABLE7, True, _ALL_R, _ALL_L, True),
    "AcR": Kind(TABLE8, True, frozenset({"R12", "R21"}), _ALL_L | {"R11", "R22"}, False),
    "Acc": Kind(TABLE9, True, frozenset(), _ALL_L | _ALL_R, True),
}

# Final value names expected in the four quadrants of C after every table.
FINAL = {"C11": "U1", "C12": "U5", "C21": "U6", "C22": "U7"}


class ScheduleError(AssertionError):
    """A schedule read a dead value, aliased, or broke a declared property."""


# ----------------------------------------------------------------------------
# temporaries
# ----------------------------------------------------------------------------
@dataclass
class Stats:
    adds: int = 0             # scalar additions of the block additions
    leaf_ops: int = 0         # scalar operations of classical leaves
    copies: int = 0           # scalar copies (modified OvL only)
    cur_tmp: int = 0          # elements of temporaries currently allocated
    peak_tmp: int = 0         # maximum of cur_tmp
    total_alloc: int = 0      # sum of all temporary allocations
    carved: int = 0           # elements carved from caller-provided scratch
    calls: Counter = field(default_factory=Counter)
    leaves: int = 0

    @property
    def ops(self) -> int:
        return self.adds + self.leaf_ops


class HeapArena:
    """Fresh temporaries for every recursion level (counted in Stats)."""

    def __init__(self, ring, stats, rng):
        self.ring, self.stats, self.rng = ring, stats, rng

    def level(self, shapes: dict):
        tmps = {}
        for name, shp in shapes.items():
            tmps[name] = self.ring.poison(self.rng, shp).astype(self.ring.dtype)
            sz = int(shp[0]) * int(shp[1])
            self.stats.cur_tmp += sz
            self.stats.total_alloc += sz
        self.stats.peak_tmp = max(self.stats.peak_tmp, self.stats.cur_tmp)
        return tmps, self

    def release(self, tmps):
        for t in tmps.values():
            self.stats.cur_tmp -= t.shape[0] * t.shape[1]


class CarveArena:
    """Temporaries carved from a caller-provided block (Algorithm 2 uses C22).

    A level's temporaries take the quadrants 11, 12, 21 of the block, in that
    order; deeper levels carve from quadrant 22.  Nothing is allocated."""

    def __init__(self, view, ring, stats, rng):
        self.view, self.ring, self.stats, self.rng = view, ring, stats, rng

    def level(self, shapes: dict):
        R, Cc = self.view.shape
        hr, hc = R // 2, Cc // 2
        quads = [self.view[:hr, :hc], self.view[:hr, hc:2 * hc], self.view[hr:2 * hr, :hc]]
        if len(shapes) > 3:
            raise ScheduleError("more than three temporaries per level")
        tmps = {}
        for (name, shp), q in zip(shapes.items(), quads):
            if shp[0] > q.shape[0] or shp[1] > q.shape[1]:
                raise ScheduleError(f"temporary {name}{shp} does not fit in scratch quadrant {q.shape}")
            t = q[: shp[0], : shp[1]]
            t[...] = self.ring.poison(self.rng, t.shape)
            tmps[name] = t
            self.stats.carved += shp[0] * shp[1]
        return tmps, CarveArena(self.view[hr:2 * hr, hc:2 * hc], self.ring, self.stats, self.rng)

    def release(self, tmps):
        pass


# ----------------------------------------------------------------------------
# interpreter
# ----------------------------------------------------------------------------
def _same_region(a: np.ndarray, b: np.ndarray) -> bool:
    return (a.__array_interface__["data"][0] == b.__array_interface__["data"][0]
            and a.shape == b.shape and a.strides == b.strides)


def _quads(M):
    r, c = M.shape[0] // 2, M.shape[1] // 2
    return {"11": M[:r, :c], "12": M[:r, c:2 * c], "21": M[r:2 * r, :c], "22": M[r:2 * r, c:2 * c]}


def _value_shapes(table, m, k, n):
    """Shape of every value of a table and bounding shape of every temporary."""
    h = {"A": (m // 2, k // 2), "B": (k // 2, n // 2), "C": (m // 2, n // 2)}
    shp = {f"{M}{i}{j}": h[M] for M in "ABC" for i in "12" for j in "12"}
    tmp = {}

    def get(v):
        if v not in shp:
            raise ScheduleError(f"value {v} is used before it is computed")
        return shp[v]

    for row in table:
        if row[0] == "add":
            _, loc, name, terms = row
            s = {get(v) for _, v in terms}
            if len(s) != 1:
                raise ScheduleError(f"{name}: operands of different shapes {s}")
            shp[name] = s.pop()
        elif row[0] == "mul":
            _, loc, name, kind, ac, left, right, acc = row
            if get(left)[1] != get(right)[0]:
                raise ScheduleError(f"{name}: inner dimensions differ")
            shp[name] = (shp[left][0], shp[right][1])
        else:
            _, loc, name, src = row
            shp[name] = get(src)
        if loc in ("X", "Y", "Z"):
            old = tmp.get(loc, (0, 0))
            tmp[loc] = (max(old[0], shp[name][0]), max(old[1], shp[name][1]))
    return shp, dict(sorted(tmp.items()))


class Interpreter:
    def __init__(self, ring, *, seed: int = 12345, poison: bool = True):
        self.ring = ring
        self.rng = np.random.default_rng(seed)
        self.poison = poison
        self.stats = Stats()

    # -- leaf ------------------------------------------------------------
    def leaf(self, alpha, beta, L, R, D):
        m, k = L.shape
        n = R.shape[1]
        prod = self.ring.matmul(L, R)
        if beta is None:
            D[...] = self.ring.lincomb([(alpha, prod)])
            self.stats.leaf_ops += m * n * (2 * k - 1)
        else:
            D[...] = self.ring.lincomb([(alpha, prod), (beta, D.copy())])
            self.stats.leaf_ops += 2 * m * n * k
        self.stats.leaves += 1

    # -- one call ----------------------------------------------------------
    def call(self, kind: str, alpha, beta, L, R, D, depth: int, arena=None):
        """D <- alpha L R (+ beta D) by schedule `kind`, `depth` Winograd levels."""
        K = KINDS[kind]
        if K.accumulate != (beta is not None):
            raise ScheduleError(f"{kind}: accumulate flag mismatch")
        m, k = L.shape
        k2, n = R.shape
        if k != k2 or D.shape != (m, n):
            raise ScheduleError("shape mismatch")
        if np.shares_memory(D, L) or np.shares_memory(D, R):
            raise ScheduleError("product destination aliases an operand")
        self.stats.calls[kind] += 1
        arena = arena or HeapArena(self.ring, self.stats, self.rng)
        keep = {b: (L if b[0] == "L" else R) for b in K.preserve}
        snap = {b: _quads(v)[b[1:]].copy() for b, v in keep.items()
                if v.shape[0] % 2 == 0 and v.shape[1] % 2 == 0}
        splittable = depth > 0 and min(m, k, n) >= 2 and m % 2 == 0 and k % 2 == 0 and n % 2 == 0
        if splittable and K.square and not (m == k == n):
            raise ScheduleError(f"{kind} needs square operands, got {m}x{k}x{n}")
        if not splittable:
            self.leaf(alpha, beta, L, R, D)
        else:
            self._table(kind, K, alpha, beta, L, R, D, depth, arena)
        for b, s in snap.items():
            if not np.array_equal(_quads(keep[b])[b[1:]], s, equal_nan=True):
                raise ScheduleError(f"{kind} modified read-only block {b}")

    def _table(self, kind, K, alpha, beta, L, R, D, depth, arena):
        ring = self.ring
        m, k = L.shape
        n = R.shape[1]
        shapes, tshapes = _value_shapes(K.table, m, k, n)
        tmps, sub_arena = arena.level(tshapes)
        loc = {}
        for M, V in (("A", L), ("B", R), ("C", D)):
            for q, v in _quads(V).items():
                loc[M + q] = v
        loc.update(tmps)
        # which value each location holds; C is garbage for C <- AB kinds
        holds = {f"{M}{i}{j}": f"{M}{i}{j}" for M in "AB" for i in "12" for j in "12"}
        for q in ("C11", "C12", "C21", "C22"):
            if K.accumulate:
                holds[q] = q
            else:
                holds[q] = None
                if self.poison:
                    loc[q][...] = ring.poison(self.rng, loc[q].shape)
        for t in tmps:
            holds[t] = None
        where = {v: l for l, v in holds.items() if v is not None}

        def coef(c):
            if c == "a":
                return alpha
            if c == "-a":
                return -alpha
            if c == "b":
                return beta
            if c == "-b":
                return -beta
            return c

        def view_of(name):
            if name not in where:
                raise ScheduleError(f"{kind}: read of dead or unknown value {name}")
            l = where[name]
            r, c = shapes[name]
            return loc[l][:r, :c]

        def store_target(l, name):
            r, c = shapes[name]
            if r > loc[l].shape[0] or c > loc[l].shape[1]:
                raise ScheduleError(f"{kind}: {name}{shapes[name]} does not fit in {l}{loc[l].shape}")
            return loc[l][:r, :c]

        def set_holder(l, name):
            old = holds.get(l)
            if old is not None and where.get(old) == l:
                del where[old]
            holds[l] = name
            where[name] = l

        def kill(l):
            old = holds.get(l)
            if old is not None and where.get(old) == l:
                del where[old]
            holds[l] = None

        for row in K.table:
            op = row[0]
            if op == "add":
                _, l, name, terms = row
                views = [view_of(v) for _, v in terms]
                dst = store_target(l, name)
                for v in views:
                    if np.shares_memory(dst, v) and not _same_region(dst, v):
                        raise ScheduleError(f"{kind}: {name} partially overlaps an operand")
                val = ring.lincomb([(coef(c), v) for (c, _), v in zip(terms, views)])
                dst[...] = val
                self.stats.adds += dst.size
                set_holder(l, name)
            elif op == "copy":
                _, l, name, src = row
                v = view_of(src)
                dst = store_target(l, name)
                if np.shares_memory(dst, v):
                    raise ScheduleError(f"{kind}: copy onto itself")
                dst[...] = v
                self.stats.copies += dst.size
                set_holder(l, name)
            else:
                _, l, name, sub, ac, left, right, acc = row
                Lv, Rv = view_of(left), view_of(right)
                dst = store_target(l, name)
                sub_beta = None
                if acc is not None:
                    bc, accv = acc
                    if where.get(accv) != l:
                        raise ScheduleError(f"{kind}: {name} accumulates into {l} which does not hold {accv}")
                    if view_of(accv).shape != dst.shape:
                        raise ScheduleError(f"{kind}: accumulation shape mismatch")
                    sub_beta = coef(bc)
                elif KINDS[sub].accumulate:
                    raise ScheduleError(f"{kind}: {sub} call without accumulation input")
                self.call(sub, coef(ac), sub_beta, Lv, Rv, dst, depth - 1, sub_arena)
                # the callee may have overwritten some operand blocks
                S = KINDS[sub]
                for side, V, vname in (("L", Lv, left), ("R", Rv, right)):
                    blocks = [b for b in S.clobber if b[0] == side]
                    if not blocks:
                        continue
                    if self.poison and V.shape[0] % 2 == 0 and V.shape[1] % 2 == 0:
                        qv = _quads(V)
                        for b in blocks:
                            qv[b[1:]][...] = ring.poison(self.rng, qv[b[1:]].shape)
                    if vname in where:
                        kill(where[vname])
                set_holder(l, name)
        for q, final in FINAL.items():
            if holds.get(q) != final:
                raise ScheduleError(f"{kind}: {q} ends holding {holds.get(q)}, expected {final}")
        arena.release(tmps)


def run(kind: str, ring, A, B, C=None, *, alpha=1, beta=None, depth: int = 1,
        seed: int = 12345, poison: bool = True):
    """Run schedule `kind` on copies of A, B (and C); return (C_out, A_after,
    B_after, stats).  A and B come back as the schedule left them, which
    matters for the overwriting kinds."""
    K = KINDS[kind]
    A = np.array(A, dtype=ring.dtype, copy=True)
    B = np.array(B, dtype=ring.dtype, copy=True)
    m, n = A.shape[0], B.shape[1]
    if K.accumulate:
        if beta is None:
            beta = 1
        D = np.array(C, dtype=ring.dtype, copy=True)
    else:
        D = ring.zeros((m, n))
        beta = None
    it = Interpreter(ring, seed=seed, poison=poison)
    it.call(kind, ring.scalar(alpha), None if beta is None else ring.scalar(beta), A, B, D, depth)
    return ring.canon(D), A, B, it.stats
