"""Schedules found by the pebble-game search (Section 4) that the library
ships as data, each with the search spec that finds it again.

A schedule here is a one-level table in the row form of search.py; it runs
through search.set_schedule and Opts(sched=swmm.CUSTOM), which replay it
under its contract before use.  regenerate(name) runs the search with the
stored spec (tens of seconds for the accumulating ones), so the data can be
checked against the search that produced it.

  acc16  C <- alpha AB + beta C, A and B read-only, two temporaries (Table
         9's contract), 16 block additions against Table 9's 17: operand
         T2 is formed again from T3 in one addition (Table 9 forms T1 and
         T2 again, two additions), and no call overwrites both operands.
         The search is restricted to Table 9's intermediate values.
  ab12   C <- alpha AB, A and B read-only, two temporaries (Table 1's
         contract), 12 block additions against Table 1's 15: three products
         are Table 2 calls that accumulate into their destination.
  aclr14 C <- alpha AB + beta C overwriting A and B, two temporaries (Table
         6's contract), 14 block additions against Table 6's 17.
  accr14 C <- alpha AB + beta C overwriting B, two temporaries (Table 7's
         contract), 14 block additions against Table 7's 17.
The last two are found at run time (a few seconds).
"""
from __future__ import annotations

from . import search as Q
from . import swmm

_AB = ("A11", "A12", "A21", "A22", "B11", "B12", "B21", "B22")
# Table 9's intermediate values are kept; the other accumulating tables'
# ones are excluded from the search for acc16
_NOT_TABLE9 = ("Z2", "P5+bC22", "P5+bC12", "P1+bC11", "P3+P5+bC12", "P4-bC21", "P7+bC22-bC12",
               "P4-bC21+bC22-bC12", "P1+P6+P7+bC22-bC12", "P1+P6+P5+bC12")

FOUND = {
    "acc16": dict(
        spec=dict(accumulate=True, preserve=_AB, temps=2,
                  kinds=(swmm.T1_DHSS, Q.SELF, swmm.T6_ACLR, swmm.T7_ACCR), recompute=True),
        search=dict(max_rows=24, max_adds=16, exclude=_NOT_TABLE9, max_states=1 << 25),
        # (op, dst, s1, s2, coef, accumulate, sign, kind)
        rows=[
            (Q.ADD, "X", "A21", "A22", 1, False, 1, 0),          # S1
            (Q.ADD, "Y", "B12", "B11", -1, False, 1, 0),         # T1
            (Q.ADD, "C22", "C22", "C12", -1, False, 1, 0),       # Z1
            (Q.ADD, "C12", "C12", "C21", -1, False, 1, 0),       # Z3
            (Q.MUL, "C11", "A12", "B21", "b", True, 1, Q.SELF),  # P2 + b C11
            (Q.MUL, "C12", "X", "Y", "b", True, 1, Q.SELF),      # P5 + b Z3
            (Q.ADD, "X", "X", "A11", -1, False, 1, 0),           # S2
            (Q.ADD, "Y", "B22", "Y", -1, False, 1, 0),           # T2
            (Q.MUL, "C21", "X", "Y", "b", True, 1, swmm.T7_ACCR),  # P6 + b C21
            (Q.ADD, "Y", "A11", "A21", -1, False, 1, 0),         # S3
            (Q.ADD, "X", "A12", "X", -1, False, 1, 0),           # S4
            (Q.ADD, "C22", "C12", "C22", "b", False, 1, 0),      # W1 = P5 + b C22 - b C21
            (Q.MUL, "C12", "X", "B22", 1, True, 1, Q.SELF),      # P3 + P5 + b Z3
            (Q.MUL, "X", "A11", "B11", 1, False, 1, swmm.T1_DHSS),  # P1
            (Q.ADD, "C21", "X", "C21", 1, False, 1, 0),          # P1 + P6 + b C21
            (Q.ADD, "C11", "X", "C11", 1, False, 1, 0),          # U1
            (Q.ADD, "X", "B22", "B12", -1, False, 1, 0),         # T3
            (Q.ADD, "C12", "C12", "C21", 1, False, 1, 0),        # U5
            (Q.MUL, "C21", "Y", "X", 1, True, 1, Q.SELF),        # P1 + P6 + P7 + b C21
            (Q.ADD, "X", "B11", "X", 1, False, 1, 0),            # T2 again, from T3
            (Q.ADD, "X", "X", "B21", -1, False, 1, 0),           # T4
            (Q.ADD, "C22", "C22", "C21", 1, False, 1, 0),        # U7
            (Q.MUL, "C21", "A22", "X", 1, True, -1, swmm.T7_ACCR),  # U6
        ]),
    "ab12": dict(
        spec=dict(accumulate=False, preserve=_AB, temps=2, kinds=(Q.SELF, swmm.T2_HLJJTT)),
        search=dict(max_adds=12),
        rows=[
            (Q.ADD, "C11", "A21", "A22", 1, False, 1, 0),        # S1
            (Q.ADD, "C12", "C11", "A11", -1, False, 1, 0),       # S2
            (Q.ADD, "C21", "A11", "A21", -1, False, 1, 0),       # S3
            (Q.ADD, "X", "A12", "C12", -1, False, 1, 0),         # S4
            (Q.ADD, "Y", "B12", "B11", -1, False, 1, 0),         # T1
            (Q.MUL, "C22", "C11", "Y", 1, False, 1, Q.SELF),     # P5
            (Q.ADD, "C11", "B22", "B12", -1, False, 1, 0),       # T3
            (Q.MUL, "Y", "C21", "C11", 1, False, 1, Q.SELF),     # P7
            (Q.ADD, "C11", "B11", "C11", 1, False, 1, 0),        # T2 = B11 + T3
            (Q.MUL, "C21", "C12", "C11", 1, False, 1, Q.SELF),   # P6
            (Q.ADD, "C12", "C11", "B21", -1, False, 1, 0),       # T4
            (Q.MUL, "C11", "A11", "B11", 1, False, 1, Q.SELF),   # P1
            (Q.ADD, "C21", "C11", "C21", 1, False, 1, 0),        # U2
            (Q.ADD, "C21", "Y", "C21", 1, False, 1, 0),          # U3
            (Q.MUL, "C11", "A12", "B21", 1, True, 1, swmm.T2_HLJJTT),   # U1 = P2 + P1
            (Q.ADD, "C22", "C22", "C21", 1, False, 1, 0),        # U7
            (Q.MUL, "C21", "A22", "C12", 1, True, -1, swmm.T2_HLJJTT),  # U6 = U3 - P4
            (Q.ADD, "C12", "C22", "Y", -1, False, 1, 0),         # U4 = U7 - P7
            (Q.MUL, "C12", "X", "B22", 1, True, 1, swmm.T2_HLJJTT),     # U5 = U4 + P3
        ]),
    "aclr14": dict(
        spec=dict(accumulate=True, preserve=(), temps=2, kinds=(swmm.T3_IP, Q.SELF)),
        search=dict(max_adds=14, max_rows=30),
        rows=None,
    ),
    "accr14": dict(
        spec=dict(accumulate=True, preserve=_AB[:4], temps=2, kinds=(swmm.T3_IP, swmm.T5_OVR, Q.SELF)),
        search=dict(max_adds=14, max_rows=30),
        rows=None,
    ),
}


def rows(name: str) -> list:
    """The stored rows of schedule `name` as search.Row objects."""
    f = FOUND[name]
    if f["rows"] is None:
        return regenerate(name)
    return [Q.Row(op, dst, s1, s2, coef, acc, sign, kind) for op, dst, s1, s2, coef, acc, sign, kind in f["rows"]]


def spec(name: str) -> dict:
    """The contract schedule `name` runs under (search.set_schedule keywords)."""
    return dict(FOUND[name]["spec"])


def regenerate(name: str) -> list:
    """Run the search that found schedule `name` again."""
    f = FOUND[name]
    o = Q.schedule_search(**f["spec"], **f["search"])
    if not o.found:
        raise RuntimeError(f"the search no longer finds {name}")
    return o.rows
