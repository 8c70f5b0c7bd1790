"""Python binding of include/swmm_search.h: the pebble-game search for the
memory schedules of one Winograd level (Section 4), and the replay of a
given schedule under the same rules.  Host code of libswmm.so; no GPU.

Locations are named as in the tables ("A11" ... "C22", "X", "Y", "Z");
recursive call kinds are the schedule codes of swmm.py (T1_DHSS ...
T9_ACC, T4M_OVL) or SELF, the schedule being searched for.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field

from . import swmm

LOCS = ("A11", "A12", "A21", "A22", "B11", "B12", "B21", "B22",
        "C11", "C12", "C21", "C22", "X", "Y", "Z")
ADD, MUL, COPY = 0, 1, 2
COEFS = (1, -1, "b", "-b")  # SWMM_COEF_ONE, NEG, BETA, NBETA
SELF = 31
MAX_ROWS = 64
ASCENDING, DESCENDING, PORTFOLIO = 0, 1, 2  # search orders


class _Spec(ctypes.Structure):
    _fields_ = [("accumulate", ctypes.c_int32), ("preserve", ctypes.c_uint32), ("temps", ctypes.c_int32),
                ("kinds", ctypes.c_uint32), ("max_written", ctypes.c_int32), ("max_copies", ctypes.c_int32),
                ("recompute", ctypes.c_int32), ("max_rows", ctypes.c_int32), ("max_adds", ctypes.c_int32),
                ("max_states", ctypes.c_int64), ("exclude", ctypes.c_uint64), ("m", ctypes.c_int32),
                ("k", ctypes.c_int32), ("n", ctypes.c_int32), ("order", ctypes.c_int32)]


class _Row(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int32) for f in ("op", "dst", "s1", "s2", "coef", "accumulate", "sign", "kind", "node")]


class _Result(ctypes.Structure):
    _fields_ = [("found", ctypes.c_int32), ("exhausted", ctypes.c_int32), ("nrows", ctypes.c_int32),
                ("written", ctypes.c_int32), ("temps_used", ctypes.c_int32), ("states", ctypes.c_int64)]


@dataclass
class Row:
    op: int                 # ADD, MUL or COPY
    dst: str                # location written
    s1: str                 # ADD: first operand; MUL: left operand; COPY: source
    s2: str | None = None   # ADD: second operand; MUL: right operand
    coef: object = 1        # ADD: coefficient of s2; MUL accumulate: of dst's value (1, -1, "b", "-b")
    accumulate: bool = False
    sign: int = 1           # MUL: sign applied to alpha
    kind: int = 0           # MUL: schedule code or SELF
    value: str = ""         # name of the value written (filled by the library)


@dataclass
class Outcome:
    found: bool
    exhausted: bool
    states: int
    written: int            # blocks of A and B written or overwritten
    temps_used: int
    rows: list = field(default_factory=list)
    first_bad_row: int = -1  # schedule_check: index of the first illegal row (-1: none)


def _lib():
    lib = swmm.load()
    if not getattr(lib, "_search_typed", False):
        lib.swmm_schedule_search.argtypes = [ctypes.POINTER(_Spec), ctypes.POINTER(_Row), ctypes.c_int32,
                                             ctypes.POINTER(_Result)]
        lib.swmm_schedule_check.argtypes = [ctypes.POINTER(_Spec), ctypes.POINTER(_Row), ctypes.c_int32,
                                            ctypes.POINTER(_Result)]
        lib.swmm_search_node_name.argtypes = [ctypes.c_int32, ctypes.c_int32]
        lib.swmm_search_node_name.restype = ctypes.c_char_p
        lib.swmm_search_node_count.argtypes = [ctypes.c_int32]
        lib.swmm_set_schedule.argtypes = [ctypes.c_void_p, ctypes.POINTER(_Spec), ctypes.POINTER(_Row),
                                          ctypes.c_int32]
        i64p = ctypes.POINTER(ctypes.c_int64)
        lib.swmm_schedule_workspace.argtypes = [ctypes.POINTER(_Spec), ctypes.POINTER(_Row), ctypes.c_int32,
                                                ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                                ctypes.POINTER(swmm._Opts), i64p, i64p,
                                                ctypes.POINTER(ctypes.c_double)]
        lib.swmm_table_rows.argtypes = [ctypes.c_int32, ctypes.POINTER(_Row), ctypes.c_int32,
                                        ctypes.POINTER(ctypes.c_int32)]
        lib._search_typed = True
    return lib


def _spec(accumulate, preserve, temps, kinds, max_written, max_copies, recompute, max_rows, max_states, max_adds=-1,
          exclude=(), shape=None, order=ASCENDING):
    pm = 0
    for b in preserve:
        i = LOCS.index(b)
        if i >= 8:
            raise ValueError(f"only blocks of A and B are preserved, not {b}")
        pm |= 1 << i
    km = 0
    for k in kinds:
        km |= 1 << int(k)
    names = node_names(accumulate) if exclude else []
    em = 0
    for v in exclude:
        em |= 1 << names.index(v)
    m, k, n = shape if shape else (0, 0, 0)
    return _Spec(int(bool(accumulate)), pm, temps, km, max_written, max_copies, int(bool(recompute)), max_rows,
                 max_adds, max_states, em, m, k, n, order)


def node_names(accumulate: bool) -> list:
    lib = _lib()
    a = int(bool(accumulate))
    return [lib.swmm_search_node_name(a, i).decode() for i in range(lib.swmm_search_node_count(a))]


def _rows_out(crows, n, accumulate):
    names = node_names(accumulate)
    out = []
    for r in crows[:n]:
        out.append(Row(op=r.op, dst=LOCS[r.dst], s1=LOCS[r.s1], s2=LOCS[r.s2] if r.op != COPY else None,
                       coef=COEFS[r.coef], accumulate=bool(r.accumulate), sign=r.sign, kind=r.kind,
                       value=names[r.node] if 0 <= r.node < len(names) else ""))
    return out


def schedule_search(*, accumulate=False, preserve=(), temps=0, kinds=(), max_written=-1, max_copies=0,
                    recompute=False, max_rows=40, max_states=0, max_adds=-1, exclude=(), shape=None,
                    order=ASCENDING) -> Outcome:
    """Search for one level's schedule: C <- alpha AB (+ beta C when
    `accumulate`), keeping the blocks named in `preserve`, with `temps`
    temporaries, recursive products of the given `kinds`, at most
    `max_adds` block additions, never forming the values named in
    `exclude` (see node_names); `shape` = relative sizes (m, k, n) of the
    operands, None for square blocks; `order`: ASCENDING, DESCENDING or
    PORTFOLIO (both in turn; often much faster to find a schedule when one
    order alone is slow)."""
    lib = _lib()
    spec = _spec(accumulate, preserve, temps, kinds, max_written, max_copies, recompute, max_rows, max_states,
                 max_adds, exclude, shape, order)
    rows = (_Row * MAX_ROWS)()
    res = _Result()
    rc = lib.swmm_schedule_search(ctypes.byref(spec), rows, MAX_ROWS, ctypes.byref(res))
    if rc != swmm.OK:
        raise swmm.SwmmError(rc, "schedule search failed")
    return Outcome(bool(res.found), bool(res.exhausted), res.states, res.written, res.temps_used,
                   _rows_out(rows, res.nrows, accumulate) if res.found else [])


def _crows(rows):
    crows = (_Row * max(len(rows), 1))()
    for i, r in enumerate(rows):
        crows[i] = _Row(r.op, LOCS.index(r.dst), LOCS.index(r.s1), LOCS.index(r.s2) if r.s2 else -1,
                        COEFS.index(r.coef), int(r.accumulate), r.sign, r.kind, -1)
    return crows


def set_schedule(handle, rows, *, accumulate=False, preserve=(), temps=0, kinds=(), max_copies=0,
                 recompute=False):
    """Give a swmm.Handle the one-level schedule `rows`; calls with
    Opts(sched=swmm.CUSTOM) then run it at every level (SELF rows recurse
    into it).  Raises SwmmError when the schedule is not a legal play."""
    lib = _lib()
    spec = _spec(accumulate, preserve, temps, kinds, -1, max_copies, recompute, MAX_ROWS, 0)
    rc = lib.swmm_set_schedule(handle.h, ctypes.byref(spec), _crows(rows), len(rows))
    if rc != swmm.OK:
        raise swmm.SwmmError(rc, lib.swmm_last_error(handle.h).decode())


def _plan(rows, m, k, n, opts, spec):
    lib = _lib()
    paper, plan, us = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
    rc = lib.swmm_schedule_workspace(ctypes.byref(spec), _crows(rows), len(rows), m, k, n, ctypes.byref(opts.c()),
                                     ctypes.byref(paper), ctypes.byref(plan), ctypes.byref(us))
    if rc != swmm.OK:
        raise swmm.SwmmError(rc, "schedule planning failed")
    return paper.value, plan.value, us.value


def schedule_workspace(rows, m, k, n, opts, *, accumulate=False, preserve=(), temps=0, kinds=(), max_copies=0,
                       recompute=False):
    """(schedule's own temporaries, planner peak) in elements for a call of
    `rows` on m x k x n with `opts` (sched must be swmm.CUSTOM); no device."""
    spec = _spec(accumulate, preserve, temps, kinds, -1, max_copies, recompute, MAX_ROWS, 0)
    return _plan(rows, m, k, n, opts, spec)[:2]


def schedule_stats(rows, m, k, n, opts, *, accumulate=False, preserve=(), temps=0, kinds=(), max_copies=0,
                   recompute=False) -> dict:
    """The plan's counts (swmm_stats fields) for a call of `rows`; no device."""
    spec = _spec(accumulate, preserve, temps, kinds, -1, max_copies, recompute, MAX_ROWS, 0)
    st = swmm._Stats()
    rc = _lib().swmm_schedule_stats(ctypes.byref(spec), _crows(rows), len(rows), m, k, n, ctypes.byref(opts.c()),
                                    ctypes.byref(st))
    if rc != swmm.OK:
        raise swmm.SwmmError(rc, "schedule planning failed")
    return {f: getattr(st, f) for f, _ in swmm._Stats._fields_ if f != "reserved"}


def schedule_model_us(rows, m, k, n, opts, *, accumulate=False, preserve=(), temps=0, kinds=(), max_copies=0,
                      recompute=False):
    """The autotuner's modelled time (microseconds) for a call of `rows`."""
    spec = _spec(accumulate, preserve, temps, kinds, -1, max_copies, recompute, MAX_ROWS, 0)
    return _plan(rows, m, k, n, opts, spec)[2]


def frontier(candidates, m, k, n, opts):
    """Memory-speed frontier of one-level schedules for an m x k x n call.

    candidates: {name: (rows, spec dict as set_schedule takes it)}.  Returns
    [(name, planned temporaries, modelled us)] of the candidates no other
    one beats on both, fewest temporaries first."""
    pts = []
    for name, (rows, spec) in candidates.items():
        _, plan, us = _plan(rows, m, k, n, opts, _spec(spec.get("accumulate", False), spec.get("preserve", ()),
                                                          spec.get("temps", 0), spec.get("kinds", ()), -1,
                                                          spec.get("max_copies", 0), spec.get("recompute", False),
                                                          MAX_ROWS, 0))
        pts.append((name, plan, us))
    keep = [a for a in pts if not any(b[1] <= a[1] and b[2] < a[2] or b[1] < a[1] and b[2] <= a[2] for b in pts)]
    return sorted(keep, key=lambda t: (t[1], t[2]))


def table_rows(sched: int) -> list:
    """The rows of the paper's table `sched` (a schedule code of swmm.py) as
    the library runs them; value names are left empty (schedule_check
    fills them)."""
    lib = _lib()
    crows = (_Row * MAX_ROWS)()
    n = ctypes.c_int32()
    rc = lib.swmm_table_rows(sched, crows, MAX_ROWS, ctypes.byref(n))
    if rc != swmm.OK:
        raise swmm.SwmmError(rc, f"no table for schedule code {sched}")
    return [Row(op=r.op, dst=LOCS[r.dst], s1=LOCS[r.s1], s2=LOCS[r.s2] if r.op != COPY else None,
                coef=COEFS[r.coef], accumulate=bool(r.accumulate), sign=r.sign, kind=r.kind)
            for r in crows[:n.value]]


def schedule_check(rows, *, accumulate=False, preserve=(), temps=0, kinds=(), max_copies=0,
                   recompute=False, shape=None) -> Outcome:
    """Replay `rows` (a list of Row) under the same rules; found is True when
    every row is a legal move and the results end in place."""
    lib = _lib()
    spec = _spec(accumulate, preserve, temps, kinds, -1, max_copies, recompute, MAX_ROWS, 0, shape=shape)
    n = len(rows)
    crows = _crows(rows)
    res = _Result()
    rc = lib.swmm_schedule_check(ctypes.byref(spec), crows, n, ctypes.byref(res))
    if rc != swmm.OK:
        raise swmm.SwmmError(rc, "schedule check failed")
    legal = res.nrows
    out = _rows_out(crows, legal, accumulate)
    return Outcome(bool(res.found), False, 0, res.written, res.temps_used, out,
                   -1 if legal == n else legal)


# contract of each printed table: (accumulates, blocks it keeps, temporaries)
_A, _B = ("A11", "A12", "A21", "A22"), ("B11", "B12", "B21", "B22")
TABLE_CONTRACT = {
    swmm.T1_DHSS: (False, _A + _B, 2), swmm.T2_HLJJTT: (True, _A + _B, 3), swmm.T3_IP: (False, (), 0),
    swmm.T4_OVL: (False, _B, 1), swmm.T4M_OVL: (False, _B + ("A12", "A22"), 1), swmm.T5_OVR: (False, _A, 1),
    swmm.T6_ACLR: (True, (), 2), swmm.T7_ACCR: (True, _A, 2), swmm.T8_ACR: (True, _A + ("B11", "B22"), 2),
    swmm.T9_ACC: (True, _A + _B, 2),
}


def tune(m, k, n, opts, *, accumulate=False, preserve=(), max_elems=None, search_states=1 << 18):
    """Pick a one-level schedule for an m x k x n call under a contract
    (accumulate or not, blocks of A and B to keep) and a memory cap.

    Candidates: every printed table whose contract covers the request; the
    same table with Table 2 for its accumulating calls and with Table 1 for
    its plain calls; the searched schedules the library ships
    (schedules_found.py) whose contract covers it; and, for C <- AB, the
    schedule the pebble-game search
    returns with the fewest block additions for each number of temporaries
    the tables use (each search bounded by `search_states`).  Each is planned
    (temporaries) and costed by the autotuner's model.  Returns (name, rows,
    spec, planned elements, modelled us) of the fastest candidate within
    `max_elems`, and the memory-speed frontier of all of them."""
    keep = set(preserve)
    cands = {}
    for code, (acc, tkeep, temps) in TABLE_CONTRACT.items():
        if acc != bool(accumulate) or not keep <= set(tkeep):
            continue
        base = table_rows(code)
        kinds0 = {r.kind for r in base if r.op == MUL}
        variants = {swmm.SCHED_NAMES[code]: base}
        for repl, tag in (({swmm.T9_ACC: swmm.T2_HLJJTT, swmm.T6_ACLR: swmm.T2_HLJJTT,
                            swmm.T7_ACCR: swmm.T2_HLJJTT, swmm.T8_ACR: swmm.T2_HLJJTT}, "/T2"),
                          ({swmm.T3_IP: swmm.T1_DHSS, swmm.T4_OVL: swmm.T1_DHSS, swmm.T5_OVR: swmm.T1_DHSS,
                            swmm.T4M_OVL: swmm.T1_DHSS}, "/T1")):
            if not kinds0 & set(repl):
                continue
            rows = [Row(**r.__dict__) for r in base]
            for r in rows:
                if r.op == MUL:
                    r.kind = repl.get(r.kind, r.kind)
            variants[swmm.SCHED_NAMES[code] + tag] = rows
        for name, rows in variants.items():
            spec = dict(accumulate=acc, preserve=tuple(tkeep), temps=temps,
                        kinds=tuple(sorted({r.kind for r in rows if r.op == MUL})),
                        max_copies=sum(r.op == COPY for r in rows), recompute=code == swmm.T9_ACC)
            if schedule_check(rows, **spec).found:
                cands[name] = (rows, spec)
    # the searched schedules the library ships (schedules_found.py)
    from . import schedules_found as found
    for fname, f in found.FOUND.items():
        fs = f["spec"]
        if fs["accumulate"] == bool(accumulate) and keep <= set(fs["preserve"]):
            cands["found:" + fname] = (found.rows(fname), dict(fs))
    # searched schedules for C <- AB (the accumulating game is too large to
    # search within a tuning call): fewest additions per table memory
    for temps in sorted({sp["temps"] for _, sp in cands.values()}) if not accumulate else ():
        kinds = (SELF, swmm.T2_HLJJTT) if len(keep) == 8 else (SELF, swmm.T3_IP)
        best = None
        for adds in range(15, 10, -1):
            o = schedule_search(preserve=tuple(keep), temps=temps, kinds=kinds, max_adds=adds, max_rows=30,
                                max_states=search_states)
            if not o.found:
                break
            best = o
        if best is not None:
            cands[f"searched t{temps}"] = (best.rows, dict(accumulate=False, preserve=tuple(keep), temps=temps,
                                                           kinds=kinds))
    scored = []
    for name, (rows, spec) in cands.items():
        _, plan, us = _plan(rows, m, k, n, opts, _spec(spec["accumulate"], spec["preserve"], spec["temps"],
                                                        spec["kinds"], -1, spec.get("max_copies", 0),
                                                        spec.get("recompute", False), MAX_ROWS, 0))
        scored.append((name, plan, us))
    ok = [t for t in scored if max_elems is None or t[1] <= max_elems]
    if not ok:
        raise ValueError("no candidate schedule fits the memory cap")
    name, plan, us = min(ok, key=lambda t: (t[2], t[1]))
    front = [a for a in scored if not any(b[1] <= a[1] and b[2] < a[2] or b[1] < a[1] and b[2] <= a[2]
                                          for b in scored)]
    return (name, cands[name][0], cands[name][1], plan, us), sorted(front, key=lambda t: (t[1], t[2]))
