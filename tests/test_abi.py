"""The C-ABI library builds, loads without a GPU, exports every entry point
include/swmm.h declares, and its planner matches the paper's memory counts
(no device work: swmm_workspace_elems accepts a NULL handle)."""
import ctypes
import os
import re

import pytest

import __graft_entry__ as g
from oracle import counts

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def S():
    g.build()
    from paper_0707_2347_gb300 import swmm
    swmm.load()
    return swmm


def declared_symbols():
    inc = os.path.join(ROOT, "include")
    text = "".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc)) if f.endswith(".h"))
    return sorted(set(re.findall(r"\b(swmm_[a-z_]+)\s*\(", text)))


def test_exports_every_declared_symbol(S):
    lib = S.load()
    decl = declared_symbols()
    assert "swmm_muladd" in decl and "swmm_mul_inplace" in decl
    for name in decl:
        assert hasattr(lib, name), name
    assert set(decl) == set(S.EXPORTS)


def test_strerror(S):
    lib = S.load()
    assert lib.swmm_strerror(0) == b"ok"
    assert lib.swmm_strerror(5) == b"device wait timed out"


def plan(S, m, k, n, **kw):
    lib = S.load()
    a, b = ctypes.c_int64(), ctypes.c_int64()
    o = S.Opts(**kw).c()
    rc = lib.swmm_workspace_elems(None, m, k, n, ctypes.byref(o), ctypes.byref(a), ctypes.byref(b))
    return rc, a.value, b.value


NAMES = {1: "T1", 2: "T2", 3: "IP", 4: "OvL", 11: "OvLM", 5: "OvR", 6: "AcLR", 7: "AccR", 8: "AcR", 9: "Acc"}


@pytest.mark.parametrize("sched", list(NAMES))
@pytest.mark.parametrize("depth", [1, 2, 3, 4])
@pytest.mark.parametrize("unfused", [True, False])
def test_planner_matches_paper_counts(S, sched, depth, unfused):
    n = 256
    rc, paper, planned = plan(S, n, n, n, sched=sched, depth=depth, flags=S.FLAG_UNFUSED if unfused else 0)
    assert rc == 0
    levels = depth if unfused else depth - 1
    assert planned == paper == counts.mem_depth(NAMES[sched], n, levels)


def test_planner_rectangular_lemma1(S):
    for m, k, n in [(512, 256, 1024), (1024, 512, 256), (256, 1024, 512)]:
        rc, paper, planned = plan(S, m, k, n, sched=1, depth=20, flags=S.FLAG_UNFUSED)
        assert rc == 0 and planned == paper == counts.E1(m, k, n)
        rc, paper, planned = plan(S, m, k, n, sched=2, depth=20, flags=S.FLAG_UNFUSED)
        assert rc == 0 and planned == paper == counts.E2(m, k, n)


def test_planner_configs(S):
    # 512^2 Table 1 depth 1: 2 * 256^2 temporaries (Table 1 X, Y)
    assert plan(S, 512, 512, 512, sched=1, depth=1, p=251, flags=S.FLAG_UNFUSED)[2] == 131072
    # 8192^2 Table 9 depth 3: 2 (4096^2 + 2048^2 + 1024^2) literal, last level fused saves 2 * 1024^2
    assert plan(S, 8192, 8192, 8192, sched=9, depth=3, flags=S.FLAG_UNFUSED)[2] == 44040192
    assert plan(S, 8192, 8192, 8192, sched=9, depth=3)[2] == 41943040
    # in-place schedules allocate nothing
    assert plan(S, 16384, 16384, 16384, sched=3, depth=4, p=251)[2] == 0
    assert plan(S, 16384, 16384, 16384, sched=10, depth=3, p=251)[2] == 0


def test_planner_rejects_bad_arguments(S):
    assert plan(S, 64, 32, 64, sched=4, depth=1)[0] == S.EINVAL   # OvL needs square
    assert plan(S, 64, 64, 64, sched=9, depth=1, p=2)[0] == S.EINVAL
    assert plan(S, 64, 64, 32, sched=10, depth=1)[0] == S.EINVAL  # IPMM needs m = n
    assert plan(S, 64, 64, 64, sched=3, depth=1, mode=7)[0] == S.EINVAL
    assert plan(S, 128, 64, 32, sched=3, depth=1)[0] == S.EINVAL  # IP needs k = n <= m
    # Algorithm 1 needs n < m, n <= k, n dividing m and k
    assert plan(S, 256, 256, 256, sched=S.IP0VMM, depth=1)[0] == S.EINVAL
    assert plan(S, 512, 128, 256, sched=S.IP0VMM, depth=1)[0] == S.EINVAL
    assert plan(S, 768, 512, 256, sched=S.IP0VMM, depth=1)[0] == 0
    assert plan(S, 640, 512, 256, sched=S.IP0VMM, depth=1)[0] == S.EINVAL


def test_planner_ip0vmm_needs_no_memory(S):
    for depth, unfused in [(1, True), (2, True), (3, False)]:
        rc, paper, planned = plan(S, 2048, 1536, 512, sched=S.IP0VMM, depth=depth,
                                  flags=S.FLAG_UNFUSED if unfused else 0)
        assert rc == 0 and paper == planned == 0


def test_autotune_choices(S):
    for shape in [(384, 384, 384), (1001, 2000, 777), (8192, 8192, 8192), (16384, 16384, 16384)]:
        s, d, t, e = S.autotune(*shape)
        assert s in (S.CLASSICAL, S.T2_HLJJTT, S.T9_ACC)
        assert 0 <= d <= 3 and t > 0 and e >= 0
        if s == S.CLASSICAL:
            assert d == 0 and e == 0
    # small problems stay classical: the additions cannot pay off
    assert S.autotune(384, 384, 384)[0] == S.CLASSICAL


def test_planner_peeling_odd_sizes(S):
    # odd dimensions are peeled: the recursion continues on the even core
    rc, paper, planned = plan(S, 1001, 1001, 1001, sched=9, depth=3, flags=S.FLAG_UNFUSED)
    assert rc == 0 and planned == paper == 2 * (500 ** 2 + 250 ** 2 + 125 ** 2)


@pytest.mark.parametrize("t,n", [(2, 1024), (3, 768), (4, 1024)])
@pytest.mark.parametrize("base", ["T2", "Acc"])
def test_planner_tblock_memory(S, t, n, base):
    """Section 7.2: the temporaries of one block call, (n/t)^2 with Table 2
    and 2 (n/t)^2 / 3 with Table 9 (Table 10), summed over the levels run."""
    acc = S.T9_ACC if base == "Acc" else 0
    b = n // t
    rc, paper, planned = plan(S, n, n, n, sched=S.TBLOCK, tblock=t, ipmm_acc=acc, depth=3, flags=S.FLAG_UNFUSED)
    assert rc == 0 and planned == paper == counts.mem_depth(base, b, 3)
    # the fused last level needs no temporaries of its own
    rc, paper, planned = plan(S, n, n, n, sched=S.TBLOCK, tblock=t, ipmm_acc=acc, depth=3)
    assert rc == 0 and planned == paper == counts.mem_depth(base, b, 2)


def test_planner_tblock_table10_leading_terms(S):
    # full recursion on 2^j blocks: n^2/4 (t = 2) and n^2/9 (t = 3) less the 1/b^2 tail of Lemma 1
    for t, n in [(2, 256), (3, 192)]:
        b = n // t
        levels = b.bit_length() - 1
        rc, paper, planned = plan(S, n, n, n, sched=S.TBLOCK, tblock=t, depth=levels, flags=S.FLAG_UNFUSED)
        assert rc == 0 and planned == paper == b * b - 1


def test_planner_tblock_rejects(S):
    assert plan(S, 1000, 1000, 1000, sched=S.TBLOCK, tblock=3, depth=1)[0] == S.EINVAL  # 3 does not divide 1000
    assert plan(S, 512, 256, 512, sched=S.TBLOCK, tblock=2, ipmm_acc=S.T9_ACC, depth=1)[0] == S.EINVAL
    assert plan(S, 512, 256, 512, sched=S.TBLOCK, tblock=2, depth=1)[0] == 0
    assert plan(S, 512, 512, 512, sched=S.TBLOCK, tblock=1, depth=1)[0] == S.EINVAL

