"""One pack for all seven fused levels under a table level.

At 8192^2 and depth 2 the top level's quadrants (4096^2, 64 MiB) are large
enough for symbolic pre-additions, so with Table 9 (read-only A and B) every
product row's operands are signed sums of operand quadrants and one launch
packs the 49 operand pairs.  Results must match the oracle's classical
product bit for bit on sampled rows, Freivalds' check on the whole result,
and the per-level packs of a bounded-staging call (SWMM_FLAG_LOWMEM, which
never packs a whole table level) bit for bit.  The staging the call reports
is the 49 pairs' (one slot, also in a graph with the dataflow capture).
Table 3 overwrites its operand quadrants, so it must keep per-level packs.
"""
import numpy as np
import pytest
import torch

from oracle import classical, probes
from paper_0707_2347_gb300 import swmm as S
from tests.gpu_util import dev, fp_inputs, host, modp_inputs

pytestmark = pytest.mark.gpu

N = 8192
PAIR = 2 * (2 * 2048 * 2048 * 2)  # one product's A and B operands: 2 limb planes of fp16
LEVEL = 49 * PAIR


@pytest.mark.parametrize("flags", [0, S.FLAG_GRAPH], ids=["eager", "graph"])
def test_level_pack_t9_modp(handle, flags):
    p = 65521
    A, B, C = modp_inputs(N, N, N, p, tag=21)
    dA, dB = dev(A), dev(B)
    dC = dev(C)
    o = S.Opts(mode=S.MODP, p=p, sched=S.T9_ACC, depth=2, flags=flags)
    for _ in range(2 if flags else 1):  # a graph: capture, then replay
        dC.copy_(dev(C))
        handle.muladd(3, dA, dB, 5, dC, o)
    handle.sync()
    st = handle.stats()
    assert st["staging_bytes"] == LEVEL
    assert st["plan_extra_elems"] == st["paper_extra_elems"] == 2 * 4096 * 4096  # Table 9: two temporaries
    out = host(dC)
    rows = np.sort(np.random.default_rng(3).choice(N, 24, replace=False))
    assert np.array_equal(out[rows], classical.rows_muladd_modp(rows, 3, A, B, 5, C, p))
    assert probes.freivalds_modp(3, A, B, 5, C, out, p, vectors=2)
    dL = dev(C)
    handle.muladd(3, dA, dB, 5, dL, S.Opts(mode=S.MODP, p=p, sched=S.T9_ACC, depth=2, flags=S.FLAG_LOWMEM))
    handle.sync()
    assert handle.stats()["staging_bytes"] <= S.LOWMEM_STAGE_BYTES
    assert torch.equal(dL, dC)
    assert np.array_equal(host(dA), A) and np.array_equal(host(dB), B)


def test_level_pack_t9_fp32(handle):
    A, B, C = fp_inputs(N, N, N, tag=22)
    dA, dB, dC = dev(A), dev(B), dev(C)
    handle.muladd(1.0, dA, dB, 1.0, dC, S.Opts(mode=S.FP32, sched=S.T9_ACC, depth=2))
    handle.sync()
    assert handle.stats()["staging_bytes"] == LEVEL + 1024  # plus the amax words
    rows = np.sort(np.random.default_rng(4).choice(N, 16, replace=False))
    exact = A[rows].astype(np.float64) @ B.astype(np.float64) + C[rows].astype(np.float64)
    scale = float(np.abs(A).max()) * float(np.abs(B).max())
    err = float(np.abs(host(dC)[rows] - exact).max()) / scale
    assert err <= probes.fp_bound(N), err


def test_inplace_table_keeps_level_packs(handle):
    """Table 3 overwrites A and B quadrants between its products, so its
    levels pack one at a time (an eager call stages one level)."""
    p = 65521
    A, B, _ = modp_inputs(N, N, N, p, tag=23)
    dA, dB = dev(A), dev(B)
    dC = torch.zeros((N, N), dtype=torch.int32, device=dA.device)
    handle.mul_inplace(dA, dB, dC, S.Opts(mode=S.MODP, p=p, sched=S.T3_IP, depth=2))
    handle.sync()
    assert handle.stats()["staging_bytes"] == 7 * PAIR
    out = host(dC)
    rows = np.sort(np.random.default_rng(5).choice(N, 16, replace=False))
    assert np.array_equal(out[rows], classical.rows_muladd_modp(rows, 1, A, B, 0, None, p))


@pytest.mark.parametrize("name", ["ab12", "acc16", "aclr14", "accr14"])
def test_searched_schedules_symbolic_at_8192(handle, name):
    """The shipped searched schedules at 8192^2 depth 2, where the top
    level's pre-additions are symbolic: ab12 parks S and T values in blocks
    of C, aclr14 and accr14 in operand quadrants they may overwrite
    (recorded, not written; packed in one pass where no product is stored
    in a quadrant a later product reads).  Sampled rows against the oracle,
    Freivalds on the whole result, and the preserved inputs bit-exact."""
    from paper_0707_2347_gb300 import schedules_found as F
    from paper_0707_2347_gb300 import search as Q
    rows_, spec = F.rows(name), F.spec(name)
    Q.set_schedule(handle, rows_, **spec)
    p, alpha, beta = 65521, 3, 5
    A, B, C = modp_inputs(N, N, N, p, tag=24)
    dA, dB, dC = dev(A), dev(B), dev(C)
    o = S.Opts(mode=S.MODP, p=p, sched=S.CUSTOM, depth=2)
    if not spec["accumulate"]:
        beta = 0
        handle.mul(dA, dB, dC, o)
        alpha = 1
    elif len(spec["preserve"]) == 8:
        handle.muladd(alpha, dA, dB, beta, dC, o)
    else:
        handle.mul_inplace(dA, dB, dC, o, alpha=alpha, beta=beta)
    handle.sync()
    if name == "ab12":
        assert handle.stats()["staging_bytes"] == LEVEL
    out = host(dC)
    rows = np.sort(np.random.default_rng(7).choice(N, 16, replace=False))
    assert np.array_equal(out[rows], classical.rows_muladd_modp(rows, alpha, A, B, beta, C if beta else None, p))
    assert probes.freivalds_modp(alpha, A, B, beta, C if beta else None, out, p, vectors=2)
    h = N // 2
    hA, hB = host(dA), host(dB)
    for blk in spec["preserve"]:
        M, M0 = (hA, A) if blk[0] == "A" else (hB, B)
        i, j = int(blk[1]) - 1, int(blk[2]) - 1
        assert np.array_equal(M[i * h:(i + 1) * h, j * h:(j + 1) * h], M0[i * h:(i + 1) * h, j * h:(j + 1) * h]), blk


@pytest.mark.parametrize("sched,keep,packs", [
    (S.T6_ACLR, "", 1), (S.T7_ACCR, "A", 1), (S.T8_ACR, "A", 1),
    (S.T3_IP, "", 0), (S.T4_OVL, "B", 0), (S.T5_OVR, "A", 0)],
    ids=["AcLR", "AccR", "AcR", "IP", "OvL", "OvR"])
def test_inplace_tables_at_level_pack_size(handle, sched, keep, packs):
    """The printed in-place tables at 2048^2 depth 2 (1024^2 quadrants, the
    smallest that pack in one pass): Tables 6-8 park their sums in operand
    quadrants as records and pack once, Tables 3-5 pack per level.  The
    whole result bit for bit against the oracle, and the blocks each table
    leaves untouched (Table 8 also B11 and B22) bit-identical."""
    p, n, alpha, beta = 65521, 2048, 3, 5
    A, B, C = modp_inputs(n, n, n, p, tag=25)
    dA, dB, dC = dev(A), dev(B), dev(C)
    o = S.Opts(mode=S.MODP, p=p, sched=sched, depth=2)
    acc = sched in (S.T6_ACLR, S.T7_ACCR, S.T8_ACR)
    if acc:
        handle.mul_inplace(dA, dB, dC, o, alpha=alpha, beta=beta)
    else:
        handle.mul_inplace(dA, dB, dC, o, alpha=alpha)
    handle.sync()
    assert handle.stats()["level_packs"] == packs
    want = classical.muladd_modp(alpha, A, B, beta if acc else 0, C, p)
    assert np.array_equal(host(dC), want)
    hA, hB = host(dA), host(dB)
    if "A" in keep:
        assert np.array_equal(hA, A)
    if "B" in keep:
        assert np.array_equal(hB, B)
    if sched == S.T8_ACR:
        h = n // 2
        assert np.array_equal(hB[:h, :h], B[:h, :h]) and np.array_equal(hB[h:, h:], B[h:, h:])
