"""Schedules found by the pebble-game search (Section 4), run on the GPU as
the handle's own schedule (SWMM_CUSTOM): at every Winograd level the found
rows, recursing into themselves, with the fused tensor-core level last.
Each result must equal the definition bit for bit over Z/pZ, and the blocks
the schedule's contract preserves must come back unchanged."""
import numpy as np
import pytest
import torch

from oracle import classical, probes
from paper_0707_2347_gb300 import search as Q
from paper_0707_2347_gb300 import swmm as S
from tests.gpu_util import DEV, dev, fp_inputs, host, modp_inputs

pytestmark = pytest.mark.gpu

A_ALL = ("A11", "A12", "A21", "A22")
B_ALL = ("B11", "B12", "B21", "B22")
CASES = {
    # found schedule: search spec (the contract it is then run under)
    "IP-4-blocks": dict(accumulate=False, preserve=(), temps=0, kinds=(S.T3_IP,), max_written=4, max_copies=3),
    "OvL": dict(accumulate=False, preserve=B_ALL, temps=1, kinds=(S.T3_IP, Q.SELF)),
    "T1": dict(accumulate=False, preserve=A_ALL + B_ALL, temps=2, kinds=(Q.SELF,)),
    "T2": dict(accumulate=True, preserve=A_ALL + B_ALL, temps=3, kinds=(S.T1_DHSS, Q.SELF)),
    "AcLR": dict(accumulate=True, preserve=(), temps=2, kinds=(S.T3_IP, Q.SELF)),
    "AccR": dict(accumulate=True, preserve=A_ALL, temps=2, kinds=(S.T3_IP, S.T5_OVR, Q.SELF)),
}


def _found(case):
    c = CASES[case]
    o = Q.schedule_search(**c)
    assert o.found
    return o.rows, {k: v for k, v in c.items() if k != "max_written"}


def _run(handle, spec, dA, dB, dC, o, alpha, beta):
    if spec["accumulate"] and len(spec["preserve"]) == 8:
        handle.muladd(alpha, dA, dB, beta, dC, o)
    elif len(spec["preserve"]) == 8:
        handle.mul(dA, dB, dC, o)
    elif spec["accumulate"]:
        handle.mul_inplace(dA, dB, dC, o, alpha=alpha, beta=beta)
    else:
        handle.mul_inplace(dA, dB, dC, o, alpha=alpha)


def _quad(M, b, h):
    i, j = int(b[1]) - 1, int(b[2]) - 1
    return M[i * h:(i + 1) * h, j * h:(j + 1) * h]


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("n,depth,flags", [(256, 2, S.FLAG_UNFUSED), (512, 2, 0), (1024, 3, S.FLAG_GRAPH)],
                         ids=["256-d2-unfused", "512-d2", "1024-d3-graph"])
def test_found_schedule_on_gpu(handle, case, n, depth, flags):
    rows, spec = _found(case)
    Q.set_schedule(handle, rows, **spec)
    p, alpha, beta = 65521, 3, 5
    A, B, C = modp_inputs(n, n, n, p, tag=31)
    dA0, dB0 = dev(A), dev(B)
    dA, dB, dC = dA0.clone(), dB0.clone(), dev(C)
    o = S.Opts(mode=S.MODP, p=p, sched=S.CUSTOM, depth=depth, flags=flags)
    _run(handle, spec, dA, dB, dC, o, alpha, beta)
    handle.sync()
    a = alpha if spec["accumulate"] or len(spec["preserve"]) < 8 else 1
    b = beta if spec["accumulate"] else 0
    out = host(dC)
    if n <= 512:
        assert np.array_equal(out, classical.muladd_modp(a, A, B, b, C, p))
    else:
        rows_idx = np.array([0, 1, n // 2 - 1, n // 2, n - 2, n - 1])
        assert np.array_equal(out[rows_idx], classical.rows_muladd_modp(rows_idx, a, A, B, b, C, p))
        x = torch.from_numpy(np.random.default_rng(3).integers(0, p, n, dtype=np.int64).astype(np.int32)).to(DEV)
        y0 = torch.empty(n, dtype=torch.int32, device=DEV)
        pop = S.Opts(mode=S.MODP, p=p)
        handle.matvec(dev(C), x, y0, pop)
        r = torch.empty(n, dtype=torch.int32, device=DEV)
        handle.residual(a, dA0, dB0, b, y0, dC, x, r, pop)
        handle.sync()
        assert not host(r).any(), "residual probe"
    h = n // 2
    hA, hB = host(dA), host(dB)
    for blk in spec["preserve"]:
        M, M0 = (hA, A) if blk[0] == "A" else (hB, B)
        assert np.array_equal(_quad(M, blk, h), _quad(M0, blk, h)), blk
    st = handle.stats()
    paper, plan = Q.schedule_workspace(rows, n, n, n, o, **spec)
    assert st["plan_extra_elems"] == plan


def test_found_schedule_fp32(handle):
    rows, spec = _found("T1")
    Q.set_schedule(handle, rows, **spec)
    n = 1024
    A, B, C = fp_inputs(n, n, n, tag=32)
    dC = dev(C)
    handle.mul(dev(A), dev(B), dC, S.Opts(mode=S.FP32, sched=S.CUSTOM, depth=3))
    handle.sync()
    err = probes.fp_error(host(dC), classical.mul_f64(A, B), A, B)["max_rel"]
    assert err <= probes.fp_bound(n), err


def test_custom_entry_point_must_match_contract(handle):
    rows, spec = _found("OvL")
    Q.set_schedule(handle, rows, **spec)
    n, p = 256, 65521
    A, B, C = modp_inputs(n, n, n, p, tag=33)
    o = S.Opts(mode=S.MODP, p=p, sched=S.CUSTOM, depth=1)
    with pytest.raises(S.SwmmError):
        handle.mul(dev(A), dev(B), dev(C), o)  # it overwrites A: only swmm_mul_inplace
    with pytest.raises(S.SwmmError):  # not square
        handle.mul_inplace(dev(A[:, :128]), dev(B[:128, :128]), dev(C[:, :128]), o)


@pytest.mark.parametrize("n,depth,flags", [(512, 2, 0), (512, 2, S.FLAG_UNFUSED), (1024, 3, S.FLAG_GRAPH)])
def test_shipped_table9_class_schedule_on_gpu(handle, n, depth, flags):
    """The shipped 16-addition schedule for Table 9's contract, bit-exact."""
    from paper_0707_2347_gb300 import schedules_found as F
    Q.set_schedule(handle, F.rows("acc16"), **F.spec("acc16"))
    p, alpha, beta = 65521, 3, 5
    A, B, C = modp_inputs(n, n, n, p, tag=34)
    dA, dB, dC = dev(A), dev(B), dev(C)
    handle.muladd(alpha, dA, dB, beta, dC, S.Opts(mode=S.MODP, p=p, sched=S.CUSTOM, depth=depth, flags=flags))
    handle.sync()
    out = host(dC)
    idx = np.arange(n) if n <= 512 else np.array([0, 1, n // 2 - 1, n // 2, n - 2, n - 1])
    assert np.array_equal(out[idx], classical.rows_muladd_modp(idx, alpha, A, B, beta, C, p))
    assert np.array_equal(host(dA), A) and np.array_equal(host(dB), B)
