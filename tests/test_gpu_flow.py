"""Graph capture with dataflow ordering (SWMM_FLAG_GRAPH without
SWMM_FLAG_SERIAL): launches wait only for the earlier launches whose memory
they touch.  Every schedule must still give the plain definition bit for
bit over Z/pZ, keep the inputs it declares read-only, and replay the same
graph to the same result."""
import numpy as np
import pytest
import torch

from oracle import classical, probes
from paper_0707_2347_gb300 import swmm as S
from tests.gpu_util import dev, fp_inputs, host, modp_inputs
from tests.test_gpu_schedules import ALL, KEEP, MUL, MULADD, INPLACE, NAME, expected

pytestmark = pytest.mark.gpu


def call(handle, sched, dA, dB, dC, o, alpha, beta):
    if sched in MUL or sched == S.IPMM:
        handle.mul(dA, dB, dC, o)
    elif sched in MULADD:
        handle.muladd(alpha, dA, dB, beta, dC, o)
    elif sched in INPLACE:
        handle.mul_inplace(dA, dB, dC, o, alpha=alpha)
    else:
        handle.mul_inplace(dA, dB, dC, o, alpha=alpha, beta=beta)


@pytest.mark.parametrize("sched", ALL, ids=[NAME[s] for s in ALL])
@pytest.mark.parametrize("n,depth,unfused", [(1024, 3, False), (512, 2, True), (998, 3, False)])
def test_flow_graph_matches_definition(handle, sched, n, depth, unfused):
    p, alpha, beta = 65521, 3, 5
    if n % 4 and sched not in MUL + MULADD:
        pytest.skip("odd sizes: the read-only schedules cover peeling under a flow")
    A, B, C = modp_inputs(n, n, n, p, tag=11)
    want = expected(sched, A, B, C, alpha, beta, p)
    flags = S.FLAG_GRAPH | (S.FLAG_UNFUSED if unfused else 0)
    o = S.Opts(mode=S.MODP, p=p, sched=sched, depth=depth, flags=flags)
    dA, dB, dC = dev(A), dev(B), dev(C)
    keepA, keepB = dA.clone(), dB.clone()
    for rep in range(2):  # capture, then replay of the cached graph on fresh inputs
        dA.copy_(keepA)
        dB.copy_(keepB)
        dC.copy_(dev(C))
        call(handle, sched, dA, dB, dC, o, alpha, beta)
        handle.sync()
        assert np.array_equal(host(dC), want), f"replay {rep}"
        if "A" in KEEP[sched]:
            assert torch.equal(dA, keepA)
        if "B" in KEEP[sched]:
            assert torch.equal(dB, keepB)


def test_flow_and_serial_capture_agree_on_stats(handle):
    p, n = 65521, 1024
    A, B, C = modp_inputs(n, n, n, p, tag=12)
    outs = []
    for extra in (0, S.FLAG_SERIAL):
        dC = dev(C)
        o = S.Opts(mode=S.MODP, p=p, sched=S.T9_ACC, depth=3, flags=S.FLAG_GRAPH | extra)
        handle.muladd(1, dev(A), dev(B), 1, dC, o)
        handle.sync()
        outs.append((host(dC), handle.stats()))
    assert np.array_equal(outs[0][0], outs[1][0])
    a, b = outs[0][1], outs[1][1]
    for key in ("leaf_launches", "ew_launches", "plan_extra_elems", "workspace_bytes"):
        assert a[key] == b[key], key
    # the dataflow capture uses at least two staging areas in turn
    assert a["staging_bytes"] >= b["staging_bytes"] > 0


def test_flow_fp32_within_bound(handle):
    n = 2048
    A, B, C = fp_inputs(n, n, n, tag=3)
    dC = dev(C)
    o = S.Opts(mode=S.FP32, sched=S.T9_ACC, depth=2, flags=S.FLAG_GRAPH)
    handle.muladd(1.0, dev(A), dev(B), 1.0, dC, o)
    handle.sync()
    err = probes.fp_error(host(dC), classical.muladd_f64(1.0, A, B, 1.0, C), A, B)["max_rel"]
    assert err <= probes.fp_bound(n), err


def test_flow_ipmm_carves_c22(handle):
    p, n, k = 65521, 1024, 2048
    A, B, _ = modp_inputs(n, k, n, p, tag=13)
    dA, dB = dev(A), dev(B)
    dC = torch.zeros((n, n), dtype=torch.int32, device=dA.device)
    o = S.Opts(mode=S.MODP, p=p, sched=S.IPMM, depth=2, ipmm_cutoff=256, flags=S.FLAG_GRAPH)
    for _ in range(2):
        dC.zero_()
        handle.mul(dA, dB, dC, o)
        handle.sync()
        assert np.array_equal(host(dC), classical.mul_modp(A, B, p))
    assert np.array_equal(host(dA), A) and np.array_equal(host(dB), B)
