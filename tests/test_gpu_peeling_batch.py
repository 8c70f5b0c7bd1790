"""Odd dimensions (dynamic peeling), the batched entry point with the
autotuner, and CUDA-graph replay, against the CPU oracle."""
import numpy as np
import pytest

import synth
from oracle import classical, probes
from paper_0707_2347_gb300 import swmm as S
from tests.gpu_util import dev, fp_inputs, host, modp_inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("sched,shape,depth", [
    (S.T9_ACC, (1001, 1001, 1001), 3), (S.T9_ACC, (515, 515, 515), 2), (S.T2_HLJJTT, (777, 1001, 333), 2),
    (S.T1_DHSS, (999, 555, 777), 3), (S.T8_ACR, (513, 771, 259), 2), (S.T6_ACLR, (513, 513, 513), 2),
    (S.T7_ACCR, (641, 641, 641), 2), (S.T5_OVR, (385, 385, 385), 3), (S.T3_IP, (1003, 501, 501), 2),
])
@pytest.mark.parametrize("flags", [0, S.FLAG_UNFUSED], ids=["fused", "unfused"])
def test_peeling_modp(handle, sched, shape, depth, flags):
    m, k, n = shape
    p = 65521
    A, B, C = modp_inputs(m, k, n, p, tag=31)
    dA, dB, dC = dev(A), dev(B), dev(C)
    o = S.Opts(mode=S.MODP, p=p, sched=sched, depth=depth, flags=flags)
    acc = sched in (S.T9_ACC, S.T2_HLJJTT, S.T8_ACR, S.T6_ACLR, S.T7_ACCR)
    if sched == S.T1_DHSS:
        handle.mul(dA, dB, dC, o)
    elif sched in (S.T9_ACC, S.T2_HLJJTT):
        handle.muladd(3, dA, dB, 5, dC, o)
    elif acc:
        handle.mul_inplace(dA, dB, dC, o, alpha=3, beta=5)
    else:
        handle.mul_inplace(dA, dB, dC, o, alpha=3)
    handle.sync()
    if sched == S.T1_DHSS:
        ref = classical.mul_modp(A, B, p)
    elif acc:
        ref = classical.muladd_modp(3, A, B, 5, C, p)
    else:
        ref = classical.muladd_modp(3, A, B, 0, C, p)
    assert np.array_equal(host(dC), ref)


def test_peeling_fp32(handle):
    m, k, n = 1001, 999, 1003
    A, B, C = fp_inputs(m, k, n, tag=32)
    dA, dB, dC = dev(A), dev(B), dev(C)
    handle.muladd(1.0, dA, dB, 1.0, dC, S.Opts(mode=S.FP32, sched=S.T2_HLJJTT, depth=2))
    handle.sync()
    err = probes.fp_error(host(dC), classical.muladd_f64(1.0, A, B, 1.0, C), A, B)["max_rel"]
    assert err <= probes.fp_bound(1003)


def _batch(count, lo, hi, seed):
    shapes = synth.batch_shapes(count, lo, hi, seed=seed)
    probs, refs = [], []
    for i, (m, k, n) in enumerate(shapes):
        if i % 2 == 0:
            A, B, C = modp_inputs(m, k, n, 65521, tag=100 + i)
            refs.append(("modp", A, B, C))
            probs.append(dict(A=dev(A), B=dev(B), C=dev(C), mode=S.MODP, p=65521, alpha=1, beta=1))
        else:
            A, B, C = fp_inputs(m, k, n, tag=100 + i)
            refs.append(("fp", A, B, C))
            probs.append(dict(A=dev(A), B=dev(B), C=dev(C), mode=S.FP32, alpha=1.0, beta=1.0))
    return probs, refs


def _check(probs, refs):
    for q, (kind, A, B, C) in zip(probs, refs):
        out = host(q["C"])
        if kind == "modp":
            assert np.array_equal(out, classical.muladd_modp(1, A, B, 1, C, 65521))
        else:
            err = probes.fp_error(out, classical.muladd_f64(1.0, A, B, 1.0, C), A, B)["max_rel"]
            assert err <= probes.fp_bound(max(A.shape[0], A.shape[1], B.shape[1]))


@pytest.mark.parametrize("graph", [False, True], ids=["eager", "graph"])
def test_batched_auto(handle, graph):
    probs, refs = _batch(24, 96, 1200, seed=41)
    flags = S.FLAG_GRAPH if graph else 0
    chosen = handle.muladd_batched(probs, flags)
    handle.sync()
    assert all(s in (S.CLASSICAL, S.T2_HLJJTT, S.T9_ACC) for s, _ in chosen)
    _check(probs, refs)
    if graph:
        # replay the captured batch on fresh C values
        for q, (kind, A, B, C) in zip(probs, refs):
            q["C"].copy_(dev(C))
        handle.muladd_batched(probs, flags)
        handle.sync()
        _check(probs, refs)


def test_batched_forced_schedules(handle):
    probs, refs = _batch(8, 600, 1100, seed=42)
    for i, q in enumerate(probs):
        q["sched"] = [S.T2_HLJJTT, S.CLASSICAL, S.T2_HLJJTT, S.T2_HLJJTT][i % 4]
        q["depth"] = 2
    chosen = handle.muladd_batched(probs, 0)
    handle.sync()
    assert [c[0] for c in chosen] == [q["sched"] for q in probs]
    _check(probs, refs)


def test_graph_replay_single_call(handle):
    p, n = 65521, 1024
    A, B, C = modp_inputs(n, n, n, p, tag=50)
    dA, dB = dev(A), dev(B)
    o = S.Opts(mode=S.MODP, p=p, sched=S.T9_ACC, depth=2, flags=S.FLAG_GRAPH)
    dC = dev(C)
    for rep in range(3):
        dC.copy_(dev(C))
        handle.muladd(3, dA, dB, 5, dC, o)
        handle.sync()
        assert np.array_equal(host(dC), classical.muladd_modp(3, A, B, 5, C, p)), rep
    # a different scalar is a different graph
    dC.copy_(dev(C))
    handle.muladd(4, dA, dB, 5, dC, o)
    handle.sync()
    assert np.array_equal(host(dC), classical.muladd_modp(4, A, B, 5, C, p))


@pytest.mark.parametrize("graph", [False, True], ids=["eager", "graph"])
def test_batched_classical_grouped(handle, graph):
    """Classical problems of one kind run as grouped launches (up to 16
    products each): 40 problems of two kinds need at most 2 + 2 launches."""
    probs, refs = _batch(40, 64, 700, seed=43)
    for q in probs:
        q["sched"] = S.CLASSICAL
        q["depth"] = 0
    handle.muladd_batched(probs, S.FLAG_GRAPH if graph else 0)
    handle.sync()
    _check(probs, refs)
    assert handle.stats()["leaf_launches"] <= 4


@pytest.mark.parametrize("graph", [False, True], ids=["eager", "graph"])
def test_batched_measured_tuning(handle, graph):
    """SWMM_FLAG_TUNE: the large problems' schedules are chosen by timing the
    classical product and one Winograd level on the GPU; results stay exact
    (Freivalds over Z/65521) or within the FP32 bound (FP64 residual), and a
    second call reuses the measured choices."""
    shapes = [(3200, 3328, 3456), (3456, 3200, 3328), (3328, 3328, 3328), (3584, 3584, 3584)]
    probs, refs = [], []
    for i, (m, k, n) in enumerate(shapes):
        if i % 2 == 0:
            A, B, C = modp_inputs(m, k, n, 65521, tag=200 + i)
            probs.append(dict(A=dev(A), B=dev(B), C=dev(C), mode=S.MODP, p=65521, alpha=1, beta=1))
            refs.append(("modp", A, B, C))
        else:
            A, B, C = fp_inputs(m, k, n, tag=200 + i)
            probs.append(dict(A=dev(A), B=dev(B), C=dev(C), mode=S.FP32, alpha=1.0, beta=1.0))
            refs.append(("fp", A, B, C))
    flags = S.FLAG_TUNE | (S.FLAG_GRAPH if graph else 0)
    chosen = handle.muladd_batched(probs, flags)
    handle.sync()
    for (s, d), (m, k, n) in zip(chosen, shapes):
        square = m == k == n
        assert (s, d) in ((S.CLASSICAL, 0), (S.T9_ACC if square else S.T2_HLJJTT, 1))
    for q, (kind, A, B, C) in zip(probs, refs):
        out = host(q["C"])
        if kind == "modp":
            assert probes.freivalds_modp(1, A, B, 1, C, out, 65521, vectors=2)
        else:
            assert probes.residual_f64(1.0, A, B, 1.0, C, out) <= probes.fp_bound(max(A.shape + B.shape))
    for q, (kind, A, B, C) in zip(probs, refs):
        q["C"].copy_(dev(C))
    again = handle.muladd_batched(probs, flags)
    handle.sync()
    assert again == chosen
