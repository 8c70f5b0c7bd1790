"""swmm_muladd_host: operands in host memory, copied block by block in the
order the schedule reads them, the result copied back.  Results must equal
the definition bit for bit over Z/pZ (FP32 mode: within the error bound),
eager and captured, with graph replays that see new host values."""
import numpy as np
import pytest
import torch

from oracle import classical, probes
from paper_0707_2347_gb300 import swmm as S
from tests.gpu_util import fp_inputs, modp_inputs

pytestmark = pytest.mark.gpu


def pinned(x):
    return torch.from_numpy(np.ascontiguousarray(x)).pin_memory()


@pytest.mark.parametrize("sched,depth,n", [(S.T9_ACC, 3, 1024), (S.T9_ACC, 2, 1000), (S.T2_HLJJTT, 2, 768),
                                           (S.CLASSICAL, 0, 999), (S.TBLOCK, 1, 1536)])
@pytest.mark.parametrize("graph", [False, True], ids=["eager", "graph"])
def test_host_operands_modp(handle, sched, depth, n, graph):
    p = 65521
    A, B, C = modp_inputs(n, n, n, p, tag=40)
    hA, hB, hC = pinned(A), pinned(B), pinned(C)
    o = S.Opts(mode=S.MODP, p=p, sched=sched, depth=depth, flags=S.FLAG_GRAPH if graph else 0)
    for rep in range(2):
        hC.copy_(torch.from_numpy(C + rep))  # new values at the same address
        handle.muladd_host(3, hA, hB, 5, hC, o)
        handle.sync()
        want = classical.muladd_modp(3, A, B, 5, C + rep, p)
        assert np.array_equal(hC.numpy(), want), rep
    assert np.array_equal(hA.numpy(), A) and np.array_equal(hB.numpy(), B)


def test_host_operands_rectangular_strided(handle):
    p, m, k, n = 65521, 600, 1030, 514
    A, B, C = modp_inputs(m, k, n, p, tag=41)
    # host views with a wider leading dimension
    bufA = torch.zeros((m, k + 6), dtype=torch.int32).pin_memory()
    bufA[:, :k] = torch.from_numpy(A)
    hA = bufA[:, :k]
    hB, hC = pinned(B), pinned(C)
    handle.muladd_host(1, hA, hB, 1, hC, S.Opts(mode=S.MODP, p=p, sched=S.T2_HLJJTT, depth=2))
    handle.sync()
    assert np.array_equal(hC.numpy(), classical.muladd_modp(1, A, B, 1, C, p))


def test_host_operands_fp32(handle):
    n = 1024
    A, B, C = fp_inputs(n, n, n, tag=42)
    hA, hB, hC = pinned(A), pinned(B), pinned(C)
    handle.muladd_host(1.0, hA, hB, 1.0, hC, S.Opts(mode=S.FP32, sched=S.T9_ACC, depth=2, flags=S.FLAG_GRAPH))
    handle.sync()
    err = probes.fp_error(hC.numpy(), classical.muladd_f64(1.0, A, B, 1.0, C), A, B)["max_rel"]
    assert err <= probes.fp_bound(n), err


def test_host_operands_reject_device_tensors(handle):
    A, B, C = modp_inputs(64, 64, 64, 251)
    with pytest.raises(ValueError):
        handle.muladd_host(1, torch.from_numpy(A).cuda(), pinned(B), 1, pinned(C), S.Opts(mode=S.MODP, p=251))
