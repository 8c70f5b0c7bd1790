"""Pre-additions kept symbolic (formed while the fused level packs) on
quadrants large enough to use them (6144^2 at depth 2: 3072^2 quadrants).
Every schedule must still give the definition bit for bit: spot rows
against the oracle plus the device residual probe over the whole result."""
import numpy as np
import pytest
import torch

from oracle import classical, probes
from paper_0707_2347_gb300 import swmm as S
from tests.gpu_util import DEV, dev, fp_inputs, host, modp_inputs
from tests.test_gpu_schedules import ALL, KEEP, MUL, MULADD, INPLACE, NAME

pytestmark = pytest.mark.gpu

N = 6144
ROWS = np.array([0, 1, 1535, 3071, 3072, 4600, 6142, 6143])


@pytest.fixture(scope="module")
def inputs():
    return modp_inputs(N, N, N, 65521, tag=21)


@pytest.mark.parametrize("sched", ALL, ids=[NAME[s] for s in ALL])
@pytest.mark.parametrize("graph", [False, True], ids=["eager", "graph"])
def test_symbolic_preadditions(handle, inputs, sched, graph):
    p, alpha, beta = 65521, 3, 5
    A, B, C = inputs
    accumulate = sched in MULADD or sched not in MUL + INPLACE
    b = beta if accumulate else 0
    a = 1 if sched in MUL else alpha
    dA0, dB0, dC0 = dev(A), dev(B), dev(C)
    dA, dB, dC = dA0.clone(), dB0.clone(), dC0.clone()
    o = S.Opts(mode=S.MODP, p=p, sched=sched, depth=2, flags=S.FLAG_GRAPH if graph else 0)
    if sched in MUL:
        handle.mul(dA, dB, dC, o)
    elif sched in MULADD:
        handle.muladd(alpha, dA, dB, beta, dC, o)
    elif sched in INPLACE:
        handle.mul_inplace(dA, dB, dC, o, alpha=alpha)
    else:
        handle.mul_inplace(dA, dB, dC, o, alpha=alpha, beta=beta)
    x = torch.from_numpy(np.random.default_rng(5).integers(0, p, N, dtype=np.int64).astype(np.int32)).to(DEV)
    y0 = torch.empty(N, dtype=torch.int32, device=DEV)
    pop = S.Opts(mode=S.MODP, p=p)
    handle.matvec(dC0, x, y0, pop)
    r = torch.empty(N, dtype=torch.int32, device=DEV)
    handle.residual(a, dA0, dB0, b, y0, dC, x, r, pop)
    handle.sync()
    assert not host(r).any(), "residual probe"
    want = classical.rows_muladd_modp(ROWS, a, A, B, b, C, p)
    assert np.array_equal(host(dC)[ROWS], want)
    if "A" in KEEP[sched]:
        assert torch.equal(dA, dA0)
    if "B" in KEEP[sched]:
        assert torch.equal(dB, dB0)


def test_symbolic_preadditions_fp32(handle):
    A, B, C = fp_inputs(N, N, N, tag=22)
    dC = dev(C)
    handle.muladd(1.0, dev(A), dev(B), 1.0, dC, S.Opts(mode=S.FP32, sched=S.T9_ACC, depth=2))
    handle.sync()
    ref = A[ROWS].astype(np.float64) @ B.astype(np.float64) + C[ROWS].astype(np.float64)
    err = np.abs(host(dC)[ROWS] - ref).max() / (np.abs(A).max() * np.abs(B).max())
    assert err <= probes.fp_bound(N), err
