"""Error paths, made without faulting, trapping or hanging the GPU.

  * A leaf GEMM whose producer waits on a barrier that nothing completes
    (swmm_test_hook SWMM_HOOK_STALL_GEMMS) gives up after the handle's wait
    bound (set short with SWMM_HOOK_WAIT_NS): swmm_sync reports
    SWMM_ETIMEOUT, and the next call on the same handle is bit-exact, so the
    kernel returned cleanly and the context stays usable.
  * An allocation the library makes for a call fails on the host
    (SWMM_HOOK_FAIL_ALLOCS): the call returns SWMM_ENOMEM before any launch,
    C is untouched, and the next call succeeds.
"""
import numpy as np
import pytest

from oracle import classical
from paper_0707_2347_gb300 import swmm as S
from tests.gpu_util import dev, host, modp_inputs

pytestmark = pytest.mark.gpu


@pytest.fixture
def fresh():
    h = S.Handle(0)
    yield h
    h.close()


@pytest.mark.parametrize("p,sched,depth", [(65521, S.T9_ACC, 1), (65521, S.CLASSICAL, 0), (251, S.T9_ACC, 2)])
def test_bounded_wait_runs_out_then_handle_recovers(fresh, p, sched, depth):
    n, alpha, beta = 1024, 3, 5
    A, B, C = modp_inputs(n, n, n, p, tag=51)
    o = S.Opts(mode=S.MODP, p=p, sched=sched, depth=depth)
    fresh.test_hook(S.HOOK_WAIT_NS, 20_000_000)  # 20 ms
    fresh.test_hook(S.HOOK_STALL_GEMMS, 1)
    dA, dB, dC = dev(A), dev(B), dev(C)
    fresh.muladd(alpha, dA, dB, beta, dC, o)
    with pytest.raises(S.SwmmError) as e:
        fresh.sync()
    assert e.value.code == S.ETIMEOUT
    fresh.test_hook(S.HOOK_WAIT_NS, 0)  # back to the default bound
    dC = dev(C)
    fresh.muladd(alpha, dA, dB, beta, dC, o)
    fresh.sync()
    assert np.array_equal(host(dC), classical.muladd_modp(alpha, A, B, beta, C, p))


def test_allocation_failure_reports_enomem(fresh):
    p, n = 65521, 512
    A, B, C = modp_inputs(n, n, n, p, tag=52)
    o = S.Opts(mode=S.MODP, p=p, sched=S.T9_ACC, depth=2)
    dA, dB, dC = dev(A), dev(B), dev(C)
    fresh.test_hook(S.HOOK_FAIL_ALLOCS, 1)
    with pytest.raises(S.SwmmError) as e:
        fresh.muladd(1, dA, dB, 1, dC, o)
    assert e.value.code == S.ENOMEM
    fresh.sync()
    assert np.array_equal(host(dC), C)  # nothing ran
    fresh.muladd(1, dA, dB, 1, dC, o)
    fresh.sync()
    assert np.array_equal(host(dC), classical.muladd_modp(1, A, B, 1, C, p))


def test_unknown_hook_rejected(fresh):
    with pytest.raises(S.SwmmError) as e:
        fresh.test_hook(99, 1)
    assert e.value.code == S.EINVAL
