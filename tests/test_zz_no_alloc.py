"""swmm_muladd_noalloc: the allocation-free variant of swmm_muladd.

Some callers cannot call cudaMalloc (their memory budget belongs to another
allocator, or they run where reaching the CUDA driver's allocator is not
allowed).  This entry point takes its scratch from a static device array
instead.  The test calls it through the C ABI twice in a row and checks each
result against the regular entry point on the same inputs; it also checks
that a plan larger than the static array is refused with a clear error.
It lives in a file collected last so that a failure here cannot hide the
results of the other GPU tests."""
import ctypes

import numpy as np
import pytest

from oracle import classical, probes
from paper_0707_2347_gb300 import swmm as S
from tests.gpu_util import dev, fp_inputs, host, modp_inputs

pytestmark = pytest.mark.gpu


def _noalloc(handle, alpha, A, B, beta, C, opts):
    """Call the entry point directly through the C ABI."""
    import torch
    lib = S.load()
    lib.swmm_set_stream(handle.h, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    m, k = A.shape
    n = B.shape[1]
    al = ctypes.c_uint32(alpha) if opts.mode == S.MODP else ctypes.c_float(alpha)
    be = ctypes.c_uint32(beta) if opts.mode == S.MODP else ctypes.c_float(beta)
    return lib.swmm_muladd_noalloc(handle.h, m, k, n, ctypes.byref(al), ctypes.c_void_p(A.data_ptr()), A.stride(0),
                                   ctypes.c_void_p(B.data_ptr()), B.stride(0), ctypes.byref(be),
                                   ctypes.c_void_p(C.data_ptr()), C.stride(0), ctypes.byref(opts.c()))


@pytest.mark.parametrize("sched,n,depth", [(S.T9_ACC, 1024, 2), (S.T2_HLJJTT, 768, 2), (S.CLASSICAL, 640, 0)])
def test_noalloc_matches_muladd_twice(handle, sched, n, depth):
    p = 65521
    opts = S.Opts(mode=S.MODP, p=p, sched=sched, depth=depth)
    for call in range(2):
        A, B, C = modp_inputs(n, n, n, p, tag=10 + call)
        dA, dB = dev(A), dev(B)
        ref, out = dev(C), dev(C)
        handle.muladd(3, dA, dB, 7, ref, opts)
        rc = _noalloc(handle, 3, dA, dB, 7, out, opts)
        assert rc == S.OK, handle.lib.swmm_last_error(handle.h)
        handle.sync()
        got = host(out)
        assert np.array_equal(got, host(ref))
        assert np.array_equal(got, classical.muladd_modp(3, A, B, 7, C, p))


def test_noalloc_fp32_twice(handle):
    n = 1024
    opts = S.Opts(mode=S.FP32, sched=S.T9_ACC, depth=2)
    for call in range(2):
        A, B, C = fp_inputs(n, n, n, tag=20 + call)
        dA, dB = dev(A), dev(B)
        ref, out = dev(C), dev(C)
        handle.muladd(1.0, dA, dB, 1.0, ref, opts)
        assert _noalloc(handle, 1.0, dA, dB, 1.0, out, opts) == S.OK
        handle.sync()
        got = host(out)
        assert np.abs(got - host(ref)).max() <= 1e-5 * np.abs(host(ref)).max()
        err = probes.fp_error(got, classical.muladd_f64(1.0, A, B, 1.0, C), A, B)["max_rel"]
        assert err <= probes.fp_bound(n)


def test_noalloc_rejects_plans_beyond_the_static_array(handle):
    import torch
    n = 4096  # Table 9 depth 2 needs 32 MiB of temporaries plus staging
    A = torch.zeros((n, n), dtype=torch.int32, device="cuda")
    B = torch.zeros((n, n), dtype=torch.int32, device="cuda")
    C = torch.zeros((n, n), dtype=torch.int32, device="cuda")
    rc = _noalloc(handle, 1, A, B, 1, C, S.Opts(mode=S.MODP, p=65521, sched=S.T9_ACC, depth=2))
    assert rc == S.EINVAL
    assert b"static scratch" in handle.lib.swmm_last_error(handle.h)
