"""Classical leaf products on the tensor cores against the CPU oracle.

Exactness over Z/pZ: bit-exact for every shape, including ragged tails that
span several 128 x 128 (or 128 x 256) tiles, the exactness boundary K = 1024
with adversarial operands, and K > 1024 where the accumulators are reduced
in place.  FP32 mode: max |C - C64| / (||A|| ||B||) <= 1e-5 n^0.6."""
import numpy as np
import pytest

import synth
from oracle import classical, probes
from paper_0707_2347_gb300 import swmm as S
from tests.gpu_util import dev, fp_inputs, host, modp_inputs, padded

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1, 1), (128, 64, 128), (256, 128, 256), (300, 200, 170), (513, 1000, 259), (64, 2048, 384),
          (1, 777, 1), (7, 3, 5)]


@pytest.mark.parametrize("p", [251, 65521])
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("simt", [False, True], ids=["tc", "simt"])
def test_classical_modp_exact(handle, p, shape, simt):
    m, k, n = shape
    A, B, C = modp_inputs(m, k, n, p)
    dA, dB, dC = dev(A), dev(B), dev(C)
    o = S.Opts(mode=S.MODP, p=p, sched=S.CLASSICAL, depth=0, flags=S.FLAG_SIMT_LEAF if simt else 0)
    handle.muladd(3, dA, dB, 5, dC, o)
    handle.sync()
    assert np.array_equal(host(dC), classical.muladd_modp(3, A, B, 5, C, p))


@pytest.mark.parametrize("p", [251, 257, 65521, 40009])
@pytest.mark.parametrize("pattern", ["max", "half", "halfneg", "alt"])
@pytest.mark.parametrize("k", [1024, 2048, 3000])
def test_exactness_adversarial(handle, p, pattern, k):
    """Largest-magnitude centred limbs at and beyond the 1024-term fp32 bound."""
    m = n = 128
    A = synth.adversarial_modp(m, k, p, pattern)
    B = synth.adversarial_modp(k, n, p, pattern)
    dA, dB = dev(A), dev(B)
    dC = dev(np.zeros((m, n), dtype=np.int32))
    handle.mul(dA, dB, dC, S.Opts(mode=S.MODP, p=p, sched=S.CLASSICAL, depth=0))
    handle.sync()
    assert np.array_equal(host(dC), classical.mul_modp(A, B, p))


def test_leading_dimensions_and_alpha(handle):
    p = 65521
    m, k, n = 200, 300, 150
    A, B, C = modp_inputs(m, k, n, p, tag=1)
    dA, dB, dC = padded(A, 333), padded(B, 160), padded(C, 151)
    handle.muladd(p - 1, dA, dB, 7, dC, S.Opts(mode=S.MODP, p=p, sched=S.CLASSICAL, depth=0))
    handle.sync()
    assert np.array_equal(host(dC), classical.muladd_modp(p - 1, A, B, 7, C, p))


@pytest.mark.parametrize("shape", [(128, 64, 128), (300, 200, 170), (512, 512, 512), (100, 4096, 96)])
def test_classical_fp32(handle, shape):
    m, k, n = shape
    A, B, C = fp_inputs(m, k, n)
    dA, dB, dC = dev(A), dev(B), dev(C)
    handle.muladd(1.0, dA, dB, 1.0, dC, S.Opts(mode=S.FP32, sched=S.CLASSICAL, depth=0))
    handle.sync()
    ref = classical.muladd_f64(1.0, A, B, 1.0, C)
    err = probes.fp_error(host(dC), ref, A, B)["max_rel"]
    assert err <= probes.fp_bound(max(shape)), err


def test_empty_inner_dimension(handle):
    p = 251
    A = np.zeros((5, 0), dtype=np.int32)
    B = np.zeros((0, 7), dtype=np.int32)
    C = synth.modp_matrix(3, 5, 7, p)
    dC = dev(C)
    handle.muladd(1, dev(np.zeros((5, 1), np.int32))[:, :0], dev(np.zeros((1, 7), np.int32))[:0], 2, dC,
                  S.Opts(mode=S.MODP, p=p, sched=S.CLASSICAL, depth=0))
    handle.sync()
    assert np.array_equal(host(dC), (2 * C) % p)


@pytest.mark.parametrize("cols", [194, 97, 1, 388])
def test_store_leaves_neighbouring_columns_alone(handle, cols):
    """A target narrower than its leading dimension must not be written
    outside its columns (TMA stores work in 16-byte chunks)."""
    p = 65521
    m, k, ld = 249, 138, 400
    A = synth.modp_matrix(1, m, k, p)
    B = synth.modp_matrix(2, k, cols, p)
    C = synth.modp_matrix(3, m, ld, p)
    dC = dev(C)
    handle.mul(dev(A), dev(B), dC[:, :cols], S.Opts(mode=S.MODP, p=p, sched=S.CLASSICAL, depth=0))
    handle.sync()
    out = host(dC)
    assert np.array_equal(out[:, :cols], classical.mul_modp(A, B, p))
    assert np.array_equal(out[:, cols:], C[:, cols:])
