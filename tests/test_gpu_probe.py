"""Residual probe (swmm_matvec / swmm_residual) against the definitions.

The matrix-vector product is checked exactly (mod p, numpy int64) or to
FP64 rounding (FP32 mode); the residual of a correct product must vanish
over Z/pZ, and for a wrong C it must equal (C - alpha A B - beta C_in) x
computed on the host."""
import numpy as np
import pytest
import torch

import synth
from oracle import classical
from paper_0707_2347_gb300 import swmm as S
from tests.gpu_util import DEV, dev, fp_inputs, host, modp_inputs, padded

pytestmark = pytest.mark.gpu


def xvec_modp(n, p, tag=0):
    return synth.modp_matrix(synth.SEED_X, 1, n, p, tag).ravel()


def xvec_f64(n, tag=0):
    return synth.normal_matrix(synth.SEED_X, 1, n, tag).ravel().astype(np.float64)


@pytest.mark.parametrize("p", [251, 65521])
@pytest.mark.parametrize("rows,cols,pad", [(1, 1, 0), (37, 1000, 0), (256, 1027, 0), (513, 4096, 0), (300, 900, 3),
                                           (64, 0, 0)])
def test_matvec_modp_exact(handle, p, rows, cols, pad):
    M = synth.modp_matrix(synth.SEED_A, rows, cols, p, tag=rows)
    x = xvec_modp(cols, p, tag=cols)
    dM = padded(M, cols + pad) if pad else dev(M)
    y = torch.empty(rows, dtype=torch.int32, device=DEV)
    handle.matvec(dM, dev(x), y, S.Opts(mode=S.MODP, p=p))
    want = (M.astype(np.int64) @ x.astype(np.int64)) % p if cols else np.zeros(rows, np.int64)
    np.testing.assert_array_equal(host(y).astype(np.int64), want)


def test_matvec_modp_reduces_any_representative(handle):
    p = 65521
    rng = np.random.default_rng(7)
    M = rng.integers(0, 2**31 - 1, size=(40, 777), dtype=np.int64).astype(np.int32)
    x = xvec_modp(777, p)
    y = torch.empty(40, dtype=torch.int32, device=DEV)
    handle.matvec(dev(M), dev(x), y, S.Opts(mode=S.MODP, p=p))
    want = ((M.astype(np.int64) % p) @ x.astype(np.int64)) % p
    np.testing.assert_array_equal(host(y).astype(np.int64), want)


@pytest.mark.parametrize("rows,cols,pad", [(37, 1000, 0), (513, 4096, 0), (300, 901, 1)])
def test_matvec_fp64(handle, rows, cols, pad):
    M = synth.normal_matrix(synth.SEED_A, rows, cols, tag=rows)
    x = xvec_f64(cols)
    dM = padded(M, cols + pad) if pad else dev(M)
    y = torch.empty(rows, dtype=torch.float64, device=DEV)
    handle.matvec(dM, dev(x), y, S.Opts(mode=S.FP32))
    want = M.astype(np.float64) @ x
    scale = np.abs(M).astype(np.float64) @ np.abs(x)
    assert np.max(np.abs(host(y) - want) / scale) < 1e-13


@pytest.mark.parametrize("sched,n,depth", [(S.T9_ACC, 1024, 2), (S.T2_HLJJTT, 1000, 2), (S.CLASSICAL, 777, 0)])
def test_residual_vanishes_for_correct_product(handle, sched, n, depth):
    p = 65521
    A, B, C = modp_inputs(n, n, n, p, tag=n)
    x = xvec_modp(n, p)
    opts = S.Opts(mode=S.MODP, p=p, sched=sched, depth=depth)
    dA, dB, dC, dx = dev(A), dev(B), dev(C), dev(x)
    y0 = torch.empty(n, dtype=torch.int32, device=DEV)
    handle.matvec(dC, dx, y0, opts)
    handle.muladd(3, dA, dB, 5, dC, opts)
    r = torch.empty(n, dtype=torch.int32, device=DEV)
    handle.residual(3, dA, dB, 5, y0, dC, dx, r, opts)
    handle.sync()
    assert not host(r).any()


def test_residual_of_wrong_product_equals_definition(handle):
    # C is left as C_in (no product): r = (C_in - alpha A B - beta C_in) x
    p, m, k, n = 65521, 300, 500, 700
    A, B, C = modp_inputs(m, k, n, p, tag=1)
    x = xvec_modp(n, p)
    opts = S.Opts(mode=S.MODP, p=p)
    dC, dx = dev(C), dev(x)
    y0 = torch.empty(m, dtype=torch.int32, device=DEV)
    handle.matvec(dC, dx, y0, opts)
    r = torch.empty(m, dtype=torch.int32, device=DEV)
    handle.residual(2, dev(A), dev(B), 7, y0, dC, dx, r, opts)
    AB = classical.mul_modp(A, B, p).astype(np.int64)
    E = (C.astype(np.int64) - 2 * AB - 7 * C.astype(np.int64)) % p
    want = (E @ x.astype(np.int64)) % p
    np.testing.assert_array_equal(host(r).astype(np.int64), want)


def test_residual_beta_zero_needs_no_y0(handle):
    p, n = 251, 512
    A, B, _ = modp_inputs(n, n, n, p)
    x = xvec_modp(n, p)
    opts = S.Opts(mode=S.MODP, p=p, sched=S.T1_DHSS, depth=1)
    dA, dB, dx = dev(A), dev(B), dev(x)
    dC = torch.zeros((n, n), dtype=torch.int32, device=DEV)
    handle.mul(dA, dB, dC, opts)
    r = torch.empty(n, dtype=torch.int32, device=DEV)
    handle.residual(1, dA, dB, 0, None, dC, dx, r, opts)
    handle.sync()
    assert not host(r).any()


def test_residual_fp32_matches_host_fp64(handle):
    n = 1024
    A, B, C = fp_inputs(n, n, n, tag=2)
    x = xvec_f64(n)
    opts = S.Opts(mode=S.FP32, sched=S.T9_ACC, depth=2)
    dA, dB, dC, dx = dev(A), dev(B), dev(C), dev(x)
    y0 = torch.empty(n, dtype=torch.float64, device=DEV)
    handle.matvec(dC, dx, y0, opts)
    handle.muladd(1.0, dA, dB, 1.0, dC, opts)
    r = torch.empty(n, dtype=torch.float64, device=DEV)
    handle.residual(1.0, dA, dB, 1.0, y0, dC, dx, r, opts)
    Cout = host(dC).astype(np.float64)
    A64, B64, C64 = A.astype(np.float64), B.astype(np.float64), C.astype(np.float64)
    want = Cout @ x - A64 @ (B64 @ x) - C64 @ x
    scale = np.abs(A64) @ (np.abs(B64) @ np.abs(x)) + np.abs(C64) @ np.abs(x)
    assert np.max(np.abs(host(r) - want) / scale) < 1e-12
    # the product itself is FP32-accurate: |r| is a small fraction of the scale
    assert np.max(np.abs(host(r)) / scale) < 1e-4


def test_residual_rejects_missing_y0(handle):
    p, n = 251, 64
    A, B, C = modp_inputs(n, n, n, p)
    r = torch.empty(n, dtype=torch.int32, device=DEV)
    with pytest.raises(S.SwmmError):
        handle.residual(1, dev(A), dev(B), 1, None, dev(C), dev(xvec_modp(n, p)), r, S.Opts(mode=S.MODP, p=p))
