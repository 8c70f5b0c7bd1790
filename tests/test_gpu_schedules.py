"""Every schedule through the C ABI against the CPU oracle.

For each table the GPU result must equal the plain definition bit for bit
over Z/pZ, inputs the table declares read-only must come back bit-identical,
and the temporaries the plan allocates must equal the paper's count."""
import numpy as np
import pytest

import synth
from oracle import classical, counts, probes
from paper_0707_2347_gb300 import swmm as S
from tests.gpu_util import dev, fp_inputs, host, modp_inputs

pytestmark = pytest.mark.gpu

MUL = [S.T1_DHSS]
MULADD = [S.T2_HLJJTT, S.T9_ACC]
INPLACE = [S.T3_IP, S.T4_OVL, S.T4M_OVL, S.T5_OVR]
INPLACE_ACC = [S.T6_ACLR, S.T7_ACCR, S.T8_ACR]
NAME = {S.T1_DHSS: "T1", S.T2_HLJJTT: "T2", S.T9_ACC: "Acc", S.T3_IP: "IP", S.T4_OVL: "OvL", S.T4M_OVL: "OvLM",
        S.T5_OVR: "OvR", S.T6_ACLR: "AcLR", S.T7_ACCR: "AccR", S.T8_ACR: "AcR"}
# operand blocks each schedule leaves untouched (Sections 3, 5, 6)
KEEP = {S.T1_DHSS: "AB", S.T2_HLJJTT: "AB", S.T9_ACC: "AB", S.T4_OVL: "B", S.T4M_OVL: "B", S.T5_OVR: "A",
        S.T7_ACCR: "A", S.T8_ACR: "A", S.T3_IP: "", S.T6_ACLR: ""}


def run(handle, sched, A, B, C, opts, alpha, beta):
    dA, dB, dC = dev(A), dev(B), dev(C)
    if sched in MUL or sched == S.IPMM:
        handle.mul(dA, dB, dC, opts)
    elif sched in MULADD:
        handle.muladd(alpha, dA, dB, beta, dC, opts)
    elif sched in INPLACE:
        handle.mul_inplace(dA, dB, dC, opts, alpha=alpha)
    else:
        handle.mul_inplace(dA, dB, dC, opts, alpha=alpha, beta=beta)
    handle.sync()
    return host(dC), host(dA), host(dB)


def expected(sched, A, B, C, alpha, beta, p):
    if sched in MULADD or sched in INPLACE_ACC:
        return classical.muladd_modp(alpha, A, B, beta, C, p)
    a = 1 if sched in MUL or sched == S.IPMM else alpha
    return classical.muladd_modp(a, A, B, 0, C, p)


ALL = MUL + MULADD + INPLACE + INPLACE_ACC


@pytest.mark.parametrize("sched", ALL, ids=[NAME[s] for s in ALL])
@pytest.mark.parametrize("n,depth", [(256, 1), (512, 2), (1024, 3)])
@pytest.mark.parametrize("variant", ["fused", "unfused", "simt"])
@pytest.mark.parametrize("p", [251, 65521])
def test_schedule_modp(handle, sched, n, depth, variant, p):
    if variant == "simt" and n > 512:
        pytest.skip("the SIMT diagnostic leaf is slow")
    flags = {"fused": 0, "unfused": S.FLAG_UNFUSED, "simt": S.FLAG_SIMT_LEAF}[variant]
    A, B, C = modp_inputs(n, n, n, p, tag=depth)
    alpha, beta = 3, 5
    o = S.Opts(mode=S.MODP, p=p, sched=sched, depth=depth, flags=flags)
    out, A2, B2 = run(handle, sched, A, B, C, o, alpha, beta)
    assert np.array_equal(out, expected(sched, A, B, C, alpha, beta, p))
    keep = KEEP[sched]
    if "A" in keep:
        assert np.array_equal(A2, A)
    if "B" in keep:
        assert np.array_equal(B2, B)
    if sched == S.T4M_OVL:
        h = n // 2
        assert np.array_equal(A2[:, h:], A[:, h:])  # A12, A22 preserved
    if sched == S.T8_ACR:
        h = n // 2
        assert np.array_equal(B2[:h, :h], B[:h, :h]) and np.array_equal(B2[h:, h:], B[h:, h:])
    st = handle.stats()
    lv = depth if variant == "unfused" else depth - 1
    assert st["plan_extra_elems"] == st["paper_extra_elems"] == counts.mem_depth(NAME[sched], n, lv)


@pytest.mark.parametrize("sched,shape", [(S.T1_DHSS, (512, 256, 1024)), (S.T1_DHSS, (256, 1024, 512)),
                                         (S.T2_HLJJTT, (512, 256, 1024)), (S.T8_ACR, (256, 512, 1024)),
                                         (S.T3_IP, (1024, 512, 512)), (S.T2_HLJJTT, (384, 640, 256))])
def test_rectangular(handle, sched, shape):
    m, k, n = shape
    p = 65521
    A, B, C = modp_inputs(m, k, n, p, tag=7)
    o = S.Opts(mode=S.MODP, p=p, sched=sched, depth=2)
    out, _, _ = run(handle, sched, A, B, C, o, 2, 3)
    assert np.array_equal(out, expected(sched, A, B, C, 2, 3, p))


@pytest.mark.parametrize("n,k,depth,cutoff,acc", [(512, 512, 1, 128, 0), (1024, 2048, 2, 256, 0),
                                                  (1024, 1024, 2, 256, S.T9_ACC)])
def test_ipmm(handle, n, k, depth, cutoff, acc):
    p = 65521
    A, B, _ = modp_inputs(n, k, n, p, tag=3)
    C = np.zeros((n, n), dtype=np.int32)
    o = S.Opts(mode=S.MODP, p=p, sched=S.IPMM, depth=depth, ipmm_cutoff=cutoff, ipmm_acc=acc)
    out, A2, B2 = run(handle, S.IPMM, A, B, C, o, 1, 0)
    assert np.array_equal(out, classical.mul_modp(A, B, p))
    assert np.array_equal(A2, A) and np.array_equal(B2, B)
    st = handle.stats()
    assert st["plan_extra_elems"] == 0 and st["workspace_bytes"] == 0


@pytest.mark.parametrize("sched", [S.T9_ACC, S.T2_HLJJTT, S.T1_DHSS], ids=["Acc", "T2", "T1"])
@pytest.mark.parametrize("n,depth", [(1024, 1), (1024, 2), (2048, 2)])
def test_fp32_mode(handle, sched, n, depth):
    A, B, C = fp_inputs(n, n, n)
    dA, dB, dC = dev(A), dev(B), dev(C)
    o = S.Opts(mode=S.FP32, sched=sched, depth=depth)
    if sched == S.T1_DHSS:
        handle.mul(dA, dB, dC, o)
        ref = classical.mul_f64(A, B)
    else:
        handle.muladd(1.0, dA, dB, 1.0, dC, o)
        ref = classical.muladd_f64(1.0, A, B, 1.0, C)
    handle.sync()
    err = probes.fp_error(host(dC), ref, A, B)["max_rel"]
    assert err <= probes.fp_bound(n), err


def test_config1_t1_512_p251(handle):
    """C <- A B over Z/251, 512 x 512, one Table 1 level, 256^3 leaves."""
    p, n = 251, 512
    A, B, _ = modp_inputs(n, n, n, p)
    for flags in (0, S.FLAG_UNFUSED):
        C = np.zeros((n, n), dtype=np.int32)
        out, A2, B2 = run(handle, S.T1_DHSS, A, B, C, S.Opts(mode=S.MODP, p=p, sched=S.T1_DHSS, depth=1, flags=flags),
                          1, 0)
        assert np.array_equal(out, np.array(classical.mul_modp(A, B, p)))
        assert np.array_equal(A2, A) and np.array_equal(B2, B)
    assert handle.stats()["plan_extra_elems"] == 131072  # 2 * 256^2 (Table 1)


def test_config2_full_size_spot(handle):
    """C <- A B + C over Z/65521 at 8192^2, Table 9 depth 3: 64 spot rows
    bit-exact plus a two-vector Freivalds residual of the whole result."""
    p, n = 65521, 8192
    A, B, C = modp_inputs(n, n, n, p)
    dA, dB, dC = dev(A), dev(B), dev(C)
    handle.muladd(1, dA, dB, 1, dC, S.Opts(mode=S.MODP, p=p, sched=S.T9_ACC, depth=3))
    handle.sync()
    out = host(dC)
    rows = np.random.default_rng(0).choice(n, 64, replace=False)
    assert np.array_equal(out[rows], classical.rows_muladd_modp(rows, 1, A, B, 1, C, p))
    assert probes.freivalds_modp(1, A, B, 1, C, out, p, vectors=2)
    assert handle.stats()["plan_extra_elems"] == 2 * (4096 ** 2 + 2048 ** 2)  # fused third level


def test_invalid_arguments(handle):
    p = 65521
    A, B, C = modp_inputs(64, 32, 64, p)
    dA, dB, dC = dev(A), dev(B), dev(C)
    with pytest.raises(S.SwmmError) as e:
        handle.mul_inplace(dA, dB, dC, S.Opts(mode=S.MODP, p=p, sched=S.T4_OVL, depth=1))
    assert e.value.code == S.EINVAL
    with pytest.raises(S.SwmmError):
        handle.mul(dA, dB, dC, S.Opts(mode=S.MODP, p=1, sched=S.T1_DHSS, depth=1))
    with pytest.raises(S.SwmmError):
        handle.muladd(1, dA, dB, 1, dC, S.Opts(mode=S.MODP, p=p, sched=S.T3_IP, depth=1))


@pytest.mark.parametrize("m,k,n,depth", [(1024, 1024, 512, 2), (2048, 1536, 512, 3), (1536, 512, 256, 1),
                                         (768, 768, 256, 2)])
@pytest.mark.parametrize("p", [251, 65521])
@pytest.mark.parametrize("unfused", [False, True])
def test_ip0vmm(handle, m, k, n, depth, p, unfused):
    """Algorithm 1: C <- alpha A B overwriting A only, no extra memory."""
    A, B, C = modp_inputs(m, k, n, p, tag=5)
    o = S.Opts(mode=S.MODP, p=p, sched=S.IP0VMM, depth=depth, flags=S.FLAG_UNFUSED if unfused else 0)
    dA, dB, dC = dev(A), dev(B), dev(C)
    handle.mul_inplace(dA, dB, dC, o, alpha=7)
    handle.sync()
    assert np.array_equal(host(dC), classical.muladd_modp(7, A, B, 0, C, p))
    assert np.array_equal(host(dB), B)
    st = handle.stats()
    assert st["plan_extra_elems"] == 0 and st["workspace_bytes"] == 0


def test_ip0vmm_fp32(handle):
    m, k, n = 2048, 1024, 512
    A, B, C = fp_inputs(m, k, n, tag=4)
    dA, dB, dC = dev(A), dev(B), dev(C)
    handle.mul_inplace(dA, dB, dC, S.Opts(mode=S.FP32, sched=S.IP0VMM, depth=2))
    handle.sync()
    err = probes.fp_error(host(dC), classical.mul_f64(A, B), A, B)["max_rel"]
    assert err <= probes.fp_bound(k), err


@pytest.mark.parametrize("t,n,depth", [(2, 1024, 3), (3, 768, 2), (4, 1024, 1)])
@pytest.mark.parametrize("base", [0, S.T9_ACC], ids=["T2", "Acc"])
@pytest.mark.parametrize("unfused", [False, True])
def test_tblock(handle, t, n, depth, base, unfused):
    """Section 7.2: C <- alpha A B + beta C by t x t blocks of accumulating
    Winograd calls; inputs read-only; one block call's temporaries."""
    p = 65521
    A, B, C = modp_inputs(n, n, n, p, tag=t)
    o = S.Opts(mode=S.MODP, p=p, sched=S.TBLOCK, depth=depth, tblock=t, ipmm_acc=base,
               flags=S.FLAG_UNFUSED if unfused else 0)
    dA, dB, dC = dev(A), dev(B), dev(C)
    handle.muladd(3, dA, dB, 5, dC, o)
    handle.sync()
    assert np.array_equal(host(dC), classical.muladd_modp(3, A, B, 5, C, p))
    assert np.array_equal(host(dA), A) and np.array_equal(host(dB), B)
    st = handle.stats()
    lv = depth if unfused else depth - 1
    assert st["plan_extra_elems"] == st["paper_extra_elems"] == counts.mem_depth("Acc" if base else "T2", n // t, lv)


def test_tblock_rectangular_fp32(handle):
    m, k, n = 1536, 1024, 768
    A, B, C = fp_inputs(m, k, n, tag=6)
    dC = dev(C)
    handle.muladd(1.0, dev(A), dev(B), 1.0, dC, S.Opts(mode=S.FP32, sched=S.TBLOCK, depth=2, tblock=2))
    handle.sync()
    err = probes.fp_error(host(dC), classical.muladd_f64(1.0, A, B, 1.0, C), A, B)["max_rel"]
    assert err <= probes.fp_bound(k), err


@pytest.mark.parametrize("n,depth", [(2048, 4), (4096, 4)])
def test_fp32_mode_depth4_within_bound(handle, n, depth):
    """Four Winograd levels keep the FP32-mode error within 1e-5 n^0.6: the
    leaves split each scaled operand into fp16 hi + lo (22 bits)."""
    A, B, C = fp_inputs(n, n, n, tag=9)
    dC = dev(C)
    handle.muladd(1.0, dev(A), dev(B), 1.0, dC, S.Opts(mode=S.FP32, sched=S.T9_ACC, depth=depth))
    handle.sync()
    idx = np.linspace(0, n - 1, 32).astype(np.int64)
    ref = A[idx].astype(np.float64) @ B.astype(np.float64) + C[idx].astype(np.float64)
    err = np.abs(host(dC)[idx] - ref).max() / (np.abs(A).max() * np.abs(B).max())
    assert err <= probes.fp_bound(n), err


def test_fp32_scaling_handles_large_and_small_magnitudes(handle):
    """Operands far outside fp16's range are scaled by a power of two."""
    n = 1024
    A, B, C = fp_inputs(n, n, n, tag=10)
    for sa, sb in [(1e6, 1e-3), (1e-8, 1e-8), (3e4, 3e4)]:
        A2, B2 = (A * sa).astype(np.float32), (B * sb).astype(np.float32)
        dC = dev(C)
        handle.muladd(1.0, dev(A2), dev(B2), 0.0, dC, S.Opts(mode=S.FP32, sched=S.T9_ACC, depth=2))
        handle.sync()
        err = probes.fp_error(host(dC), classical.mul_f64(A2, B2), A2, B2)["max_rel"]
        assert err <= probes.fp_bound(n), (sa, sb, err)


@pytest.mark.parametrize("graph", [False, True], ids=["eager", "graph"])
def test_small_fused_levels_share_launches(handle, graph):
    """Table 9 depth 3 at 2048^2: 49 fused levels of 7 x 256^3 products; the
    independent ones (different targets, or reduce-adds into one target)
    share grouped launches, and the result stays exact."""
    p, n = 65521, 2048
    A, B, C = modp_inputs(n, n, n, p, tag=31)
    dC = dev(C)
    o = S.Opts(mode=S.MODP, p=p, sched=S.T9_ACC, depth=3, flags=S.FLAG_GRAPH if graph else 0)
    handle.muladd(3, dev(A), dev(B), 5, dC, o)
    handle.sync()
    assert np.array_equal(host(dC), classical.muladd_modp(3, A, B, 5, C, p))
    st = handle.stats()
    assert st["leaf_products"] == 343
    assert st["leaf_launches"] < 49
