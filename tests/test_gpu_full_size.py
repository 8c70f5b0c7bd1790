"""Full-size parity for the large configurations, through the C ABI.

At these sizes the oracle cannot form the whole product, so each test checks
  * sampled rows of the result bit for bit (mod p) or against FP64 (FP32
    mode) with the oracle's classical product, and
  * the whole result with a randomized residual (Freivalds) on the host,
plus the contract of the schedule: inputs a schedule keeps read-only come
back bit-identical, and the planned temporaries equal the paper's count.

  * Table 3 (IP, Section 5.1), C <- A B over Z/251, 16384^2, depth 2.
  * Algorithm 2 (IPMM, Section 7.1), same product, classical first level,
    cut-off 4096: A and B bit-identical, no temporaries outside C.
  * FP32 mode, 16384^2, Table 9 at depths 1-4: max |C - C64| / (|A| |B|)
    on spot rows within 1e-5 n^0.6.
  * 512 uneven C <- A B + C problems (m, k, n uniform in [384, 6144]; even
    index mod 65521, odd FP32) in one batched call, the large problems'
    schedules measured on the GPU (SWMM_FLAG_TUNE): every problem checked
    by its residual.
  * The shipped searched schedules for Tables 6 and 7's contracts and the
    mixed schedule Table 9 over Table 2, bit-exact at 512^2 and 1024^2.
"""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest
import torch

import synth
from oracle import classical, probes
from paper_0707_2347_gb300 import search as Q
from paper_0707_2347_gb300 import swmm as S
from tests.gpu_util import DEV, dev, fp_inputs, host, modp_inputs

pytestmark = pytest.mark.gpu

THREADS = 4


def spot_rows_modp(rows, alpha, A, B, beta, C, p):
    """The oracle's rows of alpha A B + beta C mod p, a few rows per host thread."""
    chunks = np.array_split(np.asarray(rows), THREADS)
    with ThreadPoolExecutor(THREADS) as ex:
        parts = list(ex.map(lambda r: classical.rows_muladd_modp(r, alpha, A, B, beta, C, p), chunks))
    return np.concatenate(parts, axis=0)


def _rows(n, count, seed=0):
    return np.sort(np.random.default_rng(seed).choice(n, count, replace=False))


@pytest.mark.parametrize("sched", [S.T3_IP, S.IPMM], ids=["IP-table3", "IPMM-alg2"])
def test_config3_inplace_16384_p251(handle, sched):
    p, n = 251, 16384
    A, B, _ = modp_inputs(n, n, n, p)
    dA, dB = dev(A), dev(B)
    dC = torch.zeros((n, n), dtype=torch.int32, device=DEV)
    if sched == S.T3_IP:
        handle.mul_inplace(dA, dB, dC, S.Opts(mode=S.MODP, p=p, sched=S.T3_IP, depth=2))
    else:
        handle.mul(dA, dB, dC, S.Opts(mode=S.MODP, p=p, sched=S.IPMM, depth=2, ipmm_cutoff=4096))
    handle.sync()
    st = handle.stats()
    assert st["plan_extra_elems"] == 0 and st["workspace_bytes"] == 0  # Table 3 and Algorithm 2: none
    out = host(dC)
    rows = _rows(n, 64)
    assert np.array_equal(out[rows], spot_rows_modp(rows, 1, A, B, 0, None, p))
    assert probes.freivalds_modp(1, A, B, None, None, out, p, vectors=2)
    if sched == S.IPMM:  # read-only inputs (Algorithm 2)
        assert np.array_equal(host(dA), A) and np.array_equal(host(dB), B)


def test_config4_fp32_16384_depths(handle):
    n = 16384
    A, B, C = fp_inputs(n, n, n)
    rows = _rows(n, 16)
    ref = A[rows].astype(np.float64) @ B.astype(np.float64) + C[rows].astype(np.float64)
    scale = float(np.abs(A).max()) * float(np.abs(B).max())
    dA, dB, dC0 = dev(A), dev(B), dev(C)
    bound = probes.fp_bound(n)
    for depth in (1, 2, 3, 4):
        dC = dC0.clone()
        handle.muladd(1.0, dA, dB, 1.0, dC, S.Opts(mode=S.FP32, sched=S.T9_ACC, depth=depth))
        handle.sync()
        got = dC[torch.from_numpy(rows).to(DEV)].double().cpu().numpy()
        err = float(np.abs(got - ref).max()) / scale
        assert err <= bound, (depth, err, bound)
        del dC
    torch.cuda.empty_cache()


def _check_problem(q):
    """Freivalds (mod p), or the FP64 residual of one batched problem against
    the FP32-mode bound: |(C - C64) x|_inf <= max|C - C64| |x|_1, so a
    result within 1e-5 n^0.6 |A| |B| elementwise has a residual, divided by
    |A| |B| |x|_1 as residual_f64 does, within the same bound."""
    A, B, C0, C1, mode = q
    if mode == S.MODP:
        return probes.freivalds_modp(1, A, B, 1, C0, C1, 65521, vectors=2)
    return probes.residual_f64(1.0, A, B, 1.0, C0, C1, vectors=2) <= probes.fp_bound(max(A.shape + B.shape))


def test_config5_batch512(handle):
    shapes = synth.batch_shapes(512, 384, 6144)
    gen = torch.Generator(device=DEV)
    gen.manual_seed(2024)
    probs, keep = [], []
    for i, (m, k, n) in enumerate(shapes):
        if i % 2 == 0:
            mk = lambda r, c: torch.randint(0, 65521, (r, c), generator=gen, device=DEV, dtype=torch.int32)
            mode = S.MODP
        else:
            mk = lambda r, c: torch.randn((r, c), generator=gen, device=DEV, dtype=torch.float32)
            mode = S.FP32
        A, B, C = mk(m, k), mk(k, n), mk(m, n)
        keep.append(C.clone())
        probs.append(dict(A=A, B=B, C=C, mode=mode, p=65521, alpha=1, beta=1, sched=S.AUTO))
    chosen = handle.muladd_batched(probs, S.FLAG_GRAPH | S.FLAG_TUNE)
    handle.sync()
    assert len(chosen) == 512
    measured = [c for c, (m, k, n) in zip(chosen, shapes) if m * k * n >= 3072 ** 3]
    assert measured and set(measured) <= {(S.CLASSICAL, 0), (S.T2_HLJJTT, 1), (S.T9_ACC, 1)}

    def job(i):
        q = probs[i]
        return _check_problem((host(q["A"]), host(q["B"]), host(keep[i]), host(q["C"]), q["mode"]))

    bad = []
    for lo in range(0, 512, 32):  # bounded host memory: 32 problems at a time
        with ThreadPoolExecutor(THREADS) as ex:
            ok = list(ex.map(job, range(lo, min(512, lo + 32))))
        bad += [lo + i for i, o in enumerate(ok) if not o]
    assert not bad, bad


def _mixed_t9_over_t2():
    rows = Q.table_rows(S.T9_ACC)
    for r in rows:
        if r.op == Q.MUL and r.kind == S.T9_ACC:
            r.kind = S.T2_HLJJTT
    spec = dict(accumulate=True, preserve=("A11", "A12", "A21", "A22", "B11", "B12", "B21", "B22"), temps=2,
                kinds=sorted({r.kind for r in rows if r.op == Q.MUL}), recompute=True)
    return rows, spec


@pytest.mark.parametrize("name", ["aclr14", "accr14", "t9_over_t2"])
@pytest.mark.parametrize("n,depth", [(512, 2), (1024, 3)])
def test_shipped_and_mixed_schedules(handle, name, n, depth):
    from paper_0707_2347_gb300 import schedules_found as F
    if name == "t9_over_t2":
        rows, spec = _mixed_t9_over_t2()
    else:
        rows, spec = F.rows(name), F.spec(name)
    Q.set_schedule(handle, rows, **spec)
    p, alpha, beta = 65521, 3, 5
    A, B, C = modp_inputs(n, n, n, p, tag=41)
    dA, dB, dC = dev(A), dev(B), dev(C)
    o = S.Opts(mode=S.MODP, p=p, sched=S.CUSTOM, depth=depth)
    if len(spec["preserve"]) == 8:
        handle.muladd(alpha, dA, dB, beta, dC, o)
    else:
        handle.mul_inplace(dA, dB, dC, o, alpha=alpha, beta=beta)
    handle.sync()
    assert np.array_equal(host(dC), classical.muladd_modp(alpha, A, B, beta, C, p))
    h = n // 2
    hA, hB = host(dA), host(dB)
    for blk in spec["preserve"]:
        M, M0 = (hA, A) if blk[0] == "A" else (hB, B)
        i, j = int(blk[1]) - 1, int(blk[2]) - 1
        assert np.array_equal(M[i * h:(i + 1) * h, j * h:(j + 1) * h], M0[i * h:(i + 1) * h, j * h:(j + 1) * h]), blk
    paper, plan = Q.schedule_workspace(rows, n, n, n, o, **spec)
    assert handle.stats()["plan_extra_elems"] == plan
