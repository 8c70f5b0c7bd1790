"""Bounded operand staging (SWMM_FLAG_LOWMEM), through the C ABI.

The schedules' own temporaries are the paper's count (Table 10); the
tensor-core operand staging sits on top of them.  With SWMM_FLAG_LOWMEM the
staging is one area of at most the bound: a fused level packs and
multiplies its seven products in groups that fit.  Results must stay
bit-exact, the reported staging must respect the bound, and the measured
device-memory high-water mark must not exceed temporaries plus the bound.
"""
import numpy as np
import pytest
import torch

from oracle import classical, probes
from paper_0707_2347_gb300 import swmm as S
from tests.gpu_util import DEV, dev, host, modp_inputs

pytestmark = pytest.mark.gpu

MIB = 1 << 20


@pytest.fixture
def fresh():
    h = S.Handle(0)
    yield h
    h.close()


@pytest.mark.parametrize("budget_kib", [300, 1024, 3072])
@pytest.mark.parametrize("sched,entry,p", [(S.T9_ACC, "muladd", 65521), (S.T1_DHSS, "mul", 251),
                                           (S.T3_IP, "inplace", 65521), (S.T2_HLJJTT, "muladd", 251)])
@pytest.mark.parametrize("graph", [0, S.FLAG_GRAPH])
def test_grouped_fused_levels_bit_exact(fresh, budget_kib, sched, entry, p, graph):
    """A small bound forces groups of 1 to 6 products per fused level (a
    product's operands: 2 x 256^2 entries in 1 or 2 fp16 limb planes)."""
    n, depth, alpha, beta = 1024, 2, 3, 5
    fresh.test_hook(S.HOOK_LOWMEM_BYTES, budget_kib * 1024)
    A, B, C = modp_inputs(n, n, n, p, tag=61)
    dA, dB, dC = dev(A), dev(B), dev(C)
    o = S.Opts(mode=S.MODP, p=p, sched=sched, depth=depth, flags=S.FLAG_LOWMEM | graph)
    if entry == "muladd":
        fresh.muladd(alpha, dA, dB, beta, dC, o)
        ref = classical.muladd_modp(alpha, A, B, beta, C, p)
    elif entry == "mul":
        fresh.mul(dA, dB, dC, o)
        ref = classical.mul_modp(A, B, p)
    else:
        fresh.mul_inplace(dA, dB, dC, o, alpha=alpha)
        ref = classical.muladd_modp(alpha, A, B, 0, C, p)
    fresh.sync()
    assert np.array_equal(host(dC), ref)
    one_product = 2 * 256 * 256 * (1 if p <= 256 else 2) * 2
    assert fresh.stats()["staging_bytes"] <= max(budget_kib * 1024, one_product)


def test_config2_lowmem_full_size(fresh):
    """The 8192^2 accumulate configuration (Table 9, depth 3, Z/65521) with
    staging bounded by 64 MiB: bit-exact spot rows and Freivalds, staging
    within the bound, measured peak within temporaries + bound."""
    p, n = 65521, 8192
    A, B, C = modp_inputs(n, n, n, p)
    dA, dB, dC = dev(A), dev(B), dev(C)
    o = S.Opts(mode=S.MODP, p=p, sched=S.T9_ACC, depth=3, flags=S.FLAG_LOWMEM)
    with fresh.measure_peak() as m:
        fresh.muladd(1, dA, dB, 1, dC, o)
        fresh.sync()
    st = fresh.stats()
    assert st["staging_bytes"] <= S.LOWMEM_STAGE_BYTES
    assert st["plan_extra_elems"] == st["paper_extra_elems"] == 2 * (4096 ** 2 + 2048 ** 2)
    assert 0 < m.peak <= 4 * st["plan_extra_elems"] + S.LOWMEM_STAGE_BYTES + MIB
    out = host(dC)
    rows = np.random.default_rng(1).choice(n, 16, replace=False)
    assert np.array_equal(out[rows], classical.rows_muladd_modp(rows, 1, A, B, 1, C, p))
    assert probes.freivalds_modp(1, A, B, 1, C, out, p, vectors=2)


@pytest.mark.parametrize("sched", [S.T3_IP, S.IPMM], ids=["IP-table3", "IPMM-alg2"])
def test_config3_lowmem_staging(fresh, sched):
    """Table 3 and Algorithm 2 at 16384^2 over Z/251 (depth 2; IPMM cut-off
    4096) allocate no temporaries; with SWMM_FLAG_LOWMEM their staging stays
    within 64 MiB as well.  Spot rows bit-exact."""
    p, n = 251, 16384
    A, B, _ = modp_inputs(n, n, n, p)
    dA, dB = dev(A), dev(B)
    dC = torch.zeros((n, n), dtype=torch.int32, device=DEV)
    with fresh.measure_peak() as m:
        if sched == S.T3_IP:
            fresh.mul_inplace(dA, dB, dC, S.Opts(mode=S.MODP, p=p, sched=S.T3_IP, depth=2, flags=S.FLAG_LOWMEM))
        else:
            fresh.mul(dA, dB, dC, S.Opts(mode=S.MODP, p=p, sched=S.IPMM, depth=2, ipmm_cutoff=4096,
                                         flags=S.FLAG_LOWMEM))
        fresh.sync()
    st = fresh.stats()
    assert st["workspace_bytes"] == 0
    assert st["staging_bytes"] <= S.LOWMEM_STAGE_BYTES
    assert 0 < m.peak <= S.LOWMEM_STAGE_BYTES + MIB
    out = host(dC)
    rows = np.random.default_rng(2).choice(n, 8, replace=False)
    assert np.array_equal(out[rows], classical.rows_muladd_modp(rows, 1, A, B, 0, None, p))
