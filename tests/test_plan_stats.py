"""The planning pass's counts on the CPU (swmm_plan_stats): level packs,
staging, additions and launches derived from the tables by hand.

Table 9 at 8192^2 depth 2 (C <- AB + C, read-only A and B): the top level's
eight S/T rows are recorded as sums and its seven fused levels are packed in
one pass per side (2 launches) reading A and B once (2 x 8192^2 x 4 B) and
writing 49 operand pairs of 2 limb planes of 2048 x 2048 fp16 per operand;
the seven C-side rows (Z1, Z3, W1, U2, U1, U5, U7) each touch a 4096^2
block, and the product P1, which Table 9 writes into a temporary without
accumulation, needs that temporary zeroed first: 10 elementwise launches.
Table 1 at 16384^2 depth 3: the top level runs its 15 rows; each of the
seven level-2 Table 1 calls packs in one pass (2), runs its 7 C-side rows
and zeroes the destination of each of its 7 non-accumulating fused levels:
15 + 7 x 16 = 127.
"""
import pytest

from paper_0707_2347_gb300 import swmm as S

PAIR = 2 * (2 * 2048 * 2048 * 2)  # A and B operand of one 2048^3 product, 2 fp16 limb planes each


def test_table9_level_pack_counts():
    n = 8192
    st = S.plan_stats(n, n, n, S.Opts(mode=S.MODP, p=65521, sched=S.T9_ACC, depth=2))
    assert st["level_packs"] == 1
    assert st["staging_bytes"] == 49 * PAIR
    assert st["pack_bytes"] == 4 * 2 * n * n + 49 * PAIR
    assert st["ew_launches"] == 2 + 7 + 1
    assert st["add_elems"] == 7 * (n // 2) ** 2
    assert st["leaf_products"] == 49 and st["leaf_flops"] == 49 * 2 * (n // 4) ** 3
    assert st["plan_extra_elems"] == st["paper_extra_elems"] == 2 * (n // 2) ** 2


def test_bounded_staging_and_inplace_tables():
    """Bounded staging never packs a whole level.  Tables 3, 4 and 5 store
    products in operand quadrants that later products read, so their
    levels pack one at a time; Tables 6, 7 and 8 only park S and T sums in
    operand quadrants (recorded, the blocks keep their input values until
    the products are written), so they pack in one pass."""
    n = 8192
    low = S.plan_stats(n, n, n, S.Opts(mode=S.MODP, p=65521, sched=S.T9_ACC, depth=2, flags=S.FLAG_LOWMEM))
    assert low["level_packs"] == 0 and low["staging_bytes"] <= S.LOWMEM_STAGE_BYTES
    for sched in (S.T3_IP, S.T4_OVL, S.T5_OVR):
        st = S.plan_stats(n, n, n, S.Opts(mode=S.MODP, p=65521, sched=sched, depth=2))
        assert st["level_packs"] == 0 and st["staging_bytes"] == 7 * PAIR, sched
    for sched in (S.T6_ACLR, S.T7_ACCR, S.T8_ACR):
        st = S.plan_stats(n, n, n, S.Opts(mode=S.MODP, p=65521, sched=sched, depth=2))
        assert st["level_packs"] == 1 and st["staging_bytes"] == 49 * PAIR, sched


def test_table9_depth3_every_level2_call_packs_once():
    """8192^2 depth 3: all seven level-2 calls (four by Table 9, one by
    Table 1, one each by Tables 6 and 7) pack in one pass, two areas in
    turn."""
    n = 8192
    st = S.plan_stats(n, n, n, S.Opts(mode=S.MODP, p=65521, sched=S.T9_ACC, depth=3))
    assert st["level_packs"] == 7
    assert st["staging_bytes"] == 2 * 49 * (2 * (2 * 1024 * 1024 * 2))


def test_table1_depth3_counts():
    """Every level-2 table of Table 1 (read-only, C <- AB) packs in one pass;
    planned with disjoint placeholder addresses, no recorded sum is written
    out because some unrelated block was written (with every placeholder at
    address 0 the count was higher)."""
    n = 16384
    st = S.plan_stats(n, n, n, S.Opts(mode=S.MODP, p=65521, sched=S.T1_DHSS, depth=3))
    assert st["level_packs"] == 7
    assert st["ew_launches"] == 15 + 7 * (2 + 7 + 7)
    assert st["leaf_products"] == 343


def test_fp32_level_pack_stages_amax_words():
    n = 16384
    st = S.plan_stats(n, n, n, S.Opts(mode=S.FP32, sched=S.T9_ACC, depth=2))
    pair = 2 * (2 * 4096 * 4096 * 2)
    assert st["level_packs"] == 1
    assert st["staging_bytes"] == 49 * pair + 1024  # the amax words share the area
    assert st["ew_launches"] == 3 + 7 + 1  # amax pass, two level-pack launches


def test_plan_stats_rejects_bad_options():
    with pytest.raises(S.SwmmError):  # Table 3 needs k = n <= m
        S.plan_stats(500, 1000, 1000, S.Opts(mode=S.MODP, p=65521, sched=S.T3_IP, depth=2))
    with pytest.raises(S.SwmmError):  # p must satisfy 2 < p < 2^16
        S.plan_stats(100, 100, 100, S.Opts(mode=S.MODP, p=1, sched=S.T9_ACC, depth=1))


def test_searched_schedules_level_packs():
    """The shipped searched schedules at 8192^2 depth 2: ab12 (parks S and T
    in C), acc16 and accr14 pack all seven fused levels in one pass;
    aclr14 stores a product in an operand quadrant that a later product
    reads and packs per level.  Planned temporaries equal the contract's."""
    from paper_0707_2347_gb300 import schedules_found as F
    from paper_0707_2347_gb300 import search as Q
    n = 8192
    o = S.Opts(mode=S.MODP, p=65521, sched=S.CUSTOM, depth=2)
    packs = {"ab12": 1, "acc16": 1, "accr14": 1, "aclr14": 0}
    for name, want in packs.items():
        st = Q.schedule_stats(F.rows(name), n, n, n, o, **F.spec(name))
        assert st["level_packs"] == want, name
        assert st["staging_bytes"] == (49 if want else 7) * PAIR, name
        assert st["plan_extra_elems"] == st["paper_extra_elems"], name


def test_cost_model_tracks_measured_times():
    """The autotuner's model of Table 9 (mod 65521) against times measured
    on a GB300 with graph replays (inputs resident): 16384^2 depth 1 18.63
    ms, depth 2 18.84 ms, 8192^2 depth 3 4.149 ms, 32768^2 depth 2 135.0
    ms.  Within 5% each; a ranking aid, not a measurement."""
    from paper_0707_2347_gb300 import search as Q
    rows = Q.table_rows(S.T9_ACC)
    keep = ("A11", "A12", "A21", "A22", "B11", "B12", "B21", "B22")
    for n, depth, ms in [(16384, 1, 18.63), (16384, 2, 18.84), (8192, 3, 4.149), (32768, 2, 135.0)]:
        o = S.Opts(mode=S.MODP, p=65521, sched=S.CUSTOM, depth=depth)
        us = Q.schedule_model_us(rows, n, n, n, o, accumulate=True, preserve=keep, temps=2, kinds=(1, 6, 7, 9),
                                 recompute=True)
        assert abs(us / 1000.0 - ms) < 0.05 * ms, (n, depth, us, ms)
