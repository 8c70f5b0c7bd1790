#!/usr/bin/env python
"""Benchmark of the memory-efficient Strassen-Winograd library on GB300.

Default workload (the accumulate configuration): C <- A B + C over Z/65521,
A, B, C 8192 x 8192 with entries uniform in [0, 65520], Table 9 (Acc,
read-only inputs, two temporaries) at three Winograd levels, last level
fused.  Metric: effective GOP/s = 2 m n k / t over the whole call.

Printed JSON line (rank 0): value (device-resident inputs), e2e (host
buffers, copies inside the timed region), the classical tcgen05 GEMM of the
same library on the same inputs, the roofline of the leaf GEMM kernel
(event-timed inside the timed region), peak extra device bytes against the
paper's count, clocks sampled during the timed region, and a CPU baseline
(the oracle on a bounded sample).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
       python bench.py --impl reference ...   (the CPU oracle on samples)
Under torchrun every rank runs an independent replica (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

MODP, FP32 = 0, 1
CLASSICAL, T1, T2, IP, T9, IPMM, IP0VMM, TBLOCK, CUSTOM = 0, 1, 2, 3, 9, 10, 12, 13, 14

WORKLOADS = {
    # the accumulate schedule at 8192^2, three levels (default)
    "t9_8192_p65521": dict(desc="C<-AB+C over Z/65521, 8192^2, Table 9 (Acc) depth 3, fused last level",
                           m=8192, k=8192, n=8192, mode=MODP, p=65521, sched=T9, depth=3, entry="muladd"),
    "t9_16384_p65521": dict(desc="C<-AB+C over Z/65521, 16384^2, Table 9 (Acc) depth 2, fused last level",
                            m=16384, k=16384, n=16384, mode=MODP, p=65521, sched=T9, depth=2, entry="muladd"),
    "t9_16384_p65521_d1": dict(desc="C<-AB+C over Z/65521, 16384^2, Table 9 (Acc) depth 1 (fused level)",
                               m=16384, k=16384, n=16384, mode=MODP, p=65521, sched=T9, depth=1, entry="muladd"),
    "t9_2048_p65521_d1": dict(desc="C<-AB+C over Z/65521, 2048^2, Table 9 (Acc) depth 1: one fused level, 7 x 1024^3",
                              m=2048, k=2048, n=2048, mode=MODP, p=65521, sched=T9, depth=1, entry="muladd"),
    "t9_4096_p65521_d2": dict(desc="C<-AB+C over Z/65521, 4096^2, Table 9 (Acc) depth 2, fused last level",
                              m=4096, k=4096, n=4096, mode=MODP, p=65521, sched=T9, depth=2, entry="muladd"),
    "classical_4096_p65521": dict(desc="C<-AB+C over Z/65521, 4096^2, classical tcgen05 product",
                                  m=4096, k=4096, n=4096, mode=MODP, p=65521, sched=CLASSICAL, depth=0,
                                  entry="muladd"),
    "t1_512_p251": dict(desc="C<-AB over Z/251, 512^2, Table 1 depth 1", m=512, k=512, n=512, mode=MODP, p=251,
                        sched=T1, depth=1, entry="mul"),
    "ip_16384_p251": dict(desc="C<-AB over Z/251, 16384^2, Table 3 (IP) depth 2", m=16384, k=16384, n=16384,
                          mode=MODP, p=251, sched=IP, depth=2, entry="inplace"),
    "ipmm_16384_p251": dict(desc="C<-AB over Z/251, 16384^2, Algorithm 2 (IPMM), depth 2, cut-off 4096",
                            m=16384, k=16384, n=16384, mode=MODP, p=251, sched=IPMM, depth=2, entry="mul",
                            cutoff=4096),
    "batch512": dict(desc="512 independent C<-AB+C, m,k,n uniform in [384,6144], even index mod 65521, odd FP32, "
                          "schedule/depth per problem measured on the GPU for the large ones (model for the rest), "
                          "odd sizes peeled, one CUDA graph",
                     m=0, k=0, n=0, mode=MODP, p=65521, sched=-1, depth=0, entry="batch", count=512, lo=384,
                     hi=6144),
    "t1_16384_p251": dict(desc="C<-AB over Z/251, 16384^2, Table 1 depth 2", m=16384, k=16384, n=16384, mode=MODP,
                          p=251, sched=T1, depth=2, entry="mul"),
    "fp32_t9_8192": dict(desc="C<-AB+C FP32 mode (3 fp16 split products), 8192^2, Table 9 depth 2",
                         m=8192, k=8192, n=8192, mode=FP32, p=0, sched=T9, depth=2, entry="muladd"),
    "t9_32768_p65521": dict(desc="C<-AB+C over Z/65521, 32768^2, Table 9 (Acc) depth 2, fused last level",
                            m=32768, k=32768, n=32768, mode=MODP, p=65521, sched=T9, depth=2, entry="muladd"),
    "tblock2_16384_p65521": dict(desc="C<-AB+C over Z/65521, 16384^2, Section 7.2 t=2 blocks by Table 9, depth 1",
                                 m=16384, k=16384, n=16384, mode=MODP, p=65521, sched=TBLOCK, depth=1,
                                 entry="muladd", tblock=2, acc=T9),
    "ip0vmm_16384x8192x4096_p251": dict(desc="C<-AB over Z/251, m=16384 k=8192 n=4096, Algorithm 1 (IP0vMM) depth 2",
                                        m=16384, k=8192, n=4096, mode=MODP, p=251, sched=IP0VMM, depth=2,
                                        entry="inplace"),
    # Table 1 against the schedule the pebble-game search finds for the same
    # contract (read-only C <- AB, two temporaries) when recursive calls may
    # accumulate: 12 block additions per level instead of 15
    "t1_16384_p65521_d3": dict(desc="C<-AB over Z/65521, 16384^2, Table 1 depth 3", m=16384, k=16384, n=16384,
                               mode=MODP, p=65521, sched=T1, depth=3, entry="mul"),
    "searched12_16384_p65521_d3": dict(desc="C<-AB over Z/65521, 16384^2, searched read-only schedule with two "
                                            "temporaries and 12 block additions (Table 2 calls accumulate), depth 3",
                                       m=16384, k=16384, n=16384, mode=MODP, p=65521, sched=CUSTOM, depth=3,
                                       entry="mul", found="ab12"),
    # Table 9's contract with 16 block additions instead of 17: a schedule the
    # pebble-game search found, shipped in schedules_found.py
    "searched16_8192_p65521_d3": dict(desc="C<-AB+C over Z/65521, 8192^2, searched read-only schedule with two "
                                           "temporaries and 16 block additions (Table 9: 17), depth 3",
                                      m=8192, k=8192, n=8192, mode=MODP, p=65521, sched=CUSTOM, depth=3,
                                      entry="muladd", found="acc16"),
    # a mixed schedule: Table 9 at the top level, Table 2 (14 block additions
    # instead of 17, one more temporary) for its accumulating calls below
    "t9_over_t2_8192_p65521": dict(desc="C<-AB+C over Z/65521, 8192^2, Table 9 rows at every Table 9 level with "
                                        "Table 2 for their accumulating calls, depth 3",
                                   m=8192, k=8192, n=8192, mode=MODP, p=65521, sched=CUSTOM, depth=3,
                                   entry="muladd", table=T9, replace={T9: T2, 6: T2, 7: T2}),
    # FP32 mode: error and speed per size and depth
    "fp32_sweep": dict(desc="C<-AB+C FP32 mode (3 fp16 split products), n in {4096, 8192, 16384}, "
                            "Table 9 depth 1-4 vs classical",
                       m=16384, k=16384, n=16384, mode=FP32, p=0, sched=T9, depth=0, entry="sweep",
                       ns=(4096, 8192, 16384), depths=(1, 2, 3, 4)),
}
DEFAULT = "t9_8192_p65521"

# DRAM bytes (read + write) of the leaf GEMM per fused level.  One ncu
# capture of the same kernel build on one fused level (7 products of
# 1024^3, the 2048^2 depth-1 workload) read 75.6 MB and wrote 1.4 MB; the
# 8192^2 depth-3 step merges its 49 fused levels of that size into fewer
# launches with the same operands and targets per level, so the average
# launch moves 77.0 MB x 49 / (launches per step).
TRAFFIC_PER_LEVEL = 77.0e6
FUSED_LEVELS = {"t9_8192_p65521": 49, "t9_2048_p65521_d1": 1}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d["bf16_tflops"], d["bf16_tflops_sustained"], d["hbm_gbs"], "measured"
    except Exception:
        return 1900.0, 1700.0, 6800.0, "fallback"


def make_inputs(w):
    m, k, n = w["m"], w["k"], w["n"]
    if w["mode"] == MODP:
        p = w["p"]
        return (synth.modp_matrix(synth.SEED_A, m, k, p), synth.modp_matrix(synth.SEED_B, k, n, p),
                synth.modp_matrix(synth.SEED_C, m, n, p))
    return (synth.normal_matrix(synth.SEED_A, m, k), synth.normal_matrix(synth.SEED_B, k, n),
            synth.normal_matrix(synth.SEED_C, m, n))


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons while timing."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        loaded = [s for s in sm if s > 0.5 * mx] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _oracle_rows(w, A, B, C, sel):
    from oracle import classical
    if w["mode"] == MODP:
        classical.rows_muladd_modp(sel, 1, A, B, 1, C, w["p"])
    else:
        classical.rows_muladd_f64(sel, 1.0, A, B, 1.0, C)


def _oracle_parallel(w, A, B, C, rows, threads, seed):
    """The oracle's classical product on `threads` host threads at once, each
    on its own sample of `rows` rows (numpy's integer and float matmul loops
    release the interpreter lock, so the threads run on separate cores).
    Returns the wall time."""
    from concurrent.futures import ThreadPoolExecutor
    m = w["m"]
    rng = np.random.default_rng(seed)
    sels = [rng.choice(m, rows, replace=False) for _ in range(threads)]
    with ThreadPoolExecutor(threads) as ex:
        t0 = time.perf_counter()
        list(ex.map(lambda sel: _oracle_rows(w, A, B, C, sel), sels))
        return time.perf_counter() - t0


def cpu_baseline(w, A, B, C, budget_s: float = 16.0):
    """The oracle's classical product on every host core, each core on a
    bounded sample of rows of the same product; the one-core figure beside it."""
    m, k, n = w["m"], w["k"], w["n"]
    cores = os.cpu_count() or 1
    rows = 2
    while True:  # one core: size the sample to about a quarter of the budget
        t0 = time.perf_counter()
        _oracle_rows(w, A, B, C, np.random.default_rng(5).choice(m, rows, replace=False))
        dt1 = time.perf_counter() - t0
        if dt1 > budget_s / 8 or rows >= m:
            break
        rows = min(m, max(rows * 2, int(rows * budget_s / 8 / max(dt1, 1e-3))))
    one = 2.0 * rows * n * k / dt1 / 1e9
    dt = _oracle_parallel(w, A, B, C, rows, cores, 7)
    gops = 2.0 * rows * cores * n * k / dt / 1e9
    return {"value": round(gops, 4), "unit": "GOP/s", "cores": cores, "kind": "oracle",
            "single_core_value": round(one, 4),
            "sample": (f"{cores} threads x {rows} of {m} rows of the same product (numpy "
                       f"{'int64 matmul mod p' if w['mode'] == MODP else 'float64 matmul'}), {dt:.1f} s; "
                       f"one core {rows} rows in {dt1:.1f} s")}


def run_reference(args, w, rank, world):
    if rank != 0:
        return
    A, B, C = make_inputs(w)
    m, k, n = w["m"], w["k"], w["n"]
    cores = os.cpu_count() or 1
    rows = 8
    ts = []
    for step in range(args.warmup + args.steps):
        dt = _oracle_parallel(w, A, B, C, rows, cores, 6 + step)
        if step >= args.warmup:
            ts.append(dt)
    t = sum(ts) / len(ts)
    value = 2.0 * rows * cores * n * k / t / 1e9
    line = {
        "impl": "reference", "metric": "effective GOP/s (2mnk/t)", "value": round(value, 4), "unit": "GOP/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int64 mod p" if w["mode"] == MODP else "f64", "data": "synthetic",
        "config": {"workload": w["desc"], "m": m, "k": k, "n": n, "p": w["p"],
                   "schedule": "classical definition (the oracle)", "depth": 0},
        "cpu_baseline": {"value": round(value, 4), "unit": "GOP/s", "cores": cores, "kind": "oracle",
                         "sample": f"{cores} threads x {rows} rows of the {m}x{n} product per step"},
        "e2e": {"value": round(value, 4), "unit": "GOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_sweep(args, w, S, h, torch, dev, rank):
    """FP32 mode per size and depth: effective GOP/s (graph replay, device-
    resident inputs) and max |C - C64| / (|A|max |B|max) on 16 spot rows
    against FP64 on the host, next to the classical split-bf16 product."""
    rows = []
    for n in w["ns"]:
        A, B, C = (synth.normal_matrix(synth.SEED_A, n, n), synth.normal_matrix(synth.SEED_B, n, n),
                   synth.normal_matrix(synth.SEED_C, n, n))
        idx = np.linspace(0, n - 1, 16).astype(np.int64)
        ref = A[idx].astype(np.float64) @ B.astype(np.float64) + C[idx].astype(np.float64)
        scale = float(np.abs(A).max()) * float(np.abs(B).max())
        dA, dB = torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev)
        dC0 = torch.from_numpy(C).to(dev)
        dC = dC0.clone()
        for depth in (0,) + tuple(w["depths"]):
            sched = S.CLASSICAL if depth == 0 else S.T9_ACC
            o = S.Opts(mode=S.FP32, sched=sched, depth=depth, flags=S.FLAG_GRAPH)
            dC.copy_(dC0)
            h.muladd(1.0, dA, dB, 1.0, dC, o)
            h.sync()
            err = float(np.abs(dC[torch.from_numpy(idx).to(dev)].double().cpu().numpy() - ref).max()) / scale
            for _ in range(args.warmup):
                h.muladd(1.0, dA, dB, 1.0, dC, o)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(args.steps):
                h.muladd(1.0, dA, dB, 1.0, dC, o)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.steps
            st = h.stats()
            bound = 1e-5 * n ** 0.6
            rows.append({"n": n, "depth": depth, "schedule": "classical" if depth == 0 else "Acc",
                         "gops": round(2.0 * n ** 3 / (ms * 1e-3) / 1e9, 1), "ms": round(ms, 3),
                         "max_rel_err": float(f"{err:.3e}"), "bound": float(f"{bound:.3e}"),
                         "within_bound": err <= bound, "workspace_bytes": st["workspace_bytes"]})
        del dA, dB, dC, dC0
        torch.cuda.empty_cache()
    for r in rows:
        base = next(x for x in rows if x["n"] == r["n"] and x["depth"] == 0)
        r["vs_classical"] = round(r["gops"] / base["gops"], 4)
    head = next(r for r in rows if r["n"] == max(w["ns"]) and r["depth"] == 2)
    line = {
        "metric": "effective GOP/s (2mnk/t)", "value": head["gops"], "unit": "GOP/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (3 fp16 split products)", "data": "synthetic",
        "config": {"workload": w["desc"], "value_is": f"n={head['n']} depth 2",
                   "l2": "inputs > 129 MB L2, no flush", "parallelism": "replicas x1"},
        "sweep": rows,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_batch(args, w, S, h, torch, dev, dist, world, rank):
    """The batched workload: every rank runs its share of the problems (LPT
    partition on the modelled cost), inputs drawn on the device from a seeded
    generator (tens of GB of operands)."""
    from paper_0707_2347_gb300 import partition
    shapes = synth.batch_shapes(w["count"], w["lo"], w["hi"])
    modes = [S.MODP if i % 2 == 0 else S.FP32 for i in range(len(shapes))]
    parts, cost = partition.assign(shapes, world, modes)
    mine = parts[rank]
    gen = torch.Generator(device=dev)
    gen.manual_seed(1000 + rank)
    probs, ref_probs = [], []
    for i in mine:
        m, k, n = shapes[i]
        if modes[i] == S.MODP:
            mk = lambda r, c: torch.randint(0, 65521, (r, c), generator=gen, device=dev, dtype=torch.int32)
        else:
            mk = lambda r, c: torch.randn((r, c), generator=gen, device=dev, dtype=torch.float32)
        A, B, C = mk(m, k), mk(k, n), mk(m, n)
        q = dict(A=A, B=B, C=C, mode=modes[i], p=65521, alpha=1, beta=1, sched=S.AUTO)
        probs.append(q)
        ref_probs.append(dict(q, sched=S.CLASSICAL, depth=0))
    total = sum(2.0 * shapes[i][0] * shapes[i][1] * shapes[i][2] for i in range(len(shapes)))

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(pl, flags=S.FLAG_GRAPH):
        for _ in range(args.warmup):
            h.muladd_batched(pl, flags)
        h.sync()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            h.muladd_batched(pl, flags)
        e1.record()
        barrier()
        ms = e0.elapsed_time(e1) / args.steps
        if dist is not None:
            t = torch.tensor([ms], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        return ms

    # the large problems' schedules are measured on the GPU (SWMM_FLAG_TUNE)
    # during the first warm-up call; the timed calls replay the captured graph
    tflags = S.FLAG_GRAPH | S.FLAG_TUNE
    with Clocks(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        ms = timed(probs, tflags)
    chosen = h.muladd_batched(probs, tflags)
    h.sync()
    st = h.stats()
    cms = timed(ref_probs) if not args.no_classical else None
    value = total / (ms * 1e-3) / 1e9
    picks = {}
    for s_, d_ in chosen:
        key = f"{S.SCHED_NAMES[s_]}{d_ if s_ else ''}"
        picks[key] = picks.get(key, 0) + 1
    line = {
        "metric": "effective GOP/s (2mnk/t)", "value": round(value, 2), "unit": "GOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "i32 mod p (fp16 limbs) / f32 (3 fp16 split products)",
        "data": "synthetic (device generator)",
        "config": {"workload": w["desc"], "problems": len(shapes), "sum_2mnk": total, "this_rank": len(mine),
                   "autotuner_picks_rank0": picks, "l2": "operands far larger than L2, no flush",
                   "parallelism": f"LPT shards x{world}"},
        "gpu_launches": int((st["leaf_launches"] + st["ew_launches"]) * args.steps),
        "memory": {"workspace_bytes": st["workspace_bytes"], "staging_bytes": st["staging_bytes"]},
        "clocks": clk.summary(),
    }
    if cms:
        line["classical"] = {"value": round(total / (cms * 1e-3) / 1e9, 2), "ms_per_step": round(cms, 3)}
        line["speedup_vs_classical"] = round(cms / ms, 4)
    if rank == 0:
        print(json.dumps(line), flush=True)
    h.close()
    if dist is not None:
        dist.destroy_process_group()


# Large accumulate products (the n >= 16384 range): Table 9 at the depths
# that pay against the classical product of the same library.
LARGE = ((16384, (1, 2)), (32768, (2,)))


def run_large(args, S, h, torch, dev):
    """C <- A B + C over Z/65521 at n = 16384 (Table 9 depth 1 and 2) and
    n = 32768 (depth 2), each against this library's classical tcgen05
    product on the same inputs: ms per step (CUDA events, graph replays,
    inputs resident and far larger than L2), clocks sampled while timing.
    n = 16384 inputs come from the seeded host generator; n = 32768 inputs
    are drawn on the device (a seeded torch generator) to keep the run short."""
    p = 65521
    out = []
    steps = max(3, min(args.steps, 5))
    for n, depths in LARGE:
        if n <= 16384:
            A, B, C = (torch.from_numpy(synth.modp_matrix(sd, n, n, p)).to(dev)
                       for sd in (synth.SEED_A, synth.SEED_B, synth.SEED_C))
        else:
            gen = torch.Generator(device=dev)
            gen.manual_seed(n)
            A, B, C = (torch.randint(0, p, (n, n), generator=gen, device=dev, dtype=torch.int32) for _ in range(3))
        flops = 2.0 * n ** 3

        def timed(o):
            for _ in range(args.warmup):
                h.muladd(1, A, B, 1, C, o)
            h.sync()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with Clocks(torch.cuda.current_device()) as clk:
                e0.record()
                for _ in range(steps):
                    h.muladd(1, A, B, 1, C, o)
                e1.record()
                torch.cuda.synchronize()
            h.sync()
            return e0.elapsed_time(e1) / steps, clk.summary()

        cms, cclk = timed(S.Opts(mode=S.MODP, p=p, sched=S.CLASSICAL, depth=0, flags=S.FLAG_GRAPH))
        for d in depths:
            ms, clk = timed(S.Opts(mode=S.MODP, p=p, sched=S.T9_ACC, depth=d, flags=S.FLAG_GRAPH))
            st = h.stats()
            out.append({"n": n, "schedule": "Acc (Table 9)", "depth": d, "ms_per_step": round(ms, 3),
                        "gops": round(flops / (ms * 1e-3) / 1e9, 1), "classical_ms_per_step": round(cms, 3),
                        "classical_gops": round(flops / (cms * 1e-3) / 1e9, 1),
                        "speedup_vs_classical": round(cms / ms, 4),
                        "extra_elems": st["plan_extra_elems"], "paper_extra_elems": st["paper_extra_elems"],
                        "staging_bytes": st["staging_bytes"], "clocks": clk, "classical_clocks": cclk,
                        "inputs": "seeded host generator" if n <= 16384 else "seeded device generator"})
        del A, B, C
        torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="swmm", choices=["swmm", "reference"])
    ap.add_argument("--workload", default=DEFAULT, choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-classical", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="launch kernels directly instead of a CUDA graph")
    ap.add_argument("--serial", action="store_true",
                    help="capture the graph in row order on one stream (no dataflow overlap)")
    ap.add_argument("--depth", type=int, default=None, help="override the workload's recursion depth")
    ap.add_argument("--cutoff", type=int, default=None, help="override an IPMM workload's cut-off")
    ap.add_argument("--shape", default=None, help="override the workload's m,k,n")
    ap.add_argument("--sched", type=int, default=None, help="override the workload's schedule id")
    ap.add_argument("--fp32", action="store_true", help="run the workload in FP32 mode")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the n = 16384 / 32768 Table 9 vs classical record of the default workload")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    # the recorded DRAM traffic belongs to the named workloads as they are
    args.overridden = args.fp32 or any(x is not None for x in (args.depth, args.cutoff, args.shape, args.sched))
    w = dict(WORKLOADS[args.workload])
    if args.depth is not None:
        w["depth"] = args.depth
        w["desc"] = w["desc"] + f" (depth {args.depth})"
    if args.cutoff is not None:
        w["cutoff"] = args.cutoff
        w["desc"] = w["desc"] + f" (cut-off {args.cutoff})"
    if args.shape is not None:
        w["m"], w["k"], w["n"] = (int(x) for x in args.shape.split(","))
        w["desc"] = w["desc"] + f" (shape {args.shape})"
    if args.sched is not None:
        w["sched"] = args.sched
        w["desc"] = w["desc"] + f" (schedule {args.sched})"
    if args.fp32:
        w["mode"], w["p"] = FP32, 0
        w["desc"] = w["desc"] + " (FP32 mode)"

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, w, rank, world)
        return

    import torch
    import __graft_entry__ as g
    g.build()
    from paper_0707_2347_gb300 import swmm as S

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    h = S.Handle(local)
    if w["entry"] == "batch":
        run_batch(args, w, S, h, torch, dev, dist, world, rank)
        return
    if w["entry"] == "sweep":
        run_sweep(args, w, S, h, torch, dev, rank)
        return
    searched = None
    if w["sched"] == CUSTOM and "table" in w:
        # a paper table as the library runs it, with other kinds for some calls
        from paper_0707_2347_gb300 import search as Q
        rows = Q.table_rows(w["table"])
        for r in rows:
            if r.op == Q.MUL:
                r.kind = w["replace"].get(r.kind, r.kind)
        kinds = sorted({r.kind for r in rows if r.op == Q.MUL})
        Q.set_schedule(h, rows, accumulate=True, preserve=("A11", "A12", "A21", "A22", "B11", "B12", "B21", "B22"),
                       temps=2, kinds=kinds, recompute=True)
        searched = {"table": S.SCHED_NAMES[w["table"]], "kinds": [S.SCHED_NAMES[k] for k in kinds]}
    elif w["sched"] == CUSTOM and "found" in w:
        from paper_0707_2347_gb300 import schedules_found as F
        from paper_0707_2347_gb300 import search as Q
        rows = F.rows(w["found"])
        Q.set_schedule(h, rows, **F.spec(w["found"]))
        searched = {"found": w["found"], "rows": len(rows), "adds": sum(r.op == Q.ADD for r in rows)}
    m, k, n = w["m"], w["k"], w["n"]
    A, B, C = make_inputs(w)
    dA, dB = torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev)
    dC0 = torch.from_numpy(C).to(dev)
    dC = dC0.clone()
    mode, p = w["mode"], w["p"]

    def call(opts, Cdev, Adev=dA, Bdev=dB):
        if w["entry"] == "muladd":
            h.muladd(1, Adev, Bdev, 1, Cdev, opts)
        elif w["entry"] == "mul" or opts.sched == CLASSICAL:
            h.mul(Adev, Bdev, Cdev, opts)
        else:
            h.mul_inplace(Adev, Bdev, Cdev, opts)

    # the in-place schedules overwrite A and B: give them scratch copies
    inplace = w["entry"] == "inplace"
    sA = dA.clone() if inplace else dA
    sB = dB.clone() if inplace else dB

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(opts, steps, warmup, a=sA, b=sB):
        for _ in range(warmup):
            call(opts, dC, a, b)
        h.sync()
        h.leaf_timing(reset=True)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            call(opts, dC, a, b)
        e1.record()
        barrier()
        ms = e0.elapsed_time(e1) / steps
        h.sync()
        if dist is not None:
            t = torch.tensor([ms], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        return ms

    gflag = 0 if args.no_graph else (S.FLAG_GRAPH | (S.FLAG_SERIAL if args.serial else 0))
    extra = dict(ipmm_cutoff=w.get("cutoff", 0), tblock=w.get("tblock", 0), ipmm_acc=w.get("acc", 0))
    opts = S.Opts(mode=mode, p=p or 65521, sched=w["sched"], depth=w["depth"], flags=gflag, **extra)
    with Clocks(local) as clk:
        ms = timed(opts, args.steps, args.warmup)
    # device memory one call holds, measured on an eager call (graph memory
    # is shared between the graphs a handle keeps, so its marks do not
    # separate one call's use)
    eager = S.Opts(mode=mode, p=p or 65521, sched=w["sched"], depth=w["depth"], flags=0, **extra)
    with h.measure_peak() as mpk:
        call(eager, dC, sA, sB)
        h.sync()
    # Per-launch GEMM durations: the same K steps again with an event pair
    # around every leaf GEMM launch (recorded on the launching stream, inside
    # the graph).  The event nodes cost ~5 us each, so the value above is
    # timed without them; and this pass captures in row order, so a GEMM's
    # duration is its own, not shared with additions that overlap it in the
    # dataflow capture of the value pass.
    tflag = S.FLAG_TIMING | (gflag | S.FLAG_SERIAL if gflag else 0)
    topts = S.Opts(mode=mode, p=p or 65521, sched=w["sched"], depth=w["depth"], flags=tflag, **extra)
    tms = timed(topts, args.steps, args.warmup)
    gemm_ms, gemm_launches, tensor_flops = h.leaf_timing(reset=True)
    st = h.stats()
    flops = 2.0 * m * n * k
    value = world * flops / (ms * 1e-3) / 1e9
    burst, sustained, hbm, peak_kind = peaks()
    achieved = (tensor_flops / gemm_launches) / (gemm_ms / gemm_launches * 1e-3) / 1e12 if gemm_launches else 0.0

    line = {
        "metric": "effective GOP/s (2mnk/t)", "value": round(value, 2), "unit": "GOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "i32 mod p (fp16 limbs, fp32 accum)" if mode == MODP else "f32 (3 fp16 split products)",
        "data": "synthetic",
        "config": {"workload": w["desc"], "m": m, "k": k, "n": n, "p": p, "schedule": S.SCHED_NAMES[w["sched"]],
                   "depth": w["depth"], "l2": (f"inputs {(m * k + k * n + m * n) * 4 / 1e6:.0f} MB "
                          + ("> 129 MB L2, no flush" if (m * k + k * n + m * n) * 4 > 129e6 else "fit in L2")),
                   "parallelism": f"replicas x{world}"},
        "gpu_launches": int((st["leaf_launches"] + st["ew_launches"]) * args.steps),
        "cuda_graph": not args.no_graph,
        "memory": {"workspace_bytes": st["workspace_bytes"], "plan_extra_elems": st["plan_extra_elems"],
                   "paper_extra_elems_same_levels": st["paper_extra_elems"], "staging_bytes": st["staging_bytes"],
                   "measured_peak_bytes": mpk.peak,
                   "measured": "rise of the device's default memory pool during one eager call"},
        # the leaf launches are short (a step lasts milliseconds): the burst
        # figure is the denominator; the sustained one is kept beside it
        "roofline": {"bound": "tensor", "achieved": round(achieved, 1), "peak": burst, "unit": "TFLOP/s",
                     "frac": round(achieved / burst, 4),
                     "traffic": (round(TRAFFIC_PER_LEVEL * FUSED_LEVELS[args.workload] / st["leaf_launches"])
                                 if args.workload in FUSED_LEVELS and st["leaf_launches"] and not args.overridden
                                 else None),
                     "kernel": "gemm_kernel (leaf products, fp16 limb MMAs counted)",
                     "peak_kind": f"{peak_kind} bf16 burst", "peak_sustained": sustained,
                     "frac_of_sustained": round(achieved / sustained, 4), "launches_per_step": st["leaf_launches"],
                     "gemm_ms_per_step": round(gemm_ms / max(gemm_launches, 1) * st["leaf_launches"], 4),
                     "timing_pass_ms_per_step": round(tms, 4),
                     "timing_pass": "event pair per GEMM launch, graph captured in row order"},
    }
    line["clocks"] = clk.summary()
    if searched:
        line["config"]["custom_schedule"] = searched

    if not args.no_classical and w["sched"] != CLASSICAL:
        dC.copy_(dC0)
        cms = timed(S.Opts(mode=mode, p=p or 65521, sched=CLASSICAL, depth=0, flags=gflag), args.steps, args.warmup)
        dC.copy_(dC0)
        copts = S.Opts(mode=mode, p=p or 65521, sched=CLASSICAL, depth=0, flags=S.FLAG_TIMING | gflag)
        timed(copts, args.steps, args.warmup)
        cg_ms, cg_n, cg_fl = h.leaf_timing(reset=True)
        cval = world * flops / (cms * 1e-3) / 1e9
        line["classical"] = {"value": round(cval, 2), "ms_per_step": round(cms, 4),
                             "gemm_tflops": round(cg_fl / (cg_ms * 1e-3) / 1e12, 1) if cg_ms else None}
        line["speedup_vs_classical"] = round(value / cval, 4)

    if not args.no_e2e and w["entry"] == "muladd":
        # through the library's host-operand entry point: A, B, C in page-
        # locked host memory, copied in block by block as the schedule needs
        # them and C copied back, all inside the timed region
        pin = [torch.from_numpy(x).pin_memory() for x in (A, B, C)]
        opts_e = S.Opts(mode=mode, p=p or 65521, sched=w["sched"], depth=w["depth"], flags=gflag, **extra)

        def e2e_step():
            h.muladd_host(1, pin[0], pin[1], 1, pin[2], opts_e)

        for _ in range(args.warmup):
            e2e_step()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            e2e_step()
        e1.record()
        barrier()
        ems = e0.elapsed_time(e1) / args.steps
        h.sync()
        line["e2e"] = {"value": round(world * flops / (ems * 1e-3) / 1e9, 2), "unit": "GOP/s",
                       "h2d_bytes_per_step": int(A.nbytes + B.nbytes + C.nbytes), "d2h_bytes_per_step": int(C.nbytes),
                       "ms_per_step": round(ems, 4), "entry": "swmm_muladd_host"}
    elif not args.no_e2e:
        # C <- A B entry points: host copies around the device call
        pin = [torch.from_numpy(x).pin_memory() for x in (A, B)]
        out = torch.empty(C.shape, dtype=torch.from_numpy(C[:0]).dtype).pin_memory()
        opts_e = S.Opts(mode=mode, p=p or 65521, sched=w["sched"], depth=w["depth"], flags=gflag, **extra)

        def e2e_step():
            dA.copy_(pin[0], non_blocking=True)
            dB.copy_(pin[1], non_blocking=True)
            call(opts_e, dC, dA, dB)
            out.copy_(dC, non_blocking=True)

        for _ in range(args.warmup):
            e2e_step()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            e2e_step()
        e1.record()
        barrier()
        ems = e0.elapsed_time(e1) / args.steps
        h.sync()
        line["e2e"] = {"value": round(world * flops / (ems * 1e-3) / 1e9, 2), "unit": "GOP/s",
                       "h2d_bytes_per_step": int(A.nbytes + B.nbytes), "d2h_bytes_per_step": int(C.nbytes),
                       "ms_per_step": round(ems, 4), "entry": "device call, torch copies"}
    if args.workload == DEFAULT and not args.no_large:
        # the same step with operand staging bounded (SWMM_FLAG_LOWMEM)
        dC.copy_(dC0)
        lo = S.Opts(mode=mode, p=p or 65521, sched=w["sched"], depth=w["depth"], flags=gflag | S.FLAG_LOWMEM)
        with Clocks(local) as lclk:
            lms = timed(lo, args.steps, args.warmup)
        lst = h.stats()
        with h.measure_peak() as lpk:
            call(S.Opts(mode=mode, p=p or 65521, sched=w["sched"], depth=w["depth"], flags=S.FLAG_LOWMEM), dC)
            h.sync()
        line["bounded_staging"] = {
            "flag": "SWMM_FLAG_LOWMEM", "ms_per_step": round(lms, 4), "value": round(world * flops / (lms * 1e-3) / 1e9, 2),
            "slowdown": round(lms / ms, 4), "staging_bytes": lst["staging_bytes"],
            "workspace_bytes": lst["workspace_bytes"], "measured_peak_bytes": lpk.peak,
            "paper_extra_bytes": 4 * lst["paper_extra_elems"], "clocks": lclk.summary()}
        line["large"] = run_large(args, S, h, torch, dev)
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(w, A, B, C)
    if rank == 0:
        print(json.dumps(line), flush=True)
    h.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
