#!/usr/bin/env python3
"""BSW seed-extension benchmark: GCUPS on one GB300 (batched vs plain kernel).

A step is one pass of the whole extension path over one batch: length
bucketing, the per-class extension kernels and the exact 32-bit re-run, for
every pair of the 250 bp read workload (4,000,000 pairs, inputs resident in
HBM), the largest configuration that fits one GPU.  GCUPS counts the DP cells
the scalar algorithm computes (the oracle's count, which the library
reproduces exactly).  The default run also measures the 151 bp and long-query
workloads the same way, a bounded serving sweep (p50/p99 latency at three
offered loads), N bases, the seed-extension driver, suffix array lookup and
SMEM search, each checked against the oracle or the definition.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                  [--config read250] [--pairs N] [--only] [--serve]

--impl reference times the CPU oracle on the host cores, on a bounded sample of
the same workload.  --serve runs the full serving sweep (ten offered loads)
instead of the batch benchmark.  Under torchrun each rank runs its own batch
(weak scaling, no collective on the data path); rank 0 prints the JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

# 32-bit integer lane-operations one SM issues per clock (4 schedulers x 32 lanes).
LANE_OPS_PER_CLK_PER_SM = 128
METRIC = "BSW GCUPS on 1 GB300 (batched vs plain kernel, bit-exact); p50/p99 serve latency"
# DRAM bytes read + written per launch of a workload's dominant kernel, from
# one ncu capture of the current kernel (bytes, source); other kernels and
# workloads report null.
MEASURED_TRAFFIC = {
    ("read250", "k_inter<128,u8>"): (49_626_624, "ncu dram__bytes_read.sum + dram__bytes_write.sum of the dominant "
                                                 "launch, profiles/k_inter128_u8_read250.md"),
}

SECONDARY = ("read151", "long10k")

U8_NMAX = (256, 224, 192, 160, 128, 96, 64, 32)
I16_NMAX = (256, 128, 64, 32)

WORKLOAD_TEXT = {
    "read151": "151 bp short-read seed extensions: 2,000,000 left/right pairs from 1,000,000 reads of a 100 Mbp "
               "random reference (0.1% SNPs, 1% sequencing substitutions), seeds 19-151 bp, query 0-132 bp, "
               "target = query + 100; match 1, mismatch 4, gap 6+1k, w 100, zdrop 100, end bonus 5",
    "read250": "250 bp read seed extensions: 4,000,000 left/right pairs from 2,000,000 reads of the 100 Mbp "
               "reference with 2% divergence (10% of it 1-10 bp indels), seeds 19-250 bp, query 0-231 bp, "
               "target = query + 100; match 1, mismatch 4, gap 6+1k, w 100, zdrop 100, end bonus 5",
    "plain10k": "10,000 pairs, queries 1-130 bp with 1% substitutions and 0.1% 1-3 bp indels, w 100, zdrop 100",
    "long10k": "20,000 long-query pairs, query log-uniform 1-10 kbp, 12% error, w 500, zdrop 400",
}


def parse():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--config", default="read250")
    ap.add_argument("--pairs", type=int, default=None)
    ap.add_argument("--serve", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline leg")
    ap.add_argument("--no-tune", action="store_true", help="keep the default plan (no autotune)")
    ap.add_argument("--no-driver", action="store_true", help="skip the seed-extension driver leg")
    ap.add_argument("--no-sal", action="store_true", help="skip the suffix-array lookup leg")
    ap.add_argument("--no-smem", action="store_true", help="skip the SMEM search leg")
    ap.add_argument("--no-nbases", action="store_true", help="skip the N-bases leg")
    ap.add_argument("--plan", default=None,
                    help="fixed plan short_max,u8_bounds,i16_bounds,packed,warp_cols,inter_warps[,cta_min[,warp_x2]] "
                         "(no autotune)")
    ap.add_argument("--serve-requests", type=int, default=1000, help="requests per offered-load point (--serve)")
    ap.add_argument("--serve-quick", type=int, default=200,
                    help="requests per point of the bounded serving leg of the default run (0: skip it)")
    ap.add_argument("--only", action="store_true",
                    help="measure the --config workload alone (no other workloads or legs)")
    return ap.parse_args()


# ------------------------------------------------------------------ helpers

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class Dist:
    """Barrier and max-over-ranks for torchrun launches (no data-path collective)."""

    def __init__(self, backend="nccl"):
        import torch
        import torch.distributed as td
        self.world, self.rank, self.local = dist_env()
        self.td = td
        self.on = self.world > 1
        if self.on and not td.is_initialized():
            td.init_process_group(backend=backend)
        self.torch = torch
        self.device = "cuda" if backend == "nccl" else "cpu"

    def barrier(self):
        if self.on:
            self.td.barrier()

    def max(self, x: float) -> float:
        if not self.on:
            return x
        t = self.torch.tensor([float(x)], dtype=self.torch.float64, device=self.device)
        self.td.all_reduce(t, op=self.td.ReduceOp.MAX)
        return float(t.item())

    def sum(self, x: float) -> float:
        if not self.on:
            return x
        t = self.torch.tensor([float(x)], dtype=self.torch.float64, device=self.device)
        self.td.all_reduce(t, op=self.td.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.on and self.td.is_initialized():
            self.td.destroy_process_group()


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _smallest_class(n, nmax, mask, first):
    """Index (first + k) of the smallest enabled bound nmax[k] >= n (bit 0 always on)."""
    c = np.full(n.shape, first, np.int64)
    for k in range(1, len(nmax)):
        if (mask >> k) & 1:
            c = np.where(n <= nmax[k], first + k, c)
    return c


def class_of(q_len, t_len, h0, match, plan):
    """Kernel class of each pair under a plan, as the library buckets it: 0-7
    8-bit lanes (class bounds 256..16), 8-11 16-bit lanes (256..32), 12 block
    per pair (16-bit range, at least cta_min bases), 13 warp per pair with
    16-bit-range scores, 14 with 32-bit scores, -1 empty."""
    n = np.asarray(q_len, np.int64)
    m = np.asarray(t_len, np.int64)
    bound = np.asarray(h0, np.int64) + match * np.minimum(n, m)
    u8 = _smallest_class(n, U8_NMAX, plan.u8_bounds | 1, 0)
    i16 = _smallest_class(n, I16_NMAX, plan.i16_bounds | 1, 8)
    cta_min = getattr(plan, "cta_min", 0)
    w16 = np.where((cta_min > 0) & (n >= max(cta_min, 1)), 12, 13)
    if getattr(plan, "warp_x2", 0) and match <= 3:
        # the two-columns kernel re-runs pairs of bound 2^(15 - z) and above with 32-bit lanes
        z = int(np.ceil(np.log2(match + 1)))
        w16 = np.where((w16 == 13) & (bound >= (1 << (15 - z))), 14, w16)
    c = np.where(n > plan.short_max, np.where(bound <= 32767, w16, 14),
                 np.where(bound <= 255, u8, np.where(bound <= 32767, i16, 14)))
    return np.where((n <= 0) | (m <= 0), -1, c)


def class_kernel(c, plan, scoring):
    """Name of the kernel that runs class c under the plan."""
    packable = (scoring.match + min(scoring.mismatch, 255 - scoring.match)
                + max(min(scoring.o_del + scoring.e_del, 255), min(scoring.o_ins + scoring.e_ins, 255)) <= 256)
    if c < 8:
        nm = U8_NMAX[c]
        if plan.packed and nm <= 128 and packable:
            return "k_inter2<%d>" % (128 if nm > 64 else 64 if nm > 32 else 32)
        return "k_inter<%d,u8>" % nm
    if c < 12:
        return "k_inter<%d,i16>" % I16_NMAX[c - 8]
    if c == 12:
        return "k_cta<8,s16>"
    if c == 13 and getattr(plan, "warp_x2", 0) and scoring.match <= 3:
        return "k_warp_x2"
    return "k_warp<%d,s16>" % plan.warp_cols if c == 13 else "k_warp<8,s32>"


# ------------------------------------------------------------------ arms

def cpu_baseline(wl, min_s: float = 10.0, single_s: float = 4.0):
    """The oracle on the host cores: whole-workload passes on every core until
    min_s seconds have passed, then single-thread passes over the first pairs
    until single_s seconds have passed.  Returns the first pass's results too."""
    import oracle
    cores = os.cpu_count() or 1
    res = None
    passes, cells_all, t_all = 0, 0, 0.0
    while t_all < min_s and passes < 50:
        t0 = time.perf_counter()
        r, cells, _ = oracle.extend_batch(wl, nthreads=cores)
        t_all += time.perf_counter() - t0
        cells_all += int(cells.sum())
        passes += 1
        if res is None:
            res = r
    n1 = min(wl.n_pairs, 50_000)
    one = wl.subset(np.arange(n1))
    p1, cells_1, t_1 = 0, 0, 0.0
    while t_1 < single_s and p1 < 50:
        t0 = time.perf_counter()
        _, cells, _ = oracle.extend_batch(one, nthreads=1)
        t_1 += time.perf_counter() - t0
        cells_1 += int(cells.sum())
        p1 += 1
    return {"value": round(cells_all / t_all / 1e9, 4), "unit": "GCUPS", "cores": cores, "kind": "oracle",
            "sample": "%d pass(es) over all %d pairs on %d threads, %.1f s" % (passes, wl.n_pairs, cores, t_all),
            "single_thread": {"value": round(cells_1 / t_1 / 1e9, 4), "unit": "GCUPS", "cores": 1,
                              "sample": "%d pass(es) over the first %d pairs, %.1f s" % (p1, n1, t_1)}}, res


def run_reference(args):
    """The CPU oracle, timed on the host cores on a bounded sample per step."""
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    from paper_1907_12931_gb300 import workload as W
    import oracle
    wl = W.make(args.config, n_pairs=args.pairs)
    per_step = min(wl.n_pairs, 100_000 if args.config in ("read151", "read250") else 2000)
    cores = os.cpu_count() or 1
    steps = max(1, min(args.steps, 20))
    times, cells_tot = [], 0
    for s in range(args.warmup + steps):
        lo = (s * per_step) % max(1, wl.n_pairs - per_step + 1)
        sub = wl.subset(np.arange(lo, lo + per_step))
        t0 = time.perf_counter()
        _, cells, _ = oracle.extend_batch(sub, nthreads=cores)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
            cells_tot += int(cells.sum())
    total = sum(times)
    value = cells_tot / total / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "GCUPS", "n_gpus": args.gpus,
        "steps": steps, "warmup": args.warmup, "ms_per_step": round(1e3 * total / steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": args.config, "description": WORKLOAD_TEXT.get(args.config, args.config),
                   "pairs": wl.n_pairs, "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": round(value, 4), "unit": "GCUPS", "cores": cores, "kind": "oracle",
                         "sample": "%d consecutive pairs per step of the %d-pair workload" % (per_step, wl.n_pairs)},
        "e2e": {"value": round(value, 4), "unit": "GCUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def driver_leg(bsw, args):
    """The seed-extension driver (bsw_extend_seeds) on 500 000 151 bp reads
    with 2 seeds each, end to end through the C ABI (host inputs, the copies
    and both extension sides inside the timed call), its parity with the
    driver oracle on the first 5 000 reads, and the oracle's rate there."""
    from paper_1907_12931_gb300 import workload as W
    from oracle import driver
    sw = W.make_seeds("seeds151")
    ctx = bsw.Context(sw.params, mem_budget_bytes=40 << 30)
    ctx.set_reference(sw.ref)
    prep = ctx.prepare_seeds(sw)
    out = np.zeros(sw.n_seeds, bsw.ALN_DTYPE)
    ctx.extend_prepared(prep, out=out)
    times = []
    for _ in range(5):
        t0 = time.perf_counter()
        _, cells = ctx.extend_prepared(prep, out=out)
        times.append(time.perf_counter() - t0)
    t = statistics.median(times)
    nsub = 50_000
    sub = W.make_seeds("seeds151", n_reads=nsub)
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    ref = driver.extend_seeds(sub, nthreads=cores)
    tcpu = time.perf_counter() - t0
    k = sub.n_seeds
    fields = ("qb", "qe", "rb", "re", "score", "w_left", "w_right", "kept")
    mism = int(sum((out[f][:k] != ref[f]).sum() for f in fields))
    # the same seeds with N in 0.2% of the read bases outside the seeds and reference N runs
    nw = W.inject_n_seeds(sw, 0.002, 0.0005, seed=4)
    ctx.set_reference(nw.ref)
    nprep = ctx.prepare_seeds(nw)
    nout = np.zeros(nw.n_seeds, bsw.ALN_DTYPE)
    ctx.extend_prepared(nprep, out=nout)
    ntimes = []
    for _ in range(5):
        t0 = time.perf_counter()
        _, ncells = ctx.extend_prepared(nprep, out=nout)
        ntimes.append(time.perf_counter() - t0)
    tn = statistics.median(ntimes)
    n_first = W.SeedWorkload(nw.name, nw.params, nw.reads, nw.read_off, nw.read_len, nw.ref, sub.seed_read, sub.qbeg,
                             sub.slen, sub.rbeg)
    nref = driver.extend_seeds(n_first, nthreads=cores)
    nmism = int(sum((nout[f][:k] != nref[f]).sum() for f in fields))
    ctx.close()
    return {"workload": "seeds151: 500,000 151 bp reads (read151 recipe) x 2 seeds of 19-50 bp, w 100, "
                        "2 band tries", "seeds": sw.n_seeds, "ms": round(t * 1e3, 3),
            "seeds_per_s": round(sw.n_seeds / t, 1), "gcups": round(cells / t / 1e9, 3), "cells": cells,
            "kept_fraction": round(float(out["kept"].mean()), 4),
            "retried_fraction": round(float(((out["w_left"] > 100) | (out["w_right"] > 100)).mean()), 5),
            "timing": "median of 5 calls, wall clock around the synchronous C-ABI call",
            "parity_sample": {"seeds_checked": k, "fields": 8, "mismatches": mism},
            "cpu_oracle": {"seeds_per_s": round(k / tcpu, 1), "cores": cores,
                           "sample": "the first %d reads (%d seeds), %.2f s" % (nsub, k, tcpu)},
            "with_n": {"reads_n_fraction": round(float((nw.reads == 4).sum() / nw.read_len.sum()), 5),
                       "ref_n_fraction": round(float((nw.ref == 4).mean()), 5), "ms": round(tn * 1e3, 3),
                       "seeds_per_s": round(nw.n_seeds / tn, 1), "gcups": round(ncells / tn / 1e9, 3),
                       "parity_sample": {"seeds_checked": k, "fields": 8, "mismatches": nmism}}}


def n_bases_leg(bsw, wl, plan, gcups_no_n, stream):
    """The headline workload with N bases: each query base an N with
    probability 0.1 % (sequencer no-calls), each target base the start of a
    run of 1-40 N's with probability 0.02 % (reference gaps).  Device inputs,
    the same plan, timed with CUDA events on the stream; every pair checked
    against the oracle, whose run on the host cores is also timed."""
    import torch
    from paper_1907_12931_gb300 import workload as W
    import oracle
    nw = W.inject_n(wl, 0.001, 0.0002, seed=77)
    qn = np.concatenate([[0], np.cumsum(nw.q == 4)])
    tn = np.concatenate([[0], np.cumsum(nw.t == 4)])
    has_n = ((qn[nw.q_off + nw.q_len] - qn[nw.q_off]) > 0) | ((tn[nw.t_off + nw.t_len] - tn[nw.t_off]) > 0)
    ctx = bsw.Context(nw.params, mem_budget_bytes=40 << 30)
    ctx.set_plan(plan)
    db = bsw.DeviceBatch(bsw.HostBatch(nw))
    for _ in range(3):
        ctx.extend_device(db, 0, stream.cuda_stream)
    stream.synchronize()
    reps = 50
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        ctx.extend_device(db, 0, stream.cuda_stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    ctx.sync(stream.cuda_stream)
    cells = int(db.cells.item())
    got = db.out.cpu().numpy()
    ctx.extend_device(db, bsw.BSW_TIME_KERNELS | bsw.BSW_NO_GRAPH, stream.cuda_stream)
    _, class_ms = ctx.kernel_times()
    ctx.sync(stream.cuda_stream)
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    res, ocells, _ = oracle.extend_batch(nw, nthreads=cores)
    tcpu = time.perf_counter() - t0
    mism = int((res != got).any(axis=1).sum())
    ctx.close()
    gcups = cells / (ms * 1e-3) / 1e9
    return {"workload": "%s with N: query bases N with p 0.001, target N runs of 1-40 starting with p 0.0002"
                        % wl.name,
            "pairs": nw.n_pairs, "pairs_with_n": int(has_n.sum()), "ms": round(ms, 4), "gcups": round(gcups, 3),
            "vs_without_n": round(gcups / gcups_no_n, 4) if gcups_no_n else None,
            "timing": "CUDA events on the stream, mean of %d calls, device inputs" % reps,
            "class_ms_in_step": {bsw.CLASS_NAMES[c]: round(t, 4) for c, t in enumerate(class_ms) if t > 0},
            "parity": {"pairs_checked": nw.n_pairs, "fields": 6, "mismatches": mism,
                       "cells_equal": cells == int(ocells.sum())},
            "cpu_oracle": {"gcups": round(int(ocells.sum()) / tcpu / 1e9, 4), "cores": cores,
                           "sample": "all pairs once, %.2f s" % tcpu}}


def sal_leg(bsw, args, stream, hbm_peak):
    """Suffix array lookup (Eq. 1) over 8,000,000 SA intervals of a 64 Mbp
    reference prefix: the uncompressed suffix array (256 MB, larger than L2)
    in HBM, intervals and output on the device, timed with CUDA events on the
    stream; bandwidth against the measured copy peak."""
    import torch
    from paper_1907_12931_gb300 import workload as W
    from oracle import sal as sal_oracle
    ref = W.reference()[:64_000_000]
    t0 = time.perf_counter()
    sa = bsw.bsw_sa_build(ref)
    t_build = time.perf_counter() - t0
    n_sa = sa.shape[0]
    rng = np.random.default_rng(77)
    n_int = 8_000_000
    cnt = np.minimum(rng.geometric(0.25, n_int), 500).astype(np.int32)
    k = rng.integers(0, n_sa - cnt, dtype=np.int64)
    off = np.zeros(n_int, np.int64)
    np.cumsum(cnt[:-1], out=off[1:])
    total = int(cnt.sum())
    ctx = bsw.Context(W.Params(), mem_budget_bytes=8 << 30)
    ctx.sal_set_index(sa)
    dk, dc, do = (torch.from_numpy(x).cuda() for x in (k, cnt, off))
    out = torch.empty(total, dtype=torch.int32, device="cuda")
    for _ in range(3):
        ctx.sal_lookup_device(dk, dc, do, out, stream.cuda_stream)
    stream.synchronize()
    reps = 20
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        ctx.sal_lookup_device(dk, dc, do, out, stream.cuda_stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    ctx.sync(stream.cuda_stream)
    got = out.cpu().numpy()
    ns = 200_000
    want = sal_oracle.lookup(sa, k[:ns], cnt[:ns])
    mism = int((got[:want.shape[0]] != want).sum())
    t0 = time.perf_counter()
    sal_oracle.lookup(sa, k[:ns], cnt[:ns])
    tcpu = time.perf_counter() - t0
    nbytes = n_int * (8 + 4 + 8) + total * (4 + 4)
    gbs = nbytes / (ms * 1e-3) / 1e9
    ctx.close()
    return {"workload": "64 Mbp reference prefix, suffix array of 64,000,001 int32 (256 MB); 8,000,000 intervals, "
                        "counts geometric(0.25) capped at 500 (%d positions)" % total,
            "ms": round(ms, 4), "positions_per_s": round(total / (ms * 1e-3), 1),
            "roofline": {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm_peak, "unit": "GB/s",
                         "frac": round(gbs / hbm_peak, 4) if hbm_peak else None,
                         "bytes": "per interval k, count, offset (20 B) + per position S read and output write (8 B)"},
            "index_build_s": round(t_build, 2),
            "parity_sample": {"intervals_checked": ns, "mismatches": mism},
            "cpu_oracle": {"positions_per_s": round(want.shape[0] / tcpu, 1), "cores": 1,
                           "sample": "the first %d intervals, %.3f s" % (ns, tcpu)}}


class _KmerIndex:
    """Occurrence counts of patterns of 16 bases or more in a text: the text's
    positions sorted by their 16-mer, a pattern's candidates found by binary
    search on its first 16 bases and kept where the rest matches (numpy)."""

    K = 16

    def __init__(self, T):
        T = np.asarray(T, np.uint8)
        n = T.shape[0] - self.K + 1
        key = np.zeros(n, np.uint32)
        for d in range(self.K):
            key = (key << np.uint32(2)) | T[d:d + n].astype(np.uint32)
        order = np.argsort(key)
        self.T, self.key, self.pos = T, key[order], order

    def count(self, p):
        p = np.asarray(p, np.uint8)
        k = 0
        for d in range(self.K):
            k = (k << 2) | int(p[d])
        kk = np.uint32(k)                       # a key of the array's own type (no cast of the array)
        lo, hi = np.searchsorted(self.key, kk, "left"), np.searchsorted(self.key, kk, "right")
        cand = self.pos[lo:hi]
        cand = cand[cand + p.shape[0] <= self.T.shape[0]]
        for d in range(self.K, p.shape[0]):
            cand = cand[self.T[cand + d] == p[d]]
        return int(cand.shape[0])


def smem_leg(bsw, args):
    """SMEM search over 200,000 151 bp reads (both strands) of a 48 Mbp
    reference prefix: the FM-index of ref + revcomp(ref) (a 96 MB occurrence
    table), the search end to end through the C ABI; 2,000 sampled records
    checked against the definition.  The CPU oracle's rate and its exact
    parity come from a bounded sample where the oracle fits a bench run: 60
    reads of a 20 kbp prefix."""
    from paper_1907_12931_gb300 import workload as W
    from oracle import smem as smem_oracle
    n_ref = 48_000_000
    ref = W.reference()[:n_ref]
    ctx = bsw.Context(W.Params(), mem_budget_bytes=16 << 30)
    t0 = time.perf_counter()
    ctx.fm_build(ref)
    t_build = time.perf_counter() - t0
    codes, off, rl, _ = W.make_reads(200_000, 151, ref_limit=n_ref)
    packed = bsw.bsw_pack_2bit(codes)
    recs, first = ctx.smem(packed, off, rl, min_len=19)
    cap = recs.shape[0] + 16
    times = []
    for _ in range(3):
        t0 = time.perf_counter()
        recs, first = ctx.smem(packed, off, rl, min_len=19, cap=cap)
        times.append(time.perf_counter() - t0)
    t = statistics.median(times)

    # property check: occurrence counts in ref + revcomp(ref), maximality
    t0 = time.perf_counter()
    kx = _KmerIndex(np.concatenate([ref, (3 - ref[::-1]).astype(np.uint8)]))
    rng = np.random.default_rng(5)
    bad = 0
    pick = rng.choice(recs.shape[0], size=min(2000, recs.shape[0]), replace=False)
    for j in pick:
        r, q, ln, cnt = int(recs["read_id"][j]), int(recs["qbeg"][j]), int(recs["len"][j]), int(recs["s"][j])
        x = codes[off[r]:off[r] + rl[r]]
        ok = kx.count(x[q:q + ln]) == cnt
        if q + ln < rl[r]:
            ok &= kx.count(x[q:q + ln + 1]) == 0     # not extendable to the right
        if q > 0:
            ok &= kx.count(x[q - 1:q + ln]) == 0     # not extendable to the left
        bad += 0 if ok else 1
    t_check = time.perf_counter() - t0
    del kx

    # the oracle on a bounded sample, and the GPU's records there compared with it
    n_small = 20_000
    sref = ref[:n_small]
    scodes, soff, srl, _ = W.make_reads(60, 151, ref_limit=n_small, seed=11)
    sreads = [scodes[soff[r]:soff[r] + srl[r]] for r in range(srl.shape[0])]
    t0 = time.perf_counter()
    want = smem_oracle.smems(sref, sreads, 19)
    t_oracle = time.perf_counter() - t0
    ctx.fm_build(sref)
    srecs, sfirst = ctx.smem(bsw.bsw_pack_2bit(scodes), soff, srl, min_len=19)
    ctx.close()
    got = [[(int(srecs["qbeg"][k]), int(srecs["len"][k]), int(srecs["k"][k]), int(srecs["s"][k]))
            for k in range(int(sfirst[r]), int(sfirst[r + 1]))] for r in range(srl.shape[0])]
    sample_mismatch = sum(1 for a, b in zip(got, want) if a != [tuple(map(int, w)) for w in b])
    return {"workload": "200,000 151 bp reads (read151 recipe, every other read from the reverse strand) of a "
                        "48 Mbp reference prefix; min_len 19",
            "ms": round(t * 1e3, 3), "reads_per_s": round(rl.shape[0] / t, 1),
            "smems": int(recs.shape[0]), "smems_per_s": round(recs.shape[0] / t, 1),
            "timing": "median of 3 calls, wall clock around the synchronous C-ABI call (reads copied in, "
                      "records copied out)",
            "index_build_s": round(t_build, 2), "index_bytes": int(2 * n_ref),
            "property_check": {"records_checked": int(pick.shape[0]), "failures": bad, "check_s": round(t_check, 1),
                               "checks": "occurrence count in ref + revcomp(ref) (16-mer index, numpy), no "
                                         "extension by one base to the right or to the left"},
            "cpu_oracle": {"value": round(srl.shape[0] / t_oracle, 2), "unit": "reads/s", "cores": 1,
                           "kind": "oracle",
                           "sample": "60 151 bp reads of a 20 kbp reference prefix (a 40 kbp text; the "
                                     "oracle's interval narrowing over the 96 Mbp text does not fit a bench run), "
                                     "%.1f s" % t_oracle},
            "parity_sample": {"reads": int(srl.shape[0]), "reads_with_differences": sample_mismatch,
                              "smems": int(srecs.shape[0]),
                              "what": "every record (qbeg, len, k, s) of the GPU on the 20 kbp index equal to "
                                      "the oracle's"}}


def pinned_host_batch(bsw, hb):
    """Copy a HostBatch's arrays into pinned host memory (for the end-to-end leg)."""
    import torch
    for name in ("q", "t", "q_off", "q_len", "t_off", "t_len", "h0"):
        a = getattr(hb, name)
        p = torch.empty(a.shape, dtype={np.uint8: torch.uint8, np.int32: torch.int32,
                                        np.int64: torch.int64}[a.dtype.type], pin_memory=True)
        p.numpy()[...] = a
        setattr(hb, "_pin_" + name, p)
        setattr(hb, name, p.numpy())
    return hb


def time_device(ctx, db, flags, steps, warmup, stream, dist):
    import torch
    for _ in range(warmup):
        ctx.extend_device(db, flags, stream.cuda_stream)
    stream.synchronize()
    ctx.sync(stream.cuda_stream)
    dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        ctx.extend_device(db, flags, stream.cuda_stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    ctx.sync(stream.cuda_stream)
    dist.barrier()
    return dist.max(ms) / steps


def ops_per_cell(scoring) -> int:
    """Algorithmic integer operations per cell: 7 when deletions and insertions
    cost the same (E and F open from one shared M - o - e), else 8."""
    return 7 if (scoring.o_del == scoring.o_ins and scoring.e_del == scoring.e_ins) else 8


def tune(bsw, ctx, name, n_pairs, seed, args):
    """The execution plan: given (--plan), the default (--no-tune), or
    autotuned on a batch of the same recipe drawn from another seed, so the
    plan is not fitted to the timed batch itself.  Returns (plan, seconds)."""
    from paper_1907_12931_gb300 import workload as W
    t0 = time.perf_counter()
    if args.plan:
        ctx.set_plan(bsw.make_plan(*[int(x, 0) for x in args.plan.split(",")]))
        plan = ctx.get_plan()
    elif args.no_tune:
        plan = ctx.get_plan()
    else:
        twl = W.make(name, n_pairs=n_pairs, seed=seed)
        tdb = bsw.DeviceBatch(bsw.HostBatch(twl))
        plan = ctx.autotune(tdb, sample_pairs=twl.n_pairs)
        del tdb, twl
    return plan, time.perf_counter() - t0


def plain_leg(bsw, ctx, db, plan, steps, warmup, stream, dist, out_ref, cells_ref):
    """The plain baselines on the same inputs: the warp-per-pair kernels over
    pairs in input order, the int2 ring kernel with 4, 8 and 16 columns per
    lane and the two-columns kernel ("x2"; the best of the four is the plain
    kernel), and the naive global-memory kernel."""
    per = {}
    for cols in (4, 8, 16, "x2"):
        x2 = cols == "x2"
        ctx.set_plan(bsw.make_plan(plan.short_max, plan.u8_bounds, plan.i16_bounds, plan.packed, 8 if x2 else cols,
                                   plan.inter_warps, plan.cta_min, 1 if x2 else 0))
        ms = time_device(ctx, db, bsw.BSW_PLAIN_KERNEL, steps, warmup, stream, dist)
        equal = bool(np.array_equal(db.out.cpu().numpy(), out_ref)) and int(db.cells.item()) == cells_ref
        per[cols] = (ms, equal)
    ctx.set_plan(plan)
    best = min(per, key=lambda c: per[c][0])
    g_steps = max(2, steps // 3)
    ms_g = time_device(ctx, db, bsw.BSW_PLAIN_GLOBAL, g_steps, 1, stream, dist)
    g_equal = bool(np.array_equal(db.out.cpu().numpy(), out_ref)) and int(db.cells.item()) == cells_ref
    return best, per, ms_g, g_equal


def dominant_leg(bsw, ctx, wl, plan, stream, dist, steps, clk_mhz, sms):
    """The dominant kernel: the class with the most cells under the plan, run
    as a batch of its own; its duration from CUDA events recorded on its own
    stream just before and after its launch, averaged over launches."""
    all_cls = class_of(wl.q_len, wl.t_len, wl.h0, wl.params.scoring.match, plan)
    est = wl.q_len.astype(np.float64) * np.minimum(wl.t_len, 2 * wl.params.w + 1)
    dom = int(np.argmax([float(est[all_cls == c].sum()) for c in range(15)]))
    sub = wl.subset(np.nonzero(all_cls == dom)[0])
    sdb = bsw.DeviceBatch(bsw.HostBatch(sub))
    for _ in range(2):
        ctx.extend_device(sdb, bsw.BSW_NO_GRAPH, stream.cuda_stream)
    dom_ms = []
    for _ in range(max(3, steps // 4)):
        ctx.extend_device(sdb, bsw.BSW_TIME_KERNELS | bsw.BSW_NO_GRAPH, stream.cuda_stream)
        dom_ms.append(ctx.kernel_times()[1][dom])
    ctx.sync(stream.cuda_stream)
    ms_dom = dist.max(statistics.mean(dom_ms))
    dom_cells = int(sdb.cells.item())
    del sdb
    k = ops_per_cell(wl.params.scoring)
    f_mhz = clk_mhz or 1470.0
    achieved = dom_cells * k / (ms_dom * 1e-3) / 1e12
    peak = sms * f_mhz * 1e6 * LANE_OPS_PER_CLK_PER_SM / 1e12
    kernel = class_kernel(dom, plan, wl.params.scoring)
    return {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 3), "unit": "Tops/s",
            "frac": round(achieved / peak, 4),
            "frac_at_8_ops": round(achieved * 8 / k / peak, 4),
            "kernel": "%s (batch of its own class: %d pairs, %d cells; CUDA events around the kernel on its "
                      "stream, mean of %d launches)" % (kernel, sub.n_pairs, dom_cells, len(dom_ms)),
            "kernel_name": kernel, "launch_ms": round(ms_dom, 4), "cells_per_launch": dom_cells,
            "ops_per_cell": k,
            "ops_basis": "diagonal add, zero-diagonal rule, 3-way max for H, M - (o + e) (shared by E and F "
                         "when the gap costs are symmetric, else one each), the E and F add-max-clamps, the row "
                         "max with its argmax",
            "peak_basis": "%d SMs x %.0f MHz (median under load) x %d lane-ops/clk (4 schedulers x 32 lanes)"
                          % (sms, f_mhz, LANE_OPS_PER_CLK_PER_SM)}


def measure(bsw, args, name, dist, stream, local, world, rank, headline):
    """One workload: batched GCUPS (timed with clocks sampled), the plain
    baselines, the dominant kernel's roofline, and every pair checked against
    the oracle on rank 0.  The headline workload also gets the end-to-end
    C-ABI leg, the two-pairs-per-thread variant and the CPU baseline."""
    import torch
    from paper_1907_12931_gb300 import workload as W
    base = W.CONFIGS[name]
    wl = W.make(name, n_pairs=args.pairs if headline else None, seed=base["seed"] + rank)
    ctx = bsw.Context(wl.params, mem_budget_bytes=40 << 30)
    hb = bsw.HostBatch(wl)
    db = bsw.DeviceBatch(hb)
    in_bytes = hb.nbytes()
    plan, t_tune = tune(bsw, ctx, name, wl.n_pairs, base["seed"] + 1000 + rank, args)
    steps = args.steps if headline else max(3, args.steps // 2)

    clocks = ClockSampler(local)
    clocks.start()
    ms = time_device(ctx, db, 0, steps, args.warmup, stream, dist)
    clk = clocks.stop()
    cells = int(db.cells.item())
    total_cells = dist.sum(cells)
    gcups = total_cells / (ms * 1e-3) / 1e9
    out_batched = db.out.cpu().numpy().copy()

    # kernels per step and each class kernel's time within one step
    ctx.extend_device(db, bsw.BSW_TIME_KERNELS | bsw.BSW_NO_GRAPH, stream.cuda_stream)
    launches_per_step, step_class_ms = ctx.kernel_times()
    ctx.sync(stream.cuda_stream)

    p_steps = max(3, steps // 10)
    best_c, per, ms_g, g_equal = plain_leg(bsw, ctx, db, plan, p_steps, max(1, args.warmup // 2), stream, dist,
                                           out_batched, cells)
    ms_plain = per[best_c][0]
    gcups_plain = total_cells / (ms_plain * 1e-3) / 1e9
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    roof = dominant_leg(bsw, ctx, wl, plan, stream, dist, steps, clk["sm_mhz"], sms)
    traffic = MEASURED_TRAFFIC.get((name, roof["kernel_name"])) if args.pairs is None or not headline else None
    roof["traffic"] = traffic[0] if traffic else None
    roof["traffic_source"] = traffic[1] if traffic else None
    roof["dram_gbs"] = round(traffic[0] / (roof["launch_ms"] * 1e-3) / 1e9, 1) if traffic else None

    rec = {
        "workload": name, "description": WORKLOAD_TEXT.get(name, name), "pairs": wl.n_pairs,
        "cells_per_step": cells, "value": round(gcups, 3), "unit": "GCUPS", "ms_per_step": round(ms, 4),
        "steps": steps,
        "plain": {"value": round(gcups_plain, 3), "unit": "GCUPS", "ms_per_step": round(ms_plain, 4),
                  "kernel": (("k_plain_x2: the two-columns warp-per-pair kernel, one pair per warp in input "
                              "order, no bucketing or classes (pairs it cannot take run in the 32-bit warp kernel "
                              "after it)") if best_c == "x2" else
                             ("k_plain<%d>: the warp-per-pair ring kernel, one pair per warp in input order, no "
                              "bucketing, classes or re-run list" % best_c))
                            + "; the best of the ring kernel with 4, 8, 16 columns per lane and the two-columns "
                              "kernel",
                  "by_columns": {str(c): {"gcups": round(total_cells / (per[c][0] * 1e-3) / 1e9, 3),
                                          "ms_per_step": round(per[c][0], 4), "bit_exact_vs_batched": per[c][1]}
                                 for c in per},
                  "bit_exact_vs_batched": all(v[1] for v in per.values())},
        "speedup_vs_plain": round(gcups / gcups_plain, 3) if gcups_plain else None,
        "plain_global": {"value": round(total_cells / (ms_g * 1e-3) / 1e9, 3), "unit": "GCUPS",
                         "ms_per_step": round(ms_g, 4),
                         "kernel": "k_plain_global: one column per lane, the row in global memory, input order",
                         "bit_exact_vs_batched": g_equal},
        "roofline": roof,
        "kernels_per_step": launches_per_step,
        "class_ms_in_step": {bsw.CLASS_NAMES[c]: round(t, 4) for c, t in enumerate(step_class_ms) if t > 0},
        "plan": dict(plan.as_dict(), tuned=not (args.no_tune or args.plan), tune_s=round(t_tune, 2),
                     tuned_on="another batch of the same recipe (seed %d)" % (base["seed"] + 1000 + rank)
                     if not (args.no_tune or args.plan) else None),
        "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"], "reasons": clk["reasons"],
                   "samples": clk["samples"]},
        "l2": "inputs larger than L2 (%.0f MB resident packed inputs + %.0f MB results)"
              % (in_bytes / 1e6, wl.n_pairs * 24 / 1e6),
    }

    if headline:
        s_steps = max(3, steps // 10)
        ms_packed = time_device(ctx, db, bsw.BSW_PACKED_PAIRS, s_steps, max(1, args.warmup // 2), stream, dist)
        rec["two_pairs_per_thread"] = {"value": round(total_cells / (ms_packed * 1e-3) / 1e9, 3), "unit": "GCUPS",
                                       "ms_per_step": round(ms_packed, 4),
                                       "bit_exact_vs_batched": bool(np.array_equal(db.out.cpu().numpy(),
                                                                                   out_batched))}
        # end to end through the C ABI with pinned host buffers
        hbp = pinned_host_batch(bsw, bsw.HostBatch(wl))
        pout = torch.empty((wl.n_pairs, 6), dtype=torch.int32, pin_memory=True).numpy()
        e_steps = max(3, steps // 20)
        for _ in range(2):
            ctx.extend_host(hbp, out=pout)
        dist.barrier()
        t0 = time.perf_counter()
        for _ in range(e_steps):
            out_h, cells_h = ctx.extend_host(hbp, out=pout)
        t_e2e = dist.max((time.perf_counter() - t0) / e_steps)
        n = wl.n_pairs
        qb = int((wl.q_off[-1] + wl.q_len[-1] + 3) // 4) if n else 0
        tb = int((wl.t_off[-1] + wl.t_len[-1] + 3) // 4) if n else 0
        rec["e2e"] = {"value": round(dist.sum(cells_h) / t_e2e / 1e9, 3), "unit": "GCUPS",
                      "h2d_bytes_per_step": qb + tb + n * (8 + 4 + 8 + 4 + 4),
                      "d2h_bytes_per_step": n * 24 + 8 + 4 + 40, "ms_per_step": round(t_e2e * 1e3, 3),
                      "bit_exact_vs_device": bool(np.array_equal(out_h, out_batched))}
        rec["in_bytes"] = in_bytes
        rec["_wl"] = wl
        rec["_plan"] = plan

    # every pair against the oracle (rank 0); the headline's pass also times it
    if rank == 0 and not args.no_cpu:
        if headline:
            cpu, res = cpu_baseline(wl)
            rec["cpu_baseline"] = cpu
        else:
            import oracle
            res, _, _ = oracle.extend_batch(wl, nthreads=os.cpu_count() or 1)
        rec["parity"] = {"pairs_checked": int(res.shape[0]), "fields": 6,
                         "mismatches": int((res != out_batched).any(axis=1).sum())}
    ctx.close()
    del db
    return rec


def serve_leg(args):
    """A bounded serving sweep: three offered loads, --serve-quick requests each."""
    import serve_bench
    r = serve_bench.sweep(loads=(0.25, 0.5, 1.0), nreq=args.serve_quick, calib=args.serve_quick)
    return r


def run_gb300(args):
    import torch
    from paper_1907_12931_gb300 import bsw

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = Dist("nccl")
    stream = torch.cuda.Stream()
    head = measure(bsw, args, args.config, dist, stream, local, world, rank, headline=True)
    wl, plan = head.pop("_wl"), head.pop("_plan")
    others = {}
    if not args.only and args.pairs is None:
        for name in SECONDARY:
            if name != args.config:
                r = measure(bsw, args, name, dist, stream, local, world, rank, headline=False)
                others[name] = r

    short_read = args.config in ("read151", "read250") and args.pairs is None
    nb_line = None
    if rank == 0 and not args.no_nbases and short_read and not args.only:
        nb_line = n_bases_leg(bsw, wl, plan, head["value"] / world, stream)
    drv = sal_line = smem_line = serve = None
    if rank == 0 and args.pairs is None and not args.only:
        if not args.no_driver:
            drv = driver_leg(bsw, args)
        if not args.no_sal:
            sal_line = sal_leg(bsw, args, stream, measured_peaks().get("hbm_gbs"))
        if not args.no_smem:
            smem_line = smem_leg(bsw, args)
        if args.serve_quick > 0:
            serve = serve_leg(args)

    if rank == 0:
        line = {
            "metric": METRIC, "value": head["value"], "unit": "GCUPS", "n_gpus": world, "steps": head["steps"],
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "u8 storage, s16x2 arithmetic (two rows per instruction)" if args.config != "long10k"
                     else "int16 storage, s16x2 arithmetic (two columns per instruction)",
            "dtype_note": "per-pair lane storage by the exact score bound h0 + match*min(n, m) (8-bit when <= 255, "
                          "16-bit when <= 32767, else 32-bit); the 8-bit pairs without N bases compute two rows "
                          "per packed s16x2 DPX instruction and the long queries' warp kernel two columns, the "
                          "other kernels in 32-bit registers; pairs whose scores leave their lane range are re-run "
                          "exactly in 32 bits",
            "data": "synthetic",
            "config": {"workload": args.config, "description": head["description"],
                       "pairs_per_gpu": head["pairs"], "cells_per_step": head["cells_per_step"], "l2": head["l2"],
                       "parallelism": "replicas x%d (pairs sharded by rank, no collective)" % world},
            "plain": head["plain"], "speedup_vs_plain": head["speedup_vs_plain"],
            "plain_global": head["plain_global"],
            "two_pairs_per_thread": head["two_pairs_per_thread"],
            "roofline": head["roofline"],
            "cpu_baseline": head.get("cpu_baseline"),
            "parity_sample": head.get("parity"),
            "e2e": head["e2e"],
            "gpu_launches": head["kernels_per_step"] * head["steps"],
            "kernels_per_step": head["kernels_per_step"],
            "class_ms_in_step": head["class_ms_in_step"],
            "plan": head["plan"],
            "clocks": head["clocks"],
            "workloads": others,
            "serving": serve,
            "n_bases": nb_line,
            "extension_driver": drv,
            "suffix_array_lookup": sal_line,
            "smem_search": smem_line,
            "peaks_file": {k: measured_peaks().get(k) for k in ("hbm_gbs", "bf16_tflops", "sm_max_mhz")},
        }
        print(json.dumps(line), flush=True)
    dist.close()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.serve:
        import serve_bench
        return serve_bench.main(args)
    return run_gb300(args)


if __name__ == "__main__":
    sys.exit(main())
