"""Serving benchmark: Poisson arrivals of mixed-size extension requests.

Each request is a batch of 1..50 000 pairs drawn from one of three pools with
probability 1/3 each: the 151 bp and 250 bp short-read workloads (one context:
w 100, zdrop 100) and the long-query workload (a second context: w 500,
zdrop 400); the two contexts share a 20 GB device budget.  Requests are
submitted with bsw_stream_submit at their arrival times and collected with
bsw_stream_poll.  The peak is the throughput with every request queued at
once; the offered load is then swept from 10% to 100% of it, and p50/p99
latency (arrival to completion) and throughput are reported per load point.
Every request's results are compared with the CPU oracle.  Submissions draw
from 48 distinct requests (16 per pool, each packed once).  Before the sweep
each context's plan is autotuned on its pool (the short-read context on the
250 bp pool, which spans both short-read length ranges).
"""
from __future__ import annotations

import json
import os
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1907_12931_gb300 import bsw, workload as W  # noqa: E402

POOL_PAIRS = {"read151": 200_000, "read250": 200_000, "long10k": 20_000}
MAX_REQ = 50_000


class Pool:
    def __init__(self, name, nthreads):
        import oracle
        self.name = name
        self.wl = W.make(name, n_pairs=POOL_PAIRS[name])
        self.ref, self.cells, _ = oracle.extend_batch(self.wl, nthreads=nthreads)

    def request(self, rng, size):
        idx = rng.integers(0, self.wl.n_pairs, size)
        sub = self.wl.subset(idx)
        return sub, self.ref[idx], int(self.cells[idx].sum())


def _percentile(x, q):
    return float(np.percentile(np.asarray(x), q)) if len(x) else None


def run_point(ctxs, reqs, rate, verify):
    """Submit reqs (list of (pool_idx, HostBatch, ref, cells)) at Poisson times
    with the given rate (requests/s; None = all at once).  Returns latencies,
    wall time, cells and mismatches."""
    for c in set(ctxs):
        c.stream_stats(reset=True)
    n = len(reqs)
    rng = np.random.default_rng(12345)
    gaps = rng.exponential(1.0 / rate, n) if rate else np.zeros(n)
    arrivals = np.cumsum(gaps)
    outs = [np.full((r[1].n, 6), -1, np.int32) for r in reqs]
    tickets = [None] * n
    submit_t = [0.0] * n
    done_t = [None] * n
    lock = threading.Lock()
    finished = threading.Event()
    t0 = time.perf_counter()

    def poller():
        pending = set()
        nxt = 0
        while True:
            with lock:
                while nxt < n and tickets[nxt] is not None:
                    pending.add(nxt)
                    nxt += 1
            for k in list(pending):
                rc = ctxs[reqs[k][0]].poll(tickets[k], 0)
                if rc == bsw.BSW_OK:
                    done_t[k] = time.perf_counter()
                    pending.discard(k)
                elif rc != bsw.BSW_PENDING:
                    raise RuntimeError("request %d failed: %s" % (k, bsw.bsw_strerror(rc)))
            if nxt == n and not pending:
                finished.set()
                return
            time.sleep(5e-5)

    th = threading.Thread(target=poller, daemon=True)
    th.start()
    for k in range(n):
        target = t0 + arrivals[k]
        while True:
            now = time.perf_counter()
            if now >= target:
                break
            time.sleep(min(target - now, 1e-3))
        submit_t[k] = t0 + arrivals[k]
        tk = ctxs[reqs[k][0]].submit(reqs[k][1], outs[k])
        with lock:
            tickets[k] = tk
    finished.wait()
    th.join()
    wall = max(done_t) - t0
    lat = [(done_t[k] - submit_t[k]) * 1e3 for k in range(n)]
    cells = sum(r[3] for r in reqs)
    mism = 0
    if verify:
        for k in range(n):
            mism += int((outs[k] != reqs[k][2]).any(axis=1).sum())
    return lat, wall, cells, mism


def sweep(loads=(0.1, 0.2, 0.3, 0.4, 0.5, 0.6, 0.7, 0.8, 0.9, 1.0), nreq=1000, calib=200, verify=True):
    """The serving sweep: pools, contexts, tuned plans, the all-queued peak,
    then one point per offered load.  Returns the result record."""
    nth = os.cpu_count() or 1
    names = ["read151", "read250", "long10k"]
    pools = [Pool(nm, nth) for nm in names]
    ctx_short = bsw.Context(pools[0].wl.params, 14 << 30)
    ctx_long = bsw.Context(pools[2].wl.params, 6 << 30)
    ctxs = [ctx_short, ctx_short, ctx_long]
    plans = {"short": ctx_short.autotune(bsw.HostBatch(pools[1].wl)).as_dict(),
             "long": ctx_long.autotune(bsw.HostBatch(pools[2].wl)).as_dict()}
    rng = np.random.default_rng(2024)

    # A set of distinct requests (packed once); submissions draw from it.
    distinct = []
    for p in range(3):
        for _ in range(16):
            size = int(rng.integers(1, MAX_REQ + 1))
            sub, ref, cells = pools[p].request(rng, size)
            distinct.append((p, bsw.HostBatch(sub), ref, cells))
            del sub

    def make_reqs(count):
        return [distinct[int(k)] for k in rng.integers(0, len(distinct), count)]

    # peak: every request queued at once
    creqs = make_reqs(min(nreq, calib))
    run_point(ctxs, creqs[:20], None, False)                   # warm-up
    lat, wall, cells, mism = run_point(ctxs, creqs, None, verify)
    peak_gcups = cells / wall / 1e9
    mean_cells = cells / len(creqs)
    points = []
    total_mism = mism
    reqs = make_reqs(nreq)
    for load in loads:
        rate = load * peak_gcups * 1e9 / mean_cells
        lat, wall, cells, mism = run_point(ctxs, reqs, rate, verify)
        total_mism += mism
        st = [c.stream_stats() for c in (ctx_short, ctx_long)]
        busy = sum(x["busy_ms"] for x in st)
        points.append({"offered_load": load, "offered_req_per_s": round(rate, 2),
                       "p50_ms": round(_percentile(lat, 50), 3), "p99_ms": round(_percentile(lat, 99), 3),
                       "throughput_gcups": round(cells / wall / 1e9, 2), "requests": len(reqs),
                       "mismatches": mism,
                       "launches": sum(x["launches"] for x in st),
                       "merged_requests": sum(x["merged"] for x in st),
                       "budget_waits": sum(x["budget_waits"] for x in st),
                       "device_busy_ms_per_context": [round(x["busy_ms"], 2) for x in st],
                       "overlap_per_context": [round(x["busy_ms"] / x["union_ms"], 3) if x["union_ms"] else None
                                               for x in st],
                       "max_concurrent_launches": [x["max_concurrent"] for x in st],
                       "wall_ms": round(wall * 1e3, 2),
                       "device_busy_fraction_of_wall": round(busy / (wall * 1e3), 3)})
    ctx_short.close()
    ctx_long.close()
    return {
        "workload": "serve: Poisson arrivals, requests of 1-50000 pairs from read151/read250/long10k "
                    "pools (p = 1/3 each), 20 GB budget over two contexts",
        "requests_per_point": nreq, "peak_gcups_all_queued": round(peak_gcups, 2),
        "mean_cells_per_request": int(mean_cells), "plans": plans,
        "points": points, "bit_exact_mismatches": total_mism,
        "parity": "every result of every request compared with the oracle" if verify else "not checked",
    }


def main(args) -> int:
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if int(os.environ.get("RANK", "0")) != 0:
        return 0
    nreq = int(getattr(args, "serve_requests", 0) or 1000)
    r = sweep(nreq=nreq)
    points = r["points"]
    line = {
        "metric": "BSW serve p50/p99 latency vs offered load (continuous batching)",
        "value": points[-1]["p99_ms"], "unit": "ms (p99 at 100% offered load)", "n_gpus": world,
        "higher_is_better": False, "data": "synthetic",
        "config": {"workload": r["workload"], "requests_per_point": nreq,
                   "peak_gcups_all_queued": r["peak_gcups_all_queued"],
                   "mean_cells_per_request": r["mean_cells_per_request"], "plans": r["plans"]},
        "points": points, "bit_exact_mismatches": r["bit_exact_mismatches"],
    }
    print(json.dumps(line), flush=True)
    return 0 if r["bit_exact_mismatches"] == 0 else 1
