"""Host logic of bench.py (no GPU): the class mapping it uses to isolate the
dominant kernel, and the CPU-baseline record."""
import itertools

import numpy as np

import bench
from paper_1907_12931_gb300 import workload as W


class _Plan:
    def __init__(self, short_max=256, u8_bounds=0xff, i16_bounds=0xf, packed=0, warp_cols=8, cta_min=0):
        self.short_max, self.u8_bounds, self.i16_bounds = short_max, u8_bounds, i16_bounds
        self.packed, self.warp_cols, self.cta_min = packed, warp_cols, cta_min


def _class_one(n, m, h0, match, plan):
    """One pair, written out from the plan's definition in include/bsw.h."""
    if n <= 0 or m <= 0:
        return -1
    bound = h0 + match * min(n, m)
    if n > plan.short_max:
        if bound > 32767:
            return 14
        return 12 if plan.cta_min and n >= plan.cta_min else 13
    if bound <= 255:
        kept = [k for k in range(8) if k == 0 or (plan.u8_bounds >> k) & 1]
        return max((k for k in kept if bench.U8_NMAX[k] >= n), key=lambda k: k)
    if bound <= 32767:
        kept = [k for k in range(4) if k == 0 or (plan.i16_bounds >> k) & 1]
        return 8 + max(k for k in kept if bench.I16_NMAX[k] >= n)
    return 14


def test_class_of_matches_definition():
    rng = np.random.default_rng(7)
    n = np.concatenate([np.arange(0, 300), rng.integers(0, 20000, 500)])
    m = rng.integers(0, 400, n.shape[0])
    m[::7] = 0
    h0 = rng.integers(0, 300, n.shape[0])
    h0[::11] = 40000
    plans = [_Plan(), _Plan(short_max=64), _Plan(short_max=128, u8_bounds=0x5, i16_bounds=0x1),
             _Plan(u8_bounds=0x0, i16_bounds=0x0), _Plan(short_max=192, u8_bounds=0xa3, i16_bounds=0xb),
             _Plan(short_max=96, cta_min=1024), _Plan(cta_min=128)]
    for plan, match in itertools.product(plans, (1, 2)):
        got = bench.class_of(n, m, h0, match, plan)
        want = [_class_one(int(a), int(b), int(c), match, plan) for a, b, c in zip(n, m, h0)]
        np.testing.assert_array_equal(got, want)


def test_class_kernel_names():
    sc = W.Scoring()
    assert bench.class_kernel(5, _Plan(), sc) == "k_inter<96,u8>"
    assert bench.class_kernel(3, _Plan(), sc) == "k_inter<160,u8>"
    assert bench.class_kernel(5, _Plan(packed=1), sc) == "k_inter2<128>"
    assert bench.class_kernel(3, _Plan(packed=1), sc) == "k_inter<160,u8>"   # packed pairs: bounds up to 128
    assert bench.class_kernel(0, _Plan(packed=1), sc) == "k_inter<256,u8>"
    assert bench.class_kernel(9, _Plan(), sc) == "k_inter<128,i16>"
    assert bench.class_kernel(12, _Plan(cta_min=1024), sc) == "k_cta<8,s16>"
    assert bench.class_kernel(13, _Plan(warp_cols=16), sc) == "k_warp<16,s16>"
    assert bench.class_kernel(14, _Plan(), sc) == "k_warp<8,s32>"
    # large gap costs: the packed kernel does not apply
    assert bench.class_kernel(5, _Plan(packed=1), W.Scoring(1, 200, 100, 1, 100, 1)) == "k_inter<96,u8>"


def test_cpu_baseline_record():
    wl = W.make("plain10k", n_pairs=300)
    cpu, res = bench.cpu_baseline(wl, min_s=0.05, single_s=0.02)
    assert res.shape == (300, 6)
    assert cpu["kind"] == "oracle" and cpu["cores"] >= 1 and cpu["value"] > 0
    assert cpu["single_thread"]["cores"] == 1 and cpu["single_thread"]["value"] > 0


def test_reference_arm_json_line():
    """`bench.py --impl reference` (the oracle on the host cores) prints one
    JSON line with the keys the benchmark contract names."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--config", "plain10k",
                        "--steps", "1", "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["unit"] == "GCUPS" and d["value"] > 0
    assert d["config"]["workload"] == "plain10k"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "GCUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
