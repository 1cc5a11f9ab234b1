"""Execution plans, the autotuner and per-kernel timing (needs a GPU).

Every plan (which kernel runs which pairs: the per-thread/warp boundary, the
per-thread length classes, one or two pairs per thread, the warp kernel's
columns per lane, warps per block) must give the oracle's results bit for bit;
the autotuner only chooses among them.
"""
import numpy as np
import pytest

import oracle
from paper_1907_12931_gb300 import workload as W
from test_gpu_parity import NTH, adversarial, assert_same, workload_and_oracle

pytestmark = pytest.mark.gpu

PLANS = [
    {},
    {"short_max": 64},
    {"short_max": 64, "warp_cols": 4},
    {"short_max": 96, "warp_cols": 16},
    {"u8_bounds": 0x1, "i16_bounds": 0x1},
    {"u8_bounds": 0x55, "i16_bounds": 0x5, "inter_warps": 1},
    {"packed": 1, "inter_warps": 4},
    {"short_max": 128, "packed": 1, "u8_bounds": 0x0, "warp_cols": 16},
    {"short_max": 64, "cta_min": 128},
    {"short_max": 96, "warp_cols": 16, "cta_min": 1024},
    {"cta_min": 4096, "warp_cols": 4},
    {"warp_x2": 1},
    {"short_max": 64, "warp_x2": 1, "u8_bounds": 0x55},
    {"short_max": 96, "warp_x2": 1, "cta_min": 1024},
]


@pytest.fixture(scope="module")
def bsw():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_12931_gb300 import bsw as _b
    _b.lib()
    return _b


def run_plan(bsw, wl, plan, flags=0, w_override=None, device=False):
    with bsw.Context(wl.params, 16 << 30) as ctx:
        ctx.set_plan(bsw.make_plan(**plan))
        hb = bsw.HostBatch(wl, w_override=w_override)
        if not device:
            return ctx.extend_host(hb, flags)
        import torch
        db = bsw.DeviceBatch(hb)
        ctx.extend_device(db, flags)
        ctx.sync()
        torch.cuda.synchronize()
        return db.out.cpu().numpy(), int(db.cells.item())


@pytest.mark.parametrize("plan", PLANS, ids=[str(sorted(p.items())) for p in PLANS])
@pytest.mark.parametrize("config", [("read250", 40_000), ("long10k", 400)])
def test_plan_parity_workloads(bsw, plan, config):
    wl, ref, cells = workload_and_oracle(*config)
    got, gc = run_plan(bsw, wl, plan, device=True)
    assert_same(got, ref, "%s plan %s" % (config[0], plan))
    assert gc == cells


@pytest.mark.parametrize("plan", PLANS, ids=[str(sorted(p.items())) for p in PLANS])
def test_plan_parity_adversarial(bsw, plan):
    """Band edges, w = 0/1/unbounded (the unbounded band leaves the shared-memory
    ring for the global slot path), u8 bound edges, every query length class."""
    wl, ws = adversarial()
    wl.params = W.Params(W.Scoring(), w=100, zdrop=100, end_bonus=5)
    ref, cells, _ = oracle.extend_batch(wl, nthreads=NTH, w_override=ws)
    got, gc = run_plan(bsw, wl, plan, w_override=ws)
    assert_same(got, ref, "adversarial plan %s" % plan)
    assert gc == int(cells.sum())


@pytest.mark.parametrize("flag", ["BSW_FORCE_I8", "BSW_FORCE_I16", "BSW_FORCE_I32"])
def test_forced_lanes_under_plan(bsw, flag):
    """Forced lane widths keep every query up to 256 on the per-thread kernels
    whatever short_max says, and saturating pairs are re-run exactly."""
    wl, ws = adversarial()
    wl.params = W.Params(W.Scoring(), w=100, zdrop=100, end_bonus=5)
    ref, cells, _ = oracle.extend_batch(wl, nthreads=NTH, w_override=ws)
    plan = {"short_max": 64, "u8_bounds": 0x1, "i16_bounds": 0x3, "warp_cols": 4}
    got, gc = run_plan(bsw, wl, plan, flags=getattr(bsw, flag), w_override=ws)
    assert_same(got, ref, "adversarial %s" % flag)
    assert gc == int(cells.sum())


def test_set_plan_rejects_bad_fields(bsw):
    wl, _, _ = workload_and_oracle("plain10k")
    bad = [{"short_max": 63}, {"short_max": 257}, {"warp_cols": 5}, {"warp_cols": 32}, {"inter_warps": 3},
           {"packed": 2}, {"u8_bounds": 0x100}, {"i16_bounds": 0x10}, {"cta_min": 64}, {"cta_min": 1000},
           {"cta_min": 32832}, {"cta_min": -64}, {"warp_x2": 2}, {"warp_x2": -1}]
    with bsw.Context(wl.params) as ctx:
        before = ctx.get_plan().as_dict()
        assert before == {"short_max": 256, "u8_bounds": 0xff, "i16_bounds": 0xf, "packed": 0, "warp_cols": 8,
                          "inter_warps": 2, "cta_min": 0, "warp_x2": 0, "ms": 0.0}
        for b in bad:
            with pytest.raises(bsw.BswError) as ei:
                ctx.set_plan(bsw.make_plan(**b))
            assert ei.value.code == bsw.BSW_EINVAL
        assert ctx.get_plan().as_dict() == before
        ctx.set_plan(bsw.make_plan(short_max=128, u8_bounds=0x0))
        p = ctx.get_plan()
        assert p.short_max == 128 and p.u8_bounds == 0x1   # the 256 class is always kept


@pytest.mark.parametrize("device", [False, True])
def test_autotune_then_parity(bsw, device):
    wl, ref, cells = workload_and_oracle("read151", 200_000)
    with bsw.Context(wl.params, 16 << 30) as ctx:
        hb = bsw.HostBatch(wl)
        if device:
            import torch
            db = bsw.DeviceBatch(hb)
            p = ctx.autotune(db, sample_pairs=100_000, reps=2)
        else:
            p = ctx.autotune(hb, sample_pairs=100_000, reps=2)
        assert p.ms > 0
        q = ctx.get_plan()
        assert q.as_dict() == p.as_dict()
        assert 64 <= p.short_max <= 256 and p.warp_cols in (4, 8, 16) and p.inter_warps in (1, 2, 4)
        if device:
            ctx.extend_device(db)
            ctx.sync()
            torch.cuda.synchronize()
            got, gc = db.out.cpu().numpy(), int(db.cells.item())
        else:
            got, gc = ctx.extend_host(hb)
    assert_same(got, ref, "read151 after autotune (%s)" % p.as_dict())
    assert gc == cells


def test_autotune_long_queries(bsw):
    wl, ref, cells = workload_and_oracle("long10k", 2000)
    with bsw.Context(wl.params, 16 << 30) as ctx:
        hb = bsw.HostBatch(wl)
        p = ctx.autotune(hb, reps=1)
        got, gc = ctx.extend_host(hb)
    assert p.ms > 0
    assert_same(got, ref, "long10k after autotune (%s)" % p.as_dict())
    assert gc == cells


def test_autotune_rejects_flags_and_empty_is_noop(bsw):
    wl, _, _ = workload_and_oracle("plain10k")
    with bsw.Context(wl.params) as ctx:
        hb = bsw.HostBatch(wl)
        rc, _ = bsw.bsw_autotune(ctx.handle, hb.struct(bsw.BSW_PLAIN_KERNEL), 0, 1)
        assert rc == bsw.BSW_EINVAL
        rc, p = bsw.bsw_autotune(ctx.handle, hb.struct(0), -5, 1)   # <= 0: the default sample
        assert rc == bsw.BSW_OK and p.ms > 0
        empty = hb.struct(0)
        empty.n_pairs = 0
        before = ctx.get_plan().as_dict()
        rc, p = bsw.bsw_autotune(ctx.handle, empty, 0, 1)
        assert rc == bsw.BSW_OK and p.as_dict() == before


def test_kernel_times(bsw):
    import torch
    wl, ref, _ = workload_and_oracle("read151", 200_000)
    with bsw.Context(wl.params, 16 << 30) as ctx:
        rc, _ = bsw.bsw_kernel_times(ctx.handle)
        assert rc == bsw.BSW_ESTATE                       # no timed call yet
        db = bsw.DeviceBatch(bsw.HostBatch(wl))
        with pytest.raises(bsw.BswError):                 # events inside a graph: refused
            ctx.extend_device(db, bsw.BSW_TIME_KERNELS)
        ctx.extend_device(db, bsw.BSW_TIME_KERNELS | bsw.BSW_NO_GRAPH)
        launches, ms = ctx.kernel_times()
        ctx.sync()
        torch.cuda.synchronize()
        assert_same(db.out.cpu().numpy(), ref, "timed launch")
        assert launches == 18                              # 3 bucketing + 14 classes (no block class) + re-run
        assert ms[5] > 0 and ms[15] > 0                    # u8<96> carries most cells; re-run always launches
        assert ms[12] == 0                                 # cta_min 0: no block-per-pair launch
        assert all(t >= 0 for t in ms)
        # a plan with fewer classes launches fewer kernels
        ctx.set_plan(bsw.make_plan(short_max=128, u8_bounds=0x5, i16_bounds=0x1))
        ctx.extend_device(db, bsw.BSW_TIME_KERNELS | bsw.BSW_NO_GRAPH)
        launches2, ms2 = ctx.kernel_times()
        # bounds kept: 256 and 192.  u8<256> would hold only queries over 192
        # bases, which short_max 128 sends to the warp kernel, so it is
        # skipped; live: u8<192> (every query up to 128), i16<256>, the two
        # warp classes and the re-run
        assert launches2 == 3 + 5
        assert ms2[0] == 0 and ms2[1] == 0 and ms2[3] == 0 and ms2[2] > 0
        ctx.sync()
        torch.cuda.synchronize()
        assert_same(db.out.cpu().numpy(), ref, "timed launch, reduced plan")


@pytest.mark.parametrize("cols,cta", [(4, 0), (8, 0), (16, 0), (8, 128)])
def test_ring_wrap_band_edges(bsw, cols, cta):
    """Band widths just under a power of two with full-width bands (near
    identical sequences): the chunks' out-of-band lanes reach furthest past the
    band there, and must never read a band column through the ring's wrap."""
    rng = np.random.default_rng(99)
    qs, ts, hs = [], [], []
    for n in (700, 1100, 1600, 2300):
        for _ in range(3):
            ref = rng.integers(0, 4, n + 1200)
            q = ref[:n].copy()
            flip = rng.random(n) < 0.01
            q[flip] = (q[flip] + 1) % 4
            qs.append(q.astype(np.uint8)); ts.append(ref[: n + 600].astype(np.uint8)); hs.append(int(rng.integers(20, 60)))
    wl = W.from_lists(qs, ts, hs, align=4)
    for w in (126, 127, 254, 255, 500, 508, 510, 511):
        wl.params = W.Params(W.Scoring(), w=w, zdrop=0, end_bonus=5)
        ref, cells, _ = oracle.extend_batch(wl, nthreads=NTH)
        got, gc = run_plan(bsw, wl, {"short_max": 64, "warp_cols": cols, "cta_min": cta}, device=True)
        assert_same(got, ref, "w=%d cols=%d cta_min=%d" % (w, cols, cta))
        assert gc == int(cells.sum())


@pytest.mark.parametrize("w", [3, 40, 100, 127, 128, 129, 383, 384, 500, 1000, 2100])
def test_block_per_pair_band_widths(bsw, w):
    """One pair per block over band widths that give one chunk, several chunks
    in one round, and several rounds (4 warps x 256 columns per round), with
    z-drop on, for long near-copies and for queries with indels."""
    rng = np.random.default_rng(1000 + w)
    qs, ts, hs = [], [], []
    for n in (130, 300, 900, 2500, 5000):
        for err in (0.0, 0.02, 0.12):
            ref = rng.integers(0, 4, n + w + 600).astype(np.uint8)
            q = list(ref[:n])
            k = 0
            out = []
            while k < len(q):                                  # substitutions and 1-3 bp indels
                u = rng.random()
                if u < err / 2:
                    out.append(int((q[k] + 1 + rng.integers(0, 3)) % 4)); k += 1
                elif u < 3 * err / 4:
                    k += int(rng.integers(1, 4))
                elif u < err:
                    out.extend(int(x) for x in rng.integers(0, 4, int(rng.integers(1, 4)))); 
                else:
                    out.append(int(q[k])); k += 1
            qs.append(np.array(out, np.uint8)); ts.append(ref[: len(out) + w]); hs.append(int(rng.integers(19, 61)))
    wl = W.from_lists(qs, ts, hs, align=4)
    for zd in (100, 0):
        wl.params = W.Params(W.Scoring(), w=w, zdrop=zd, end_bonus=5)
        ref, cells, _ = oracle.extend_batch(wl, nthreads=NTH)
        got, gc = run_plan(bsw, wl, {"short_max": 64, "cta_min": 128}, device=True)
        assert_same(got, ref, "block per pair w=%d zdrop=%d" % (w, zd))
        assert gc == int(cells.sum())


def test_block_per_pair_other_scorings(bsw):
    """Asymmetric gap costs and extensions above 1 take the kernel's general
    variants (no shared M - o - e, no immediate offsets)."""
    wl = W.make("long10k", n_pairs=600)
    for sc in ((1, 4, 6, 1, 6, 1), (2, 3, 5, 2, 4, 1), (1, 6, 1, 1, 1, 1), (5, 9, 3, 3, 8, 2), (1, 4, 6, 2, 6, 2)):
        wl.params = W.Params(W.Scoring(*sc), w=300, zdrop=200, end_bonus=3)
        ref, cells, _ = oracle.extend_batch(wl, nthreads=NTH)
        got, gc = run_plan(bsw, wl, {"short_max": 96, "cta_min": 512}, device=True)
        assert_same(got, ref, "block per pair scoring %s" % (sc,))
        assert gc == int(cells.sum())


def test_block_per_pair_band_override(bsw):
    """Per-pair bands wider than the context's ring go to the re-run list."""
    wl = W.make("long10k", n_pairs=500)
    ws = np.where(np.arange(wl.n_pairs) % 3 == 0, 1500, np.where(np.arange(wl.n_pairs) % 3 == 1, 50, 500))
    ws = ws.astype(np.int32)
    ref, cells, _ = oracle.extend_batch(wl, nthreads=NTH, w_override=ws)
    got, gc = run_plan(bsw, wl, {"short_max": 96, "cta_min": 256}, w_override=ws)
    assert_same(got, ref, "block per pair, band overrides")
    assert gc == int(cells.sum())
