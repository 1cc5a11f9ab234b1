"""N bases (code 4) through the CUDA path against the oracle (needs a GPU).

An N scores -1 against any base, N included, on either side.  Pairs with an
N run in the 8-bit per-thread kernels (N columns select the -1 byte of the
row profile, N rows use an all -1 profile) or, when their scores do not fit
8 bits, in the 32-bit warp kernel with N-aware scoring; the packed two-pair
kernel and the 16-bit classes never see them.  Every result field and the
cell count must match the oracle exactly.
"""
import numpy as np
import pytest

import oracle
from paper_1907_12931_gb300 import workload as W
from test_gpu_parity import NTH, adversarial, assert_same, flag_of, run

pytestmark = pytest.mark.gpu

FLAGS = [0, "plain", "plainglobal", "i8", "i16", "i32", "packed", "i8packed"]


@pytest.fixture(scope="module")
def bsw():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_12931_gb300 import bsw as _b
    _b.lib()
    return _b


def oracle_of(wl, w_override=None):
    res, cells, _ = oracle.extend_batch(wl, nthreads=NTH, w_override=w_override)
    return res, int(cells.sum())


def hand_cases():
    """N at the ends, in the middle, as whole sequences and runs, on each
    side, across the 8-bit, 16-bit and 32-bit score ranges."""
    rng = np.random.default_rng(404)
    qs, ts, hs = [], [], []

    def add(q, t, h0):
        qs.append(np.asarray(q, np.uint8)); ts.append(np.asarray(t, np.uint8)); hs.append(h0)

    for n in (1, 2, 7, 8, 9, 31, 32, 33, 64, 100, 151, 255, 256, 300, 700):
        ref = rng.integers(0, 4, 2 * n + 40).astype(np.uint8)
        q = ref[:n].copy()
        for h0 in (0, 5, 60, 250, 2000, 40000):
            a = q.copy(); a[0] = 4
            add(a, ref[:n + 20], h0)                             # N first
            a = q.copy(); a[-1] = 4
            add(a, ref[:n + 20], h0)                             # N last
            a = q.copy(); a[n // 2] = 4
            add(a, ref[:n + 20], h0)                             # N in the middle
            t = ref[:n + 20].copy(); t[n // 3: n // 3 + 5] = 4
            add(q, t, h0)                                        # run of N in the target
            add(np.full(n, 4), ref[:n + 20], h0)                 # all-N query
            add(q, np.full(n + 20, 4), h0)                       # all-N target
            a = np.where(rng.random(n) < 0.2, 4, q)
            t = np.where(rng.random(n + 20) < 0.2, 4, ref[:n + 20])
            add(a, t, h0)                                        # N on both sides
    return W.from_lists(qs, ts, hs, align=4)


@pytest.mark.parametrize("flags", FLAGS)
def test_hand_cases(bsw, flags):
    wl = hand_cases()
    ref, cells = oracle_of(wl)
    got, gc = run(bsw, wl, flag_of(bsw, flags))
    assert_same(got, ref, "N hand cases/%s" % flags)
    assert gc == cells


@pytest.mark.parametrize("zdrop", [100, 0, 7])
@pytest.mark.parametrize("flags", [0, "plain", "i16", "i32", "i8"])
def test_adversarial_with_n(bsw, zdrop, flags):
    base, ws = adversarial()
    wl = W.inject_n(base, 0.03, 0.01, seed=17)
    wl = W.Workload(wl.name, W.Params(W.Scoring(), w=100, zdrop=zdrop, end_bonus=5), wl.q, wl.q_off, wl.q_len,
                    wl.t, wl.t_off, wl.t_len, wl.h0)
    ref, cells = oracle_of(wl, w_override=ws)
    got, gc = run(bsw, wl, flag_of(bsw, flags), w_override=ws)
    assert_same(got, ref, "adversarial+N zdrop=%d/%s" % (zdrop, flags))
    assert gc == cells


_cache = {}


def n_workload(config, n_pairs, q_rate, t_runs):
    key = (config, n_pairs, q_rate, t_runs)
    if key not in _cache:
        wl = W.inject_n(W.make(config, n_pairs=n_pairs), q_rate, t_runs, seed=5)
        _cache[key] = (wl,) + oracle_of(wl)
    return _cache[key]


@pytest.mark.parametrize("flags", [0, "plain", "i32", "packed"])
@pytest.mark.parametrize("config,n_pairs", [("read151", 200_000), ("read250", 100_000)])
def test_reads_with_n(bsw, config, n_pairs, flags):
    """Reads with 0.2 % scattered N and reference targets with N runs: most
    pairs have none and keep the fast lanes, the rest take the N-aware ones."""
    wl, ref, cells = n_workload(config, n_pairs, 0.002, 0.0005)
    got, gc = run(bsw, wl, flag_of(bsw, flags))
    assert_same(got, ref, "%s+N/%s" % (config, flags))
    assert gc == cells


def test_long_with_n(bsw):
    wl, ref, cells = n_workload("long10k", 2_000, 0.001, 0.0002)
    got, gc = run(bsw, wl, 0)
    assert_same(got, ref, "long10k+N")
    assert gc == cells


@pytest.mark.parametrize("plan", [(256, 0xff, 0xf, 0, 8, 2), (64, 0x0, 0x0, 1, 4, 1), (128, 0x55, 0x5, 0, 16, 4),
                                  (96, 0xff, 0xf, 0, 8, 2, 0, 1)])
def test_plans_with_n(bsw, plan):
    wl, ref, cells = n_workload("read151", 200_000, 0.002, 0.0005)
    with bsw.Context(wl.params, 16 << 30) as ctx:
        ctx.set_plan(bsw.make_plan(*plan))
        got, gc = ctx.extend_host(bsw.HostBatch(wl))
    assert_same(got, ref, "read151+N plan %s" % (plan,))
    assert gc == cells


def test_device_pointers_with_n(bsw):
    import torch
    wl = hand_cases()
    ref, cells = oracle_of(wl)
    with bsw.Context(wl.params, 16 << 30) as ctx:
        db = bsw.DeviceBatch(bsw.HostBatch(wl))
        ctx.extend_device(db, 0)
        ctx.sync()
        torch.cuda.synchronize()
        got, gc = db.out.cpu().numpy(), int(db.cells.item())
    assert_same(got, ref, "N hand cases, device pointers")
    assert gc == cells


def test_autotune_with_n(bsw):
    wl, ref, cells = n_workload("read151", 200_000, 0.002, 0.0005)
    with bsw.Context(wl.params, 16 << 30) as ctx:
        hb = bsw.HostBatch(wl)
        ctx.autotune(hb, reps=1)
        got, gc = ctx.extend_host(hb)
    assert_same(got, ref, "read151+N after autotune")
    assert gc == cells


def test_serving_with_n(bsw):
    """Batches with N bitmaps through the serving loop, merged with N-free
    batches and with each other (some copied at submit): every request gives
    the oracle's results, and the same as alone."""
    hc = hand_cases()
    r151 = W.make("read151", n_pairs=60_000)
    nw = W.inject_n(r151, 0.01, 0.002, seed=9)
    ref_hc, _ = oracle_of(hc)
    ref_nw, _ = oracle_of(nw)
    ref_151, _ = oracle_of(r151)
    rng = np.random.default_rng(31)
    reqs = [(hc, ref_hc)]
    for k in range(12):
        src, ref = ((nw, ref_nw), (r151, ref_151))[k % 2]
        size = int(rng.integers(1, 9000))
        start = int(rng.integers(0, src.n_pairs - size))
        idx = np.arange(start, start + size)
        reqs.append((src.subset(idx), ref[idx]))
    with bsw.Context(hc.params, mem_budget_bytes=4 << 30) as ctx:
        tickets, outs, hbs = [], [], []
        for k, (sub, _) in enumerate(reqs):
            hb = bsw.HostBatch(sub)
            out = np.full((sub.n_pairs, 6), -7, np.int32)
            tickets.append(ctx.submit(hb, out, bsw.BSW_COPY_INPUTS if k % 3 == 1 else 0))
            outs.append(out)
            hbs.append(hb)
        for t in tickets:
            assert ctx.poll(t, 60_000_000) == bsw.BSW_OK
        for (sub, ref), out, hb in zip(reqs, outs, hbs):
            assert_same(out, ref, "served request with N")
            alone, _ = ctx.extend_host(hb)
            np.testing.assert_array_equal(alone, out)
