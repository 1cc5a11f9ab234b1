"""Parity of the CUDA path with the CPU oracle (needs a GPU).

Every comparison is bit-exact on all six result fields, plus the total cell
count.  The oracle runs on the host cores over the same seeded inputs.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1907_12931_gb300 import workload as W

pytestmark = pytest.mark.gpu

NTH = os.cpu_count() or 4


@pytest.fixture(scope="module")
def bsw():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_12931_gb300 import bsw as _b
    _b.lib()
    return _b


_cache = {}


def workload_and_oracle(config, n_pairs=None):
    key = (config, n_pairs)
    if key not in _cache:
        wl = W.make(config, n_pairs=n_pairs)
        res, cells, _ = oracle.extend_batch(wl, nthreads=NTH)
        _cache[key] = (wl, res, int(cells.sum()))
    return _cache[key]


def assert_same(got, ref, what):
    bad = np.nonzero((got != ref).any(axis=1))[0]
    if bad.size:
        k = bad[0]
        raise AssertionError("%s: %d of %d pairs differ; first pair %d: gpu %s oracle %s"
                             % (what, bad.size, ref.shape[0], k, got[k].tolist(), ref[k].tolist()))


def run(bsw, wl, flags=0, device=False, budget=16 << 30, w_override=None, params=None, warp_cols=None, cta_min=0,
        warp_x2=0):
    with bsw.Context(params or wl.params, budget) as ctx:
        if warp_cols is not None or cta_min or warp_x2:
            ctx.set_plan(bsw.make_plan(warp_cols=warp_cols or 8, cta_min=cta_min, warp_x2=warp_x2))
        hb = bsw.HostBatch(wl, w_override=w_override)
        if not device:
            return ctx.extend_host(hb, flags)
        import torch
        db = bsw.DeviceBatch(hb)
        ctx.extend_device(db, flags)
        ctx.sync()
        torch.cuda.synchronize()
        return db.out.cpu().numpy(), int(db.cells.item())


def flag_of(bsw, name):
    return {0: 0, "plain": bsw.BSW_PLAIN_KERNEL, "plainglobal": bsw.BSW_PLAIN_GLOBAL,
            "i8": bsw.BSW_FORCE_I8, "i16": bsw.BSW_FORCE_I16,
            "i32": bsw.BSW_FORCE_I32, "packed": bsw.BSW_PACKED_PAIRS,
            "i8packed": bsw.BSW_FORCE_I8 | bsw.BSW_PACKED_PAIRS}[name]


@pytest.mark.parametrize("flags", [0, "plain", "plainglobal", "i8", "i16", "i32", "packed", "i8packed"])
def test_plain10k(bsw, flags):
    wl, ref, cells = workload_and_oracle("plain10k")
    f = flag_of(bsw, flags)
    got, gc = run(bsw, wl, f)
    assert_same(got, ref, "plain10k/%s" % flags)
    assert gc == cells


@pytest.mark.parametrize("device", [False, True])
def test_plain10k_device_pointers(bsw, device):
    wl, ref, cells = workload_and_oracle("plain10k")
    got, gc = run(bsw, wl, 0, device=device)
    assert_same(got, ref, "plain10k device=%s" % device)
    assert gc == cells


@pytest.mark.parametrize("config", ["read151", "read250", "long10k"])
def test_full_workloads_batched(bsw, config):
    wl, ref, cells = workload_and_oracle(config)
    got, gc = run(bsw, wl, 0, device=True)
    assert_same(got, ref, config)
    assert gc == cells


@pytest.mark.parametrize("config", ["read151", "read250"])
def test_full_workloads_packed_pairs(bsw, config):
    wl, ref, cells = workload_and_oracle(config)
    got, gc = run(bsw, wl, bsw.BSW_PACKED_PAIRS, device=True)
    assert_same(got, ref, config + "/packed")
    assert gc == cells


@pytest.mark.parametrize("config", ["read151", "read250", "long10k"])
@pytest.mark.parametrize("warp_cols", [4, 8, 16])
def test_full_workloads_plain(bsw, config, warp_cols):
    """The plain baseline (the ring warp kernel over pairs in input order) with
    each column count, on every pair of the full workloads."""
    wl, ref, cells = workload_and_oracle(config)
    got, gc = run(bsw, wl, bsw.BSW_PLAIN_KERNEL, device=True, warp_cols=warp_cols)
    assert_same(got, ref, "%s/plain C=%d" % (config, warp_cols))
    assert gc == cells


@pytest.mark.parametrize("config", ["read151", "long10k"])
def test_full_workloads_plain_global(bsw, config):
    wl, ref, cells = workload_and_oracle(config)
    got, gc = run(bsw, wl, bsw.BSW_PLAIN_GLOBAL, device=True)
    assert_same(got, ref, config + "/plain global")
    assert gc == cells


def test_read151_forced_lanes(bsw):
    """int8 lanes without the bound check on long-seed pairs whose scores pass
    255 force the exact 32-bit re-run (Section V-D1); int16 and int32 too."""
    wl, ref, cells = workload_and_oracle("read151", 200_000)
    big = wl.subset(np.arange(0, 4000))
    hb_h0 = big.h0.copy()
    big.h0[:] = np.minimum(hb_h0 + 200, 250)   # many bounds above 255
    ref2, c2, _ = oracle.extend_batch(big, nthreads=NTH)
    for name in ("BSW_FORCE_I8", "BSW_FORCE_I16", "BSW_FORCE_I32"):
        got, gc = run(bsw, big, getattr(bsw, name))
        assert_same(got, ref2, name)
        assert gc == int(c2.sum())
    got, gc = run(bsw, wl, bsw.BSW_FORCE_I8)
    assert_same(got, ref, "read151 i8")


def adversarial():
    rng = np.random.default_rng(12345)
    qs, ts, hs, ws = [], [], [], []

    def add(q, t, h0, w=100):
        qs.append(np.asarray(q, np.uint8)); ts.append(np.asarray(t, np.uint8)); hs.append(h0); ws.append(w)

    lens = [0, 1, 2, 3, 4, 5, 15, 16, 17, 31, 32, 33, 63, 64, 65, 95, 96, 97, 127, 128, 129, 159, 160, 161, 191, 192,
            193, 223, 224, 225, 255, 256, 257, 300, 600]
    for n in lens:
        for m in (0, 1, n, n + 100, max(1, n // 2)):
            ref = rng.integers(0, 4, n + m + 8)
            q = ref[:n].copy()
            flip = rng.random(n) < 0.05
            q = np.where(flip, (q + 1) % 4, q)
            add(q, ref[:m], int(rng.integers(0, 90)))
            add(q, ref[:m], 0)
            add(np.zeros(n), np.full(m, 1), 40)                    # all mismatch
            add(np.full(n, 2), np.full(m, 2), 30)                   # homopolymer match
            add(q, ref[:m], max(0, 255 - min(n, m)))                 # u8 bound edge
            add(q, ref[:m], max(0, 256 - min(n, m)))                 # just over
            add(q, ref[:m], int(rng.integers(0, 50)), w=0)
            add(q, ref[:m], int(rng.integers(0, 50)), w=1)
            add(q, ref[:m], int(rng.integers(0, 50)), w=n + m + 5)
    # adjacent insertion/deletion, long indels
    for _ in range(300):
        n = int(rng.integers(10, 200))
        t = rng.integers(0, 4, n + 120)
        q = list(t[:n])
        p = int(rng.integers(1, n - 2))
        k = int(rng.integers(1, 12))
        q = q[:p] + list(rng.integers(0, 4, k)) + q[p + k + int(rng.integers(0, 5)):]
        add(q, t, int(rng.integers(5, 80)))
    return W.from_lists(qs, ts, hs, align=4), np.array(ws, np.int32)


@pytest.mark.parametrize("zdrop", [100, 0, 1, 7])
@pytest.mark.parametrize("flags", [0, "plain", "plain4", "plain16", "plainglobal", "i16", "i32", "i8", "packed"])
def test_adversarial(bsw, zdrop, flags):
    wl, ws = adversarial()
    params = W.Params(W.Scoring(), w=100, zdrop=zdrop, end_bonus=5)
    wl.params = params
    ref, cells, _ = oracle.extend_batch(wl, nthreads=NTH, w_override=ws)
    cols = None
    if flags in ("plain4", "plain16"):
        cols = int(flags[5:])
        flags = "plain"
    f = flag_of(bsw, flags)
    got, gc = run(bsw, wl, f, w_override=ws, warp_cols=cols)
    assert_same(got, ref, "adversarial zdrop=%d flags=%s" % (zdrop, flags))
    assert gc == int(cells.sum())


@pytest.mark.parametrize("sc", [(1, 4, 6, 1, 6, 1), (2, 3, 5, 2, 4, 1), (1, 6, 1, 1, 1, 1), (5, 9, 3, 3, 8, 2)])
def test_other_scorings(bsw, sc):
    wl = W.make("read250", n_pairs=30000)
    params = W.Params(W.Scoring(*sc), w=60, zdrop=40, end_bonus=3)
    wl.params = params
    ref, cells, _ = oracle.extend_batch(wl, nthreads=NTH)
    for f in (0, bsw.BSW_PLAIN_KERNEL, bsw.BSW_FORCE_I32, bsw.BSW_PACKED_PAIRS):
        got, gc = run(bsw, wl, f)
        assert_same(got, ref, "scoring %s flags %d" % (sc, f))
        assert gc == int(cells.sum())


def test_split_equals_whole(bsw):
    """Pairs are independent: k-way splits of one batch give the same results."""
    wl, ref, cells = workload_and_oracle("read151", 200_000)
    whole, _ = run(bsw, wl)
    parts = []
    for idx in np.array_split(np.arange(wl.n_pairs), 5):
        g, _ = run(bsw, wl.subset(idx))
        parts.append(g)
    np.testing.assert_array_equal(np.concatenate(parts), whole)
    assert_same(whole, ref, "whole")


def test_graph_replay_sees_new_inputs(bsw):
    """Device-pointer calls replay a captured graph; new contents of the same
    buffers give the new results."""
    import torch
    a, ref_a, _ = workload_and_oracle("plain10k")
    b = W.make("plain10k", seed=99)
    ref_b, _, _ = oracle.extend_batch(b, nthreads=NTH)
    with bsw.Context(a.params) as ctx:
        ha, hb = bsw.HostBatch(a), bsw.HostBatch(b)
        db = bsw.DeviceBatch(ha)
        for _ in range(2):
            ctx.extend_device(db)
            ctx.sync()
            assert_same(db.out.cpu().numpy(), ref_a, "replay a")
        # same shapes? copy b's arrays into a's buffers where they fit
        if hb.q.nbytes <= db.q.numel() and hb.t.nbytes <= db.t.numel():
            db.q[: hb.q.nbytes].copy_(torch.from_numpy(hb.q))
            db.t[: hb.t.nbytes].copy_(torch.from_numpy(hb.t))
            for name in ("q_off", "q_len", "t_off", "t_len", "h0"):
                getattr(db, name).copy_(torch.from_numpy(getattr(hb, name)))
            ctx.extend_device(db)
            ctx.sync()
            assert_same(db.out.cpu().numpy(), ref_b, "replay b")


def test_invalid_inputs_and_recovery(bsw):
    wl, ref, _ = workload_and_oracle("plain10k")
    with bsw.Context(wl.params) as ctx:
        for field, val in (("q_len", -1), ("h0", -5), ("q_off", 2)):
            hb = bsw.HostBatch(wl)
            getattr(hb, field)[7] = val
            with pytest.raises(bsw.BswError) as e:
                ctx.extend_host(hb)
            assert e.value.code == bsw.BSW_EINVAL
        # the device-pointer path reports the same through bsw_sync
        hb = bsw.HostBatch(wl)
        db = bsw.DeviceBatch(hb)
        db.q_len[3] = -1
        ctx.extend_device(db, bsw.BSW_NO_GRAPH)
        with pytest.raises(bsw.BswError):
            ctx.sync()
        got, _ = ctx.extend_host(bsw.HostBatch(wl))
        assert_same(got, ref, "after errors")


def test_invalid_inputs_large_batch(bsw):
    """Batches above the host-check size are checked on the device before any
    sequence is copied: the same errors, and the context stays usable."""
    wl, ref, _ = workload_and_oracle("read151", 200_000)
    with bsw.Context(wl.params, 16 << 30) as ctx:
        for field, k, val in (("q_len", 99_999, -1), ("h0", 50_000, -5), ("t_off", 3, 6), ("q_len", 12, 40_000)):
            hb = bsw.HostBatch(wl)
            getattr(hb, field)[k] = val
            with pytest.raises(bsw.BswError) as e:
                ctx.extend_host(hb)
            assert e.value.code == bsw.BSW_EINVAL, (field, k, val)
        hb = bsw.HostBatch(wl, w_override=np.full(wl.n_pairs, 100, np.int32))
        hb.w[777] = -1
        with pytest.raises(bsw.BswError) as e:
            ctx.extend_host(hb)
        assert e.value.code == bsw.BSW_EINVAL
        got, cells = ctx.extend_host(bsw.HostBatch(wl))
        assert_same(got, ref, "large batch after errors")


def test_budget_too_small(bsw):
    wl, _, _ = workload_and_oracle("plain10k")
    with bsw.Context(wl.params, mem_budget_bytes=1 << 16) as ctx:
        with pytest.raises(bsw.BswError) as e:
            ctx.extend_host(bsw.HostBatch(wl))
        assert e.value.code == bsw.BSW_EBUDGET


def test_empty_batch_and_empty_sides(bsw):
    wl = W.from_lists([[], [0, 1], [], [2] * 40], [[1, 2], [], [], [2] * 50], [7, 9, 11, 13])
    ref, cells, _ = oracle.extend_batch(wl)
    got, gc = run(bsw, wl)
    assert_same(got, ref, "empty sides")
    assert gc == int(cells.sum())
    empty = W.from_lists([], [], [])
    got, gc = run(bsw, empty)
    assert got.shape == (0, 6) and gc == 0


def test_serving_each_request_same_alone_and_mixed(bsw):
    """Continuous batching: requests submitted together (merged into shared
    launches, overlapped across lanes) give exactly their results alone."""
    rng = np.random.default_rng(5)
    pools = [workload_and_oracle("read151", 200_000), workload_and_oracle("read250")]
    reqs = []
    for k in range(40):
        wl, ref, _ = pools[k % 2]
        size = int(rng.integers(1, 20000)) if k % 7 else int(rng.integers(30000, 50001))
        start = int(rng.integers(0, wl.n_pairs - size))
        idx = np.arange(start, start + size)
        reqs.append((wl.subset(idx), ref[idx]))
    with bsw.Context(pools[0][0].params, mem_budget_bytes=4 << 30) as ctx:
        tickets, outs, hbs = [], [], []
        for k, (sub, _) in enumerate(reqs):
            hb = bsw.HostBatch(sub)
            out = np.full((sub.n_pairs, 6), -7, np.int32)
            tickets.append(ctx.submit(hb, out, bsw.BSW_COPY_INPUTS if k % 3 == 0 else 0))
            outs.append(out)
            hbs.append(hb)
        for t in tickets:
            assert ctx.poll(t, 60_000_000) == bsw.BSW_OK
        assert ctx.poll(tickets[0], 0) == bsw.BSW_ENOTFOUND
        for (sub, ref), out, hb in zip(reqs, outs, hbs):
            assert_same(out, ref, "served request")
            alone, _ = ctx.extend_host(hb)
            np.testing.assert_array_equal(alone, out)


def test_serving_waits_for_memory(bsw):
    """A budget that holds one launch but not two: while one lane runs, the
    next admission is put back to wait for its memory (counted in the serving
    statistics), and every request still comes back with the oracle's results."""
    wl, ref, _ = workload_and_oracle("read151", 200_000)
    reqs = [np.arange(k * 40_000, (k + 1) * 40_000) for k in range(5)]
    hbs = [bsw.HostBatch(wl.subset(idx)) for idx in reqs]          # packed first: the submits come together
    outs = [np.full((idx.shape[0], 6), -7, np.int32) for idx in reqs]
    with bsw.Context(wl.params, mem_budget_bytes=30 << 20) as ctx:
        tickets = [ctx.submit(hb, out) for hb, out in zip(hbs, outs)]
        for t in tickets:
            assert ctx.poll(t, 120_000_000) == bsw.BSW_OK
        st = ctx.stream_stats()
        for idx, out in zip(reqs, outs):
            assert_same(out, ref[idx], "request served under a small budget")
    assert st["requests"] == len(reqs)
    assert st["budget_waits"] >= 1
    assert st["launches"] >= 2


def test_serving_launches_overlap(bsw):
    """Long-query requests larger than one merge run as several launches over
    the execution lanes; the statistics show their device intervals and that
    they overlapped, and every result is the oracle's."""
    wl, ref, _ = workload_and_oracle("long10k")
    rng = np.random.default_rng(8)
    idxs = [np.sort(rng.choice(wl.n_pairs, 2500, replace=False)) for _ in range(24)]
    hbs = [bsw.HostBatch(wl.subset(idx)) for idx in idxs]          # packed first: the submits come together
    outs = [np.full((idx.shape[0], 6), -7, np.int32) for idx in idxs]
    with bsw.Context(wl.params, mem_budget_bytes=8 << 30) as ctx:
        ctx.stream_stats(reset=True)
        tickets = [ctx.submit(hb, out) for hb, out in zip(hbs, outs)]
        for t in tickets:
            assert ctx.poll(t, 120_000_000) == bsw.BSW_OK
        st = ctx.stream_stats(reset=True)
        assert ctx.stream_stats()["requests"] == 0              # reset
    for idx, out in zip(idxs, outs):
        assert_same(out, ref[idx], "long request")
    assert st["requests"] == 24 and st["launches"] >= 2
    assert st["union_ms"] > 0 and st["busy_ms"] >= st["union_ms"] * 0.999
    assert st["max_concurrent"] >= 2, st


def test_serving_rejects_and_times_out(bsw):
    wl, _, _ = workload_and_oracle("plain10k")
    with bsw.Context(wl.params, mem_budget_bytes=1 << 16) as ctx:
        with pytest.raises(bsw.BswError) as e:
            ctx.submit(bsw.HostBatch(wl), np.zeros((wl.n_pairs, 6), np.int32))
        assert e.value.code == bsw.BSW_EBUDGET
    with bsw.Context(wl.params) as ctx:
        hb = bsw.HostBatch(wl)
        out = np.zeros((wl.n_pairs, 6), np.int32)
        t = ctx.submit(hb, out)
        rc = ctx.poll(t, 0)
        assert rc in (bsw.BSW_OK, bsw.BSW_PENDING)
        if rc == bsw.BSW_PENDING:
            assert ctx.poll(t, 60_000_000) == bsw.BSW_OK
        assert ctx.poll(12345678, 0) == bsw.BSW_ENOTFOUND


def test_maximum_query_length(bsw):
    """Queries of BSW_MAX_QLEN bases (band 500, the long-read parameters): a
    near-copy, an exact copy whose score leaves the 16-bit range (the 32-bit
    kernel), a query of that length against a 9 kbp target (score bound
    under the two-columns kernel's limit, columns up to the last) and a short
    pair beside them; one base more is rejected."""
    L = bsw.BSW_MAX_QLEN
    rng = np.random.default_rng(77)
    t = rng.integers(0, 4, L + 500).astype(np.uint8)
    near = t[:L].copy()
    flips = rng.random(L) < 0.05
    near[flips] = (near[flips] + 1) % 4
    params = W.Params(W.Scoring(), w=500, zdrop=400, end_bonus=5)
    wl = W.from_lists([near, t[:L], near, t[:50]], [t, t, t[:9000], t[:150]], [40, 40, 40, 20], params=params,
                      align=4)
    ref, cells, _ = oracle.extend_batch(wl, nthreads=NTH)
    assert ref[1][0] == 40 + L                        # the exact copy: h0 + L
    for flags in (0, "plain", "i32"):
        got, gc = run(bsw, wl, flag_of(bsw, flags), params=params)
        assert_same(got, ref, "max qlen/%s" % flags)
        assert gc == int(cells.sum())
    got, gc = run(bsw, wl, 0, params=params, cta_min=128)             # one pair per block
    assert_same(got, ref, "max qlen/block per pair")
    assert gc == int(cells.sum())
    for flags in (0, "plain"):                                         # two columns per instruction
        got, gc = run(bsw, wl, flag_of(bsw, flags), params=params, warp_x2=1)
        assert_same(got, ref, "max qlen/x2/%s" % flags)
        assert gc == int(cells.sum())
    too = W.from_lists([t[:L + 1]], [t], [40], params=params, align=4)
    with bsw.Context(params) as ctx:
        with pytest.raises(bsw.BswError) as e:
            ctx.extend_host(bsw.HostBatch(too))
        assert e.value.code == bsw.BSW_EINVAL
