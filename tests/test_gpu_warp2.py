"""The two-columns-per-instruction warp kernel against the oracle (needs a GPU).

The plan field warp_x2 sends the 16-bit warp-per-pair class to the kernel that
packs columns k and k + 4 of each 8-column granule into the halves of one
register.  It must give the oracle's results bit for bit wherever it runs:
band widths that give 1 to 4 granules per lane and several chunks per row,
rows ending on every column of a granule, bands just under the ring size,
every scoring it accepts, pairs above its score limit (re-run with 32-bit
lanes), per-pair bands wider than its ring, and the full long-query workload;
and as the plain baseline over pairs in input order.
"""
import numpy as np
import pytest

import oracle
from paper_1907_12931_gb300 import workload as W
from test_gpu_parity import NTH, adversarial, assert_same, workload_and_oracle

pytestmark = pytest.mark.gpu

X2 = {"short_max": 64, "warp_x2": 1}


@pytest.fixture(scope="module")
def bsw():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_12931_gb300 import bsw as _b
    _b.lib()
    return _b


def run_plan(bsw, wl, plan, flags=0, w_override=None):
    import torch
    with bsw.Context(wl.params, 16 << 30) as ctx:
        ctx.set_plan(bsw.make_plan(**plan))
        db = bsw.DeviceBatch(bsw.HostBatch(wl, w_override=w_override))
        ctx.extend_device(db, flags)
        ctx.sync()
        torch.cuda.synchronize()
        return db.out.cpu().numpy(), int(db.cells.item())


def check(bsw, wl, plan, what, w_override=None):
    ref, cells, _ = oracle.extend_batch(wl, nthreads=NTH, w_override=w_override)
    got, gc = run_plan(bsw, wl, plan, w_override=w_override)
    assert_same(got, ref, what)
    assert gc == int(cells.sum()), what


def mutated(rng, ref, n, err):
    """A query from ref[:n] with substitutions and 1-3 bp indels at rate err."""
    q, k, out = ref[:n], 0, []
    while k < len(q):
        u = rng.random()
        if u < err / 2:
            out.append(int((q[k] + 1 + rng.integers(0, 3)) % 4)); k += 1
        elif u < 3 * err / 4:
            k += int(rng.integers(1, 4))
        elif u < err:
            out.extend(int(x) for x in rng.integers(0, 4, int(rng.integers(1, 4))))
        else:
            out.append(int(q[k])); k += 1
    return np.array(out, np.uint8)


@pytest.mark.parametrize("config", ["long10k", "read250"])
def test_full_workloads(bsw, config):
    wl, ref, cells = workload_and_oracle(config)
    got, gc = run_plan(bsw, wl, X2)
    assert_same(got, ref, config + "/x2")
    assert gc == cells


@pytest.mark.parametrize("w", [3, 40, 100, 127, 128, 129, 250, 383, 384, 500, 508, 511, 1000, 1020, 1100])
def test_band_widths(bsw, w):
    """Bands of 1 to 4 granules per lane and of several chunks per row (over
    1024 columns), z-drop on and off, near copies and noisy queries."""
    rng = np.random.default_rng(2000 + w)
    qs, ts, hs = [], [], []
    for n in (65, 130, 300, 900, 2500, 4000):
        for err in (0.0, 0.02, 0.12):
            ref = rng.integers(0, 4, n + w + 600).astype(np.uint8)
            q = mutated(rng, ref, n, err)
            qs.append(q); ts.append(ref[: len(q) + w]); hs.append(int(rng.integers(19, 61)))
    wl = W.from_lists(qs, ts, hs, align=4)
    for zd in (100, 0):
        wl.params = W.Params(W.Scoring(), w=w, zdrop=zd, end_bonus=5)
        check(bsw, wl, X2, "x2 w=%d zdrop=%d" % (w, zd))


def test_granule_edges(bsw):
    """Query lengths around granule, 256-column and ring boundaries, so rows
    end on every column of a granule and at a chunk's last column."""
    rng = np.random.default_rng(77)
    qs, ts, hs = [], [], []
    lens = [65, 66, 71, 72, 73, 79, 80, 255, 256, 257, 263, 264, 511, 512, 513, 767, 768, 769, 1023, 1024, 1025,
            1031, 1032, 1033, 2047, 2048, 2049]
    for n in lens:
        ref = rng.integers(0, 4, 2 * n + 64).astype(np.uint8)
        for err, dm in ((0.0, 0), (0.01, 40), (0.05, n // 3), (0.0, -n // 2)):
            q = mutated(rng, ref, n, err)
            qs.append(q); ts.append(ref[: max(1, len(q) + dm)]); hs.append(int(rng.integers(0, 90)))
    wl = W.from_lists(qs, ts, hs, align=4)
    for w in (100, 255, 256, 600):
        wl.params = W.Params(W.Scoring(), w=w, zdrop=100, end_bonus=5)
        check(bsw, wl, X2, "x2 granule edges w=%d" % w)


def test_ring_wrap_band_edges(bsw):
    """Full-width bands just under a power of two (near-identical sequences):
    the last chunk's out-of-band granules reach furthest past the band there
    and must never read a band column through the ring's wrap."""
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
    for w in (120, 123, 124, 126, 127, 252, 254, 255, 500, 504, 508, 510, 511, 1016, 1020):
        wl.params = W.Params(W.Scoring(), w=w, zdrop=0, end_bonus=5)
        check(bsw, wl, X2, "x2 ring edges w=%d" % w)


@pytest.mark.parametrize("sc", [(1, 4, 6, 1, 6, 1), (2, 3, 5, 2, 4, 1), (1, 6, 1, 1, 1, 1), (3, 9, 3, 3, 8, 2),
                                (1, 4, 6, 2, 6, 2), (2, 1, 0, 1, 0, 1), (1, 1, 2, 3, 1, 2)])
def test_scorings(bsw, sc):
    """Match 1 to 3 (zero-rule shift 1 or 2), asymmetric gap costs and
    extensions above 1 (the general variant without a shared M - o - e)."""
    wl = W.make("long10k", n_pairs=500)
    wl.params = W.Params(W.Scoring(*sc), w=300, zdrop=200, end_bonus=3)
    check(bsw, wl, X2, "x2 scoring %s" % (sc,))


def test_unsupported_match_falls_back(bsw):
    """Match above 3 keeps the int2 ring kernel (warp_x2 does not apply)."""
    wl = W.make("long10k", n_pairs=300)
    wl.params = W.Params(W.Scoring(5, 9, 3, 3, 8, 2), w=300, zdrop=200, end_bonus=3)
    check(bsw, wl, X2, "x2 plan, match 5")


def test_score_limit_reruns(bsw):
    """Pairs whose score bound reaches 2^14 (match 1) or 2^13 (match 2 and 3)
    take the 32-bit re-run, the rest stay; both exact, including pairs right
    at the limit."""
    rng = np.random.default_rng(5)
    for sc, lim in (((1, 4, 6, 1, 6, 1), 1 << 14), ((2, 4, 6, 1, 6, 1), 1 << 13)):
        a = sc[0]
        qs, ts, hs = [], [], []
        for n in (300, 1200, 3000):
            ref = rng.integers(0, 4, n + 300).astype(np.uint8)
            q = mutated(rng, ref, n, 0.02)
            for h0 in (lim - 1 - a * len(q), lim - a * len(q), lim + 5 - a * len(q), 10, 4000):
                if 0 <= h0 < 30000:
                    qs.append(q); ts.append(ref[: len(q) + 200]); hs.append(int(h0))
        wl = W.from_lists(qs, ts, hs, align=4)
        wl.params = W.Params(W.Scoring(*sc), w=150, zdrop=100, end_bonus=5)
        check(bsw, wl, X2, "x2 score limit %s" % (sc,))


def test_band_override(bsw):
    """Per-pair bands wider than the context's ring go to the re-run list;
    narrower ones stay in the kernel."""
    wl = W.make("long10k", n_pairs=500)
    k = np.arange(wl.n_pairs) % 4
    ws = np.select([k == 0, k == 1, k == 2], [1500, 50, 7], 500).astype(np.int32)
    check(bsw, wl, X2, "x2 band overrides", w_override=ws)


@pytest.mark.parametrize("zdrop", [100, 0, 1, 7])
def test_adversarial(bsw, zdrop):
    wl, ws = adversarial()
    wl.params = W.Params(W.Scoring(), w=100, zdrop=zdrop, end_bonus=5)
    check(bsw, wl, X2, "x2 adversarial zdrop=%d" % zdrop, w_override=ws)


def test_plan_roundtrip_and_bad_values(bsw):
    wl = W.make("plain10k", n_pairs=100)
    with bsw.Context(wl.params, 1 << 30) as ctx:
        ctx.set_plan(bsw.make_plan(warp_x2=1))
        assert ctx.get_plan().warp_x2 == 1
        for bad in (2, -1):
            with pytest.raises(bsw.BswError):
                ctx.set_plan(bsw.make_plan(warp_x2=bad))
        assert ctx.get_plan().warp_x2 == 1


@pytest.mark.parametrize("config", ["long10k", "read250", "plain10k"])
def test_plain_kernel(bsw, config):
    """The plain baseline with the two-columns kernel (pairs in input order;
    pairs it cannot take run in the 32-bit kernel afterwards)."""
    wl, ref, cells = workload_and_oracle(config)
    got, gc = run_plan(bsw, wl, {"warp_x2": 1}, flags=bsw.BSW_PLAIN_KERNEL)
    assert_same(got, ref, config + "/plain x2")
    assert gc == cells


def test_plain_kernel_leftovers(bsw):
    """Pairs the plain two-columns kernel leaves to the 32-bit kernel: N
    bases, score bounds at its limit, bands wider than its ring, empty sides
    (answered in place) and the adversarial set's band widths."""
    from test_gpu_nbase import hand_cases
    hc = hand_cases()
    ref, cells, _ = oracle.extend_batch(hc, nthreads=NTH)
    got, gc = run_plan(bsw, hc, {"warp_x2": 1}, flags=bsw.BSW_PLAIN_KERNEL)
    assert_same(got, ref, "plain x2, N hand cases")
    assert gc == int(cells.sum())
    wl, ws = adversarial()
    wl.params = W.Params(W.Scoring(), w=100, zdrop=100, end_bonus=5)
    ref, cells, _ = oracle.extend_batch(wl, nthreads=NTH, w_override=ws)
    got, gc = run_plan(bsw, wl, {"warp_x2": 1}, flags=bsw.BSW_PLAIN_KERNEL, w_override=ws)
    assert_same(got, ref, "plain x2, adversarial")
    assert gc == int(cells.sum())
