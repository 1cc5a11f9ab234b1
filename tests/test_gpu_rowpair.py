"""The 8-bit per-thread kernel's row pairs against the oracle (needs a GPU).

Pairs of the 8-bit classes without N bases run two rows per packed
instruction: rows i and i+1, one column apart, with row i+1's band ends taken
from row i once row i has ended (its start before the packed loop, its end
from the last column where row i's H is positive).  The cases here aim at
that logic: odd and even row counts down to one row, rows whose band end
moves back by several columns (a tail of zeros in row i), reads of slots past
the previous row's end that still hold values of earlier rows, band clips of
one to a few columns, every gap-cost split, match scores that change the
zero-diagonal shift, and score bounds either side of 255 (above it the pair
goes to the 16-bit class).  Every comparison is bit-exact on all six
result fields and the cell count.
"""
import numpy as np
import pytest

import oracle
from paper_1907_12931_gb300 import workload as W
from test_gpu_parity import NTH, assert_same, run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bsw():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_12931_gb300 import bsw as _b
    _b.lib()
    return _b


def random_pairs(rng, count, nmax, mmax, match, h0_cap=120):
    """Query/target pairs: near copies at several error rates, unrelated
    targets, and h0 within the 8-bit bound h0 + match * min(n, m) <= 255."""
    qs, ts, hs = [], [], []
    while len(qs) < count:
        n = int(rng.integers(1, nmax + 1))
        m = int(rng.integers(1, mmax + 1))
        left = 255 - match * min(n, m)
        if left < 0:
            continue
        ref = rng.integers(0, 4, n + m + 10)
        q = ref[:n].copy()
        err = rng.choice([0.0, 0.02, 0.1, 0.4])
        flip = rng.random(n) < err
        q[flip] = rng.integers(0, 4, int(flip.sum()))
        off = int(rng.integers(0, 6))
        t = ref[off:off + m].copy() if rng.random() < 0.7 else rng.integers(0, 4, m)
        if len(t) < m:
            t = np.concatenate([t, rng.integers(0, 4, m - len(t))])
        qs.append(q.astype(np.uint8))
        ts.append(t.astype(np.uint8))
        hs.append(int(rng.integers(0, min(left, h0_cap) + 1)))
    return qs, ts, hs


def check(bsw, wl, what):
    ref, cells, stale = oracle.extend_batch(wl, nthreads=NTH)
    got, gc = run(bsw, wl, device=True)
    assert_same(got, ref, what)
    assert gc == int(cells.sum()), what
    return stale


SCORINGS = [
    ((1, 4, 6, 1, 6, 1), 100, 100, 5),
    ((1, 4, 6, 1, 6, 1), 3, 0, 0),
    ((2, 3, 5, 2, 4, 1), 8, 20, 3),
    ((3, 5, 0, 2, 0, 2), 1, 5, 4),
    ((1, 1, 1, 1, 2, 2), 20, 1, 2),
    ((2, 1, 0, 1, 3, 1), 2, 0, 6),
    ((1, 2, 0, 1, 0, 1), 5, 30, 1),
]


@pytest.mark.parametrize("k", range(len(SCORINGS)))
def test_random_pairs(bsw, k):
    """Symmetric and split gap costs, match 1 to 3, bands of 1 to 100."""
    sc, w, zd, eb = SCORINGS[k]
    rng = np.random.default_rng(300 + k)
    qs, ts, hs = random_pairs(rng, 3000, 60, 90, sc[0])
    wl = W.from_lists(qs, ts, hs, W.Params(W.Scoring(*sc), w=w, zdrop=zd, end_bonus=eb), align=4)
    check(bsw, wl, "row pairs %s w=%d zdrop=%d" % (sc, w, zd))


@pytest.mark.parametrize("w", [1, 2, 3, 5, 8])
def test_stale_slot_reads(bsw, w):
    """Narrow bands over near copies with large h0: the band end grows by two
    columns past the previous row's, so rows read slots that an earlier row
    wrote.  The oracle counts those reads; the batch must hold many."""
    rng = np.random.default_rng(40 + w)
    qs, ts, hs = [], [], []
    for _ in range(4000):
        n, m = int(rng.integers(2, 50)), int(rng.integers(2, 60))
        q = rng.integers(0, 4, n)
        t = q[rng.integers(0, n, m)] if rng.random() < 0.5 else rng.integers(0, 4, m)
        qs.append(q.astype(np.uint8)); ts.append(t.astype(np.uint8))
        hs.append(int(rng.integers(0, min(255 - min(n, m), 80) + 1)))
    with_stale = 0
    for sc in ((1, 4, 6, 1, 6, 1), (1, 2, 0, 1, 0, 1), (2, 3, 1, 2, 4, 1)):
        hs2 = [min(h, 255 - sc[0] * min(len(q), len(t))) for h, q, t in zip(hs, qs, ts)]
        wl = W.from_lists(qs, ts, hs2, W.Params(W.Scoring(*sc), w=w, zdrop=30, end_bonus=3), align=4)
        stale = check(bsw, wl, "stale reads w=%d %s" % (w, sc))
        with_stale += int((stale > 0).sum())
    assert with_stale >= 20, with_stale


def test_row_counts(bsw):
    """Every target length from 1 to 9 (the last row alone when odd) against
    query lengths 1 to 12, at several h0 and band widths."""
    rng = np.random.default_rng(9)
    qs, ts, hs = [], [], []
    for m in range(1, 10):
        for n in range(1, 13):
            for h0 in (0, 1, 7, 30, 200):
                if h0 + min(n, m) > 255:
                    continue
                q = rng.integers(0, 4, n).astype(np.uint8)
                t = np.where(rng.random(m) < 0.8, np.resize(q, m), rng.integers(0, 4, m)).astype(np.uint8)
                qs.append(q); ts.append(t); hs.append(h0)
    for w in (0, 1, 2, 100):
        for zd in (100, 1):
            wl = W.from_lists(qs, ts, hs, W.Params(W.Scoring(), w=w, zdrop=zd, end_bonus=5), align=4)
            check(bsw, wl, "row counts w=%d zdrop=%d" % (w, zd))


def test_score_bound_edges(bsw):
    """h0 + match * min(n, m) at 254, 255 (row pairs) and 256, 257 (the
    16-bit class), including 256-base queries whose row key holds column
    255."""
    rng = np.random.default_rng(12)
    for a in (1, 2):
        qs, ts, hs = [], [], []
        for n in (40, 100, 127, 200, 256):
            for m in (n - 1, n, n + 30):
                ref = rng.integers(0, 4, max(n, m) + 5)
                q = ref[:n].astype(np.uint8)
                t = ref[:m].astype(np.uint8)
                for d in (-1, 0, 1, 2):
                    h0 = 255 - a * min(n, m) + d
                    if 0 <= h0:
                        qs.append(q); ts.append(t); hs.append(h0)
        wl = W.from_lists(qs, ts, hs, W.Params(W.Scoring(a, 4, 6, 1, 6, 1), w=100, zdrop=100, end_bonus=5), align=4)
        check(bsw, wl, "bound edges match %d" % a)
