"""The 8-bit row-pair scheme against the oracle, on the host (no GPU).

`rowpair_model.extend` restates the kernel's two-rows-per-instruction pass
bit by bit (packed instructions emulated on 32-bit words).  These tests pin
the scheme itself: every result field and the cell count equal the oracle's
for random pairs under symmetric and split gap costs, match scores 1 to 3
and bands of 0 to 100 columns; for pairs whose rows read slots past the
previous row's end (the oracle counts those reads); and for every row count
from 1 to 9.  The GPU tests in `test_gpu_rowpair.py` check the kernel on the
same kinds of input.
"""
import numpy as np
import pytest

import oracle
import rowpair_model
from paper_1907_12931_gb300 import workload as W


def random_case(rng):
    a = int(rng.integers(1, 4))
    b = int(rng.integers(1, 6))
    od, ed = int(rng.integers(0, 8)), int(rng.integers(1, 3))
    oi, ei = (od, ed) if rng.random() < 0.5 else (int(rng.integers(0, 8)), int(rng.integers(1, 3)))
    n, m = int(rng.integers(1, 61)), int(rng.integers(1, 91))
    ref = rng.integers(0, 4, n + m + 10)
    q = ref[:n].copy()
    flip = rng.random(n) < rng.choice([0.0, 0.02, 0.1, 0.4])
    q[flip] = rng.integers(0, 4, int(flip.sum()))
    off = int(rng.integers(0, 6))
    t = ref[off:off + m].copy() if rng.random() < 0.7 else rng.integers(0, 4, m)
    left = 255 - a * min(n, m)
    h0 = int(rng.integers(0, min(left, 120) + 1)) if left >= 0 else None
    params = W.Params(W.Scoring(a, b, od, ed, oi, ei), w=int(rng.choice([0, 1, 2, 3, 5, 10, 30, 100])),
                      zdrop=int(rng.choice([0, 1, 5, 20, 100])), end_bonus=int(rng.integers(0, 8)))
    return params, q.astype(np.uint8), t.astype(np.uint8), h0


def same(params, q, t, h0, what):
    ref, cells, stale = oracle.extend_one(params, q, t, h0)
    got, gc = rowpair_model.extend(params, q, t, h0)
    assert got == ref and gc == cells, (what, len(q), len(t), h0, params, ref, cells, got, gc)
    return stale


@pytest.mark.parametrize("seed", range(4))
def test_random_pairs(seed):
    rng = np.random.default_rng(900 + seed)
    done = 0
    while done < 400:
        params, q, t, h0 = random_case(rng)
        if h0 is None:
            continue
        same(params, q, t, h0, "random %d" % seed)
        done += 1


def test_stale_slot_reads():
    """Narrow bands and large h0 over near copies: rows whose band end grows
    by two columns read slots an earlier row wrote."""
    rng = np.random.default_rng(77)
    with_stale = tries = 0
    while with_stale < 60 and tries < 60000:
        tries += 1
        a = int(rng.integers(1, 4))
        n, m = int(rng.integers(2, 50)), int(rng.integers(2, 60))
        q = rng.integers(0, 4, n).astype(np.uint8)
        t = (q[rng.integers(0, n, m)] if rng.random() < 0.5 else rng.integers(0, 4, m)).astype(np.uint8)
        left = 255 - a * min(n, m)
        if left < 0:
            continue
        h0 = int(rng.integers(0, min(left, 80) + 1))
        od, ed = int(rng.integers(0, 6)), int(rng.integers(1, 3))
        params = W.Params(W.Scoring(a, int(rng.integers(1, 6)), od, ed, od, ed),
                          w=int(rng.choice([1, 2, 3, 5, 8])), zdrop=int(rng.choice([0, 3, 30])),
                          end_bonus=int(rng.integers(0, 6)))
        ref, cells, stale = oracle.extend_one(params, q, t, h0)
        if stale == 0:
            continue
        with_stale += 1
        same(params, q, t, h0, "stale")
    assert with_stale >= 60, with_stale


def test_row_counts():
    """Target lengths 1 to 9 (the last row alone when odd) against queries
    of 1 to 12 bases."""
    rng = np.random.default_rng(3)
    for m in range(1, 10):
        for n in range(1, 13):
            for h0 in (0, 1, 7, 30, 200):
                if h0 + min(n, m) > 255:
                    continue
                q = rng.integers(0, 4, n).astype(np.uint8)
                t = np.where(rng.random(m) < 0.8, np.resize(q, m), rng.integers(0, 4, m)).astype(np.uint8)
                for w in (0, 1, 2, 100):
                    same(W.Params(W.Scoring(), w=w, zdrop=1, end_bonus=5), q, t, h0, "rows")


def test_packed_helpers():
    """The emulated packed instructions act on each 16-bit half alone."""
    m = rowpair_model
    for lo_a, hi_a, lo_b, hi_b, lo_c, hi_c in [(5, -3, 2, 7, 4, -9), (-100, 200, 50, -50, 0, 0), (255, 0, 3, -4, 256, 1)]:
        a, b, c = m.pack(lo_a, hi_a), m.pack(lo_b, hi_b), m.pack(lo_c, hi_c)
        assert m.viaddmin_s16x2(a, b, c) == m.pack(min(lo_a + lo_b, lo_c), min(hi_a + hi_b, hi_c))
        assert m.viaddmax_s16x2_relu(a, b, c) == m.pack(max(lo_a + lo_b, lo_c, 0), max(hi_a + hi_b, hi_c, 0))
        assert m.vimax3_s16x2(a, b, c) == m.pack(max(lo_a, lo_b, lo_c), max(hi_a, hi_b, hi_c))
    # the selector of slot j gives s(t_i, q_j) low and s(t_{i+1}, q_{j-1}) high, sign-extended
    prof0, prof1 = 0x01FCFCFC, 0xFCFC01FC        # row i: base 3 matches; row i+1: base 1
    for qj in range(4):
        for qjm in range(4):
            sel = qj * 0x11 + qjm * 0x1100 + 0xC480
            r = m.prmt(prof0, prof1, sel)
            assert m.lo16(r) == (1 if qj == 3 else -4) and m.hi16(r) == (1 if qjm == 1 else -4)
