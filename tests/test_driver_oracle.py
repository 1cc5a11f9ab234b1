"""Pins of the seed-extension driver oracle (oracle/driver.py), no GPU.

Each expected value below is worked out by hand from the readings D1-D5 in
the oracle's header and the extension's definition (Eq. 2, Eq. 3, rules a-c):
with match 1, mismatch 4, gaps 6+1k, end bonus 5."""
import numpy as np
import pytest

import oracle
from oracle import driver
from paper_1907_12931_gb300 import workload as W

P = W.Params(W.Scoring(), w=100, zdrop=100, end_bonus=5)


def _ref(n, seed=5):
    return W.random_codes(seed, n)


def _one(reads, ref, seeds, params=P, tries=2):
    sw = W.seeds_from_lists(reads, ref, seeds, params=params)
    return driver.extend_seeds(sw, params=params, max_band_try=tries)


def test_exact_read_extends_to_both_ends():
    ref = _ref(2000)
    p = 700
    read = ref[p:p + 40].copy()
    out = _one([read], ref, [(0, 10, 20, p + 10)])
    # left: 10 matches from h0 = 20 reach the read start: gscore 30 > score - 5
    # right: 10 matches from 30 reach the read end: 40
    assert (out["qb"][0], out["qe"][0], out["rb"][0], out["re"][0], out["score"][0]) == (0, 40, p, p + 40, 40)
    assert out["kept"][0] == 1 and out["w_left"][0] == 100 and out["w_right"][0] == 100


def test_n_in_read_and_reference():
    """R11 inside the driver.  Seed [0, 20) at p, so the left side is empty
    and the right side starts from h0 = 20 with 20 query bases.  An N at read
    position 30 costs 1 instead of the mismatch's 4: 20 + 10 - 1 + 9 = 38, and
    the extension still reaches the read end (38 > 33).  An N in the
    reference opposite read position 35 gives the same 38; both together
    give 36; an N run of 8 reference bases opposite read positions 25-32
    gives 20 + 5 - 8 + 7 = 24 at the read end against a local best of 25 at
    read position 25: 24 > 25 - 5, so the read end is kept."""
    ref = _ref(2000, seed=9)
    p = 500
    read = ref[p:p + 40].copy()
    a = read.copy(); a[30] = 4
    out = _one([a], ref, [(0, 0, 20, p)])
    assert (out["qb"][0], out["qe"][0], out["rb"][0], out["re"][0], out["score"][0]) == (0, 40, p, p + 40, 38)
    r2 = ref.copy(); r2[p + 35] = 4
    out = _one([read], r2, [(0, 0, 20, p)])
    assert (out["qe"][0], out["re"][0], out["score"][0]) == (40, p + 40, 38)
    out = _one([a], r2, [(0, 0, 20, p)])
    assert (out["qe"][0], out["re"][0], out["score"][0]) == (40, p + 40, 36)
    r3 = ref.copy(); r3[p + 25:p + 33] = 4
    out = _one([read], r3, [(0, 0, 20, p)])
    assert (out["qe"][0], out["re"][0], out["score"][0]) == (40, p + 40, 24)


def test_end_mismatches_clip_or_extend():
    ref = _ref(2000, seed=6)
    p = 300
    read = ref[p:p + 40].copy()
    one = read.copy()
    one[39] = (one[39] + 1) % 4
    # one mismatch at the end: local best 39 at column 38, reaching the end
    # gives 39 - 4 = 35 > 39 - 5, so the read end is taken with score 35
    out = _one([one], ref, [(0, 0, 20, p)])
    assert (out["qb"][0], out["qe"][0], out["re"][0], out["score"][0]) == (0, 40, p + 40, 35)
    two = read.copy()
    two[38] = (two[38] + 1) % 4
    two[39] = (two[39] + 1) % 4
    # two mismatches: the end gives 38 - 8 = 30 <= 38 - 5, so the local best
    # (38 at read position 38) is kept
    out = _one([two], ref, [(0, 0, 20, p)])
    assert (out["qb"][0], out["qe"][0], out["re"][0], out["score"][0]) == (0, 38, p + 38, 38)


def test_seed_at_read_start_and_reference_start():
    ref = _ref(500, seed=7)
    read = ref[0:30].copy()
    # seed at read start: no left query (w_left 0); at reference start: the
    # left side has no target either
    out = _one([read], ref, [(0, 0, 20, 0)])
    assert (out["qb"][0], out["rb"][0], out["qe"][0], out["score"][0], out["w_left"][0]) == (0, 0, 30, 30, 0)
    # a seed inside the read at reference start: empty left target, so the
    # left side stays at the seed (gscore -1 keeps the local best)
    read2 = np.concatenate([_ref(5, seed=8), ref[0:30]])
    out = _one([read2], ref, [(0, 5, 20, 0)])
    assert (out["qb"][0], out["rb"][0], out["qe"][0], out["score"][0]) == (5, 0, 35, 30)


def test_post_filter_drops_covered_seeds():
    ref = _ref(3000, seed=9)
    p = 1000
    read = ref[p:p + 60].copy()
    other = ref[2000:2060].copy()
    seeds = [(0, 5, 20, p + 5), (0, 30, 20, p + 30), (1, 10, 25, 2010)]
    out = _one([read, other], ref, seeds)
    # the first seed's alignment covers the whole read, so the second seed is
    # covered; the other read's seed is kept
    assert list(out["kept"]) == [1, 0, 1]
    assert (out["qb"][1], out["qe"][1], out["score"][1]) == (0, 60, 60)


def test_band_retry_matches_the_wider_band():
    # right side with a 4-base and later a 2-base deletion from the read: with
    # w = 4 the best path leaves the diagonal by 4 >= (4 >> 1) + (4 >> 2) = 3
    # but cannot follow the second deletion; the extension is rerun with w = 8,
    # which can, and the result must equal one extension with w = 8
    ref = _ref(4000, seed=10)
    p = 1500
    read = np.concatenate([ref[p:p + 30], ref[p + 34:p + 64], ref[p + 66:p + 100]])
    params = W.Params(W.Scoring(), w=4, zdrop=100, end_bonus=5)
    out = _one([read], ref, [(0, 0, 20, p)], params=params)
    q = read[20:]
    t = ref[p + 20:p + 20 + len(q) + 4]   # D1: query length + w, w = 4
    r8 = oracle.extend_one(params, q, t, 20, w=8)[0]
    r4 = oracle.extend_one(params, q, t, 20, w=4)[0]
    assert r4["max_off"] >= 3 and r4 != r8
    assert out["w_right"][0] == 8
    local = r8["gscore"] <= 0 or r8["gscore"] <= r8["score"] - 5
    assert out["qe"][0] == 20 + (r8["qle"] if local else len(q))
    assert out["score"][0] == (r8["score"] if local else r8["gscore"])
    # one try only: the w = 4 result stands
    out1 = _one([read], ref, [(0, 0, 20, p)], params=params, tries=1)
    assert out1["w_right"][0] == 4
    local4 = r4["gscore"] <= 0 or r4["gscore"] <= r4["score"] - 5
    assert out1["score"][0] == (r4["score"] if local4 else r4["gscore"])


def test_generated_seeds_invariants():
    sw = W.make_seeds("seeds151", n_reads=400)
    out = driver.extend_seeds(sw, nthreads=4)
    q0, L, r0 = sw.qbeg, sw.slen, sw.rbeg
    assert np.all(out["qb"] <= q0) and np.all(out["qe"] >= q0 + L)
    assert np.all(out["rb"] <= r0) and np.all(out["re"] >= r0 + L)
    assert np.all(out["qb"] >= 0) and np.all(out["qe"] <= sw.read_len[sw.seed_read])
    # the first seed of every read is kept
    first = np.r_[True, sw.seed_read[1:] != sw.seed_read[:-1]]
    assert np.all(out["kept"][first] == 1)
    # most seeds of a 1%-error read extend to the whole read
    assert np.mean((out["qb"] == 0) & (out["qe"] == 151)) > 0.5
