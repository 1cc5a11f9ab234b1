"""Pins for the CPU oracle (no GPU).

The oracle is checked against things fixed independently of it: hand-worked
examples (tests/golden), closed forms of the method, an independent
full-matrix brute-force DP on tiny inputs, and invariants.
"""
import itertools
import os

import numpy as np
import pytest

import oracle
from oracle import brute
from paper_1907_12931_gb300 import workload as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_worked.txt")
P = W.Params()


def grid_workload(Q, T, H0, params=P):
    """Pairs with equal shapes: Q [B, n], T [B, m] -> Workload (offsets multiple of 4)."""
    Q = np.asarray(Q, np.uint8)
    T = np.asarray(T, np.uint8)
    B, n = Q.shape
    m = T.shape[1]
    sn, sm = max(4, (n + 3) // 4 * 4), max(4, (m + 3) // 4 * 4)
    q = np.zeros((B, sn), np.uint8)
    q[:, :n] = Q
    t = np.zeros((B, sm), np.uint8)
    t[:, :m] = T
    return W.Workload("grid", params, q.reshape(-1), np.arange(B, dtype=np.int64) * sn,
                      np.full(B, n, np.int32), t.reshape(-1), np.arange(B, dtype=np.int64) * sm,
                      np.full(B, m, np.int32), np.asarray(H0, np.int32))


def read_golden():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        head, res, cells = [x.split() for x in line.split("|")]
        name, q, t, h0, w, zd, eb = head
        q = "" if q == "-" else q
        t = "" if t == "-" else t
        rows.append((name, q, t, int(h0), int(w), int(zd), int(eb), [int(x) for x in res], int(cells[0])))
    return rows


@pytest.mark.parametrize("row", read_golden(), ids=lambda r: r[0])
def test_hand_worked(row):
    name, q, t, h0, w, zd, eb, expect, cells = row
    params = W.Params(W.Scoring(), w=w, zdrop=zd, end_bonus=eb)
    res, ncell, _ = oracle.extend_one(params, W.encode(q) if q else np.zeros(0, np.uint8),
                                      W.encode(t) if t else np.zeros(0, np.uint8), h0)
    assert [res[k] for k in oracle.FIELDS] == expect
    assert ncell == cells


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("L", [1, 2, 5, 17, 64, 130, 300])
@pytest.mark.parametrize("extra", [0, 7, 120])
def test_identical_prefix(L, extra):
    """q equal to the first L bases of t: the diagonal is the only best path,
    so the extension takes all of q with score h0 + match*L."""
    rng = np.random.default_rng(L * 1000 + extra)
    t = rng.integers(0, 4, L + extra).astype(np.uint8)
    q = t[:L].copy()
    for s in [W.Scoring(), W.Scoring(2, 3, 5, 2, 4, 1)]:
        params = W.Params(s, w=max(L, 1) + 5, zdrop=0, end_bonus=5)
        h0 = 30
        res, _, _ = oracle.extend_one(params, q, t, h0)
        full = h0 + s.match * L
        assert res == dict(score=full, qle=L, tle=L, gtle=L, gscore=full, max_off=0)


@pytest.mark.parametrize("seed", range(20))
def test_all_mismatch(seed):
    """No query base equals any target base: every M is below its diagonal, so
    no cell ever exceeds h0 and the best stays at the seed."""
    rng = np.random.default_rng(seed)
    qb = rng.integers(0, 4)
    n, m = rng.integers(1, 60), rng.integers(1, 90)
    q = np.full(n, qb, np.uint8)
    t = ((qb + rng.integers(1, 4, m)) % 4).astype(np.uint8)
    h0 = int(rng.integers(1, 80))
    res, _, _ = oracle.extend_one(P, q, t, h0)
    assert (res["score"], res["qle"], res["tle"], res["max_off"]) == (h0, 0, 0, 0)
    assert res["gscore"] < h0


@pytest.mark.parametrize("n", [1, 3, 40, 101])
def test_zero_seed_score(n):
    """h0 = 0: the first row of Eq. 3 is all zero, every diagonal is zero, so
    row 0 is all zero; when the band reaches the query end, gscore = 0 at
    row 0 and the sweep stops there."""
    rng = np.random.default_rng(n)
    q = rng.integers(0, 4, n).astype(np.uint8)
    t = rng.integers(0, 4, n + 10).astype(np.uint8)
    params = W.Params(W.Scoring(), w=n + 1, zdrop=100, end_bonus=5)
    res, cells, _ = oracle.extend_one(params, q, t, 0)
    assert res == dict(score=0, qle=0, tle=0, gtle=1, gscore=0, max_off=0)
    assert cells == n


def test_band_clip_values():
    """R1: trunc((n*a + end_bonus - o)/e + 1), at least 1, then min with w."""
    assert oracle.band_width(P, 4) == 4            # (4 + 5 - 6)/1 + 1
    assert oracle.band_width(P, 130) == 100        # w binds
    assert oracle.band_width(P, 1) == 1            # (1 + 5 - 6) + 1 = 1
    s = W.Scoring(1, 4, 6, 3, 6, 2)
    p = W.Params(s, w=100, zdrop=100, end_bonus=0)
    # ins: (10 - 6)/2 + 1 = 3 ; del: (10 - 6)/3 + 1 = 2.33 -> 2
    assert oracle.band_width(p, 10) == 2
    # negative numerator truncates toward zero, then the floor of 1 applies
    assert oracle.band_width(p, 1) == 1
    for n in range(0, 300):
        for w in (1, 7, 100, 500):
            assert oracle.band_width(P, n, w) == brute.band_clip(n, w, 1, 5, 6, 1, 6, 1)


# ---------------------------------------------------------------- brute force

def _oracle_grid(Q, T, H0, flags, params=P):
    wl = grid_workload(Q, T, H0, params)
    res, cells, stale = oracle.extend_batch(wl, flags=flags, nthreads=4)
    return res, cells, stale


def test_brute_exhaustive_4x4():
    """Every pair of 4-base sequences, no band/trim/z-drop: the one-row sweep
    equals the full-matrix DP (pins the in-place row bookkeeping and Eq. 3)."""
    allseq = np.array(list(itertools.product(range(4), repeat=4)), np.uint8)
    Q = np.repeat(allseq, len(allseq), axis=0)
    T = np.tile(allseq, (len(allseq), 1))
    for h0 in (0, 3, 7, 12):
        H0 = np.full(len(Q), h0, np.int32)
        got, _, _ = _oracle_grid(Q, T, H0, oracle.NO_BAND | oracle.NO_TRIM | oracle.NO_ZDROP)
        ref = brute.extend_full(P, Q, T, H0)
        np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("n,m", [(1, 1), (1, 8), (8, 1), (3, 5), (5, 3), (6, 8), (8, 8), (2, 7)])
def test_brute_random_small(n, m):
    rng = np.random.default_rng(n * 31 + m)
    B = 4000
    Q = rng.integers(0, 4, (B, n))
    T = rng.integers(0, 4, (B, m))
    # read-like: half the targets copy the query with a few substitutions
    half = B // 2
    k = min(n, m)
    T[:half, :k] = Q[:half, :k]
    flip = rng.random((half, k)) < 0.15
    T[:half, :k] = np.where(flip, (T[:half, :k] + 1) % 4, T[:half, :k])
    H0 = rng.integers(0, 20, B)
    for sc in (W.Scoring(), W.Scoring(2, 3, 2, 1, 3, 2)):
        params = W.Params(sc, w=100, zdrop=100, end_bonus=5)
        got, _, _ = _oracle_grid(Q, T, H0, oracle.NO_BAND | oracle.NO_TRIM | oracle.NO_ZDROP, params)
        np.testing.assert_array_equal(got, brute.extend_full(params, Q, T, H0))


@pytest.mark.parametrize("w", [0, 1, 2, 3])
def test_brute_static_band(w):
    """Band on, trim off: equals the full-matrix DP restricted to |i - j| <= w'."""
    rng = np.random.default_rng(100 + w)
    for n, m in [(6, 8), (8, 6), (8, 8), (3, 8)]:
        B = 3000
        Q = rng.integers(0, 4, (B, n))
        T = rng.integers(0, 4, (B, m))
        T[: B // 2, :min(n, m)] = Q[: B // 2, :min(n, m)]
        H0 = rng.integers(0, 25, B)
        params = W.Params(W.Scoring(), w=w, zdrop=100, end_bonus=5)
        got, _, _ = _oracle_grid(Q, T, H0, oracle.NO_TRIM | oracle.NO_ZDROP, params)
        np.testing.assert_array_equal(got, brute.extend_full(params, Q, T, H0, band=True))


@pytest.mark.parametrize("zd", [1, 2, 4, 8])
def test_brute_zdrop(zd):
    """z-drop (R5) on a banded, untrimmed sweep equals the brute force with the
    same row rule; small thresholds so that it fires often."""
    rng = np.random.default_rng(200 + zd)
    n, m = 8, 8
    B = 5000
    Q = rng.integers(0, 4, (B, n))
    T = rng.integers(0, 4, (B, m))
    T[: B // 2] = Q[: B // 2]
    T[: B // 2, 3] = (T[: B // 2, 3] + 1) % 4
    H0 = rng.integers(5, 25, B)
    sc = W.Scoring(1, 4, 3, 1, 2, 2)
    params = W.Params(sc, w=3, zdrop=zd, end_bonus=5)
    got, _, _ = _oracle_grid(Q, T, H0, oracle.NO_TRIM, params)
    ref = brute.extend_full(params, Q, T, H0, band=True, zdrop=True)
    np.testing.assert_array_equal(got, ref)
    # z-drop fired on some pairs (the comparison is not vacuous)
    nozd = brute.extend_full(params, Q, T, H0, band=True, zdrop=False)
    assert (nozd != ref).any()


def test_trim_never_raises_score():
    """With rule c on, cells cut from the band count as zero, and every value
    in Eq. 2 is monotone in its inputs (M is monotone once clamped at 0), so the
    trimmed score never exceeds the full DP's -- unless a read of a row entry
    left by an earlier row (R6) brings in a larger value, which the oracle counts."""
    rng = np.random.default_rng(7)
    n, m = 8, 8
    B = 20000
    Q = rng.integers(0, 4, (B, n))
    T = rng.integers(0, 4, (B, m))
    T[: B // 2] = Q[: B // 2]
    flip = rng.random((B // 2, n)) < 0.2
    T[: B // 2] = np.where(flip, (T[: B // 2] + 2) % 4, T[: B // 2])
    H0 = rng.integers(0, 12, B)
    params = W.Params(W.Scoring(), w=100, zdrop=100, end_bonus=5)
    got, _, stale = _oracle_grid(Q, T, H0, oracle.NO_ZDROP, params)
    ref = brute.extend_full(params, Q, T, H0, band=True)
    clean = stale == 0
    assert clean.mean() > 0.5
    assert (got[clean, 0] <= ref[clean, 0]).all()
    assert (got[:, 0] == ref[:, 0]).mean() > 0.9


def _readlike(rng, B, n, m, flip_p=0.2):
    Q = rng.integers(0, 4, (B, n))
    T = rng.integers(0, 4, (B, m))
    k = min(n, m)
    T[: B // 2, :k] = Q[: B // 2, :k]
    flip = rng.random((B // 2, k)) < flip_p
    T[: B // 2, :k] = np.where(flip, (T[: B // 2, :k] + 1) % 4, T[: B // 2, :k])
    return Q, T


TRIM_PARAMS = [
    W.Params(W.Scoring(), w=100, zdrop=100, end_bonus=5),
    W.Params(W.Scoring(1, 4, 2, 1, 2, 1), w=3, zdrop=3, end_bonus=5),
    W.Params(W.Scoring(1, 6, 1, 1, 1, 1), w=100, zdrop=5, end_bonus=0),
    W.Params(W.Scoring(2, 3, 3, 2, 1, 1), w=2, zdrop=0, end_bonus=1),
]


def test_trimmed_exhaustive_4x4():
    """The full heuristic on every pair of 4-base sequences equals the
    explicit-matrix restatement with band adjustment (rule c)."""
    allseq = np.array(list(itertools.product(range(4), repeat=4)), np.uint8)
    Q = np.repeat(allseq, len(allseq), axis=0)
    T = np.tile(allseq, (len(allseq), 1))
    for params in TRIM_PARAMS[:2]:
        for h0 in (2, 9):
            H0 = np.full(len(Q), h0, np.int32)
            got, _, _ = _oracle_grid(Q, T, H0, 0, params)
            np.testing.assert_array_equal(got, brute.extend_trimmed(params, Q, T, H0))


@pytest.mark.parametrize("pi", range(len(TRIM_PARAMS)))
@pytest.mark.parametrize("n,m", [(1, 5), (5, 1), (8, 8), (12, 16), (24, 30), (40, 20)])
def test_trimmed_random(pi, n, m):
    """As above on random read-like pairs, including pairs where the band
    regrows over slots written by earlier rows (R6)."""
    params = TRIM_PARAMS[pi]
    rng = np.random.default_rng(1000 * pi + 10 * n + m)
    B = 3000
    Q, T = _readlike(rng, B, n, m, 0.25)
    H0 = rng.integers(0, 20, B)
    got, _, stale = _oracle_grid(Q, T, H0, 0, params)
    np.testing.assert_array_equal(got, brute.extend_trimmed(params, Q, T, H0))
    got2, _, _ = _oracle_grid(Q, T, H0, oracle.NO_ZDROP, params)
    np.testing.assert_array_equal(got2, brute.extend_trimmed(params, Q, T, H0, zdrop=False))


def test_stale_reads_occur_and_match():
    """R6 is exercised: a narrow band over noisy pairs makes the band regrow
    over slots from earlier rows with non-zero values, and the results still
    equal the explicit-matrix restatement."""
    params = W.Params(W.Scoring(1, 4, 2, 1, 2, 1), w=3, zdrop=0, end_bonus=5)
    rng = np.random.default_rng(11)
    B = 6000
    Q, T = _readlike(rng, B, 24, 24, 0.3)
    H0 = rng.integers(0, 20, B)
    got, _, stale = _oracle_grid(Q, T, H0, 0, params)
    assert (stale > 0).sum() >= 20
    np.testing.assert_array_equal(got, brute.extend_trimmed(params, Q, T, H0))


def test_gap_reading_differs():
    """R3: with gaps opening from M an insertion cannot directly follow a
    deletion; opening from H (Eq. 2 as printed) allows it.  The two readings
    agree on gap-free alignments and differ on some adjacent-gap inputs."""
    rng = np.random.default_rng(3)
    params = W.Params(W.Scoring(1, 4, 1, 1, 1, 1), w=100, zdrop=0, end_bonus=0)
    n, m = 8, 8
    B = 20000
    Q = rng.integers(0, 4, (B, n))
    T = rng.integers(0, 4, (B, m))
    H0 = np.full(B, 10)
    a, _, _ = _oracle_grid(Q, T, H0, 0, params)
    b, _, _ = _oracle_grid(Q, T, H0, oracle.GAP_FROM_H, params)
    assert (a != b).any(axis=1).sum() > 0
    # the default reading is the one the brute force states (gaps open from M)
    full, _, _ = _oracle_grid(Q, T, H0, oracle.NO_BAND | oracle.NO_TRIM | oracle.NO_ZDROP, params)
    np.testing.assert_array_equal(full, brute.extend_full(params, Q, T, H0))
    np.testing.assert_array_equal(a, brute.extend_trimmed(params, Q, T, H0, zdrop=False))
    same = np.tile(np.arange(8) % 4, (50, 1))
    a2, _, _ = _oracle_grid(same, same, np.full(50, 10), 0, params)
    b2, _, _ = _oracle_grid(same, same, np.full(50, 10), oracle.GAP_FROM_H, params)
    np.testing.assert_array_equal(a2, b2)


# ---------------------------------------------------------------- invariants

@pytest.mark.parametrize("config", ["plain10k", "read151", "read250", "long10k"])
def test_invariants_on_workloads(config):
    n = {"plain10k": 10000, "read151": 20000, "read250": 20000, "long10k": 300}[config]
    wl = W.make(config, n_pairs=n)
    res, cells, _ = oracle.extend_batch(wl, nthreads=8)
    score, qle, tle, gtle, gscore, moff = res.T
    assert (score >= wl.h0).all()
    assert ((qle >= 0) & (qle <= wl.q_len)).all()
    assert ((tle >= 0) & (tle <= wl.t_len)).all()
    assert ((gtle >= 0) & (gtle <= wl.t_len)).all()
    assert (gscore <= score).all()
    assert ((moff >= 0) & (moff <= np.maximum(wl.q_len, wl.t_len))).all()
    # qle = tle = 0 exactly when the best stayed at the seed
    assert ((qle == 0) == (score == wl.h0)).all()
    # z-drop only stops rows early: switching it off never lowers a score
    res2, cells2, _ = oracle.extend_batch(wl, flags=oracle.NO_ZDROP, nthreads=8)
    assert (res2[:, 0] >= score).all()
    assert (cells2 >= cells).all()
    # cells are bounded by the band area
    assert (cells <= wl.q_len.astype(np.int64) * wl.t_len).all()


def test_threads_do_not_change_results():
    wl = W.make("plain10k", n_pairs=3000)
    a = oracle.extend_batch(wl, nthreads=1)
    b = oracle.extend_batch(wl, nthreads=7)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


def test_generator_deterministic():
    a = W.make("read250", n_pairs=1000, nthreads=1)
    b = W.make("read250", n_pairs=1000, nthreads=5)
    for k in ("q", "q_off", "q_len", "t", "t_off", "t_len", "h0"):
        np.testing.assert_array_equal(getattr(a, k), getattr(b, k))
    assert a.q.max() <= 3 and a.t.max() <= 3


def test_n_scores_minus_one():
    """R11 by hand: one cell, h0 = 10.  Against N (either side, or both) the
    cell gets M = 10 - 1 = 9 < h0, so the best stays h0 at (0, 0) and the
    query end is reached with 9 at row 0: {10, 0, 0, 1, 9, 0}.  A match
    gives 11 instead."""
    for q, t in ((4, 4), (4, 0), (0, 4), (2, 4)):
        got, _, _ = _oracle_grid([[q]], [[t]], [10], oracle.NO_BAND | oracle.NO_TRIM | oracle.NO_ZDROP)
        assert got[0].tolist() == [10, 0, 0, 1, 9, 0], (q, t, got[0])
    got, _, _ = _oracle_grid([[2]], [[2]], [10], 0)
    assert got[0].tolist() == [11, 1, 1, 1, 11, 0]


def test_all_n_diagonal():
    """A query of n N's against a target of N's: along the diagonal H drops by
    1 per cell (the gaps cost more), so the best stays h0 and the query end is
    first reached at row n - 1 with h0 - n."""
    n, h0 = 6, 20
    got, _, _ = _oracle_grid([[4] * n], [[4] * (n + 4)], [h0], 0)
    assert got[0][0] == h0 and got[0][1] == 0
    assert got[0][4] == h0 - n and got[0][3] >= n


@pytest.mark.parametrize("n,m", [(1, 1), (3, 5), (5, 3), (6, 8), (8, 8)])
def test_brute_random_small_with_n(n, m):
    """Codes 0..4 (N) on both sides: the one-row sweep equals the full-matrix
    DP, each applying R11 on its own."""
    rng = np.random.default_rng(n * 53 + m)
    B = 3000
    Q = rng.integers(0, 4, (B, n))
    T = rng.integers(0, 4, (B, m))
    half = B // 2
    k = min(n, m)
    T[:half, :k] = Q[:half, :k]
    Q = np.where(rng.random((B, n)) < 0.15, 4, Q)
    T = np.where(rng.random((B, m)) < 0.15, 4, T)
    H0 = rng.integers(0, 20, B)
    got, _, _ = _oracle_grid(Q, T, H0, oracle.NO_BAND | oracle.NO_TRIM | oracle.NO_ZDROP)
    np.testing.assert_array_equal(got, brute.extend_full(P, Q, T, H0))
    got, _, _ = _oracle_grid(Q, T, H0, 0)
    np.testing.assert_array_equal(got, brute.extend_trimmed(P, Q, T, H0))
