"""Pins of the SMEM oracle (oracle/smem.py) against brute force, no GPU:
occurrences by substring search in T = ref + revcomp(ref), SA intervals by
ranking the pattern among the sorted suffixes of T + terminator."""
import numpy as np
import pytest

from oracle import smem


def brute(ref, x, min_len):
    T = "".join("ACGT"[c] for c in smem.text(ref))
    xs = "".join("ACGTN"[c] for c in x)                              # N (code 4) occurs nowhere in T
    suffixes = sorted(T[i:] + "\x00" for i in range(len(T) + 1))   # "\x00" sorts before A: the terminator
    ends = []
    for i in range(len(xs)):
        j = i
        while j < len(xs) and xs[i:j + 1] in T:
            j += 1
        ends.append(j)
    res = []
    for i in range(len(xs)):
        if (i == 0 or ends[i - 1] < ends[i]) and ends[i] - i >= min_len:
            p = xs[i:ends[i]]
            k = sum(1 for s in suffixes if s < p)
            cnt = sum(1 for s in suffixes if s.startswith(p))
            res.append((i, ends[i] - i, k, cnt))
    return res


@pytest.mark.parametrize("seed", range(6))
def test_oracle_matches_brute_force(seed):
    rng = np.random.default_rng(seed)
    ref = rng.integers(0, 4, 80 + 20 * seed)
    reads = []
    for _ in range(6):
        L = int(rng.integers(1, 30))
        if rng.random() < 0.6:
            p = int(rng.integers(0, ref.shape[0] - L))
            x = ref[p:p + L].copy()
            if rng.random() < 0.5:
                x = 3 - x[::-1]                                   # from the other strand
            flips = rng.random(L) < 0.08
            x[flips] = (x[flips] + 1) % 4
        else:
            x = rng.integers(0, 4, L)
        reads.append(x)
    got = smem.smems(ref, reads, min_len=1)
    for x, g in zip(reads, got):
        assert g == brute(ref, x, 1), (list(x), g)


def test_hand_example():
    # ref = ACGTAC, revcomp = GTACGT, T = ACGTACGTACGT.  Read CGTACGA: from 0
    # the longest match is CGTACG (T[1:7] and T[5:11]: 2 occurrences; CGTACGA
    # does not occur); from 1..5 the matches end at 6 as well (no new SMEM);
    # from 6, "A" occurs 3 times.  So the SMEMs are (0, 6) x2 and (6, 1) x3.
    ref = np.array([0, 1, 2, 3, 0, 1])
    x = np.array([1, 2, 3, 0, 1, 2, 0])
    got = smem.smems(ref, [x], min_len=1)[0]
    assert [(q, n, s) for q, n, _, s in got] == [(0, 6, 2), (6, 1, 3)]
    assert got == brute(ref, x, 1)
    # min_len drops the short ones
    assert smem.smems(ref, [x], min_len=3)[0] == [g for g in got if g[1] >= 3]


@pytest.mark.parametrize("seed", range(3))
def test_oracle_with_n_matches_brute_force(seed):
    """Reads with N: no match contains an N, and a match may start right
    after one."""
    rng = np.random.default_rng(50 + seed)
    ref = rng.integers(0, 4, 120)
    reads = []
    for _ in range(8):
        L = int(rng.integers(2, 30))
        p = int(rng.integers(0, ref.shape[0] - L))
        x = ref[p:p + L].copy()
        x[rng.random(L) < 0.15] = 4
        reads.append(x)
    reads.append(np.array([4, 4, 4]))
    for min_len in (1, 3):
        got = smem.smems(ref, reads, min_len)
        for x, g in zip(reads, got):
            assert [tuple(int(v) for v in t) for t in g] == brute(ref, x, min_len)
