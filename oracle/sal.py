"""CPU oracle of the suffix array lookup (test infrastructure: only tests/
and bench.py's CPU legs use it).

Section IV-D keeps the suffix array S of the reference uncompressed, so a
lookup is Eq. 1, j = S[i].  S here is the suffix array of the text followed
by a terminator smaller than every base (n + 1 entries, S[0] = n): the
starting positions of all suffixes in lexicographic order.  `suffix_array`
computes it by prefix doubling, written plainly: suffixes are ranked by
their first symbol, then repeatedly by the pair (rank of the first 2^d
symbols, rank of the next 2^d), until all ranks differ.  `lookup` is Eq. 1
over SA intervals.
"""
from __future__ import annotations

import numpy as np


def suffix_array(codes) -> np.ndarray:
    s = np.asarray(codes, np.int64)
    n = s.shape[0] + 1
    rank = np.empty(n, np.int64)
    rank[:-1] = s + 1            # bases 1..4, the terminator 0
    rank[-1] = 0
    k = 1
    sa = np.argsort(rank, kind="stable")
    while True:
        second = np.full(n, -1, np.int64)          # rank of the suffix k further on (-1 past the end)
        second[:n - k] = rank[k:]
        sa = np.lexsort((second, rank))            # by (rank, second)
        key_r, key_s = rank[sa], second[sa]
        new = np.empty(n, np.int64)
        new[sa] = np.concatenate([[0], np.cumsum((key_r[1:] != key_r[:-1]) | (key_s[1:] != key_s[:-1]))])
        rank = new
        if rank.max() == n - 1:
            return sa.astype(np.int32)
        k *= 2


def lookup(sa: np.ndarray, k, cnt) -> np.ndarray:
    """The reference coordinates S[k[t]], ..., S[k[t] + cnt[t] - 1] of every
    interval t, concatenated in interval order."""
    parts = [sa[int(a):int(a) + int(c)] for a, c in zip(k, cnt)]
    return np.concatenate(parts).astype(np.int32) if parts else np.zeros(0, np.int32)
