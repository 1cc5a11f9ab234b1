"""CPU oracle of the SMEM search (test infrastructure: only tests/ and
bench.py's CPU legs use it).

Section IV searches super-maximal exact matches (Li 2012) of a read in the
reference and its reverse complement: T = ref + revcomp(ref) (the reverse
complement of base c is 3 - c).  For a read X, e(i) is the end of the
longest prefix of X[i:] that occurs in T; the SMEMs are the intervals
[i, e(i)) with i = 0 or e(i-1) < e(i): exact matches that no longer exact
match contains.  Each is reported as (qbeg, len, k, s) with [k, k + s) its
interval in the suffix array of T + terminator ($ smaller than every base),
so s is its number of occurrences in T.  The interval of a pattern is found
by narrowing the suffix array one symbol at a time: suffixes that share the
first d symbols are consecutive and sorted by their next symbol.
"""
from __future__ import annotations

import numpy as np

from oracle import sal


def text(ref) -> np.ndarray:
    ref = np.asarray(ref, np.int64)
    return np.concatenate([ref, 3 - ref[::-1]])


class Index:
    def __init__(self, ref):
        self.T = text(ref)
        self.sa = sal.suffix_array(self.T).astype(np.int64)
        self.n = self.T.shape[0]

    def sym(self, rows, d):
        """Symbol d of the suffixes at SA rows (-1 past the end, the terminator)."""
        p = self.sa[rows] + d
        return np.where(p < self.n, self.T[np.minimum(p, self.n - 1)], -1)

    def narrow(self, lo, hi, d, c):
        """Rows in [lo, hi) (suffixes sharing d symbols) whose symbol d is c."""
        rows = np.arange(lo, hi)
        col = self.sym(rows, d)
        return lo + int(np.searchsorted(col, c, "left")), lo + int(np.searchsorted(col, c, "right"))


def smems(ref, reads, min_len: int):
    """reads: code arrays.  Returns a list per read of (qbeg, len, k, s)."""
    ix = Index(ref)
    out = []
    for x in reads:
        x = np.asarray(x, np.int64)
        L = x.shape[0]
        ends, ivs = [], []
        for i in range(L):
            lo, hi, j = 0, ix.n + 1, i
            while j < L:
                l2, h2 = ix.narrow(lo, hi, j - i, x[j])
                if l2 >= h2:
                    break
                lo, hi, j = l2, h2, j + 1
            ends.append(j)
            ivs.append((lo, hi))
        res = []
        for i in range(L):
            if (i == 0 or ends[i - 1] < ends[i]) and ends[i] - i >= min_len:
                lo, hi = ivs[i]
                res.append((i, ends[i] - i, lo, hi - lo))
        out.append(res)
    return out
