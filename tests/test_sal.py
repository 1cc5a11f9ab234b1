"""Suffix array and its lookup (Section IV-D, Eq. 1), no GPU: the oracle
against brute-force suffix sorting, and the library's index builder
(bsw_sa_build, host code) against the oracle."""
import numpy as np
import pytest

from oracle import sal
from paper_1907_12931_gb300 import workload as W


def brute(s):
    n = len(s)
    return sorted(range(n + 1), key=lambda i: list(s[i:]) + [-1])


@pytest.mark.parametrize("alpha", [1, 2, 4])
def test_oracle_suffix_array_is_sorted_suffixes(alpha):
    rng = np.random.default_rng(alpha)
    for n in list(range(0, 14)) + [40, 200]:
        for _ in range(12):
            s = rng.integers(0, alpha, n)
            assert list(sal.suffix_array(s)) == brute(s), (n, list(s))


def test_oracle_lookup_is_eq1():
    sa = np.array([7, 3, 0, 5, 1, 6, 2, 4], np.int32)
    np.testing.assert_array_equal(sal.lookup(sa, [2, 0, 7, 5], [3, 1, 1, 0]), [0, 5, 1, 7, 4])
    assert sal.lookup(sa, [], []).shape == (0,)


def lib():
    from paper_1907_12931_gb300 import bsw
    bsw.lib()
    return bsw


@pytest.mark.parametrize("n", [0, 1, 2, 7, 1000, 65_537, 300_000])
def test_library_builder_matches_oracle(n):
    bsw = lib()
    rng = np.random.default_rng(n)
    for alpha in (1, 2, 4):
        s = rng.integers(0, alpha, n).astype(np.uint8)
        np.testing.assert_array_equal(bsw.bsw_sa_build(s), sal.suffix_array(s))


def test_library_builder_on_the_reference_prefix():
    bsw = lib()
    s = W.reference()[:1_000_000]
    sa = bsw.bsw_sa_build(s)
    np.testing.assert_array_equal(sa, sal.suffix_array(s))


def test_library_builder_rejects_bad_codes():
    bsw = lib()
    with pytest.raises(bsw.BswError):
        bsw.bsw_sa_build(np.array([0, 1, 4, 2], np.uint8))
