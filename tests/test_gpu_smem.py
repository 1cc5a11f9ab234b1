"""SMEM search on the GPU (bsw_fm_build + bsw_smem) against the oracle
(oracle/smem.py), needs a GPU: every record (read, start, length, SA
interval) must match."""
import numpy as np
import pytest

from oracle import smem
from paper_1907_12931_gb300 import workload as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bsw():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_12931_gb300 import bsw as _b
    _b.lib()
    return _b


def pack(reads):
    rl = np.array([len(r) for r in reads], np.int32)
    off, total = W.layout(rl, 4)
    codes = np.zeros(total, np.uint8)
    for o, r in zip(off, reads):
        codes[o:o + len(r)] = r
    from paper_1907_12931_gb300 import bsw as b
    return b.bsw_pack_2bit(codes), off, rl


def check(bsw, ref, reads, min_len):
    want = smem.smems(ref, reads, min_len)
    packed, off, rl = pack(reads)
    with bsw.Context(W.Params()) as ctx:
        ctx.fm_build(ref)
        got, first = ctx.smem(packed, off, rl, min_len=min_len, cap=1)   # cap 1: exercises the retry
    for r, w in enumerate(want):
        g = got[first[r]:first[r + 1]]
        assert np.all(g["read_id"] == r)
        assert [tuple(int(v) for v in x) for x in g[["qbeg", "len", "k", "s"]]] == [tuple(x) for x in w], r


@pytest.mark.parametrize("seed", range(4))
def test_small_references(bsw, seed):
    rng = np.random.default_rng(100 + seed)
    ref = rng.integers(0, 4, 500 + 300 * seed).astype(np.uint8)
    reads = []
    for _ in range(40):
        L = int(rng.integers(0, 60))
        if rng.random() < 0.7 and L:
            p = int(rng.integers(0, ref.shape[0] - L))
            x = ref[p:p + L].copy()
            if rng.random() < 0.5:
                x = (3 - x[::-1]).astype(np.uint8)
            flips = rng.random(L) < 0.05
            x[flips] = (x[flips] + 1) % 4
        else:
            x = rng.integers(0, 4, L).astype(np.uint8)
        reads.append(x)
    for min_len in (1, 5, 19):
        check(bsw, ref, reads, min_len)


def test_generated_reads(bsw):
    """151 bp reads from both strands of a 60 kbp reference prefix."""
    ref = W.reference()[:60_000]
    codes, off, rl, _ = W.make_reads(120, 151, ref_limit=60_000)
    reads = [codes[o:o + n] for o, n in zip(off, rl)]
    check(bsw, ref, reads, 19)


@pytest.mark.parametrize("period", [1, 2, 3, 7])
def test_repetitive_reference(bsw, period):
    """A tandem repeat with a few point changes: the forward pass shrinks the
    occurrence count by a little per base, so the lists of many reads exceed
    the shared-memory capacity and those reads take the global-list launch."""
    rng = np.random.default_rng(200 + period)
    unit = rng.integers(0, 4, period).astype(np.uint8)
    n = 3000
    ref = np.tile(unit, n // period + 1)[:n]
    ref = np.where(rng.random(n) < 0.01, rng.integers(0, 4, n), ref).astype(np.uint8)
    reads = []
    for _ in range(30):
        L = int(rng.integers(20, 80))
        p = int(rng.integers(0, n - L))
        x = ref[p:p + L].copy()
        if rng.random() < 0.5:
            x = (3 - x[::-1]).astype(np.uint8)
        flips = rng.random(L) < 0.02
        x[flips] = (x[flips] + 1) % 4
        reads.append(x)
    reads.append(np.tile(unit, 100 // period + 1)[:100].astype(np.uint8))   # the pure repeat
    for min_len in (1, 19):
        check(bsw, ref, reads, min_len)


def test_reads_with_n(bsw):
    """N in reads (15% of bases, and runs): matches stop at an N and start
    after one; reads passed with their N bitmap."""
    rng = np.random.default_rng(300)
    ref = rng.integers(0, 4, 1500).astype(np.uint8)
    reads = []
    for _ in range(50):
        L = int(rng.integers(1, 70))
        p = int(rng.integers(0, ref.shape[0] - L))
        x = ref[p:p + L].copy()
        if rng.random() < 0.5:
            x = (3 - x[::-1]).astype(np.uint8)
        x[rng.random(L) < 0.15] = 4
        if L > 20 and rng.random() < 0.3:
            q = int(rng.integers(0, L - 5))
            x[q:q + 5] = 4
        reads.append(x)
    reads.append(np.full(10, 4, np.uint8))
    rl = np.array([len(r) for r in reads], np.int32)
    off, total = W.layout(rl, 4)
    codes = np.zeros(total, np.uint8)
    for o, r in zip(off, reads):
        codes[o:o + len(r)] = r
    packed, nm = bsw.bsw_pack_2bit_n(codes)
    for min_len in (1, 5):
        want = smem.smems(ref, reads, min_len)
        with bsw.Context(W.Params()) as ctx:
            ctx.fm_build(ref)
            got, first = ctx.smem(packed, off, rl, min_len=min_len, reads_n=nm)
        for r, w in enumerate(want):
            g = got[first[r]:first[r + 1]]
            assert [tuple(int(v) for v in x) for x in g[["qbeg", "len", "k", "s"]]] == [tuple(x) for x in w], r
