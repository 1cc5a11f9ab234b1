"""Seeded synthetic seed-extension workloads.

The paper's BSW measurements use pairs intercepted from BWA-MEM on real reads
(Section VI, Table V).  Neither those reads nor the reference ship here, so the
workloads are synthetic stand-ins drawn by ``bswgen.c`` (splitmix64 streams,
one per read or pair).  This module only produces inputs: sequences as codes
0..3 (A, C, G, T), offsets, lengths and the seed score h0.  It holds none of
the extension arithmetic; the CUDA path and the CPU oracle both take their
inputs from here.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bswgen.c")
_SO = os.path.join(_HERE, "_bswgen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the generator into an in-tree shared object."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-pthread", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, i32, u64, vp = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_void_p
            lib.bswgen_num_units.argtypes = [ctypes.c_int, i64]
            lib.bswgen_num_units.restype = i64
            lib.bswgen_lengths.argtypes = [ctypes.c_int, u64, i64, i32, vp, vp]
            lib.bswgen_lengths.restype = ctypes.c_int
            lib.bswgen_fill.argtypes = [ctypes.c_int, u64, i64, i32, vp, vp, vp, vp, vp, ctypes.c_int]
            lib.bswgen_fill.restype = ctypes.c_int
            lib.bswgen_random_codes.argtypes = [u64, i64, vp]
            lib.bswgen_random_codes.restype = None
            lib.bswgen_seeds.argtypes = [u64, i64, i32, i32, vp, vp, vp, vp, vp, ctypes.c_int]
            lib.bswgen_seeds.restype = ctypes.c_int
            lib.bswgen_ref_copy.argtypes = [i64, i64, vp]
            lib.bswgen_ref_copy.restype = ctypes.c_int
            lib.bswgen_ref_len.argtypes = []
            lib.bswgen_ref_len.restype = i64
            lib.bswgen_reads.argtypes = [u64, i64, i32, i64, vp, vp]
            lib.bswgen_reads.restype = ctypes.c_int
            _lib = lib
    return _lib


@dataclasses.dataclass(frozen=True)
class Scoring:
    """Match score a > 0; mismatch, gap-open and gap-extension penalties > 0.

    A gap of k bases costs o + k*e (Eq. 3 writes the boundary as
    H[0,0] - (g_o + g_e*i))."""
    match: int = 1
    mismatch: int = 4
    o_del: int = 6
    e_del: int = 1
    o_ins: int = 6
    e_ins: int = 1


@dataclasses.dataclass(frozen=True)
class Params:
    scoring: Scoring = Scoring()
    w: int = 100
    zdrop: int = 100
    end_bonus: int = 5


@dataclasses.dataclass
class Workload:
    """A batch of extension pairs.  Sequence k of q is q[q_off[k] : q_off[k] + q_len[k]]."""
    name: str
    params: Params
    q: np.ndarray       # uint8 codes 0..3 (4 = N)
    q_off: np.ndarray   # int64, in bases
    q_len: np.ndarray   # int32
    t: np.ndarray
    t_off: np.ndarray
    t_len: np.ndarray
    h0: np.ndarray      # int32

    @property
    def n_pairs(self) -> int:
        return int(self.q_len.shape[0])

    def subset(self, idx) -> "Workload":
        """Pairs idx (an index array), re-laid out compactly."""
        idx = np.asarray(idx, dtype=np.int64)
        ql, tl = self.q_len[idx], self.t_len[idx]
        qo, qt = layout(ql)
        to, tt = layout(tl)
        return Workload(self.name + "[subset]", self.params, _gather(self.q, self.q_off[idx], ql, qo, qt), qo,
                        ql.copy(), _gather(self.t, self.t_off[idx], tl, to, tt), to, tl.copy(),
                        self.h0[idx].copy())


def _gather(seq, src_off, lengths, dst_off, total):
    """Copy sequences [src_off, src_off + len) of seq to dst_off in a new array of `total` bases."""
    out = np.zeros(total, np.uint8)
    lengths = np.asarray(lengths, np.int64)
    n = int(lengths.sum())
    if n:
        starts = np.repeat(np.cumsum(lengths) - lengths, lengths)
        within = np.arange(n, dtype=np.int64) - starts
        out[np.repeat(dst_off, lengths) + within] = seq[np.repeat(src_off, lengths) + within]
    return out


def layout(lengths: np.ndarray, align: int = 16):
    """Offsets (multiples of `align` bases) for sequences of the given lengths, and the total."""
    lengths = np.asarray(lengths, dtype=np.int64)
    padded = (lengths + align - 1) // align * align
    off = np.zeros(lengths.shape[0], np.int64)
    if lengths.shape[0] > 1:
        np.cumsum(padded[:-1], out=off[1:])
    total = int(padded.sum()) + align
    return off, total


# The five workloads: id, pairs, seed, band w, z-drop.  Scoring is the same for
# all: match 1, mismatch 4, gap open 6, gap extend 1, end bonus 5.
CONFIGS = {
    "plain10k": dict(gen=0, n_pairs=10_000, seed=0, w=100, zdrop=100),
    "read151": dict(gen=1, n_pairs=2_000_000, seed=1, w=100, zdrop=100),
    "read250": dict(gen=2, n_pairs=4_000_000, seed=2, w=100, zdrop=100),
    "long10k": dict(gen=3, n_pairs=20_000, seed=3, w=500, zdrop=400),
}


def make(config: str, n_pairs: int | None = None, seed: int | None = None, align: int = 16,
         nthreads: int | None = None) -> Workload:
    """Generate workload `config` (a CONFIGS key); n_pairs/seed override the defaults."""
    c = CONFIGS[config]
    n = c["n_pairs"] if n_pairs is None else int(n_pairs)
    s = c["seed"] if seed is None else int(seed)
    params = Params(Scoring(), w=c["w"], zdrop=c["zdrop"], end_bonus=5)
    lib = _load()
    q_len = np.zeros(n, np.int32)
    t_len = np.zeros(n, np.int32)
    rc = lib.bswgen_lengths(c["gen"], s, n, params.scoring.match, q_len.ctypes.data, t_len.ctypes.data)
    if rc != 0:
        raise RuntimeError("bswgen_lengths failed: %d" % rc)
    q_off, qt = layout(q_len, align)
    t_off, tt = layout(t_len, align)
    q = np.zeros(qt, np.uint8)
    t = np.zeros(tt, np.uint8)
    h0 = np.zeros(n, np.int32)
    nth = nthreads or min(32, os.cpu_count() or 1)
    rc = lib.bswgen_fill(c["gen"], s, n, params.scoring.match, q_off.ctypes.data, t_off.ctypes.data,
                         q.ctypes.data, t.ctypes.data, h0.ctypes.data, nth)
    if rc != 0:
        raise RuntimeError("bswgen_fill failed: %d" % rc)
    return Workload(config, params, q, q_off, q_len, t, t_off, t_len, h0)


def random_codes(seed: int, n: int) -> np.ndarray:
    out = np.zeros(n, np.uint8)
    _load().bswgen_random_codes(seed, n, out.ctypes.data)
    return out


def from_lists(queries, targets, h0s, params: Params | None = None, align: int = 16,
               name: str = "custom") -> Workload:
    """Build a workload from explicit code sequences (lists/arrays of 0..3)."""
    ql = np.array([len(x) for x in queries], np.int32)
    tl = np.array([len(x) for x in targets], np.int32)
    qo, qt = layout(ql, align)
    to, tt = layout(tl, align)
    q = np.zeros(qt, np.uint8)
    t = np.zeros(tt, np.uint8)
    for k, x in enumerate(queries):
        q[qo[k]:qo[k] + len(x)] = np.asarray(x, np.uint8)
    for k, x in enumerate(targets):
        t[to[k]:to[k] + len(x)] = np.asarray(x, np.uint8)
    return Workload(name, params or Params(), q, qo, ql, t, to, tl, np.asarray(h0s, np.int32))


def encode(s: str) -> np.ndarray:
    """ACGTN string -> codes 0..4 (4 = N)."""
    lut = {"A": 0, "C": 1, "G": 2, "T": 3, "N": 4}
    return np.array([lut[ch] for ch in s.upper()], np.uint8)


def _draw_positions(off, ln, k, rng):
    """k positions drawn uniformly, with replacement, from the bases of the
    sequences [off, off + ln); also the sequence of each."""
    ln = np.asarray(ln, np.int64)
    cum = np.cumsum(ln)
    total = int(cum[-1]) if cum.size else 0
    if total == 0 or k == 0:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    r = rng.integers(0, total, k)
    i = np.searchsorted(cum, r, side="right")
    return np.asarray(off, np.int64)[i] + r - (cum[i] - ln[i]), i


def inject_n(wl: Workload, q_rate: float, t_runs: float, seed: int, run_max: int = 40) -> Workload:
    """A copy of wl with N bases (code 4): about a q_rate fraction of the
    query bases become N, scattered (sequencer no-calls), and about a t_runs
    fraction of the target bases start a run of 1..run_max N's, cut at the
    target's end (assembly gaps in the reference).  Positions are drawn with
    replacement; padding between sequences is left as it was."""
    rng = np.random.default_rng(seed)
    q, t = wl.q.copy(), wl.t.copy()
    kq = rng.binomial(int(wl.q_len.sum()), q_rate)
    pos, _ = _draw_positions(wl.q_off, wl.q_len, kq, rng)
    q[pos] = 4
    kt = rng.binomial(int(wl.t_len.sum()), t_runs)
    start, i = _draw_positions(wl.t_off, wl.t_len, kt, rng)
    if start.size:
        end = np.minimum(start + rng.integers(1, run_max + 1, start.size), wl.t_off[i] + wl.t_len[i])
        lens = end - start
        first = np.cumsum(lens) - lens
        t[np.repeat(start, lens) + np.arange(int(lens.sum())) - np.repeat(first, lens)] = 4
    return Workload(wl.name + "+N", wl.params, q, wl.q_off, wl.q_len, t, wl.t_off, wl.t_len, wl.h0)


# ------------------------------------------------------------ seeds on reads

@dataclasses.dataclass
class SeedWorkload:
    """Reads, the reference and seeds for the extension driver.  Read r is
    reads[read_off[r] : read_off[r] + read_len[r]]; seed k lies at read
    positions [qbeg[k], qbeg[k] + slen[k]) of read seed_read[k] and starts at
    reference position rbeg[k]; seeds of one read are consecutive."""
    name: str
    params: Params
    reads: np.ndarray       # uint8 codes
    read_off: np.ndarray    # int64, multiples of 4
    read_len: np.ndarray    # int32
    ref: np.ndarray         # uint8 codes (the whole reference)
    seed_read: np.ndarray   # int32
    qbeg: np.ndarray        # int32
    slen: np.ndarray        # int32
    rbeg: np.ndarray        # int64

    @property
    def n_seeds(self) -> int:
        return int(self.qbeg.shape[0])

    @property
    def n_reads(self) -> int:
        return int(self.read_len.shape[0])


def _covered(starts, ends, total):
    """Mask of positions [0, total) inside some [start, end)."""
    starts = np.asarray(starts, np.int64)
    ends = np.minimum(np.asarray(ends, np.int64), total)
    m = np.bincount(starts, minlength=total + 1)[:total + 1] - np.bincount(ends, minlength=total + 1)[:total + 1]
    return np.cumsum(m)[:total] > 0


def inject_n_seeds(sw: SeedWorkload, read_rate: float, ref_runs: float, seed: int, run_max: int = 40) -> SeedWorkload:
    """A copy of sw with N bases (code 4) outside the seeds (seeds are exact
    matches): about a read_rate fraction of the read bases become N,
    scattered, and about a ref_runs fraction of the reference bases start a
    run of 1..run_max N's."""
    rng = np.random.default_rng(seed)
    reads, ref = sw.reads.copy(), sw.ref.copy()
    qs = sw.read_off[sw.seed_read].astype(np.int64) + sw.qbeg
    in_seed = _covered(qs, qs + sw.slen, reads.shape[0])
    pos, _ = _draw_positions(sw.read_off, sw.read_len, rng.binomial(int(sw.read_len.sum()), read_rate), rng)
    pos = pos[~in_seed[pos]]
    reads[pos] = 4
    k = rng.binomial(ref.shape[0], ref_runs)
    start = rng.integers(0, ref.shape[0], k)
    runs = _covered(start, start + rng.integers(1, run_max + 1, k), ref.shape[0])
    ref[runs & ~_covered(sw.rbeg, sw.rbeg + sw.slen, ref.shape[0])] = 4
    return SeedWorkload(sw.name + "+N", sw.params, reads, sw.read_off, sw.read_len, ref, sw.seed_read, sw.qbeg,
                        sw.slen, sw.rbeg)


# Seed workloads: read length, reads, seeds per read, seed; scoring as above, w 100, zdrop 100.
SEED_CONFIGS = {
    "seeds151": dict(read_len=151, n_reads=500_000, spr=2, seed=11),
    "seeds250": dict(read_len=250, n_reads=500_000, spr=2, seed=12),
}

_ref_cache = None
_ref_lock = threading.Lock()


def reference() -> np.ndarray:
    """The 100 Mbp reference of the read workloads (codes), built once."""
    global _ref_cache
    lib = _load()
    with _ref_lock:
        if _ref_cache is None:
            n = int(lib.bswgen_ref_len())
            r = np.zeros(n, np.uint8)
            if lib.bswgen_ref_copy(0, n, r.ctypes.data) != 0:
                raise RuntimeError("bswgen_ref_copy failed")
            _ref_cache = r
    return _ref_cache


def make_seeds(config: str, n_reads: int | None = None, seed: int | None = None,
               nthreads: int | None = None) -> SeedWorkload:
    """Generate seed workload `config` (a SEED_CONFIGS key)."""
    c = SEED_CONFIGS[config]
    nr = c["n_reads"] if n_reads is None else int(n_reads)
    rl, spr = c["read_len"], c["spr"]
    ns = nr * spr
    reads = np.zeros(nr * rl, np.uint8)
    s_read = np.zeros(ns, np.int32)
    s_q = np.zeros(ns, np.int32)
    s_l = np.zeros(ns, np.int32)
    s_r = np.zeros(ns, np.int64)
    nth = nthreads or min(32, os.cpu_count() or 1)
    rc = _load().bswgen_seeds(c["seed"] if seed is None else int(seed), nr, rl, spr, reads.ctypes.data,
                              s_read.ctypes.data, s_q.ctypes.data, s_l.ctypes.data, s_r.ctypes.data, nth)
    if rc != 0:
        raise RuntimeError("bswgen_seeds failed: %d" % rc)
    read_len = np.full(nr, rl, np.int32)
    read_off, total = layout(read_len, 4)
    packed = np.zeros(total, np.uint8)
    packed[np.repeat(read_off, rl) + np.tile(np.arange(rl), nr)] = reads
    return SeedWorkload(config, Params(Scoring(), w=100, zdrop=100, end_bonus=5), packed, read_off, read_len,
                        reference(), s_read, s_q, s_l, s_r)


def seeds_from_lists(reads, ref, seeds, params: Params | None = None, name: str = "custom") -> SeedWorkload:
    """A seed workload from explicit reads (code sequences), a reference (codes)
    and seeds (read index, read start, length, reference start), the seeds of
    one read listed together."""
    rlen = np.array([len(r) for r in reads], np.int32)
    roff, total = layout(rlen, 4)
    packed = np.zeros(total, np.uint8)
    for k, r in enumerate(reads):
        packed[roff[k]:roff[k] + len(r)] = np.asarray(r, np.uint8)
    sr = np.array([s[0] for s in seeds], np.int32)
    return SeedWorkload(name, params or Params(), packed, roff, rlen, np.asarray(ref, np.uint8), sr,
                        np.array([s[1] for s in seeds], np.int32), np.array([s[2] for s in seeds], np.int32),
                        np.array([s[3] for s in seeds], np.int64))


def make_reads(n_reads: int, read_len: int = 151, ref_limit: int = 48_000_000, seed: int = 21):
    """Reads for the SMEM search copied from the reference's first ref_limit
    bases (read151 or read250 recipe), odd-numbered ones reverse-complemented.
    Returns (reads as codes laid out at read_off, read_off (multiples of 4),
    read_len, reference start of each read)."""
    reads = np.zeros(n_reads * read_len, np.uint8)
    pos = np.zeros(n_reads, np.int64)
    rc = _load().bswgen_reads(seed, n_reads, read_len, ref_limit, reads.ctypes.data, pos.ctypes.data)
    if rc != 0:
        raise RuntimeError("bswgen_reads failed: %d" % rc)
    rl = np.full(n_reads, read_len, np.int32)
    off, total = layout(rl, 4)
    codes = np.zeros(total, np.uint8)
    codes[np.repeat(off, read_len) + np.tile(np.arange(read_len), n_reads)] = reads
    return codes, off, rl, pos
