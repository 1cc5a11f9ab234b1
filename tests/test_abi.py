"""C-ABI checks that need no GPU: the library builds, loads, exports every
function include/bsw.h declares, and its host-only helpers behave."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1907_12931_gb300 import build as B

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "bsw.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    from paper_1907_12931_gb300 import bsw
    return bsw


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bsw_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_abi():
    names = declared_functions()
    for need in ("bsw_init", "bsw_extend_batch", "bsw_stream_submit", "bsw_stream_poll", "bsw_strerror",
                 "bsw_destroy", "bsw_pack_2bit", "bsw_sync"):
        assert need in names


def test_exports_every_declared_symbol(lib):
    so = ctypes.CDLL(B.LIB)
    for name in declared_functions():
        assert hasattr(so, name), name


def test_pack_2bit(lib):
    codes = np.array([0, 1, 2, 3, 3, 2, 1], np.uint8)
    packed = lib.bsw_pack_2bit(codes)
    assert packed.tolist() == [0b11100100, 0b00011011]
    np.testing.assert_array_equal(lib.bsw_pack_2bit(np.frombuffer(b"ACGTtgc", np.uint8)), packed)
    rng = np.random.default_rng(0)
    x = rng.integers(0, 4, 1001).astype(np.uint8)
    p = lib.bsw_pack_2bit(x)
    back = (p[np.arange(1001) // 4] >> (2 * (np.arange(1001) % 4))) & 3
    np.testing.assert_array_equal(back, x)
    with pytest.raises(lib.BswError) as e:
        lib.bsw_pack_2bit(np.frombuffer(b"ACNT", np.uint8))
    assert e.value.code == lib.BSW_EINVAL


def test_pack_2bit_n(lib):
    """N (code 4 or the letter) sets its bit in the bitmap and packs as 0;
    the other codes pack as bsw_pack_2bit does."""
    codes = np.array([0, 4, 2, 3, 4, 2, 1, 0, 4], np.uint8)
    packed, nm = lib.bsw_pack_2bit_n(codes)
    assert packed.tolist() == [0b11100000, 0b00011000, 0]
    assert nm.tolist() == [0b00010010, 0b1]
    p2, n2 = lib.bsw_pack_2bit_n(np.frombuffer(b"ANGTnGCAN", np.uint8))
    np.testing.assert_array_equal(p2, packed)
    np.testing.assert_array_equal(n2, nm)
    rng = np.random.default_rng(1)
    x = rng.integers(0, 5, 1003).astype(np.uint8)
    p, m = lib.bsw_pack_2bit_n(x)
    k = np.arange(1003)
    back = (p[k // 4] >> (2 * (k % 4))) & 3
    isn = (m[k // 8] >> (k % 8)) & 1
    np.testing.assert_array_equal(isn, (x == 4).astype(np.uint8))
    np.testing.assert_array_equal(back, np.where(x == 4, 0, x))
    with pytest.raises(lib.BswError) as e:
        lib.bsw_pack_2bit_n(np.array([0, 5], np.uint8))
    assert e.value.code == lib.BSW_EINVAL


def test_host_batch_carries_n_bitmaps(lib):
    from paper_1907_12931_gb300 import workload as W
    wl = W.from_lists([W.encode("ACGTN"), W.encode("ACGT")], [W.encode("ACGT"), W.encode("NNAC")], [5, 5], align=4)
    hb = lib.HostBatch(wl)
    assert hb.q_n is not None and hb.t_n is not None
    s = hb.struct()
    assert s.q_n == hb.q_n.ctypes.data and s.t_n == hb.t_n.ctypes.data
    assert hb.q_n.tolist() == [0b10000, 0]                      # queries at 0 and 8, 16 bases in all
    assert hb.t_n.tolist() == [0b110000, 0]                     # targets at 0 and 4, 12 bases
    plain = lib.HostBatch(W.from_lists([W.encode("ACGT")], [W.encode("ACGT")], [5], align=4))
    assert plain.q_n is None and plain.struct().q_n is None and plain.struct().t_n is None


def test_inject_n_keeps_padding_and_rates():
    from paper_1907_12931_gb300 import workload as W
    wl = W.make("plain10k", n_pairs=2000)
    nw = W.inject_n(wl, 0.01, 0.001, seed=3)
    qin = np.zeros(wl.q.shape[0], bool)
    for o, n in zip(wl.q_off, wl.q_len):
        qin[o:o + n] = True
    tin = np.zeros(wl.t.shape[0], bool)
    for o, n in zip(wl.t_off, wl.t_len):
        tin[o:o + n] = True
    assert not (nw.q[~qin] == 4).any() and not (nw.t[~tin] == 4).any()
    changed = nw.q != wl.q
    assert (nw.q[changed] == 4).all() and (nw.t[nw.t != wl.t] == 4).all()
    rate = (nw.q[qin] == 4).mean()
    assert 0.007 < rate < 0.013
    assert (nw.t[tin] == 4).mean() > 0.005


def test_strerror_and_version(lib):
    assert lib.bsw_strerror(0) == "ok"
    assert "budget" in lib.bsw_strerror(lib.BSW_EBUDGET)
    assert "unknown" in lib.bsw_strerror(-99)
    assert "sm_103a" in lib.bsw_version()


def test_invalid_arguments_without_gpu(lib):
    L = lib.lib()
    # bad scoring is rejected before any CUDA call
    sc = lib.bsw_scoring_t(0, 4, 6, 1, 6, 1)
    h = ctypes.c_void_p()
    assert L.bsw_init(ctypes.byref(sc), 100, 100, 5, 1 << 30, ctypes.byref(h)) == lib.BSW_EINVAL
    sc = lib.bsw_scoring_t(1, 4, 6, 0, 6, 1)
    assert L.bsw_init(ctypes.byref(sc), 100, 100, 5, 1 << 30, ctypes.byref(h)) == lib.BSW_EINVAL
    sc = lib.bsw_scoring_t(1, 4, 6, 1, 6, 1)
    assert L.bsw_init(ctypes.byref(sc), -1, 100, 5, 1 << 30, ctypes.byref(h)) == lib.BSW_EINVAL
    assert L.bsw_init(ctypes.byref(sc), 100, 100, 5, 0, ctypes.byref(h)) == lib.BSW_EINVAL
    assert L.bsw_extend_batch(None, None, None, None, None) == lib.BSW_EINVAL
    assert L.bsw_stream_poll(None, 1, 0) == lib.BSW_EINVAL
    assert L.bsw_band_width(None, 10, 10) == -1
    L.bsw_destroy(None)


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    """The product path has no fallback: a missing library is an error."""
    from paper_1907_12931_gb300 import bsw
    monkeypatch.setattr(bsw, "_lib", None)
    monkeypatch.setattr(bsw, "LIB", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        bsw.lib()


def test_header_constants_match_binding(lib):
    text = open(HEADER).read()
    import re as _re
    for name in ("BSW_MAX_QLEN", "BSW_NOALLOC_MAX_PAIRS", "BSW_NOALLOC_MAX_QLEN"):
        m = _re.search(r"#define\s+%s\s+(\d+)" % name, text)
        assert m, name
        assert int(m.group(1)) == getattr(lib, name), name


def test_inject_n_seeds_keeps_seeds_exact():
    """N goes outside the seeds only (seeds are exact matches), at about the
    asked rates; nothing else changes."""
    from paper_1907_12931_gb300 import workload as W
    sw = W.make_seeds("seeds151", n_reads=3000)
    nw = W.inject_n_seeds(sw, 0.01, 0.0005, seed=1)
    qs = sw.read_off[sw.seed_read].astype(np.int64) + sw.qbeg
    for q, ln, r in zip(qs, sw.slen, sw.rbeg):
        assert not (nw.reads[q:q + ln] == 4).any()
        assert not (nw.ref[r:r + ln] == 4).any()
    assert (nw.reads[nw.reads != sw.reads] == 4).all() and (nw.ref[nw.ref != sw.ref] == 4).all()
    rate = (nw.reads == 4).sum() / sw.read_len.sum()
    assert 0.003 < rate < 0.01
    assert 0.003 < (nw.ref == 4).mean() < 0.02


def test_package_never_imports_the_oracle():
    """Parity rests on the oracle sharing nothing with the product: no module
    of the package imports it (the checker is used only by tests, the smoke
    check and the benchmark's CPU legs)."""
    import ast
    pkg = os.path.join(os.path.dirname(os.path.dirname(__file__)), "paper_1907_12931_gb300")
    offenders = []
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if not f.endswith(".py"):
                continue
            path = os.path.join(dirpath, f)
            tree = ast.parse(open(path).read(), path)
            for node in ast.walk(tree):
                names = []
                if isinstance(node, ast.Import):
                    names = [a.name for a in node.names]
                elif isinstance(node, ast.ImportFrom):
                    names = [node.module or ""]
                if any(nm == "oracle" or nm.startswith("oracle.") for nm in names):
                    offenders.append("%s:%d" % (os.path.relpath(path, pkg), node.lineno))
    assert offenders == []
    # and the CUDA sources include nothing from the oracle's directory
    csrc = os.path.join(pkg, "csrc")
    for f in os.listdir(csrc):
        text = open(os.path.join(csrc, f), errors="replace").read()
        assert "oracle" not in re.findall(r'#include\s*[<"]([^>"]+)', text).__str__(), f


def test_fault_inject_spec(lib):
    """The fault-injection spec parser (host only): site names, optional
    :skip:count, NULL/"" to disarm; malformed specs are refused and change
    nothing."""
    for spec in ("alloc", "h2d", "launch", "thread", "host", "alloc,h2d,launch", "h2d:3", "launch:0:5",
                 "alloc,thread:2:1", "", None):
        assert lib.bsw_fault_inject(spec) == lib.BSW_OK, spec
    for spec in ("bogus", "alloc,", "alloc:x", "alloc:1:", "alloc:1:2:3", ":1", "alloc;h2d", "ALLOC",
                 "alloc:99999999999"):
        assert lib.bsw_fault_inject(spec) == lib.BSW_EINVAL, spec
    assert lib.bsw_fault_inject(None) == lib.BSW_OK


def test_fault_inject_environment(tmp_path):
    """BSW_FAULT_INJECT is read when the library loads; a malformed value is
    ignored (the library still loads and runs its host helpers)."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(__file__))
    code = ("import sys; sys.path.insert(0, %r); from paper_1907_12931_gb300 import bsw; import numpy as np; "
            "print(bsw.bsw_pack_2bit(np.array([0,1,2,3], np.uint8)).tolist())" % root)
    for val in ("alloc,launch:1:2", "not-a-site"):
        env = dict(os.environ, BSW_FAULT_INJECT=val)
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=120)
        assert r.returncode == 0, r.stderr
        assert r.stdout.strip() == "[228]"


def _band_area(params, q_len, t_len, w_override=None):
    """Each pair's band area, from the band clip's definition in include/bsw.h."""
    sc = params.scoring
    n = np.asarray(q_len, np.int64)
    m = np.asarray(t_len, np.int64)
    w = np.full(n.shape, params.w, np.int64) if w_override is None else np.asarray(w_override, np.int64)

    def cap(o, e):
        return np.maximum((n * sc.match + params.end_bonus - o + e) // e, 1)

    wb = np.minimum(w, np.minimum(cap(sc.o_ins, sc.e_ins), cap(sc.o_del, sc.e_del)))
    return n * np.minimum(m, 2 * wb + 1)


def test_partition_balances_band_area(lib):
    """bsw_partition: contiguous ranges covering every pair once, each
    boundary the first pair at which the running band area reaches k/parts of
    the total (so every part is within one pair of an equal share)."""
    from paper_1907_12931_gb300 import workload as W
    for name, n_pairs in (("read151", 50_000), ("long10k", 3000), ("plain10k", 777)):
        wl = W.make(name, n_pairs=n_pairs)
        wt = _band_area(wl.params, wl.q_len, wl.t_len).astype(np.float64)
        run = np.cumsum(wt)
        for parts in (1, 2, 3, 8, 13):
            b = lib.bsw_partition(wl.params, wl.q_len, wl.t_len, parts)
            assert b[0] == 0 and b[-1] == wl.n_pairs and (np.diff(b) >= 0).all()
            for k in range(1, parts):
                want = int(np.searchsorted(run * parts >= run[-1] * k, True)) + 1
                assert b[k] == want, (name, parts, k)
            shares = np.add.reduceat(wt, b[:-1])[np.diff(b) > 0] if parts > 1 else wt.sum()
            assert np.all(np.abs(np.atleast_1d(shares) - wt.sum() / parts) <= wt.max() + 1)
    # per-pair bands, more parts than pairs, an empty batch, bad arguments
    wl = W.make("plain10k", n_pairs=5)
    ws = np.array([1, 100, 3, 0, 50], np.int32)
    b = lib.bsw_partition(wl.params, wl.q_len, wl.t_len, 9, w_override=ws)
    assert b[0] == 0 and b[-1] == 5 and (np.diff(b) >= 0).all() and b.shape == (10,)
    e = W.make("plain10k", n_pairs=1)
    b = lib.bsw_partition(e.params, e.q_len[:0], e.t_len[:0], 4)
    assert b.tolist() == [0, 0, 0, 0, 0]
    with pytest.raises(lib.BswError):
        lib.bsw_partition(wl.params, wl.q_len, wl.t_len, 0)
    with pytest.raises(lib.BswError):
        lib.bsw_partition(wl.params, np.array([-1, 3], np.int32), np.array([4, 4], np.int32), 2)
