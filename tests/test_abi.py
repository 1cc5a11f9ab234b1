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
