"""CPU oracle for BSW seed extension - TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg import this package.  The library (``paper_1907_12931_gb300``) never does,
and the two share no code: the only common module is the seeded input
generator, which holds none of the extension arithmetic.

``bsw_oracle.c`` is the literal row sweep of Section V-A (Eq. 2 and Eq. 3 plus
the band, abort and band-adjust rules); ``brute.py`` is an independent
full-matrix DP used to pin it on tiny inputs.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bsw_oracle.c")
_SO = os.path.join(_HERE, "_bsw_oracle.so")
_lock = threading.Lock()
_lib = None

NO_BAND = 1
NO_TRIM = 2
NO_ZDROP = 4
GAP_FROM_H = 8

FIELDS = ("score", "qle", "tle", "gtle", "gscore", "max_off")


class _Params(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int32) for k in
                ("match", "mismatch", "o_del", "e_del", "o_ins", "e_ins", "w", "zdrop", "end_bonus")] + \
               [("flags", ctypes.c_uint32)]


class _Result(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int32) for k in FIELDS]


def build(force: bool = False) -> str:
    """Compile the oracle (plain C, -O2, no SIMD intrinsics) into an in-tree .so."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC", "-pthread",
                               _SRC, "-o", tmp])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
            lib.orc_extend_one.argtypes = [ctypes.POINTER(_Params), i32, vp, i32, vp, i32, i32,
                                           ctypes.POINTER(_Result), ctypes.POINTER(i64), ctypes.POINTER(i64)]
            lib.orc_extend_one.restype = ctypes.c_int
            lib.orc_extend_batch.argtypes = [ctypes.POINTER(_Params), i64, vp, vp, vp, vp, vp, vp, vp, vp,
                                             vp, vp, vp, ctypes.c_int]
            lib.orc_extend_batch.restype = ctypes.c_int
            lib.orc_band_width.argtypes = [ctypes.POINTER(_Params), i32, i32]
            lib.orc_band_width.restype = i32
            _lib = lib
    return _lib


def _params(params, flags: int = 0) -> _Params:
    s = params.scoring
    return _Params(s.match, s.mismatch, s.o_del, s.e_del, s.o_ins, s.e_ins,
                   params.w, params.zdrop, params.end_bonus, flags)


def band_width(params, n: int, w: int | None = None) -> int:
    """The band after the gap-limit clip (reading R1)."""
    return int(_load().orc_band_width(ctypes.byref(_params(params)), n, params.w if w is None else w))


def extend_one(params, q, t, h0: int, w: int | None = None, flags: int = 0):
    """One extension of query codes q against target codes t.

    Returns (dict of the six result fields, cells, stale non-zero reads)."""
    q = np.ascontiguousarray(q, np.uint8)
    t = np.ascontiguousarray(t, np.uint8)
    res = _Result()
    cells = ctypes.c_int64()
    stale = ctypes.c_int64()
    rc = _load().orc_extend_one(ctypes.byref(_params(params, flags)), len(q), q.ctypes.data, len(t),
                                t.ctypes.data, int(h0), params.w if w is None else int(w),
                                ctypes.byref(res), ctypes.byref(cells), ctypes.byref(stale))
    if rc != 0:
        raise MemoryError("oracle: allocation failed")
    return {k: getattr(res, k) for k in FIELDS}, cells.value, stale.value


def extend_batch(wl, flags: int = 0, nthreads: int = 1, w_override=None, params=None):
    """All pairs of a workload.  Returns (results int32[N, 6], cells int64[N], stale int64[N])."""
    p = _params(params or wl.params, flags)
    n = wl.n_pairs
    res = np.zeros((n, 6), np.int32)
    cells = np.zeros(n, np.int64)
    stale = np.zeros(n, np.int64)
    wo = None
    if w_override is not None:
        wo = np.ascontiguousarray(w_override, np.int32)
    arrs = [np.ascontiguousarray(x) for x in (wl.q, wl.q_off, wl.q_len, wl.t, wl.t_off, wl.t_len, wl.h0)]
    rc = _load().orc_extend_batch(ctypes.byref(p), n, *[a.ctypes.data for a in arrs],
                                  None if wo is None else wo.ctypes.data,
                                  res.ctypes.data, cells.ctypes.data, stale.ctypes.data, int(nthreads))
    if rc != 0:
        raise MemoryError("oracle: allocation failed")
    return res, cells, stale
