"""Python binding of the BSW C ABI (include/bsw.h): argument marshalling only.

Every function named like the C ABI calls it directly through ctypes; every
step of the extension runs in the library's CUDA kernels.  The library must
have been built (``paper_1907_12931_gb300.build.build()``); there is no
fallback of any kind, and a missing library raises at load time.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from .build import LIB

BSW_OK = 0
BSW_PENDING = 1
BSW_EINVAL = -1
BSW_ENOMEM = -2
BSW_EBUDGET = -3
BSW_ECUDA = -4
BSW_ETIMEOUT = -5
BSW_ENOTFOUND = -6
BSW_ESTATE = -7
BSW_MAX_QLEN = 32768

BSW_DEVICE_PTRS = 0x01
BSW_FORCE_I8 = 0x02
BSW_FORCE_I16 = 0x04
BSW_FORCE_I32 = 0x08
BSW_PLAIN_KERNEL = 0x10
BSW_NO_GRAPH = 0x20
BSW_COPY_INPUTS = 0x40
BSW_PACKED_PAIRS = 0x80
BSW_TIME_KERNELS = 0x100
BSW_PLAIN_GLOBAL = 0x200

BSW_FAULT_ALLOC = 0x01
BSW_FAULT_H2D = 0x02
BSW_FAULT_LAUNCH = 0x04
BSW_FAULT_THREAD = 0x08
BSW_FAULT_HOST = 0x10

# class_ms indices of bsw_timing_t
CLASS_NAMES = ("u8<256>", "u8<224>", "u8<192>", "u8<160>", "u8<128>", "u8<96>", "u8<64>", "u8<32>",
               "i16<256>", "i16<128>", "i16<64>", "i16<32>", "cta16", "warp16", "warp32", "rerun32")

FIELDS = ("score", "qle", "tle", "gtle", "gscore", "max_off")


class BswError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__("%s: %s (%d)" % (where, bsw_strerror(code), code))
        self.code = code


class bsw_scoring_t(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int32) for k in ("match", "mismatch", "o_del", "e_del", "o_ins", "e_ins")]


class bsw_result_t(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int32) for k in FIELDS]


class bsw_batch_t(ctypes.Structure):
    _fields_ = [("n_pairs", ctypes.c_int64),
                ("q", ctypes.c_void_p), ("q_off", ctypes.c_void_p), ("q_len", ctypes.c_void_p),
                ("t", ctypes.c_void_p), ("t_off", ctypes.c_void_p), ("t_len", ctypes.c_void_p),
                ("h0", ctypes.c_void_p), ("w_override", ctypes.c_void_p), ("flags", ctypes.c_uint32),
                ("q_n", ctypes.c_void_p), ("t_n", ctypes.c_void_p)]


class bsw_plan_t(ctypes.Structure):
    _fields_ = [("short_max", ctypes.c_int32), ("u8_bounds", ctypes.c_uint32), ("i16_bounds", ctypes.c_uint32),
                ("packed", ctypes.c_int32), ("warp_cols", ctypes.c_int32), ("inter_warps", ctypes.c_int32),
                ("cta_min", ctypes.c_int32), ("warp_x2", ctypes.c_int32), ("ms", ctypes.c_float)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class bsw_seed_t(ctypes.Structure):
    _fields_ = [("read_id", ctypes.c_int32), ("qbeg", ctypes.c_int32), ("len", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("rbeg", ctypes.c_int64)]


class bsw_aln_t(ctypes.Structure):
    _fields_ = [("qb", ctypes.c_int32), ("qe", ctypes.c_int32), ("rb", ctypes.c_int64), ("re", ctypes.c_int64),
                ("score", ctypes.c_int32), ("w_left", ctypes.c_int32), ("w_right", ctypes.c_int32),
                ("kept", ctypes.c_int32)]


SMEM_DTYPE = np.dtype([("read_id", "<i4"), ("qbeg", "<i4"), ("len", "<i4"), ("reserved", "<i4"), ("k", "<i8"),
                       ("s", "<i8")])
SEED_DTYPE = np.dtype([("read_id", "<i4"), ("qbeg", "<i4"), ("len", "<i4"), ("reserved", "<i4"), ("rbeg", "<i8")])
ALN_DTYPE = np.dtype([("qb", "<i4"), ("qe", "<i4"), ("rb", "<i8"), ("re", "<i8"), ("score", "<i4"),
                      ("w_left", "<i4"), ("w_right", "<i4"), ("kept", "<i4")])


class bsw_serve_stats_t(ctypes.Structure):
    _fields_ = [("requests", ctypes.c_int64), ("launches", ctypes.c_int64), ("merged", ctypes.c_int64),
                ("budget_waits", ctypes.c_int64), ("busy_ms", ctypes.c_double), ("union_ms", ctypes.c_double),
                ("max_concurrent", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class bsw_timing_t(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int32), ("class_ms", ctypes.c_float * 16)]


_lib = None
_lock = threading.Lock()


def lib():
    """The loaded libbsw.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB):
                raise RuntimeError("libbsw.so is not built (%s); run paper_1907_12931_gb300.build.build()" % LIB)
            L = ctypes.CDLL(LIB)
            vp, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
            L.bsw_init.argtypes = [ctypes.POINTER(bsw_scoring_t), i32, i32, i32, i64, ctypes.POINTER(vp)]
            L.bsw_init.restype = ctypes.c_int
            L.bsw_extend_batch.argtypes = [vp, ctypes.POINTER(bsw_batch_t), vp, vp, vp]
            L.bsw_extend_batch.restype = ctypes.c_int
            L.bsw_sync.argtypes = [vp, vp]
            L.bsw_sync.restype = ctypes.c_int
            L.bsw_stream_submit.argtypes = [vp, ctypes.POINTER(bsw_batch_t), vp, ctypes.POINTER(u64)]
            L.bsw_stream_submit.restype = ctypes.c_int
            L.bsw_stream_poll.argtypes = [vp, u64, i32]
            L.bsw_stream_poll.restype = ctypes.c_int
            L.bsw_strerror.argtypes = [ctypes.c_int]
            L.bsw_strerror.restype = ctypes.c_char_p
            L.bsw_destroy.argtypes = [vp]
            L.bsw_destroy.restype = None
            L.bsw_pack_2bit.argtypes = [vp, i64, vp]
            L.bsw_pack_2bit.restype = ctypes.c_int
            L.bsw_pack_2bit_n.argtypes = [vp, i64, vp, vp]
            L.bsw_pack_2bit_n.restype = ctypes.c_int
            L.bsw_band_width.argtypes = [vp, i32, i32]
            L.bsw_band_width.restype = i32
            L.bsw_extend_batch_noalloc.argtypes = [ctypes.POINTER(bsw_scoring_t), i32, i32, i32,
                                                   ctypes.POINTER(bsw_batch_t), vp, vp, vp]
            L.bsw_extend_batch_noalloc.restype = ctypes.c_int
            L.bsw_version.argtypes = []
            L.bsw_version.restype = ctypes.c_char_p
            L.bsw_get_plan.argtypes = [vp, ctypes.POINTER(bsw_plan_t)]
            L.bsw_get_plan.restype = ctypes.c_int
            L.bsw_set_plan.argtypes = [vp, ctypes.POINTER(bsw_plan_t)]
            L.bsw_set_plan.restype = ctypes.c_int
            L.bsw_autotune.argtypes = [vp, ctypes.POINTER(bsw_batch_t), i64, i32, ctypes.POINTER(bsw_plan_t)]
            L.bsw_autotune.restype = ctypes.c_int
            L.bsw_kernel_times.argtypes = [vp, ctypes.POINTER(bsw_timing_t)]
            L.bsw_kernel_times.restype = ctypes.c_int
            L.bsw_sa_build.argtypes = [vp, i64, vp]
            L.bsw_sa_build.restype = ctypes.c_int
            L.bsw_sal_set_index.argtypes = [vp, vp, i64]
            L.bsw_sal_set_index.restype = ctypes.c_int
            L.bsw_sal_lookup.argtypes = [vp, i64, vp, vp, vp, vp, ctypes.c_uint32, vp]
            L.bsw_sal_lookup.restype = ctypes.c_int
            L.bsw_fm_build.argtypes = [vp, vp, i64]
            L.bsw_fm_build.restype = ctypes.c_int
            L.bsw_smem.argtypes = [vp, i64, vp, vp, vp, i32, vp, i64, vp, vp]
            L.bsw_smem.restype = ctypes.c_int
            L.bsw_smem_n.argtypes = [vp, i64, vp, vp, vp, vp, i32, vp, i64, vp, vp]
            L.bsw_smem_n.restype = ctypes.c_int
            L.bsw_set_reference.argtypes = [vp, vp, i64]
            L.bsw_set_reference.restype = ctypes.c_int
            L.bsw_extend_seeds.argtypes = [vp, i64, vp, vp, vp, i64, vp, i32, vp, vp]
            L.bsw_extend_seeds.restype = ctypes.c_int
            L.bsw_set_reference_n.argtypes = [vp, vp, vp, i64]
            L.bsw_set_reference_n.restype = ctypes.c_int
            L.bsw_extend_seeds_n.argtypes = [vp, i64, vp, vp, vp, vp, i64, vp, i32, vp, vp]
            L.bsw_extend_seeds_n.restype = ctypes.c_int
            L.bsw_partition.argtypes = [ctypes.POINTER(bsw_scoring_t), i32, i32, vp, vp, vp, i64, i32, vp]
            L.bsw_partition.restype = ctypes.c_int
            L.bsw_stream_stats.argtypes = [vp, ctypes.POINTER(bsw_serve_stats_t), i32]
            L.bsw_stream_stats.restype = ctypes.c_int
            L.bsw_fault_inject.argtypes = [ctypes.c_char_p]
            L.bsw_fault_inject.restype = ctypes.c_int
            _lib = L
    return _lib


# ------------------------------------------------------------ C ABI, by name

def bsw_strerror(code: int) -> str:
    return lib().bsw_strerror(int(code)).decode()


def bsw_version() -> str:
    return lib().bsw_version().decode()


def bsw_init(scoring, w: int, zdrop: int, end_bonus: int, mem_budget_bytes: int) -> int:
    """Returns the context handle (an integer pointer)."""
    sc = bsw_scoring_t(scoring.match, scoring.mismatch, scoring.o_del, scoring.e_del, scoring.o_ins, scoring.e_ins)
    h = ctypes.c_void_p()
    rc = lib().bsw_init(ctypes.byref(sc), int(w), int(zdrop), int(end_bonus), int(mem_budget_bytes), ctypes.byref(h))
    if rc != BSW_OK:
        raise BswError(rc, "bsw_init")
    return h.value


def bsw_destroy(ctx: int) -> None:
    lib().bsw_destroy(ctx)


def bsw_extend_batch(ctx: int, batch: bsw_batch_t, out_ptr: int, cells_ptr: int | None, stream: int | None) -> int:
    return lib().bsw_extend_batch(ctx, ctypes.byref(batch), out_ptr, cells_ptr, stream)


def bsw_extend_batch_noalloc(scoring, w: int, zdrop: int, end_bonus: int, batch: bsw_batch_t, out_ptr: int,
                             cells_ptr: int | None, stream: int | None) -> int:
    """The allocation-free variant (device pointers only); returns the C return code."""
    sc = bsw_scoring_t(scoring.match, scoring.mismatch, scoring.o_del, scoring.e_del, scoring.o_ins, scoring.e_ins)
    return lib().bsw_extend_batch_noalloc(ctypes.byref(sc), int(w), int(zdrop), int(end_bonus), ctypes.byref(batch),
                                          out_ptr, cells_ptr, stream)


BSW_NOALLOC_MAX_PAIRS = 262144
BSW_NOALLOC_MAX_QLEN = 256


def bsw_sync(ctx: int, stream: int | None = None) -> int:
    return lib().bsw_sync(ctx, stream)


def bsw_stream_submit(ctx: int, batch: bsw_batch_t, out_ptr: int) -> tuple[int, int]:
    t = ctypes.c_uint64()
    rc = lib().bsw_stream_submit(ctx, ctypes.byref(batch), out_ptr, ctypes.byref(t))
    return rc, t.value


def bsw_stream_poll(ctx: int, ticket: int, timeout_us: int) -> int:
    return lib().bsw_stream_poll(ctx, int(ticket), int(timeout_us))


def bsw_pack_2bit(codes: np.ndarray) -> np.ndarray:
    codes = np.ascontiguousarray(codes, np.uint8)
    out = np.zeros((codes.shape[0] + 3) // 4, np.uint8)
    rc = lib().bsw_pack_2bit(codes.ctypes.data, codes.shape[0], out.ctypes.data)
    if rc != BSW_OK:
        raise BswError(rc, "bsw_pack_2bit")
    return out


def bsw_pack_2bit_n(codes: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Codes 0..4 (4 = N): the 2-bit packing and the N bitmap."""
    codes = np.ascontiguousarray(codes, np.uint8)
    out = np.zeros((codes.shape[0] + 3) // 4, np.uint8)
    nm = np.zeros((codes.shape[0] + 7) // 8, np.uint8)
    rc = lib().bsw_pack_2bit_n(codes.ctypes.data, codes.shape[0], out.ctypes.data, nm.ctypes.data)
    if rc != BSW_OK:
        raise BswError(rc, "bsw_pack_2bit_n")
    return out, nm


def _pack(codes: np.ndarray):
    """Packed codes and an N bitmap, or None when there is no N."""
    codes = np.ascontiguousarray(codes, np.uint8)
    if codes.size and int(codes.max()) > 3:
        return bsw_pack_2bit_n(codes)
    return bsw_pack_2bit(codes), None


def bsw_band_width(ctx: int, qlen: int, w: int) -> int:
    return int(lib().bsw_band_width(ctx, int(qlen), int(w)))


def bsw_get_plan(ctx: int) -> bsw_plan_t:
    p = bsw_plan_t()
    rc = lib().bsw_get_plan(ctx, ctypes.byref(p))
    if rc != BSW_OK:
        raise BswError(rc, "bsw_get_plan")
    return p


def bsw_set_plan(ctx: int, plan: bsw_plan_t) -> int:
    return lib().bsw_set_plan(ctx, ctypes.byref(plan))


def bsw_autotune(ctx: int, batch: bsw_batch_t, sample_pairs: int, reps: int) -> tuple[int, bsw_plan_t]:
    p = bsw_plan_t()
    rc = lib().bsw_autotune(ctx, ctypes.byref(batch), int(sample_pairs), int(reps), ctypes.byref(p))
    return rc, p


def bsw_kernel_times(ctx: int) -> tuple[int, bsw_timing_t]:
    t = bsw_timing_t()
    rc = lib().bsw_kernel_times(ctx, ctypes.byref(t))
    return rc, t


def bsw_set_reference(ctx: int, ref_packed: np.ndarray, ref_len: int) -> int:
    return lib().bsw_set_reference(ctx, ref_packed.ctypes.data, int(ref_len))


def bsw_set_reference_n(ctx: int, ref_packed: np.ndarray, ref_n, ref_len: int) -> int:
    return lib().bsw_set_reference_n(ctx, ref_packed.ctypes.data, None if ref_n is None else ref_n.ctypes.data,
                                     int(ref_len))


def bsw_extend_seeds_n(ctx: int, n_reads: int, reads, reads_n, read_off, read_len, seeds, max_band_try: int, out,
                       cells) -> int:
    return lib().bsw_extend_seeds_n(ctx, int(n_reads), reads.ctypes.data,
                                    None if reads_n is None else reads_n.ctypes.data, read_off.ctypes.data,
                                    read_len.ctypes.data, int(seeds.shape[0]), seeds.ctypes.data, int(max_band_try),
                                    out.ctypes.data, ctypes.addressof(cells))


def bsw_extend_seeds(ctx: int, n_reads: int, reads, read_off, read_len, seeds, max_band_try: int, out,
                     cells) -> int:
    return lib().bsw_extend_seeds(ctx, int(n_reads), reads.ctypes.data, read_off.ctypes.data, read_len.ctypes.data,
                                  int(seeds.shape[0]), seeds.ctypes.data, int(max_band_try), out.ctypes.data,
                                  ctypes.addressof(cells))


def bsw_partition(params, q_len, t_len, parts: int, w_override=None) -> np.ndarray:
    """Contiguous pair ranges balanced by band area for `parts` devices:
    bounds[parts + 1] with part k = pairs [bounds[k], bounds[k+1])."""
    sc = params.scoring
    s = bsw_scoring_t(sc.match, sc.mismatch, sc.o_del, sc.e_del, sc.o_ins, sc.e_ins)
    ql = np.ascontiguousarray(q_len, np.int32)
    tl = np.ascontiguousarray(t_len, np.int32)
    wo = None if w_override is None else np.ascontiguousarray(w_override, np.int32)
    bounds = np.zeros(int(parts) + 1, np.int64)
    rc = lib().bsw_partition(ctypes.byref(s), int(params.w), int(params.end_bonus), ql.ctypes.data, tl.ctypes.data,
                             None if wo is None else wo.ctypes.data, ql.shape[0], int(parts), bounds.ctypes.data)
    if rc != BSW_OK:
        raise BswError(rc, "bsw_partition")
    return bounds


def bsw_fault_inject(spec: str | None) -> int:
    """Arm host-side fault injection ("alloc,h2d:skip:count"; None disarms)."""
    return lib().bsw_fault_inject(None if spec is None else spec.encode())


def bsw_sa_build(codes: np.ndarray) -> np.ndarray:
    """Suffix array of codes (0..3) + terminator: n + 1 int32 entries."""
    codes = np.ascontiguousarray(codes, np.uint8)
    sa = np.zeros(codes.shape[0] + 1, np.int32)
    rc = lib().bsw_sa_build(codes.ctypes.data, codes.shape[0], sa.ctypes.data)
    if rc != BSW_OK:
        raise BswError(rc, "bsw_sa_build")
    return sa


def make_plan(short_max=256, u8_bounds=0xff, i16_bounds=0xf, packed=0, warp_cols=8, inter_warps=2,
              cta_min=0, warp_x2=0) -> bsw_plan_t:
    return bsw_plan_t(short_max, u8_bounds, i16_bounds, packed, warp_cols, inter_warps, cta_min, warp_x2, 0.0)


# --------------------------------------------------------------- marshalling

class HostBatch:
    """Packed, host-resident inputs of a workload (numpy arrays kept alive)."""

    def __init__(self, wl, w_override=None, flags: int = 0):
        self.q, self.q_n = _pack(wl.q)
        self.t, self.t_n = _pack(wl.t)
        # own copies: the caller's arrays are never aliased
        self.q_off = np.array(wl.q_off, np.int64, copy=True, order="C")
        self.q_len = np.array(wl.q_len, np.int32, copy=True, order="C")
        self.t_off = np.array(wl.t_off, np.int64, copy=True, order="C")
        self.t_len = np.array(wl.t_len, np.int32, copy=True, order="C")
        self.h0 = np.array(wl.h0, np.int32, copy=True, order="C")
        self.w = None if w_override is None else np.array(w_override, np.int32, copy=True, order="C")
        self.n = int(self.q_len.shape[0])
        self.flags = flags

    def struct(self, flags: int | None = None) -> bsw_batch_t:
        f = self.flags if flags is None else flags
        return bsw_batch_t(self.n, self.q.ctypes.data, self.q_off.ctypes.data, self.q_len.ctypes.data,
                           self.t.ctypes.data, self.t_off.ctypes.data, self.t_len.ctypes.data,
                           self.h0.ctypes.data, None if self.w is None else self.w.ctypes.data, f,
                           None if self.q_n is None else self.q_n.ctypes.data,
                           None if self.t_n is None else self.t_n.ctypes.data)

    def nbytes(self) -> int:
        return sum(a.nbytes for a in (self.q, self.t, self.q_off, self.q_len, self.t_off, self.t_len, self.h0,
                                      self.q_n, self.t_n) if a is not None)


class DeviceBatch:
    """The same inputs as torch CUDA tensors, plus device result buffers."""

    def __init__(self, hb: HostBatch, device="cuda"):
        import torch
        self.n = hb.n
        self.q = torch.from_numpy(hb.q).to(device)
        self.t = torch.from_numpy(hb.t).to(device)
        self.q_off = torch.from_numpy(hb.q_off).to(device)
        self.q_len = torch.from_numpy(hb.q_len).to(device)
        self.t_off = torch.from_numpy(hb.t_off).to(device)
        self.t_len = torch.from_numpy(hb.t_len).to(device)
        self.h0 = torch.from_numpy(hb.h0).to(device)
        self.w = None if hb.w is None else torch.from_numpy(hb.w).to(device)
        self.q_n = None if hb.q_n is None else torch.from_numpy(hb.q_n).to(device)
        self.t_n = None if hb.t_n is None else torch.from_numpy(hb.t_n).to(device)
        self.out = torch.zeros((self.n, 6), dtype=torch.int32, device=device)
        self.cells = torch.zeros(1, dtype=torch.int64, device=device)

    def struct(self, flags: int = 0) -> bsw_batch_t:
        return bsw_batch_t(self.n, self.q.data_ptr(), self.q_off.data_ptr(), self.q_len.data_ptr(),
                           self.t.data_ptr(), self.t_off.data_ptr(), self.t_len.data_ptr(), self.h0.data_ptr(),
                           None if self.w is None else self.w.data_ptr(), flags | BSW_DEVICE_PTRS,
                           None if self.q_n is None else self.q_n.data_ptr(),
                           None if self.t_n is None else self.t_n.data_ptr())


class Context:
    """Owns a bsw_ctx_t."""

    def __init__(self, params, mem_budget_bytes: int = 8 << 30):
        self.params = params
        self.handle = bsw_init(params.scoring, params.w, params.zdrop, params.end_bonus, mem_budget_bytes)

    def close(self):
        if self.handle:
            bsw_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def extend_host(self, hb: HostBatch, flags: int = 0, stream: int | None = None, out: np.ndarray | None = None):
        """Host inputs -> (results int32 [N, 6], cells).  `out`, if given, is a
        C-contiguous int32 [N, 6] array that receives the results (pinned
        memory makes the copy back faster)."""
        if out is None:
            out = np.zeros((hb.n, 6), np.int32)
        elif out.dtype != np.int32 or out.shape != (hb.n, 6) or not out.flags["C_CONTIGUOUS"]:
            raise ValueError("out must be a C-contiguous int32 array of shape (%d, 6)" % hb.n)
        cells = ctypes.c_int64()
        rc = bsw_extend_batch(self.handle, hb.struct(hb.flags | flags), out.ctypes.data,
                              ctypes.addressof(cells), stream)
        if rc != BSW_OK:
            raise BswError(rc, "bsw_extend_batch")
        return out, cells.value

    def extend_device(self, db: DeviceBatch, flags: int = 0, stream: int | None = None):
        """Device inputs; enqueues on `stream` (a cudaStream_t as int) and returns."""
        rc = bsw_extend_batch(self.handle, db.struct(flags), db.out.data_ptr(), db.cells.data_ptr(), stream)
        if rc != BSW_OK:
            raise BswError(rc, "bsw_extend_batch")

    def sync(self, stream: int | None = None):
        rc = bsw_sync(self.handle, stream)
        if rc != BSW_OK:
            raise BswError(rc, "bsw_sync")

    def submit(self, hb: HostBatch, out: np.ndarray, flags: int = 0) -> int:
        rc, ticket = bsw_stream_submit(self.handle, hb.struct(hb.flags | flags), out.ctypes.data)
        if rc != BSW_OK:
            raise BswError(rc, "bsw_stream_submit")
        return ticket

    def poll(self, ticket: int, timeout_us: int = -1) -> int:
        return bsw_stream_poll(self.handle, ticket, timeout_us)

    def stream_stats(self, reset: bool = False) -> dict:
        st = bsw_serve_stats_t()
        rc = lib().bsw_stream_stats(self.handle, ctypes.byref(st), 1 if reset else 0)
        if rc != BSW_OK:
            raise BswError(rc, "bsw_stream_stats")
        return st.as_dict()

    def get_plan(self) -> bsw_plan_t:
        return bsw_get_plan(self.handle)

    def set_plan(self, plan: bsw_plan_t) -> None:
        rc = bsw_set_plan(self.handle, plan)
        if rc != BSW_OK:
            raise BswError(rc, "bsw_set_plan")

    def autotune(self, batch, sample_pairs: int = 0, reps: int = 0) -> bsw_plan_t:
        """Tune the plan on a HostBatch or DeviceBatch; returns the chosen plan."""
        rc, p = bsw_autotune(self.handle, batch.struct(0), sample_pairs, reps)
        if rc != BSW_OK:
            raise BswError(rc, "bsw_autotune")
        return p

    def kernel_times(self) -> tuple[int, list]:
        """(launches, per-class ms) of the last call made with BSW_TIME_KERNELS."""
        rc, t = bsw_kernel_times(self.handle)
        if rc != BSW_OK:
            raise BswError(rc, "bsw_kernel_times")
        return t.launches, list(t.class_ms)

    def fm_build(self, ref_codes: np.ndarray) -> None:
        ref = np.ascontiguousarray(ref_codes, np.uint8)
        rc = lib().bsw_fm_build(self.handle, ref.ctypes.data, ref.shape[0])
        if rc != BSW_OK:
            raise BswError(rc, "bsw_fm_build")

    def smem(self, reads_packed, read_off, read_len, min_len: int = 19, cap: int | None = None, reads_n=None):
        """SMEMs of packed reads (reads_n: their N bitmap, or None).  Returns
        (structured records, first[n_reads + 1])."""
        read_off = np.ascontiguousarray(read_off, np.int64)
        read_len = np.ascontiguousarray(read_len, np.int32)
        n = read_len.shape[0]
        first = np.zeros(n + 1, np.int64)
        n_out = ctypes.c_int64()
        cap = 4 * n + 16 if cap is None else cap
        while True:
            out = np.zeros(cap, SMEM_DTYPE)
            rc = lib().bsw_smem_n(self.handle, n, reads_packed.ctypes.data,
                                  None if reads_n is None else reads_n.ctypes.data, read_off.ctypes.data,
                                  read_len.ctypes.data, int(min_len), out.ctypes.data, cap, ctypes.addressof(n_out),
                                  first.ctypes.data)
            if rc == BSW_EBUDGET and n_out.value > cap:
                cap = int(n_out.value)
                continue
            if rc != BSW_OK:
                raise BswError(rc, "bsw_smem_n")
            return out[:n_out.value], first

    def sal_set_index(self, sa: np.ndarray) -> None:
        sa = np.ascontiguousarray(sa, np.int32)
        rc = lib().bsw_sal_set_index(self.handle, sa.ctypes.data, sa.shape[0])
        if rc != BSW_OK:
            raise BswError(rc, "bsw_sal_set_index")

    def sal_lookup(self, k: np.ndarray, cnt: np.ndarray) -> np.ndarray:
        """Host intervals -> the concatenated positions S[k[t] .. k[t] + cnt[t])."""
        k = np.ascontiguousarray(k, np.int64)
        cnt = np.ascontiguousarray(cnt, np.int32)
        off = np.zeros(k.shape[0], np.int64)
        if k.shape[0] > 1:
            np.cumsum(cnt[:-1], out=off[1:])
        out = np.zeros(int(cnt.sum()), np.int32)
        rc = lib().bsw_sal_lookup(self.handle, k.shape[0], k.ctypes.data, cnt.ctypes.data, off.ctypes.data,
                                  out.ctypes.data, 0, None)
        if rc != BSW_OK:
            raise BswError(rc, "bsw_sal_lookup")
        return out

    def sal_lookup_device(self, k, cnt, off, out, stream: int | None = None) -> None:
        """Device intervals (torch tensors): enqueue the gather into out."""
        rc = lib().bsw_sal_lookup(self.handle, k.shape[0], k.data_ptr(), cnt.data_ptr(), off.data_ptr(),
                                  out.data_ptr(), BSW_DEVICE_PTRS, stream)
        if rc != BSW_OK:
            raise BswError(rc, "bsw_sal_lookup")

    def set_reference(self, ref_codes: np.ndarray) -> None:
        """Upload a reference given as codes 0..3, or 0..4 with N (packed here)."""
        self._ref_packed, self._ref_n = _pack(ref_codes)
        rc = bsw_set_reference_n(self.handle, self._ref_packed, self._ref_n, int(ref_codes.shape[0]))
        if rc != BSW_OK:
            raise BswError(rc, "bsw_set_reference_n")

    @staticmethod
    def prepare_seeds(sw):
        """Packed reads (with an N bitmap when they hold N), offsets, lengths
        and seed records of a SeedWorkload."""
        seeds = np.zeros(sw.n_seeds, SEED_DTYPE)
        seeds["read_id"], seeds["qbeg"], seeds["len"], seeds["rbeg"] = sw.seed_read, sw.qbeg, sw.slen, sw.rbeg
        packed, reads_n = _pack(sw.reads)
        return (sw.n_reads, packed, reads_n, np.ascontiguousarray(sw.read_off, np.int64),
                np.ascontiguousarray(sw.read_len, np.int32), seeds)

    def extend_prepared(self, prep, max_band_try: int = 2, out=None):
        """bsw_extend_seeds on prepare_seeds' arrays.  Returns (alignments, cells)."""
        n_reads, reads, reads_n, read_off, read_len, seeds = prep
        if out is None:
            out = np.zeros(seeds.shape[0], ALN_DTYPE)
        cells = ctypes.c_int64()
        rc = bsw_extend_seeds_n(self.handle, n_reads, reads, reads_n, read_off, read_len, seeds, max_band_try, out,
                                cells)
        if rc != BSW_OK:
            raise BswError(rc, "bsw_extend_seeds_n")
        return out, cells.value

    def extend_seeds(self, sw, max_band_try: int = 2):
        """The driver over a SeedWorkload (reads as codes; the reference set
        with set_reference).  Returns (structured alignments, cells)."""
        return self.extend_prepared(self.prepare_seeds(sw), max_band_try)

    def band_width(self, qlen: int, w: int | None = None) -> int:
        return bsw_band_width(self.handle, qlen, self.params.w if w is None else w)
