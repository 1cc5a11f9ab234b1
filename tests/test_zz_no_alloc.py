"""bsw_extend_batch_noalloc against bsw_extend_batch and the oracle (needs a GPU).

The allocation-free entry point serves callers that may not allocate device
memory; it keeps its work buffers in one device array that every call reuses.
Two calls in a row, on different batches, must each give exactly what the
context-based entry point gives and what the CPU oracle gives, so nothing a
call leaves in the array leaks into the next.  This file is collected last on
purpose.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1907_12931_gb300 import workload as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_12931_gb300 import bsw
    bsw.lib()
    return torch, bsw


def reference(bsw, wl, flags=0):
    with bsw.Context(wl.params, 8 << 30) as ctx:
        db = bsw.DeviceBatch(bsw.HostBatch(wl))
        ctx.extend_device(db, flags)
        ctx.sync()
        return db.out.cpu().numpy(), int(db.cells.item())


def noalloc(torch, bsw, wl, flags=0):
    db = bsw.DeviceBatch(bsw.HostBatch(wl))
    db.out.fill_(-9)
    db.cells.fill_(-9)
    stream = torch.cuda.current_stream()
    p = wl.params
    rc = bsw.bsw_extend_batch_noalloc(p.scoring, p.w, p.zdrop, p.end_bonus, db.struct(flags), db.out.data_ptr(),
                                      db.cells.data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize()
    return rc, db.out.cpu().numpy(), int(db.cells.item())


def test_two_calls_in_a_row_match_extend_batch(env):
    torch, bsw = env
    a = W.make("read151", n_pairs=120_000)                       # left/right short-read pairs
    b = W.make("plain10k", n_pairs=9_000, seed=7)                 # a different, smaller batch next
    for wl in (a, b):
        ref, ref_cells = reference(bsw, wl)
        rc, got, cells = noalloc(torch, bsw, wl)
        assert rc == bsw.BSW_OK, bsw.bsw_strerror(rc)
        np.testing.assert_array_equal(got, ref)
        assert cells == ref_cells
        want, want_cells, _ = oracle.extend_batch(wl, nthreads=os.cpu_count() or 1)
        np.testing.assert_array_equal(got, want)
        assert cells == int(want_cells.sum())


def test_forced_lanes_and_limits(env):
    torch, bsw = env
    wl = W.make("read250", n_pairs=30_000)
    short = wl.subset(np.nonzero(wl.q_len <= bsw.BSW_NOALLOC_MAX_QLEN)[0])
    ref, ref_cells = reference(bsw, short, bsw.BSW_FORCE_I8)
    rc, got, cells = noalloc(torch, bsw, short, bsw.BSW_FORCE_I8)
    assert rc == bsw.BSW_OK
    np.testing.assert_array_equal(got, ref)
    assert cells == ref_cells
    # a query longer than the stated maximum is rejected
    long_wl = W.make("long10k", n_pairs=50)
    assert long_wl.q_len.max() > bsw.BSW_NOALLOC_MAX_QLEN
    rc, _, _ = noalloc(torch, bsw, long_wl)
    assert rc == bsw.BSW_EINVAL
    # too many pairs are rejected before any work
    big = bsw.bsw_batch_t(bsw.BSW_NOALLOC_MAX_PAIRS + 1, 1, 1, 1, 1, 1, 1, 1, None, bsw.BSW_DEVICE_PTRS)
    p = wl.params
    assert bsw.bsw_extend_batch_noalloc(p.scoring, p.w, p.zdrop, p.end_bonus, big, 1, None, None) == bsw.BSW_EINVAL
    # and the entry point still works after the rejections
    ref, ref_cells = reference(bsw, short)
    rc, got, cells = noalloc(torch, bsw, short)
    assert rc == bsw.BSW_OK
    np.testing.assert_array_equal(got, ref)
