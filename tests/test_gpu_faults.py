"""Host-side fault injection (needs a GPU): each injected failure returns its
documented code, and the same context then computes oracle-exact results.

Nothing here faults the GPU: bsw_fault_inject makes a host call (an
allocation, a host-to-device copy, a kernel launch, a thread start, a host
container allocation) report failure before it reaches the device.
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
    wl = W.make("read151", n_pairs=40_000)
    want, cells, _ = oracle.extend_batch(wl, nthreads=os.cpu_count() or 1)
    yield torch, bsw, wl, want, int(cells.sum())
    bsw.bsw_fault_inject(None)


def _expect(bsw, code, fn):
    with pytest.raises(bsw.BswError) as e:
        fn()
    assert e.value.code == code, bsw.bsw_strerror(e.value.code)


@pytest.mark.parametrize("site,code", [("alloc", -2), ("h2d", -4), ("launch", -4)])
def test_host_batch_recovers(env, site, code):
    torch, bsw, wl, want, cells = env
    with bsw.Context(wl.params, 4 << 30) as ctx:
        hb = bsw.HostBatch(wl)
        assert bsw.bsw_fault_inject(site) == bsw.BSW_OK
        _expect(bsw, code, lambda: ctx.extend_host(hb))
        for _ in range(2):                      # the context works, twice in a row
            got, gc = ctx.extend_host(hb)
            np.testing.assert_array_equal(got, want)
            assert gc == cells


@pytest.mark.parametrize("flags", [0, "nograph"])
def test_device_batch_recovers_from_launch_failure(env, flags):
    torch, bsw, wl, want, cells = env
    f = bsw.BSW_NO_GRAPH if flags else 0
    with bsw.Context(wl.params, 4 << 30) as ctx:
        db = bsw.DeviceBatch(bsw.HostBatch(wl))
        assert bsw.bsw_fault_inject("launch") == bsw.BSW_OK
        _expect(bsw, bsw.BSW_ECUDA, lambda: ctx.extend_device(db, f))
        db.out.fill_(-7)
        ctx.extend_device(db, f)
        ctx.sync()
        np.testing.assert_array_equal(db.out.cpu().numpy(), want)
        assert int(db.cells.item()) == cells


def test_alloc_failure_after_growth(env):
    """A failed growth of the work buffers (a larger batch than before) leaves
    the context usable for both the small and the large batch."""
    torch, bsw, wl, want, cells = env
    small = wl.subset(np.arange(2000))
    with bsw.Context(wl.params, 4 << 30) as ctx:
        got, _ = ctx.extend_host(bsw.HostBatch(small))
        np.testing.assert_array_equal(got, want[:2000])
        assert bsw.bsw_fault_inject("alloc") == bsw.BSW_OK
        _expect(bsw, bsw.BSW_ENOMEM, lambda: ctx.extend_host(bsw.HostBatch(wl)))
        got, _ = ctx.extend_host(bsw.HostBatch(small))
        np.testing.assert_array_equal(got, want[:2000])
        got, gc = ctx.extend_host(bsw.HostBatch(wl))
        np.testing.assert_array_equal(got, want)
        assert gc == cells


@pytest.mark.parametrize("spec", ["thread", "host", "host:1:1"])
def test_failed_submit_registers_nothing(env, spec):
    """A submit that fails (server thread start, ticket table, queue) returns
    BSW_ENOMEM, issues no ticket and never writes its out; the next submit
    works and gets the first ticket."""
    torch, bsw, wl, want, cells = env
    sub = wl.subset(np.arange(5000))
    hb = bsw.HostBatch(sub)
    with bsw.Context(wl.params, 4 << 30) as ctx:
        out_failed = np.full((sub.n_pairs, 6), -7, np.int32)
        assert bsw.bsw_fault_inject(spec) == bsw.BSW_OK
        rc, ticket = bsw.bsw_stream_submit(ctx.handle, hb.struct(), out_failed.ctypes.data)
        assert rc == bsw.BSW_ENOMEM and ticket == 0
        assert bsw.bsw_stream_poll(ctx.handle, 1, 0) == bsw.BSW_ENOTFOUND
        out = np.zeros((sub.n_pairs, 6), np.int32)
        t = ctx.submit(hb, out)
        assert t == 1
        assert ctx.poll(t, -1) == bsw.BSW_OK
        np.testing.assert_array_equal(out, want[:5000])
        assert (out_failed == -7).all()


@pytest.mark.parametrize("spec,code", [("alloc", -2), ("h2d", -4), ("launch", -4), ("host:2:1", 0)])
def test_serving_recovers(env, spec, code):
    """A failure inside the serving thread: the request it hits reports the
    code (an admission-list allocation is retried, so that request succeeds),
    and later requests on the same context are exact."""
    torch, bsw, wl, want, cells = env
    sub = wl.subset(np.arange(8000))
    hb = bsw.HostBatch(sub)
    with bsw.Context(wl.params, 4 << 30) as ctx:
        out = np.zeros((sub.n_pairs, 6), np.int32)
        assert bsw.bsw_fault_inject(spec) == bsw.BSW_OK
        t = ctx.submit(hb, out)
        assert ctx.poll(t, -1) == code
        if code == 0:
            np.testing.assert_array_equal(out, want[:8000])
        bsw.bsw_fault_inject(None)
        for _ in range(2):
            out = np.zeros((sub.n_pairs, 6), np.int32)
            t = ctx.submit(hb, out)
            assert ctx.poll(t, -1) == bsw.BSW_OK
            np.testing.assert_array_equal(out, want[:8000])
