"""Suffix array lookup on the GPU (bsw_sal_lookup) against Eq. 1 on the
oracle's suffix array; needs a GPU."""
import numpy as np
import pytest

from oracle import sal
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


@pytest.fixture(scope="module")
def index():
    s = W.reference()[:2_000_000]
    return sal.suffix_array(s)


def intervals(n_sa, count, seed):
    rng = np.random.default_rng(seed)
    cnt = np.minimum(rng.geometric(0.25, count), 600).astype(np.int32)
    cnt[::17] = 0
    k = rng.integers(0, n_sa - cnt, dtype=np.int64)
    k[::29] = n_sa - cnt[::29]          # intervals ending at the last entry
    return k, cnt


def test_host_lookup(bsw, index):
    k, cnt = intervals(index.shape[0], 50_000, 1)
    with bsw.Context(W.Params()) as ctx:
        ctx.sal_set_index(index)
        got = ctx.sal_lookup(k, cnt)
    np.testing.assert_array_equal(got, sal.lookup(index, k, cnt))


def test_device_lookup(bsw, index):
    import torch
    k, cnt = intervals(index.shape[0], 80_000, 2)
    off = np.zeros(k.shape[0], np.int64)
    np.cumsum(cnt[:-1], out=off[1:])
    with bsw.Context(W.Params()) as ctx:
        ctx.sal_set_index(index)
        dk, dc, do = (torch.from_numpy(x).cuda() for x in (k, cnt, off))
        out = torch.full((int(cnt.sum()),), -1, dtype=torch.int32, device="cuda")
        ctx.sal_lookup_device(dk, dc, do, out)
        ctx.sync()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), sal.lookup(index, k, cnt))


def test_errors(bsw, index):
    import torch
    with bsw.Context(W.Params()) as ctx:
        with pytest.raises(bsw.BswError) as ei:
            ctx.sal_lookup(np.array([0]), np.array([1]))          # no index yet
        assert ei.value.code == bsw.BSW_ESTATE
        ctx.sal_set_index(index)
        n = index.shape[0]
        with pytest.raises(bsw.BswError) as ei:
            ctx.sal_lookup(np.array([n - 2]), np.array([3]))      # past the end
        assert ei.value.code == bsw.BSW_EINVAL
        # device pointers: the bad interval is skipped and reported by bsw_sync
        dk = torch.tensor([0, n - 2], dtype=torch.int64, device="cuda")
        dc = torch.tensor([2, 3], dtype=torch.int32, device="cuda")
        do = torch.tensor([0, 2], dtype=torch.int64, device="cuda")
        out = torch.full((5,), -1, dtype=torch.int32, device="cuda")
        ctx.sal_lookup_device(dk, dc, do, out)
        with pytest.raises(bsw.BswError) as ei:
            ctx.sync()
        assert ei.value.code == bsw.BSW_EINVAL
        assert out[:2].cpu().tolist() == index[:2].tolist() and out[2:].cpu().tolist() == [-1, -1, -1]
        np.testing.assert_array_equal(ctx.sal_lookup(np.array([5]), np.array([4])), index[5:9])


@pytest.mark.parametrize("layout", ["reversed", "gaps", "short_only"])
def test_device_lookup_output_layouts(bsw, index, layout):
    """Outputs placed at arbitrary offsets (intervals in reverse order, gaps
    between them), and consecutive outputs of short intervals only: each
    interval's positions land at its own offset, nothing else is written."""
    import torch
    k, cnt = intervals(index.shape[0], 40_000, 3)
    if layout == "short_only":
        cnt = np.minimum(cnt, 32).astype(np.int32)
    if layout == "reversed":
        off = np.zeros(k.shape[0], np.int64)
        np.cumsum(cnt[::-1][:-1], out=off[1:])
        off = off[::-1].copy()
        total = int(cnt.sum())
    elif layout == "gaps":
        gap = np.random.default_rng(4).integers(0, 3, k.shape[0])
        off = np.zeros(k.shape[0], np.int64)
        np.cumsum((cnt + gap)[:-1], out=off[1:])
        total = int(off[-1] + cnt[-1])
    else:
        off = np.zeros(k.shape[0], np.int64)
        np.cumsum(cnt[:-1], out=off[1:])
        total = int(cnt.sum())
    want = np.full(total, -1, np.int32)
    for a, c, o in zip(k, cnt, off):
        want[o:o + c] = index[a:a + c]
    with bsw.Context(W.Params()) as ctx:
        ctx.sal_set_index(index)
        dk, dc, do = (torch.from_numpy(x).cuda() for x in (k, cnt, off))
        out = torch.full((total,), -1, dtype=torch.int32, device="cuda")
        ctx.sal_lookup_device(dk, dc, do, out)
        ctx.sync()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), want)
