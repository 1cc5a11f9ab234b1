"""The seed-extension driver (bsw_extend_seeds) against its CPU oracle
(oracle/driver.py), needs a GPU.  Every alignment field and the total cell
count must match exactly."""
import numpy as np
import pytest

from oracle import driver
from paper_1907_12931_gb300 import workload as W
from test_gpu_parity import NTH

pytestmark = pytest.mark.gpu

FIELDS = ("qb", "qe", "rb", "re", "score", "w_left", "w_right", "kept")


@pytest.fixture(scope="module")
def bsw():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_12931_gb300 import bsw as _b
    _b.lib()
    return _b


def compare(bsw, sw, params=None, tries=2, what=""):
    params = params or sw.params
    ref = driver.extend_seeds(sw, params=params, max_band_try=tries, nthreads=NTH)
    with bsw.Context(params, 16 << 30) as ctx:
        ctx.set_reference(sw.ref)
        got, cells = ctx.extend_seeds(sw, max_band_try=tries)
    for f in FIELDS:
        bad = np.nonzero(got[f] != ref[f])[0]
        if bad.size:
            k = bad[0]
            raise AssertionError("%s: field %s differs on %d of %d seeds; first %d: gpu %s oracle %s"
                                 % (what, f, bad.size, sw.n_seeds, k, got[k], {g: ref[g][k] for g in FIELDS}))
    assert cells == ref["cells"], (what, cells, ref["cells"])
    return ref


def hand_cases():
    ref = W.random_codes(21, 6000)
    reads, seeds = [], []

    def add(read, sds):
        rid = len(reads)
        reads.append(np.asarray(read, np.uint8))
        seeds.extend((rid,) + tuple(s) for s in sds)

    p = 700
    add(ref[p:p + 40], [(10, 20, p + 10)])                                  # exact read
    one = ref[300:340].copy(); one[39] = (one[39] + 1) % 4
    add(one, [(0, 20, 300)])                                                # one end mismatch
    two = ref[300:340].copy(); two[38] = (two[38] + 1) % 4; two[39] = (two[39] + 1) % 4
    add(two, [(0, 20, 300)])                                                # two end mismatches
    add(ref[0:30], [(0, 20, 0)])                                            # read and reference start
    add(np.concatenate([W.random_codes(22, 5), ref[0:30]]), [(5, 20, 0)])   # empty left target
    add(ref[1000:1060], [(5, 20, 1005), (30, 20, 1030)])                    # covered second seed
    add(ref[5940:6000], [(10, 30, 5950)])                                   # right target at reference end
    add(np.concatenate([ref[1500:1530], ref[1534:1564], ref[1566:1600]]), [(0, 20, 1500)])   # two deletions
    add(W.random_codes(23, 50), [(20, 19, 4000)])                           # unrelated read
    add(ref[2000:2000 + 19], [(0, 19, 2000)])                               # seed is the whole read
    return W.seeds_from_lists(reads, ref, seeds)


@pytest.mark.parametrize("w", [100, 4, 1])
@pytest.mark.parametrize("tries", [1, 2, 3])
def test_hand_cases(bsw, w, tries):
    sw = hand_cases()
    params = W.Params(W.Scoring(), w=w, zdrop=100, end_bonus=5)
    compare(bsw, sw, params=params, tries=tries, what="hand w=%d tries=%d" % (w, tries))


@pytest.mark.parametrize("config,n_reads", [("seeds151", 20_000), ("seeds250", 10_000)])
def test_generated_seeds(bsw, config, n_reads):
    sw = W.make_seeds(config, n_reads=n_reads)
    ref = compare(bsw, sw, what=config)
    assert ref["kept"].mean() > 0.3


def test_many_band_retries(bsw):
    """A small band against 250 bp reads with indels of up to 10 bases: many
    extensions leave the diagonal by more than 3/4 of the band and run again."""
    sw = W.make_seeds("seeds250", n_reads=4_000)
    params = W.Params(W.Scoring(), w=8, zdrop=100, end_bonus=5)
    ref = compare(bsw, sw, params=params, tries=3, what="w=8 tries=3")
    assert (ref["w_right"] > 8).sum() > 50


def test_invalid_arguments(bsw):
    sw = hand_cases()
    with bsw.Context(sw.params) as ctx:
        with pytest.raises(bsw.BswError) as ei:
            ctx.extend_seeds(sw)                                            # no reference yet
        assert ei.value.code == bsw.BSW_ESTATE
        ctx.set_reference(sw.ref)
        bad = W.SeedWorkload(sw.name, sw.params, sw.reads, sw.read_off, sw.read_len, sw.ref, sw.seed_read.copy(),
                             sw.qbeg.copy(), sw.slen.copy(), sw.rbeg.copy())
        bad.qbeg[0] = 35                                                    # seed past the read end
        with pytest.raises(bsw.BswError) as ei:
            ctx.extend_seeds(bad)
        assert ei.value.code == bsw.BSW_EINVAL
        bad = W.SeedWorkload(sw.name, sw.params, sw.reads, sw.read_off, sw.read_len, sw.ref,
                             sw.seed_read[[0, 5, 6, 0]].copy(), sw.qbeg[[0, 5, 6, 0]].copy(),
                             sw.slen[[0, 5, 6, 0]].copy(), sw.rbeg[[0, 5, 6, 0]].copy())
        with pytest.raises(bsw.BswError) as ei:
            ctx.extend_seeds(bad)                                           # read 0's seeds not consecutive
        assert ei.value.code == bsw.BSW_EINVAL
        with pytest.raises(bsw.BswError) as ei:
            ctx.extend_seeds(sw, max_band_try=0)
        assert ei.value.code == bsw.BSW_EINVAL
        got, _ = ctx.extend_seeds(sw)                                       # the context still works
        assert got.shape[0] == sw.n_seeds


def n_cases():
    """Hand cases with N in reads and reference: single N, runs, N next to
    the seed, N at the read ends, all-N read flanks."""
    sw = hand_cases()
    reads = [sw.reads[o:o + n].copy() for o, n in zip(sw.read_off, sw.read_len)]
    ref = sw.ref.copy()
    seeds = [(int(r), int(q), int(l), int(b)) for r, q, l, b in zip(sw.seed_read, sw.qbeg, sw.slen, sw.rbeg)]
    reads[0][5] = 4                                  # N in the left flank
    reads[0][35] = 4                                 # and in the right one
    reads[5][:4] = 4                                 # N at the read start
    reads[5][-3:] = 4                                # and at its end
    ref[300 + 25:300 + 33] = 4                       # an N run opposite read 1's right flank
    ref[1500 + 45:1500 + 47] = 4                     # N near the deletions of read 7
    reads[8][:] = 4                                  # an all-N read against its seed's target
    for r in reads:
        r[r.shape[0] // 2:r.shape[0] // 2 + 1] = np.where(r.shape[0] > 60, 4, r[r.shape[0] // 2])
    return W.seeds_from_lists(reads, ref, seeds)


@pytest.mark.parametrize("w,tries", [(100, 2), (4, 3), (1, 1)])
def test_n_hand_cases(bsw, w, tries):
    sw = n_cases()
    params = W.Params(W.Scoring(), w=w, zdrop=100, end_bonus=5)
    compare(bsw, sw, params=params, tries=tries, what="N hand w=%d tries=%d" % (w, tries))


@pytest.mark.parametrize("config,n_reads,w,tries", [("seeds151", 20_000, 100, 2), ("seeds250", 6_000, 8, 3)])
def test_generated_seeds_with_n(bsw, config, n_reads, w, tries):
    """N in 0.2% of the read bases outside the seeds and reference N runs
    (0.05% run starts, 1-40 bases)."""
    sw = W.inject_n_seeds(W.make_seeds(config, n_reads=n_reads), 0.002, 0.0005, seed=4)
    params = W.Params(W.Scoring(), w=w, zdrop=100, end_bonus=5)
    compare(bsw, sw, params=params, tries=tries, what="%s+N" % config)
