"""CPU oracle of the seed-extension driver around BSW (test infrastructure:
only tests/, the smoke check and bench.py's CPU legs use it).

Section V-C2 extends every seed of a read and filters the results
afterwards, instead of extending seeds one after another; Section V-A is one
extension.  For each seed (read r, read interval [qbeg, qbeg + len),
reference start rbeg, taken as ungapped) the driver:

  1. extends left from the seed start: the read prefix [0, qbeg) reversed
     against the reference before rbeg reversed, from h0 = len * match;
  2. picks the left end (D2), giving the aligned start (qb, rb) and the left
     score;
  3. extends right from the seed end: the read suffix [qbeg + len, read_len)
     against the reference from rbeg + len, from h0 = the left score (D5);
  4. picks the right end (D2), giving (qe, re) and the score;
  5. drops seeds that an earlier alignment of the same read already covers
     (D4).

The paper leaves these points to BWA-MEM; the readings here:
  D1 a side's target is its query length + w reference bases, clipped at the
     reference ends;
  D2 the side is extended to the read end (query length, gtle, gscore) unless
     gscore <= 0 or gscore <= score - end_bonus, when the local best is kept
     (qle, tle, score);
  D3 an extension whose max_off is at least (w' >> 1) + (w' >> 2) for its
     band w' runs again with twice the band, up to max_band_try runs in all;
     the last run's result is used (the target window stays as in D1);
  D4 in the read's seed order, a seed whose read and reference intervals both
     lie inside the alignment of an earlier kept seed of the same read is not
     kept;
  D5 the right extension starts from the left score, and the alignment's
     score is the right side's chosen score.
Each step calls the BSW oracle (`oracle.extend_batch`); nothing here shares
code with the CUDA path.
"""
from __future__ import annotations

import numpy as np

import oracle
from paper_1907_12931_gb300 import workload as W


def _run_side(queries, targets, h0, params, max_band_try, nthreads):
    """BSW over one side's pairs with the band retry (D3).  Returns results
    int32[N, 6], the band of each pair's last run, and the cells of all runs."""
    n = len(queries)
    wl = W.from_lists(queries, targets, h0, params=params, align=4)
    w = params.w
    wcur = np.full(n, w, np.int32)
    res, cells, _ = oracle.extend_batch(wl, nthreads=nthreads, w_override=wcur)
    total = int(cells.sum())
    ran = np.ones(n, bool)
    for t in range(1, max_band_try):
        wt = wcur
        redo = np.nonzero(ran & (res[:, 5] >= (wt >> 1) + (wt >> 2)))[0]
        ran = np.zeros(n, bool)
        if redo.size == 0:
            break
        sub = wl.subset(redo)
        wnew = (w << t) * np.ones(redo.size, np.int32)
        r2, c2, _ = oracle.extend_batch(sub, nthreads=nthreads, w_override=wnew)
        res[redo] = r2
        wcur = wcur.copy()
        wcur[redo] = wnew
        ran[redo] = True
        total += int(c2.sum())
    return res, wcur, total


def _choose(res, qlen, end_bonus):
    """D2: query extent, target extent and score of each side."""
    score, qle, tle, gtle, gscore = (res[:, k].astype(np.int64) for k in range(5))
    local = (gscore <= 0) | (gscore <= score - end_bonus)
    qext = np.where(local, qle, qlen)
    text = np.where(local, tle, gtle)
    sc = np.where(local, score, gscore)
    return qext, text, sc


def extend_seeds(sw: W.SeedWorkload, params: W.Params | None = None, max_band_try: int = 2, nthreads: int = 1):
    """The driver over every seed of sw.  Returns a dict of arrays (one entry
    per seed): qb, qe, rb, re, score, w_left, w_right (band of the side's last
    run; 0 for an empty side), kept; and 'cells' (all BSW runs)."""
    P = params or sw.params
    a, w, eb = P.scoring.match, P.w, P.end_bonus
    ns = sw.n_seeds
    ref, rlen = sw.ref, sw.ref.shape[0]
    qb0 = sw.qbeg.astype(np.int64)
    L = sw.slen.astype(np.int64)
    rb0 = sw.rbeg.astype(np.int64)
    roff = sw.read_off[sw.seed_read].astype(np.int64)
    rl = sw.read_len[sw.seed_read].astype(np.int64)

    # 1. left side
    lq, lt = [], []
    for k in range(ns):
        o, q, r = roff[k], qb0[k], rb0[k]
        lq.append(sw.reads[o:o + q][::-1])
        tl = min(q + w, r)
        lt.append(ref[r - tl:r][::-1])
    h0l = (L * a).astype(np.int32)
    resl, wl_used, cells_l = _run_side(lq, lt, h0l, P, max_band_try, nthreads)
    qext, text, sl = _choose(resl, qb0, eb)
    qb = qb0 - qext
    rb = rb0 - text

    # 3. right side
    rq, rt = [], []
    for k in range(ns):
        o, qe, re = roff[k], qb0[k] + L[k], rb0[k] + L[k]
        rq.append(sw.reads[o + qe:o + rl[k]])
        tl = max(0, min(rl[k] - qe + w, rlen - re))
        rt.append(ref[re:re + tl])
    resr, wr_used, cells_r = _run_side(rq, rt, sl.astype(np.int32), P, max_band_try, nthreads)
    qext2, text2, sc = _choose(resr, rl - qb0 - L, eb)
    qe = qb0 + L + qext2
    re = rb0 + L + text2

    # 5. post-filter
    kept = np.ones(ns, np.int32)
    start = 0
    while start < ns:
        end = start
        while end < ns and sw.seed_read[end] == sw.seed_read[start]:
            end += 1
        for k in range(start, end):
            for j in range(start, k):
                if kept[j] and qb[j] <= qb0[k] and qb0[k] + L[k] <= qe[j] and rb[j] <= rb0[k] and rb0[k] + L[k] <= re[j]:
                    kept[k] = 0
                    break
        start = end

    return {"qb": qb.astype(np.int32), "qe": qe.astype(np.int32), "rb": rb, "re": re,
            "score": sc.astype(np.int32),
            "w_left": np.where(qb0 > 0, wl_used, 0).astype(np.int32),
            "w_right": np.where(rl - qb0 - L > 0, wr_used, 0).astype(np.int32),
            "kept": kept, "cells": cells_l + cells_r}
