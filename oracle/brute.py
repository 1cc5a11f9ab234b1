"""Brute-force full-matrix DP for tiny extensions - TEST INFRASTRUCTURE ONLY.

An independent restatement of the extension used to pin the row-sweep oracle
(``bsw_oracle.c``).  Where the oracle keeps one row of H and E and updates it
in place (Section V-A, last paragraph), this module fills explicit matrices
H, E, F over every cell, with the boundaries written out as the functions of
Eq. 3, so the index bookkeeping of the one-row form is not shared.

It implements:
  * Eq. 2 with the readings R2 (zero diagonal -> M = 0) and R3 (E and F open
    from M with cost o + e) of the oracle's header;
  * Eq. 3 boundaries: H[-1,-1] = h0, first row max(0, h0 - o_ins - (j+1) e_ins),
    first column max(0, h0 - o_del - (i+1) e_del), E = F = 0 on entry;
  * optionally the static diagonal band (rule a, band width clipped by R1),
    with cells outside it absent (H = E = 0, F restarts inside the band);
  * the all-zero-row abort (rule b, first half) and optionally z-drop (R5);
  * best / global-score bookkeeping with the tie rules R4.
It does NOT implement the band adjustment after each row (rule c): that is the
heuristic the comparisons are about.

The DP runs over a batch of equally-shaped pairs at once (numpy vectors over
the batch); the loops over cells are plain Python.
"""
from __future__ import annotations

import numpy as np


def band_clip(n: int, w: int, match: int, end_bonus: int, o_ins: int, e_ins: int, o_del: int, e_del: int) -> int:
    """R1 restated: the band never exceeds the widest gap the score can pay for,
    trunc((n*match + end_bonus - o)/e + 1) for each gap type, at least 1."""
    def lim(o, e):
        num = n * match + end_bonus - o + e          # (x/e + 1) = (x + e)/e
        k = abs(num) // e * (1 if num >= 0 else -1)  # truncate toward zero
        return max(k, 1)
    return min(w, lim(o_ins, e_ins), lim(o_del, e_del))


def extend_full(params, Q: np.ndarray, T: np.ndarray, H0: np.ndarray, band: bool = False,
                zdrop: bool = False, w: int | None = None):
    """Q: [B, n] codes, T: [B, m] codes, H0: [B].  Returns int64 [B, 6]
    (score, qle, tle, gtle, gscore, max_off)."""
    s = params.scoring
    Q = np.asarray(Q, np.int64)
    T = np.asarray(T, np.int64)
    H0 = np.asarray(H0, np.int64)
    B, n = Q.shape
    m = T.shape[1]
    out = np.zeros((B, 6), np.int64)
    if n == 0:                                   # R7
        out[:, 0] = H0
        out[:, 4] = H0
        return out
    oe_d, oe_i = s.o_del + s.e_del, s.o_ins + s.e_ins
    wb = band_clip(n, params.w if w is None else w, s.match, params.end_bonus,
                   s.o_ins, s.e_ins, s.o_del, s.e_del) if band else None

    def in_band(i, j):
        return wb is None or (i - wb <= j <= i + wb)

    def top(j):      # H at row -1, column j (Eq. 3 first row, column j+1)
        return np.maximum(0, H0 - s.o_ins - (j + 1) * s.e_ins)

    def left(i):     # H at row i, column -1 (Eq. 3 first column, row i+1)
        return np.maximum(0, H0 - s.o_del - (i + 1) * s.e_del)

    H = np.zeros((m, n, B), np.int64)
    E = np.zeros((m + 1, n, B), np.int64)        # E[i] enters row i; E[0] = 0
    Mm = np.zeros((m, n, B), np.int64)

    best = H0.copy()
    bi = np.full(B, -1, np.int64)
    bj = np.full(B, -1, np.int64)
    gbest = np.full(B, -1, np.int64)
    gi = np.full(B, -1, np.int64)
    moff = np.zeros(B, np.int64)
    alive = np.ones(B, bool)

    for i in range(m):
        F = np.zeros(B, np.int64)
        rm = np.zeros(B, np.int64)
        rj = np.full(B, -1, np.int64)
        for j in range(n):
            if not in_band(i, j):
                F = np.zeros(B, np.int64)
                continue
            if i == 0:
                d = H0.copy() if j == 0 else top(j - 1)
            elif j == 0:
                d = left(i - 1)
            else:
                d = H[i - 1, j - 1] if in_band(i - 1, j - 1) else np.zeros(B, np.int64)
            sc = np.where(Q[:, j] == T[:, i], s.match, -s.mismatch)
            M = np.where(d > 0, d + sc, 0)
            e = E[i, j] if (i == 0 or in_band(i - 1, j)) else np.zeros(B, np.int64)
            h = np.maximum(M, np.maximum(e, F))
            H[i, j] = h
            Mm[i, j] = M
            E[i + 1, j] = np.maximum(np.maximum(e - s.e_del, M - oe_d), 0)
            F = np.maximum(np.maximum(F - s.e_ins, M - oe_i), 0)
            ge = h >= rm
            rj = np.where(ge, j, rj)
            rm = np.maximum(rm, h)
        # the band's last column this row, and whether it is the query end
        lo = 0 if wb is None else max(0, i - wb)
        hi = n if wb is None else min(n, i + wb + 1)
        reach = max(lo, hi) == n
        if reach:
            if hi > lo:
                hend = H[i, n - 1]
            else:
                hend = left(i) if lo == 0 else np.zeros(B, np.int64)
            upd = alive & (hend >= gbest)
            gi = np.where(upd, i, gi)
            gbest = np.where(alive, np.maximum(gbest, hend), gbest)
        stop = alive & (rm == 0)
        alive = alive & ~stop
        newb = alive & (rm > best)
        off = np.abs(rj - i)
        moff = np.where(newb, np.maximum(moff, off), moff)
        bi0, bj0 = bi.copy(), bj.copy()
        best = np.where(newb, rm, best)
        bi = np.where(newb, i, bi)
        bj = np.where(newb, rj, bj)
        if zdrop and params.zdrop > 0:
            cand = alive & ~newb
            di = i - bi0
            dj = rj - bj0
            drop = np.where(di > dj,
                            best - rm - (di - dj) * s.e_del,
                            best - rm - (dj - di) * s.e_ins)
            alive = alive & ~(cand & (drop > params.zdrop))
        if not alive.any():
            break
    out[:, 0] = best
    out[:, 1] = bj + 1
    out[:, 2] = bi + 1
    out[:, 3] = gi + 1
    out[:, 4] = gbest
    out[:, 5] = moff
    return out
