"""Brute-force full-matrix DP for tiny extensions - TEST INFRASTRUCTURE ONLY.

An independent restatement of the extension used to pin the row-sweep oracle
(``bsw_oracle.c``).  Where the oracle keeps one row of H and E and updates it
in place (Section V-A, last paragraph), this module fills explicit matrices
H, E, F over every cell, with the boundaries written out as the functions of
Eq. 3, so the index bookkeeping of the one-row form is not shared.

``extend_full`` implements:
  * Eq. 2 with the readings R2 (zero diagonal -> M = 0) and R3 (E and F open
    from M with cost o + e) of the oracle's header, and R11 (N, code 4,
    scores -1 against any base);
  * Eq. 3 boundaries: H[-1,-1] = h0, first row max(0, h0 - o_ins - (j+1) e_ins),
    first column max(0, h0 - o_del - (i+1) e_del), E = F = 0 on entry;
  * optionally the static diagonal band (rule a, band width clipped by R1),
    with cells outside it absent (H = E = 0, F restarts inside the band);
  * the all-zero-row abort (rule b, first half) and optionally z-drop (R5);
  * best / global-score bookkeeping with the tie rules R4.
It does not adjust the band after each row (rule c).  ``extend_trimmed`` adds
rule c, restated over the same explicit matrices with a per-column record of
the row that last wrote each slot (see its docstring).

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
            sc = np.where((Q[:, j] > 3) | (T[:, i] > 3), -1, np.where(Q[:, j] == T[:, i], s.match, -s.mismatch))
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


def extend_trimmed(params, Q: np.ndarray, T: np.ndarray, H0: np.ndarray, zdrop: bool = True,
                   w: int | None = None):
    """The full heuristic (rules a, b and c), restated over explicit matrices.

    The one-row form of Section V-A keeps a slot per column; between rows,
    slot c holds the H of column c-1 and the E entering column c, as written
    by the last row whose band covered c.  Here that is spelled out: every
    computed cell is kept in full matrices, and for each column the row that
    last wrote its slot is recorded.  A cell's diagonal and incoming E are then
    read from that row -- the previous row when the band is unchanged, an
    earlier row (or the first row of Eq. 3) when the band regrows (R6).  The
    slot of the band's first column holds that row's first-column boundary
    (Eq. 3, 0 once the band has left column 0); the slot just past its last
    column holds the last H and an E of 0.

    Band adjustment (rule c): the next row starts at the first non-empty slot
    and ends two past the last non-empty slot, a slot being empty when its H
    and E are both 0.  Returns int64 [B, 6] like extend_full.
    """
    s = params.scoring
    Q = np.asarray(Q, np.int64)
    T = np.asarray(T, np.int64)
    H0 = np.asarray(H0, np.int64)
    B, n = Q.shape
    m = T.shape[1]
    out = np.zeros((B, 6), np.int64)
    if n == 0:
        out[:, 0] = H0
        out[:, 4] = H0
        return out
    oe_d, oe_i = s.o_del + s.e_del, s.o_ins + s.e_ins
    wb = band_clip(n, params.w if w is None else w, s.match, params.end_bonus,
                   s.o_ins, s.e_ins, s.o_del, s.e_del)
    ar = np.arange(B)

    def left(i):
        return np.maximum(0, H0 - s.o_del - (np.asarray(i) + 1) * s.e_del)

    def top_slot(j):  # the first row of Eq. 3 as the slot of column j
        return H0.copy() if j == 0 else np.maximum(0, H0 - s.o_ins - j * s.e_ins)

    H = np.zeros((max(m, 1), n, B), np.int64)      # H(i, j)
    Eo = np.zeros((max(m, 1), n, B), np.int64)     # E(i+1, j)
    LO = np.zeros((max(m, 1), B), np.int64)
    HI = np.zeros((max(m, 1), B), np.int64)
    lw = np.full((n + 1, B), -1, np.int64)         # last row that wrote slot j

    def slot(r, j):
        """(H, E) held by slot j after row r (r >= 0 per pair, j in [LO[r], HI[r]])."""
        lo_r, hi_r = LO[r, ar], HI[r, ar]
        first = np.where(lo_r == 0, left(r), 0)
        hprev = H[r, max(j - 1, 0), ar] if j > 0 else np.zeros(B, np.int64)
        hv = np.where(j == lo_r, first, hprev)
        ev = np.where(j >= hi_r, 0, Eo[r, min(j, n - 1), ar])
        return hv, ev

    best = H0.copy()
    bi = np.full(B, -1, np.int64)
    bj = np.full(B, -1, np.int64)
    gbest = np.full(B, -1, np.int64)
    gi = np.full(B, -1, np.int64)
    moff = np.zeros(B, np.int64)
    alive = np.ones(B, bool)
    lo = np.zeros(B, np.int64)
    hi = np.full(B, n, np.int64)

    for i in range(m):
        lo = np.maximum(lo, i - wb)
        hi = np.minimum(np.minimum(hi, i + wb + 1), n)
        LO[i], HI[i] = lo, hi
        F = np.zeros(B, np.int64)
        rm = np.zeros(B, np.int64)
        rj = np.full(B, -1, np.int64)
        for j in range(n):
            inb = alive & (lo <= j) & (j < hi)
            if not inb.any():
                continue
            r = lw[j]
            never = r < 0
            rr = np.where(never, 0, r)
            hv, ev = slot(rr, j)
            d = np.where(never, top_slot(j), hv)
            e = np.where(never, 0, ev)
            sc = np.where((Q[:, j] > 3) | (T[:, i] > 3), -1, np.where(Q[:, j] == T[:, i], s.match, -s.mismatch))
            M = np.where(d > 0, d + sc, 0)
            h = np.maximum(M, np.maximum(e, F))
            H[i, j] = np.where(inb, h, 0)
            Eo[i, j] = np.where(inb, np.maximum(np.maximum(e - s.e_del, M - oe_d), 0), 0)
            F = np.where(inb, np.maximum(np.maximum(F - s.e_ins, M - oe_i), 0), 0)
            ge = inb & (h >= rm)
            rj = np.where(ge, j, rj)
            rm = np.where(inb, np.maximum(rm, h), rm)
        # slots [lo, hi] now belong to row i
        for j in range(n + 1):
            cov = alive & (lo <= j) & (j <= hi)
            lw[j] = np.where(cov, i, lw[j])
        reach = np.maximum(lo, hi) == n
        hend = np.where(hi > lo, H[i, np.clip(hi - 1, 0, n - 1), ar], np.where(lo == 0, left(i), 0))
        upd = alive & reach
        gi = np.where(upd & (hend >= gbest), i, gi)
        gbest = np.where(upd, np.maximum(gbest, hend), gbest)
        alive = alive & (rm != 0)
        newb = alive & (rm > best)
        moff = np.where(newb, np.maximum(moff, np.abs(rj - i)), moff)
        bi0, bj0 = bi.copy(), bj.copy()
        best = np.where(newb, rm, best)
        bi = np.where(newb, i, bi)
        bj = np.where(newb, rj, bj)
        if zdrop and params.zdrop > 0:
            di, dj = i - bi0, rj - bj0
            drop = np.where(di > dj, best - rm - (di - dj) * s.e_del, best - rm - (dj - di) * s.e_ins)
            alive = alive & ~(~newb & (drop > params.zdrop))
        if not alive.any():
            break
        # rule c
        nz = np.zeros((n + 1, B), bool)
        for j in range(n + 1):
            cov = (lo <= j) & (j <= hi)
            if cov.any():
                hv, ev = slot(np.full(B, i), j)
                nz[j] = cov & ((hv != 0) | (ev != 0))
        idx = np.arange(n + 1)[:, None]
        cand_lo = np.where(nz & (idx < hi), idx, n + 1).min(axis=0)
        new_lo = np.where(cand_lo <= n, np.minimum(cand_lo, hi), hi)
        cand_hi = np.where(nz & (idx >= new_lo), idx, -1).max(axis=0)
        last = np.where(cand_hi >= 0, cand_hi, new_lo - 1)
        lo = np.where(alive, new_lo, lo)
        hi = np.where(alive, np.minimum(last + 2, n), hi)
    out[:, 0] = best
    out[:, 1] = bj + 1
    out[:, 2] = bi + 1
    out[:, 3] = gi + 1
    out[:, 4] = gbest
    out[:, 5] = moff
    return out
