"""A bit-level model of the 8-bit row-pair pass, for CPU tests.

The 8-bit per-thread kernel runs rows i and i+1 of a pair in the low and high
halves of s16x2 registers, row i+1 one column behind, and settles row i+1's
band ends from row i after the fact (the kernel's comment gives the
argument).  This module restates that pass in Python with every packed
instruction emulated on 32-bit words (DPX add-min / add-max / three-way max
per 16-bit half, byte permutes, multiply-adds and high multiplies), and the
slot column as a list of 32-bit words, so that `tests/test_rowpair_model.py`
can check the scheme itself against the oracle on the host: the band start
found before the packed loop, the band end L + 3 from the last positive
column of row i, row i's zeros written back past row i+1's end, reads of
slots past the previous row's end (the band rule of Section V-A), the last
row alone when the row count is odd.

It is test infrastructure: nothing outside `tests/` imports it, and it shares
no code with the CUDA path or the oracle (it calls the oracle only for the
clipped band width w').
"""
import oracle

M32 = 0xffffffff


def s16(x):
    x &= 0xffff
    return x - 0x10000 if x & 0x8000 else x


def lo16(x):
    return s16(x)


def hi16(x):
    return s16(x >> 16)


def pack(lo, hi):
    return (lo & 0xffff) | ((hi & 0xffff) << 16)


def u16lo(x):
    return x & 0xffff


def u16hi(x):
    return (x >> 16) & 0xffff


# Per-half emulations of the DPX instructions the kernel uses.
def viaddmin_s16x2(a, b, c):
    return pack(min(s16(lo16(a) + lo16(b)), lo16(c)), min(s16(hi16(a) + hi16(b)), hi16(c)))


def viaddmax_s16x2_relu(a, b, c):
    return pack(max(s16(lo16(a) + lo16(b)), lo16(c), 0), max(s16(hi16(a) + hi16(b)), hi16(c), 0))


def vimax3_s16x2(a, b, c):
    return pack(max(lo16(a), lo16(b), lo16(c)), max(hi16(a), hi16(b), hi16(c)))


def viaddmax_u16x2(a, b, c):
    return pack(max((u16lo(a) + u16lo(b)) & 0xffff, u16lo(c)), max((u16hi(a) + u16hi(b)) & 0xffff, u16hi(c)))


def viaddmin_u16x2(a, b, c):
    return pack(min((u16lo(a) + u16lo(b)) & 0xffff, u16lo(c)), min((u16hi(a) + u16hi(b)) & 0xffff, u16hi(c)))


def imad(a, b, c):
    return (a * b + c) & M32


def umulhi(a, b):
    return ((a & M32) * (b & M32)) >> 32


def prmt(a, b, sel):
    """Byte permute: output byte k is byte (nibble k & 7) of {a, b}, or that
    byte's sign replicated when the nibble's bit 3 is set."""
    by = [(a >> (8 * k)) & 0xff for k in range(4)] + [(b >> (8 * k)) & 0xff for k in range(4)]
    out = 0
    for k in range(4):
        nib = (sel >> (4 * k)) & 0xf
        v = by[nib & 7]
        if nib & 8:
            v = 0xff if v & 0x80 else 0
        out |= v << (8 * k)
    return out


def sext8(x):
    x &= 0xff
    return x - 256 if x & 0x80 else x


def extend(params, q, t, h0, w=None):
    """One pair through the row-pair pass.  Returns (results dict, cells).

    Preconditions of the kernel's row-pair path: n, m >= 1 and
    h0 + match * min(n, m) <= 255, no N bases."""
    sc = params.scoring
    a, b = sc.match, sc.mismatch
    e_del, e_ins = sc.e_del, sc.e_ins
    oe_del, oe_ins = sc.o_del + e_del, sc.o_ins + e_ins
    sym = oe_del == oe_ins and e_del == e_ins
    n, m = len(q), len(t)
    assert n >= 1 and m >= 1 and h0 + a * min(n, m) <= 255
    wb = oracle.band_width(params, n, params.w if w is None else w)
    zmul = 128                     # D * 128 >= D + s for D >= 1, below 2^15 for D <= 255
    noe_d2, noe_i2 = pack(-oe_del, -oe_del), pack(-oe_ins, -oe_ins)
    ne_d2, ne_i2 = pack(-e_del, -e_del), pack(-e_ins, -e_ins)

    # Slot j: selector (q_j, q_j | 8, 4 + q_{j-1}, (4 + q_{j-1}) | 8) in bits
    # 0-15, E in 16-23, H in 24-31; the first row of Eq. 3.
    S = []
    for j in range(n + 1):
        cj = int(q[j]) if j < n else 0
        cjm = int(q[j - 1]) if j >= 1 else 0
        hv = h0 if j == 0 else max(0, h0 - sc.o_ins - j * e_ins)
        S.append(cj * 0x11 + cjm * 0x1100 + 0xC480 + (hv << 24))
    mb8 = (-b) & 0xff
    mis4 = mb8 * 0x01010101
    flip = (a ^ mb8) & 0xff

    def profile(i):               # byte c: s(t_i, c)
        return (mis4 ^ (flip << (8 * int(t[i])))) & M32

    def slot_set(k, h, e):
        S[k] = (S[k] & 0xffff) | ((e & 0xff) << 16) | ((h & 0xff) << 24)

    def cell(d, e, f, s):
        M = min(d + s, d * zmul)
        return max(M, e, f), max(e - e_del, M - oe_del, 0), max(f - e_ins, M - oe_ins, 0)

    lo, hi = 0, n
    best, bi, bj, gbest, gi, moff = h0, -1, -1, -1, -1, 0
    ncell = 0

    def decide(row, key, lo_r, hi_r, h_end):
        """Row decisions (Section V-D): query-end score, all-zero row, best,
        z-drop.  Returns False to stop."""
        nonlocal best, bi, bj, gbest, gi, moff, ncell
        rm, rj = key >> 8, key & 255
        if hi_r > lo_r:
            ncell += hi_r - lo_r
        if max(lo_r, hi_r) == n:
            if h_end >= gbest:
                gi = row
            gbest = max(gbest, h_end)
        if rm == 0:
            return False
        if rm > best:
            best, bi, bj = rm, row, rj
            moff = max(moff, abs(rj - row))
        elif params.zdrop > 0:
            di, dj = row - bi, rj - bj
            drop = best - rm - (di - dj) * e_del if di > dj else best - rm - (dj - di) * e_ins
            if drop > params.zdrop:
                return False
        return True

    for i in range(0, m, 2):
        lo = max(lo, i - wb)
        hi = min(hi, i + wb + 1, n)
        hl0 = max(0, h0 - oe_del - i * e_del) if lo == 0 else 0
        p0 = profile(i)
        single = i + 1 == m
        p1 = profile(i + 1) if not single else 0
        # Row i alone until its first non-zero slot and row i+1's lower clip.
        f, hprev, hprev2, en_last, key_lo, Lp = 0, hl0, 0, 0, 0, 0
        found, lo1, c0 = False, hi, None
        for s in range(lo, hi):
            wv = S[s]
            h, en, f = cell(wv >> 24, (wv >> 16) & 0xff, f, s16(prmt(p0, p1, wv)))
            key_lo = max(key_lo, h * 256 + s)
            if h > 0:
                Lp = s + 1
            if not found and (hprev | en):
                found, lo1 = True, s
            hprev2, hprev, en_last = hprev, h, en
            if not single and found and s >= max(lo1, i + 1 - wb):
                c0 = s
                break
        if single:
            decide(i, key_lo, lo, hi, hprev if hi > lo else hl0)
            break
        if c0 is None:
            c0 = max(lo1, i + 1 - wb)
        bnd1 = max(0, h0 - oe_del - (i + 1) * e_del) if c0 == 0 else 0
        # Both rows: step s computes (i, s) in the low halves, (i+1, s-1) high.
        hA, hB, ENp, F2 = pack(hprev, bnd1), pack(hprev2, 0), pack(en_last, 0), pack(f, 0)
        key2, L2 = pack(key_lo, 0), pack(Lp, 0)
        for s in range(c0 + 1, hi):
            wv = S[s]
            e = (wv >> 16) & 0xff
            Hd2 = imad(hB, 65536, umulhi(wv, 256))
            Ed2 = imad(ENp, 65536, e)
            M2 = viaddmin_s16x2(Hd2, prmt(p0, p1, wv), imad(Hd2, zmul, 0))
            h2 = vimax3_s16x2(M2, Ed2, F2)
            Mi2 = viaddmax_s16x2_relu(M2, noe_i2, 0)
            Md2 = Mi2 if sym else viaddmax_s16x2_relu(M2, noe_d2, 0)
            EN2 = viaddmax_s16x2_relu(Ed2, ne_d2, Md2)
            F2 = viaddmax_s16x2_relu(F2, ne_i2, Mi2)
            h2K = imad(h2, 256, 0)
            j2 = pack(s, s - 1)
            key2 = viaddmax_u16x2(h2K, j2, key2)
            L2 = viaddmax_u16x2(viaddmin_u16x2(j2, 0x00010001, h2K), 0, L2)
            S[s - 1] = (S[s - 1] & 0xffff) | ((prmt(EN2, hA, 0x0062) & 0xffff) << 16)
            hB, hA, ENp = hA, h2, EN2
        if hi > c0 + 1:
            Hi1, Hi2, Ei1 = lo16(hA), lo16(hB), lo16(ENp)
            ce, fh, hlh = hi - 1, hi16(F2), hi16(hA)
        else:
            Hi1, Hi2, Ei1 = hprev, hprev2, en_last
            ce, fh, hlh = c0, 0, bnd1
        key_hi, Lp = u16hi(key2), u16lo(L2)
        if not decide(i, u16lo(key2), lo, hi, Hi1 if hi > lo else hl0):
            break
        # Row i+1's band is [c0, hi1); its columns from ce on run alone.
        hi1 = min(Lp + 2, n, i + 1 + wb + 1)
        for c in range(ce, hi1):
            if c == hi - 1:
                d, e = Hi2, Ei1
            elif c == hi:
                d, e = Hi1, 0
            else:                   # past row i's end: the slot as it stands
                d, e = S[c] >> 24, (S[c] >> 16) & 0xff
            h, en, fh = cell(d, e, fh, sext8(prmt(p1, 0, S[c])))
            slot_set(c, hlh, en)
            key_hi = max(key_hi, h * 256 + c)
            hlh = h
        if hi1 >= ce and hi1 > c0:
            slot_set(hi1, hlh, 0)
        if not decide(i + 1, key_hi, c0, hi1, (S[hi1] >> 24) if hi1 > c0 else bnd1):
            break
        for k in range(hi1 + 1, hi + 1):      # row i's zeros past row i+1's end
            slot_set(k, 0, 0)
        k = c0                                 # rule c on row i+1's slots
        while k < hi1 and (S[k] >> 16) == 0:
            k += 1
        lo = k
        k = hi1
        while k >= lo and (S[k] >> 16) == 0:
            k -= 1
        hi = min(k + 2, n)
    return dict(score=best, qle=bj + 1, tle=bi + 1, gtle=gi + 1, gscore=gbest, max_off=moff), ncell
