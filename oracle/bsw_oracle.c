/*
 * bsw_oracle.c - CPU oracle for banded Smith-Waterman seed extension (BSW).
 *
 * TEST INFRASTRUCTURE ONLY.  This is the plain, slow, obviously-correct
 * reference that the CUDA path is checked against.  Only the tests, the smoke
 * check and the CPU-baseline leg of the benchmark use it; the library never
 * calls it and shares no code with it.
 *
 * What it computes (paper Section V-A, "Banded Smith Waterman Algorithm Used
 * in BWA-MEM"):
 *   - the cell recurrence of Eq. 2: H = max(diagonal + S, E, F), with E and F
 *     the affine-gap terms clamped at 0;
 *   - the boundary of Eq. 3: first row / first column = max(0, H[0,0] - (g_o +
 *     g_e * k)), with H[0,0] = h0, the seed's score;
 *   - the three rules listed after Eq. 2's introduction: (a) only cells inside
 *     a band around the diagonal, (b) stop when a row is all zero or its best
 *     drops too far below the best so far (z-drop), (c) after each row, shrink
 *     the band past zero cells at both ends;
 *   - one row each of H and E kept in memory (Section V-A, last paragraph),
 *     which is why the band-adjust reads below see values left by earlier
 *     rows;
 *   - the global (query-end) score and the best score with their positions
 *     (Section V-D, items (a) and (b)).
 * The paper states its output is identical to BWA-MEM's, so every point the
 * text leaves open is read the way BWA-MEM's extension defines it:
 *   R1 band clip by the largest gap the score can pay for (uses end_bonus);
 *   R2 a zero diagonal gives M = 0 (no fresh local start inside an extension);
 *   R3 E and F open from M (cost o + e), not from H;
 *   R4 ties: row argmax -> larger column, best -> earlier row, gscore -> later row;
 *   R5 z-drop with the diagonal-offset gap correction;
 *   R6 band growth of +2 reads row entries written by earlier rows;
 *   R7 empty query -> {h0, 0, 0, 0, h0, 0}; empty target -> {h0, 0, 0, 0, -1, 0};
 *   R8 rows walk the target, columns walk the query;
 *   R11 an N (code 4; the paper's alphabet has four bases) scores -1 against
 *       any base, N included, as BWA-MEM scores it.
 * Rows are target positions i (deletion penalties on vertical moves), columns
 * are query positions j (insertion penalties on horizontal moves).
 *
 * Debug flags switch the heuristics off for the brute-force comparisons and
 * select the other reading of R3 (gaps opening from H, as Eq. 2 literally
 * writes it) so that a test can show the two readings differ.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

typedef struct {
    int32_t score, qle, tle, gtle, gscore, max_off;
} orc_result_t;

typedef struct {
    int32_t match, mismatch, o_del, e_del, o_ins, e_ins;
    int32_t w, zdrop, end_bonus;
    uint32_t flags;
} orc_params_t;

enum {
    ORC_NO_BAND = 1u,    /* no diagonal band (rule a) */
    ORC_NO_TRIM = 2u,    /* no band adjustment after rows (rule c) */
    ORC_NO_ZDROP = 4u,   /* no z-drop (second half of rule b) */
    ORC_GAP_FROM_H = 8u  /* the other reading of R3: E, F open from H */
};

static int32_t imax(int32_t a, int32_t b) { return a > b ? a : b; }
static int32_t imin(int32_t a, int32_t b) { return a < b ? a : b; }

/*
 * R1: the widest gap worth opening.  A gap of k costs o + k*e, and the most an
 * extension of a length-n query can gain is n*match + end_bonus, so the band
 * never needs to exceed (n*match + end_bonus - o)/e + 1, truncated toward zero
 * and at least 1.  The quotient is taken exactly in integers: C division
 * truncates toward zero.
 */
static int32_t gap_limit(int32_t n, int32_t match, int32_t end_bonus, int32_t o, int32_t e)
{
    int64_t x = (int64_t)n * match + end_bonus - o;
    int64_t k = (x + e) / e;
    return (int32_t)(k > 1 ? k : 1);
}

int orc_band_width(const orc_params_t *P, int32_t n, int32_t w)
{
    int32_t wi = gap_limit(n, P->match, P->end_bonus, P->o_ins, P->e_ins);
    int32_t wd = gap_limit(n, P->match, P->end_bonus, P->o_del, P->e_del);
    return imin(w, imin(wi, wd));
}

/*
 * One extension.  q: query codes (n), t: target codes (m), both 0..3 (A, C, G, T)
 * or 4 (N, R11).
 * Returns 0, or -1 if memory runs out.  cells counts the (i, j) updates made;
 * stale_nz counts reads of row entries that the previous row did not write
 * and that hold a non-zero value (R6).
 */
int orc_extend_one(const orc_params_t *P, int32_t n, const uint8_t *q, int32_t m, const uint8_t *t,
                   int32_t h0, int32_t w, orc_result_t *res, int64_t *cells, int64_t *stale_nz)
{
    const int32_t a = P->match, b = P->mismatch;
    const int32_t o_del = P->o_del, e_del = P->e_del, o_ins = P->o_ins, e_ins = P->e_ins;
    const int from_h = (P->flags & ORC_GAP_FROM_H) != 0;
    int64_t ncell = 0, nstale = 0;

    if (n == 0) {                                     /* R7 */
        res->score = h0; res->qle = 0; res->tle = 0;
        res->gtle = 0; res->gscore = h0; res->max_off = 0;
        if (cells) *cells = 0;
        if (stale_nz) *stale_nz = 0;
        return 0;
    }

    /* Band width (rule a, with R1). */
    int32_t wb = (P->flags & ORC_NO_BAND) ? n + m + 1 : orc_band_width(P, n, w);

    /* One row of H and E (Section V-A).  Entry c holds, between rows, the H of
     * the previous row at column c-1 (the next row's diagonal) and the E that
     * enters column c of the next row. */
    int32_t *Hp = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    int32_t *Ep = (int32_t *)calloc((size_t)(n + 1), sizeof(int32_t));
    if (!Hp || !Ep) { free(Hp); free(Ep); return -1; }

    /* Eq. 3, first row: H[0,0] = h0, H[0,c] = max(0, h0 - (g_o + g_e*c)). */
    Hp[0] = h0;
    for (int32_t c = 1; c <= n; ++c) Hp[c] = imax(0, h0 - o_ins - c * e_ins);

    int32_t best = h0, bi = -1, bj = -1;              /* best score and its cell */
    int32_t gbest = -1, gi = -1;                      /* best score at the query end */
    int32_t moff = 0;                                 /* largest |j - i| of a new best */
    int32_t lo = 0, hi = n;                           /* band [lo, hi) */
    int32_t prev_hi = n;                              /* entries [.., prev_hi] written last row */

    for (int32_t i = 0; i < m; ++i) {
        /* Band for this row. */
        if (!(P->flags & ORC_NO_BAND)) {
            lo = imax(lo, i - wb);
            hi = imin(hi, i + wb + 1);
        }
        hi = imin(hi, n);

        /* Eq. 3, first column: H[i,0] boundary, only while the band touches it. */
        int32_t hl = lo == 0 ? imax(0, h0 - o_del - (i + 1) * e_del) : 0;
        int32_t f = 0, rm = 0, rj = -1;
        const int32_t ti = t[i];

        int32_t j;
        for (j = lo; j < hi; ++j) {
            int32_t d = Hp[j];                        /* H(i-1, j-1) */
            int32_t e = Ep[j];                        /* E(i, j) */
            if (i > 0 && j > prev_hi && (d != 0 || e != 0)) ++nstale;
            Hp[j] = hl;                               /* H(i, j-1), for row i+1 */
            /* Eq. 2 with R2: a zero diagonal is unreached. */
            /* R11: N (code 4) scores -1 against any base, N included. */
            const int32_t sc = (q[j] > 3 || ti > 3) ? -1 : (q[j] == ti ? a : -b);
            int32_t M = d > 0 ? d + sc : 0;
            int32_t h = imax(M, imax(e, f));
            hl = h;
            if (h >= rm) rj = j;                      /* R4: ties -> larger j */
            rm = imax(rm, h);
            int32_t src = from_h ? h : M;             /* R3 */
            Ep[j] = imax(imax(e - e_del, src - o_del - e_del), 0);   /* E(i+1, j) */
            f = imax(imax(f - e_ins, src - o_ins - e_ins), 0);       /* F(i, j+1) */
            ++ncell;
        }
        Hp[hi] = hl;
        Ep[hi] = 0;
        prev_hi = hi;

        /* Global score: the band reached the end of the query (Section V-D b). */
        if (j == n) {
            if (hl >= gbest) gi = i;                  /* R4: ties -> later row */
            gbest = imax(gbest, hl);
        }
        /* Rule b, first half: an all-zero row ends the extension. */
        if (rm == 0) break;
        if (rm > best) {                              /* R4: ties keep the earlier row */
            best = rm; bi = i; bj = rj;
            int32_t off = rj - i < 0 ? i - rj : rj - i;
            moff = imax(moff, off);
        } else if (P->zdrop > 0 && !(P->flags & ORC_NO_ZDROP)) {
            /* Rule b, second half, with R5's gap correction. */
            int32_t di = i - bi, dj = rj - bj;
            if (di > dj) {
                if (best - rm - (di - dj) * e_del > P->zdrop) break;
            } else {
                if (best - rm - (dj - di) * e_ins > P->zdrop) break;
            }
        }
        /* Rule c: skip zero entries at both ends for the next row. */
        if (!(P->flags & ORC_NO_TRIM)) {
            int32_t k = lo;
            while (k < hi && Hp[k] == 0 && Ep[k] == 0) ++k;
            lo = k;
            k = hi;
            while (k >= lo && Hp[k] == 0 && Ep[k] == 0) --k;
            hi = imin(k + 2, n);
        } else {
            hi = n;
        }
    }
    free(Hp);
    free(Ep);
    res->score = best;
    res->qle = bj + 1;
    res->tle = bi + 1;
    res->gtle = gi + 1;
    res->gscore = gbest;
    res->max_off = moff;
    if (cells) *cells = ncell;
    if (stale_nz) *stale_nz = nstale;
    return 0;
}

/* ------------------------------------------------------------------- batch */

typedef struct {
    const orc_params_t *P;
    int64_t n_pairs;
    const uint8_t *q; const int64_t *q_off; const int32_t *q_len;
    const uint8_t *t; const int64_t *t_off; const int32_t *t_len;
    const int32_t *h0; const int32_t *w_override;
    orc_result_t *res; int64_t *cells; int64_t *stale;
    int64_t next;      /* shared work counter */
    int failed;
} batch_t;

static void *batch_worker(void *arg)
{
    batch_t *B = (batch_t *)arg;
    for (;;) {
        int64_t s = __atomic_fetch_add(&B->next, 1024, __ATOMIC_RELAXED);
        if (s >= B->n_pairs) break;
        int64_t e = s + 1024 < B->n_pairs ? s + 1024 : B->n_pairs;
        for (int64_t p = s; p < e; ++p) {
            int32_t w = B->w_override ? B->w_override[p] : B->P->w;
            int64_t c = 0, z = 0;
            if (orc_extend_one(B->P, B->q_len[p], B->q + B->q_off[p], B->t_len[p], B->t + B->t_off[p],
                               B->h0[p], w, &B->res[p], &c, &z) != 0)
                __atomic_store_n(&B->failed, 1, __ATOMIC_RELAXED);
            if (B->cells) B->cells[p] = c;
            if (B->stale) B->stale[p] = z;
        }
    }
    return NULL;
}

/* All pairs, on nthreads host threads taking chunks of 1024 pairs. */
int orc_extend_batch(const orc_params_t *P, int64_t n_pairs,
                     const uint8_t *q, const int64_t *q_off, const int32_t *q_len,
                     const uint8_t *t, const int64_t *t_off, const int32_t *t_len,
                     const int32_t *h0, const int32_t *w_override,
                     orc_result_t *res, int64_t *cells, int64_t *stale, int nthreads)
{
    batch_t B = {P, n_pairs, q, q_off, q_len, t, t_off, t_len, h0, w_override, res, cells, stale, 0, 0};
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    int started = 0;
    for (int k = 1; k < nthreads; ++k) {
        if (pthread_create(&th[k], NULL, batch_worker, &B) != 0) break;
        started = k;
    }
    batch_worker(&B);
    for (int k = 1; k <= started; ++k) pthread_join(th[k], NULL);
    return B.failed ? -1 : 0;
}
