/*
 * bswgen.c - seeded synthetic seed-extension workloads.
 *
 * The paper measures BSW on extension pairs intercepted from BWA-MEM runs on
 * real reads (Section VI, Table V: 48 M pairs from 76 bp reads).  Those reads
 * and the reference are not available, so every workload here is synthetic:
 * a uniform-random ACGT reference, reads copied from it with substitutions and
 * indels, a seed placed in each read, and the query/target pair on either side
 * of the seed.  This file only draws random sequences and lengths; it holds
 * none of the extension arithmetic, and both the CUDA path and the CPU oracle
 * are fed from it.
 *
 * Bases are codes 0..3 (A, C, G, T), one byte per base.
 *
 * Randomness: splitmix64 (Steele, Lea, Flood, "Fast splittable pseudorandom
 * number generators", OOPSLA 2014).  Each unit (a pair, or a read that yields
 * a left and a right pair) owns an independent stream seeded from
 * (config seed, unit index), so the output does not depend on thread count.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <pthread.h>

#define GOLDEN 0x9e3779b97f4a7c15ULL

static inline uint64_t sm_next(uint64_t *s)
{
    uint64_t z = (*s += GOLDEN);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* Stateless hash of (a, b): one splitmix64 step from a derived state. */
static inline uint64_t sm_hash(uint64_t a, uint64_t b)
{
    uint64_t s = a ^ (b * GOLDEN + 0x632be59bd9b4e019ULL);
    sm_next(&s);
    return sm_next(&s);
}

/* Uniform integer in [0, k) by 64x64->128 multiply-shift. */
static inline uint32_t uni(uint64_t *s, uint32_t k)
{
    return (uint32_t)(((unsigned __int128)sm_next(s) * k) >> 64);
}

/* Probability in parts per million -> 64-bit threshold. */
static inline uint64_t ppm_thr(uint64_t ppm)
{
    return (uint64_t)(((unsigned __int128)ppm << 64) / 1000000u);
}

/* ---------------------------------------------------------------- reference */

#define REF_SEED 0x5eedfacecafebeefULL
#define REF_LEN_SMALL 1000000LL      /* workload 0: 1 Mbp */
#define REF_LEN_LARGE 100000000LL    /* workloads 1-3: 100 Mbp */

static uint8_t *g_ref[2];
static int64_t g_ref_len[2] = {REF_LEN_SMALL, REF_LEN_LARGE};
static pthread_mutex_t g_ref_lock = PTHREAD_MUTEX_INITIALIZER;

static const uint8_t *get_ref(int which)
{
    pthread_mutex_lock(&g_ref_lock);
    if (!g_ref[which]) {
        int64_t n = g_ref_len[which];
        uint8_t *r = (uint8_t *)malloc((size_t)n);
        if (r) {
            uint64_t s = sm_hash(REF_SEED, (uint64_t)which);
            for (int64_t i = 0; i < n; i += 32) {
                uint64_t x = sm_next(&s);
                for (int k = 0; k < 32 && i + k < n; ++k) r[i + k] = (uint8_t)((x >> (2 * k)) & 3);
            }
        }
        g_ref[which] = r;
    }
    pthread_mutex_unlock(&g_ref_lock);
    return g_ref[which];
}

/* ------------------------------------------------------------- read copier */

typedef struct {
    uint64_t thr_sub;    /* per-base substitution threshold */
    uint64_t thr_indel;  /* per-base indel-event threshold (checked first) */
    uint32_t indel_max;  /* indel length uniform in 1..indel_max */
} mut_t;

/*
 * Copy `want` bases from ref starting at `pos`, applying per-base events.
 * map[k] (if non-null) receives the reference position that emitted base k
 * (for an inserted base: the reference base that follows it).
 * Returns the reference position after the last consumed base.
 */
static int64_t mutate_copy(const uint8_t *ref, int64_t ref_len, int64_t pos, int32_t want,
                           uint64_t *rng, const mut_t *mu, uint8_t *out, int64_t *map)
{
    int32_t k = 0;
    while (k < want) {
        uint64_t r = sm_next(rng);
        if (r < mu->thr_indel) {
            uint32_t len = 1 + uni(rng, mu->indel_max);
            if (uni(rng, 2) == 0) {               /* deletion from the read */
                pos += len;
            } else {                              /* insertion into the read */
                for (uint32_t x = 0; x < len && k < want; ++x) {
                    out[k] = (uint8_t)uni(rng, 4);
                    if (map) map[k] = pos;
                    ++k;
                }
                if (k >= want) break;
            }
        }
        uint8_t b = pos < ref_len ? ref[pos] : (uint8_t)uni(rng, 4);
        if (sm_next(rng) < mu->thr_sub) b = (uint8_t)((b + 1 + uni(rng, 3)) & 3);
        out[k] = b;
        if (map) map[k] = pos;
        ++k;
        ++pos;
    }
    return pos;
}

/* ---------------------------------------------------------------- workloads */

/*
 * Workload ids (the sizes, rates and parameters are the ones the synthetic
 * stand-ins are specified with):
 *  0  10 k pairs, 1 Mbp reference; query = 1..130 bp copied from a uniform
 *     position with 1% substitutions and 0.1% 1-3 bp indels; target = the
 *     reference window of query length + 100 (clipped at the reference end);
 *     h0 uniform 19..60.
 *  1  151 bp reads from a donor (reference + 0.1% SNPs) with 1% substitution
 *     errors; seed of 19..151 bp at a random offset; a left pair (reversed
 *     prefix / reversed reference window) and a right pair per read; target
 *     length = query length + 100; h0 = seed length x match.
 *  2  250 bp reads with 2% divergence (90% substitutions, 10% indels of
 *     1..10 bp); seeding as workload 1.
 *  3  long queries, length log-uniform 1..10 000, 12% error (half
 *     substitutions, half 1..3 bp indels); target = query length + 500;
 *     h0 uniform 19..60.
 */
enum { W_PLAIN = 0, W_READ151 = 1, W_READ250 = 2, W_LONG = 3 };

static int units_per_pair2(int cfg) { return cfg == W_READ151 || cfg == W_READ250; }

typedef struct {
    int32_t n_a, m_a, n_b, m_b;   /* pair lengths (b only for read units) */
    int32_t h0_a, h0_b;
    int64_t r0;                   /* reference start */
    int32_t L, s;                 /* seed length and offset (read units) */
} unit_t;

/* First draws of a unit's stream: every length is fixed before any base. */
static void unit_head(int cfg, uint64_t seed, int64_t u, int32_t match, uint64_t *rng, unit_t *x)
{
    *rng = sm_hash(seed, (uint64_t)u);
    memset(x, 0, sizeof(*x));
    if (cfg == W_PLAIN) {
        int64_t rl = REF_LEN_SMALL;
        x->n_a = 1 + (int32_t)uni(rng, 130);
        x->h0_a = 19 + (int32_t)uni(rng, 42);
        x->r0 = (int64_t)uni(rng, (uint32_t)(rl - x->n_a));
        int64_t m = x->n_a + 100;
        if (x->r0 + m > rl) m = rl - x->r0;
        x->m_a = (int32_t)m;
    } else if (cfg == W_READ151 || cfg == W_READ250) {
        int32_t rlen = cfg == W_READ151 ? 151 : 250;
        x->r0 = 400 + (int64_t)uni(rng, (uint32_t)(REF_LEN_LARGE - 2000));
        x->L = 19 + (int32_t)uni(rng, (uint32_t)(rlen - 19 + 1));
        x->s = (int32_t)uni(rng, (uint32_t)(rlen - x->L + 1));
        x->n_a = x->s;                       /* left: reversed prefix */
        x->m_a = x->n_a + 100;
        x->n_b = rlen - x->s - x->L;         /* right: suffix after the seed */
        x->m_b = x->n_b + 100;
        x->h0_a = x->h0_b = x->L * match;
    } else {                                  /* W_LONG */
        double uu = (double)(sm_next(rng) >> 11) * (1.0 / 9007199254740992.0);
        int32_t n = (int32_t)floor(exp(uu * log(10000.0)) + 0.5);
        if (n < 1) n = 1;
        if (n > 10000) n = 10000;
        x->n_a = n;
        x->h0_a = 19 + (int32_t)uni(rng, 42);
        x->r0 = (int64_t)uni(rng, (uint32_t)(REF_LEN_LARGE - 40000));
        x->m_a = n + 500;
    }
}

int64_t bswgen_num_units(int cfg, int64_t n_pairs)
{
    return units_per_pair2(cfg) ? (n_pairs + 1) / 2 : n_pairs;
}

/* Lengths of every pair (pairs beyond n_pairs of the last read are dropped). */
int bswgen_lengths(int cfg, uint64_t seed, int64_t n_pairs, int32_t match, int32_t *q_len, int32_t *t_len)
{
    if (cfg < 0 || cfg > 3 || n_pairs < 0) return -1;
    int64_t nu = bswgen_num_units(cfg, n_pairs);
    for (int64_t u = 0; u < nu; ++u) {
        uint64_t rng;
        unit_t x;
        unit_head(cfg, seed, u, match, &rng, &x);
        if (units_per_pair2(cfg)) {
            int64_t p = 2 * u;
            q_len[p] = x.n_a; t_len[p] = x.m_a;
            if (p + 1 < n_pairs) { q_len[p + 1] = x.n_b; t_len[p + 1] = x.m_b; }
        } else {
            q_len[u] = x.n_a; t_len[u] = x.m_a;
        }
    }
    return 0;
}

typedef struct {
    int cfg; uint64_t seed; int64_t n_pairs; int32_t match;
    const int64_t *q_off, *t_off; uint8_t *q, *t; int32_t *h0;
    int64_t u_beg, u_end;
} job_t;

static void *fill_range(void *arg)
{
    job_t *J = (job_t *)arg;
    const int cfg = J->cfg;
    const uint8_t *ref = get_ref(cfg == W_PLAIN ? 0 : 1);
    const int64_t rl = cfg == W_PLAIN ? REF_LEN_SMALL : REF_LEN_LARGE;
    uint8_t read[256];
    int64_t map[256];
    mut_t mu;
    const uint64_t snp_thr = ppm_thr(1000);         /* 0.1% donor SNPs */
    const uint64_t donor_seed = sm_hash(REF_SEED, 0xD0D0);
    if (cfg == W_PLAIN) { mu.thr_indel = ppm_thr(1000); mu.thr_sub = ppm_thr(10000); mu.indel_max = 3; }
    else if (cfg == W_READ151) { mu.thr_indel = 0; mu.thr_sub = ppm_thr(10000); mu.indel_max = 1; }
    else if (cfg == W_READ250) { mu.thr_indel = ppm_thr(2000); mu.thr_sub = ppm_thr(18000); mu.indel_max = 10; }
    else { mu.thr_indel = ppm_thr(60000); mu.thr_sub = ppm_thr(60000); mu.indel_max = 3; }

    for (int64_t u = J->u_beg; u < J->u_end; ++u) {
        uint64_t rng;
        unit_t x;
        unit_head(cfg, J->seed, u, J->match, &rng, &x);
        if (cfg == W_PLAIN || cfg == W_LONG) {
            uint8_t *q = J->q + J->q_off[u], *t = J->t + J->t_off[u];
            mutate_copy(ref, rl, x.r0, x.n_a, &rng, &mu, q, NULL);
            for (int32_t k = 0; k < x.m_a; ++k) t[k] = ref[x.r0 + k];
            J->h0[u] = x.h0_a;
            continue;
        }
        int32_t rlen = cfg == W_READ151 ? 151 : 250;
        if (cfg == W_READ151) {
            for (int32_t k = 0; k < rlen; ++k) {
                int64_t p = x.r0 + k;
                uint8_t b = ref[p];
                uint64_t hv = sm_hash(donor_seed, (uint64_t)p);
                if (hv < snp_thr) b = (uint8_t)((b + 1 + (uint32_t)((hv >> 8) % 3)) & 3);
                if (sm_next(&rng) < mu.thr_sub) b = (uint8_t)((b + 1 + uni(&rng, 3)) & 3);
                read[k] = b;
                map[k] = p;
            }
        } else {
            mutate_copy(ref, rl, x.r0, rlen, &rng, &mu, read, map);
        }
        /* left pair: reversed read prefix, reversed reference before the seed */
        int64_t p = 2 * u;
        {
            uint8_t *q = J->q + J->q_off[p], *t = J->t + J->t_off[p];
            int64_t lp = map[x.s];
            for (int32_t k = 0; k < x.n_a; ++k) q[k] = read[x.s - 1 - k];
            for (int32_t k = 0; k < x.m_a; ++k) t[k] = ref[lp - 1 - k];
            J->h0[p] = x.h0_a;
        }
        if (p + 1 < J->n_pairs) {
            uint8_t *q = J->q + J->q_off[p + 1], *t = J->t + J->t_off[p + 1];
            int32_t e = x.s + x.L;
            int64_t rp = e < rlen ? map[e] : map[rlen - 1] + 1;
            for (int32_t k = 0; k < x.n_b; ++k) q[k] = read[e + k];
            for (int32_t k = 0; k < x.m_b; ++k) t[k] = ref[rp + k];
            J->h0[p + 1] = x.h0_b;
        }
    }
    return NULL;
}

/*
 * Fill sequences and h0.  q_off/t_off give each pair's start (in bases) in
 * q/t, laid out by the caller from bswgen_lengths.  nthreads >= 1.
 */
int bswgen_fill(int cfg, uint64_t seed, int64_t n_pairs, int32_t match,
                const int64_t *q_off, const int64_t *t_off, uint8_t *q, uint8_t *t, int32_t *h0,
                int nthreads)
{
    if (cfg < 0 || cfg > 3 || n_pairs < 0) return -1;
    if (!get_ref(cfg == W_PLAIN ? 0 : 1)) return -2;
    int64_t nu = bswgen_num_units(cfg, n_pairs);
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 64) nthreads = 64;
    if (nu < nthreads) nthreads = nu > 0 ? (int)nu : 1;
    pthread_t th[64];
    job_t jobs[64];
    for (int i = 0; i < nthreads; ++i) {
        jobs[i] = (job_t){cfg, seed, n_pairs, match, q_off, t_off, q, t, h0,
                          nu * i / nthreads, nu * (i + 1) / nthreads};
    }
    for (int i = 1; i < nthreads; ++i) pthread_create(&th[i], NULL, fill_range, &jobs[i]);
    fill_range(&jobs[0]);
    for (int i = 1; i < nthreads; ++i) pthread_join(th[i], NULL);
    return 0;
}

/* Uniform-random codes, for small hand-made tests. */
void bswgen_random_codes(uint64_t seed, int64_t n, uint8_t *out)
{
    uint64_t s = sm_hash(seed, 0xC0DE);
    for (int64_t i = 0; i < n; ++i) out[i] = (uint8_t)uni(&s, 4);
}

/* ------------------------------------------------------ seeds on reads */

/*
 * Seed workloads for the extension driver: n_reads reads of read_len bases
 * from the 100 Mbp reference (read_len 151: the donor / 1% substitution recipe
 * of workload 1; otherwise the 2% divergence recipe of workload 2), each with
 * seeds_per_read seeds of 19..min(50, read_len) bases at uniform offsets.  A
 * seed's reference start is the reference position of its first read base
 * (the seed is taken as ungapped from there).  Seeds of one read are listed
 * together, in the order drawn.
 */
typedef struct {
    uint64_t seed; int64_t r_beg, r_end; int32_t read_len, spr;
    uint8_t *reads; int32_t *s_read, *s_qbeg, *s_len; int64_t *s_rbeg;
} sjob_t;

static void *seeds_range(void *arg)
{
    sjob_t *J = (sjob_t *)arg;
    const uint8_t *ref = get_ref(1);
    const int32_t rlen = J->read_len;
    int64_t *map = (int64_t *)malloc(sizeof(int64_t) * (size_t)rlen);
    if (!map) return NULL;
    mut_t mu;
    if (rlen == 151) { mu.thr_indel = 0; mu.thr_sub = ppm_thr(10000); mu.indel_max = 1; }
    else { mu.thr_indel = ppm_thr(2000); mu.thr_sub = ppm_thr(18000); mu.indel_max = 10; }
    const uint64_t snp_thr = ppm_thr(1000);
    const uint64_t donor_seed = sm_hash(REF_SEED, 0xD0D0);
    for (int64_t r = J->r_beg; r < J->r_end; ++r) {
        uint64_t rng = sm_hash(J->seed ^ 0x5EED5EEDULL, (uint64_t)r);
        const int64_t r0 = 400 + (int64_t)uni(&rng, (uint32_t)(REF_LEN_LARGE - 2 * (int64_t)rlen - 2000));
        uint8_t *read = J->reads + r * rlen;
        if (rlen == 151) {
            for (int32_t k = 0; k < rlen; ++k) {
                int64_t p = r0 + k;
                uint8_t b = ref[p];
                uint64_t hv = sm_hash(donor_seed, (uint64_t)p);
                if (hv < snp_thr) b = (uint8_t)((b + 1 + (uint32_t)((hv >> 8) % 3)) & 3);
                if (sm_next(&rng) < mu.thr_sub) b = (uint8_t)((b + 1 + uni(&rng, 3)) & 3);
                read[k] = b;
                map[k] = p;
            }
        } else {
            mutate_copy(ref, REF_LEN_LARGE, r0, rlen, &rng, &mu, read, map);
        }
        const int32_t lmax = rlen < 50 ? rlen : 50;
        for (int32_t k = 0; k < J->spr; ++k) {
            const int64_t s = r * J->spr + k;
            const int32_t L = 19 + (int32_t)uni(&rng, (uint32_t)(lmax - 19 + 1));
            const int32_t q = (int32_t)uni(&rng, (uint32_t)(rlen - L + 1));
            J->s_read[s] = (int32_t)r;
            J->s_qbeg[s] = q;
            J->s_len[s] = L;
            J->s_rbeg[s] = map[q];
        }
    }
    free(map);
    return NULL;
}

int bswgen_seeds(uint64_t seed, int64_t n_reads, int32_t read_len, int32_t seeds_per_read, uint8_t *reads,
                 int32_t *s_read, int32_t *s_qbeg, int32_t *s_len, int64_t *s_rbeg, int nthreads)
{
    if (n_reads < 0 || read_len < 19 || read_len > 10000 || seeds_per_read < 1) return -1;
    if (!get_ref(1)) return -2;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 64) nthreads = 64;
    if (n_reads < nthreads) nthreads = n_reads > 0 ? (int)n_reads : 1;
    pthread_t th[64];
    sjob_t jobs[64];
    for (int i = 0; i < nthreads; ++i)
        jobs[i] = (sjob_t){seed, n_reads * i / nthreads, n_reads * (i + 1) / nthreads, read_len, seeds_per_read,
                           reads, s_read, s_qbeg, s_len, s_rbeg};
    for (int i = 1; i < nthreads; ++i) pthread_create(&th[i], NULL, seeds_range, &jobs[i]);
    seeds_range(&jobs[0]);
    for (int i = 1; i < nthreads; ++i) pthread_join(th[i], NULL);
    return 0;
}

/* The 100 Mbp reference (codes), bases [start, start + n). */
int bswgen_ref_copy(int64_t start, int64_t n, uint8_t *out)
{
    const uint8_t *ref = get_ref(1);
    if (!ref || start < 0 || n < 0 || start + n > REF_LEN_LARGE) return -1;
    memcpy(out, ref + start, (size_t)n);
    return 0;
}

int64_t bswgen_ref_len(void) { return REF_LEN_LARGE; }

/*
 * Reads for the SMEM search: n_reads reads of read_len bases copied from
 * reference positions [400, ref_limit - read_len - 400) with the recipe of
 * workload 1 (read_len 151: donor SNPs, 1% substitutions) or 2 (2%
 * divergence with indels); odd-numbered reads are reverse-complemented (the
 * other strand).  pos[r] receives the reference start of read r.
 */
int bswgen_reads(uint64_t seed, int64_t n_reads, int32_t read_len, int64_t ref_limit, uint8_t *reads, int64_t *pos)
{
    const uint8_t *ref = get_ref(1);
    if (!ref || n_reads < 0 || read_len < 1 || read_len > 10000 || ref_limit > REF_LEN_LARGE ||
        ref_limit < 2 * (int64_t)read_len + 1000)
        return -1;
    mut_t mu;
    if (read_len == 151) { mu.thr_indel = 0; mu.thr_sub = ppm_thr(10000); mu.indel_max = 1; }
    else { mu.thr_indel = ppm_thr(2000); mu.thr_sub = ppm_thr(18000); mu.indel_max = 10; }
    const uint64_t snp_thr = ppm_thr(1000);
    const uint64_t donor_seed = sm_hash(REF_SEED, 0xD0D0);
    uint8_t *tmp = (uint8_t *)malloc((size_t)read_len);
    if (!tmp) return -2;
    for (int64_t r = 0; r < n_reads; ++r) {
        uint64_t rng = sm_hash(seed ^ 0x5E1EC7ULL, (uint64_t)r);
        const int64_t r0 = 400 + (int64_t)uni(&rng, (uint32_t)(ref_limit - 2 * (int64_t)read_len - 800));
        pos[r] = r0;
        if (read_len == 151) {
            for (int32_t k = 0; k < read_len; ++k) {
                int64_t p = r0 + k;
                uint8_t b = ref[p];
                uint64_t hv = sm_hash(donor_seed, (uint64_t)p);
                if (hv < snp_thr) b = (uint8_t)((b + 1 + (uint32_t)((hv >> 8) % 3)) & 3);
                if (sm_next(&rng) < mu.thr_sub) b = (uint8_t)((b + 1 + uni(&rng, 3)) & 3);
                tmp[k] = b;
            }
        } else {
            mutate_copy(ref, ref_limit, r0, read_len, &rng, &mu, tmp, NULL);
        }
        uint8_t *out = reads + r * (int64_t)read_len;
        if (r & 1) {
            for (int32_t k = 0; k < read_len; ++k) out[k] = (uint8_t)(3 - tmp[read_len - 1 - k]);
        } else {
            memcpy(out, tmp, (size_t)read_len);
        }
    }
    free(tmp);
    return 0;
}
