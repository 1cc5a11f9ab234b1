/*
 * bsw.h - C ABI of the GB300 banded Smith-Waterman seed-extension library.
 *
 * The operation is BWA-MEM's seed extension as described in Section V-A of
 * "Efficient Architecture-Aware Acceleration of BWA-MEM for Multicore Systems"
 * (Vasimuddin, Misra, Li, Aluru, IPDPS 2019): starting from a seed with score
 * h0 = H[0,0], fill the DP matrix of Eq. 2 row by row with the boundary of
 * Eq. 3, restricted to a band around the diagonal (rule a), stopping when a
 * row is all zero or drops too far below the best (rule b, z-drop), and
 * shrinking the band past zero cells at both ends after each row (rule c).
 * Rows walk the target (deletions are vertical moves), columns walk the query
 * (insertions are horizontal moves).  The result fields are the ones BWA-MEM's
 * extension returns (Section V-D, items (a) and (b)):
 *   score   best H over the computed rows, or h0 if no cell exceeds it
 *   qle,tle query / target length of the best cell (column+1, row+1; 0 = seed)
 *   gtle    target length at the best score reaching the query end (0 = none)
 *   gscore  best H in the query's last column (-1 if the band never reached it)
 *   max_off largest |column - row| of a cell that raised the best score
 * Every field is exact integer arithmetic; the library's kernels and a plain
 * CPU restatement agree bit for bit.
 *
 * Conventions
 *   - Bases are 2-bit codes A=0 C=1 G=2 T=3, packed four per byte, base k of a
 *     sequence in bits 2*(k%4)..2*(k%4)+1 of byte k/4 (bsw_pack_2bit).
 *     Offsets are in bases and must be multiples of 4, so every sequence starts
 *     on a byte.  Ambiguous bases (N) ride beside the 2-bit codes in
 *     optional per-side bitmaps (bsw_batch_t.q_n / t_n, bsw_pack_2bit_n): an
 *     N scores -1 against any base, N included.
 *   - Extension runs rightward from the seed.  A left extension is the caller's
 *     job: pass the reversed query prefix and the reversed reference window.
 *   - An empty query returns {h0, 0, 0, 0, h0, 0}; an empty target returns
 *     {h0, 0, 0, 0, -1, 0}.
 *   - Scores must satisfy h0 + match * min(qlen, tlen) < 2^30.
 *
 * Threading: a context is not thread-safe, except that bsw_stream_submit and
 * bsw_stream_poll may be called from one client thread while the context's
 * own server thread runs.
 *
 * Every function returns BSW_OK (0), BSW_PENDING (> 0, poll only) or a
 * negative BSW_E* code; nothing else crosses the ABI.  After any error except
 * BSW_ECUDA the context stays usable.  After BSW_ECUDA from a sticky device
 * error (the CUDA context is lost) only bsw_destroy is valid.
 */
#ifndef BSW_H
#define BSW_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BSW_OK        0
#define BSW_PENDING   1
#define BSW_EINVAL   (-1)   /* bad argument or input value                    */
#define BSW_ENOMEM   (-2)   /* host or device allocation failed               */
#define BSW_EBUDGET  (-3)   /* the batch cannot fit the device-memory budget  */
#define BSW_ECUDA    (-4)   /* a CUDA call failed                             */
#define BSW_ETIMEOUT (-5)   /* a bounded wait ran out                         */
#define BSW_ENOTFOUND (-6)  /* unknown or already collected ticket            */
#define BSW_ESTATE   (-7)   /* the context cannot accept the call             */

/* The longest query a batch pair may have (longer: BSW_EINVAL). */
#define BSW_MAX_QLEN 32768

/* bsw_batch_t.flags */
#define BSW_DEVICE_PTRS   0x01u  /* every batch pointer and `out` are device pointers      */
#define BSW_FORCE_I8      0x02u  /* 8-bit lanes for every pair up to 256 query bases,
                                    without the score-bound check; pairs whose scores
                                    leave 0..255 are re-run exactly with 32-bit lanes   */
#define BSW_FORCE_I16     0x04u  /* 16-bit lanes (same re-run rule above 32767)            */
#define BSW_FORCE_I32     0x08u  /* 32-bit warp-per-pair kernel for every pair             */
#define BSW_PLAIN_KERNEL  0x10u  /* baseline: one pair per warp in input order (no
                                    bucketing, classes or re-run list), each pair on
                                    the warp-per-pair ring kernel with the plan's
                                    warp_cols columns per lane                       */
#define BSW_NO_GRAPH      0x20u  /* device-pointer path: launch directly, no CUDA graph    */
#define BSW_COPY_INPUTS   0x40u  /* submit: copy host inputs at submit time                */
#define BSW_PACKED_PAIRS  0x80u  /* 8-bit classes up to 128 query bases: two pairs per
                                    thread in packed 16-bit lanes instead of one        */
#define BSW_TIME_KERNELS  0x100u /* record CUDA events around each class kernel (host
                                    pointers, or device pointers with BSW_NO_GRAPH);
                                    read them with bsw_kernel_times                     */
#define BSW_PLAIN_GLOBAL  0x200u /* naive baseline: one pair per warp in input order, one
                                    column per lane, the row's slots in global memory    */

typedef struct bsw_ctx bsw_ctx_t;

/* match > 0; mismatch, o_*, e_* > 0 are penalties (a gap of k costs o + k*e).
 * match <= 127 and mismatch <= 128. */
typedef struct {
    int32_t match, mismatch, o_del, e_del, o_ins, e_ins;
} bsw_scoring_t;

typedef struct {
    int32_t score, qle, tle, gtle, gscore, max_off;
} bsw_result_t;

typedef struct {
    int64_t n_pairs;
    const uint8_t *q;          /* packed queries                                  */
    const int64_t *q_off;      /* [n_pairs] query start, in bases, multiple of 4  */
    const int32_t *q_len;      /* [n_pairs] >= 0                                  */
    const uint8_t *t;          /* packed targets                                  */
    const int64_t *t_off;      /* [n_pairs]                                       */
    const int32_t *t_len;      /* [n_pairs] >= 0                                  */
    const int32_t *h0;         /* [n_pairs] seed score, >= 0                      */
    const int32_t *w_override; /* [n_pairs] per-pair band, or NULL for the ctx w  */
    uint32_t flags;            /* BSW_* flags above                               */
    const uint8_t *q_n;        /* N bitmap of q, or NULL (no N): bit p & 7 of     */
    const uint8_t *t_n;        /* byte p >> 3 marks base p as N (see below)       */
} bsw_batch_t;

/*
 * N bases: the 2-bit codes hold A, C, G, T only.  q_n / t_n (nullable, same
 * pointer kind as q / t) mark bases as N; an N scores -1 against any base, N
 * included (BWA-MEM's rule; the paper's alphabet has four bases), and the
 * base's 2-bit code is ignored.  Pairs with an N run in the 8-bit per-thread
 * kernels when their scores fit, else in the 32-bit warp-per-pair kernel.
 * bsw_pack_2bit_n packs text with N.  bsw_stream_submit takes them too (and
 * copies them with BSW_COPY_INPUTS).
 */

/*
 * Create a context.  sc: scoring (copied); w >= 0: band half-width before the
 * gap-limit clip; zdrop: z-drop threshold, <= 0 disables it; end_bonus >= 0:
 * used only in the band clip (the largest gap worth opening is
 * trunc((qlen*match + end_bonus - o)/e + 1)).  mem_budget_bytes > 0 caps the
 * device memory the context allocates (work buffers, staging and the serving
 * loop's slots).  On success *out owns a CUDA-side context on the current
 * device; release it with bsw_destroy.
 * Errors: BSW_EINVAL (bad scoring/arguments), BSW_ENOMEM, BSW_ECUDA.
 */
int bsw_init(const bsw_scoring_t *sc, int32_t w, int32_t zdrop, int32_t end_bonus,
             int64_t mem_budget_bytes, bsw_ctx_t **out);

/*
 * Extend every pair of a batch (Section V-A for each pair; the batch is the
 * inter-task unit of Section V-C).  out[k] receives pair k's result.
 *
 * Host pointers (default): inputs and out are host memory owned by the caller;
 * they may be released on return.  The call stages inputs to the device,
 * runs the kernels on cuda_stream (a cudaStream_t, or NULL for the context's
 * own stream), copies results back and returns when they are in out.
 *
 * BSW_DEVICE_PTRS: every pointer, including out and cells_out, is device
 * memory on the context's device.  The call only enqueues work on cuda_stream
 * and returns; results are valid once the stream reaches that point.  Input
 * errors found by the kernels are reported by bsw_sync.
 *
 * cells_out (nullable): receives the number of DP cells computed, the same
 * count the CPU restatement makes (cells inside each row's band, over the rows
 * run).  In device mode it is a device int64 that the call overwrites.
 *
 * Errors: BSW_EINVAL (n_pairs < 0, null pointer, negative length or h0,
 * offset not a multiple of 4, a query longer than BSW_MAX_QLEN, score bound
 * h0 + match * min(q_len, t_len) of 2^30 or more, bad flags), BSW_EBUDGET,
 * BSW_ENOMEM, BSW_ECUDA.
 */
int bsw_extend_batch(bsw_ctx_t *ctx, const bsw_batch_t *batch, bsw_result_t *out,
                     int64_t *cells_out, void *cuda_stream);

/*
 * Wait for cuda_stream (NULL: the context's stream) and report input errors
 * the kernels flagged since the last call (BSW_EINVAL), or BSW_ECUDA.
 */
int bsw_sync(bsw_ctx_t *ctx, void *cuda_stream);

/*
 * Serving: queue a batch of host inputs and return at once with a ticket
 * (flags: 0 or BSW_COPY_INPUTS; the other flags are rejected).  A server thread admits
 * queued batches as stream slots and device memory within the budget free up,
 * merges small ones into one launch, and overlaps launches on several streams
 * (continuous batching).  A batch may carry N bitmaps (q_n, t_n).  An
 * admission that finds the budget held by busy lanes waits for one of them to
 * finish.  Inputs and out must stay valid until poll returns
 * BSW_OK for the ticket, unless BSW_COPY_INPUTS is set (inputs are copied
 * before submit returns; out must still stay valid).
 * Errors: BSW_EINVAL, BSW_EBUDGET (the batch alone exceeds the budget),
 * BSW_ENOMEM, BSW_ESTATE (context shutting down).  A failed submit registers
 * nothing: no ticket is issued, *ticket is left as it was, and the library
 * never writes the batch's out.
 */
int bsw_stream_submit(bsw_ctx_t *ctx, const bsw_batch_t *batch, bsw_result_t *out,
                      uint64_t *ticket);

/*
 * Serving counters since the context was made or last reset (reset != 0
 * zeroes them after reading).  A launch is one merged batch on one
 * execution lane; its device interval runs from the event recorded before its
 * host-to-device copy to the event after its results are copied back (CUDA
 * events on the lane's stream), kept for the latest 65536 launches.
 *   requests        requests finished (any status)
 *   launches        launches finished
 *   merged          requests that shared their launch with another request
 *   budget_waits    admissions put back to wait for device memory that busy
 *                   lanes held (the budget, not a failure)
 *   busy_ms         the sum of the launches' intervals
 *   union_ms        the time at least one launch was on the device (busy_ms /
 *                   union_ms > 1: launches overlapped)
 *   max_concurrent  the most launches on the device at one moment
 * Errors: BSW_EINVAL (null argument).
 */
typedef struct {
    int64_t requests, launches, merged, budget_waits;
    double busy_ms, union_ms;
    int32_t max_concurrent;
} bsw_serve_stats_t;
int bsw_stream_stats(bsw_ctx_t *ctx, bsw_serve_stats_t *out, int32_t reset);

/*
 * Wait up to timeout_us microseconds (0: just check; < 0: wait without limit)
 * for a ticket.  BSW_OK: out is filled and the ticket is released.
 * BSW_PENDING: not yet.  A negative code: the request failed (the ticket is
 * released) or the ticket is unknown (BSW_ENOTFOUND).
 */
int bsw_stream_poll(bsw_ctx_t *ctx, uint64_t ticket, int32_t timeout_us);

/*
 * Host-side fault injection, for tests of the error paths.  The paper has no
 * counterpart.  Nothing here touches the GPU: a named host call is made to
 * fail as if the runtime had refused it, so the caller sees the documented
 * code and the context must stay usable afterwards.  Sites:
 *   alloc   a device (cudaMalloc) or pinned host (cudaMallocHost) allocation
 *           of a context's buffers: the call returns BSW_ENOMEM
 *   h2d     a host-to-device copy of a host batch (bsw_extend_batch with host
 *           pointers, the serving loop's staging): BSW_ECUDA
 *   launch  the launch of a batch's kernels: BSW_ECUDA
 *   thread  the start of a context's serving thread: bsw_stream_submit
 *           returns BSW_ENOMEM and registers nothing
 *   host    a host container allocation in the serving path (ticket table,
 *           queue, admission list): BSW_ENOMEM from bsw_stream_submit, or a
 *           retried admission in the serving thread
 * spec: a comma-separated list of site names, optionally followed by
 * ":skip" and ":count" (defaults 0 and 1): of the later hits on any listed
 * site the first `skip` pass and the next `count` fail; then injection stops.
 * NULL or "" disarms.  The environment variable BSW_FAULT_INJECT, if set when
 * the library loads, is applied the same way.  Process-wide; not meant for
 * production use.  Returns BSW_OK, or BSW_EINVAL for a spec it cannot parse
 * (the previous setting is then kept).
 */
#define BSW_FAULT_ALLOC  0x01u
#define BSW_FAULT_H2D    0x02u
#define BSW_FAULT_LAUNCH 0x04u
#define BSW_FAULT_THREAD 0x08u
#define BSW_FAULT_HOST   0x10u
int bsw_fault_inject(const char *spec);

/* Static English description of a return code. */
const char *bsw_strerror(int code);

/* Stop the server thread, wait for queued work, free everything.  NULL is a no-op. */
void bsw_destroy(bsw_ctx_t *ctx);

/*
 * Pack n bases into out[(n + 3) / 4] (layout above).  Input bytes are codes
 * 0..3 or the letters ACGT/acgt.  Returns BSW_OK, or BSW_EINVAL on any other
 * byte (out is then unspecified).
 */
int bsw_pack_2bit(const uint8_t *in, int64_t n, uint8_t *out);

/*
 * As bsw_pack_2bit, also accepting N (code 4 or the letters N/n): N is
 * packed as code 0 and marked in out_n[(n + 7) / 8] (bit p & 7 of byte
 * p >> 3 for base p; other bits 0).  Returns BSW_OK or BSW_EINVAL.
 */
int bsw_pack_2bit_n(const uint8_t *in, int64_t n, uint8_t *out, uint8_t *out_n);

/*
 * The band half-width after the gap-limit clip for a query of qlen bases:
 * min(w, trunc((qlen*match + end_bonus - o)/e + 1) for both gap kinds), each
 * limit at least 1.  Returns -1 on bad arguments.
 */
int32_t bsw_band_width(const bsw_ctx_t *ctx, int32_t qlen, int32_t w);

/*
 * Split one batch over several devices (pairs are independent, so there is
 * no exchange step: each device runs its part with its own context and the
 * parts' results, concatenated in order, are the batch's results).  Part k
 * is the contiguous pair range [bounds[k], bounds[k+1]); bounds[0] = 0 and
 * bounds[parts] = n_pairs.  The ranges balance the estimated work: pair p
 * weighs q_len[p] * min(t_len[p], 2w' + 1), its band area, w' its band after
 * the gap-limit clip (bsw_band_width's rule, w_override[p] when given), and
 * the boundaries are where the running weight first reaches k/parts of the
 * total.  Host pointers (q_len, t_len, w_override nullable); no device work,
 * so it needs no context.  sc, w, end_bonus: as bsw_init.
 * Errors: BSW_EINVAL (null pointers, n_pairs < 0, parts < 1, a negative
 * length or band).
 */
int bsw_partition(const bsw_scoring_t *sc, int32_t w, int32_t end_bonus, const int32_t *q_len,
                  const int32_t *t_len, const int32_t *w_override, int64_t n_pairs, int32_t parts,
                  int64_t *bounds);

/*
 * bsw_extend_batch_noalloc: the batched extension for callers that cannot
 * allocate device memory.  The paper has no counterpart; it exists for code
 * that may not call cudaMalloc where it extends seeds (a memory pool that owns
 * the whole device, an allocator that forbids allocation at that point, or a
 * library inside a process whose device memory is managed by someone else).
 *
 * It computes exactly what bsw_extend_batch computes for the same scoring and
 * parameters, and allocates nothing: no context, no cudaMalloc/cudaFree, no
 * streams or events.  Its work buffers live in one file-scope device array of
 * BSW_NOALLOC_SCRATCH_BYTES bytes that every GPU which loads this library holds
 * until the process exits.
 *
 *   sc, w, zdrop, end_bonus  as for bsw_init
 *   batch    device pointers only (flags must include BSW_DEVICE_PTRS; the
 *            BSW_FORCE_* flags are honoured, others are rejected)
 *   out      device array of n_pairs results
 *   cells_out  nullable device int64, overwritten with the cell count
 *   cuda_stream  the stream to run on (NULL: the legacy default stream)
 *
 * Limits: n_pairs <= BSW_NOALLOC_MAX_PAIRS, every query <= BSW_NOALLOC_MAX_QLEN
 * bases.  A larger n_pairs returns BSW_EINVAL before any work; a longer query
 * is found by the kernels and the call returns BSW_EINVAL (out is then
 * unspecified for that batch).  The call enqueues the work, waits for the
 * stream and returns the status (BSW_OK, BSW_EINVAL for bad inputs, BSW_ECUDA).
 *
 * The first call on a device looks up the array's device address for that
 * device and sets kernel attributes; make that first call before any stream
 * capture on the device.  All calls share the one array: two calls whose work
 * overlaps on the GPU (different streams, or different host threads) race on
 * it and give wrong results; serialize them.
 */
#define BSW_NOALLOC_MAX_PAIRS 262144
#define BSW_NOALLOC_MAX_QLEN 256
#define BSW_NOALLOC_SCRATCH_BYTES (16u << 20)
int bsw_extend_batch_noalloc(const bsw_scoring_t *sc, int32_t w, int32_t zdrop, int32_t end_bonus,
                             const bsw_batch_t *batch, bsw_result_t *out, int64_t *cells_out,
                             void *cuda_stream);

/*
 * Execution plan of the batched path: which kernel runs which pairs.  The
 * paper fixes these choices for 512-bit vectors (Section V-C: sort by length,
 * 8-bit lanes first, 16-bit re-run); here they are parameters.  Every plan
 * computes the same results; plans differ only in speed.
 *
 *   short_max    queries of up to short_max bases run one pair per thread (the
 *                per-thread length classes); longer ones one pair per warp.
 *                64 <= short_max <= 256.
 *   u8_bounds    bit k (k = 1..7) keeps the 8-bit class boundary at
 *                224, 192, 160, 128, 96, 64, 32 bases; the 256 class (bit 0) is
 *                always kept.  A query runs in the smallest kept class that
 *                holds it (a class of bound N keeps N + 1 slots per thread).
 *   i16_bounds   the same for the 16-bit classes: bits 1..3 = 128, 64, 32.
 *   packed       1: the 8-bit classes up to 128 bases run two pairs per thread
 *                in packed 16-bit lanes, where the scoring allows it (small
 *                mismatch and gap costs); 0: one pair per thread.
 *   warp_cols    columns each lane owns per row chunk in the 16-bit
 *                warp-per-pair kernel: 4, 8 or 16.
 *   inter_warps  warps per block of the per-thread kernels: 1, 2 or 4.
 *   cta_min      queries of at least cta_min bases whose scores fit 16 bits
 *                (and that hold no N) run one pair per block of 4 warps, the
 *                row's band split across the warps (uneven batches: the
 *                longest pairs no longer set the batch's tail); 0: none.  A
 *                multiple of 64 in [128, BSW_MAX_QLEN], or 0.
 *   warp_x2      1: the 16-bit warp-per-pair class runs the kernel that
 *                computes two columns per instruction (16-bit halves of one
 *                register, 8-column granules, 1 to 4 granules per lane chosen
 *                per row), for pairs whose score bound h0 + match*min(n, m)
 *                is below 2^(15 - z), 2^z >= match + 1 (16384 for match 1);
 *                the class's other pairs run with 32-bit lanes.  Applies when
 *                match <= 3 and o + e <= 8192, e <= 2048 on both sides;
 *                warp_cols is then unused by that class.  0 or 1.
 *   ms           output of bsw_autotune (the plan's time on its sample, in
 *                milliseconds); ignored by bsw_set_plan.
 */
typedef struct {
    int32_t short_max;
    uint32_t u8_bounds, i16_bounds;
    int32_t packed, warp_cols, inter_warps, cta_min, warp_x2;
    float ms;
} bsw_plan_t;

/* The context's current plan (a new context has {256, 0xff, 0xf, 0, 8, 2, 0, 0}).
 * Errors: BSW_EINVAL (null argument). */
int bsw_get_plan(const bsw_ctx_t *ctx, bsw_plan_t *plan);

/* Use `plan` for every later call on the context.  Errors: BSW_EINVAL (a field
 * out of range), BSW_ESTATE (submitted work still pending). */
int bsw_set_plan(bsw_ctx_t *ctx, const bsw_plan_t *plan);

/*
 * Autotune the plan on a sample of `batch`: its first min(n_pairs,
 * sample_pairs) pairs (sample_pairs <= 0: 2097152).  Each candidate plan is
 * timed with CUDA events as the fastest of `reps` launches (reps <= 0: 3)
 * after one warm-up launch, on the context's stream.  The search is
 * coordinate descent from the default plan: short_max (256, 192, 128, 96,
 * 64), warp_x2 (0, 1), warp_cols (8, 4, 16; when warp_x2 stays 0),
 * cta_min (0, 8192, 4096, 2048, 1024, 512),
 * packed, inter_warps (2, 1, 4), then each class
 * boundary removed in turn (8-bit from 192 down, then 16-bit); a change is
 * kept when it is at least 1% faster than the best so far.  A knob that only
 * affects classes holding no pair of the sample is not tried, and the
 * boundary of a class holding no pair of the sample is removed untimed.  The
 * fastest plan becomes the context's plan and is written to *chosen
 * (nullable), with its time measured again.
 *
 * batch: host pointers, or device pointers with BSW_DEVICE_PTRS (other flags
 * are rejected); the sample's results are computed and discarded.  The call
 * returns when tuning is done.  Errors: as bsw_extend_batch, and BSW_ESTATE
 * (submitted work still pending).
 */
int bsw_autotune(bsw_ctx_t *ctx, const bsw_batch_t *batch, int64_t sample_pairs, int32_t reps,
                 bsw_plan_t *chosen);

/*
 * Kernel times of the last bsw_extend_batch call made with BSW_TIME_KERNELS.
 * Waits for that call's work, then class_ms[c] = the time between the CUDA
 * events recorded on the stream of class c's kernel just before and just
 * after its launch (0 if the class was not launched).  Classes: 0-7 the 8-bit
 * per-thread classes of bound 256, 224, 192, 160, 128, 96, 64, 32; 8-11 the
 * 16-bit classes of bound 256, 128, 64, 32; 12 the block-per-pair kernel; 13
 * the 16-bit warp-per-pair kernel; 14 the 32-bit one; 15 the 32-bit re-run.
 * launches = the kernels
 * the last batched call launched (timed or not; the plain kernel counts 1).
 * Errors: BSW_EINVAL (null argument), BSW_ESTATE (no timed call yet),
 * BSW_ECUDA.
 */
typedef struct {
    int32_t launches;
    float class_ms[16];
} bsw_timing_t;
int bsw_kernel_times(bsw_ctx_t *ctx, bsw_timing_t *out);

/*
 * Seed-extension driver (Section V-C2: every seed of a read is extended and
 * the results are filtered afterwards; Section V-A for each extension).
 *
 * bsw_set_reference uploads the reference once per context: ref_len bases,
 * 2-bit packed as for batches (4 per byte, first base in the low bits).  The
 * copy is charged to the context's budget and replaces any earlier one.
 * Errors: BSW_EINVAL, BSW_EBUDGET, BSW_ENOMEM, BSW_ECUDA, BSW_ESTATE
 * (submitted work pending).
 */
int bsw_set_reference(bsw_ctx_t *ctx, const uint8_t *ref, int64_t ref_len);

/* The same with an N bitmap of the reference (ref_n: bit p & 7 of byte p >> 3
 * marks base p as N; (ref_len + 7) / 8 bytes; NULL: no N).  N bases score as
 * in BSW batches (-1 against anything). */
int bsw_set_reference_n(bsw_ctx_t *ctx, const uint8_t *ref, const uint8_t *ref_n, int64_t ref_len);

typedef struct {
    int32_t read_id;   /* the seed's read, 0..n_reads-1                          */
    int32_t qbeg;      /* seed start in the read                                 */
    int32_t len;       /* seed length: read bases [qbeg, qbeg + len)             */
    int32_t reserved;  /* 0                                                      */
    int64_t rbeg;      /* seed start in the reference (the seed is ungapped)     */
} bsw_seed_t;

typedef struct {
    int32_t qb, qe;          /* aligned read interval [qb, qe)                   */
    int64_t rb, re;          /* aligned reference interval [rb, re)              */
    int32_t score;           /* score of the chosen ends                          */
    int32_t w_left, w_right; /* band of each side's last run; 0: no read bases    */
    int32_t kept;            /* 0: covered by an earlier kept seed of the read    */
} bsw_aln_t;

/*
 * Extend every seed against the context's reference (bsw_set_reference):
 *   1. left: the read bases before the seed, reversed, against the qbeg + w
 *      reference bases before rbeg (fewer at the reference start), reversed,
 *      from h0 = len * match;
 *   2. the left end: the read start (gtle, gscore) unless gscore <= 0 or
 *      gscore <= score - end_bonus, else the local best (qle, tle, score);
 *      this gives (qb, rb) and the left score;
 *   3. right: the read bases after the seed against the following
 *      (read bases + w) reference bases, from h0 = the left score;
 *   4. the right end as in 2, giving (qe, re) and score;
 *   each extension whose max_off reaches (w' >> 1) + (w' >> 2) for its band
 *   w' runs again with twice the band, up to max_band_try runs (1..8), and
 *   the last run counts;
 *   5. in each read's seed order, a seed whose read and reference intervals
 *   lie inside the alignment of an earlier kept seed is not kept.
 * The extensions use the context's scoring, w, zdrop, end_bonus and plan.
 *
 * Host pointers: reads 2-bit packed, read r at base offset read_off[r]
 * (a multiple of 4) with read_len[r] bases; seeds[n_seeds] with the seeds of
 * one read consecutive, each inside its read and the reference; out[n_seeds]
 * (caller-owned) receives the alignments; cells_out (nullable) the DP cells
 * of all extensions.  The call returns when out is filled.
 * Errors: BSW_EINVAL (bad argument, a seed outside its read or the
 * reference, a read's seeds not consecutive), BSW_ESTATE (no reference, or
 * submitted work pending), BSW_EBUDGET, BSW_ENOMEM, BSW_ECUDA.
 */
int bsw_extend_seeds(bsw_ctx_t *ctx, int64_t n_reads, const uint8_t *reads, const int64_t *read_off,
                     const int32_t *read_len, int64_t n_seeds, const bsw_seed_t *seeds, int32_t max_band_try,
                     bsw_aln_t *out, int64_t *cells_out);

/* The same with an N bitmap of the reads (reads_n: bit p & 7 of byte p >> 3
 * marks read base p, as addressed by read_off, as N; NULL: no N).  With N in
 * the reads or the reference, each side's pairs carry N bitmaps and score N
 * as -1. */
int bsw_extend_seeds_n(bsw_ctx_t *ctx, int64_t n_reads, const uint8_t *reads, const uint8_t *reads_n,
                       const int64_t *read_off, const int32_t *read_len, int64_t n_seeds, const bsw_seed_t *seeds,
                       int32_t max_band_try, bsw_aln_t *out, int64_t *cells_out);

/*
 * Suffix array lookup (Section IV-D, Eq. 1: j = S[i]).
 *
 * bsw_sa_build (host only, no context): the suffix array of codes[0..n)
 * (bases 0..3) followed by a terminator smaller than every base, written to
 * sa[0..n] (n + 1 entries; sa[0] = n).  Built by induced sorting in linear
 * time; an index step, run once per reference.  n < 2^31 - 2.
 * Errors: BSW_EINVAL (bad argument or a code > 3), BSW_ENOMEM.
 */
int bsw_sa_build(const uint8_t *codes, int64_t n, int32_t *sa);

/*
 * bsw_sal_set_index: upload a suffix array of sa_n entries (host pointer) to
 * the context, uncompressed (4 bytes per entry, charged to the budget); it
 * replaces any earlier one.  Errors: BSW_EINVAL, BSW_EBUDGET, BSW_ENOMEM,
 * BSW_ECUDA, BSW_ESTATE (submitted work pending).
 *
 * bsw_sal_lookup: for each SA interval t, positions[off[t] + i] = S[k[t] + i]
 * for 0 <= i < cnt[t] (the reference coordinates of the interval's matches).
 * off[] is the caller's layout of the output (for example the exclusive
 * prefix sum of cnt).  Host pointers (flags 0): the call checks every
 * interval, stages, gathers on the GPU and returns with positions filled.
 * BSW_DEVICE_PTRS: k, cnt, off, positions are device memory; the call only
 * enqueues on cuda_stream (NULL: the context's stream), and an interval
 * outside [0, sa_n) is skipped and reported by bsw_sync.
 * Errors: BSW_EINVAL, BSW_ESTATE (no suffix array), BSW_EBUDGET, BSW_ECUDA.
 */
int bsw_sal_set_index(bsw_ctx_t *ctx, const int32_t *sa, int64_t sa_n);
int bsw_sal_lookup(bsw_ctx_t *ctx, int64_t n_intervals, const int64_t *k, const int32_t *cnt, const int64_t *off,
                   int32_t *positions, uint32_t flags, void *cuda_stream);

/*
 * Super-maximal exact matches (Section IV; Li 2012).
 *
 * bsw_fm_build: index the reference for SMEM search.  The text is
 * T = ref + its reverse complement (the SMEM search covers both strands);
 * the call builds, on the host, the FM-index of T (its suffix array by
 * induced sorting, the occurrence table in buckets of 32 BWT positions) and
 * uploads it (2 bytes per reference base; the suffix array is not kept).
 * ref: codes 0..3, n bases, n < 2^30.
 * Errors: BSW_EINVAL, BSW_ENOMEM, BSW_EBUDGET, BSW_ECUDA, BSW_ESTATE
 * (submitted work pending).
 *
 * bsw_smem: for each read X (2-bit packed at base offset read_off[r], a
 * multiple of 4, with read_len[r] bases), with e(i) the end of the longest
 * prefix of X[i:] occurring in T, the SMEMs are the intervals [i, e(i)) with
 * i = 0 or e(i-1) < e(i) (no longer exact match contains them); those of at
 * least min_len bases are written to out, grouped by read in read order and
 * by qbeg within a read, with [k, k + s) the interval of X[i, e(i)) in the
 * suffix array of T.  first[r] (n_reads + 1 entries, nullable) receives the
 * index of read r's first record.  *n_out receives the number of records;
 * if it exceeds out_cap nothing is written to out and BSW_EBUDGET is
 * returned (call again with a larger out).  Device memory: about 300 bytes
 * per read besides the reads, plus 16 * (max(read_len) + 1) bytes per read
 * whose search needs more than 24 match intervals at once.
 * bsw_smem_n also takes an N bitmap of the reads (bit p & 7 of byte p >> 3
 * marks base p as N; NULL: none): an N occurs nowhere in T, so no match
 * contains one.
 * Errors: BSW_EINVAL, BSW_ESTATE (no index), BSW_EBUDGET, BSW_ECUDA.
 */
typedef struct {
    int32_t read_id;   /* the read                                              */
    int32_t qbeg, len; /* the match: read bases [qbeg, qbeg + len)              */
    int32_t reserved;
    int64_t k, s;      /* its suffix-array interval [k, k + s) in T (s = count) */
} bsw_smem_t;

int bsw_fm_build(bsw_ctx_t *ctx, const uint8_t *ref, int64_t n);
int bsw_smem(bsw_ctx_t *ctx, int64_t n_reads, const uint8_t *reads, const int64_t *read_off,
             const int32_t *read_len, int32_t min_len, bsw_smem_t *out, int64_t out_cap, int64_t *n_out,
             int64_t *first);
int bsw_smem_n(bsw_ctx_t *ctx, int64_t n_reads, const uint8_t *reads, const uint8_t *reads_n, const int64_t *read_off,
               const int32_t *read_len, int32_t min_len, bsw_smem_t *out, int64_t out_cap, int64_t *n_out,
               int64_t *first);

/* Library version string. */
const char *bsw_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BSW_H */
