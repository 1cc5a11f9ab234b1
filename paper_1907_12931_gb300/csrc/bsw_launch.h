// bsw_launch.h - host-side entry points into the BSW kernels.
#pragma once

#include <cuda_runtime.h>
#include <vector>
#include "bsw_device.cuh"

namespace bsw {

// Shared memory a warp-per-pair block may use for its slot rings.
constexpr size_t kRingSmemMax = 96 * 1024;

// Warp-per-pair kernels: 8 warps per block, 2 blocks per SM.
constexpr int kWarpKernelThreads = 256;
constexpr int kWarpBlocksPerSM = 2;

// Query-length upper bounds of the 8-bit (classes 0-7) and 16-bit (classes
// 8-11) per-thread kernels.
constexpr int kU8Nmax[8] = {256, 224, 192, 160, 128, 96, 64, 32};
constexpr int kI16Nmax[4] = {256, 128, 64, 32};

struct Streams {
    cudaStream_t main;
    cudaStream_t side[3];
    cudaEvent_t fork;
    cudaEvent_t join[3];
};

// How one batch is laid out over the kernels: which query lengths run one
// pair per thread and which one pair per warp, the per-thread length classes
// (bucket boundaries), two pairs per thread or one, the warp kernel's columns
// per lane (tile width) and the per-thread kernels' warps per block.  Every
// plan computes the same results; only the speed differs.
struct Plan {
    int32_t short_max;
    ClassTable cls;
    bool packed;
    int32_t warp_cols;     // 4, 8 or 16
    int32_t inter_warps;   // 1, 2 or 4
    int32_t cta_min;       // queries of at least this many bases in the 16-bit range run one pair per block (0: none)
    bool warp_x2;          // the 16-bit warp class runs the two-columns-per-instruction kernel (where it applies)
};

// u8_mask bit k enables kU8Nmax[k] as a class (bit 0 is always on), i16_mask
// bit k enables kI16Nmax[k]; a query goes to the smallest enabled class that
// holds it.  cta_min: 0, or a multiple of 64 in [128, kLongMax].  Returns
// false for values out of range.
bool make_plan(int short_max, uint32_t u8_mask, uint32_t i16_mask, bool packed, int warp_cols, int inter_warps,
               int cta_min, bool warp_x2, Plan *out);
Plan default_plan();

// The 16-bit warp kernel with two columns per instruction (bsw_warp2.cu):
// whether the scoring suits it (match <= 3, so scores up to 2^13 fit, and
// gap costs that fit 16-bit halves), the
// ring for the context's band (0: too large for shared memory), the
// per-device set-up, and the launch over one class list.
bool x2_usable(const Params &P);
int x2_ring_log2(const Params &P);
cudaError_t prepare_x2(int sms);
cudaError_t launch_x2(const Batch &B, const Params &P, const Work &W, int cls, cudaStream_t st, int sms);
// Its plain baseline over pairs in input order (the pairs it cannot take are
// left on the re-run list, which the caller runs with the 32-bit kernel).
cudaError_t launch_plain_x2(const Batch &B, const Params &P, const Work &W, cudaStream_t st, int sms);

// Whether the scoring lets the packed two-pairs-per-thread kernel run.
bool packed_scoring_ok(const Params &P);

// Kernels one launch_batched call makes under the plan and batch flags.
int batched_launches(const Plan &L, uint32_t flags);

// Optional CUDA events around each class kernel (timing-enabled events,
// recorded on the stream the kernel is launched on).
struct ClassTimer {
    cudaEvent_t t0[kNumClass + 1], t1[kNumClass + 1];
    bool used[kNumClass + 1];
};

// Kernel attributes and occupancy; call once per device before any launch
// (and before any stream capture).
cudaError_t prepare_kernels(int sms);

// Number of per-warp slot regions the warp-per-pair kernels use.
int warp_slots_needed(int sms);

// Length-bucketed batched path: classify + counting sort + per-class
// persistent kernels (forked over the side streams) + 32-bit re-run.
// W.hist must be zero on entry (k_scan leaves it zero); W.cells and W.status
// accumulate.  T (nullable) records each launched class kernel's events.
cudaError_t launch_batched(const Batch &B, const Params &P, const Work &W, const Streams &S, int sms, const Plan &L,
                           ClassTimer *T = nullptr);

// The same path on one stream (no side streams, no events); the warp-per-pair
// kernels use warp_blocks blocks of kWarpKernelThreads threads.
cudaError_t launch_batched_serial(const Batch &B, const Params &P, const Work &W, cudaStream_t st, int sms,
                                  int warp_blocks, const Plan &L);

// Baseline: one pair per warp in input order, the warp kernel with the
// plan's columns per lane, or the two-columns kernel when the plan selects it
// (then the 32-bit kernel over the pairs it left), or, with BSW_PLAIN_GLOBAL
// in P.flags, the naive one-column-per-lane kernel with its row in global
// memory.
cudaError_t launch_plain(const Batch &B, const Params &P, const Work &W, cudaStream_t st, int sms, const Plan &L);
// Kernels launch_plain makes under the plan and flags.
int plain_launches(const Params &P, const Plan &L, uint32_t flags);

// Per-pair arrays of a host batch already on the device, checked and reduced
// there: whether any pair is invalid (the checks of bsw_extend_batch) and, over
// the pairs with both sides non-empty, the packed-byte extents of q and t and
// the longest query.
struct PairMeta {
    const int64_t *q_off;
    const int32_t *q_len;
    const int64_t *t_off;
    const int32_t *t_len;
    const int32_t *h0;
    const int32_t *w;   // nullable
};
struct Extents32 {
    unsigned long long q_lo, t_lo;   // start at ~0
    unsigned long long q_hi, t_hi;   // the rest start at 0
    int32_t maxn;
    uint32_t inval;
};
cudaError_t launch_extents(const PairMeta &M, int64_t n, const Params &P, Extents32 *X, cudaStream_t st, int sms);

// ---------------------------------------------------- seed-extension driver

// Device inputs of bsw_extend_seeds (packed reads and reference, seeds).
struct DriverIn {
    const bsw_seed_t *seeds;
    const uint8_t *reads;
    const int64_t *read_off;
    const int32_t *read_len;
    const uint8_t *ref;
    int64_t ref_len;
    const uint8_t *reads_n, *ref_n;   // N bitmaps (bit p & 7 of byte p >> 3), nullable
};

// One side's pairs: packed sequences in fixed per-seed slots of qslot/tslot
// bases, the pair arrays of a Batch, the band of each pair's last run and
// the results.
struct DriverSide {
    uint8_t *q, *t;
    int64_t *q_off, *t_off;
    int32_t *q_len, *t_len, *h0, *w_cur;
    bsw_result_t *res;
    int qslot, tslot;
    uint8_t *q_n, *t_n;   // N bitmaps of the slots (both or neither), nullable
};

// Checks of bsw_extend_seeds' inputs, on the device: every read's offset and
// length, every seed inside its read and the reference, each read's seeds
// consecutive (runs[r] counts the runs of read r's seeds; zeroed by the
// caller), the right side's score bound.  Also the packed-read extent and the
// longest read.  read_bytes and maxrl start at 0, inval at 0.
struct DriverCheck {
    unsigned long long read_bytes;
    int32_t maxrl;
    uint32_t inval;
};
cudaError_t launch_driver_check(const DriverIn &D, int64_t n_reads, int64_t n_seeds, int match, uint32_t *runs,
                                DriverCheck *X, cudaStream_t st, int sms);

// The compact batch of a band retry (the sequences stay in DriverSide).
struct DriverCompact {
    int64_t *q_off, *t_off;
    int32_t *q_len, *t_len, *h0, *w;
    bsw_result_t *res;
};

cudaError_t launch_side(bool left, const DriverIn &D, const DriverSide &S, int64_t n, int w, int match,
                        cudaStream_t st, int sms);
cudaError_t launch_retry_select(const DriverSide &S, int64_t n, int wt, int32_t *list, uint32_t *count,
                                cudaStream_t st, int sms);
cudaError_t launch_retry_gather(const DriverSide &S, const int32_t *list, const uint32_t *count, int64_t n_max,
                                int wnext, const DriverCompact &C, cudaStream_t st, int sms);
cudaError_t launch_retry_scatter(const DriverSide &S, const int32_t *list, const uint32_t *count, int64_t n_max,
                                 int wnext, const DriverCompact &C, cudaStream_t st, int sms);
cudaError_t launch_decide(bool left, const DriverIn &D, const DriverSide &S, int64_t n, int end_bonus,
                          bsw_aln_t *out, cudaStream_t st, int sms);
cudaError_t launch_filter(const DriverIn &D, int64_t n, bsw_aln_t *out, cudaStream_t st, int sms);

// ----------------------------------------------------- FM-index and SMEMs

// One bucket of the occurrence table: counts of each base in BWT[0, 32t)
// and the bucket's 32 BWT bases, 2-bit packed (32 bytes, one DRAM sector).
struct FmEntry {
    uint32_t cnt[4];
    uint64_t bwt;
    uint64_t pad;
};

// Host copy of one FM-index: n = text length + 1 BWT rows, the $ row, the
// first row of each base's block (C[0] = 1 for $, C[4] = n).
struct FmHost {
    int64_t n = 0, primary = -1;
    int64_t C[5] = {0, 0, 0, 0, 0};
    std::vector<FmEntry> occ;
};

struct FmDev {
    const FmEntry *occ;
    int64_t n, primary;
    int64_t C[5];
};

// Reads of an SMEM search: packed 2-bit, read r at base offset read_off[r]
// with read_len[r] <= lmax bases.
struct SmemIn {
    const uint8_t *reads;
    const int64_t *read_off;
    const int32_t *read_len;
    int64_t n_reads;
    int lmax;
    const uint8_t *reads_n;   // N bitmap of the reads, nullable
};

// The index of text[0..n) from its suffix array sa[0..n] (host).
void fm_from_sa(const uint8_t *text, int64_t n, const int32_t *sa, FmHost &out);
// end[r * lmax + i] = the end of the longest prefix of read r from i that
// occurs in the text of Frev's reverse.
// One bi-interval (Algorithm 2): [k, k + s) the suffix-array interval of a
// match P in T, [l, l + s) that of revcomp(P), e the match's end in the read.
struct BiIv {
    uint32_t k, l, s;
    int32_t e;
};
constexpr int kSmemThreads = 128, kListCap = 24, kSmemBlocksPerSm = 4, kSmemKeep = 8;

// Buffers of one SMEM search.  Store mode: count[r] (-1 and r appended to
// ovf_list[atomicAdd(ovf_n)] when the read's list exceeds kListCap) and up to
// kSmemKeep records at scratch[r * kSmemKeep].  Write mode: records at
// out[first[r]].  next: the launch's read counter (zeroed by the launchers).
struct SmemWork {
    int64_t *count;
    bsw_smem_t *scratch;
    const int64_t *first;
    bsw_smem_t *out;
    uint32_t *next;
    uint32_t *ovf_n;
    int32_t *ovf_list;
};
cudaError_t launch_smem_store(const SmemIn &R, const FmDev &F, int min_len, const SmemWork &W, cudaStream_t st, int sms);
// The reads ids[0..n_ids) in store or write mode with lists in `lists` (cap
// entries per lane, n_ids lanes at most).
cudaError_t launch_smem_global(bool write, const SmemIn &R, const FmDev &F, int min_len, const SmemWork &W,
                               const int32_t *ids, int64_t n_ids, BiIv *lists, int cap, cudaStream_t st, int sms);
// Records of reads with count <= kSmemKeep from the scratch to out[first[r]].
cudaError_t launch_smem_gather(int64_t n_reads, const SmemWork &W, cudaStream_t st, int sms);

// Suffix array lookup: out[off[t] + i] = sa[k[t] + i] for i < cnt[t].
// Intervals outside [0, sa_n) set kStInval in *status and write nothing.
cudaError_t launch_sal(const int32_t *sa, int64_t sa_n, const int64_t *k, const int32_t *cnt, const int64_t *off,
                       int64_t n_int, int32_t *out, uint32_t *status, cudaStream_t st, int sms);

}  // namespace bsw
