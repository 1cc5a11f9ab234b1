// bsw_device.cuh - device-side types shared by the BSW kernels and their launcher.
#pragma once

#include <cstdint>
#include "bsw.h"

namespace bsw {

// Query lengths up to kShortMax run in the per-thread (inter-task) kernels;
// longer ones, and every pair of the 32-bit re-run, in the warp-per-pair kernel.
constexpr int kShortMax = 256;
// Longest query the warp-per-pair kernel's slot scratch is sized for.
constexpr int kLongMax = BSW_MAX_QLEN;

// Pair classes.  Classes 0-7: 8-bit lanes for query lengths (192,256],
// (128,192], (96,128], (64,96], (48,64], (32,48], (16,32], [1,16]; 8-11:
// 16-bit lanes for (128,256], (64,128], (32,64], [1,32]; 12: block (several
// warps) per pair, the longest queries of the 16-bit range; 13: warp per pair
// with 16-bit-range scores; 14: warp per pair with 32-bit scores; 15: the
// re-run list.
constexpr int kNumClass = 15;
constexpr int kRerun = 15;
constexpr int kClsCTA = 12, kClsW16 = 13, kClsW32 = 14;
// Work counters: one per class and the re-run list, then the 64-bit counter
// (two words, 8-byte aligned) of the two-columns warp kernel's first wave.
constexpr int kStrata = kNumClass + 1;
constexpr int kNumCounters = kNumClass + 3;

// Counting-sort bins.  Within a class the bins run from long to short queries,
// so the persistent kernels take the longest work first.  The 8-bit bins also
// split each query length by h0 (16 buckets of 16, largest first): a pair's
// band starts about h0 columns wide, so 32 pairs of one bucket keep the lanes
// of a warp on similar trip counts.
constexpr int kU8H0Buckets = 16;
constexpr int kBinU8 = 0, kBinI16 = 256 * kU8H0Buckets, kBinW16 = kBinI16 + 256, kBinW32 = kBinW16 + 640,
              kNumBins = kBinW32 + 640;

// Status bits written by the kernels.
constexpr uint32_t kStInval = 1u;      // an input value is out of range
constexpr uint32_t kStTooLong = 2u;    // a query exceeds the slot scratch

struct Params {
    int32_t a, b, o_del, e_del, o_ins, e_ins, w, zdrop, end_bonus;
    uint32_t flags;
    int32_t max_qlen;   // longer queries are rejected (kStTooLong)
    // 1<<8, 1<<16, 1<<24 as launch parameters: multiplying by them moves a
    // byte with a multiply-add (FMA pipe) instead of a permute or shift (ALU).
    uint32_t k8, k16, k24;
    // Queries longer than this run one pair per warp (the per-thread classes
    // take the rest, up to kShortMax); a tuning choice, 64 <= short_max <= 256.
    int32_t short_max;
};

// Class c covers the counting-sort bins [b[c], b[c+1]); a class with an empty
// range is not launched.  Set from the tuning plan (bucket boundaries).
struct ClassTable {
    int32_t b[kNumClass + 1];
};

struct Batch {
    int64_t n;
    const uint8_t *q;
    const int64_t *q_off;
    const int32_t *q_len;
    const uint8_t *t;
    const int64_t *t_off;
    const int32_t *t_len;
    const int32_t *h0;
    const int32_t *w_override;
    bsw_result_t *out;
    // N bitmaps (nullable): bit (p & 7) of byte p >> 3 marks base p of q / t
    // as N, which scores -1 against any base
    const uint8_t *q_n, *t_n;
};

// One pair's fields as the counting sort lays them out in sorted order (32
// bytes), so the class kernels read them coalesced instead of gathering six
// arrays at random positions.
struct __align__(16) PairRec {
    int64_t q_off, t_off;
    int32_t n, m, h0, w;
};

// Device scratch for one batch launch (allocated and owned by the host runtime).
struct Work {
    int32_t *key;              // [n] counting-sort bin, -1 = done or invalid
    int32_t *order;            // [n] pair ids grouped by bin
    PairRec *rec;              // [n] the pairs' fields in the same order (nullable)
    uint32_t *hist;            // [kNumBins], zero between launches
    uint32_t *cursor;          // [kNumBins]
    int32_t *cls_start;        // [kNumClass + 1]
    int32_t *cls_count;        // [kNumClass + 1]
    uint32_t *cls_next;        // [kNumCounters] work counters of the persistent kernels
    int32_t *rerun;            // [n] pairs to redo with 32-bit lanes
    unsigned long long *cells; // DP cells computed
    uint32_t *status;          // kSt* bits
    uint8_t *slots;            // warp-per-pair slot scratch
    int64_t slot_bytes_per_warp;
};

// Device helpers shared by the kernel translation units.
#ifdef __CUDACC__
constexpr unsigned kFull = 0xffffffffu;
__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel)
{
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}

// Largest gap worth opening: trunc((n*match + end_bonus - o)/e + 1), at least 1.
__device__ __forceinline__ int gap_cap(int n, int a, int eb, int o, int e)
{
    long long x = (long long)n * a + eb - o + e;
    long long k = x / e;
    return (int)(k > 1 ? k : 1);
}

__device__ __forceinline__ int clip_band(const Params &P, int n, int w)
{
    int wi = gap_cap(n, P.a, P.end_bonus, P.o_ins, P.e_ins);
    int wd = gap_cap(n, P.a, P.end_bonus, P.o_del, P.e_del);
    return min(w, min(wi, wd));
}

__device__ __forceinline__ void store_result(bsw_result_t *out, int score, int qle, int tle, int gtle,
                                             int gscore, int moff)
{
    bsw_result_t r;
    r.score = score; r.qle = qle; r.tle = tle; r.gtle = gtle; r.gscore = gscore; r.max_off = moff;
    *out = r;
}
#endif

}  // namespace bsw
