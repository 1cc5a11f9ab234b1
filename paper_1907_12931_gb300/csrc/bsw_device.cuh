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

// Pair classes.  Classes 0-7: 8-bit lanes for query lengths (224,256],
// (192,224], (160,192], (128,160], (96,128], (64,96], (32,64], [1,32] (a
// class of bound N keeps N + 1 slots per thread, so bounds 32 apart keep the
// shared memory a warp holds, and thus the warps per SM, close to what its
// queries need); 8-11:
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

// Whether bases [off, off + len) of an N bitmap hold an N.
__device__ __forceinline__ bool range_has_n(const uint8_t *nm, int64_t off, int len)
{
    if (!nm || len <= 0) return false;
    const int64_t a = off, b = off + len;                 // bits [a, b)
    const int64_t b0 = a >> 3, b1 = (b - 1) >> 3;         // first and last byte
    auto masked = [&](int64_t byte, uint32_t v) {
        if (byte == b0) v &= 0xffu << (a & 7);
        if (byte == b1) v &= 0xffu >> (7 - ((b - 1) & 7));
        return v;
    };
    if (masked(b0, __ldg(nm + b0))) return true;
    int64_t byte = b0 + 1;
    for (; byte <= b1 && (reinterpret_cast<uintptr_t>(nm + byte) & 7); ++byte)   // up to an 8-byte boundary
        if (masked(byte, __ldg(nm + byte))) return true;
    for (; byte + 8 <= b1; byte += 8)                    // 8 whole bytes strictly between b0 and b1
        if (__ldg(reinterpret_cast<const unsigned long long *>(nm + byte)) != 0ull) return true;
    for (; byte <= b1; ++byte)
        if (masked(byte, __ldg(nm + byte))) return true;
    return false;
}

__device__ __forceinline__ bool pair_has_n(const Batch &B, int64_t qo, int n, int64_t to, int m)
{
    return range_has_n(B.q_n, qo, n) || range_has_n(B.t_n, to, m);
}

// Checks of one pair for the plain kernels (the checks k_classify makes);
// answers pairs with an empty side.  Returns the pair's score bound, or -1
// when there is nothing to compute.
__device__ __forceinline__ long long plain_check(const Batch &B, const Params &P, const Work &W, int64_t p,
                                                 int lane)
{
    const int n = B.q_len[p], m = B.t_len[p], h0 = B.h0[p];
    const int64_t qo = B.q_off[p], to = B.t_off[p];
    const int w = B.w_override ? B.w_override[p] : P.w;
    if (n < 0 || m < 0 || h0 < 0 || w < 0 || qo < 0 || to < 0 || (qo & 3) || (to & 3)) {
        if (lane == 0) atomicOr(W.status, kStInval);
        return -1;
    }
    if (n == 0 || m == 0) {
        if (lane == 0) store_result(&B.out[p], h0, 0, 0, 0, n == 0 ? h0 : -1, 0);
        return -1;
    }
    const long long bound = (long long)h0 + (long long)P.a * min(n, m);
    if (bound >= (1ll << 30)) {
        if (lane == 0) atomicOr(W.status, kStInval);
        return -1;
    }
    if (n > P.max_qlen) {
        if (lane == 0) atomicOr(W.status, kStTooLong);
        return -1;
    }
    return bound;
}
#endif

}  // namespace bsw
