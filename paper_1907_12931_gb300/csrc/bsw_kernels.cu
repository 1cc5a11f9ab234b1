// bsw_kernels.cu - sm_103a kernels for banded Smith-Waterman seed extension.
//
// The extension of one pair follows Section V-A of the paper: Eq. 2 per cell,
// the Eq. 3 boundary, the band (rule a), the all-zero / z-drop stop (rule b)
// and the band adjustment after each row (rule c), keeping one row of H and E
// (the "slots"), with BWA-MEM's semantics where the text leaves a choice.
// Slot c holds, between rows, H of column c-1 (the next row's diagonal) and the
// E entering column c.  A row writes slots [lo, hi] only; slots past the band
// keep what an earlier row left there, and a band that regrows reads them.
//
// Kernels
//   k_classify/k_scan/k_scatter  length bucketing (Section V-C1's sort by
//                                length, as a device counting sort)
//   k_inter<NMAX, U8>            one pair per thread: the paper's inter-task
//                                SIMD (Section V-C) mapped onto SIMT lanes;
//                                8-bit or 16-bit lanes (Section V-D1)
//   k_warp<C, S16>               one pair per warp, row-synchronous: each lane
//                                owns C consecutive columns of a row chunk and
//                                F is a max-plus scan across lanes; used for
//                                long queries and the 32-bit re-run
//   k_plain<C>                   the baseline: the warp-per-pair ring kernel
//                                over pairs in input order, no batching
//   k_plain_global               the naive baseline: one column per lane and
//                                the row in global memory
#include <cuda_runtime.h>
#include <cstdint>

#include "bsw_device.cuh"
#include "bsw_launch.h"

namespace bsw {

constexpr int kNeg = -(1 << 29);

// ------------------------------------------------------------------ bucketing

__device__ __forceinline__ int pick_bin(int n, long long bound, uint32_t flags, int short_max, int h0, bool has_n)
{
    const int u8 = kBinU8 + (kShortMax - n) * kU8H0Buckets + (kU8H0Buckets - 1 - min(h0 >> 4, kU8H0Buckets - 1));
    const int rank = 639 - min(n >> 6, 639);
    if (flags & BSW_FORCE_I32) return kBinW32 + rank;
    // Pairs with an N base: the 8-bit per-thread kernels score N, the 32-bit
    // warp kernel does; the 16-bit and packed kernels do not take them.
    if (has_n) {
        const bool f8 = (flags & BSW_FORCE_I8) != 0;
        if (!(flags & BSW_FORCE_I16) && n <= (f8 ? kShortMax : short_max) && (f8 || bound <= 255)) return u8;
        return kBinW32 + rank;
    }
    // The forced lane widths are test modes: they keep every query up to
    // kShortMax on the per-thread kernels whatever the plan says.
    if (n <= ((flags & (BSW_FORCE_I8 | BSW_FORCE_I16)) ? kShortMax : short_max)) {
        if (flags & BSW_FORCE_I8) return u8;
        if (flags & BSW_FORCE_I16) return kBinI16 + (kShortMax - n);
        if (bound <= 255) return u8;
        if (bound <= 32767) return kBinI16 + (kShortMax - n);
        return kBinW32 + rank;
    }
    return bound <= 32767 ? kBinW16 + rank : kBinW32 + rank;
}

__device__ __forceinline__ int n_bit(const uint8_t *nm, int64_t pos)
{
    return (__ldg(nm + (pos >> 3)) >> (pos & 7)) & 1;
}

// Validate each pair, answer the empty ones, and histogram the rest by bin.
__global__ void __launch_bounds__(512) k_classify(Batch B, Params P, Work W)
{
    __shared__ uint32_t sh[kNumBins];
    for (int k = threadIdx.x; k < kNumBins; k += blockDim.x) sh[k] = 0;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < B.n; p += stride) {
        const int n = B.q_len[p], m = B.t_len[p], h0 = B.h0[p];
        const int64_t qo = B.q_off[p], to = B.t_off[p];
        const int w = B.w_override ? B.w_override[p] : P.w;
        int key = -1;
        if (n < 0 || m < 0 || h0 < 0 || w < 0 || qo < 0 || to < 0 || (qo & 3) || (to & 3)) {
            atomicOr(W.status, kStInval);
        } else if (n == 0) {
            store_result(&B.out[p], h0, 0, 0, 0, h0, 0);
        } else if (m == 0) {
            store_result(&B.out[p], h0, 0, 0, 0, -1, 0);
        } else {
            const long long bound = (long long)h0 + (long long)P.a * min(n, m);
            if (bound >= (1ll << 30)) atomicOr(W.status, kStInval);
            else if (n > P.max_qlen) atomicOr(W.status, kStTooLong);
            else {
                // an 8-bit pair stays in its bin with or without N: scan the
                // N bitmaps only for the others
                key = pick_bin(n, bound, P.flags, P.short_max, h0, false);
                const bool u8 = key < kBinI16 && !(P.flags & BSW_FORCE_I16);
                if (!u8 && (B.q_n || B.t_n) && pair_has_n(B, qo, n, to, m))
                    key = pick_bin(n, bound, P.flags, P.short_max, h0, true);
            }
        }
        W.key[p] = key;
        if (key >= 0) atomicAdd(&sh[key], 1u);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kNumBins; k += blockDim.x)
        if (sh[k]) atomicAdd(&W.hist[k], sh[k]);
}

// One block of 1024 threads: exclusive scan of the histogram into the scatter
// cursors, class ranges (class c covers bins [T.b[c], T.b[c+1])), and a reset
// of the histogram and work counters.  Thread t scans kScanPer consecutive bins.
constexpr int kScanPer = (kNumBins + 1023) / 1024;

__global__ void __launch_bounds__(1024) k_scan(Work W, ClassTable T)
{
    __shared__ uint32_t pre[kNumBins + 1];
    __shared__ uint32_t wsum[32];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    uint32_t v[kScanPer];
    uint32_t s = 0;
#pragma unroll
    for (int u = 0; u < kScanPer; ++u) {
        const int idx = t * kScanPer + u;
        v[u] = idx < kNumBins ? W.hist[idx] : 0u;
        s += v[u];
    }
    uint32_t x = s;
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t y = __shfl_up_sync(kFull, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t w = wsum[lane];
        for (int d = 1; d < 32; d <<= 1) {
            uint32_t y = __shfl_up_sync(kFull, w, d);
            if (lane >= d) w += y;
        }
        wsum[lane] = w;
    }
    __syncthreads();
    uint32_t run = x - s + (wid ? wsum[wid - 1] : 0u);
#pragma unroll
    for (int u = 0; u < kScanPer; ++u) {
        const int idx = t * kScanPer + u;
        if (idx < kNumBins) {
            pre[idx] = run;
            W.cursor[idx] = run;
            W.hist[idx] = 0;
        }
        run += v[u];
    }
    if (t == 0) pre[kNumBins] = wsum[31];
    __syncthreads();
    if (t < kNumClass) {
        W.cls_start[t] = (int32_t)pre[T.b[t]];
        W.cls_count[t] = (int32_t)(pre[T.b[t + 1]] - pre[T.b[t]]);
    }
    if (t == kRerun) { W.cls_start[t] = 0; W.cls_count[t] = 0; }
    if (t < kNumCounters) W.cls_next[t] = 0;
}

// Place every pair in its bin.  Each block takes tiles of kScatterTile pairs:
// ranks within the tile come from shared-memory atomics, and one global atomic
// per non-empty bin reserves the tile's range in that bin.
constexpr int kScatterThreads = 512, kScatterPer = 8, kScatterTile = kScatterThreads * kScatterPer;

__global__ void __launch_bounds__(kScatterThreads) k_scatter(Batch B, Params P, Work W)
{
    const int64_t n = B.n;
    __shared__ uint32_t cnt[kNumBins];
    __shared__ uint32_t base[kNumBins];
    for (int64_t tile = (int64_t)blockIdx.x * kScatterTile; tile < n; tile += (int64_t)gridDim.x * kScatterTile) {
        for (int k = threadIdx.x; k < kNumBins; k += kScatterThreads) cnt[k] = 0;
        __syncthreads();
        int key[kScatterPer];
        uint32_t rank[kScatterPer];
#pragma unroll
        for (int u = 0; u < kScatterPer; ++u) {
            const int64_t p = tile + u * kScatterThreads + threadIdx.x;
            key[u] = p < n ? W.key[p] : -1;
            rank[u] = key[u] >= 0 ? atomicAdd(&cnt[key[u]], 1u) : 0u;
        }
        __syncthreads();
        for (int k = threadIdx.x; k < kNumBins; k += kScatterThreads)
            if (cnt[k]) base[k] = atomicAdd(&W.cursor[k], cnt[k]);
        __syncthreads();
#pragma unroll
        for (int u = 0; u < kScatterPer; ++u) {
            if (key[u] < 0) continue;
            const int64_t p = tile + u * kScatterThreads + threadIdx.x;
            const uint32_t pos = base[key[u]] + rank[u];
            W.order[pos] = (int32_t)p;
            if (W.rec) {
                PairRec r;
                r.q_off = B.q_off[p];
                r.t_off = B.t_off[p];
                r.n = B.q_len[p];
                r.m = B.t_len[p];
                r.h0 = B.h0[p];
                r.w = B.w_override ? B.w_override[p] : P.w;
                W.rec[pos] = r;
            }
        }
        __syncthreads();
    }
}

// Checks and packed-byte extents of a batch's pairs (block reduction, then one
// atomic per field and block).
__global__ void __launch_bounds__(256) k_extents(PairMeta M, int64_t n, Params P, Extents32 *X)
{
    unsigned long long qlo = ~0ull, qhi = 0, tlo = ~0ull, thi = 0;
    int maxn = 0;
    uint32_t bad = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
        const int32_t ql = M.q_len[k], tl = M.t_len[k], h0 = M.h0[k];
        const int64_t qo = M.q_off[k], to = M.t_off[k];
        const int32_t w = M.w ? M.w[k] : P.w;
        if (ql < 0 || tl < 0 || h0 < 0 || w < 0 || qo < 0 || to < 0 || (qo & 3) || (to & 3)) {
            bad = 1;
            continue;
        }
        if (ql > 0 && tl > 0) {
            if ((long long)h0 + (long long)P.a * min(ql, tl) >= (1ll << 30) || ql > kLongMax) bad = 1;
            qlo = min(qlo, (unsigned long long)(qo >> 2));
            qhi = max(qhi, (unsigned long long)((qo + ql + 3) >> 2));
            tlo = min(tlo, (unsigned long long)(to >> 2));
            thi = max(thi, (unsigned long long)((to + tl + 3) >> 2));
            maxn = max(maxn, ql);
        }
    }
    for (int d = 16; d > 0; d >>= 1) {
        qlo = min(qlo, __shfl_xor_sync(kFull, qlo, d));
        qhi = max(qhi, __shfl_xor_sync(kFull, qhi, d));
        tlo = min(tlo, __shfl_xor_sync(kFull, tlo, d));
        thi = max(thi, __shfl_xor_sync(kFull, thi, d));
        maxn = max(maxn, __shfl_xor_sync(kFull, maxn, d));
        bad |= __shfl_xor_sync(kFull, bad, d);
    }
    __shared__ unsigned long long s[8][4];
    __shared__ int sm[8];
    __shared__ uint32_t sb[8];
    const int wid = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        s[wid][0] = qlo; s[wid][1] = qhi; s[wid][2] = tlo; s[wid][3] = thi;
        sm[wid] = maxn;
        sb[wid] = bad;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int u = 1; u < (int)(blockDim.x >> 5); ++u) {
            qlo = min(qlo, s[u][0]); qhi = max(qhi, s[u][1]);
            tlo = min(tlo, s[u][2]); thi = max(thi, s[u][3]);
            maxn = max(maxn, sm[u]);
            bad |= sb[u];
        }
        atomicMin(&X->q_lo, qlo);
        atomicMax(&X->q_hi, qhi);
        atomicMin(&X->t_lo, tlo);
        atomicMax(&X->t_hi, thi);
        atomicMax(&X->maxn, maxn);
        if (bad) atomicOr(&X->inval, 1u);
    }
}

// ------------------------------------------------------- one pair per thread

// Slot word layouts (32 bits per column, column j of lane L at S[j*32 + L]):
//   8-bit lanes : bits 0-15 a byte-permute selector for the query base q
//                 (q*0x1111 | 0x8880 picks byte q of the row's score profile
//                 and sign-extends it), bits 16-23 E, bits 24-31 H.  E is
//                 read with a byte load of the lane's own word and E, H are
//                 written back with one 16-bit store (shared-memory pipe)
//                 instead of masks and permutes (integer pipe).
//   16-bit lanes: bits 0-14 H, bits 15-29 E, bits 30-31 q.
template <bool U8>
__device__ __forceinline__ uint32_t slot_init(int q, int h)
{
    return U8 ? ((uint32_t)q * 0x1111u | 0x8880u | ((uint32_t)h << 24)) : ((uint32_t)h | ((uint32_t)q << 30));
}

// Whether a slot word holds a nonzero H or E.
template <bool U8>
__device__ __forceinline__ bool slot_nonzero(uint32_t w)
{
    return U8 ? (w >> 16) != 0u : (w & 0x3fffffffu) != 0u;
}

// Extend pair p; the calling thread owns the slot column S[0], S[32], ...
// Returns the cells computed, or 0 after queueing the pair for the 32-bit
// re-run when a score leaves the lane range.
// NM: the batch has N bitmaps (8-bit lanes only); kernels of batches without
// them carry no N code.
template <int NMAX, bool U8, bool NM>
__device__ __forceinline__ unsigned long long inter_pair(const Batch &B, const Params &P, const Work &W,
                                                         int p, const PairRec &R, uint32_t *S)
{
    constexpr int VMAX = U8 ? 255 : 32767;
    const int n = R.n, m = R.m, h0 = R.h0;
    const int wb = clip_band(P, n, R.w);
    const int e_del = P.e_del, e_ins = P.e_ins;
    const int oe_del = P.o_del + e_del, oe_ins = P.o_ins + e_ins;
    if (h0 > VMAX || n > NMAX) {
        W.rerun[atomicAdd(&W.cls_count[kRerun], 1)] = p;
        return 0;
    }

    // Eq. 3, first row: H = h0 at column 0, max(0, h0 - o_ins - c*e_ins) after.
    // 8-bit lanes: an N column gets the selector of byte 4 (the -1 profile).
    const int64_t q_off = R.q_off;
    const uint8_t *qp = B.q + (q_off >> 2);
    for (int c = 0; c <= n; c += 4) {
        const uint32_t byte = c < n ? __ldg(qp + (c >> 2)) : 0u;
        const uint32_t nb = (NM && B.q_n && c < n) ? (uint32_t)__ldg(B.q_n + ((q_off + c) >> 3)) >> ((q_off + c) & 7) : 0u;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int j = c + k;
            if (j <= n) {
                const int hv = j == 0 ? h0 : max(0, h0 - P.o_ins - j * e_ins);
                S[j * 32] = slot_init<U8>((nb >> k) & 1 ? 4 : (byte >> (2 * k)) & 3, hv);
            }
        }
    }
    const uint8_t *tn = NM ? B.t_n : nullptr;
    const int64_t t_off = R.t_off;

    const uint8_t *tp = B.t + (t_off >> 2);
    const uint32_t mb8 = (uint32_t)(-P.b) & 0xffu;
    const uint32_t mis4 = mb8 * 0x01010101u;
    const uint32_t flip = ((uint32_t)P.a ^ mb8) & 0xffu;
    int lo = 0, hi = n;
    int best = h0, bi = -1, bj = -1, gbest = -1, gi = -1, moff = 0;
    unsigned long long ncell = 0;
    uint32_t tbyte = 0;
    for (int i = 0; i < m; ++i) {
        if ((i & 3) == 0) {
            tbyte = __ldg(tp + (i >> 2));
            if (NM && tn) tbyte |= (((uint32_t)__ldg(tn + ((t_off + i) >> 3)) >> ((t_off + i) & 7)) & 15u) << 8;
        }
        const int tb = (tbyte >> (2 * (i & 3))) & 3;
        lo = max(lo, i - wb);
        hi = min(min(hi, i + wb + 1), n);
        // Eq. 3, first column, while the band still touches it.
        int hl = lo == 0 ? max(0, h0 - oe_del - i * e_del) : 0;
        int f = 0, key = 0;   // key = H*256 + j (j < 256): its max is the row max, ties to larger j
        if (U8) {
            // byte c: score of (t_i, c); all -1 for an N row (byte 4, N columns, is -1 too)
            uint32_t prof = mis4 ^ (flip << (8 * tb));
            if (NM && ((tbyte >> (8 + (i & 3))) & 1u)) prof = 0xffffffffu;
            const uint32_t k8 = P.k8;
            // E is loaded as a byte before the word: a byte load issued after
            // the word load would be folded into a shift and mask of the word
            // (integer pipe); issued first it stays a shared-memory load.
            const uint8_t *SE = reinterpret_cast<const uint8_t *>(S) + 2;     // E byte of column 0's word
            uint16_t *SEH = reinterpret_cast<uint16_t *>(reinterpret_cast<uint8_t *>(S) + 2);   // E | H << 8
            if (oe_del == oe_ins && e_del == e_ins) {
#pragma unroll 4
                for (int j = lo; j < hi; ++j) {
                    const int e = SE[j * 128];                                 // E(i, j)
                    const uint32_t wv = S[j * 32];
                    const int sc = (int)prmt(prof, 0xffffffffu, wv);
                    const int d = (int)(wv >> 24);                             // H(i-1, j-1)
                    const int M = __viaddmin_s32(d, sc, (int)((uint32_t)d * k8));   // d > 0 ? d + sc : <= 0
                    const int h = __vimax3_s32(M, e, f);                       // Eq. 2
                    key = max(key, (int)((uint32_t)h * k8) + j);
                    const int t = M - oe_del;
                    const int e2 = __viaddmax_s32_relu(e, -e_del, t);          // E(i+1, j)
                    f = __viaddmax_s32_relu(f, -e_ins, t);                     // F(i, j+1)
                    SEH[j * 64] = (uint16_t)((uint32_t)hl * k8 + (uint32_t)e2);   // H(i, j-1), E(i+1, j)
                    hl = h;
                }
            } else {
#pragma unroll 4
                for (int j = lo; j < hi; ++j) {
                    const int e = SE[j * 128];
                    const uint32_t wv = S[j * 32];
                    const int sc = (int)prmt(prof, 0xffffffffu, wv);
                    const int d = (int)(wv >> 24);
                    const int M = __viaddmin_s32(d, sc, (int)((uint32_t)d * k8));
                    const int h = __vimax3_s32(M, e, f);
                    key = max(key, (int)((uint32_t)h * k8) + j);
                    const int e2 = __viaddmax_s32_relu(e, -e_del, M - oe_del);
                    f = __viaddmax_s32_relu(f, -e_ins, M - oe_ins);
                    SEH[j * 64] = (uint16_t)((uint32_t)hl * k8 + (uint32_t)e2);
                    hl = h;
                }
            }
            SEH[hi * 64] = (uint16_t)((uint32_t)(hl & 0xff) * k8);   // H(i, hi-1), E = 0
        } else {
            const int a = P.a, mb = -P.b;
#pragma unroll 4
            for (int j = lo; j < hi; ++j) {
                const uint32_t wv = S[j * 32];
                const int d = (int)(wv & 0x7fffu);
                const int e = (int)((wv >> 15) & 0x7fffu);
                const int sc = (int)(wv >> 30) == tb ? a : mb;
                const int M = __viaddmin_s32(d, sc, d << 16);
                const int h = __vimax3_s32(M, e, f);
                key = max(key, h * 512 + j);
                const int e2 = __viaddmax_s32_relu(e, -e_del, M - oe_del);
                f = __viaddmax_s32_relu(f, -e_ins, M - oe_ins);
                S[j * 32] = (wv & 0xc0000000u) | ((uint32_t)(e2 & 0x7fff) << 15) | (uint32_t)(hl & 0x7fff);
                hl = h;
            }
            const uint32_t wh = S[hi * 32];
            S[hi * 32] = (wh & 0xc0000000u) | (uint32_t)(hl & 0x7fff);
        }
        const int rm = U8 ? key >> 8 : key >> 9, rj = U8 ? key & 255 : key & 511;
        if (rm > VMAX) {                                   // Section V-D1: widen and redo
            W.rerun[atomicAdd(&W.cls_count[kRerun], 1)] = p;
            return 0;
        }
        if (hi > lo) ncell += (unsigned)(hi - lo);
        if (max(lo, hi) == n) {                            // band reached the query end
            if (hl >= gbest) gi = i;
            gbest = max(gbest, hl);
        }
        if (rm == 0) break;                                // rule b: all-zero row
        if (rm > best) {
            best = rm; bi = i; bj = rj;
            moff = max(moff, abs(rj - i));
        } else if (P.zdrop > 0) {                          // rule b: z-drop
            const int di = i - bi, dj = rj - bj;
            const int drop = di > dj ? best - rm - (di - dj) * e_del : best - rm - (dj - di) * e_ins;
            if (drop > P.zdrop) break;
        }
        int k = lo;                                        // rule c
        while (k < hi && !slot_nonzero<U8>(S[k * 32])) ++k;
        lo = k;
        k = hi;
        while (k >= lo && !slot_nonzero<U8>(S[k * 32])) --k;
        hi = min(k + 2, n);
    }
    store_result(&B.out[p], best, bj + 1, bi + 1, gi + 1, gbest, moff);
    return ncell;
}

// ------------------------------------------ two rows per instruction (8-bit)
//
// The 8-bit class pairs without N bases take rows in pairs: rows i and i+1 sit
// in the low and high halves of s16x2 registers, row i+1 one column behind
// (step s computes cells (i, s) and (i+1, s-1)), so every DPX instruction of
// the cell update (Eq. 2, Eq. 3's affine gaps) advances two cells.  Row i+1
// takes its diagonal H(i, s-2) and its E(i+1, s-1) from row i's registers;
// only row i+1's results go back to the slot column, slot s-1 <- {H(i+1, s-2),
// E(i+2, s-1)}, so a pass reads each slot once and writes it once for two
// rows.  The row selector in bits 0-15 of slot s picks byte q_s of row i's
// profile for the low half and byte 4 + q_{s-1} (row i+1's profile) for the
// high half, both sign-extended, so one byte permute gives both scores.
//
// Row i+1's band depends on row i's rule-c trims, which are known only after
// row i ends.  Its left end is found before the packed loop starts: row i
// runs alone until its first non-zero slot (its trimmed start) is known and
// the band's lower clip is reached.  Its right end, min(last + 2, n) with
// `last` row i's last non-zero slot, equals L + 3 for L the last column where
// H(i, .) > 0 (a slot past L + 1 has H(i, k-1) = 0, and E(i+1, k) > 0 would
// imply H(i, k) > 0); the packed loop tracks L and runs row i+1 up to row i's
// end.  Row i+1's cells past L + 2 see a zero diagonal and a zero E, so they
// hold only F, which is below the in-band row maximum: the row key is
// unchanged, and after the pass their slots get row i's zeros back (the
// values a row-by-row pass leaves there).  The last two or three columns of
// row i+1 run after the loop, once L is known, reading the slot past row i's
// end as a row-by-row pass does (a value an earlier row left there, read when
// the band grows past the previous row's end).
template <int NMAX, bool SYM>
__device__ __forceinline__ unsigned long long inter_pair_rp(const Batch &B, const Params &P, const PairRec &R,
                                                            bsw_result_t *out, uint32_t *S)
{
    const int n = R.n, m = R.m, h0 = R.h0;
    const int wb = clip_band(P, n, R.w);
    const int e_del = P.e_del, e_ins = P.e_ins;
    const int oe_del = P.o_del + e_del, oe_ins = P.o_ins + e_ins;
    const uint32_t k8 = P.k8, k16 = P.k16;          // 2^8, 2^16 (run-time: multiply-adds, not shifts)
    // Zero-diagonal rule: M = min(D + s, D * 128), D * 128 >= D + s for D >= 1
    // (match <= 127) and below 2^15 for D <= 255.  The factor comes from a
    // run-time value so that the product stays a multiply-add (FMA pipe)
    // instead of becoming a shift (integer pipe).
    const uint32_t zmul = k8 >> 1;
    const uint32_t noe_d2 = (uint32_t)(-oe_del & 0xffff) * 0x10001u, noe_i2 = (uint32_t)(-oe_ins & 0xffff) * 0x10001u;
    const uint32_t ne_d2 = (uint32_t)(-e_del & 0xffff) * 0x10001u, ne_i2 = (uint32_t)(-e_ins & 0xffff) * 0x10001u;

    // Eq. 3, first row, and the selectors: slot j = q_j * 0x11 + q_{j-1} * 0x1100
    // + 0xc480 (nibbles q_j, q_j | 8, 4 + q_{j-1}, (4 + q_{j-1}) | 8).
    const int64_t q_off = R.q_off;
    const uint8_t *qp = B.q + (q_off >> 2);
    uint32_t cprev = 0;
    for (int c = 0; c <= n; c += 4) {
        const uint32_t byte = c < n ? __ldg(qp + (c >> 2)) : 0u;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int j = c + k;
            if (j <= n) {
                const uint32_t cj = j < n ? (byte >> (2 * k)) & 3u : 0u;
                const int hv = j == 0 ? h0 : max(0, h0 - P.o_ins - j * e_ins);
                S[j * 32] = cj * 0x11u + cprev * 0x1100u + 0xc480u + ((uint32_t)hv << 24);
                cprev = cj;
            }
        }
    }
    const uint8_t *tp = B.t + (R.t_off >> 2);
    const uint32_t mb8 = (uint32_t)(-P.b) & 0xffu;
    const uint32_t mis4 = mb8 * 0x01010101u;
    const uint32_t flip = ((uint32_t)P.a ^ mb8) & 0xffu;
    const uint8_t *SE8 = reinterpret_cast<const uint8_t *>(S) + 2;                          // E byte of slot 0
    uint16_t *SEH = reinterpret_cast<uint16_t *>(reinterpret_cast<uint8_t *>(S) + 2);     // E | H << 8 of slot 0

    int lo = 0, hi = n;
    int best = h0, bi = -1, bj = -1, gbest = -1, gi = -1, moff = 0;
    unsigned long long ncell = 0;
    uint32_t tbyte = 0, tnext = __ldg(tp);                  // target bases, fetched one byte (4 rows) ahead
    for (int i = 0; i < m; i += 2) {
        if ((i & 3) == 0) {
            tbyte = tnext;
            tnext = i + 4 < m ? __ldg(tp + (i >> 2) + 1) : 0u;
        }
        const int tb0 = (tbyte >> (2 * (i & 3))) & 3, tb1 = (tbyte >> (2 * (i & 3) + 2)) & 3;
        const uint32_t p0 = mis4 ^ (flip << (8 * tb0));      // row i: byte c = s(t_i, c)
        const uint32_t p1 = mis4 ^ (flip << (8 * tb1));      // row i+1
        const bool single = i + 1 == m;
        lo = max(lo, i - wb);
        hi = min(min(hi, i + wb + 1), n);
        const int hl0 = lo == 0 ? max(0, h0 - oe_del - i * e_del) : 0;   // H(i, lo-1), Eq. 3 first column

        // Row i alone from lo until its first non-zero slot and the lower clip
        // of row i+1's band (c0), or to its end.
        int f = 0, hprev = hl0, hprev2 = 0, en_last = 0, key_lo = 0, Lp = 0;
        int lo1 = hi, c0 = -1;
        bool found = false;
        for (int s = lo; s < hi; ++s) {
            const uint32_t wv = S[s * 32];
            const int d = (int)(wv >> 24), e = (int)((wv >> 16) & 0xffu);
            const int sc = (int)(short)prmt(p0, p1, wv);
            const int M = __viaddmin_s32(d, sc, d * (int)zmul);
            const int h = __vimax3_s32(M, e, f);
            const int en = __viaddmax_s32_relu(e, -e_del, M - oe_del);
            f = __viaddmax_s32_relu(f, -e_ins, M - oe_ins);
            key_lo = max(key_lo, h * 256 + s);
            if (h > 0) Lp = s + 1;
            if (!found && (hprev | en)) { found = true; lo1 = s; }
            hprev2 = hprev; hprev = h; en_last = en;
            if (!single && found && s >= max(lo1, i + 1 - wb)) { c0 = s; break; }
        }
        if (single) {                                        // the last row of an odd count
            const int rm = key_lo >> 8, rj = key_lo & 255;
            if (hi > lo) ncell += (unsigned)(hi - lo);
            if (max(lo, hi) == n) {
                const int hl = hi > lo ? hprev : hl0;
                if (hl >= gbest) gi = i;
                gbest = max(gbest, hl);
            }
            if (rm > 0) {
                if (rm > best) {
                    best = rm; bi = i; bj = rj;
                    moff = max(moff, abs(rj - i));
                }
            }
            break;
        }
        if (c0 < 0) c0 = max(lo1, i + 1 - wb);
        const int bnd1 = c0 == 0 ? max(0, h0 - oe_del - (i + 1) * e_del) : 0;   // H(i+1, c0-1)

        // Both rows: step s computes (i, s) low and (i+1, s-1) high.
        uint32_t hA = (uint32_t)hprev | ((uint32_t)bnd1 << 16);   // h of step s-1
        uint32_t hB = (uint32_t)hprev2;                            // h of step s-2 (low half used)
        uint32_t ENp = (uint32_t)en_last;                          // E out of step s-1 (low half used)
        uint32_t F2 = (uint32_t)f;                                 // F(i, s) | F(i+1, s-1) << 16
        uint32_t key2 = (uint32_t)key_lo, L2 = (uint32_t)Lp;       // row keys H * 256 + column; L + 1
        uint32_t j2 = (uint32_t)(c0 + 1) | ((uint32_t)c0 << 16);
#pragma unroll 8
        for (int s = c0 + 1; s < hi; ++s) {
            const uint32_t e = SE8[s * 128];                       // E(i, s): byte load before the word
            const uint32_t wv = S[s * 32];
            const uint32_t Hd2 = hB * k16 + __umulhi(wv, k8);      // H(i-1, s-1) | H(i, s-2) << 16
            const uint32_t Ed2 = ENp * k16 + e;                     // E(i, s) | E(i+1, s-1) << 16
            const uint32_t M2 = __viaddmin_s16x2(Hd2, prmt(p0, p1, wv), Hd2 * zmul);
            const uint32_t h2 = __vimax3_s16x2(M2, Ed2, F2);
            const uint32_t Mi2 = __viaddmax_s16x2_relu(M2, noe_i2, 0u);
            const uint32_t Md2 = SYM ? Mi2 : __viaddmax_s16x2_relu(M2, noe_d2, 0u);
            const uint32_t EN2 = __viaddmax_s16x2_relu(Ed2, ne_d2, Md2);
            F2 = __viaddmax_s16x2_relu(F2, ne_i2, Mi2);
            const uint32_t h2K = h2 * k8;
            key2 = __viaddmax_u16x2(h2K, j2, key2);
            L2 = __viaddmax_u16x2(__viaddmin_u16x2(j2, 0x00010001u, h2K), 0u, L2);   // s + 1 where H(i, s) > 0
            SEH[(s - 1) * 64] = (uint16_t)prmt(EN2, hA, 0x0062u);             // slot s-1 <- E(i+2, s-1), H(i+1, s-2)
            j2 += 0x00010001u;
            hB = hA; hA = h2; ENp = EN2;
        }
        int Hi1, Hi2, Ei1, ce, fh, hlh;                            // row i's last values; row i+1's state
        if (hi > c0 + 1) {
            Hi1 = (int)(hA & 0xffffu); Hi2 = (int)(hB & 0xffffu); Ei1 = (int)(ENp & 0xffffu);
            ce = hi - 1; fh = (int)(F2 >> 16); hlh = (int)(hA >> 16);
        } else {
            Hi1 = hprev; Hi2 = hprev2; Ei1 = en_last;
            ce = c0; fh = 0; hlh = bnd1;
        }
        key_lo = (int)(key2 & 0xffffu);
        int key_hi = (int)(key2 >> 16);
        Lp = (int)(L2 & 0xffffu);

        // Row i: Section V-D's decisions.
        {
            const int rm = key_lo >> 8, rj = key_lo & 255;
            if (hi > lo) ncell += (unsigned)(hi - lo);
            if (max(lo, hi) == n) {
                const int hl = hi > lo ? Hi1 : hl0;
                if (hl >= gbest) gi = i;
                gbest = max(gbest, hl);
            }
            if (rm == 0) break;
            if (rm > best) {
                best = rm; bi = i; bj = rj;
                moff = max(moff, abs(rj - i));
            } else if (P.zdrop > 0) {
                const int di = i - bi, dj = rj - bj;
                const int drop = di > dj ? best - rm - (di - dj) * e_del : best - rm - (dj - di) * e_ins;
                if (drop > P.zdrop) break;
            }
        }
        // Row i+1's band is [c0, hi1); its columns from ce on run here.
        const int i1 = i + 1;
        const int hi1 = min(min(Lp + 2, n), i1 + wb + 1);
        for (int c = ce; c < hi1; ++c) {
            const uint32_t wc = S[c * 32];
            int d, e;
            if (c == hi - 1) { d = Hi2; e = Ei1; }
            else if (c == hi) { d = Hi1; e = 0; }
            else { d = (int)(wc >> 24); e = (int)((wc >> 16) & 0xffu); }   // past row i: the slot as it stands
            const int sc = (int)(signed char)prmt(p1, 0u, wc);
            const int M = __viaddmin_s32(d, sc, d * (int)zmul);
            const int h = __vimax3_s32(M, e, fh);
            const int en = __viaddmax_s32_relu(e, -e_del, M - oe_del);
            fh = __viaddmax_s32_relu(fh, -e_ins, M - oe_ins);
            SEH[c * 64] = (uint16_t)(((uint32_t)hlh << 8) | (uint32_t)en);
            key_hi = max(key_hi, h * 256 + c);
            hlh = h;
        }
        if (hi1 >= ce && hi1 > c0) SEH[hi1 * 64] = (uint16_t)((uint32_t)hlh << 8);   // row end, E = 0
        {
            const int rm = key_hi >> 8, rj = key_hi & 255;
            if (hi1 > c0) ncell += (unsigned)(hi1 - c0);
            if (max(c0, hi1) == n) {
                const int hl = hi1 > c0 ? (int)(S[hi1 * 32] >> 24) : bnd1;
                if (hl >= gbest) gi = i1;
                gbest = max(gbest, hl);
            }
            if (rm == 0) break;
            if (rm > best) {
                best = rm; bi = i1; bj = rj;
                moff = max(moff, abs(rj - i1));
            } else if (P.zdrop > 0) {
                const int di = i1 - bi, dj = rj - bj;
                const int drop = di > dj ? best - rm - (di - dj) * e_del : best - rm - (dj - di) * e_ins;
                if (drop > P.zdrop) break;
            }
        }
        for (int k = hi1 + 1; k <= hi; ++k) SEH[k * 64] = 0;       // row i's zeros past row i+1's end
        int k = c0;                                                // rule c on row i+1
        while (k < hi1 && !slot_nonzero<true>(S[k * 32])) ++k;
        lo = k;
        k = hi1;
        while (k >= lo && !slot_nonzero<true>(S[k * 32])) --k;
        hi = min(k + 2, n);
    }
    store_result(out, best, bj + 1, bi + 1, gi + 1, gbest, moff);
    return ncell;
}

// Whether the row-pair path takes the pair: no N bases (the caller's kernel
// runs it only for batches without N bitmaps), scores and gap terms inside
// the packed 8-bit range.
__device__ __forceinline__ bool rp_eligible(const Params &P, const PairRec &R, int nmax)
{
    return R.n >= 1 && R.m >= 1 && R.n <= nmax && R.h0 >= 0 &&
           (long long)R.h0 + (long long)P.a * min(R.n, R.m) <= 255 && P.a <= 127 && P.o_del + P.e_del <= 30000 &&
           P.o_ins + P.e_ins <= 30000 && P.e_del <= 30000 && P.e_ins <= 30000;
}

template <int NMAX, bool U8, bool NM = false>
__global__ void __launch_bounds__(256) k_inter(Batch B, Params P, Work W, int cls)
{
    extern __shared__ uint32_t smem[];
    const int lane = threadIdx.x & 31;
    uint32_t *S = smem + (threadIdx.x >> 5) * ((NMAX + 1) * 32) + lane;
    const int start = W.cls_start[cls], count = W.cls_count[cls];
    const int ngroups = (count + 31) >> 5;
    unsigned long long cells = 0;
    for (;;) {
        int g = 0;
        if (lane == 0) g = (int)atomicAdd(&W.cls_next[cls], 1u);
        g = __shfl_sync(kFull, g, 0);
        if (g >= ngroups) break;
        const int idx = (g << 5) + lane;
        if (idx < count) {
            const int p = W.order[start + idx];
            PairRec R;
            if (W.rec) {
                R = W.rec[start + idx];
            } else {
                R.q_off = B.q_off[p]; R.t_off = B.t_off[p];
                R.n = B.q_len[p]; R.m = B.t_len[p]; R.h0 = B.h0[p];
                R.w = B.w_override ? B.w_override[p] : P.w;
            }
            if (U8 && !NM && rp_eligible(P, R, NMAX)) {
                cells += (P.o_del == P.o_ins && P.e_del == P.e_ins) ? inter_pair_rp<NMAX, true>(B, P, R, &B.out[p], S)
                                                                   : inter_pair_rp<NMAX, false>(B, P, R, &B.out[p], S);
            } else {
                cells += inter_pair<NMAX, U8, NM>(B, P, W, p, R, S);
            }
        }
        __syncwarp();
    }
    for (int d = 16; d > 0; d >>= 1) cells += __shfl_xor_sync(kFull, cells, d);
    if (lane == 0 && cells) atomicAdd(W.cells, cells);
}

// --------------------------------------------- two pairs per thread (s16x2)
//
// The paper's inter-task SIMD with 16-bit lanes (Section V-C, V-D1), two pairs
// per 32-bit register: one warp holds 64 pairs.  Opt-in (BSW_PACKED_PAIRS).

// Packed 16-bit integer SIMD (two lanes per 32-bit register).
__device__ __forceinline__ uint32_t add2(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("add.s16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ uint32_t max2(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("max.s16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ uint32_t max2relu(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("max.s16x2.relu %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ uint32_t minu2(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

// Scores scaled by 128 in 16-bit lanes: the low 7 bits of H*128 + j carry
// the column (queries up to 128 bases), so one packed max tracks each pair's
// row best with ties to the larger column.
constexpr int kS2 = 7;

// Per-thread state of the two-pair kernel for one row.
struct Row2 {
    uint32_t f2, key2, dprev2, hlast2, tbit2;
};

// Constants of the packed cell update.
struct Cell2K {
    uint32_t nK;      // 0x10000 - (match + mismatch)*128: packed negation of the mismatch cost
    uint32_t noed2;   // -(o_del + e_del)*128 in each lane
    uint32_t noei2;   // -(o_ins + e_ins)*128
    uint32_t ned2;    // -e_del*128
    uint32_t nei2;    // -e_ins*128
    uint32_t a128;    // match*128
};

// Cells [j0, j1) of one row for both lanes.  m: lanes whose band covers the
// range (0xffff per lane); lanes outside it are computed but neither stored
// nor counted.  Slot words: SD[j*32] = D*128 per lane (D = H + match for
// H > 0, else 0: the previous row's H at column j-1); SE[j*32] = E*128 per
// lane in bits 7-14 / 23-30 and the lane's query mismatch mask in bits
// 0-3 / 16-19.
template <bool MASKED>
__device__ __forceinline__ void cells2(uint32_t *SD, uint32_t *SE, int j0, int j1, uint32_t m, Row2 &R,
                                       const Cell2K &K)
{
    const uint32_t keep_e = MASKED ? (m & 0xff80ff80u) : 0xff80ff80u;
    uint32_t J2 = (uint32_t)j0 * 0x00010001u;
#pragma unroll 2
    for (int j = j0; j < j1; ++j) {
        const uint32_t wd = SD[j * 32], we = SE[j * 32];
        const uint32_t e2 = we & 0x7f807f80u;                          // E(i, j)*128
        const uint32_t mm = minu2(we & R.tbit2, 0x00010001u);          // 1 where base != t_i
        const uint32_t M2 = add2(wd, mm * K.nK);                       // Eq. 2 diagonal term
        const uint32_t h2 = max2(max2(M2, e2), R.f2);                  // H(i, j)
        uint32_t hj = add2(h2, J2);
        if (MASKED) hj &= m;
        R.key2 = max2(R.key2, hj);
        const uint32_t en = max2relu(add2(e2, K.ned2), add2(M2, K.noed2));   // E(i+1, j)
        R.f2 = max2relu(add2(R.f2, K.nei2), add2(M2, K.noei2));              // F(i, j+1)
        if (MASKED) {
            SD[j * 32] = (R.dprev2 & m) | (wd & ~m);
            SE[j * 32] = (en & keep_e) | (we & ~keep_e);
        } else {
            SD[j * 32] = R.dprev2;
            SE[j * 32] = en | (we & 0x000f000fu);
        }
        R.dprev2 = minu2(h2, 0x00010001u) * K.a128 + h2;               // D of H(i, j)
        R.hlast2 = h2;
        J2 += 0x00010001u;
    }
}

// Per-pair bookkeeping of the two-pair kernel.
struct Pair2 {
    int p, n, m, h0, wb;
    int lo, hi, best, bi, bj, gbest, gi, moff;
    bool live;
    unsigned long long ncell;
    const uint8_t *tp;
};

__device__ __forceinline__ void pair2_open(Pair2 &X, const Batch &B, const Params &P, int p)
{
    X.p = p;
    X.live = p >= 0;
    if (!X.live) return;
    X.n = B.q_len[p];
    X.m = B.t_len[p];
    X.h0 = B.h0[p];
    X.wb = clip_band(P, X.n, B.w_override ? B.w_override[p] : P.w);
    X.lo = 0; X.hi = X.n;
    X.best = X.h0; X.bi = X.bj = -1; X.gbest = X.gi = -1; X.moff = 0;
    X.ncell = 0;
    X.tp = B.t + (B.t_off[p] >> 2);
}

// Extend pairs pa (low lanes) and pb (high lanes, -1 for none) on one thread.
// Returns the cells computed; pairs whose scores leave the lane range go to
// the 32-bit re-run and count nothing here.
template <int NMAX>
__device__ unsigned long long inter2_pairs(const Batch &B, const Params &P, const Work &W, int pa, int pb,
                                           uint32_t *SD, uint32_t *SE)
{
    const int a = P.a;
    const int vmax = 255 - a;
    Pair2 X[2];
    pair2_open(X[0], B, P, pa);
    pair2_open(X[1], B, P, pb);
    // First row of Eq. 3 and the query masks, per lane.
    const int nmax = max(X[0].live ? X[0].n : 0, X[1].live ? X[1].n : 0);
    for (int j = 0; j <= nmax; ++j) { SD[j * 32] = 0u; SE[j * 32] = 0u; }
    for (int h = 0; h < 2; ++h) {
        if (!X[h].live) continue;
        if (X[h].h0 > vmax || X[h].n > NMAX) {
            W.rerun[atomicAdd(&W.cls_count[kRerun], 1)] = X[h].p;
            X[h].live = false;
            continue;
        }
        const uint8_t *qp = B.q + (B.q_off[X[h].p] >> 2);
        const int sh = 16 * h;
        for (int c = 0; c <= X[h].n; c += 4) {
            const uint32_t byte = c < X[h].n ? __ldg(qp + (c >> 2)) : 0u;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int j = c + k;
                if (j <= X[h].n) {
                    const int hv = j == 0 ? X[h].h0 : max(0, X[h].h0 - P.o_ins - j * P.e_ins);
                    const uint32_t d = hv > 0 ? (uint32_t)(hv + a) << kS2 : 0u;
                    const uint32_t q = (~(1u << ((byte >> (2 * k)) & 3)) & 0xfu);
                    SD[j * 32] |= d << sh;
                    SE[j * 32] |= q << sh;
                }
            }
        }
    }
    const int bm = min(P.b, 255 - a);
    Cell2K K;
    const uint32_t kmis = (uint32_t)((a + bm) << kS2);
    K.nK = 0x10000u - kmis;
    auto rep = [](int v) { return ((uint32_t)v & 0xffffu) * 0x00010001u; };
    K.noed2 = rep(-(min(P.o_del + P.e_del, 255) << kS2));
    K.noei2 = rep(-(min(P.o_ins + P.e_ins, 255) << kS2));
    K.ned2 = rep(-(min(P.e_del, 255) << kS2));
    K.nei2 = rep(-(min(P.e_ins, 255) << kS2));
    K.a128 = (uint32_t)(a << kS2);

    const int oe_del = P.o_del + P.e_del;
    uint32_t tbyte[2] = {0u, 0u};
    for (int i = 0; X[0].live || X[1].live; ++i) {
        int lo[2], hi[2], left[2];
        bool on[2];
        Row2 R;
        R.f2 = 0u; R.key2 = 0u; R.dprev2 = 0u; R.hlast2 = 0u; R.tbit2 = 0u;
        for (int h = 0; h < 2; ++h) {
            if (X[h].live && i >= X[h].m) {                 // every target row done
                store_result(&B.out[X[h].p], X[h].best, X[h].bj + 1, X[h].bi + 1, X[h].gi + 1, X[h].gbest, X[h].moff);
                X[h].live = false;
            }
            on[h] = X[h].live;
            if (!on[h]) { lo[h] = hi[h] = 0; left[h] = 0; continue; }
            if ((i & 3) == 0) tbyte[h] = __ldg(X[h].tp + (i >> 2));
            const int tb = (tbyte[h] >> (2 * (i & 3))) & 3;
            R.tbit2 |= (1u << tb) << (16 * h);
            X[h].lo = max(X[h].lo, i - X[h].wb);
            X[h].hi = min(min(X[h].hi, i + X[h].wb + 1), X[h].n);
            lo[h] = X[h].lo; hi[h] = X[h].hi;
            left[h] = lo[h] == 0 ? max(0, X[h].h0 - oe_del - i * P.e_del) : 0;
        }
        if (!on[0] && !on[1]) break;
        const bool band0 = on[0] && lo[0] < hi[0], band1 = on[1] && lo[1] < hi[1];
        uint32_t hl2 = 0u;                      // H(i, hi-1)*128 per lane (or the left boundary)
        for (int h = 0; h < 2; ++h)
            if (on[h]) hl2 |= ((uint32_t)left[h] << kS2) << (16 * h);
        // Walk the union of the two bands in segments where the active lanes do not change.
        int j = 1 << 30, jend = 0;
        if (band0) { j = min(j, lo[0]); jend = max(jend, hi[0]); }
        if (band1) { j = min(j, lo[1]); jend = max(jend, hi[1]); }
        while (j < jend) {
            int nb = jend;
            uint32_t m = 0u;
            for (int h = 0; h < 2; ++h) {
                const bool bh = h ? band1 : band0;
                if (!bh) continue;
                if (lo[h] > j) nb = min(nb, lo[h]);
                if (hi[h] > j) nb = min(nb, hi[h]);
                if (lo[h] <= j && j < hi[h]) {
                    m |= 0xffffu << (16 * h);
                    if (j == lo[h]) {           // lane h enters its band: fresh F, left boundary
                        const uint32_t lh = (uint32_t)left[h] << kS2;
                        const uint32_t dl = left[h] > 0 ? lh + ((uint32_t)a << kS2) : 0u;
                        R.f2 &= ~(0xffffu << (16 * h));
                        R.dprev2 = (R.dprev2 & ~(0xffffu << (16 * h))) | (dl << (16 * h));
                    }
                }
            }
            if (m == 0xffffffffu) cells2<false>(SD, SE, j, nb, m, R, K);
            else if (m) cells2<true>(SD, SE, j, nb, m, R, K);
            for (int h = 0; h < 2; ++h) {
                const bool bh = h ? band1 : band0;
                if (bh && hi[h] == nb && (m >> (16 * h)) & 1u)     // lane h leaves its band
                    hl2 = (hl2 & ~(0xffffu << (16 * h))) | (R.hlast2 & (0xffffu << (16 * h)));
            }
            j = nb;
        }
        for (int h = 0; h < 2; ++h) {
            if (!on[h]) continue;
            Pair2 &Y = X[h];
            const int sh = 16 * h;
            const int hl = (int)((hl2 >> sh) & 0xffffu) >> kS2;
            // slot hi: H(i, hi-1) and E = 0 for this lane
            const uint32_t dl = hl > 0 ? (uint32_t)(hl + a) << kS2 : 0u;
            SD[Y.hi * 32] = (SD[Y.hi * 32] & ~(0xffffu << sh)) | (dl << sh);
            SE[Y.hi * 32] &= ~(0xff80u << sh);
            const int key = (int)((R.key2 >> sh) & 0xffffu);
            const int rm = key >> kS2, rj = key & ((1 << kS2) - 1);
            if (rm > vmax) {                                   // Section V-D1: widen and redo
                W.rerun[atomicAdd(&W.cls_count[kRerun], 1)] = Y.p;
                Y.live = false;
                Y.ncell = 0;
                continue;
            }
            if (Y.hi > Y.lo) Y.ncell += (unsigned)(Y.hi - Y.lo);
            if (max(Y.lo, Y.hi) == Y.n) {
                if (hl >= Y.gbest) Y.gi = i;
                Y.gbest = max(Y.gbest, hl);
            }
            bool stop = rm == 0;
            if (!stop) {
                if (rm > Y.best) {
                    Y.best = rm; Y.bi = i; Y.bj = rj;
                    Y.moff = max(Y.moff, abs(rj - i));
                } else if (P.zdrop > 0) {
                    const int di = i - Y.bi, dj = rj - Y.bj;
                    const int drop = di > dj ? Y.best - rm - (di - dj) * P.e_del : Y.best - rm - (dj - di) * P.e_ins;
                    stop = drop > P.zdrop;
                }
            }
            if (stop) {
                store_result(&B.out[Y.p], Y.best, Y.bj + 1, Y.bi + 1, Y.gi + 1, Y.gbest, Y.moff);
                Y.live = false;
                continue;
            }
            const uint32_t mk = 0xffffu << sh, mke = 0xff80u << sh;
            int k = Y.lo;                                      // rule c
            while (k < Y.hi && !((SD[k * 32] & mk) | (SE[k * 32] & mke))) ++k;
            Y.lo = k;
            k = Y.hi;
            while (k >= Y.lo && !((SD[k * 32] & mk) | (SE[k * 32] & mke))) --k;
            Y.hi = min(k + 2, Y.n);
        }
    }
    unsigned long long cells = 0;
    for (int h = 0; h < 2; ++h) {
        if (X[h].p < 0) continue;
        cells += X[h].ncell;
    }
    return cells;
}

// Persistent kernel: each warp takes groups of 64 consecutive pairs of its
// class (thread L takes entries 2L and 2L+1, pairs of nearly equal length).
template <int NMAX>
__global__ void __launch_bounds__(256) k_inter2(Batch B, Params P, Work W, int cls)
{
    extern __shared__ uint32_t smem[];
    const int lane = threadIdx.x & 31;
    uint32_t *SD = smem + (threadIdx.x >> 5) * ((NMAX + 1) * 64) + lane;
    uint32_t *SE = SD + (NMAX + 1) * 32;
    const int start = W.cls_start[cls], count = W.cls_count[cls];
    const int ngroups = (count + 63) >> 6;
    unsigned long long cells = 0;
    for (;;) {
        int g = 0;
        if (lane == 0) g = (int)atomicAdd(&W.cls_next[cls], 1u);
        g = __shfl_sync(kFull, g, 0);
        if (g >= ngroups) break;
        const int i0 = (g << 6) + 2 * lane;
        const int pa = i0 < count ? W.order[start + i0] : -1;
        const int pb = i0 + 1 < count ? W.order[start + i0 + 1] : -1;
        if (pa >= 0) cells += inter2_pairs<NMAX>(B, P, W, pa, pb, SD, SE);
        __syncwarp();
    }
    for (int d = 16; d > 0; d >>= 1) cells += __shfl_xor_sync(kFull, cells, d);
    if (lane == 0 && cells) atomicAdd(W.cells, cells);
}

// ---------------------------------------------------------- one pair per warp

// Slot storage for the warp kernels: 16-bit (H low half, E high half of a
// 32-bit word) or 32-bit (an int2 {H, E}).
template <bool S16> struct SlotIO;

template <> struct SlotIO<true> {
    static constexpr int kBytes = 4;
    __device__ static void load(const uint8_t *base, int j, int &h, int &e)
    {
        const uint32_t v = reinterpret_cast<const uint32_t *>(base)[j];
        h = (int)(v & 0xffffu); e = (int)(v >> 16);
    }
    __device__ static void store(uint8_t *base, int j, int h, int e)
    {
        reinterpret_cast<uint32_t *>(base)[j] = (uint32_t)h | ((uint32_t)e << 16);
    }
};

template <> struct SlotIO<false> {
    static constexpr int kBytes = 8;
    __device__ static void load(const uint8_t *base, int j, int &h, int &e)
    {
        const int2 v = reinterpret_cast<const int2 *>(base)[j];
        h = v.x; e = v.y;
    }
    __device__ static void store(uint8_t *base, int j, int h, int e)
    {
        reinterpret_cast<int2 *>(base)[j] = make_int2(h, e);
    }
};

// Extend pair p with the whole warp.  Rows are processed one after the other;
// each row is cut into chunks of 32*C columns, lane L owning columns
// [cb + L*C, cb + L*C + C) of a chunk starting at cb.  M and E are lane-local;
// F(i,j) = max(0, max_k<j (M_k - o_ins - e_ins - (j-1-k) e_ins)) is a max-plus
// prefix over the row, computed per lane and then as a warp scan of the lanes'
// maps f -> max(f - cnt*e_ins, b).  Row decisions (band, stop, best, trim) are
// warp-uniform.  `slots` holds n + 1 + 32*C slots.
//
// RING: the slots live in a shared-memory ring of mask + 1 entries (a power of
// two >= 2*w' + 3) indexed by column & mask.  The band never spans more than
// 2*w' + 2 columns, so a column's ring entry is not reused while the column
// can still be read, including the band-regrowth reads of earlier rows'
// values.  Columns never written before get their first-row value of Eq. 3
// when the band first reaches them (hw is the highest column set so far).
// NM: the batch has N bitmaps; an N on either side scores -1.
template <int C, bool S16, bool RING, bool NM = false>
__device__ unsigned long long warp_pair(const Batch &B, const Params &P, int p, uint8_t *slots, int mask)
{
    using IO = SlotIO<S16>;
    const int lane = threadIdx.x & 31;
    const int n = B.q_len[p], m = B.t_len[p], h0 = B.h0[p];
    const int wb = clip_band(P, n, B.w_override ? B.w_override[p] : P.w);
    const int a = P.a, mb = -P.b;
    const int e_del = P.e_del, e_ins = P.e_ins;
    const int oe_del = P.o_del + e_del, oe_ins = P.o_ins + e_ins;
    auto at = [mask](int j) { return RING ? (j & mask) : j; };
    int hw = -1;
    if (!RING) {
        for (int c = lane; c <= n; c += 32)
            IO::store(slots, c, c == 0 ? h0 : max(0, h0 - P.o_ins - c * e_ins), 0);
        hw = n;
        __syncwarp();
    }

    const int64_t qoff = B.q_off[p];
    const uint8_t *tp = B.t + (B.t_off[p] >> 2);
    int lo = 0, hi = n;
    int best = h0, bi = -1, bj = -1, gbest = -1, gi = -1, moff = 0;
    unsigned long long ncell = 0;
    for (int i = 0; i < m; ++i) {
        const int tb = (__ldg(tp + (i >> 2)) >> (2 * (i & 3))) & 3;
        const bool tn = NM && B.t_n && n_bit(B.t_n, B.t_off[p] + i);
        lo = max(lo, i - wb);
        hi = min(min(hi, i + wb + 1), n);
        if (RING && hi - 1 > hw) {             // first visit of columns (hw, hi-1]
            for (int c = hw + 1 + lane; c <= hi - 1; c += 32)
                IO::store(slots, c & mask, c == 0 ? h0 : max(0, h0 - P.o_ins - c * e_ins), 0);
            hw = hi - 1;
            __syncwarp();
        }
        const int hl0 = lo == 0 ? max(0, h0 - oe_del - i * e_del) : 0;
        int carry_f = 0, carry_h = hl0;
        int rm_l = 0, rj_l = -1;
        for (int cb = (lo / C) * C; cb < hi; cb += 32 * C) {
            const int j0 = cb + lane * C;
            int M[C], E0[C], Fl[C], H[C];
            bool act[C];
            int cnt = 0, floc = 0;
            uint32_t qbits = 0, nq = 0;
            if (j0 < hi && j0 + C > lo) {
#pragma unroll
                for (int k = 0; k < C; k += 4) {
                    const int64_t pos = qoff + j0 + k;
                    if (j0 + k < n) qbits |= (uint32_t)__ldg(B.q + (pos >> 2)) << (2 * k);
                }
                if (C < 4) qbits >>= 2 * ((qoff + j0) & 3);
                if (NM && B.q_n) {                       // N bits of the lane's columns
                    const int64_t pos = qoff + j0;
                    const int bits = (int)(pos & 7) + min(C, n - j0);   // bitmap bits up to the last column
                    const uint8_t *src = B.q_n + (pos >> 3);
                    uint32_t w = __ldg(src);
#pragma unroll
                    for (int b = 1; b <= (C + 7) / 8; ++b)
                        if (8 * b < bits) w |= (uint32_t)__ldg(src + b) << (8 * b);
                    nq = w >> (pos & 7);
                }
            }
#pragma unroll
            for (int k = 0; k < C; ++k) {
                const int j = j0 + k;
                act[k] = j >= lo && j < hi;
                int d = 0, e = 0;
                if (act[k]) IO::load(slots, at(j), d, e);
                int sc = (int)((qbits >> (2 * k)) & 3u) == tb ? a : mb;
                if (NM && (tn || ((nq >> k) & 1u))) sc = -1;
                M[k] = d > 0 ? d + sc : 0;
                E0[k] = e;
                Fl[k] = floc;
                if (act[k]) {
                    floc = __viaddmax_s32_relu(floc, -e_ins, M[k] - oe_ins);
                    ++cnt;
                }
            }
            // Warp scan of f -> max(f - A, Bv), earlier lanes applied first.
            int A = cnt * e_ins, Bv = cnt ? floc : kNeg;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int Ae = __shfl_up_sync(kFull, A, d), Be = __shfl_up_sync(kFull, Bv, d);
                if (lane >= d) { Bv = max(Be - A, Bv); A = Ae + A; }
            }
            int Aex = __shfl_up_sync(kFull, A, 1), Bex = __shfl_up_sync(kFull, Bv, 1);
            if (lane == 0) { Aex = 0; Bex = kNeg; }
            int g = max(carry_f - Aex, Bex);
            int hlast = 0;
#pragma unroll
            for (int k = 0; k < C; ++k) {
                if (act[k]) {
                    const int F = max(Fl[k], g);
                    g -= e_ins;
                    const int h = __vimax3_s32(M[k], E0[k], F);
                    H[k] = h;
                    if (h >= rm_l) { rm_l = h; rj_l = j0 + k; }
                    hlast = h;
                } else {
                    H[k] = 0;
                }
            }
            int hin = __shfl_up_sync(kFull, hlast, 1);
            if (lane == 0 || j0 <= lo) hin = carry_h;
#pragma unroll
            for (int k = 0; k < C; ++k) {
                if (act[k]) {
                    const int e2 = __viaddmax_s32_relu(E0[k], -e_del, M[k] - oe_del);
                    IO::store(slots, at(j0 + k), hin, e2);
                    hin = H[k];
                }
            }
            const int A31 = __shfl_sync(kFull, A, 31), B31 = __shfl_sync(kFull, Bv, 31);
            carry_f = max(carry_f - A31, B31);
            const int end = min(cb + 32 * C, hi);
            carry_h = __shfl_sync(kFull, hlast, (end - 1 - cb) / C);
        }
        const int hl = carry_h;
        __syncwarp();
        if (lane == 0) IO::store(slots, at(hi), hl, 0);
        hw = max(hw, hi);
        __syncwarp();
        const int rm = __reduce_max_sync(kFull, (unsigned)rm_l);
        const int rj = (int)__reduce_max_sync(kFull, (unsigned)(rm_l == rm ? rj_l + 1 : 0)) - 1;
        if (hi > lo) ncell += (unsigned)(hi - lo);
        if (max(lo, hi) == n) {
            if (hl >= gbest) gi = i;
            gbest = max(gbest, hl);
        }
        if (rm == 0) break;
        if (rm > best) {
            best = rm; bi = i; bj = rj;
            moff = max(moff, abs(rj - i));
        } else if (P.zdrop > 0) {
            const int di = i - bi, dj = rj - bj;
            const int drop = di > dj ? best - rm - (di - dj) * e_del : best - rm - (dj - di) * e_ins;
            if (drop > P.zdrop) break;
        }
        // rule c with ballots over 32 slots at a time
        int nlo = hi;
        for (int base = lo; base < hi; base += 32) {
            const int j = base + lane;
            int h = 0, e = 0;
            if (j < hi) IO::load(slots, at(j), h, e);
            const unsigned bal = __ballot_sync(kFull, (h | e) != 0);
            if (bal) { nlo = base + __ffs(bal) - 1; break; }
        }
        lo = nlo;
        int last = lo - 1;
        for (int top = hi; top >= lo; top -= 32) {
            const int j = top - lane;
            int h = 0, e = 0;
            if (j >= lo) IO::load(slots, at(j), h, e);
            const unsigned bal = __ballot_sync(kFull, (h | e) != 0);
            if (bal) { last = top - (__ffs(bal) - 1); break; }
        }
        hi = min(last + 2, n);
    }
    if (lane == 0) store_result(&B.out[p], best, bj + 1, bi + 1, gi + 1, gbest, moff);
    return ncell;
}

// Ring position (in 8-byte slots) of column j with one padding slot per C:
// lane L of a full chunk reads column cb + C*L + k (cb a multiple of C), at
// slot const + (C+1)*L + k.  A warp's 64-bit accesses are served a half-warp
// at a time; 2(C+1) words apart, the 16 lanes of a half cover 32 distinct
// banks.  (The smaller last chunks of a row, C/2 or C/4 columns per lane,
// see up to 2-way conflicts.)
template <int C>
__device__ __forceinline__ int ring_pos(int j, int mask)
{
    const int r = j & mask;
    return r + r / C;
}

// Columns the chunks of one row cover from the first chunk's start, for a
// span of s columns from there to hi: full chunks of 32*C, then a last chunk
// of 32*C, 16*C or 8*C columns (the ring kernel's choice).  Nondecreasing in s.
template <int C>
__host__ __device__ constexpr int chunk_cover(int s)
{
    return s <= 0 ? 0
         : 32 * C * ((s - 1) / (32 * C)) +
               ((s - 32 * C * ((s - 1) / (32 * C))) > 16 * C ? 32 * C
                : (s - 32 * C * ((s - 1) / (32 * C))) > 8 * C ? 16 * C : 8 * C);
}

// The ring kernels keep one int2 {H(i-1, j-1), E(i, j)} per column, so a
// cell costs one 64-bit load and one 64-bit store of shared memory.
//
// One row chunk of the ring kernel: lane L owns the CC columns
// [cb + CC*L, cb + CC*L + CC) of a ring laid out for C columns per lane (CC
// = C, C/2 or C/4: the lane's columns stay consecutive ring slots).  Columns
// outside the band read empty slots (ring invariant below), so no load is
// masked.  Each lane loads its slots, computes M and the E of the next row
// for every column, and a local F pass; the F entering each lane is a prefix
// max over the warp of floc + (lane+1)*CC*e_ins (F(i,j) = max(0, max_{k<j}
// (M_k - o - e - (j-1-k)e)), Eq. 2 with the affine gap of Eq. 3); then H and
// the stores.  Slot j receives H(i, j-1) (the next row's diagonal) and
// E(i+1, j); the lane stores slot j0 + k once H of column j0 + k - 1 is
// known, and slot j0 last, with H of the previous lane's last column.  F
// entering the chunk is carry_f, H of the column before it carry_h.  LAST:
// the chunk holding column hi - 1; it stores columns up to and including hi
// (slot hi gets H(i, hi-1) with E = 0, the row-end value) and none beyond.
// SYM: o_del = o_ins and e_del = e_ins (E and F open from one M - o - e).
// E1: e_del = e_ins = 1 (the F offsets are immediates).
template <int C, int CC, bool LAST, bool SYM, bool E1>
__device__ __forceinline__ void ring_chunk(const uint8_t *qp, int n, uint32_t tmask, int2 *RG, int mask, int cb,
                                           int hi, int a, int mb, int e_del, int e_ins, int oe_del, int oe_ins,
                                           int lane, int &carry_f, int &carry_h, int &key_l)
{
    const int ed = E1 ? 1 : e_del, ei = E1 ? 1 : e_ins;
    const int j0 = cb + lane * CC;
    uint32_t qbits = 0;
    if (CC >= 4) {
#pragma unroll
        for (int u = 0; u < CC / 4; ++u)
            if (j0 + 4 * u < n) qbits |= (uint32_t)__ldg(qp + (j0 >> 2) + u) << (8 * u);
    } else if (j0 < n) {
        qbits = (uint32_t)__ldg(qp + (j0 >> 2)) >> (2 * (j0 & 3));
    }
    const uint32_t x = qbits ^ tmask;                       // field k is zero where query base j0 + k is t_i
    int2 *rg = RG + ring_pos<C>(j0, mask);
    int M[CC], Ev[CC], Fl[CC];
    int floc = 0;
#pragma unroll
    for (int k = 0; k < CC; ++k) {
        const int2 v = rg[k];                               // H(i-1, j-1), E(i, j)
        const int sc = (x & (3u << (2 * k))) ? mb : a;
        M[k] = __viaddmin_s32(v.x, sc, v.x << 16);          // v.x > 0 ? v.x + sc : <= 0
        Ev[k] = v.y;
        Fl[k] = floc;
        floc = __viaddmax_s32_relu(floc, -ei, M[k] - oe_ins);
    }
    const int ce = CC * ei;
    int v = floc + (lane + 1) * ce;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) v = max(v, __shfl_up_sync(kFull, v, d));
    int vex = __shfl_up_sync(kFull, v, 1);
    if (lane == 0) vex = carry_f;
    const int g = max(carry_f, vex) - lane * ce;            // F entering the lane's first column
    const int vall = __shfl_sync(kFull, v, 31);
    const int kst = LAST ? hi - j0 : CC;                    // columns j0 + k, k <= kst, are stored
    int kk = 0, hp = 0, e20 = 0;
#pragma unroll
    for (int k = 0; k < CC; ++k) {
        const int F = __viaddmax_s32(g, -k * ei, Fl[k]);
        const int h = __vimax3_s32(M[k], Ev[k], F);
        kk = max(kk, h * 32768 + k);                        // row key H*32768 + column: ties to the larger column
        const int e2 = __viaddmax_s32_relu(Ev[k], -ed, M[k] - (SYM ? oe_ins : oe_del));   // E(i+1, j)
        if (k == 0) e20 = e2;
        else if (!LAST || k <= kst) rg[k] = make_int2(hp, e2);
        hp = h;
    }
    int hin = __shfl_up_sync(kFull, hp, 1);
    if (lane == 0) hin = carry_h;
    if (!LAST || kst >= 0) rg[0] = make_int2(hin, e20);
    key_l = max(key_l, kk + j0);
    carry_f = max(carry_f, vall) - 32 * ce;
    if (!LAST) {
        carry_h = __shfl_sync(kFull, hp, 31);
    } else if (hi == cb + 32 * CC && lane == 31) {
        RG[ring_pos<C>(hi, mask)] = make_int2(hp, 0);
    }
}

// The warp-per-pair extension with its row in a shared-memory ring (scores
// up to 32767, for the row key H * 32768 + column), C columns per lane (4, 8
// or 16).  Each row runs chunks of 32*C columns and a last chunk of 32*C,
// 16*C or 8*C columns, whichever is the smallest that holds the rest of the
// band.
//
// Ring invariant: at the start of a row every slot outside [lo, hi) is zero
// (H = E = 0) unless the band will initialise it on first visit.  It holds
// because the band only ever drops all-zero slots at the right (rule c), the
// slots it leaves at the left are zeroed when it leaves them (rule a) or are
// zero already (rule c), the slot at hi is zeroed at the start of the row
// (its value, the previous row-end, is not read in this row), and the ring is
// cleared when the pair starts.  So out-of-band lanes read empty slots: at the
// left they compute H = E = F = 0 and store zeros, and at the right their H is
// an F below some in-band M, strictly below the row best, and they store
// nothing.  The ring is sized by ring_slots, so that no out-of-band lane
// (at most chunk_cover(2w' + C) columns from the first chunk's start) reads a
// slot of a band column through the ring's wrap.
template <int C, bool SYM, bool E1>
__device__ unsigned long long warp_pair_ring16(const Batch &B, const Params &P, int p, int2 *RG, int mask)
{
    static_assert(C == 4 || C == 8 || C == 16, "columns per lane");
    const int lane = threadIdx.x & 31;
    const int n = B.q_len[p], m = B.t_len[p], h0 = B.h0[p];
    const int wb = clip_band(P, n, B.w_override ? B.w_override[p] : P.w);
    const int a = P.a, mb = -P.b;
    const int e_del = P.e_del, e_ins = P.e_ins;
    const int oe_del = P.o_del + e_del, oe_ins = P.o_ins + e_ins;
    const uint8_t *qp = B.q + (B.q_off[p] >> 2);
    const uint8_t *tp = B.t + (B.t_off[p] >> 2);
    const int words = mask + 1 + (mask + 1) / C;
    for (int w = lane; w < words; w += 32) RG[w] = make_int2(0, 0);
    int hw = -1, lo = 0, hi = n;
    int best = h0, bi = -1, bj = -1, gbest = -1, gi = -1, moff = 0;
    unsigned long long ncell = 0;
    for (int i = 0; i < m; ++i) {
        const int tb = (__ldg(tp + (i >> 2)) >> (2 * (i & 3))) & 3;
        const uint32_t tmask = (uint32_t)tb * 0x55555555u;    // t_i in each 2-bit field
        const int lo_new = max(lo, i - wb);
        for (int c = lo + lane; c < lo_new; c += 32)             // left the band
            RG[ring_pos<C>(c, mask)] = make_int2(0, 0);
        lo = lo_new;
        hi = min(min(hi, i + wb + 1), n);
        for (int c = hw + 1 + lane; c <= hi - 1; c += 32)     // first visit of columns (hw, hi-1]
            RG[ring_pos<C>(c, mask)] = make_int2(c == 0 ? h0 : max(0, h0 - P.o_ins - c * e_ins), 0);
        hw = max(hw, hi - 1);
        if (lane == 0) RG[ring_pos<C>(hi, mask)] = make_int2(0, 0);
        __syncwarp();
        const int hl0 = lo == 0 ? max(0, h0 - oe_del - i * e_del) : 0;
        int carry_f = 0, carry_h = hl0, key_l = 0;
        int cb = (lo / C) * C;
        if (lo < hi) {
            while (hi - cb > 32 * C) {
                ring_chunk<C, C, false, SYM, E1>(qp, n, tmask, RG, mask, cb, hi, a, mb, e_del, e_ins, oe_del, oe_ins,
                                                 lane, carry_f, carry_h, key_l);
                cb += 32 * C;
            }
            if (hi - cb > 16 * C)
                ring_chunk<C, C, true, SYM, E1>(qp, n, tmask, RG, mask, cb, hi, a, mb, e_del, e_ins, oe_del, oe_ins,
                                                lane, carry_f, carry_h, key_l);
            else if (hi - cb > 8 * C)
                ring_chunk<C, C / 2, true, SYM, E1>(qp, n, tmask, RG, mask, cb, hi, a, mb, e_del, e_ins, oe_del,
                                                    oe_ins, lane, carry_f, carry_h, key_l);
            else
                ring_chunk<C, C / 4, true, SYM, E1>(qp, n, tmask, RG, mask, cb, hi, a, mb, e_del, e_ins, oe_del,
                                                    oe_ins, lane, carry_f, carry_h, key_l);
        } else if (lane == 0) {
            RG[ring_pos<C>(hi, mask)] = make_int2(hl0, 0);    // empty band: the row-end value is the first column's
        }
        __syncwarp();
        hw = max(hw, hi);                                      // slot hi holds the row-end value now
        const int key = (int)__reduce_max_sync(kFull, (unsigned)key_l);
        const int rm = key >> 15, rj = key & 32767;
        if (hi > lo) ncell += (unsigned)(hi - lo);
        if (max(lo, hi) == n) {                                // H(i, n-1), now in slot hi
            const int hl = RG[ring_pos<C>(hi, mask)].x;
            if (hl >= gbest) gi = i;
            gbest = max(gbest, hl);
        }
        if (rm == 0) break;
        if (rm > best) {
            best = rm; bi = i; bj = rj;
            moff = max(moff, abs(rj - i));
        } else if (P.zdrop > 0) {
            const int di = i - bi, dj = rj - bj;
            const int drop = di > dj ? best - rm - (di - dj) * e_del : best - rm - (dj - di) * e_ins;
            if (drop > P.zdrop) break;
        }
        int nlo = hi;                                          // rule c with ballots
        for (int base = lo; base < hi; base += 32) {
            const int j = base + lane;
            int2 sv = make_int2(0, 0);
            if (j < hi) sv = RG[ring_pos<C>(j, mask)];
            const unsigned bal = __ballot_sync(kFull, (sv.x | sv.y) != 0);
            if (bal) { nlo = base + __ffs(bal) - 1; break; }
        }
        lo = nlo;
        int last = lo - 1;
        for (int top = hi; top >= lo; top -= 32) {
            const int j = top - lane;
            int2 sv = make_int2(0, 0);
            if (j >= lo) sv = RG[ring_pos<C>(j, mask)];
            const unsigned bal = __ballot_sync(kFull, (sv.x | sv.y) != 0);
            if (bal) { last = top - (__ffs(bal) - 1); break; }
        }
        hi = min(last + 2, n);
    }
    if (lane == 0) store_result(&B.out[p], best, bj + 1, bi + 1, gi + 1, gbest, moff);
    return ncell;
}

// The ring kernel's variant for the scoring: symmetric gap costs share
// M - o - e, and unit extensions make the F offsets immediates.
template <int C>
__device__ __forceinline__ unsigned long long ring16_pair(const Batch &B, const Params &P, int p, int2 *RG, int mask)
{
    const bool sym = P.o_del == P.o_ins && P.e_del == P.e_ins;
    if (sym && P.e_del == 1) return warp_pair_ring16<C, true, true>(B, P, p, RG, mask);
    return sym ? warp_pair_ring16<C, true, false>(B, P, p, RG, mask) : warp_pair_ring16<C, false, false>(B, P, p, RG, mask);
}

// ------------------------------------------------------- one pair per block
//
// The longest queries run one pair per block of kCtaWarps warps.  Each row's
// band is cut into chunks of 32*C columns (lane L of a chunk owns C
// consecutive columns, as in the warp kernel) dealt to the warps in rounds:
// chunk r*kCtaWarps + w is warp w's in round r.  The warps of a round
// compute their chunks at the same time.  F crosses chunk boundaries as a
// max-plus map: a chunk turns the F entering it into max(f, B) - 32*C*e_ins
// at its end, where B is its lanes' scan total, so after one block barrier
// each warp folds the maps of the chunks before it.  H of a chunk's last
// column is the next chunk's diagonal input: within a round the chunk's lane
// 31 writes it into the next chunk's first slot (after the barrier, so after
// that chunk has read the slot's old value); across rounds it goes through
// shared memory.  Row decisions are the warp kernel's, taken by every thread
// from values the warps publish in shared memory before a second barrier:
// each warp's row key, the row-end value, and the first and last non-zero
// slot that the warps owning the band's ends find in their own chunks (the
// rare row whose end chunk is all zero scans the rest after the barrier).
// The ring and its invariant are the warp kernel's, sized for full chunks.
constexpr int kCtaWarps = 4;
constexpr int kCtaNone = -0x40000000;

struct CtaCtl {
    int sf[2][kCtaWarps];   // by round parity: each chunk's F map total
    int sh[2];              // by round parity: H of the round's last column
    int skey[kCtaWarps];    // each warp's row key (H * 32768 + column)
    int slo, shi, shl;      // first / last non-zero slot found by the owning warps, H(i, hi-1)
    int pair;               // the block's next pair
};

// Ring slots for band w' with full chunks of 32*C columns: a power of two, at
// least 2w' + 3 and at least the columns of the chunks that cover 2w' + C
// columns from a C-aligned start.
template <int C>
__host__ __device__ inline int cta_ring_slots(int wb)
{
    const int cover = 32 * C * ((2 * wb + C + 32 * C - 1) / (32 * C));
    int need = 64;
    while (need < 2 * wb + 3 || need < cover) need <<= 1;
    return need;
}

template <int C, bool SYM, bool E1>
__device__ unsigned long long cta_pair(const Batch &B, const Params &P, int p, int2 *RG, int mask, CtaCtl &S)
{
    constexpr int NT = kCtaWarps * 32, CW = 32 * C;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n = B.q_len[p], m = B.t_len[p], h0 = B.h0[p];
    const int wb = clip_band(P, n, B.w_override ? B.w_override[p] : P.w);
    const int a = P.a, mb = -P.b;
    const int e_del = E1 ? 1 : P.e_del, e_ins = E1 ? 1 : P.e_ins;
    const int oe_del = P.o_del + e_del, oe_ins = P.o_ins + e_ins;
    const int ce = C * e_ins;
    const uint8_t *qp = B.q + (B.q_off[p] >> 2);
    const uint8_t *tp = B.t + (B.t_off[p] >> 2);
    const int words = mask + 1 + (mask + 1) / C;
    for (int w = tid; w < words; w += NT) RG[w] = make_int2(0, 0);
    __syncthreads();
    int hw = -1, lo = 0, hi = n;
    int best = h0, bi = -1, bj = -1, gbest = -1, gi = -1, moff = 0;
    unsigned long long ncell = 0;
    for (int i = 0; i < m; ++i) {
        const int tb = (__ldg(tp + (i >> 2)) >> (2 * (i & 3))) & 3;
        const uint32_t tmask = (uint32_t)tb * 0x55555555u;
        const int lo_new = max(lo, i - wb);
        const int hi_new = min(min(hi, i + wb + 1), n);
        const int cb0 = (lo_new / C) * C;
        const int nch = lo_new < hi_new ? (hi_new - cb0 + CW - 1) / CW : 0;
        // Ring set-up, each slot by the warp whose chunk reads it: the slots
        // that left the band (left of or in chunk 0: warp 0), first visits of
        // columns (hw, hi_new - 1] and the empty slot at hi_new.
        if (warp == 0)
            for (int c = lo + lane; c < lo_new; c += 32) RG[ring_pos<C>(c, mask)] = make_int2(0, 0);
        for (int c = hw + 1 + lane; c <= hi_new - 1; c += 32)
            if (((c - cb0) / CW) % kCtaWarps == warp)
                RG[ring_pos<C>(c, mask)] = make_int2(c == 0 ? h0 : max(0, h0 - P.o_ins - c * e_ins), 0);
        if (lane == 0 && ((hi_new - cb0) / CW) % kCtaWarps == warp) RG[ring_pos<C>(hi_new, mask)] = make_int2(0, 0);
        hw = max(hw, hi_new - 1);
        __syncwarp();
        const int hl0 = lo_new == 0 ? max(0, h0 - oe_del - i * e_del) : 0;
        int key_l = 0, cf_round = 0;
        for (int r = 0; r * kCtaWarps < nch; ++r) {
            const int c = r * kCtaWarps + warp;
            const bool active = c < nch, last = c == nch - 1;
            const int cb = cb0 + c * CW, j0 = cb + lane * C;
            int M[C], Ev[C], Fl[C];
            int2 *rg = RG + ring_pos<C>(j0, mask);
            int v = 0;
            if (active) {
                uint32_t qbits = 0;
#pragma unroll
                for (int u = 0; u < C / 4; ++u)
                    if (j0 + 4 * u < n) qbits |= (uint32_t)__ldg(qp + (j0 >> 2) + u) << (8 * u);
                const uint32_t x = qbits ^ tmask;
                int floc = 0;
#pragma unroll
                for (int k = 0; k < C; ++k) {
                    const int2 sv = rg[k];
                    const int sc = (x & (3u << (2 * k))) ? mb : a;
                    M[k] = __viaddmin_s32(sv.x, sc, sv.x << 16);
                    Ev[k] = sv.y;
                    Fl[k] = floc;
                    floc = __viaddmax_s32_relu(floc, -e_ins, M[k] - oe_ins);
                }
                v = floc + (lane + 1) * ce;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) v = max(v, __shfl_up_sync(kFull, v, d));
                if (lane == 31) S.sf[r & 1][warp] = v;
            }
            __syncthreads();
            // F entering this chunk (the maps of the round's chunks before
            // it applied to the round's carry), and entering the next round
            const int nact = min(kCtaWarps, nch - r * kCtaWarps);
            int cf = cf_round, cf_mine = 0;
            for (int w2 = 0; w2 < nact; ++w2) {
                if (w2 == warp) cf_mine = cf;
                cf = max(cf, S.sf[r & 1][w2]) - 32 * ce;
            }
            cf_round = cf;
            if (active) {
                int vex = __shfl_up_sync(kFull, v, 1);
                if (lane == 0) vex = cf_mine;
                const int g = max(cf_mine, vex) - lane * ce;
                const int kst = last ? hi_new - j0 : C;
                int kk = 0, hp = 0, e20 = 0;
#pragma unroll
                for (int k = 0; k < C; ++k) {
                    const int F = __viaddmax_s32(g, -k * e_ins, Fl[k]);
                    const int h = __vimax3_s32(M[k], Ev[k], F);
                    kk = max(kk, h * 32768 + k);
                    const int e2 = __viaddmax_s32_relu(Ev[k], -e_del, M[k] - (SYM ? oe_ins : oe_del));
                    if (k == 0) e20 = e2;
                    else if (!last || k <= kst) rg[k] = make_int2(hp, e2);
                    hp = h;
                }
                key_l = max(key_l, kk + j0);
                const int hin = __shfl_up_sync(kFull, hp, 1);
                if (!last || kst >= 0) {
                    if (lane > 0) rg[0] = make_int2(hin, e20);
                    else if (warp == 0) rg[0] = make_int2(r == 0 ? hl0 : S.sh[(r - 1) & 1], e20);
                    else rg[0].y = e20;                 // .x comes from the previous warp's chunk
                }
                if (lane == 31) {
                    if (!last && warp < kCtaWarps - 1) RG[ring_pos<C>(cb + CW, mask)].x = hp;
                    else if (!last) S.sh[r & 1] = hp;
                    else if (hi_new == cb + CW) RG[ring_pos<C>(hi_new, mask)] = make_int2(hp, 0);
                }
            }
        }
        // publish the warp's row key, the row-end value and the band-end scans
        const int kw = (int)__reduce_max_sync(kFull, (unsigned)key_l);
        if (lane == 0) S.skey[warp] = kw;
        __syncwarp();
        if (nch == 0) {
            if (tid == 0) {
                RG[ring_pos<C>(hi_new, mask)] = make_int2(hl0, 0);
                S.shl = hl0;
            }
        } else {
            const int wl = (nch - 1) % kCtaWarps;       // the warp of the chunk holding hi_new - 1
            const int cbl = cb0 + (nch - 1) * CW;
            if (warp == wl && lane == 0) S.shl = RG[ring_pos<C>(hi_new, mask)].x;
            if (warp == 0) {                            // first non-zero slot in chunk 0
                const int end = min(hi_new, cb0 + CW);
                int f = kCtaNone;
                for (int base = lo_new; base < end; base += 32) {
                    const int j = base + lane;
                    int2 sv = make_int2(0, 0);
                    if (j < end) sv = RG[ring_pos<C>(j, mask)];
                    const unsigned bal = __ballot_sync(kFull, (sv.x | sv.y) != 0);
                    if (bal) { f = base + __ffs(bal) - 1; break; }
                }
                if (lane == 0) S.slo = f;
            }
            if (warp == wl) {                           // last non-zero slot in the last chunk
                // its first slot's H comes from another warp unless it starts a round
                const int low = max(lo_new, (nch - 1) % kCtaWarps == 0 ? cbl : cbl + 1);
                int f = kCtaNone;
                for (int top = hi_new; top >= low; top -= 32) {
                    const int j = top - lane;
                    int2 sv = make_int2(0, 0);
                    if (j >= low) sv = RG[ring_pos<C>(j, mask)];
                    const unsigned bal = __ballot_sync(kFull, (sv.x | sv.y) != 0);
                    if (bal) { f = top - (__ffs(bal) - 1); break; }
                }
                if (lane == 0) S.shi = f;
            }
        }
        __syncthreads();
        int key = 0;
#pragma unroll
        for (int w2 = 0; w2 < kCtaWarps; ++w2) key = max(key, S.skey[w2]);
        const int rm = key >> 15, rj = key & 32767;
        const int hl = S.shl;
        lo = lo_new;
        hi = hi_new;
        hw = max(hw, hi);                                  // slot hi holds the row-end value now
        if (hi > lo) ncell += (unsigned)(hi - lo);
        if (max(lo, hi) == n) {
            if (hl >= gbest) gi = i;
            gbest = max(gbest, hl);
        }
        if (rm == 0) break;
        if (rm > best) {
            best = rm; bi = i; bj = rj;
            moff = max(moff, abs(rj - i));
        } else if (P.zdrop > 0) {
            const int di = i - bi, dj = rj - bj;
            const int drop = di > dj ? best - rm - (di - dj) * e_del : best - rm - (dj - di) * e_ins;
            if (drop > P.zdrop) break;
        }
        // rule c: rm > 0, so a chunk was active and both scans ran
        int nlo = S.slo, last = S.shi;
        const bool more = nlo == kCtaNone || last == kCtaNone;
        if (nlo == kCtaNone) {                             // chunk 0 is all zero: scan the rest
            nlo = hi;
            for (int base = min(hi, cb0 + CW); base < hi; base += 32) {
                const int j = base + lane;
                int2 sv = make_int2(0, 0);
                if (j < hi) sv = RG[ring_pos<C>(j, mask)];
                const unsigned bal = __ballot_sync(kFull, (sv.x | sv.y) != 0);
                if (bal) { nlo = base + __ffs(bal) - 1; break; }
            }
        }
        if (last == kCtaNone) {                            // the last chunk is all zero: scan below it
            const int cbl = cb0 + (nch - 1) * CW;
            const int top0 = max(lo, (nch - 1) % kCtaWarps == 0 ? cbl : cbl + 1) - 1;
            last = nlo - 1;
            for (int top = top0; top >= nlo; top -= 32) {
                const int j = top - lane;
                int2 sv = make_int2(0, 0);
                if (j >= nlo) sv = RG[ring_pos<C>(j, mask)];
                const unsigned bal = __ballot_sync(kFull, (sv.x | sv.y) != 0);
                if (bal) { last = top - (__ffs(bal) - 1); break; }
            }
        }
        if (more) __syncthreads();                         // the scans read slots the next row rewrites
        lo = nlo;
        hi = min(last + 2, n);
    }
    if (tid == 0) store_result(&B.out[p], best, bj + 1, bi + 1, gi + 1, gbest, moff);
    return ncell;
}

template <int C>
__device__ __forceinline__ unsigned long long cta_pair_any(const Batch &B, const Params &P, int p, int2 *RG, int mask,
                                                           CtaCtl &S)
{
    const bool sym = P.o_del == P.o_ins && P.e_del == P.e_ins;
    if (sym && P.e_del == 1) return cta_pair<C, true, true>(B, P, p, RG, mask, S);
    return sym ? cta_pair<C, true, false>(B, P, p, RG, mask, S) : cta_pair<C, false, false>(B, P, p, RG, mask, S);
}

// Persistent block-per-pair kernel over a class list.  A pair whose band
// needs a larger ring than the block has (a per-pair band override wider
// than the context's) goes to the 32-bit re-run list, whose warp kernel
// takes any band.
template <int C>
__global__ void __launch_bounds__(kCtaWarps * 32, 5) k_cta(Batch B, Params P, Work W, int cls, int ring_log2)
{
    extern __shared__ int2 cta_ring[];
    __shared__ CtaCtl S;
    const int count = W.cls_count[cls];
    const int32_t *list = W.order + W.cls_start[cls];
    unsigned long long cells = 0;
    for (;;) {
        if (threadIdx.x == 0) S.pair = (int)atomicAdd(&W.cls_next[cls], 1u);
        __syncthreads();
        const int g = S.pair;
        __syncthreads();
        if (g >= count) break;
        const int p = list[g];
        const int n = B.q_len[p];
        const int wb = clip_band(P, n, B.w_override ? B.w_override[p] : P.w);
        const int need = cta_ring_slots<C>(wb);
        if (ring_log2 > 0 && need <= (1 << ring_log2)) {
            const unsigned long long c = cta_pair_any<C>(B, P, p, cta_ring, need - 1, S);
            if (threadIdx.x == 0) cells += c;
        } else if (threadIdx.x == 0) {
            W.rerun[atomicAdd(&W.cls_count[kRerun], 1)] = p;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && cells) atomicAdd(W.cells, cells);
}

// Slots of the ring for band w' and C columns per lane: a power of two, at
// least 2w' + 3 (the band spans at most 2w' + 2 slots with the row end) and
// at least the columns a row's chunks cover for the widest span 2w' + C (so
// out-of-band lanes, which reach that far past lo, never alias a band slot).
template <int C>
__host__ __device__ inline int ring_slots(int wb)
{
    int need = 64;
    while (need < 2 * wb + 3 || need < chunk_cover<C>(2 * wb + C)) need <<= 1;
    return need;
}

// Bytes of one warp's ring of 2^lg slots of 8 bytes; the 16-bit kernel's
// also has one padding slot per C (ring_pos).
template <bool S16, int C>
__host__ __device__ constexpr size_t ring_bytes(int lg)
{
    return S16 ? ((size_t)8 << lg) + ((size_t)8 << lg) / C : (size_t)8 << lg;
}

// Persistent warp-per-pair kernel over a class list (or the re-run list).
// ring_log2 > 0: each warp has a shared-memory slot ring of 1 << ring_log2
// entries (dynamic shared memory); a pair whose band needs a larger ring uses
// the warp's global slot scratch instead.  16 columns per lane need more
// registers than two resident blocks of 8 warps leave: that kernel runs
// blocks of 4 warps, 3 per SM.
template <int C> constexpr int warp_threads() { return C >= 16 ? 128 : kWarpKernelThreads; }

template <int C, bool S16>
__global__ void __launch_bounds__(C >= 16 ? 128 : 256, C >= 16 ? 3 : 2) k_warp(Batch B, Params P, Work W, int cls, int ring_log2)
{
    extern __shared__ uint8_t ring_mem[];
    const int lane = threadIdx.x & 31;
    const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    uint8_t *slots = W.slots + gw * W.slot_bytes_per_warp;
    uint8_t *ring = ring_mem + (size_t)(threadIdx.x >> 5) * ring_bytes<S16, C>(ring_log2);
    const int count = W.cls_count[cls];
    const int32_t *list = cls == kRerun ? W.rerun : W.order + W.cls_start[cls];
    unsigned long long cells = 0;
    for (;;) {
        int g = 0;
        if (lane == 0) g = (int)atomicAdd(&W.cls_next[cls], 1u);
        g = __shfl_sync(kFull, g, 0);
        if (g >= count) break;
        const int p = list[g];
        const int n = B.q_len[p];
        if (ring_log2 > 0) {
            const int wb = clip_band(P, n, B.w_override ? B.w_override[p] : P.w);
            // the 16-bit ring: ring_slots; the 32-bit one at least 2w'+3
            // and 64 >= 8 columns
            int need = S16 ? ring_slots<C>(wb) : 64;
            while (need < 2 * wb + 3) need <<= 1;
            if (need <= (1 << ring_log2)) {
                if (S16) {
                    cells += ring16_pair<C>(B, P, p, reinterpret_cast<int2 *>(ring), need - 1);
                } else if (B.q_n || B.t_n) {
                    cells += warp_pair<C, false, true, true>(B, P, p, ring, need - 1);
                } else {
                    cells += warp_pair<C, false, true, false>(B, P, p, ring, need - 1);
                }
                continue;
            }
        }
        if ((int64_t)(n + 1 + 32 * C) * SlotIO<S16>::kBytes > W.slot_bytes_per_warp) {
            if (lane == 0) atomicOr(W.status, kStTooLong);
            continue;
        }
        if (!S16 && (B.q_n || B.t_n)) cells += warp_pair<C, S16, false, true>(B, P, p, slots, 0);
        else cells += warp_pair<C, S16, false, false>(B, P, p, slots, 0);
    }
    if (lane == 0 && cells) atomicAdd(W.cells, cells);
}

// The plain baseline: the best one-pair-per-warp kernel with no batching
// around it.  Each warp takes pairs in input order (grid stride), with no
// bucketing, no classes and no re-run list, and extends each with the
// warp-per-pair ring kernel of C columns per lane (16-bit slots when the
// score bound allows and the pair has no N; the 32-bit kernel otherwise).  A
// pair whose band needs a larger ring than the warp has uses the warp's
// global slot scratch.  ring16_log2 / ring32_log2: the warp's rings (0: none).
template <int C>
__global__ void __launch_bounds__(C >= 16 ? 128 : 256, C >= 16 ? 3 : 2)
    k_plain(Batch B, Params P, Work W, int ring16_log2, int ring32_log2, int64_t ring_bytes_per_warp)
{
    extern __shared__ uint8_t ring_mem[];
    const int lane = threadIdx.x & 31;
    const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    uint8_t *slots = W.slots + gw * W.slot_bytes_per_warp;
    uint8_t *ring = ring_mem + (size_t)(threadIdx.x >> 5) * ring_bytes_per_warp;
    unsigned long long cells = 0;
    for (int64_t p = gw; p < B.n; p += nw) {
        const long long bound = plain_check(B, P, W, p, lane);
        if (bound < 0) continue;
        const int n = B.q_len[p];
        const int wb = clip_band(P, n, B.w_override ? B.w_override[p] : P.w);
        const bool has_n = (B.q_n || B.t_n) && pair_has_n(B, B.q_off[p], n, B.t_off[p], B.t_len[p]);
        if (bound <= 32767 && !has_n) {
            const int need = ring_slots<C>(wb);
            if (ring16_log2 > 0 && need <= (1 << ring16_log2)) {
                cells += ring16_pair<C>(B, P, (int)p, reinterpret_cast<int2 *>(ring), need - 1);
                continue;
            }
        } else {
            int need = 64;
            while (need < 2 * wb + 3) need <<= 1;
            if (ring32_log2 > 0 && need <= (1 << ring32_log2)) {
                cells += has_n ? warp_pair<8, false, true, true>(B, P, (int)p, ring, need - 1)
                               : warp_pair<8, false, true, false>(B, P, (int)p, ring, need - 1);
                continue;
            }
        }
        if ((int64_t)(n + 1 + 32 * 8) * 8 > W.slot_bytes_per_warp) {
            if (lane == 0) atomicOr(W.status, kStTooLong);
            continue;
        }
        cells += has_n ? warp_pair<8, false, false, true>(B, P, (int)p, slots, 0)
                       : warp_pair<8, false, false, false>(B, P, (int)p, slots, 0);
    }
    if (lane == 0 && cells) atomicAdd(W.cells, cells);
}

// The naive baseline (BSW_PLAIN_GLOBAL): one pair per warp in input order,
// one column per lane, the row's slots in global memory; 16-bit slots when
// the score bound allows.
__global__ void __launch_bounds__(256) k_plain_global(Batch B, Params P, Work W)
{
    const int lane = threadIdx.x & 31;
    const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    uint8_t *slots = W.slots + gw * W.slot_bytes_per_warp;
    unsigned long long cells = 0;
    for (int64_t p = gw; p < B.n; p += nw) {
        const int n = B.q_len[p], m = B.t_len[p], h0 = B.h0[p];
        const int64_t qo = B.q_off[p], to = B.t_off[p];
        const int w = B.w_override ? B.w_override[p] : P.w;
        if (n < 0 || m < 0 || h0 < 0 || w < 0 || qo < 0 || to < 0 || (qo & 3) || (to & 3)) {
            if (lane == 0) atomicOr(W.status, kStInval);
            continue;
        }
        if (n == 0 || m == 0) {
            if (lane == 0) store_result(&B.out[p], h0, 0, 0, 0, n == 0 ? h0 : -1, 0);
            continue;
        }
        const long long bound = (long long)h0 + (long long)P.a * min(n, m);
        if (bound >= (1ll << 30)) {
            if (lane == 0) atomicOr(W.status, kStInval);
            continue;
        }
        const bool s16 = bound <= 32767;
        if ((int64_t)(n + 1 + 32) * (s16 ? 4 : 8) > W.slot_bytes_per_warp) {
            if (lane == 0) atomicOr(W.status, kStTooLong);
            continue;
        }
        if (B.q_n || B.t_n)
            cells += s16 ? warp_pair<1, true, false, true>(B, P, (int)p, slots, 0)
                         : warp_pair<1, false, false, true>(B, P, (int)p, slots, 0);
        else
            cells += s16 ? warp_pair<1, true, false>(B, P, (int)p, slots, 0) : warp_pair<1, false, false>(B, P, (int)p, slots, 0);
    }
    if (lane == 0 && cells) atomicAdd(W.cells, cells);
}


// ------------------------------------------------------------------ launcher

bool make_plan(int short_max, uint32_t u8_mask, uint32_t i16_mask, bool packed, int warp_cols, int inter_warps,
               int cta_min, bool warp_x2, Plan *out)
{
    if (short_max < 64 || short_max > kShortMax) return false;
    if (cta_min != 0 && (cta_min < 128 || cta_min > kLongMax || (cta_min & 63))) return false;
    if (warp_cols != 4 && warp_cols != 8 && warp_cols != 16) return false;
    if (inter_warps != 1 && inter_warps != 2 && inter_warps != 4) return false;
    if ((u8_mask & ~0xffu) || (i16_mask & ~0xfu)) return false;
    Plan L;
    L.short_max = short_max;
    L.packed = packed;
    L.warp_cols = warp_cols;
    L.inter_warps = inter_warps;
    L.cta_min = cta_min;
    L.warp_x2 = warp_x2;
    int32_t *b = L.cls.b;
    // A disabled class gets an empty range; its queries fall to the next
    // larger enabled class.
    b[0] = kBinU8;
    b[8] = kBinI16;
    for (int c = 7; c >= 1; --c)
        b[c] = ((u8_mask >> c) & 1u) ? kBinU8 + (kShortMax - kU8Nmax[c]) * kU8H0Buckets : b[c + 1];
    // the 16-bit warp bins run from long to short queries (bin kBinW16 + 639
    // - n / 64): the block-per-pair class takes those of n >= cta_min
    b[kClsCTA] = kBinW16;
    b[kClsW16] = kBinW16 + (cta_min ? 640 - (cta_min >> 6) : 0);
    for (int c = 11; c >= 9; --c) b[c] = ((i16_mask >> (c - 8)) & 1u) ? kBinI16 + kShortMax - kI16Nmax[c - 8] : b[c + 1];
    b[kClsW32] = kBinW32;
    b[kNumClass] = kNumBins;
    *out = L;
    return true;
}

Plan default_plan()
{
    Plan L;
    make_plan(kShortMax, 0xffu, 0xfu, false, 8, 2, 0, false, &L);
    return L;
}

namespace {

// Resident blocks per SM of each k_inter instantiation with 1, 2 and 4 warps
// per block, set by prepare_kernels.
int g_inter_blocks[12][3];
int g_inter_blocks_n[8][3];     // the N-aware 8-bit instantiations

int warps_index(int warps) { return warps <= 1 ? 0 : warps == 2 ? 1 : 2; }

template <int NMAX, bool U8> size_t inter_smem(int warps) { return (size_t)warps * (NMAX + 1) * 32 * 4; }
template <int NMAX, bool U8> constexpr int inter_index()
{
    return U8 ? (NMAX >= 256 ? 0 : NMAX >= 224 ? 1 : NMAX >= 192 ? 2 : NMAX >= 160 ? 3 : NMAX >= 128 ? 4 : NMAX >= 96 ? 5
                 : NMAX >= 64 ? 6 : 7)
              : 8 + (NMAX >= 256 ? 0 : NMAX >= 128 ? 1 : NMAX >= 64 ? 2 : 3);
}

template <int NMAX, bool U8, bool NM>
cudaError_t prepare_inter_one(int *blocks)
{
    cudaError_t e = cudaFuncSetAttribute(k_inter<NMAX, U8, NM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)inter_smem<NMAX, U8>(4));
    if (e != cudaSuccess) return e;
    for (int wi = 0; wi < 3; ++wi) {
        const int warps = 1 << wi;
        int nb = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_inter<NMAX, U8, NM>, warps * 32,
                                                          inter_smem<NMAX, U8>(warps));
        if (e != cudaSuccess) return e;
        blocks[wi] = nb > 0 ? nb : 1;
    }
    return cudaSuccess;
}

template <int NMAX, bool U8>
cudaError_t prepare_inter()
{
    cudaError_t e = prepare_inter_one<NMAX, U8, false>(g_inter_blocks[inter_index<NMAX, U8>()]);
    if (e != cudaSuccess || !U8) return e;
    return prepare_inter_one<NMAX, true, true>(g_inter_blocks_n[inter_index<NMAX, U8>()]);
}

template <int NMAX, bool U8>
cudaError_t launch_inter(const Batch &B, const Params &P, const Work &W, int cls, cudaStream_t st, int sms, int warps)
{
    if (U8 && (B.q_n || B.t_n)) {
        const int blocks = sms * g_inter_blocks_n[inter_index<NMAX, U8>()][warps_index(warps)];
        k_inter<NMAX, true, true><<<blocks, warps * 32, inter_smem<NMAX, U8>(warps), st>>>(B, P, W, cls);
    } else {
        const int blocks = sms * g_inter_blocks[inter_index<NMAX, U8>()][warps_index(warps)];
        k_inter<NMAX, U8, false><<<blocks, warps * 32, inter_smem<NMAX, U8>(warps), st>>>(B, P, W, cls);
    }
    return cudaGetLastError();
}

int g_inter2_blocks[3] = {1, 1, 1};

template <int NMAX> constexpr int inter2_warps() { return NMAX >= 128 ? 2 : NMAX >= 64 ? 4 : 8; }
template <int NMAX> constexpr size_t inter2_smem() { return (size_t)inter2_warps<NMAX>() * (NMAX + 1) * 64 * 4; }
template <int NMAX> constexpr int inter2_index() { return NMAX >= 128 ? 0 : NMAX >= 64 ? 1 : 2; }

template <int NMAX>
cudaError_t prepare_inter2()
{
    cudaError_t e = cudaFuncSetAttribute(k_inter2<NMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)inter2_smem<NMAX>());
    if (e != cudaSuccess) return e;
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_inter2<NMAX>, inter2_warps<NMAX>() * 32,
                                                      inter2_smem<NMAX>());
    if (e != cudaSuccess) return e;
    g_inter2_blocks[inter2_index<NMAX>()] = nb > 0 ? nb : 1;
    return cudaSuccess;
}

// The packed kernel holds every intermediate in a signed 16-bit lane only when
// the mismatch and gap-open costs (clamped where larger ones act the same) fit.
bool inter2_scoring_ok(const Params &P)
{
    const int bm = P.b < 255 - P.a ? P.b : 255 - P.a;
    const int od = P.o_del + P.e_del < 255 ? P.o_del + P.e_del : 255;
    const int oi = P.o_ins + P.e_ins < 255 ? P.o_ins + P.e_ins : 255;
    return P.a + bm + od <= 256 && P.a + bm + oi <= 256;
}

// 8-bit class with queries up to NMAX: one pair per thread, or two pairs per
// thread in packed 16-bit lanes when the plan (or the batch flag) asks for it
// and the scoring allows.
template <int NMAX>
cudaError_t launch_u8(const Batch &B, const Params &P, const Work &W, int cls, cudaStream_t st, int sms, const Plan &L)
{
    constexpr int N2 = NMAX > 64 ? 128 : NMAX > 32 ? 64 : 32;   // the packed kernel's sizes
    if (NMAX <= 128 && (L.packed || (P.flags & BSW_PACKED_PAIRS)) && inter2_scoring_ok(P) && !B.q_n && !B.t_n) {
        const int blocks = sms * g_inter2_blocks[inter2_index<N2>()];
        k_inter2<N2><<<blocks, inter2_warps<N2>() * 32, inter2_smem<N2>(), st>>>(B, P, W, cls);
        return cudaGetLastError();
    }
    return launch_inter<NMAX, true>(B, P, W, cls, st, sms, L.inter_warps);
}

// Ring size for the context's band: the smallest power of two >= 2*w + 3,
// capped so that a block's rings fit in shared memory (0: no ring).
template <bool S16, int C>
int ring_log2_for(const Params &P)
{
    int lg = 6;
    const int need = S16 ? ring_slots<C>(P.w) : 2 * P.w + 3;
    while ((1 << lg) < need && lg < 16) ++lg;
    const size_t per_block = (size_t)(warp_threads<C>() / 32) * ring_bytes<S16, C>(lg);
    return per_block <= kRingSmemMax ? lg : 0;
}

// Ring of the block-per-pair kernel for the context's band (0: none fits).
constexpr int kCtaCols = 8;
int g_cta_blocks = 1;   // resident blocks per SM, set by prepare_kernels

int cta_ring_log2(const Params &P)
{
    int lg = 6;
    const int need = cta_ring_slots<kCtaCols>(P.w);
    while ((1 << lg) < need && lg < 16) ++lg;
    return ring_bytes<true, kCtaCols>(lg) <= kRingSmemMax ? lg : 0;
}

cudaError_t launch_cta(const Batch &B, const Params &P, const Work &W, int cls, cudaStream_t st, int sms)
{
    const int lg = cta_ring_log2(P);
    const size_t smem = lg ? ring_bytes<true, kCtaCols>(lg) : 0;
    k_cta<kCtaCols><<<sms * g_cta_blocks, kCtaWarps * 32, smem, st>>>(B, P, W, cls, lg);
    return cudaGetLastError();
}

template <int C, bool S16>
cudaError_t launch_warp(const Batch &B, const Params &P, const Work &W, int cls, cudaStream_t st, int blocks)
{
    const int lg = ring_log2_for<S16, C>(P);
    // blocks counts blocks of kWarpKernelThreads; the same number of warps in
    // blocks of warp_threads<C>()
    constexpr int tpb = warp_threads<C>();
    const size_t smem = lg ? (size_t)(tpb / 32) * ring_bytes<S16, C>(lg) : 0;
    k_warp<C, S16><<<blocks * (kWarpKernelThreads / tpb), tpb, smem, st>>>(B, P, W, cls, lg);
    return cudaGetLastError();
}

// One class kernel: the per-thread kernels take the SM count, the warp
// kernels a block count.
using ClassLaunch = cudaError_t (*)(const Batch &, const Params &, const Work &, int, cudaStream_t, int, int,
                                   const Plan &);

template <int NMAX>
cudaError_t cls_u8(const Batch &B, const Params &P, const Work &W, int c, cudaStream_t st, int sms, int, const Plan &L)
{
    return launch_u8<NMAX>(B, P, W, c, st, sms, L);
}

template <int NMAX>
cudaError_t cls_i16(const Batch &B, const Params &P, const Work &W, int c, cudaStream_t st, int sms, int, const Plan &L)
{
    return launch_inter<NMAX, false>(B, P, W, c, st, sms, L.inter_warps);
}

cudaError_t cls_w16(const Batch &B, const Params &P, const Work &W, int c, cudaStream_t st, int sms, int wblocks,
                    const Plan &L)
{
    if (L.warp_x2 && x2_usable(P) && x2_ring_log2(P) > 0) return launch_x2(B, P, W, c, st, sms);
    if (L.warp_cols == 4) return launch_warp<4, true>(B, P, W, c, st, wblocks);
    if (L.warp_cols == 16) return launch_warp<16, true>(B, P, W, c, st, wblocks);
    return launch_warp<8, true>(B, P, W, c, st, wblocks);
}

cudaError_t cls_w32(const Batch &B, const Params &P, const Work &W, int c, cudaStream_t st, int, int wblocks,
                    const Plan &)
{
    return launch_warp<8, false>(B, P, W, c, st, wblocks);
}

cudaError_t cls_cta(const Batch &B, const Params &P, const Work &W, int c, cudaStream_t st, int sms, int,
                    const Plan &)
{
    return launch_cta(B, P, W, c, st, sms);
}

constexpr ClassLaunch kClassLaunch[kNumClass + 1] = {
    cls_u8<256>, cls_u8<224>, cls_u8<192>, cls_u8<160>, cls_u8<128>, cls_u8<96>, cls_u8<64>, cls_u8<32>,
    cls_i16<256>, cls_i16<128>, cls_i16<64>, cls_i16<32>, cls_cta, cls_w16, cls_w32, cls_w32};

// Launch order of the classes in the forked path and the side stream of each:
// the longest work first (block-per-pair pairs, then the long 8-bit
// classes), each stream ending with shorter work.
constexpr int kForkOrder[kNumClass] = {kClsCTA, 0, 1, 2, 3, 4, 5, 6, 7, kClsW16, kClsW32, 8, 9, 10, 11};
constexpr int kClassStream[kNumClass] = {0, 0, 0, 1, 1, 1, 2, 2, 2, 2, 2, 2, 0, 2, 2};

// Whether class c can hold pairs under the plan and the batch flags (classes
// that cannot are not launched).
bool class_live(int c, const Plan &L, uint32_t flags)
{
    if (c == kClsCTA) return L.cls.b[kClsCTA] != L.cls.b[kClsW16];
    if (c >= kClsW16) return true;
    if (flags & BSW_FORCE_I32) return false;
    const bool u8 = c < 8;
    if ((flags & BSW_FORCE_I8) && !u8) return false;
    if ((flags & BSW_FORCE_I16) && u8) return false;
    if (L.cls.b[c] == L.cls.b[c + 1]) return false;
    if (flags & (BSW_FORCE_I8 | BSW_FORCE_I16)) return true;
    const int nmin = u8 ? kShortMax - (L.cls.b[c + 1] - kBinU8) / kU8H0Buckets + 1   // the class's shortest query
                        : kShortMax - (L.cls.b[c + 1] - kBinI16) + 1;
    return nmin <= L.short_max;
}

cudaError_t launch_class(int c, const Batch &B, const Params &P, const Work &W, cudaStream_t st, int sms, int wblocks,
                         const Plan &L, ClassTimer *T)
{
    cudaError_t e;
    if (T && (e = cudaEventRecord(T->t0[c], st)) != cudaSuccess) return e;
    if ((e = kClassLaunch[c](B, P, W, c, st, sms, wblocks, L)) != cudaSuccess) return e;
    if (T) {
        if ((e = cudaEventRecord(T->t1[c], st)) != cudaSuccess) return e;
        T->used[c] = true;
    }
    return cudaSuccess;
}

cudaError_t launch_prepass(const Batch &B, const Params &P, const Work &W, cudaStream_t st, int sms, const Plan &L)
{
    const int cblocks = (int)((B.n + 511) / 512 < (int64_t)sms * 4 ? (B.n + 511) / 512 : (int64_t)sms * 4);
    k_classify<<<cblocks, 512, 0, st>>>(B, P, W);
    k_scan<<<1, 1024, 0, st>>>(W, L.cls);
    const int sblocks = (int)((B.n + kScatterTile - 1) / kScatterTile < (int64_t)sms * 2
                                  ? (B.n + kScatterTile - 1) / kScatterTile : (int64_t)sms * 2);
    k_scatter<<<sblocks, kScatterThreads, 0, st>>>(B, P, W);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_extents(const PairMeta &M, int64_t n, const Params &P, Extents32 *X, cudaStream_t st, int sms)
{
    const int64_t b = (n + 255) / 256;
    const int blocks = (int)(b < (int64_t)sms * 4 ? (b > 0 ? b : 1) : (int64_t)sms * 4);
    k_extents<<<blocks, 256, 0, st>>>(M, n, P, X);
    return cudaGetLastError();
}

bool packed_scoring_ok(const Params &P) { return inter2_scoring_ok(P); }

int batched_launches(const Plan &L, uint32_t flags)
{
    int k = 3;   // classify, scan, scatter
    for (int c = 0; c <= kNumClass; ++c) k += class_live(c, L, flags) ? 1 : 0;
    return k;
}

cudaError_t prepare_kernels(int sms)
{
    (void)sms;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_warp<4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRingSmemMax)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_warp<8, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRingSmemMax)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_warp<16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRingSmemMax)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_warp<8, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRingSmemMax)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_plain<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRingSmemMax)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_cta<kCtaCols>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRingSmemMax)) !=
        cudaSuccess)
        return e;
    {
        // resident blocks for the ring of a w = 500 band (the long-query workload's)
        const int nb_smem = (int)ring_bytes<true, kCtaCols>(11);
        int nb = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_cta<kCtaCols>, kCtaWarps * 32, nb_smem)) !=
            cudaSuccess)
            return e;
        g_cta_blocks = nb > 0 ? nb : 1;
    }
    if ((e = cudaFuncSetAttribute(k_plain<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRingSmemMax)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_plain<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRingSmemMax)) != cudaSuccess)
        return e;
    if ((e = prepare_x2(sms)) != cudaSuccess) return e;
    if ((e = prepare_inter<256, true>()) != cudaSuccess) return e;
    if ((e = prepare_inter<192, true>()) != cudaSuccess) return e;
    if ((e = prepare_inter<128, true>()) != cudaSuccess) return e;
    if ((e = prepare_inter<96, true>()) != cudaSuccess) return e;
    if ((e = prepare_inter<64, true>()) != cudaSuccess) return e;
    if ((e = prepare_inter<224, true>()) != cudaSuccess) return e;
    if ((e = prepare_inter<32, true>()) != cudaSuccess) return e;
    if ((e = prepare_inter<160, true>()) != cudaSuccess) return e;
    if ((e = prepare_inter<256, false>()) != cudaSuccess) return e;
    if ((e = prepare_inter<128, false>()) != cudaSuccess) return e;
    if ((e = prepare_inter<64, false>()) != cudaSuccess) return e;
    if ((e = prepare_inter<32, false>()) != cudaSuccess) return e;
    if ((e = prepare_inter2<128>()) != cudaSuccess) return e;
    if ((e = prepare_inter2<64>()) != cudaSuccess) return e;
    return prepare_inter2<32>();
}

int warp_slots_needed(int sms) { return sms * kWarpBlocksPerSM * (kWarpKernelThreads / 32); }

cudaError_t launch_batched(const Batch &B, const Params &P0, const Work &W, const Streams &S, int sms, const Plan &L,
                           ClassTimer *T)
{
    cudaError_t e;
    if (B.n <= 0) return cudaSuccess;
    Params P = P0;
    P.short_max = L.short_max;
    if ((e = launch_prepass(B, P, W, S.main, sms, L)) != cudaSuccess) return e;
    // Fork: classes run concurrently on the side streams so that one class's
    // tail overlaps the next class's start.
    if ((e = cudaEventRecord(S.fork, S.main)) != cudaSuccess) return e;
    for (int k = 0; k < 3; ++k)
        if ((e = cudaStreamWaitEvent(S.side[k], S.fork, 0)) != cudaSuccess) return e;
    const int wblocks = sms * kWarpBlocksPerSM;
    // The two-columns warp kernel runs after the other classes: it leaves a
    // quarter of each SM's block slots free (3 blocks of its 4, so the
    // longest pairs get a twelfth of an SM, not a sixteenth), and kernels of
    // other classes in them would take issue slots from those pairs.
    const bool x2_after = L.warp_x2 && x2_usable(P) && x2_ring_log2(P) > 0;
    for (int c : kForkOrder)
        if (class_live(c, L, P.flags) && !(x2_after && c == kClsW16) &&
            (e = launch_class(c, B, P, W, S.side[kClassStream[c]], sms, wblocks, L, T)) != cudaSuccess)
            return e;
    for (int k = 0; k < 3; ++k) {
        if ((e = cudaEventRecord(S.join[k], S.side[k])) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(S.main, S.join[k], 0)) != cudaSuccess) return e;
    }
    if (x2_after && (e = launch_class(kClsW16, B, P, W, S.main, sms, wblocks, L, T)) != cudaSuccess) return e;
    // Section V-D1: pairs whose scores left their lane range, exactly, in 32 bits.
    return launch_class(kRerun, B, P, W, S.main, sms, wblocks, L, T);
}

cudaError_t launch_batched_serial(const Batch &B, const Params &P0, const Work &W, cudaStream_t st, int sms,
                                  int warp_blocks, const Plan &L)
{
    cudaError_t e;
    if (B.n <= 0) return cudaSuccess;
    Params P = P0;
    P.short_max = L.short_max;
    if ((e = launch_prepass(B, P, W, st, sms, L)) != cudaSuccess) return e;
    for (int c = 0; c <= kNumClass; ++c)
        if (class_live(c, L, P.flags) && (e = launch_class(c, B, P, W, st, sms, warp_blocks, L, nullptr)) != cudaSuccess)
            return e;
    return cudaSuccess;
}

namespace {

template <int C>
cudaError_t launch_plain_c(const Batch &B, const Params &P, const Work &W, cudaStream_t st, int sms)
{
    // rings for the context's band: 16-bit for C columns per lane, 32-bit as
    // the warp kernel's 32-bit class has them; a warp's share of shared
    // memory holds the larger
    const int lg16 = ring_log2_for<true, C>(P), lg32 = ring_log2_for<false, 8>(P);
    const size_t r16 = lg16 ? ring_bytes<true, C>(lg16) : 0, r32 = lg32 ? ring_bytes<false, 8>(lg32) : 0;
    const size_t per_warp = r16 > r32 ? r16 : r32;
    constexpr int tpb = warp_threads<C>();
    constexpr int bps = C >= 16 ? 3 : 2;   // blocks per SM of the launch bounds
    const size_t smem = per_warp * (tpb / 32);
    if (smem > kRingSmemMax) return cudaErrorInvalidValue;
    // at most as many warps as the work buffers have slot regions
    k_plain<C><<<sms * bps, tpb, smem, st>>>(B, P, W, lg16, lg32, (int64_t)per_warp);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_plain(const Batch &B, const Params &P, const Work &W, cudaStream_t st, int sms, const Plan &L)
{
    if (B.n <= 0) return cudaSuccess;
    if (P.flags & BSW_PLAIN_GLOBAL) {
        k_plain_global<<<sms * kWarpBlocksPerSM, kWarpKernelThreads, 0, st>>>(B, P, W);
        return cudaGetLastError();
    }
    if (L.warp_x2 && x2_usable(P) && x2_ring_log2(P) > 0) {
        cudaError_t e;
        if ((e = launch_plain_x2(B, P, W, st, sms)) != cudaSuccess) return e;
        return launch_warp<8, false>(B, P, W, kRerun, st, sms * kWarpBlocksPerSM);
    }
    if (L.warp_cols == 4) return launch_plain_c<4>(B, P, W, st, sms);
    if (L.warp_cols == 16) return launch_plain_c<16>(B, P, W, st, sms);
    return launch_plain_c<8>(B, P, W, st, sms);
}

int plain_launches(const Params &P, const Plan &L, uint32_t flags)
{
    if (flags & BSW_PLAIN_GLOBAL) return 1;
    return (L.warp_x2 && x2_usable(P) && x2_ring_log2(P) > 0) ? 2 : 1;
}

}  // namespace bsw
