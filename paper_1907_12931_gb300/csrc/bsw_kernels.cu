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
//   k_plain                      the baseline: one pair per warp, input order
#include <cuda_runtime.h>
#include <cstdint>

#include "bsw_device.cuh"
#include "bsw_launch.h"

namespace bsw {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kNeg = -(1 << 29);

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

// ------------------------------------------------------------------ bucketing

__device__ __forceinline__ int pick_bin(int n, long long bound, uint32_t flags)
{
    const int rank = 639 - min(n >> 6, 639);
    if (flags & BSW_FORCE_I32) return kBinW32 + rank;
    if (n <= kShortMax) {
        if (flags & BSW_FORCE_I8) return kBinU8 + (kShortMax - n);
        if (flags & BSW_FORCE_I16) return kBinI16 + (kShortMax - n);
        if (bound <= 255) return kBinU8 + (kShortMax - n);
        if (bound <= 32767) return kBinI16 + (kShortMax - n);
        return kBinW32 + rank;
    }
    return bound <= 32767 ? kBinW16 + rank : kBinW32 + rank;
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
            else key = pick_bin(n, bound, P.flags);
        }
        W.key[p] = key;
        if (key >= 0) atomicAdd(&sh[key], 1u);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kNumBins; k += blockDim.x)
        if (sh[k]) atomicAdd(&W.hist[k], sh[k]);
}

// Class c covers bins [kClassBins[c], kClassBins[c+1]).
__constant__ int kClassBins[kNumClass + 1] = {0, 128, 192, 224, 256, 384, 448, 480, 512, 1152, 1792};

// One block of 1024 threads: exclusive scan of the histogram into the scatter
// cursors, class ranges, and a reset of the histogram and work counters.
__global__ void __launch_bounds__(1024) k_scan(Work W)
{
    __shared__ uint32_t pre[kNumBins + 1];
    __shared__ uint32_t wsum[32];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const uint32_t a = (2 * t < kNumBins) ? W.hist[2 * t] : 0u;
    const uint32_t b = (2 * t + 1 < kNumBins) ? W.hist[2 * t + 1] : 0u;
    const uint32_t s = a + b;
    uint32_t x = s;
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t y = __shfl_up_sync(kFull, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t v = wsum[lane];
        for (int d = 1; d < 32; d <<= 1) {
            uint32_t y = __shfl_up_sync(kFull, v, d);
            if (lane >= d) v += y;
        }
        wsum[lane] = v;
    }
    __syncthreads();
    const uint32_t excl = x - s + (wid ? wsum[wid - 1] : 0u);
    if (2 * t < kNumBins) { pre[2 * t] = excl; W.cursor[2 * t] = excl; W.hist[2 * t] = 0; }
    if (2 * t + 1 < kNumBins) { pre[2 * t + 1] = excl + a; W.cursor[2 * t + 1] = excl + a; W.hist[2 * t + 1] = 0; }
    if (t == 0) pre[kNumBins] = wsum[31];
    __syncthreads();
    if (t < kNumClass) {
        W.cls_start[t] = (int32_t)pre[kClassBins[t]];
        W.cls_count[t] = (int32_t)(pre[kClassBins[t + 1]] - pre[kClassBins[t]]);
    }
    if (t == kRerun) { W.cls_start[t] = 0; W.cls_count[t] = 0; }
    if (t <= kNumClass) W.cls_next[t] = 0;
}

// Place every pair in its bin.  Each block takes tiles of kScatterTile pairs:
// ranks within the tile come from shared-memory atomics, and one global atomic
// per non-empty bin reserves the tile's range in that bin.
constexpr int kScatterThreads = 512, kScatterPer = 8, kScatterTile = kScatterThreads * kScatterPer;

__global__ void __launch_bounds__(kScatterThreads) k_scatter(int64_t n, Work W)
{
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
        for (int u = 0; u < kScatterPer; ++u)
            if (key[u] >= 0) W.order[base[key[u]] + rank[u]] = (int32_t)(tile + u * kScatterThreads + threadIdx.x);
        __syncthreads();
    }
}

// ------------------------------------------------------- one pair per thread

// Slot word layouts (32 bits per column, column j of lane L at S[j*32 + L]):
//   8-bit lanes : bits 0-15 a byte-permute selector for the query base q
//                 (q*0x1111 | 0x8880 picks byte q of the row's score profile
//                 and sign-extends it), bits 16-23 H, bits 24-31 E.
//   16-bit lanes: bits 0-14 H, bits 15-29 E, bits 30-31 q.
template <bool U8>
__device__ __forceinline__ uint32_t slot_init(int q, int h)
{
    return U8 ? ((uint32_t)q * 0x1111u | 0x8880u | ((uint32_t)h << 16)) : ((uint32_t)h | ((uint32_t)q << 30));
}

template <bool U8>
__device__ __forceinline__ bool slot_nonzero(uint32_t w)
{
    return U8 ? (w >> 16) != 0u : (w & 0x3fffffffu) != 0u;
}

// Extend pair p; the calling thread owns the slot column S[0], S[32], ...
// Returns the cells computed, or 0 after queueing the pair for the 32-bit
// re-run when a score leaves the lane range.
template <int NMAX, bool U8>
__device__ __forceinline__ unsigned long long inter_pair(const Batch &B, const Params &P, const Work &W,
                                                         int p, uint32_t *S)
{
    constexpr int VMAX = U8 ? 255 : 32767;
    const int n = B.q_len[p], m = B.t_len[p], h0 = B.h0[p];
    const int wb = clip_band(P, n, B.w_override ? B.w_override[p] : P.w);
    const int e_del = P.e_del, e_ins = P.e_ins;
    const int oe_del = P.o_del + e_del, oe_ins = P.o_ins + e_ins;
    if (h0 > VMAX || n > NMAX) {
        W.rerun[atomicAdd(&W.cls_count[kRerun], 1)] = p;
        return 0;
    }

    // Eq. 3, first row: H = h0 at column 0, max(0, h0 - o_ins - c*e_ins) after.
    const uint8_t *qp = B.q + (B.q_off[p] >> 2);
    for (int c = 0; c <= n; c += 4) {
        const uint32_t byte = c < n ? __ldg(qp + (c >> 2)) : 0u;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int j = c + k;
            if (j <= n) {
                const int hv = j == 0 ? h0 : max(0, h0 - P.o_ins - j * e_ins);
                S[j * 32] = slot_init<U8>((byte >> (2 * k)) & 3, hv);
            }
        }
    }

    const uint8_t *tp = B.t + (B.t_off[p] >> 2);
    const uint32_t mb8 = (uint32_t)(-P.b) & 0xffu;
    const uint32_t mis4 = mb8 * 0x01010101u;
    const uint32_t flip = ((uint32_t)P.a ^ mb8) & 0xffu;
    int lo = 0, hi = n;
    int best = h0, bi = -1, bj = -1, gbest = -1, gi = -1, moff = 0;
    unsigned long long ncell = 0;
    uint32_t tbyte = 0;
    for (int i = 0; i < m; ++i) {
        if ((i & 3) == 0) tbyte = __ldg(tp + (i >> 2));
        const int tb = (tbyte >> (2 * (i & 3))) & 3;
        lo = max(lo, i - wb);
        hi = min(min(hi, i + wb + 1), n);
        // Eq. 3, first column, while the band still touches it.
        int hl = lo == 0 ? max(0, h0 - oe_del - i * e_del) : 0;
        int f = 0, key = 0;   // key = H*512 + j: its max is the row max, ties to larger j
        if (U8) {
            const uint32_t prof = mis4 ^ (flip << (8 * tb));   // byte c: score of (t_i, c)
#pragma unroll 4
            for (int j = lo; j < hi; ++j) {
                const uint32_t wv = S[j * 32];
                const int sc = (int)prmt(prof, 0u, wv);
                const int d = (int)prmt(wv, 0u, 0x4442u);         // H(i-1, j-1)
                const int d8 = (int)prmt(wv, 0u, 0x4424u);        // d << 8
                const int M = __viaddmin_s32(d, sc, d8);          // d > 0 ? d + sc : <= 0
                const int e = (int)(wv >> 24);                    // E(i, j)
                const int h = __vimax3_s32(M, e, f);              // Eq. 2
                key = max(key, h * 512 + j);
                const int e2 = __viaddmax_s32_relu(e, -e_del, M - oe_del);   // E(i+1, j)
                f = __viaddmax_s32_relu(f, -e_ins, M - oe_ins);              // F(i, j+1)
                S[j * 32] = prmt(wv, prmt((uint32_t)hl, (uint32_t)e2, 0x0040u), 0x5410u);
                hl = h;
            }
            const uint32_t wh = S[hi * 32];
            S[hi * 32] = (wh & 0xffffu) | ((uint32_t)(hl & 0xff) << 16);
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
        const int rm = key >> 9, rj = key & 511;
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

template <int NMAX, bool U8>
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
        if (idx < count) cells += inter_pair<NMAX, U8>(B, P, W, W.order[start + idx], S);
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
template <int C, bool S16>
__device__ unsigned long long warp_pair(const Batch &B, const Params &P, int p, uint8_t *slots)
{
    using IO = SlotIO<S16>;
    const int lane = threadIdx.x & 31;
    const int n = B.q_len[p], m = B.t_len[p], h0 = B.h0[p];
    const int wb = clip_band(P, n, B.w_override ? B.w_override[p] : P.w);
    const int a = P.a, mb = -P.b;
    const int e_del = P.e_del, e_ins = P.e_ins;
    const int oe_del = P.o_del + e_del, oe_ins = P.o_ins + e_ins;

    for (int c = lane; c <= n; c += 32)
        IO::store(slots, c, c == 0 ? h0 : max(0, h0 - P.o_ins - c * e_ins), 0);
    __syncwarp();

    const int64_t qoff = B.q_off[p];
    const uint8_t *tp = B.t + (B.t_off[p] >> 2);
    int lo = 0, hi = n;
    int best = h0, bi = -1, bj = -1, gbest = -1, gi = -1, moff = 0;
    unsigned long long ncell = 0;
    for (int i = 0; i < m; ++i) {
        const int tb = (__ldg(tp + (i >> 2)) >> (2 * (i & 3))) & 3;
        lo = max(lo, i - wb);
        hi = min(min(hi, i + wb + 1), n);
        const int hl0 = lo == 0 ? max(0, h0 - oe_del - i * e_del) : 0;
        int carry_f = 0, carry_h = hl0;
        int rm_l = 0, rj_l = -1;
        for (int cb = (lo / C) * C; cb < hi; cb += 32 * C) {
            const int j0 = cb + lane * C;
            int M[C], E0[C], Fl[C], H[C];
            bool act[C];
            int cnt = 0, floc = 0;
            uint32_t qbits = 0;
            if (j0 < hi && j0 + C > lo) {
#pragma unroll
                for (int k = 0; k < C; k += 4) {
                    const int64_t pos = qoff + j0 + k;
                    if (j0 + k < n) qbits |= (uint32_t)__ldg(B.q + (pos >> 2)) << (2 * k);
                }
                if (C < 4) qbits >>= 2 * ((qoff + j0) & 3);
            }
#pragma unroll
            for (int k = 0; k < C; ++k) {
                const int j = j0 + k;
                act[k] = j >= lo && j < hi;
                int d = 0, e = 0;
                if (act[k]) IO::load(slots, j, d, e);
                const int sc = (int)((qbits >> (2 * k)) & 3u) == tb ? a : mb;
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
                    IO::store(slots, j0 + k, hin, e2);
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
        if (lane == 0) IO::store(slots, hi, hl, 0);
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
            if (j < hi) IO::load(slots, j, h, e);
            const unsigned bal = __ballot_sync(kFull, (h | e) != 0);
            if (bal) { nlo = base + __ffs(bal) - 1; break; }
        }
        lo = nlo;
        int last = lo - 1;
        for (int top = hi; top >= lo; top -= 32) {
            const int j = top - lane;
            int h = 0, e = 0;
            if (j >= lo) IO::load(slots, j, h, e);
            const unsigned bal = __ballot_sync(kFull, (h | e) != 0);
            if (bal) { last = top - (__ffs(bal) - 1); break; }
        }
        hi = min(last + 2, n);
    }
    if (lane == 0) store_result(&B.out[p], best, bj + 1, bi + 1, gi + 1, gbest, moff);
    return ncell;
}

// Persistent warp-per-pair kernel over a class list (or the re-run list).
template <int C, bool S16>
__global__ void __launch_bounds__(256) k_warp(Batch B, Params P, Work W, int cls)
{
    const int lane = threadIdx.x & 31;
    const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    uint8_t *slots = W.slots + gw * W.slot_bytes_per_warp;
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
        if ((int64_t)(n + 1 + 32 * C) * SlotIO<S16>::kBytes > W.slot_bytes_per_warp) {
            if (lane == 0) atomicOr(W.status, kStTooLong);
            continue;
        }
        cells += warp_pair<C, S16>(B, P, p, slots);
    }
    if (lane == 0 && cells) atomicAdd(W.cells, cells);
}

// Baseline: one pair per warp in input order, no bucketing, no persistence
// beyond a grid-stride loop; 16-bit slots when the score bound allows.
__global__ void __launch_bounds__(256) k_plain(Batch B, Params P, Work W)
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
        cells += s16 ? warp_pair<1, true>(B, P, (int)p, slots) : warp_pair<1, false>(B, P, (int)p, slots);
    }
    if (lane == 0 && cells) atomicAdd(W.cells, cells);
}

// ------------------------------------------------------------------ launcher

namespace {

// Resident blocks per SM of each k_inter instantiation, set by prepare_kernels.
int g_inter_blocks[8] = {1, 1, 1, 1, 1, 1, 1, 1};

template <int NMAX> constexpr int inter_warps() { return NMAX >= 256 ? 2 : NMAX >= 128 ? 4 : 8; }
template <int NMAX> constexpr size_t inter_smem() { return (size_t)inter_warps<NMAX>() * (NMAX + 1) * 32 * 4; }
template <int NMAX, bool U8> constexpr int inter_index()
{
    return (U8 ? 0 : 4) + (NMAX >= 256 ? 0 : NMAX >= 128 ? 1 : NMAX >= 64 ? 2 : 3);
}

template <int NMAX, bool U8>
cudaError_t prepare_inter()
{
    cudaError_t e = cudaFuncSetAttribute(k_inter<NMAX, U8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)inter_smem<NMAX>());
    if (e != cudaSuccess) return e;
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_inter<NMAX, U8>, inter_warps<NMAX>() * 32,
                                                      inter_smem<NMAX>());
    if (e != cudaSuccess) return e;
    g_inter_blocks[inter_index<NMAX, U8>()] = nb > 0 ? nb : 1;
    return cudaSuccess;
}

template <int NMAX, bool U8>
cudaError_t launch_inter(const Batch &B, const Params &P, const Work &W, int cls, cudaStream_t st, int sms)
{
    const int blocks = sms * g_inter_blocks[inter_index<NMAX, U8>()];
    k_inter<NMAX, U8><<<blocks, inter_warps<NMAX>() * 32, inter_smem<NMAX>(), st>>>(B, P, W, cls);
    return cudaGetLastError();
}

template <int C, bool S16>
cudaError_t launch_warp(const Batch &B, const Params &P, const Work &W, int cls, cudaStream_t st, int blocks)
{
    k_warp<C, S16><<<blocks, kWarpKernelThreads, 0, st>>>(B, P, W, cls);
    return cudaGetLastError();
}

}  // namespace

cudaError_t prepare_kernels(int sms)
{
    (void)sms;
    cudaError_t e;
    if ((e = prepare_inter<256, true>()) != cudaSuccess) return e;
    if ((e = prepare_inter<128, true>()) != cudaSuccess) return e;
    if ((e = prepare_inter<64, true>()) != cudaSuccess) return e;
    if ((e = prepare_inter<32, true>()) != cudaSuccess) return e;
    if ((e = prepare_inter<256, false>()) != cudaSuccess) return e;
    if ((e = prepare_inter<128, false>()) != cudaSuccess) return e;
    if ((e = prepare_inter<64, false>()) != cudaSuccess) return e;
    return prepare_inter<32, false>();
}

int warp_slots_needed(int sms) { return sms * kWarpBlocksPerSM * (kWarpKernelThreads / 32); }

cudaError_t launch_batched(const Batch &B, const Params &P, const Work &W, const Streams &S, int sms)
{
    cudaError_t e;
    if (B.n <= 0) return cudaSuccess;
    const int cblocks = (int)((B.n + 511) / 512 < (int64_t)sms * 4 ? (B.n + 511) / 512 : (int64_t)sms * 4);
    k_classify<<<cblocks, 512, 0, S.main>>>(B, P, W);
    k_scan<<<1, 1024, 0, S.main>>>(W);
    const int sblocks = (int)((B.n + kScatterTile - 1) / kScatterTile < (int64_t)sms * 2 ? (B.n + kScatterTile - 1) / kScatterTile : (int64_t)sms * 2);
    k_scatter<<<sblocks, kScatterThreads, 0, S.main>>>(B.n, W);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // Fork: classes run concurrently on the side streams so that one class's
    // tail overlaps the next class's start.
    if ((e = cudaEventRecord(S.fork, S.main)) != cudaSuccess) return e;
    for (int k = 0; k < 3; ++k)
        if ((e = cudaStreamWaitEvent(S.side[k], S.fork, 0)) != cudaSuccess) return e;
    const int wblocks = sms * kWarpBlocksPerSM;
    if ((e = launch_inter<256, true>(B, P, W, 0, S.side[0], sms)) != cudaSuccess) return e;
    if ((e = launch_inter<128, true>(B, P, W, 1, S.side[0], sms)) != cudaSuccess) return e;
    if ((e = launch_inter<64, true>(B, P, W, 2, S.side[1], sms)) != cudaSuccess) return e;
    if ((e = launch_inter<32, true>(B, P, W, 3, S.side[1], sms)) != cudaSuccess) return e;
    if ((e = launch_warp<4, true>(B, P, W, 8, S.side[2], wblocks)) != cudaSuccess) return e;
    if ((e = launch_warp<4, false>(B, P, W, 9, S.side[2], wblocks)) != cudaSuccess) return e;
    if ((e = launch_inter<256, false>(B, P, W, 4, S.side[2], sms)) != cudaSuccess) return e;
    if ((e = launch_inter<128, false>(B, P, W, 5, S.side[2], sms)) != cudaSuccess) return e;
    if ((e = launch_inter<64, false>(B, P, W, 6, S.side[2], sms)) != cudaSuccess) return e;
    if ((e = launch_inter<32, false>(B, P, W, 7, S.side[2], sms)) != cudaSuccess) return e;
    for (int k = 0; k < 3; ++k) {
        if ((e = cudaEventRecord(S.join[k], S.side[k])) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(S.main, S.join[k], 0)) != cudaSuccess) return e;
    }
    // Section V-D1: pairs whose scores left their lane range, exactly, in 32 bits.
    return launch_warp<4, false>(B, P, W, kRerun, S.main, wblocks);
}

cudaError_t launch_batched_serial(const Batch &B, const Params &P, const Work &W, cudaStream_t st, int sms,
                                  int warp_blocks)
{
    cudaError_t e;
    if (B.n <= 0) return cudaSuccess;
    const int cblocks = (int)((B.n + 511) / 512 < (int64_t)sms * 4 ? (B.n + 511) / 512 : (int64_t)sms * 4);
    k_classify<<<cblocks, 512, 0, st>>>(B, P, W);
    k_scan<<<1, 1024, 0, st>>>(W);
    const int sblocks = (int)((B.n + kScatterTile - 1) / kScatterTile < (int64_t)sms * 2 ? (B.n + kScatterTile - 1) / kScatterTile : (int64_t)sms * 2);
    k_scatter<<<sblocks, kScatterThreads, 0, st>>>(B.n, W);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = launch_inter<256, true>(B, P, W, 0, st, sms)) != cudaSuccess) return e;
    if ((e = launch_inter<128, true>(B, P, W, 1, st, sms)) != cudaSuccess) return e;
    if ((e = launch_inter<64, true>(B, P, W, 2, st, sms)) != cudaSuccess) return e;
    if ((e = launch_inter<32, true>(B, P, W, 3, st, sms)) != cudaSuccess) return e;
    if ((e = launch_inter<256, false>(B, P, W, 4, st, sms)) != cudaSuccess) return e;
    if ((e = launch_inter<128, false>(B, P, W, 5, st, sms)) != cudaSuccess) return e;
    if ((e = launch_inter<64, false>(B, P, W, 6, st, sms)) != cudaSuccess) return e;
    if ((e = launch_inter<32, false>(B, P, W, 7, st, sms)) != cudaSuccess) return e;
    if ((e = launch_warp<4, true>(B, P, W, 8, st, warp_blocks)) != cudaSuccess) return e;
    if ((e = launch_warp<4, false>(B, P, W, 9, st, warp_blocks)) != cudaSuccess) return e;
    return launch_warp<4, false>(B, P, W, kRerun, st, warp_blocks);
}

cudaError_t launch_plain(const Batch &B, const Params &P, const Work &W, cudaStream_t st, int sms)
{
    if (B.n <= 0) return cudaSuccess;
    k_plain<<<sms * kWarpBlocksPerSM, kWarpKernelThreads, 0, st>>>(B, P, W);
    return cudaGetLastError();
}

}  // namespace bsw
