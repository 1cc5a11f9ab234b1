// bsw_fm.cu - FM-index and super-maximal exact matches (Section IV).
//
// The text is T = ref + revcomp(ref) (Section IV-A: the SMEM search works on
// the reference with its reverse complement), followed by a terminator $
// smaller than every base.  One FM-index of T serves both directions: since
// revcomp(T) = T, a pattern P and revcomp(P) occur equally often, and the
// pair of their suffix-array intervals (the bi-interval [k, l, s] of
// Algorithms 2-3) can be extended by one base on either side.
//
// O (Algorithm 1) is kept in buckets of eta = 32 BWT positions: entry t holds
// the counts of each base in BWT[0, 32t) and the 32 BWT bases of the bucket,
// 2-bit packed in one 64-bit word: 32 bytes, one DRAM sector per lookup (the
// paper's CPU layout uses 64-byte entries with a byte per base for AVX2
// compares; a 2-bit word and population counts serve the GPU).  One lookup
// gives the occurrences of all four bases; the $ row is stored as base 0 and
// subtracted.
//
// SMEMs of a read X (Li 2012; Algorithm 4): from a position x, extend X[x]
// forward base by base, keeping the bi-interval each time its size is about to
// shrink (one per distinct occurrence count, longest match last); then extend
// those matches backward one base at a time, longest first.  A match that can
// no longer be extended while no longer one survives at that base is an SMEM.
// The next x is the end of the longest match from x; every SMEM holds exactly
// one of the visited x.  One thread takes one read at a time; its list of
// bi-intervals lives in shared memory (kListCap entries), and a read whose
// list would grow beyond that is finished by a launch with lists in global
// memory.  One pass keeps up to kSmemKeep records per read in a scratch
// buffer; after the host's prefix sum a gather puts them in place, and the
// rare reads with more are searched again, writing in place.
#include <cuda_runtime.h>
#include <climits>
#include <cstdint>
#include <vector>

#include "bsw.h"
#include "bsw_launch.h"

namespace bsw {

// ------------------------------------------------------------------ host build

// Index of one text (codes 0..3, length n) from its suffix array sa[0..n].
void fm_from_sa(const uint8_t *text, int64_t n, const int32_t *sa, FmHost &out)
{
    const int64_t N = n + 1;
    out.n = N;
    out.occ.assign((size_t)(N / 32 + 1), FmEntry{{0, 0, 0, 0}, 0, 0});
    uint32_t cnt[4] = {0, 0, 0, 0};
    out.primary = -1;
    for (int64_t i = 0; i < N; ++i) {
        if ((i & 31) == 0) {
            FmEntry &e = out.occ[(size_t)(i >> 5)];
            for (int c = 0; c < 4; ++c) e.cnt[c] = cnt[c];
        }
        int b;
        if (sa[i] == 0) {
            out.primary = i;                              // the $ row: stored as 0, not counted
            b = 0;
        } else {
            b = text[sa[i] - 1];
            ++cnt[b];
        }
        out.occ[(size_t)(i >> 5)].bwt |= (uint64_t)b << (2 * (i & 31));
    }
    if ((N & 31) == 0) {
        FmEntry &e = out.occ[(size_t)(N >> 5)];
        for (int c = 0; c < 4; ++c) e.cnt[c] = cnt[c];
    }
    out.C[0] = 1;                                         // the terminator sorts first
    for (int c = 0; c < 4; ++c) out.C[c + 1] = out.C[c] + cnt[c];
}

// --------------------------------------------------------------------- device

namespace {

// Occurrences of each base in BWT[0, i) (Algorithm 1, all four from one bucket).
__device__ __forceinline__ void occ4(const FmDev &F, uint32_t i, uint32_t o[4])
{
    const FmEntry *e = F.occ + (i >> 5);
    const int y = (int)(i & 31);
    const uint4 c = __ldg(reinterpret_cast<const uint4 *>(e->cnt));
    const uint64_t w = __ldg(&e->bwt);
    const uint64_t m = (y ? (~0ull >> (64 - 2 * y)) : 0ull) & 0x5555555555555555ull;   // bit 2j, j < y
    const uint64_t lo = w & m, hi = (w >> 1) & m;                                        // the two bits of base j
    o[0] = c.x + (uint32_t)__popcll(m & ~lo & ~hi);
    o[1] = c.y + (uint32_t)__popcll(lo & ~hi);
    o[2] = c.z + (uint32_t)__popcll(hi & ~lo);
    o[3] = c.w + (uint32_t)__popcll(lo & hi);
    if (F.primary >= (int64_t)(i - y) && F.primary < (int64_t)i) --o[0];   // the $ row, stored as base 0
}

// The bi-interval of bP from that of P (Algorithm 2's backward extension).
// A forward extension (Algorithm 3) is the same step: the bi-interval of Pc
// is that of comp(c) revcomp(P) with the two intervals swapped.
// [k', k'+s') holds the suffixes of [k, k+s) preceded by b.  revcomp(bP) =
// revcomp(P) comp(b), whose interval inside [l, l+s) comes after the suffix
// revcomp(P)$ (if any) and the extensions by bases smaller than comp(b), i.e.
// after as many rows as P has occurrences preceded by the terminator or by a
// base larger than b.
__device__ __forceinline__ BiIv back_ext(const FmDev &F, const uint32_t C[5], BiIv v, int b)
{
    uint32_t ok[4], oe[4];
    occ4(F, v.k, ok);
    occ4(F, v.k + v.s, oe);
    uint32_t above = 0;
#pragma unroll
    for (int c = 3; c > 0; --c)
        if (c > b) above += oe[c] - ok[c];
    const uint32_t sent = (F.primary >= (int64_t)v.k && F.primary < (int64_t)v.k + v.s) ? 1u : 0u;
    uint32_t kb = ok[0], sb = oe[0] - ok[0];
#pragma unroll
    for (int c = 1; c < 4; ++c)
        if (c == b) { kb = ok[c]; sb = oe[c] - ok[c]; }
    return BiIv{C[b] + kb, v.l + sent + above, sb, v.e};
}

// Base pos of the reads: 0..3, or 4 for an N.
__device__ __forceinline__ int read_base(const SmemIn &R, int64_t pos)
{
    if (R.reads_n && ((__ldg(R.reads_n + (pos >> 3)) >> (pos & 7)) & 1)) return 4;
    return (__ldg(R.reads + (pos >> 2)) >> (2 * (pos & 3))) & 3;
}

// All SMEMs of at least min_len bases of the reads t < t_end taken from the
// counter *W.next (read ids[t], or t when ids is null), in increasing start
// order.  Store mode: count[r], and the first kSmemKeep records at
// scratch[r * kSmemKeep]; a read with more is finished by a write-mode launch.
// Write mode: the records at out[first[r]].  A lane's list holds cap entries
// at list[0], list[stride], ...; in store mode a read that needs more is
// dropped (count -1, its id appended to ovf_list) and finished by a launch
// with longer lists.
//
// The lane is a small state machine so that every pass of the main loop makes
// exactly one bi-interval extension on every lane that has work (the memory
// lookups of Algorithm 1 dominate; lanes of a warp run in step instead of
// each following its own loop nest).  States between extensions:
//   kRead  take the next read;     kCall  start the search from x;
//   kBack  forward pass over, start the backward pass;
//   kEnd   the search from x is over;
//   kFwd   pending: extend v forward by X[i];
//   kBwd   pending: extend list[p] backward by X[j].
template <bool WRITE>
__device__ void smem_lanes(const SmemIn &R, const FmDev &F, const uint32_t C[5], int min_len, int64_t t_end,
                           const int32_t *ids, BiIv *list, int stride, int cap, const SmemWork &W)
{
    enum { kRead, kCall, kBack, kEnd, kFwd, kBwd };
    int state = kRead;
    int64_t r = 0, base = 0, o = 0, n = 0, call0 = 0;
    int L = 0, x = 0, i = 0, j = 0, p = 0, m = 0, mc = 0, next = 0, last = 0;
    BiIv v{0, 0, 0, 0};
    auto emit = [&](int start, int len, const BiIv &u) {
        if (len < min_len) return;
        bsw_smem_t sm;
        sm.read_id = (int32_t)r;
        sm.qbeg = start;
        sm.len = len;
        sm.reserved = 0;
        sm.k = u.k;
        sm.s = u.s;
        if (WRITE) W.out[o + n] = sm;
        else if (n < kSmemKeep) W.scratch[o + n] = sm;
        ++n;
    };
    for (;;) {
        // settle: run the bookkeeping up to the next extension
        while (state < kFwd) {
            if (state == kRead) {
                const int64_t t = atomicAdd(W.next, 1u);
                if (t >= t_end) return;
                r = ids ? ids[t] : t;
                L = R.read_len[r];
                base = R.read_off[r];
                o = WRITE ? W.first[r] : r * kSmemKeep;
                n = 0;
                x = 0;
                state = kCall;
            } else if (state == kCall) {
                if (x >= L) {
                    if (!WRITE) W.count[r] = n;
                    state = kRead;
                    continue;
                }
                const int c0 = read_base(R, base + x);
                if (c0 > 3) {                                           // no match starts at an N
                    ++x;
                    continue;
                }
                v = BiIv{C[c0], C[3 - c0], C[c0 + 1] - C[c0], 0};
                m = 0;
                i = x + 1;
                if (i < L) {
                    state = kFwd;
                } else {
                    v.e = L;
                    list[(m++) * stride] = v;
                    state = kBack;
                }
            } else if (state == kBack) {
                for (int a = 0, b = m - 1; a < b; ++a, --b) {          // longest first
                    const BiIv u = list[a * stride];
                    list[a * stride] = list[b * stride];
                    list[b * stride] = u;
                }
                next = list[0].e;
                call0 = n;
                last = INT_MAX;
                j = x - 1;
                p = 0;
                mc = 0;
                if (j >= 0) {
                    state = kBwd;
                } else {                                                // at the read start: the longest is an SMEM
                    emit(0, list[0].e, list[0]);
                    state = kEnd;
                }
            } else {                                                    // kEnd
                // this search emitted starts in decreasing order
                bsw_smem_t *seg = WRITE ? W.out : W.scratch;
                if (WRITE || n <= kSmemKeep)
                    for (int64_t a = o + call0, b = o + n - 1; a < b; ++a, --b) {
                        const bsw_smem_t u = seg[a];
                        seg[a] = seg[b];
                        seg[b] = u;
                    }
                x = next;
                state = kCall;
            }
        }

        // one extension (Algorithm 2), the same code on every lane
        const bool fwd = state == kFwd;
        const BiIv u = fwd ? BiIv{v.l, v.k, v.s, 0} : list[p * stride];
        const int cb = read_base(R, base + (fwd ? i : j));
        BiIv w = back_ext(F, C, u, fwd ? 3 - (cb & 3) : cb & 3);
        if (cb > 3) w.s = 0;                                        // an N extends nothing

        if (fwd) {
            w = BiIv{w.l, w.k, w.s, 0};
            if (w.s != v.s) {                                       // X[x..i) is the longest with its count
                if (m == cap) goto overflow;
                v.e = i;
                list[(m++) * stride] = v;
                if (w.s == 0) {
                    state = kBack;
                    continue;
                }
            }
            v = w;
            if (++i == L) {                                         // the match reaches the read end
                if (m == cap) goto overflow;
                v.e = L;
                list[(m++) * stride] = v;
                state = kBack;
            }
            continue;
        } else {
            if (w.s == 0) {
                if (mc == 0 && j + 1 < last) {                      // no longer match survives: an SMEM
                    last = j + 1;
                    emit(last, u.e - last, u);
                }
            } else if (mc == 0 || w.s != list[(mc - 1) * stride].s) {
                w.e = u.e;
                list[(mc++) * stride] = w;
            }
            if (++p == m) {
                if (mc == 0) {
                    state = kEnd;
                } else {
                    m = mc;
                    mc = 0;
                    p = 0;
                    if (--j < 0) {                                  // at the read start
                        emit(0, list[0].e, list[0]);
                        state = kEnd;
                    }
                }
            }
            continue;
        }
    overflow:
        if (!WRITE) {
            W.count[r] = -1;
            W.ovf_list[atomicAdd(W.ovf_n, 1u)] = (int32_t)r;
        }
        state = kRead;
    }
}

__device__ __forceinline__ void load_c(const FmDev &F, uint32_t C[5])
{
#pragma unroll
    for (int c = 0; c < 5; ++c) C[c] = (uint32_t)F.C[c];
}

// Store mode over all reads with the lists in shared memory.
__global__ void __launch_bounds__(kSmemThreads) k_smem_store(SmemIn R, FmDev F, int min_len, SmemWork W)
{
    extern __shared__ BiIv lists[];
    uint32_t C[5];
    load_c(F, C);
    smem_lanes<false>(R, F, C, min_len, R.n_reads, nullptr, lists + threadIdx.x, blockDim.x, kListCap, W);
}

// The reads ids[0..n_ids) with lists in global memory, cap entries per lane
// (enough for any read of the batch).
template <bool WRITE>
__global__ void __launch_bounds__(256) k_smem_global(SmemIn R, FmDev F, int min_len, SmemWork W, const int32_t *ids,
                                                     int64_t n_ids, BiIv *lists, int cap)
{
    uint32_t C[5];
    load_c(F, C);
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_ids) return;                     // at most n_ids lanes take reads: list slots g < n_ids
    smem_lanes<WRITE>(R, F, C, min_len, n_ids, ids, lists + g * cap, 1, cap, W);
}

// Records of the reads with at most kSmemKeep from the scratch to out[first[r]].
__global__ void __launch_bounds__(256) k_smem_gather(int64_t n_reads, SmemWork W)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n_reads; r += stride) {
        const int64_t c = W.count[r];
        if (c > kSmemKeep) continue;
        for (int64_t k = 0; k < c; ++k) W.out[W.first[r] + k] = W.scratch[r * kSmemKeep + k];
    }
}

int grid_for(int64_t n, int per_block, int sms, int per_sm)
{
    const int64_t b = (n + per_block - 1) / per_block;
    return (int)(b < (int64_t)sms * per_sm ? (b > 0 ? b : 1) : (int64_t)sms * per_sm);
}

}  // namespace

cudaError_t launch_smem_store(const SmemIn &R, const FmDev &F, int min_len, const SmemWork &W, cudaStream_t st, int sms)
{
    if (R.n_reads <= 0) return cudaSuccess;
    const size_t smem = sizeof(BiIv) * kListCap * kSmemThreads;
    cudaError_t e = cudaFuncSetAttribute(k_smem_store, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(W.next, 0, 4, st);
    if (e != cudaSuccess) return e;
    k_smem_store<<<grid_for(R.n_reads, kSmemThreads, sms, kSmemBlocksPerSm), kSmemThreads, smem, st>>>(R, F, min_len, W);
    return cudaGetLastError();
}

cudaError_t launch_smem_global(bool write, const SmemIn &R, const FmDev &F, int min_len, const SmemWork &W,
                               const int32_t *ids, int64_t n_ids, BiIv *lists, int cap, cudaStream_t st, int sms)
{
    if (n_ids <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(W.next, 0, 4, st);
    if (e != cudaSuccess) return e;
    const int blocks = grid_for(n_ids, 256, sms, 8);
    if (write) k_smem_global<true><<<blocks, 256, 0, st>>>(R, F, min_len, W, ids, n_ids, lists, cap);
    else k_smem_global<false><<<blocks, 256, 0, st>>>(R, F, min_len, W, ids, n_ids, lists, cap);
    return cudaGetLastError();
}

cudaError_t launch_smem_gather(int64_t n_reads, const SmemWork &W, cudaStream_t st, int sms)
{
    if (n_reads <= 0) return cudaSuccess;
    k_smem_gather<<<grid_for(n_reads, 256, sms, 8), 256, 0, st>>>(n_reads, W);
    return cudaGetLastError();
}

}  // namespace bsw
