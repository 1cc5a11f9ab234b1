// bsw_fm.cu - FM-index and super-maximal exact matches (Section IV).
//
// The text is T = ref + revcomp(ref) (Section IV-A: the SMEM search works on
// the reference with its reverse complement), followed by a terminator $
// smaller than every base.  Two FM-indexes are kept: of T, for the SA
// intervals of the matches, and of reverse(T), whose backward search takes a
// read's bases left to right, i.e. extends a match forward.
//
// O (Algorithm 1) is kept in buckets of eta = 32 BWT positions: entry t holds
// the counts of each base in BWT[0, 32t) and the 32 BWT bases of the bucket,
// 2-bit packed in one 64-bit word: 32 bytes, one DRAM sector per lookup (the
// paper's CPU layout uses 64-byte entries with a byte per base for AVX2
// compares; a 2-bit word and a population count serve the GPU).  O(c, i) =
// count + the matches of c among the bucket's first i mod 32 bases; the $ row
// is stored as base 0 and subtracted.
//
// SMEMs of a read X (Li 2012; the paper's Algorithm 4 finds the same set
// position by position): with e(i) the end of the longest prefix of X[i:]
// occurring in T, the SMEMs are [i, e(i)) for i = 0 or e(i-1) < e(i).
// e(i) is computed for every read position in parallel (one thread each),
// then one thread per read lists its SMEMs of at least min_len bases and
// finds each one's SA interval [k, k + s) in T by backward search.
#include <cuda_runtime.h>
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

// Occurrences of c in BWT[0, i) (Algorithm 1).
__device__ __forceinline__ uint32_t get_o(const FmDev &F, int c, int64_t i)
{
    const FmEntry *e = F.occ + (i >> 5);
    const int y = (int)(i & 31);
    const uint64_t x = __ldg(&e->bwt) ^ (0x5555555555555555ull * (uint64_t)c);
    const uint64_t same = ~(x | (x >> 1)) & 0x5555555555555555ull;   // bit 2j: base j == c
    const uint64_t below = y ? (~0ull >> (64 - 2 * y)) : 0ull;
    uint32_t w = __ldg(&e->cnt[c]) + (uint32_t)__popcll(same & below);
    if (c == 0 && F.primary >= i - y && F.primary < i) --w;   // the $ row is stored as base 0
    return w;
}

// Backward search step: the SA interval of bX from that of X.
__device__ __forceinline__ void back_step(const FmDev &F, int c, int64_t &lo, int64_t &hi)
{
    lo = F.C[c] + get_o(F, c, lo);
    hi = F.C[c] + get_o(F, c, hi);
}

__device__ __forceinline__ int read_base(const uint8_t *reads, int64_t pos)
{
    return (__ldg(reads + (pos >> 2)) >> (2 * (pos & 3))) & 3;
}

// e(i) for every position of every read: one thread per (read, position),
// position i of read r at r * lmax + i, backward search on the index of
// reverse(T) with the read's bases from i onward.
__global__ void __launch_bounds__(256) k_match_end(SmemIn R, FmDev Frev, int32_t *end)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t n_pos = R.n_reads * (int64_t)R.lmax;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n_pos; g += stride) {
        const int64_t r = g / R.lmax;
        const int i = (int)(g - r * R.lmax);
        const int L = R.read_len[r];
        if (i >= L) continue;
        const int64_t base = R.read_off[r];
        int64_t lo = 0, hi = Frev.n;
        int j = i;
        while (j < L) {
            int64_t l2 = lo, h2 = hi;
            back_step(Frev, read_base(R.reads, base + j), l2, h2);
            if (l2 >= h2) break;
            lo = l2;
            hi = h2;
            ++j;
        }
        end[g] = j;
    }
}

// One thread per read: count (write = false) or write its SMEMs.
template <bool WRITE>
__global__ void __launch_bounds__(256) k_smem(SmemIn R, FmDev F, const int32_t *end, int min_len, int64_t *count,
                                             const int64_t *first, bsw_smem_t *out)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < R.n_reads; r += stride) {
        const int L = R.read_len[r];
        const int32_t *e = end + r * (int64_t)R.lmax;
        int64_t n = 0, o = WRITE ? first[r] : 0;
        for (int i = 0; i < L; ++i) {
            const int ei = e[i];
            if ((i > 0 && e[i - 1] >= ei) || ei - i < min_len) continue;
            if (WRITE) {
                int64_t lo = 0, hi = F.n;
                for (int j = ei - 1; j >= i; --j) back_step(F, read_base(R.reads, R.read_off[r] + j), lo, hi);
                bsw_smem_t s;
                s.read_id = (int32_t)r;
                s.qbeg = i;
                s.len = ei - i;
                s.reserved = 0;
                s.k = lo;
                s.s = hi - lo;
                out[o + n] = s;
            }
            ++n;
        }
        if (!WRITE) count[r] = n;
    }
}

int grid_for(int64_t n, int per_block, int sms)
{
    const int64_t b = (n + per_block - 1) / per_block;
    return (int)(b < (int64_t)sms * 16 ? (b > 0 ? b : 1) : (int64_t)sms * 16);
}

}  // namespace

cudaError_t launch_match_end(const SmemIn &R, const FmDev &Frev, int32_t *end, cudaStream_t st, int sms)
{
    const int64_t n_pos = R.n_reads * (int64_t)R.lmax;
    if (n_pos <= 0) return cudaSuccess;
    k_match_end<<<grid_for(n_pos, 256, sms), 256, 0, st>>>(R, Frev, end);
    return cudaGetLastError();
}

cudaError_t launch_smem(bool write, const SmemIn &R, const FmDev &F, const int32_t *end, int min_len, int64_t *count,
                        const int64_t *first, bsw_smem_t *out, cudaStream_t st, int sms)
{
    if (R.n_reads <= 0) return cudaSuccess;
    if (write) k_smem<true><<<grid_for(R.n_reads, 256, sms), 256, 0, st>>>(R, F, end, min_len, count, first, out);
    else k_smem<false><<<grid_for(R.n_reads, 256, sms), 256, 0, st>>>(R, F, end, min_len, count, first, out);
    return cudaGetLastError();
}

}  // namespace bsw
