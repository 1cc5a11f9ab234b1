// bsw_driver.cu - kernels of the seed-extension driver (bsw_extend_seeds).
//
// Section V-C2: every seed of a read is extended, and the results are filtered
// afterwards.  Per seed the driver extends left (the read prefix before the
// seed, reversed, against the reference before it, reversed), decides the left
// end, extends right (the read suffix against the reference after the seed)
// from the left score, decides the right end, and finally drops seeds that an
// earlier alignment of the same read covers.  Readings where the paper is
// silent (BWA-MEM's behaviour): a side's target is its query length + w bases;
// the read end is taken unless gscore <= 0 or gscore <= score - end_bonus; an
// extension whose max_off reaches (w >> 1) + (w >> 2) of its band runs again
// with twice the band; a seed inside an earlier kept alignment of its read is
// not kept.  The extensions themselves run in the batched kernels.
#include <cuda_runtime.h>
#include <cstdint>

#include "bsw.h"
#include "bsw_device.cuh"
#include "bsw_launch.h"

namespace bsw {

namespace {

__device__ __forceinline__ uint32_t base_at(const uint8_t *packed, int64_t pos)
{
    return (__ldg(packed + (pos >> 2)) >> (2 * (pos & 3))) & 3u;
}

__device__ __forceinline__ uint32_t n_at(const uint8_t *nm, int64_t pos)
{
    return nm ? (__ldg(nm + (pos >> 3)) >> (pos & 7)) & 1u : 0u;
}

// One warp per seed: the side's query and target as 2-bit packed sequences in
// the seed's fixed slots (qslot, tslot bases, multiples of 16), their N
// bitmaps when the side has them, plus the pair's lengths, offsets and h0.
template <bool LEFT>
__global__ void __launch_bounds__(256) k_side(DriverIn D, DriverSide S, int64_t n, int w, int match)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t k = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); k < n; k += nw) {
        const bsw_seed_t sd = D.seeds[k];
        const int64_t roff = D.read_off[sd.read_id];
        const int rl = D.read_len[sd.read_id];
        int qlen, tlen;
        int64_t qsrc, tsrc;                                  // first source base (LEFT: the one before)
        if (LEFT) {
            qlen = sd.qbeg;
            tlen = (int)min((int64_t)sd.qbeg + w, sd.rbeg);
            qsrc = roff + sd.qbeg - 1;
            tsrc = sd.rbeg - 1;
        } else {
            const int qe = sd.qbeg + sd.len;
            const int64_t re = sd.rbeg + sd.len;
            qlen = rl - qe;
            tlen = (int)max((int64_t)0, min((int64_t)qlen + w, D.ref_len - re));
            qsrc = roff + qe;
            tsrc = re;
        }
        const int64_t qo = k * (int64_t)S.qslot, to = k * (int64_t)S.tslot;
        for (int b = lane; b < (qlen + 3) / 4; b += 32) {
            uint32_t v = 0;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int j = 4 * b + u;
                if (j < qlen) v |= base_at(D.reads, LEFT ? qsrc - j : qsrc + j) << (2 * u);
            }
            S.q[(qo >> 2) + b] = (uint8_t)v;
        }
        for (int b = lane; b < (tlen + 3) / 4; b += 32) {
            uint32_t v = 0;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int j = 4 * b + u;
                if (j < tlen) v |= base_at(D.ref, LEFT ? tsrc - j : tsrc + j) << (2 * u);
            }
            S.t[(to >> 2) + b] = (uint8_t)v;
        }
        if (S.q_n) {                                         // slots start on a byte of the bitmaps
            for (int b = lane; b < (qlen + 7) / 8; b += 32) {
                uint32_t v = 0;
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int j = 8 * b + u;
                    if (j < qlen) v |= n_at(D.reads_n, LEFT ? qsrc - j : qsrc + j) << u;
                }
                S.q_n[(qo >> 3) + b] = (uint8_t)v;
            }
            for (int b = lane; b < (tlen + 7) / 8; b += 32) {
                uint32_t v = 0;
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int j = 8 * b + u;
                    if (j < tlen) v |= n_at(D.ref_n, LEFT ? tsrc - j : tsrc + j) << u;
                }
                S.t_n[(to >> 3) + b] = (uint8_t)v;
            }
        }
        if (lane == 0) {
            S.q_off[k] = qo;
            S.q_len[k] = qlen;
            S.t_off[k] = to;
            S.t_len[k] = tlen;
            S.h0[k] = LEFT ? sd.len * match : S.h0[k];      // the right side's h0 was set by the left decision
            S.w_cur[k] = w;
        }
    }
}

// Pairs whose last run (band wt) reached max_off >= (wt >> 1) + (wt >> 2): the
// compact list for the next run with band wnext.
__global__ void k_retry_select(DriverSide S, int64_t n, int wt, int32_t *list, uint32_t *count)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride)
        if (S.w_cur[k] == wt && S.res[k].max_off >= (wt >> 1) + (wt >> 2))
            list[atomicAdd(count, 1u)] = (int32_t)k;
}

__global__ void k_retry_gather(DriverSide S, const int32_t *list, const uint32_t *count, int wnext, DriverCompact C)
{
    const int64_t cnt = *count;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += stride) {
        const int k = list[i];
        C.q_off[i] = S.q_off[k];
        C.q_len[i] = S.q_len[k];
        C.t_off[i] = S.t_off[k];
        C.t_len[i] = S.t_len[k];
        C.h0[i] = S.h0[k];
        C.w[i] = wnext;
    }
}

__global__ void k_retry_scatter(DriverSide S, const int32_t *list, const uint32_t *count, int wnext, DriverCompact C)
{
    const int64_t cnt = *count;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += stride) {
        const int k = list[i];
        S.res[k] = C.res[i];
        S.w_cur[k] = wnext;
    }
}

// The end of one side: the read end unless gscore <= 0 or gscore <= score -
// end_bonus.  Left: the aligned start and the right side's h0.  Right: the
// aligned end and the score.
template <bool LEFT>
__global__ void k_decide(DriverIn D, DriverSide S, int64_t n, int end_bonus, bsw_aln_t *out)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
        const bsw_result_t r = S.res[k];
        const bsw_seed_t sd = D.seeds[k];
        const bool local = r.gscore <= 0 || r.gscore <= r.score - end_bonus;
        const int qext = local ? r.qle : S.q_len[k];
        const int text = local ? r.tle : r.gtle;
        const int sc = local ? r.score : r.gscore;
        bsw_aln_t a = out[k];
        if (LEFT) {
            a.qb = sd.qbeg - qext;
            a.rb = sd.rbeg - text;
            a.w_left = S.q_len[k] > 0 ? S.w_cur[k] : 0;
            S.h0[k] = sc;                                    // the right extension starts from the left score
        } else {
            a.qe = sd.qbeg + sd.len + qext;
            a.re = sd.rbeg + sd.len + text;
            a.score = sc;
            a.w_right = S.q_len[k] > 0 ? S.w_cur[k] : 0;
            a.kept = 1;
        }
        out[k] = a;
    }
}

// One thread per read (the thread at the read's first seed): in seed order, a
// seed whose read and reference intervals lie inside the alignment of an
// earlier kept seed of the read is not kept.
__global__ void k_filter(DriverIn D, int64_t n, bsw_aln_t *out)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += stride) {
        const int rid = D.seeds[s].read_id;
        if (s > 0 && D.seeds[s - 1].read_id == rid) continue;
        int64_t e = s;
        while (e < n && D.seeds[e].read_id == rid) ++e;
        for (int64_t k = s + 1; k < e; ++k) {
            const bsw_seed_t sd = D.seeds[k];
            for (int64_t j = s; j < k; ++j) {
                const bsw_aln_t a = out[j];
                if (a.kept && a.qb <= sd.qbeg && sd.qbeg + sd.len <= a.qe && a.rb <= sd.rbeg && sd.rbeg + sd.len <= a.re) {
                    out[k].kept = 0;
                    break;
                }
            }
        }
    }
}

// Reads: offsets on a base multiple of 4, lengths in [0, kLongMax]; the
// packed extent and the longest read.
__global__ void __launch_bounds__(256) k_check_reads(DriverIn D, int64_t n_reads, DriverCheck *X)
{
    unsigned long long rb = 0;
    int mx = 0;
    uint32_t bad = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n_reads; r += stride) {
        const int64_t o = D.read_off[r];
        const int32_t l = D.read_len[r];
        if (o < 0 || (o & 3) || l < 0 || l > kLongMax) { bad = 1; continue; }
        rb = max(rb, (unsigned long long)((o + l + 3) >> 2));
        mx = max(mx, l);
    }
    for (int d = 16; d > 0; d >>= 1) {
        rb = max(rb, __shfl_xor_sync(0xffffffffu, rb, d));
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, d));
        bad |= __shfl_xor_sync(0xffffffffu, bad, d);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&X->read_bytes, rb);
        atomicMax(&X->maxrl, mx);
        if (bad) atomicOr(&X->inval, 1u);
    }
}

// Seeds: inside their read and the reference, the right side's score bound
// within 2^30, and each read's seeds one consecutive run.  Reads are checked
// by k_check_reads in the same stream before this kernel's results are used;
// a seed of an invalid read only reads that read's length.
__global__ void __launch_bounds__(256) k_check_seeds(DriverIn D, int64_t n_reads, int64_t n_seeds, int match,
                                                     uint32_t *runs, DriverCheck *X)
{
    uint32_t bad = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_seeds; k += stride) {
        const bsw_seed_t sd = D.seeds[k];
        if (sd.read_id < 0 || sd.read_id >= n_reads) { bad = 1; continue; }
        const int32_t rl = D.read_len[sd.read_id];
        if (sd.qbeg < 0 || sd.len < 0 || (int64_t)sd.qbeg + sd.len > rl || sd.rbeg < 0 || sd.rbeg + sd.len > D.ref_len ||
            (long long)match * (2 * (long long)rl + 1) >= (1ll << 30))
            bad = 1;
        if ((k == 0 || D.seeds[k - 1].read_id != sd.read_id) && atomicAdd(&runs[sd.read_id], 1u) != 0u) bad = 1;
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&X->inval, 1u);
}

int grid_for(int64_t n, int per_block, int sms)
{
    const int64_t b = (n + per_block - 1) / per_block;
    return (int)(b < (int64_t)sms * 8 ? (b > 0 ? b : 1) : (int64_t)sms * 8);
}

}  // namespace

cudaError_t launch_side(bool left, const DriverIn &D, const DriverSide &S, int64_t n, int w, int match,
                        cudaStream_t st, int sms)
{
    const int blocks = grid_for(n, 8, sms);
    if (left) k_side<true><<<blocks, 256, 0, st>>>(D, S, n, w, match);
    else k_side<false><<<blocks, 256, 0, st>>>(D, S, n, w, match);
    return cudaGetLastError();
}

cudaError_t launch_retry_select(const DriverSide &S, int64_t n, int wt, int32_t *list, uint32_t *count,
                                cudaStream_t st, int sms)
{
    k_retry_select<<<grid_for(n, 256, sms), 256, 0, st>>>(S, n, wt, list, count);
    return cudaGetLastError();
}

cudaError_t launch_retry_gather(const DriverSide &S, const int32_t *list, const uint32_t *count, int64_t n_max,
                                int wnext, const DriverCompact &C, cudaStream_t st, int sms)
{
    k_retry_gather<<<grid_for(n_max, 256, sms), 256, 0, st>>>(S, list, count, wnext, C);
    return cudaGetLastError();
}

cudaError_t launch_retry_scatter(const DriverSide &S, const int32_t *list, const uint32_t *count, int64_t n_max,
                                 int wnext, const DriverCompact &C, cudaStream_t st, int sms)
{
    k_retry_scatter<<<grid_for(n_max, 256, sms), 256, 0, st>>>(S, list, count, wnext, C);
    return cudaGetLastError();
}

cudaError_t launch_decide(bool left, const DriverIn &D, const DriverSide &S, int64_t n, int end_bonus,
                          bsw_aln_t *out, cudaStream_t st, int sms)
{
    if (left) k_decide<true><<<grid_for(n, 256, sms), 256, 0, st>>>(D, S, n, end_bonus, out);
    else k_decide<false><<<grid_for(n, 256, sms), 256, 0, st>>>(D, S, n, end_bonus, out);
    return cudaGetLastError();
}

cudaError_t launch_driver_check(const DriverIn &D, int64_t n_reads, int64_t n_seeds, int match, uint32_t *runs,
                                DriverCheck *X, cudaStream_t st, int sms)
{
    if (n_reads > 0) k_check_reads<<<grid_for(n_reads, 256, sms), 256, 0, st>>>(D, n_reads, X);
    if (n_seeds > 0) k_check_seeds<<<grid_for(n_seeds, 256, sms), 256, 0, st>>>(D, n_reads, n_seeds, match, runs, X);
    return cudaGetLastError();
}

cudaError_t launch_filter(const DriverIn &D, int64_t n, bsw_aln_t *out, cudaStream_t st, int sms)
{
    k_filter<<<grid_for(n, 256, sms), 256, 0, st>>>(D, n, out);
    return cudaGetLastError();
}

}  // namespace bsw
