// bsw_sal.cu - suffix array lookup (Section IV-D, Eq. 1: j = S[i]).
//
// With the suffix array kept uncompressed in HBM, the reference coordinates
// of an SA interval [k, k + cnt) are S[k], ..., S[k + cnt - 1]: one read per
// position.  Each warp takes 32 intervals at a time: the lanes load the 32
// intervals' k, count and output offset with coalesced loads, every lane
// copies its own interval if it has at most 32 positions (32 independent
// random reads of S in flight per warp, which the latency of HBM needs), and
// the whole warp copies each longer interval together, 32 positions per step.
// Bound: HBM latency and bandwidth.
#include <cuda_runtime.h>
#include <cstdint>

#include "bsw_launch.h"

namespace bsw {

namespace {

__global__ void __launch_bounds__(256) k_sal(const int32_t *__restrict__ sa, int64_t sa_n,
                                             const int64_t *__restrict__ k, const int32_t *__restrict__ cnt,
                                             const int64_t *__restrict__ off, int64_t n_int,
                                             int32_t *__restrict__ out, uint32_t *status)
{
    constexpr unsigned kAll = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t base = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; base < n_int;
         base += nw * 32) {
        const int64_t t = base + lane;
        int64_t k0 = 0, o = 0;
        int c = 0;
        bool ok = false;
        if (t < n_int) {
            k0 = k[t];
            c = cnt[t];
            o = off[t];
            ok = k0 >= 0 && c >= 0 && k0 + c <= sa_n;
            if (!ok) atomicOr(status, kStInval);
        }
        if (ok && c <= 32) {
#pragma unroll 4
            for (int i = 0; i < c; ++i) out[o + i] = __ldg(sa + k0 + i);
        }
        unsigned longs = __ballot_sync(kAll, ok && c > 32);
        while (longs) {
            const int src = __ffs(longs) - 1;
            longs &= longs - 1;
            const int64_t kk = __shfl_sync(kAll, k0, src), oo = __shfl_sync(kAll, o, src);
            const int cc = __shfl_sync(kAll, c, src);
            for (int i = lane; i < cc; i += 32) out[oo + i] = __ldg(sa + kk + i);
        }
    }
}

}  // namespace

cudaError_t launch_sal(const int32_t *sa, int64_t sa_n, const int64_t *k, const int32_t *cnt, const int64_t *off,
                       int64_t n_int, int32_t *out, uint32_t *status, cudaStream_t st, int sms)
{
    if (n_int <= 0) return cudaSuccess;
    const int64_t want = (n_int + 255) / 256;             // 8 warps of 32 intervals per block
    const int blocks = (int)(want < (int64_t)sms * 16 ? want : (int64_t)sms * 16);
    k_sal<<<blocks, 256, 0, st>>>(sa, sa_n, k, cnt, off, n_int, out, status);
    return cudaGetLastError();
}

}  // namespace bsw
