// int_rates.cu - issue rate of the integer instructions the BSW cell loop uses.
//
// The extension is bound by integer issue, not by HBM or tensor cores, so its
// roofline is SMs x clock x (lane-ops per clock per SM) / (ops per cell).  This
// program measures lane-ops per clock per SM for each instruction kind on the
// running GPU: one block of 1024 threads per SM, eight dependent chains per
// thread that feed each other (so nothing folds), SM cycles from clock64().
// Output: one JSON object per line.  It is a measurement program, not part of
// the library; build it with
//   nvcc -O3 -gencode arch=compute_103a,code=sm_103a -o _build/int_rates int_rates.cu
#include <cuda_runtime.h>
#include <cstdio>
#include <vector>

#define CHAIN8(OP)                      \
    x0 = OP(x0, x1, x2);                \
    x1 = OP(x1, x2, x3);                \
    x2 = OP(x2, x3, x4);                \
    x3 = OP(x3, x4, x5);                \
    x4 = OP(x4, x5, x6);                \
    x5 = OP(x5, x6, x7);                \
    x6 = OP(x6, x7, x0);                \
    x7 = OP(x7, x0, x1);

__device__ __forceinline__ unsigned prmt_(unsigned a, unsigned b, unsigned s)
{
    unsigned d;
    asm volatile("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(s));
    return d;
}

#define OP_IADD(a, b, c) ((a) + (b))
#define OP_IADD3(a, b, c) ((a) + (b) + (c))
#define OP_MAX(a, b, c) max((a), (b))
#define OP_MAX3(a, b, c) __vimax3_s32((a), (b), (c))
#define OP_ADDMAX(a, b, c) __viaddmax_s32((a), (b), (c))
#define OP_ADDMAXRELU(a, b, c) __viaddmax_s32_relu((a), (b), (c))
#define OP_ADDMIN(a, b, c) __viaddmin_s32((a), (b), (c))
#define OP_IMAD(a, b, c) ((a) * (b) + (c))
#define OP_PRMT(a, b, c) (int)prmt_((unsigned)(a), (unsigned)(b), (unsigned)(c) & 0x7777u)
#define OP_SHR(a, b, c) (int)((unsigned)(a) >> ((b) & 31))
#define OP_LOP3(a, b, c) (((a) & (b)) ^ (c))
#define OP_MAX_S16X2(a, b, c) (int)__vimax_s16x2_relu((unsigned)(a), (unsigned)(b))
#define OP_ADDMAX_S16X2(a, b, c) (int)__viaddmax_s16x2((unsigned)(a), (unsigned)(b), (unsigned)(c))
#define OP_MAX3_S16X2(a, b, c) (int)__vimax3_s16x2((unsigned)(a), (unsigned)(b), (unsigned)(c))
#define OP_SEL(a, b, c) ((a) > (c) ? (b) : (c))

#define KERNEL(NAME, OP)                                                                         \
    __global__ void __launch_bounds__(1024) k_##NAME(int iters, int seed, int *out, long long *cyc) \
    {                                                                                            \
        int x0 = seed + threadIdx.x, x1 = seed ^ 0x55, x2 = seed * 3, x3 = seed + 7;            \
        int x4 = seed - threadIdx.x, x5 = seed ^ 0x3c3c, x6 = seed + 11, x7 = seed * 5;         \
        __syncthreads();                                                                         \
        long long t0 = clock64();                                                                \
        for (int it = 0; it < iters; ++it) {                                                     \
            _Pragma("unroll") for (int u = 0; u < 8; ++u) { CHAIN8(OP) }                         \
        }                                                                                        \
        __syncthreads();                                                                         \
        long long t1 = clock64();                                                                \
        out[blockIdx.x * blockDim.x + threadIdx.x] = x0 ^ x1 ^ x2 ^ x3 ^ x4 ^ x5 ^ x6 ^ x7;     \
        if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;                                         \
    }

KERNEL(iadd, OP_IADD)
KERNEL(iadd3, OP_IADD3)
KERNEL(imax, OP_MAX)
KERNEL(vimax3, OP_MAX3)
KERNEL(viaddmax, OP_ADDMAX)
KERNEL(viaddmax_relu, OP_ADDMAXRELU)
KERNEL(viaddmin, OP_ADDMIN)
KERNEL(imad, OP_IMAD)
KERNEL(prmt, OP_PRMT)
KERNEL(shr, OP_SHR)
KERNEL(lop3, OP_LOP3)
KERNEL(sel, OP_SEL)
KERNEL(vimax_s16x2_relu, OP_MAX_S16X2)
KERNEL(viaddmax_s16x2, OP_ADDMAX_S16X2)
KERNEL(vimax3_s16x2, OP_MAX3_S16X2)

typedef void (*kfn)(int, int, int *, long long *);

int main()
{
    int sms = 0, clk = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, 0);
    struct { const char *name; kfn f; int ops_per_chain_step; } ks[] = {
        {"iadd", k_iadd, 1}, {"iadd3", k_iadd3, 1}, {"imnmx", k_imax, 1}, {"vimax3_s32", k_vimax3, 1},
        {"viaddmax_s32", k_viaddmax, 1}, {"viaddmax_s32_relu", k_viaddmax_relu, 1}, {"viaddmin_s32", k_viaddmin, 1},
        {"imad", k_imad, 1}, {"prmt", k_prmt, 1}, {"shf", k_shr, 1}, {"lop3", k_lop3, 1}, {"isetp+sel", k_sel, 1},
        {"vimax_s16x2_relu", k_vimax_s16x2_relu, 1}, {"viaddmax_s16x2", k_viaddmax_s16x2, 1},
        {"vimax3_s16x2", k_vimax3_s16x2, 1}};
    const int threads = 1024, iters = 4096;
    int *out = nullptr;
    long long *cyc = nullptr;
    if (cudaMalloc(&out, sizeof(int) * sms * threads) != cudaSuccess) return 1;
    if (cudaMalloc(&cyc, sizeof(long long) * sms) != cudaSuccess) return 1;
    std::vector<long long> h(sms);
    printf("{\"sms\": %d, \"clock_khz_attr\": %d}\n", sms, clk);
    for (auto &k : ks) {
        for (int rep = 0; rep < 2; ++rep) {   // first pass warms up
            k.f<<<sms, threads>>>(iters, 12345, out, cyc);
            if (cudaDeviceSynchronize() != cudaSuccess) { printf("{\"error\": \"%s\"}\n", k.name); return 1; }
        }
        cudaMemcpy(h.data(), cyc, sizeof(long long) * sms, cudaMemcpyDeviceToHost);
        double mean = 0;
        for (long long c : h) mean += (double)c;
        mean /= sms;
        const double lane_ops = (double)threads * iters * 8.0 * 8.0 * k.ops_per_chain_step;
        printf("{\"op\": \"%s\", \"lane_ops_per_clk_per_sm\": %.2f, \"cycles\": %.0f}\n", k.name, lane_ops / mean, mean);
    }
    cudaFree(out);
    cudaFree(cyc);
    return 0;
}
