// bsw_noalloc.cu - bsw_extend_batch_noalloc: the batched extension without any
// allocation, for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they extend seeds: code
// running under an allocator that forbids it (a pool that owns all device
// memory, a stream-ordered allocator in the middle of a graph capture it
// controls), or a host library linked into a process whose memory is managed
// elsewhere.  For them this entry point takes its work buffers from one
// file-scope device array instead of a context's arena.  It runs the same
// bucketing and per-thread extension kernels as bsw_extend_batch, all on the
// caller's stream.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "bsw.h"
#include "bsw_device.cuh"
#include "bsw_launch.h"

using namespace bsw;

namespace {

constexpr int64_t kNaMaxPairs = BSW_NOALLOC_MAX_PAIRS;
constexpr int kNaMaxQlen = BSW_NOALLOC_MAX_QLEN;
constexpr int kNaWarpBlocks = 304;                     // 2432 warps of slot scratch
constexpr int64_t kNaSlotBytes = ((kNaMaxQlen + 1 + 32 * 8) * 8 + 255) / 256 * 256;

constexpr size_t al(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t kOffKey = 0;
constexpr size_t kOffOrder = kOffKey + al(4 * kNaMaxPairs);
constexpr size_t kOffRerun = kOffOrder + al(4 * kNaMaxPairs);
constexpr size_t kOffHist = kOffRerun + al(4 * kNaMaxPairs);
constexpr size_t kOffCursor = kOffHist + al(4 * kNumBins);
constexpr size_t kOffClsStart = kOffCursor + al(4 * kNumBins);
constexpr size_t kOffClsCount = kOffClsStart + al(4 * (kNumClass + 1));
constexpr size_t kOffClsNext = kOffClsCount + al(4 * (kNumClass + 1));
constexpr size_t kOffCells = kOffClsNext + al(4 * kNumCounters);
constexpr size_t kOffStatus = kOffCells + al(8);
constexpr size_t kOffSlots = kOffStatus + al(4);
constexpr size_t kNaBytes = kOffSlots + (size_t)kNaSlotBytes * kNaWarpBlocks * (kWarpKernelThreads / 32);
static_assert(kNaBytes <= BSW_NOALLOC_SCRATCH_BYTES, "scratch layout exceeds the stated size");

// The scratch every call uses.  Held by each GPU that loads the library until
// the process exits; its contents persist from one call to the next.
static __device__ __align__(256) uint8_t g_scratch[BSW_NOALLOC_SCRATCH_BYTES];

struct DeviceSetup {
    bool done = false;
    uint8_t *scratch = nullptr;   // device address of g_scratch on that device
    int sms = 0;
};

std::mutex g_setup_lock;
DeviceSetup g_setup[64];

// Once per device, with that device current: the array's device address (in
// host code the symbol is only a host-side stand-in), SM count, kernel
// attributes.  A device counts as set up only when every step succeeded; a
// failed set-up (for example a first call made during a stream capture)
// records nothing and is tried again by the next call.
int setup_device(int dev, DeviceSetup **out)
{
    if (dev < 0 || dev >= 64) return BSW_EINVAL;
    std::lock_guard<std::mutex> lk(g_setup_lock);
    DeviceSetup &s = g_setup[dev];
    if (!s.done) {
        void *p = nullptr;
        int sms = 0;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            prepare_kernels(sms) != cudaSuccess) {
            cudaGetLastError();
            return BSW_ECUDA;
        }
        s.scratch = (uint8_t *)p;
        s.sms = sms;
        s.done = true;
    }
    *out = &s;
    return BSW_OK;
}

}  // namespace

extern "C" int bsw_extend_batch_noalloc(const bsw_scoring_t *sc, int32_t w, int32_t zdrop, int32_t end_bonus,
                                        const bsw_batch_t *b, bsw_result_t *out, int64_t *cells_out,
                                        void *cuda_stream)
{
    if (!sc || !b || w < 0 || end_bonus < 0) return BSW_EINVAL;
    if (sc->match <= 0 || sc->match > 127 || sc->mismatch <= 0 || sc->mismatch > 128 || sc->o_del < 0 ||
        sc->o_ins < 0 || sc->e_del <= 0 || sc->e_ins <= 0 || sc->o_del > (1 << 20) || sc->o_ins > (1 << 20) ||
        sc->e_del > (1 << 20) || sc->e_ins > (1 << 20) || end_bonus > (1 << 20))
        return BSW_EINVAL;
    const uint32_t allowed = BSW_DEVICE_PTRS | BSW_FORCE_I8 | BSW_FORCE_I16 | BSW_FORCE_I32;
    if (!(b->flags & BSW_DEVICE_PTRS) || (b->flags & ~allowed)) return BSW_EINVAL;
    const uint32_t forced = b->flags & (BSW_FORCE_I8 | BSW_FORCE_I16 | BSW_FORCE_I32);
    if (forced & (forced - 1)) return BSW_EINVAL;
    if (b->n_pairs < 0 || b->n_pairs > kNaMaxPairs) return BSW_EINVAL;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (b->n_pairs == 0) {
        if (cells_out && cudaMemsetAsync(cells_out, 0, 8, st) != cudaSuccess) { cudaGetLastError(); return BSW_ECUDA; }
        return BSW_OK;
    }
    if (!b->q || !b->q_off || !b->q_len || !b->t || !b->t_off || !b->t_len || !b->h0 || !out) return BSW_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return BSW_ECUDA; }
    DeviceSetup *s = nullptr;
    int rc = setup_device(dev, &s);
    if (rc != BSW_OK) return rc;

    uint8_t *base = s->scratch;
    Work W;
    W.key = (int32_t *)(base + kOffKey);
    W.order = (int32_t *)(base + kOffOrder);
    W.rec = nullptr;   // the class kernels gather the pairs' fields from the batch
    W.rerun = (int32_t *)(base + kOffRerun);
    W.hist = (uint32_t *)(base + kOffHist);
    W.cursor = (uint32_t *)(base + kOffCursor);
    W.cls_start = (int32_t *)(base + kOffClsStart);
    W.cls_count = (int32_t *)(base + kOffClsCount);
    W.cls_next = (uint32_t *)(base + kOffClsNext);
    W.cells = cells_out ? (unsigned long long *)cells_out : (unsigned long long *)(base + kOffCells);
    W.status = (uint32_t *)(base + kOffStatus);
    W.slots = base + kOffSlots;
    W.slot_bytes_per_warp = kNaSlotBytes;

    Params P{sc->match, sc->mismatch, sc->o_del, sc->e_del, sc->o_ins, sc->e_ins, w, zdrop, end_bonus, b->flags,
             kNaMaxQlen, 1u << 8, 1u << 16, 1u << 24, kShortMax};
    Batch B{b->n_pairs, b->q, b->q_off, b->q_len, b->t, b->t_off, b->t_len, b->h0, b->w_override, out,
            b->q_n, b->t_n};
    // The histogram, the cell count and the status word must start at zero;
    // the array keeps whatever the previous call left.
    if (cudaMemsetAsync(W.hist, 0, 4 * kNumBins, st) != cudaSuccess || cudaMemsetAsync(W.cells, 0, 8, st) != cudaSuccess ||
        cudaMemsetAsync(W.status, 0, 4, st) != cudaSuccess) {
        cudaGetLastError();
        return BSW_ECUDA;
    }
    if (launch_batched_serial(B, P, W, st, s->sms, kNaWarpBlocks, default_plan()) != cudaSuccess) {
        cudaGetLastError();
        return BSW_ECUDA;
    }
    uint32_t status = 0;
    if (cudaMemcpyAsync(&status, W.status, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return BSW_ECUDA;
    }
    return status ? BSW_EINVAL : BSW_OK;
}
