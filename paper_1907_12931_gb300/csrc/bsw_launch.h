// bsw_launch.h - host-side entry points into the BSW kernels.
#pragma once

#include <cuda_runtime.h>
#include "bsw_device.cuh"

namespace bsw {

// Warp-per-pair kernels: 8 warps per block, 2 blocks per SM.
constexpr int kWarpKernelThreads = 256;
constexpr int kWarpBlocksPerSM = 2;

struct Streams {
    cudaStream_t main;
    cudaStream_t side[3];
    cudaEvent_t fork;
    cudaEvent_t join[3];
};

// Kernel attributes and occupancy; call once per device before any launch
// (and before any stream capture).
cudaError_t prepare_kernels(int sms);

// Number of per-warp slot regions the warp-per-pair kernels use.
int warp_slots_needed(int sms);

// Length-bucketed batched path: classify + counting sort + per-class
// persistent kernels (forked over the side streams) + 32-bit re-run.
// W.hist must be zero on entry (k_scan leaves it zero); W.cells and W.status
// accumulate.
cudaError_t launch_batched(const Batch &B, const Params &P, const Work &W, const Streams &S, int sms);

// The same path on one stream (no side streams, no events); the warp-per-pair
// kernels use warp_blocks blocks of kWarpKernelThreads threads.
cudaError_t launch_batched_serial(const Batch &B, const Params &P, const Work &W, cudaStream_t st, int sms,
                                  int warp_blocks);

// Baseline: one pair per warp in input order.
cudaError_t launch_plain(const Batch &B, const Params &P, const Work &W, cudaStream_t st, int sms);

}  // namespace bsw
