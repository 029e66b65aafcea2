// Internal interface between the host API (sm_api.cu) and the kernel
// translation units.  Not part of the public C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sm_common.cuh"

namespace smgpu {

// Kernel ids.  Every plan maps to exactly one of them.
enum KernelId : int {
    K_SO32H = 0,  // Shift-And, 32-bit state, 16 match flags kept (m <= 17)
    K_SO32A = 1,  // Shift-And, 32-bit state, per-chunk accumulator (m <= 32)
    K_SO64H = 2,  // Shift-And, 64-bit state, 16 match flags kept (m <= 49)
    K_SO64A = 3,  // Shift-And, 64-bit state, accumulator (m <= 64)
    K_QGRAM = 4,  // exact q-gram stride filter + warp verification
    K_LINEAR = 5, // per-segment Knuth-Morris-Pratt
    K_COUNT = 6
};

struct KernelShape {
    const void *fn;
    int threads;
    size_t smem;
    int blocks_per_sm;  // filled by kernels_init
};

// Fill shapes (sets shared-memory attributes, queries occupancy).  Must run
// once per device before the first launch.
cudaError_t kernels_init(int sms);
const KernelShape &kernel_shape(int kid);

// Start positions covered by one work item of kernel `kid` for plan `hdr`.
uint64_t kernel_tile_starts(int kid, const PlanDev &hdr);

// Work units of a query (0 when m > n): staged sub-tiles for the
// bit-parallel kernels, base ranges (tile_starts positions) otherwise.
uint64_t kernel_ntiles(int kid, const PlanDev &hdr, const uint8_t *text, uint64_t n);

// Persistent launch of kernel `kid` over `a` with `grid` blocks.
cudaError_t kernel_launch(int kid, const LaunchArgs &a, int grid, cudaStream_t stream);

// Writes 0 to each count of `ptrs` (queries that have no work item).
cudaError_t launch_zero_counts(uint64_t *const *ptrs, uint32_t count, cudaStream_t stream);

// Device text generator (sm_gen_text).
cudaError_t launch_gen_text(uint8_t *out, uint64_t start, uint64_t count, uint64_t key,
                            uint32_t sigma, const uint32_t *thresholds, uint32_t nthr,
                            const uint8_t *byte_map, cudaStream_t stream);

}  // namespace smgpu
