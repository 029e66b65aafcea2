// Internal interface between the host API (sm_api.cu) and the kernel
// translation units.  Not part of the public C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sm_common.cuh"

namespace smgpu {

// Kernel ids.  Every plan maps to exactly one of them.  The bit-parallel
// kernels differ in state width (32/64 bits), mask-table entry width (1, 2,
// 4 or 8 bytes) and how match flags are read ("H": 16 flags kept above bit
// m-1 of the state; "A": accumulator plus rescan of flagged chunks).
enum KernelId : int {
    K_SO8H = 0,   // 32-bit state, byte masks, m = 7..8 (m <= 8 where asked by id)
    K_SO16H = 1,  // 32-bit state, half-word masks, m <= 16
    K_SO32H = 2,  // 32-bit state, word masks, m <= 17
    K_SO32A = 3,  // 32-bit state, word masks, m <= 32
    K_SO64H = 4,  // 64-bit state, m <= 49
    K_SO64A = 5,  // 64-bit state, m <= 64
    K_QGRAM = 6,  // exact q-gram stride filter + warp verification
    K_LINEAR = 7, // per-segment Knuth-Morris-Pratt
    K_SOMULTI = 8, // several Shift-And patterns (m <= 16) of one text in one state (batches only)
    K_DFA = 9,     // per-segment string-matching automaton, table in shared memory
    K_SO6P = 10,   // 32-bit state, byte masks, two text bytes per step, m = 5..6 (m <= 6 by id)
    K_SO4Q = 11,   // 32-bit state, byte masks, four text bytes per step, m <= 4
    K_COUNT = 12
};

// The bit-parallel kernels (staged sub-tiles, one-warp blocks).  Patterns
// of m <= 4, 5..6 and 7..8 have kernels of their own (four-, two- and
// one-byte steps), so a launch holds one scan loop's code, not several.
inline bool so_kid(int kid) { return kid <= K_SO64A || kid == K_SO6P || kid == K_SO4Q; }
// Kernels that stage sub-tiles and use the per-block spill area.
inline bool staged_kid(int kid) { return so_kid(kid) || kid == K_SOMULTI; }
inline uint32_t so_entry_bytes(int kid) {
    return kid == K_SO8H || kid == K_SO6P || kid == K_SO4Q ? 1u : kid == K_SO16H ? 2u : (kid <= K_SO32A ? 4u : 8u);
}
inline uint32_t so_word_bits(int kid) { return kid <= K_SO32A || kid == K_SO6P || kid == K_SO4Q ? 32u : 64u; }
inline bool so_hist(int kid) { return kid != K_SO32A && kid != K_SO64A; }
// Bit-parallel kernel for length m and state width wb (0 = choose), or -1.
inline int so_kid_for(uint32_t m, uint32_t wb) {
    if (wb == 0) wb = m <= 32 ? 32u : 64u;
    if (wb == 32)
        return m <= 4 ? K_SO4Q : m <= 6 ? K_SO6P : m <= 8 ? K_SO8H : m <= 16 ? K_SO16H : m <= 17 ? K_SO32H : m <= 32 ? K_SO32A : -1;
    if (wb == 64) return m <= 49 ? K_SO64H : m <= 64 ? K_SO64A : -1;
    return -1;
}

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

// Adds k to the library's kernel-launch counter (sm_kernel_launches).
void count_launches(uint64_t k);

// Persistent launch of kernel `kid` over `a` with `grid` blocks.
cudaError_t kernel_launch(int kid, const LaunchArgs &a, int grid, cudaStream_t stream);

// Writes 0 to each count of `ptrs` (queries that have no work item).
cudaError_t launch_zero_counts(uint64_t *const *ptrs, uint32_t count, cudaStream_t stream);

// Device text generator (sm_gen_text).
cudaError_t launch_gen_text(uint8_t *out, uint64_t start, uint64_t count, uint64_t key,
                            uint32_t sigma, const uint32_t *thresholds, uint32_t nthr,
                            const uint8_t *byte_map, cudaStream_t stream);

}  // namespace smgpu
