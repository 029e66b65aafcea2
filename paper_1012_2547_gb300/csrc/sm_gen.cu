// Device twin of the seeded input generator, and a tiny helper kernel that
// zeroes the counts of queries without work items.  Neither is part of the
// matching method.
#include "sm_internal.h"

namespace smgpu {

namespace {

// splitmix64 output function (Steele, Lea and Flood, OOPSLA 2014).
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void gen_kernel(uint8_t *out, uint64_t start, uint64_t count, uint64_t key,
                           uint32_t sigma, const uint32_t *thr, uint32_t nthr,
                           const uint8_t *bmap) {
    __shared__ uint32_t s_thr[256];
    __shared__ uint8_t s_map[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
        s_thr[i] = (thr && i < static_cast<int>(nthr)) ? thr[i] : 0xFFFFFFFFu;
        s_map[i] = bmap ? bmap[i] : static_cast<uint8_t>(i);
    }
    __syncthreads();
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < count;
         i += stride) {
        const uint64_t r = mix64(key + (start + i + 1) * 0x9E3779B97F4A7C15ull);
        const uint64_t u = r >> 32;
        uint32_t sym;
        if (sigma) {
            sym = static_cast<uint32_t>((u * sigma) >> 32);
        } else {
            sym = 0;
            for (uint32_t k = 0; k < nthr; ++k) sym += u >= s_thr[k];
        }
        out[i] = s_map[sym & 255u];
    }
}

__global__ void zero_counts_kernel(uint64_t *const *ptrs, uint32_t count) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) *ptrs[i] = 0ull;
}

}  // namespace

cudaError_t launch_gen_text(uint8_t *out, uint64_t start, uint64_t count, uint64_t key,
                            uint32_t sigma, const uint32_t *thresholds, uint32_t nthr,
                            const uint8_t *byte_map, cudaStream_t stream) {
    if (count == 0) return cudaSuccess;
    const uint64_t want = (count + 255) / 256;
    const int grid = static_cast<int>(want < 65536 ? want : 65536);
    gen_kernel<<<grid, 256, 0, stream>>>(out, start, count, key, sigma, thresholds, nthr, byte_map);
    return cudaGetLastError();
}

cudaError_t launch_zero_counts(uint64_t *const *ptrs, uint32_t count, cudaStream_t stream) {
    if (count == 0) return cudaSuccess;
    zero_counts_kernel<<<(count + 255) / 256, 256, 0, stream>>>(ptrs, count);
    return cudaGetLastError();
}

}  // namespace smgpu
