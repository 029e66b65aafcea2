/*
 * smgen.h - device twin of the seeded text generator used by the tests and
 * the benchmark to build large synthetic texts directly in device memory.
 * It is not part of the matching method (the paper has no counterpart); it
 * exists so that an 8 GiB text need not cross PCIe/C2C.
 *
 * Byte i (i = start .. start+count-1) is
 *     r   = splitmix64_mix(key + (i + 1) * 0x9E3779B97F4A7C15)
 *     u   = r >> 32
 *     sym = sigma ? (u * sigma) >> 32                      (uniform)
 *                 : #{k < nthr : thresholds[k] <= u}       (skewed)
 *     out[i - start] = byte_map ? byte_map[sym] : sym
 * where splitmix64_mix is the splitmix64 output function (Steele, Lea and
 * Flood, OOPSLA 2014).  The host module paper_1012_2547_gb300/gen.py
 * implements the same definition.
 *
 * out       : device pointer to `count` bytes (any alignment).
 * thresholds: device pointer to nthr ascending uint32 thresholds, or NULL
 *             when sigma != 0.  nthr <= 255.
 * byte_map  : device pointer to 256 bytes, or NULL for the identity.
 * Enqueued on `stream`; returns SM_EINVAL for bad arguments.
 */
#ifndef SMGEN_H
#define SMGEN_H

#include <stdint.h>

#include "smgpu.h"

#ifdef __cplusplus
extern "C" {
#endif

sm_status sm_gen_text(uint8_t *out, uint64_t start, uint64_t count, uint64_t key, uint32_t sigma,
                      const uint32_t *thresholds, uint32_t nthr, const uint8_t *byte_map,
                      sm_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* SMGEN_H */
