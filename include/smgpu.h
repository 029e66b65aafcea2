/*
 * smgpu.h - C ABI of the GB300 exact string matching library (libsmgpu.so).
 *
 * The operation (Faro & Lecroq, Section 1, problem statement): for a text t
 * of n bytes and a pattern p of m bytes, report ALL occurrences of p in t,
 * i.e. every 0-based start position i in [0, n-m] with t[i..i+m-1] = p,
 * overlapping occurrences included, as strictly increasing uint64 values.
 * Symbols are arbitrary bytes 0..255; the alphabet size sigma is only a
 * tuning hint.  This is the online setting the paper studies (Section 1):
 * the pattern is preprocessed (sm_prepare), the text is not indexed.
 *
 * Memory and ownership
 *   - `text`, `out_pos` and `out_count` are DEVICE pointers owned by the
 *     caller (e.g. torch tensors).  `pattern` is a HOST pointer; it is only
 *     read during the call.  `sm_query` arrays are HOST arrays read during
 *     the call.
 *   - Plans (sm_plan) and batches (sm_batch) are owned by the library and
 *     released with sm_plan_free / sm_batch_free.  Per-stream workspace
 *     (look-back state, claim counters) is owned by the library and kept
 *     until sm_shutdown().
 *   - `text` may have any alignment.  The kernels may read the bytes of the
 *     16-byte-aligned blocks that hold t[0] and t[n-1]; those bytes never
 *     influence a result.  `out_pos` and `out_count` must be 8-byte aligned.
 *
 * Asynchrony
 *   - Every search is enqueued on `stream` (a cudaStream_t; NULL is the
 *     legacy default stream) and returns before the GPU work ends.
 *     *out_count is written on the device: it holds the TOTAL number of
 *     occurrences even when that exceeds `cap`; the first min(total, cap)
 *     positions are written to out_pos.  Truncation is not an error at this
 *     level; higher layers report it (SM_ETRUNC) after reading the count.
 *   - Device-side waits are bounded.  A wait that runs out sets a device
 *     error word; sm_sync() reports it as SM_ETIMEOUT and the stream stays
 *     usable.
 *
 * Errors: argument errors are detected on the host before any launch and
 * return SM_EINVAL without enqueuing work; CUDA runtime failures return
 * SM_ECUDA; failed allocations SM_ENOMEM.
 */
#ifndef SMGPU_H
#define SMGPU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same object as cudaStream_t; declared here so callers need no CUDA header. */
typedef struct CUstream_st *sm_stream_t;

typedef enum {
    SM_OK = 0,
    SM_EINVAL = 1,   /* bad argument: null pointer, m = 0, misaligned output... */
    SM_ENOMEM = 2,   /* device or host allocation failed */
    SM_ECUDA = 3,    /* a CUDA runtime call failed (no device, launch error) */
    SM_ETIMEOUT = 4, /* a bounded device-side wait ran out (see sm_sync) */
    SM_ETRUNC = 5    /* more occurrences than `cap` (reported by sync wrappers) */
} sm_status;

/* Kernel families.  All compute the same set; they differ in speed. */
typedef enum {
    SM_VARIANT_AUTO = 0,     /* tuning table, else built-in rule */
    SM_VARIANT_SHIFTOR = 1,  /* bit-parallel Shift-And/Shift-Or, m <= 64 */
    SM_VARIANT_QGRAM = 2,    /* exact q-gram stride filter + warp verify */
    SM_VARIANT_LINEAR = 3,   /* per-segment Knuth-Morris-Pratt (dense fallback) */
    SM_VARIANT_DFA = 4       /* per-segment string-matching automaton (the
                              * AUT/DFA algorithm of Figs. 1-3): one table
                              * step per text byte whatever m and the hit
                              * density.  Needs (m+1) x C x 2 <= 32,512 bytes
                              * of table, C = distinct bytes of p + 1; an
                              * explicit config that exceeds it is SM_EINVAL */
} sm_variant;

typedef struct sm_plan sm_plan;   /* opaque, library-owned */
typedef struct sm_batch sm_batch; /* opaque, library-owned */

/*
 * Explicit plan configuration (sm_prepare_ex).  Zero fields mean "choose".
 *   variant  : sm_variant.
 *   q        : q-gram length for SM_VARIANT_QGRAM, 1..8 and <= m.
 *   word_bits: Shift-Or state width, 32 or 64 (m <= 32 or m <= 64).
 *   tile     : log2 hint of the work-item size.  QGRAM/LINEAR/DFA: bytes
 *              of start positions per thread range.  SHIFTOR (whose staged
 *              sub-tile is fixed at 4,608 end positions): the shortest work
 *              item in bytes, rounded up to whole sub-tiles and capped at 64
 *              of them; 0 lets the launch size items from the grid alone.
 */
typedef struct {
    uint32_t variant;
    uint32_t q;
    uint32_t word_bits;
    uint32_t tile;
} sm_config;

/* Read-only description of a plan (sm_plan_info). */
typedef struct {
    uint32_t m;
    uint32_t variant;     /* resolved sm_variant (never AUTO) */
    uint32_t q;           /* q-gram length (QGRAM), else 0 */
    uint32_t word_bits;   /* Shift-Or width (SHIFTOR), else 0 */
    uint32_t hist;        /* 1 if the Shift-Or state carries 16 match flags */
    uint32_t tile_starts; /* start positions per work item */
    uint64_t device_bytes;/* size of the plan's device tables */
    uint32_t kernel;      /* internal kernel id (0..11): batches run one launch per id */
    uint32_t reserved;
} sm_plan_desc;

/*
 * sm_prepare - preprocess a pattern (paper Section 1: online matching
 * preprocesses the pattern only).  Builds, on the host, the tables of the
 * chosen kernel family and copies them to device memory on `stream`:
 *   - Shift-Or masks: bit j of B[c] is 1 iff p[j] = c (the one-bit-per-
 *     pattern-symbol encoding of the bit-parallel algorithms, Section 1);
 *   - for long patterns, the exact q-gram table of p (the Hash-q idea of
 *     Fig. 1 with q-grams compared exactly, never by hash alone);
 *   - the Knuth-Morris-Pratt border table for the linear fallback;
 *   - the string-matching automaton of p over its byte classes, for DFA
 *     plans and for q-gram plans of periodic patterns (smallest period
 *     <= m/2, table within the DFA limit), whose dense work items then run
 *     the automaton instead of Knuth-Morris-Pratt.
 * pattern    : host pointer to m bytes.  m >= 1 (m = 0 -> SM_EINVAL).
 * sigma_hint : expected alphabet size of the texts (0 = unknown); only
 *              changes the kernel choice and q, never the result.
 * out_plan   : receives a library-owned plan; free with sm_plan_free.
 * The plan is usable by work enqueued on any stream after this call returns
 * (the copy is synchronous with respect to the host).
 */
sm_status sm_prepare(const uint8_t *pattern, uint32_t m, uint32_t sigma_hint,
                     sm_stream_t stream, sm_plan **out_plan);

/* sm_prepare with an explicit configuration (tests, autotuner).  A config
 * that cannot serve the pattern (e.g. SHIFTOR with m > 64, q > m) returns
 * SM_EINVAL. */
sm_status sm_prepare_ex(const uint8_t *pattern, uint32_t m, uint32_t sigma_hint,
                        const sm_config *config, sm_stream_t stream, sm_plan **out_plan);

/*
 * sm_prepare_many - preprocess `count` patterns in one call; the device
 * tables of all plans share one allocation and one host-to-device copy.
 * patterns : host pointer to the concatenated pattern bytes.
 * lengths  : host array of count lengths (each >= 1).
 * sigma_hint, config: as in sm_prepare_ex (config may be NULL = auto).
 * out_plans: host array of count plan pointers to fill.  Each plan must be
 *            freed with sm_plan_free; the shared allocation is released
 *            when the last of them is freed.
 */
sm_status sm_prepare_many(const uint8_t *patterns, const uint32_t *lengths, uint32_t count,
                          uint32_t sigma_hint, const sm_config *config, sm_stream_t stream,
                          sm_plan **out_plans);

/* Release a plan.  Work that uses it must have completed.  NULL is a no-op. */
sm_status sm_plan_free(sm_plan *plan);

/*
 * Release `count` plans (e.g. all plans of one sm_prepare_many call) in one
 * call, as sm_plan_free on each.  plans: host array of count plan pointers
 * (NULL entries are skipped); NULL with count > 0 -> SM_EINVAL.  Work that
 * uses any of them must have completed.
 */
sm_status sm_plan_free_many(sm_plan *const *plans, uint32_t count);

/* Describe a plan (host only, no GPU work). */
sm_status sm_plan_info(const sm_plan *plan, sm_plan_desc *out);

/*
 * Layout of a plan's device image (sm_plan_image).  Offsets are bytes from
 * the start of the image; an offset of 0 means the table is absent.
 *   masks      : 256 Shift-And masks of entry_bytes each (SHIFTOR plans),
 *                little-endian; bit j (j < m) of mask c is 1 iff p[j] = c,
 *                every bit >= m is 1 (Section 1's one-bit-per-symbol masks).
 *   pattern    : the m pattern bytes.
 *   border     : u32 fail[0..m], fail[q] = length of the longest proper
 *                border of p[0..q-1] (Knuth-Morris-Pratt, Fig. 1).
 *   qgram_*    : QGRAM plans.  slots: 1 << slot_bits entries of {u64 key
 *                (q-gram, byte 0 in bits 0..7), u32 first, u32 count}
 *                (count 0 = empty); offsets: u32, the offsets j of each key
 *                at [first, first + count) in decreasing order; slot of a
 *                key: (key * 0x9E3779B97F4A7C15) >> (64 - slot_bits), then
 *                linear probing; bitmap: 1 << bitmap_bits bits, bit
 *                h >> (32 - bitmap_bits) set for every key, with the 32-bit
 *                h = (lo * 0x9E3779B1) ^ (hi * 0x85EBCA77), lo and hi the
 *                key's low and high 32 bits.
 *   automaton  : DFA plans, and QGRAM plans of periodic patterns (smallest
 *                period <= m/2) whose table fits.  classes_tab: u16[256],
 *                2 x the class of each byte (class 0: bytes absent from p);
 *                automaton: u16[(m+1) x classes], the entry at byte offset
 *                r + classes_tab[c] for r = 2 x classes x q is
 *                2 x classes x delta(q, c), delta(q, c) = length of the
 *                longest prefix of p that is a suffix of p[0..q-1] c.
 */
typedef struct {
    uint32_t m;
    uint32_t variant;      /* resolved sm_variant */
    uint32_t kernel;       /* internal kernel id, as sm_plan_desc */
    uint32_t bytes;        /* image size */
    uint32_t q, s;         /* q-gram length and probe stride m - q + 1 */
    uint32_t word_bits, hist, entry_bytes;
    uint32_t tile_starts;  /* start positions per work unit */
    uint32_t off_masks, off_pattern, off_border;
    uint32_t off_qgram_bitmap, bitmap_bits, off_qgram_slots, slot_bits, off_qgram_offsets;
    uint32_t off_classes_tab, off_automaton, classes;
    uint32_t reserved;
} sm_plan_layout;

/*
 * sm_plan_image - build the device image of a plan in host memory, exactly
 * the bytes sm_prepare_ex would upload for (pattern, sigma_hint, config),
 * without any CUDA call (plan inspection, tests, caching plans).
 * image    : host buffer of `capacity` bytes, or NULL to ask only for the
 *            layout (layout->bytes is the size needed).
 * layout   : receives the layout; required.
 * Errors: SM_EINVAL for the arguments sm_prepare_ex rejects, a null layout,
 * or capacity < layout->bytes with a non-null image (nothing is copied).
 */
sm_status sm_plan_image(const uint8_t *pattern, uint32_t m, uint32_t sigma_hint,
                        const sm_config *config, void *image, size_t capacity,
                        sm_plan_layout *layout);

/*
 * sm_search - all occurrences of pattern (host, m bytes) in text (device,
 * n bytes).  Plans are cached per pattern content, so repeated searches for
 * the same pattern skip preprocessing.
 *   out_pos  : device array of cap uint64 slots (may be NULL iff cap = 0).
 *   out_count: device uint64; receives the total count.
 * m > n is valid and yields a count of 0.
 */
sm_status sm_search(const uint8_t *text, uint64_t n, const uint8_t *pattern, uint32_t m,
                    uint64_t *out_pos, uint64_t cap, uint64_t *out_count, sm_stream_t stream);

/*
 * sm_search_noalloc - sm_search for patterns of up to 64 bytes that makes no
 * device allocation at all.  The paper has no counterpart.  It is for
 * callers that are not allowed to call cudaMalloc on their request path:
 * serving loops that reserve all device memory when they start (an
 * allocation later could fail or stall every stream while the allocator
 * synchronises), and plugins running inside a host framework that owns
 * every device byte through its own allocator.  Those callers pass inputs
 * and outputs only.
 *   m          : 1..64 (longer patterns -> SM_EINVAL).
 *   n          : at most 65536 * 64 * 4608 - 16 bytes (about 19 GB); a longer
 *                text -> SM_EINVAL, before any CUDA call.
 *   Other arguments as in sm_search.
 * The plan and the kernel's scratch (claim counter, error word, one
 * look-back word per work item; 4.25 KiB + 512 KiB) sit in one statically
 * sized device array that every GPU loading the library keeps until the
 * process exits.  The first call on a device looks up that array's address
 * with cudaGetSymbolAddress; make that first call before any stream
 * capture.  All calls share the array and it keeps the last call's
 * contents: each call rewrites the plan with a small kernel (the pattern
 * travels by value in its launch arguments) and clears what must start at
 * zero, on `stream`.  Calls whose GPU work overlaps (e.g. on two streams at
 * once) race on the array: order them on one stream.
 * Completion: *out_count is set to UINT64_MAX before the search and holds
 * the total once it completes.  A one-thread kernel enqueued after the
 * search sets it back to UINT64_MAX if any bounded device wait of the
 * search ran out (then out_pos may be incomplete), so once the stream is
 * idle a count of UINT64_MAX means "failed, retry" and any other value is
 * the exact total.  Each call adds 3 to sm_kernel_launches.
 */
sm_status sm_search_noalloc(const uint8_t *text, uint64_t n, const uint8_t *pattern, uint32_t m,
                            uint64_t *out_pos, uint64_t cap, uint64_t *out_count,
                            sm_stream_t stream);

/* sm_search with a prepared plan (no host preprocessing, no host sync). */
sm_status sm_search_plan(const sm_plan *plan, const uint8_t *text, uint64_t n,
                         uint64_t *out_pos, uint64_t cap, uint64_t *out_count,
                         sm_stream_t stream);

/* One (pattern, text) pair of a batch.  Pointers as in sm_search_plan. */
typedef struct {
    const uint8_t *text;
    uint64_t n;
    const sm_plan *plan;
    uint64_t *out_pos;
    uint64_t cap;
    uint64_t *out_count;
} sm_query;

/*
 * sm_search_batch - run nq independent searches.  Queries are grouped by
 * kernel family; each family runs as ONE persistent launch whose blocks claim
 * (query, tile) work items from a device counter, so thousands of uneven
 * queries share the GPU without one launch per query.  Equivalent to nq
 * sm_search_plan calls.  `queries` is a host array read during the call.
 */
sm_status sm_search_batch(const sm_query *queries, uint32_t nq, sm_stream_t stream);

/*
 * Asynchronous batch in caller-provided device memory (for serving loops that
 * own their memory budget).  sm_batch_workspace_size returns the bytes a
 * batch of these queries needs (claim counters, one look-back word per work
 * item, descriptors, spill area); sm_search_batch_async lays the batch out in
 * `workspace` (device, 256-byte aligned, at least that many bytes), enqueues
 * the descriptor upload, the workspace reset and one persistent launch per
 * kernel family on `stream`, and returns.  The workspace, texts, plans and
 * outputs must stay valid until the stream reaches this point; the call
 * allocates nothing.  The descriptor upload is from pageable host memory, so
 * the call may wait for work already enqueued on `stream`.  Too small a
 * workspace -> SM_EINVAL.
 */
sm_status sm_batch_workspace_size(const sm_query *queries, uint32_t nq, size_t *bytes);
sm_status sm_search_batch_async(const sm_query *queries, uint32_t nq, void *workspace,
                                size_t workspace_bytes, sm_stream_t stream);

/*
 * Reusable batch: sm_batch_create uploads the query descriptors once and
 * records the whole batch (workspace reset + one persistent launch per
 * kernel family) as a CUDA graph; sm_batch_launch replays it on `stream`.
 * The texts, plans and output buffers named by the queries must stay valid
 * for the life of the batch.  flags: bit 0 set = plain launches (no graph);
 * bit 1 set = no multi-pattern packs.
 *
 * Multi-pattern packs (sm_search_batch, sm_search_batch_async and
 * sm_batch_create unless flag bit 1): Shift-Or queries with m <= 16 on the
 * same text (same pointer and length), prepared with an alphabet-size hint
 * sigma such that sigma^m >= 2^16 (occurrences expected sparse; for a
 * skewed text, pass an effective alphabet size), are packed
 * side by side into one 32-bit Shift-And state (at most 32 bits and 16
 * patterns a pack) and scanned together.  Results are the same as without
 * packing for any text (dense texts are only slower).
 */
sm_status sm_batch_create(const sm_query *queries, uint32_t nq, uint32_t flags,
                          sm_stream_t stream, sm_batch **out_batch);
sm_status sm_batch_launch(sm_batch *batch, sm_stream_t stream);
sm_status sm_batch_free(sm_batch *batch);

/*
 * Tuning table: per (m bucket, sigma bucket) kernel configuration used by
 * SM_VARIANT_AUTO.  m buckets are the bit lengths floor(log2 m) (0..10 for
 * m up to 2047, 11 for longer); sigma buckets are 0 = unknown, then
 * floor(log2 sigma) (1..8).  `entries` holds one sm_config per
 * (m_bucket, sigma_bucket) pair, row-major over 12 x 9 cells; a cell whose
 * variant is 0 keeps the built-in rule.  sm_tuning_set copies the table;
 * sm_tuning_get reads the current table into `entries` (12*9 cells).
 * sm_tuning_reset restores the built-in rule.
 */
#define SM_TUNE_M_BUCKETS 12
#define SM_TUNE_S_BUCKETS 9
sm_status sm_tuning_set(const sm_config *entries, uint32_t count);
sm_status sm_tuning_get(sm_config *entries, uint32_t count);
sm_status sm_tuning_reset(void);

/*
 * sm_sync - wait for all work on `stream`, then report (and clear) any
 * device-side timeout raised by a search since the last sm_sync:
 * SM_ETIMEOUT if a bounded wait ran out, SM_ECUDA on a CUDA error.
 */
sm_status sm_sync(sm_stream_t stream);

/*
 * sm_kernel_launches - number of kernel launches this library has issued
 * in this process (graph replays count their kernels).  For accounting.
 */
uint64_t sm_kernel_launches(void);

/*
 * sm_selftest_wait - failure-reporting check.  Enqueues on `stream` one
 * warp that resolves a look-back word whose predecessor nothing ever
 * publishes: the library's bounded wait runs out after its limit (2 s of
 * device time), the kernel records the timeout in the device error word
 * and returns, and the next sm_sync(stream) reports SM_ETIMEOUT (and clears
 * it).  The stream and context stay usable.  Returns SM_ECUDA if the launch
 * fails.
 */
sm_status sm_selftest_wait(sm_stream_t stream);

/* Release library-owned workspace and cached plans.  No work may be pending. */
sm_status sm_shutdown(void);

/* Human-readable text for a status code (static storage). */
const char *sm_strerror(sm_status status);

#ifdef __cplusplus
}
#endif

#endif /* SMGPU_H */
