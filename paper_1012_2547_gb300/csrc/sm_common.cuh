// Shared device/host definitions of libsmgpu: plan and query layouts,
// mbarrier / bulk-copy helpers and the decoupled look-back used to turn
// per-tile hit counts into sorted global output offsets.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace smgpu {

// ---------------------------------------------------------------- layouts

enum : uint32_t { VAR_SHIFTOR = 1, VAR_QGRAM = 2, VAR_LINEAR = 3, VAR_DFA = 4 };

// Largest automaton (transition table bytes) a DFA plan may have: the table
// lives in shared memory beside the kernel's other buffers.
constexpr uint32_t DFA_MAX_TABLE = 32768 - 256;

// Device header of a plan blob.  The blob is one contiguous, 256-byte
// aligned allocation: header, then the tables at the listed byte offsets.
struct PlanDev {
    uint32_t m;
    uint32_t variant;     // VAR_*
    uint32_t word_bits;   // Shift-Or state width (32 / 64)
    uint32_t hist;        // 1: Shift-Or words keep 16 match flags above bit m-1
    uint32_t q;           // q-gram length (QGRAM)
    uint32_t s;           // probe stride m - q + 1 (QGRAM)
    uint32_t bm_bits;     // log2 of q-gram bitmap size in bits
    uint32_t slot_bits;   // log2 of q-gram hash slots
    uint32_t off_tbl;     // 256 Shift-And masks (u32 or u64)
    uint32_t off_pat;     // pattern bytes, zero padded to a multiple of 16 (+16)
    uint32_t off_bitmap;  // q-gram presence bitmap (u32 words)
    uint32_t off_slots;   // QSlot[1 << slot_bits]
    uint32_t off_offs;    // u16 offsets j of each q-gram, descending per key
    uint32_t off_fail;    // u32 border table fail[0..m] (Knuth-Morris-Pratt)
    uint32_t tile_starts; // start positions per work item (QGRAM / LINEAR / DFA)
    uint32_t bytes;       // blob size
    // String-matching automaton over a class-reduced alphabet (DFA plans,
    // and q-gram plans of periodic patterns for their dense fallback; 0 =
    // none).  Rows are addressed by byte offset r = 2 * C * state and
    // cls[c] = 2 * class of byte c (class 0: bytes absent from p); the u16 at
    // byte offset r + cls[c] of the table is the row offset of the next
    // state, so a step is two loads and one add.
    uint32_t off_cls;     // 256 x u8
    uint32_t off_dfa;     // (m + 1) x C x u16
    uint32_t classes;     // C
    uint32_t dfa_final;   // row offset of state m (a match ends here)
    uint32_t reserved[12];
};
static_assert(sizeof(PlanDev) == 128, "PlanDev is one 128-byte header");

struct QSlot {
    uint64_t key;    // q-gram packed little-endian (byte 0 in bits 0..7)
    uint32_t first;  // index of its first offset in the offsets array
    uint32_t count;  // number of offsets; 0 marks an empty slot
};

// One query as the kernels see it.
struct QueryDev {
    const uint8_t *text;
    uint64_t n;
    const PlanDev *plan;
    uint64_t *out_pos;
    uint64_t cap;
    uint64_t *out_count;
    uint64_t *state;        // look-back words, one per work item
    uint64_t ntiles;        // work items of this query
    uint64_t first_ticket;  // tickets [first_ticket, first_ticket + ntiles)
    uint64_t nsub;          // bit-parallel kernel: staged sub-tiles of the query
    uint32_t sub_per_item;  // bit-parallel kernel: sub-tiles per work item
    uint32_t pad;
};

// Arguments of one persistent launch over a group of queries that share a
// kernel.  nq == 1 uses the inline `one`, otherwise `qs` (device array).
struct LaunchArgs {
    const QueryDev *qs;
    QueryDev one;
    uint32_t nq;
    uint32_t pad;
    unsigned long long *ticket;  // claim counter, zero at launch
    unsigned long long total;    // total tickets
    uint32_t *err;               // device error word (bit flags)
    uint8_t *spill;              // bit-parallel kernel: per-block flag spill area, or null
    // Ticket map, or null.  Entry t is (query index << 40) | item: the
    // launch's items in the order the host chose (items of queries that
    // share a text interleaved by text position, so the text streams
    // through L2 once for all of them).  Each query's items still come in
    // increasing order, which the look-back needs.  Null: tickets run
    // query by query, [first_ticket, first_ticket + ntiles) per query.
    const uint64_t *tmap;
};

constexpr uint64_t TMAP_ITEM_MASK = (1ull << 40) - 1;

enum : uint32_t { ERR_TIMEOUT = 1u, ERR_COPY = 2u };

// A multi-pattern pack, built by the host for a batch: up to MP_MAXK
// Shift-And patterns over one text, packed side by side into one 32-bit
// state.  The pack's own QueryDev (text, item split, tickets) has `plan`
// pointing at this block; each pattern keeps its own query (output,
// capacity, count, look-back words).
constexpr int MP_MAXK = 16;
struct PackPlan {
    uint32_t k;                       // patterns in the pack
    uint32_t I;                       // the first bit of every field
    uint32_t F;                       // the last bit of every field
    uint32_t maxm;                    // longest pattern
    uint8_t shift[MP_MAXK];           // field of pattern p: bits shift[p] ..
    uint8_t len[MP_MAXK];             //   shift[p] + len[p] - 1 (len = m)
    const QueryDev *member[MP_MAXK];  // the patterns' own queries
    uint32_t table[256];              // OR over p of (mask_p[c] << shift[p])
};
constexpr size_t MP_PLAN_BYTES = (sizeof(PackPlan) + 255) & ~size_t(255);

// Look-back word: status in bits 62..63, value in bits 0..61.
constexpr uint64_t LB_EMPTY = 0ull;
constexpr uint64_t LB_AGG = 1ull << 62;
constexpr uint64_t LB_INC = 2ull << 62;
constexpr uint64_t LB_ERR = 3ull << 62;
constexpr uint64_t LB_VAL = (1ull << 62) - 1;

// Bound of every device-side wait, in globaltimer nanoseconds.
constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;

#ifdef __CUDACC__

// ---------------------------------------------------------------- PTX helpers

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// Test (and, with a suspend-time hint, wait up to `hint_ns` for) completion
// of phase `parity`.  A suspended warp issues nothing, so waiting warps do
// not take issue slots from warps that have work.
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity,
                                              uint32_t hint_ns = 1000000u) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}

// Bounded wait for phase `parity` of `bar`; false if the limit ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (global_ns() - t0 > WAIT_LIMIT_NS) return false;
    }
    return true;
}

// Order earlier generic-proxy shared accesses before later async-proxy ones.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// 1-D bulk copy global -> shared, completion counted on `bar` (bytes and
// both addresses must be multiples of 16).
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ uint64_t ld_relaxed(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed(uint64_t *p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------- look-back

// Single-pass decoupled look-back (Merrill and Garland, "Single-pass
// Parallel Prefix Scan with Decoupled Look-back", 2016), written from the
// published method.  Called by one full warp of the block that owns work
// item k of a query once the item's hit count `agg` is known.  A window is
// the 32 nearest unread predecessors (one coalesced load per lane).  While
// a window holds only aggregates the next round reads 8 windows at once, so
// a far inclusive prefix costs few round trips; a window blocked on an
// unpublished item backs off exponentially, so spinning warps do not flood
// L2.  Items of a query are claimed in increasing ticket order, so every
// item waited on is already owned by a running block and the wait ends.
// Returns the number of hits in items 0..k-1; `*ok` turns false if a wait
// ran out or a predecessor failed, in which case the item is marked failed
// so successors stop waiting.
constexpr int LB_WINDOWS = 8;

// Publishes item k's own count: inclusive at once for item 0, an aggregate
// otherwise.  (Whole warp; lane 0 stores.)
__device__ __forceinline__ void lookback_publish(uint64_t *state, uint64_t k, uint64_t agg) {
    if ((threadIdx.x & 31) == 0) st_relaxed(&state[k], (k == 0 ? LB_INC : LB_AGG) | agg);
}

// Exclusive prefix of item k, whose count `agg` lookback_publish has
// already made visible; publishes the inclusive prefix when found.
__device__ __forceinline__ uint64_t lookback_resolve(uint64_t *state, uint64_t k, uint64_t agg,
                                                     uint32_t *err, bool *ok) {
    const int lane = threadIdx.x & 31;
    *ok = true;
    if (k == 0) return 0;
    uint64_t excl = 0;
    int64_t j = static_cast<int64_t>(k) - 1;  // nearest predecessor not yet summed
    int nwin = 1;
    uint32_t sleep_ns = 32;
    uint64_t t0 = 0;
    bool timed = false;
    while (true) {
        uint64_t w[LB_WINDOWS];
#pragma unroll
        for (int i = 0; i < LB_WINDOWS; ++i) {
            const int64_t idx = j - lane - 32 * i;
            w[i] = (i < nwin && idx >= 0) ? ld_relaxed(&state[idx]) : LB_INC;
        }
        bool found = false, blocked = false, failed = false;
        int consumed = 0;  // windows summed in full
        uint64_t part = 0;
#pragma unroll
        for (int i = 0; i < LB_WINDOWS; ++i) {
            if (i < nwin && !found && !blocked) {
                const uint64_t st = w[i] & ~LB_VAL;
                const unsigned done = __ballot_sync(0xffffffffu, st == LB_INC || st == LB_ERR);
                const unsigned empty = __ballot_sync(0xffffffffu, st == LB_EMPTY);
                const int first = done ? __ffs(done) - 1 : 32;
                const unsigned before = first == 32 ? 0xffffffffu : ((1u << first) - 1u);
                if (empty & before) {
                    blocked = true;
                } else {
                    if (lane <= first) part += w[i] & LB_VAL;
                    if (first < 32) {
                        found = true;
                        failed = __shfl_sync(0xffffffffu, st, first) == LB_ERR;
                    } else {
                        consumed = i + 1;
                    }
                }
            }
        }
        excl += warp_sum_u64(part);
        if (failed) {
            if (lane == 0) st_relaxed(&state[k], LB_ERR);
            *ok = false;
            return 0;
        }
        if (found) break;
        j -= 32 * consumed;
        if (blocked) {
            if (!timed) {
                t0 = global_ns();
                timed = true;
            } else if (global_ns() - t0 > WAIT_LIMIT_NS) {
                if (lane == 0) {
                    atomicOr(err, ERR_TIMEOUT);
                    st_relaxed(&state[k], LB_ERR);
                }
                *ok = false;
                return 0;
            }
            __nanosleep(sleep_ns);
            sleep_ns = min(sleep_ns * 2, 1024u);
            nwin = 1;
        } else {
            nwin = LB_WINDOWS;  // only aggregates so far: read further per round
            timed = false;
        }
    }
    if (lane == 0) st_relaxed(&state[k], LB_INC | ((excl + agg) & LB_VAL));
    return excl;
}

// Publish and resolve in one go (the item's warp waits for its prefix).
__device__ __forceinline__ uint64_t lookback_exclusive(uint64_t *state, uint64_t k, uint64_t agg,
                                                       uint32_t *err, bool *ok) {
    lookback_publish(state, k, agg);
    return lookback_resolve(state, k, agg, err, ok);
}

// Ticket -> (query index, tile) for a launch.
__device__ __forceinline__ void resolve_ticket(const LaunchArgs &a, unsigned long long t,
                                               uint32_t *qi, uint64_t *tile) {
    if (a.tmap) {
        const uint64_t e = __ldg(&a.tmap[t]);
        *qi = static_cast<uint32_t>(e >> 40);
        *tile = e & TMAP_ITEM_MASK;
        return;
    }
    if (a.nq == 1) {
        *qi = 0;
        *tile = t;
        return;
    }
    uint32_t lo = 0, hi = a.nq - 1;
    while (lo < hi) {  // last query with first_ticket <= t
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (a.qs[mid].first_ticket <= t) lo = mid;
        else hi = mid - 1;
    }
    *qi = lo;
    *tile = t - a.qs[lo].first_ticket;
}

__device__ __forceinline__ const QueryDev &query_of(const LaunchArgs &a, uint32_t qi) {
    return a.nq == 1 ? a.one : a.qs[qi];
}

#endif  // __CUDACC__

}  // namespace smgpu
