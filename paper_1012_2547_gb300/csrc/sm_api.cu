// Host side of libsmgpu: the C ABI of include/smgpu.h and include/smgen.h.
//
//   sm_prepare*   pattern -> plan: chooses the kernel family (tuning table
//                 or built-in rule), builds its tables on the host and copies
//                 them to device memory as one blob.
//   sm_search*    one query -> workspace reset + one persistent launch.
//   sm_batch_*    many queries -> descriptors uploaded once; per kernel
//                 family one persistent launch over all its (query, tile)
//                 work items; the sequence is captured as a CUDA graph.
//   sm_tuning_*   the (m bucket, sigma bucket) -> configuration table.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <condition_variable>
#include <functional>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "sm_internal.h"
#include "smgen.h"
#include "smgpu.h"

namespace smgpu {
const void *so_kernel_fn(int kid);
size_t so_kernel_smem(int kid);
int so_kernel_threads();
uint64_t so_tile_starts();
uint32_t so_hit_buffer();
uint32_t so_spill_bytes();
uint32_t so_max_sub();
const void *mp_kernel_fn();
size_t mp_kernel_smem();
const void *qg_kernel_fn(int kid);
int qg_kernel_threads();
}  // namespace smgpu

using namespace smgpu;

namespace {

constexpr uint32_t kMaxM = 1u << 24;
constexpr size_t kTicketBytes = 256;  // up to 32 claim counters per launch set

// Device blocks for plans are recycled instead of freed: cudaFree waits for
// the whole device, which would stall every stream each time a batch's plans
// are released (e.g. by a serving loop).  Released blocks go to a free list
// by power-of-two size class (bounded in total bytes); larger requests and
// overflow use cudaMalloc / cudaFree directly.
class BlockPool {
  public:
    static BlockPool &get() {
        static BlockPool *P = new BlockPool();  // never destroyed: used at exit
        return *P;
    }
    cudaError_t acquire(size_t bytes, void **out, size_t *cls_bytes) {
        const size_t cls = size_class(bytes);
        {
            std::lock_guard<std::mutex> g(mu_);
            auto &fl = free_[index(cls)];
            if (cls <= kMaxClass && !fl.empty()) {
                *out = fl.back();
                fl.pop_back();
                cached_ -= cls;
                *cls_bytes = cls;
                return cudaSuccess;
            }
        }
        *cls_bytes = cls;
        return cudaMalloc(out, cls);
    }
    void release(void *p, size_t cls) {
        if (!p) return;
        {
            std::lock_guard<std::mutex> g(mu_);
            if (cls <= kMaxClass && cached_ + cls <= kMaxCached) {
                free_[index(cls)].push_back(p);
                cached_ += cls;
                return;
            }
        }
        cudaFree(p);
    }

  private:
    static constexpr size_t kMinClass = 4096;
    static constexpr size_t kMaxClass = size_t(64) << 20;
    static constexpr size_t kMaxCached = size_t(512) << 20;
    static size_t size_class(size_t b) {
        size_t c = kMinClass;
        while (c < b) c <<= 1;
        return c;
    }
    static int index(size_t cls) {
        int i = 0;
        while ((kMinClass << i) < cls) ++i;
        return i;
    }
    std::mutex mu_;
    std::vector<void *> free_[48];
    size_t cached_ = 0;
};

struct DevArena {
    void *ptr = nullptr;
    size_t cls = 0;  // pooled block size (0: plain cudaMalloc)
    ~DevArena() {
        if (!ptr) return;
        if (cls) BlockPool::get().release(ptr, cls);
        else cudaFree(ptr);
    }
};

struct Workspace {
    uint8_t *mem = nullptr;
    size_t bytes = 0;
};

struct Lib {
    std::mutex mu;
    bool inited = false;
    int device = -1;
    int sms = 0;
    uint32_t *err = nullptr;
    KernelShape shapes[K_COUNT];
    std::unordered_map<cudaStream_t, Workspace> ws;
    std::unordered_map<std::string, sm_plan *> cache;
    sm_config tuning[SM_TUNE_M_BUCKETS * SM_TUNE_S_BUCKETS];
    std::atomic<uint64_t> launches{0};
    uint32_t item_cap = 64;  // most units per work item (SMGPU_ITEM_UNITS overrides)
};

Lib &lib() {
    static Lib *L = new Lib();  // never destroyed: may be used at exit
    return *L;
}

sm_status from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return SM_OK;
    if (e == cudaErrorMemoryAllocation) return SM_ENOMEM;
    return SM_ECUDA;
}

#define SM_TRY_CUDA(expr)                          \
    do {                                           \
        cudaError_t e_ = (expr);                   \
        if (e_ != cudaSuccess) return from_cuda(e_); \
    } while (0)

// Device init: kernel shapes and the error word.  Caller holds no lock.
sm_status ensure_init() {
    Lib &L = lib();
    std::lock_guard<std::mutex> g(L.mu);
    if (L.inited) return SM_OK;
    int dev = 0;
    SM_TRY_CUDA(cudaGetDevice(&dev));
    int sms = 0;
    SM_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    SM_TRY_CUDA(kernels_init(sms));
    for (int k = 0; k < K_COUNT; ++k) L.shapes[k] = kernel_shape(k);
    SM_TRY_CUDA(cudaMalloc(&L.err, 256));
    SM_TRY_CUDA(cudaMemset(L.err, 0, 256));
    L.device = dev;
    L.sms = sms;
    if (const char *e = std::getenv("SMGPU_ITEM_UNITS")) {
        const long v = std::strtol(e, nullptr, 10);
        if (v >= 1 && v <= 4096) L.item_cap = static_cast<uint32_t>(v);
    }
    L.inited = true;
    return SM_OK;
}

bool aligned8(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 7u) == 0; }

// ---------------------------------------------------------------- plans

uint32_t ceil_log2(uint64_t x) {
    uint32_t b = 0;
    while ((1ull << b) < x) ++b;
    return b;
}

uint32_t m_bucket(uint32_t m) {
    uint32_t b = 0;
    while (b < 11 && (2u << b) <= m) ++b;
    return b;  // floor(log2 m), capped at 11
}

uint32_t s_bucket(uint32_t sigma) {
    if (sigma == 0) return 0;
    uint32_t b = 0;
    while (b < 8 && (2u << b) <= sigma) ++b;
    return std::max(1u, b);  // floor(log2 sigma) in 1..8
}

// Built-in q-gram length: the smallest q with sigma^q >= 2^11 m, clamped to
// 3..8 (sigma 4 when unknown), so that a probe of a text q-gram that is not
// one of the pattern's m - q + 1 q-grams passes the filter rarely: a warp's
// round of 32 probes then reaches the key table in a few percent of rounds.
uint32_t rule_q(uint32_t m, uint32_t sigma) {
    const double sg = sigma >= 2 ? static_cast<double>(sigma) : 4.0;
    int q = static_cast<int>(std::ceil(std::log(2048.0 * m) / std::log(sg) - 1e-9));
    q = std::min(8, std::max(3, q));
    return std::min<uint32_t>(static_cast<uint32_t>(q), m);
}

// Built-in kernel family: the bit-parallel scan for short patterns, and for
// m <= 64 on binary and ternary alphabets (where even 8-grams filter
// poorly); the q-gram stride filter otherwise (from m = 17 its probes, one
// per m - q + 1 bytes, cost fewer instructions per byte than the scan's
// step per byte).
uint32_t rule_variant(uint32_t m, uint32_t sigma) {
    if (m <= 16) return SM_VARIANT_SHIFTOR;
    if (m <= 64 && sigma >= 2 && sigma <= 3) return SM_VARIANT_SHIFTOR;
    return SM_VARIANT_QGRAM;
}

size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

uint64_t pack_qgram(const uint8_t *p, uint32_t q) {
    uint64_t g = 0;
    for (uint32_t b = 0; b < q; ++b) g |= static_cast<uint64_t>(p[b]) << (8 * b);
    return g;
}

}  // namespace

struct sm_plan {
    PlanDev hdr;
    const PlanDev *dev = nullptr;
    std::shared_ptr<DevArena> arena;
    int kid = 0;
    uint32_t min_units = 1;  // shortest work item in units (config `tile`, bit-parallel kernels)
    uint32_t sigma = 0;      // alphabet-size hint given at preparation (0 = unknown)
    std::vector<uint8_t> pattern;
};

struct sm_batch {
    std::shared_ptr<DevArena> arena;  // owning allocation (null for caller workspace)
    uint8_t *base = nullptr;          // tickets | states | descriptors | zero list | spill
    struct Group {
        int kid;
        LaunchArgs args;
        int grid;
    };
    std::vector<Group> groups;
    uint64_t **zero_list = nullptr;
    uint32_t nzero = 0;
    size_t reset_bytes = 0;  // tickets + states, zeroed before each launch
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint32_t kernels = 0;
};

namespace {

// Host blob for one pattern.  Returns SM_EINVAL if `cfg` cannot serve it.
// Builds the device image of one plan and appends it to `arena` (at a
// multiple of 256 bytes past its start; *at receives the offset).
// `tuning` is a snapshot of the tuning table, or null to read the
// library's under its lock.  Scratch tables are kept per thread, so many
// plans built in a row allocate nothing but the arena's growth.
sm_status build_blob(const uint8_t *p, uint32_t m, uint32_t sigma, const sm_config *cfg,
                     const sm_config *tuning, std::vector<uint8_t> *arena, size_t *at,
                     PlanDev *hdr_out, int *kid_out, uint32_t *min_units_out) {
    Lib &L = lib();
    sm_config tc{};
    const size_t cell = m_bucket(m) * SM_TUNE_S_BUCKETS + s_bucket(sigma);
    if (tuning) {
        tc = tuning[cell];
    } else {
        std::lock_guard<std::mutex> g(L.mu);
        tc = L.tuning[cell];
    }
    // Border table (Knuth-Morris-Pratt): fail[q] = length of the longest
    // proper border of p[0..q-1]; m - fail[m] is the smallest period of p.
    thread_local std::vector<uint32_t> fail;
    fail.assign(m + 1, 0);
    for (uint32_t i = 1, kk = 0; i < m; ++i) {
        while (kk > 0 && p[kk] != p[i]) kk = fail[kk];
        if (p[kk] == p[i]) ++kk;
        fail[i + 1] = kk;
    }
    // Byte classes of the automaton: 0 for bytes absent from p, then one
    // class per distinct pattern byte in order of first occurrence.
    uint16_t cls_of[256] = {};
    uint32_t C = 1;
    for (uint32_t j = 0; j < m; ++j)
        if (!cls_of[p[j]]) cls_of[p[j]] = static_cast<uint16_t>(C++);
    const uint64_t dfa_bytes = static_cast<uint64_t>(m + 1) * C * 2;
    const bool dfa_fits = dfa_bytes <= DFA_MAX_TABLE;

    uint32_t variant = cfg && cfg->variant ? cfg->variant : tc.variant;
    if (variant == SM_VARIANT_AUTO) variant = rule_variant(m, sigma);
    // A tuned (not explicit) choice that cannot serve p falls back to the rule.
    const bool explicit_cfg = cfg && cfg->variant;
    if (!explicit_cfg && variant == SM_VARIANT_SHIFTOR && m > 64) variant = SM_VARIANT_QGRAM;
    if (!explicit_cfg && variant == SM_VARIANT_DFA && !dfa_fits) variant = rule_variant(m, sigma);
    const sm_config *src = explicit_cfg ? cfg : &tc;

    PlanDev h{};
    h.m = m;
    int kid = 0;
    uint32_t q = 0, wb = 0;
    uint64_t R = 0;
    if (variant == SM_VARIANT_SHIFTOR) {
        wb = src->word_bits ? src->word_bits : (m <= 32 ? 32u : 64u);
        if (!explicit_cfg && m > wb) wb = 64;
        if ((wb != 32 && wb != 64) || m > wb) return SM_EINVAL;
        kid = so_kid_for(m, wb);
        if (kid < 0) return SM_EINVAL;
        h.hist = so_hist(kid) ? 1u : 0u;
        h.variant = VAR_SHIFTOR;
        h.word_bits = wb;
        h.tile_starts = static_cast<uint32_t>(so_tile_starts());
        // tile: log2 of the shortest work item in bytes, whole sub-tiles.
        if (src->tile) {
            const uint64_t bytes = 1ull << std::min(src->tile, 40u);
            *min_units_out = static_cast<uint32_t>(std::min<uint64_t>(
                so_max_sub(), std::max<uint64_t>(1, (bytes + so_tile_starts() - 1) / so_tile_starts())));
        }
    } else if (variant == SM_VARIANT_QGRAM) {
        q = src->q ? src->q : rule_q(m, sigma);
        if (!explicit_cfg) q = std::min(q, m);
        if (q < 1 || q > 8 || q > m) return SM_EINVAL;
        const uint32_t s = m - q + 1;
        // Base range per thread ~4 KiB of start positions; a launch may give
        // a thread several base ranges (sub_per_item).
        // Probes per thread range: about 1 KiB of starts (2 to 256 probes;
        // fewer only where 128 ranges would pass 2^32 starts).  Short units
        // keep many blocks busy on a short text, including when an item falls
        // back to the linear scan (one thread per range); a launch over a
        // long text gives each work item many units (sub_per_item), so the
        // filter still runs many probe rounds per item there.
        uint32_t ppt = src->tile ? (1u << std::min(src->tile, 20u)) / s : 1024u / s;
        ppt = std::max(2u, std::min(ppt, 256u));
        while (ppt > 2 && static_cast<uint64_t>(ppt) * s * qg_kernel_threads() >= (1ull << 32)) ppt /= 2;
        R = static_cast<uint64_t>(ppt) * s;
        if (R * qg_kernel_threads() >= (1ull << 32)) return SM_EINVAL;
        h.variant = VAR_QGRAM;
        h.q = q;
        h.s = s;
        h.tile_starts = static_cast<uint32_t>(R * qg_kernel_threads());
        kid = K_QGRAM;
    } else if (variant == SM_VARIANT_LINEAR) {
        R = std::max<uint64_t>(1024, 4ull * m);
        if (src->tile) R = std::max<uint64_t>(R, 1ull << std::min(src->tile, 24u));
        if (R * qg_kernel_threads() >= (1ull << 32)) return SM_EINVAL;
        h.variant = VAR_LINEAR;
        h.tile_starts = static_cast<uint32_t>(R * qg_kernel_threads());
        kid = K_LINEAR;
    } else if (variant == SM_VARIANT_DFA) {
        if (!dfa_fits) return SM_EINVAL;
        // Each thread runs the automaton over m - 1 bytes past its last
        // start.  Base ranges of max(1024, m) starts keep enough threads for
        // texts of a few MiB; a launch over a long text gives each thread
        // several base ranges (sub_per_item), which dilutes the overlap.
        R = std::max<uint64_t>(1024, m);
        if (src->tile) R = std::max<uint64_t>(R, 1ull << std::min(src->tile, 24u));
        R = (R + 15) & ~uint64_t(15);
        if (R * qg_kernel_threads() >= (1ull << 32)) return SM_EINVAL;
        h.variant = VAR_DFA;
        h.tile_starts = static_cast<uint32_t>(R * qg_kernel_threads());
        kid = K_DFA;
    } else {
        return SM_EINVAL;
    }
    // The automaton: for DFA plans, and for q-gram plans of periodic
    // patterns (smallest period <= m/2), whose dense tiles use it.  Only a
    // periodic pattern can have occurrences closer than m/2 apart.
    const bool with_dfa =
        h.variant == VAR_DFA || (h.variant == VAR_QGRAM && dfa_fits && 2ull * (m - fail[m]) <= m);

    // q-gram table, in O(m): the packed q-gram of every offset j (rolled
    // from the previous one), inserted into a scratch slot table sized for
    // m - q + 1 keys (the same hash and probing as the plan's table), which
    // counts the distinct ones; they size the plan's table.  When that size
    // is the scratch table's (every aperiodic pattern) the scratch table is
    // the plan's table.
    thread_local std::vector<uint64_t> keys;
    thread_local std::vector<QSlot> tslots;
    thread_local std::vector<uint32_t> slot_of;
    uint32_t nkeys = 0, sbits = 0;
    if (h.variant == VAR_QGRAM) {
        const uint32_t ng = m - q + 1;
        keys.resize(ng);
        slot_of.resize(ng);
        uint64_t g = pack_qgram(p, q);
        const uint32_t top = 8 * (q - 1);
        for (uint32_t j = 0; j < ng; ++j) {
            keys[j] = g;
            if (j + q < m) g = (g >> 8) | (static_cast<uint64_t>(p[j + q]) << top);
        }
        sbits = std::max(4u, ceil_log2(2ull * ng));
        tslots.assign(size_t(1) << sbits, QSlot{0, 0, 0});
        const uint32_t smask = (1u << sbits) - 1;
        for (uint32_t j = 0; j < ng; ++j) {
            const uint64_t key = keys[j];
            uint32_t sl = static_cast<uint32_t>((key * 0x9E3779B97F4A7C15ull) >> (64 - sbits));
            while (tslots[sl].count && tslots[sl].key != key) sl = (sl + 1) & smask;
            if (!tslots[sl].count) {
                tslots[sl].key = key;
                ++nkeys;
            }
            ++tslots[sl].count;
            slot_of[j] = sl;
        }
        h.slot_bits = std::max(4u, ceil_log2(2ull * nkeys));
        // Presence bitmap of 2^(slot_bits + 8) bits, 512 to 1024 per key (a
        // probe of a non-key passes it with probability under 1/512), at most
        // 2^16 bits.
        h.bm_bits = std::min(16u, std::max(12u, h.slot_bits + 8));
    }

    // Layout.
    size_t off = sizeof(PlanDev);
    h.off_tbl = static_cast<uint32_t>(off);
    const uint32_t esz = h.variant == VAR_SHIFTOR ? so_entry_bytes(kid) : 0;
    off += 256 * esz;
    off = align16(off);
    h.off_pat = static_cast<uint32_t>(off);
    off += align16(m) + 16;
    h.off_bitmap = static_cast<uint32_t>(off);
    off += h.variant == VAR_QGRAM ? (size_t(1) << h.bm_bits) / 8 : 0;
    off = align16(off);
    h.off_slots = static_cast<uint32_t>(off);
    off += h.variant == VAR_QGRAM ? (size_t(1) << h.slot_bits) * sizeof(QSlot) : 0;
    h.off_offs = static_cast<uint32_t>(off);
    off += h.variant == VAR_QGRAM ? align16(4ull * (m - q + 1)) : 0;
    h.off_fail = static_cast<uint32_t>(off);
    off += align16(4ull * (m + 1));
    if (with_dfa) {
        h.off_cls = static_cast<uint32_t>(off);
        off += 256 * 2;
        h.off_dfa = static_cast<uint32_t>(off);
        off += align16(dfa_bytes);
        h.classes = C;
        h.dfa_final = m * C * 2;
    }
    off = (off + 255) & ~size_t(255);
    if (off >= (1ull << 32)) return SM_EINVAL;
    h.bytes = static_cast<uint32_t>(off);

    const size_t base = (arena->size() + 255) & ~size_t(255);
    arena->resize(base + off);  // new bytes are zero
    uint8_t *b = arena->data() + base;
    *at = base;
    if (h.variant == VAR_SHIFTOR) {
        // Shift-And masks: bit j of B[c] is 1 iff p[j] = c; bits >= m are 1
        // so that older match flags survive the AND.  Entries keep the low
        // esz bytes (the kernel supplies the ones above them); stored
        // little-endian, as the device reads them.
        const uint64_t low = m >= 64 ? ~0ull : ((1ull << m) - 1);
        uint64_t B[256];
        for (int c = 0; c < 256; ++c) B[c] = ~low;
        for (uint32_t j = 0; j < m; ++j) B[p[j]] |= 1ull << j;
        uint8_t *tb = b + h.off_tbl;
        switch (esz) {  // typed stores: the low esz bytes, little-endian as the device reads them
            case 1: for (int c = 0; c < 256; ++c) tb[c] = static_cast<uint8_t>(B[c]); break;
            case 2: for (int c = 0; c < 256; ++c) reinterpret_cast<uint16_t *>(tb)[c] = static_cast<uint16_t>(B[c]); break;
            case 4: for (int c = 0; c < 256; ++c) reinterpret_cast<uint32_t *>(tb)[c] = static_cast<uint32_t>(B[c]); break;
            default: for (int c = 0; c < 256; ++c) reinterpret_cast<uint64_t *>(tb)[c] = B[c]; break;
        }
    }
    std::memcpy(b + h.off_pat, p, m);
    if (h.variant == VAR_QGRAM) {
        uint32_t *bitmap = reinterpret_cast<uint32_t *>(b + h.off_bitmap);
        QSlot *slots = reinterpret_cast<QSlot *>(b + h.off_slots);
        uint32_t *offs = reinterpret_cast<uint32_t *>(b + h.off_offs);
        const uint32_t mask = (1u << h.slot_bits) - 1;
        const uint32_t ng = m - q + 1;
        // Each key gets a slot (linear probing from its hash) and a count;
        // then each slot a run of the offsets array; then the runs are
        // filled with j descending, the order the kernel emits candidates.
        if (h.slot_bits == sbits) {
            std::memcpy(slots, tslots.data(), (size_t(1) << sbits) * sizeof(QSlot));
        } else {  // fewer distinct q-grams than offsets (periodic p): a smaller table
            for (uint32_t j = 0; j < ng; ++j) {
                const uint64_t g = keys[j];
                uint32_t sl = static_cast<uint32_t>((g * 0x9E3779B97F4A7C15ull) >> (64 - h.slot_bits));
                while (slots[sl].count && slots[sl].key != g) sl = (sl + 1) & mask;
                slots[sl].key = g;
                ++slots[sl].count;
                slot_of[j] = sl;
            }
        }
        // Bitmap bit of every key: top bm_bits bits of the two 32-bit
        // halves' multiplicative hashes xored (the same function as the
        // kernel's probe loop).  `first` is first set one past each run,
        // then moved down as the run is filled with j ascending, so the run
        // holds j descending and `first` ends at the run's start.
        uint32_t run = 0;
        for (uint32_t sl = 0; sl <= mask; ++sl) {
            if (slots[sl].count) {
                const uint64_t g = slots[sl].key;
                const uint32_t h32 = (static_cast<uint32_t>(g) * 0x9E3779B1u) ^
                                     (static_cast<uint32_t>(g >> 32) * 0x85EBCA77u);
                const uint32_t bb = h32 >> (32 - h.bm_bits);
                bitmap[bb >> 5] |= 1u << (bb & 31);
            }
            run += slots[sl].count;
            slots[sl].first = run;
        }
        for (uint32_t j = 0; j < ng; ++j) offs[--slots[slot_of[j]].first] = j;
    }
    std::memcpy(b + h.off_fail, fail.data(), 4ull * (m + 1));
    if (with_dfa) {
        // Rows by byte offset (row of state q at 2*C*q); entries are the
        // row offsets of the next states.  Row 0 goes to 1 on p[0] only;
        // row q copies the row of X, the state the automaton reaches on
        // p[1..q-1] (the longest proper border of p[0..q-1]), and goes to
        // q+1 on p[q]; row m is the row of X after p[1..m-1].
        uint16_t *cls = reinterpret_cast<uint16_t *>(b + h.off_cls);
        for (int c = 0; c < 256; ++c) cls[c] = static_cast<uint16_t>(2 * cls_of[c]);
        uint16_t *T = reinterpret_cast<uint16_t *>(b + h.off_dfa);
        const uint32_t row = 2 * C;  // bytes per row
        T[cls_of[p[0]]] = static_cast<uint16_t>(row);
        uint32_t X = 0;
        for (uint32_t q = 1; q <= m; ++q) {
            std::memcpy(T + q * C, T + X * C, 2ull * C);
            if (q < m) {
                T[q * C + cls_of[p[q]]] = static_cast<uint16_t>((q + 1) * row);
                X = T[X * C + cls_of[p[q]]] / row;
            }
        }
    }
    std::memcpy(b, &h, sizeof(h));
    *hdr_out = h;
    *kid_out = kid;
    return SM_OK;
}

// Host worker threads for plan building, started on first use and kept:
// starting threads on every call cost more than building a thousand plans.
// run(n, fn) calls fn(0..n-1) on the workers and the calling thread and
// returns when all calls have returned; concurrent run()s take turns.
class HostPool {
  public:
    static HostPool &get() {
        static HostPool *P = new HostPool();  // never destroyed: workers may be idle at exit
        return *P;
    }
    unsigned threads() const { return static_cast<unsigned>(workers_.size()) + 1; }
    void run(unsigned n, const std::function<void(unsigned)> &fn) {
        std::lock_guard<std::mutex> one(run_mu_);
        {
            std::lock_guard<std::mutex> g(mu_);
            job_ = &fn;
            njob_ = n;
            next_ = 0;
            remaining_ = n;
            ++gen_;
        }
        cv_.notify_all();
        work();
        std::unique_lock<std::mutex> g(mu_);
        done_cv_.wait(g, [&] { return remaining_ == 0; });
        job_ = nullptr;
    }

  private:
    HostPool() {
        const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
        const unsigned n = std::min(hw, 32u) - 1;
        for (unsigned i = 0; i < n; ++i) workers_.emplace_back([this] { loop(); });
    }
    // Takes tasks of the current job until none is left.
    void work() {
        while (true) {
            unsigned t;
            const std::function<void(unsigned)> *fn;
            {
                std::lock_guard<std::mutex> g(mu_);
                if (!job_ || next_ >= njob_) return;
                t = next_++;
                fn = job_;
            }
            (*fn)(t);
            std::lock_guard<std::mutex> g(mu_);
            if (--remaining_ == 0) done_cv_.notify_all();
        }
    }
    void loop() {
        uint64_t seen = 0;
        while (true) {
            {
                std::unique_lock<std::mutex> g(mu_);
                cv_.wait(g, [&] { return gen_ != seen; });
                seen = gen_;
            }
            work();
        }
    }
    std::mutex run_mu_, mu_;
    std::condition_variable cv_, done_cv_;
    std::vector<std::thread> workers_;
    const std::function<void(unsigned)> *job_ = nullptr;
    unsigned njob_ = 0, next_ = 0, remaining_ = 0;
    uint64_t gen_ = 0;
};

// Pinned host staging for plan uploads, reused across calls: a copy from
// pageable memory goes through a driver bounce buffer at a fraction of the
// link's rate.  Its mutex is held from the fill to the stream sync that
// follows the copy, so the buffer is never rewritten while in flight.
struct PinnedStaging {
    std::mutex mu;
    uint8_t *p = nullptr;
    size_t cap = 0;
    // Buffers outgrown are kept, not freed: cudaFreeHost waits for the whole
    // device, which stalled a serving loop's scheduler for tens of
    // milliseconds.  Growth doubles, so they add up to less than the buffer
    // in use.
    std::vector<uint8_t *> outgrown;
};

PinnedStaging &pinned_staging() {
    static PinnedStaging *s = new PinnedStaging();  // never destroyed: may be used at exit
    return *s;
}

constexpr size_t kStagingMax = size_t(1) << 30;  // larger uploads stage in pageable memory

sm_status prepare_many(const uint8_t *patterns, const uint32_t *lengths, uint32_t count,
                       uint32_t sigma, const sm_config *cfg, cudaStream_t stream, sm_plan **out) {
    sm_status st = ensure_init();
    if (st != SM_OK) return st;
    std::vector<PlanDev> hdrs(count);
    std::vector<int> kids(count);
    std::vector<uint32_t> min_units(count, 1);
    std::vector<size_t> pat_off(count);
    size_t pos = 0;
    for (uint32_t i = 0; i < count; ++i) {
        if (lengths[i] == 0 || lengths[i] > kMaxM) return SM_EINVAL;
        pat_off[i] = pos;
        pos += lengths[i];
    }
    // Host tables of many patterns are built on the pool's threads (small
    // calls on the caller's thread alone), each thread appending its plans
    // to an arena of its own, with one snapshot of the tuning table.
    std::vector<sm_status> sts(count, SM_OK);
    const bool many = count >= 64;
    const unsigned nth = many ? HostPool::get().threads() : 1u;
    auto on_threads = [&](const std::function<void(unsigned)> &fn) {
        if (!many) fn(0);
        else HostPool::get().run(nth, fn);
    };
    std::vector<sm_config> tuning(SM_TUNE_M_BUCKETS * SM_TUNE_S_BUCKETS);
    {
        std::lock_guard<std::mutex> g(lib().mu);
        std::copy(lib().tuning, lib().tuning + tuning.size(), tuning.begin());
    }
    std::vector<std::vector<uint8_t>> arenas(nth);
    std::vector<size_t> offs(count);
    on_threads([&](unsigned t) {
        size_t guess = 0;  // a little above a typical plan's size: few regrowths
        for (uint32_t i = t; i < count; i += nth) guess += 1024 + 48ull * lengths[i];
        arenas[t].reserve(guess);
        for (uint32_t i = t; i < count; i += nth)
            sts[i] = build_blob(patterns + pat_off[i], lengths[i], sigma, cfg, tuning.data(), &arenas[t],
                                &offs[i], &hdrs[i], &kids[i], &min_units[i]);
    });
    for (uint32_t i = 0; i < count; ++i)
        if (sts[i] != SM_OK) return sts[i];
    // Arena t goes to [arena_at[t], arena_at[t] + size) of the device block.
    std::vector<size_t> arena_at(nth);
    size_t total = 0;
    for (unsigned t = 0; t < nth; ++t) {
        arena_at[t] = total;
        total += (arenas[t].size() + 255) & ~size_t(255);
    }
    for (uint32_t i = 0; i < count; ++i) offs[i] += arena_at[i % nth];
    auto arena = std::make_shared<DevArena>();
    SM_TRY_CUDA(BlockPool::get().acquire(std::max<size_t>(total, 256), &arena->ptr, &arena->cls));
    PinnedStaging &ps = pinned_staging();
    std::lock_guard<std::mutex> staging_lock(ps.mu);
    uint8_t *stage = nullptr;
    std::vector<uint8_t> pageable;
    if (total <= kStagingMax) {
        if (ps.cap < total) {
            const size_t want = std::min(kStagingMax, std::max({total + total / 2, 2 * ps.cap, size_t(64) << 20}));
            uint8_t *np = nullptr;
            if (cudaHostAlloc(reinterpret_cast<void **>(&np), want, cudaHostAllocDefault) == cudaSuccess) {
                if (ps.p) ps.outgrown.push_back(ps.p);
                ps.p = np;
                ps.cap = want;
            } else {
                (void)cudaGetLastError();  // not sticky: stage in pageable memory instead
            }
        }
        if (ps.cap >= total) stage = ps.p;
    }
    if (!stage) {
        pageable.resize(total);
        stage = pageable.data();
    }
    on_threads([&](unsigned t) {
        if (!arenas[t].empty()) std::memcpy(stage + arena_at[t], arenas[t].data(), arenas[t].size());
    });
    // Upload on the caller's stream, then wait for it: the plans are usable
    // by work on any stream once this returns, and no legacy-default-stream
    // copy serialises with other streams' work.
    SM_TRY_CUDA(cudaMemcpyAsync(arena->ptr, stage, total, cudaMemcpyHostToDevice, stream));
    SM_TRY_CUDA(cudaStreamSynchronize(stream));
    pos = 0;
    for (uint32_t i = 0; i < count; ++i) {
        sm_plan *pl = new sm_plan();
        pl->hdr = hdrs[i];
        pl->dev = reinterpret_cast<const PlanDev *>(static_cast<uint8_t *>(arena->ptr) + offs[i]);
        pl->arena = arena;
        pl->kid = kids[i];
        pl->min_units = min_units[i];
        pl->sigma = sigma;
        pl->pattern.assign(patterns + pos, patterns + pos + lengths[i]);
        pos += lengths[i];
        out[i] = pl;
    }
    return SM_OK;
}

// ---------------------------------------------------------------- launches

// Workspace of at least `bytes` for `stream` (grows; growth synchronises).
sm_status get_workspace(cudaStream_t stream, size_t bytes, uint8_t **out) {
    Lib &L = lib();
    std::lock_guard<std::mutex> g(L.mu);
    Workspace &w = L.ws[stream];
    if (w.bytes < bytes) {
        if (w.mem) cudaFree(w.mem);
        w.mem = nullptr;
        w.bytes = 0;
        const size_t want = std::max<size_t>(bytes, std::max<size_t>(2 * w.bytes, 1 << 20));
        cudaError_t e = cudaMalloc(&w.mem, want);
        if (e != cudaSuccess) return from_cuda(e);
        w.bytes = want;
    }
    *out = w.mem;
    return SM_OK;
}

int grid_for(int kid, uint64_t tickets) {
    const KernelShape &s = lib().shapes[kid];
    const uint64_t full = static_cast<uint64_t>(lib().sms) * std::max(1, s.blocks_per_sm);
    return static_cast<int>(std::max<uint64_t>(1, std::min(full, tickets)));
}

// Units per work item for a launch that covers `units` units (staged
// sub-tiles of the bit-parallel kernels, base ranges of the others): at most
// `rounds` (default four) work items per resident block, rounded so that
// the last round of items fills the grid (a round with a few items would
// leave most blocks idle for a whole item); a large launch gets long work
// items and a small one keeps every block busy.
uint32_t sub_per_item(int kid, uint64_t units, uint64_t rounds = 4);

// Rounds of work items for a q-gram plan searched alone: two for strides of
// 512 and more, whose items hold few probes each, so that the per-item
// block scan and look-back weigh less (8 GiB at m = 1024: 33.4 -> 36.0
// TB/s of scanned text); four otherwise (two cost m = 32 1 %).
uint64_t solo_rounds(const sm_plan *plan) {
    return plan->kid == K_QGRAM && plan->hdr.s >= 512 ? 2 : 4;
}

uint32_t sub_per_item(int kid, uint64_t units, uint64_t rounds) {
    const KernelShape &s = lib().shapes[kid];
    const uint64_t resident = static_cast<uint64_t>(lib().sms) * std::max(1, s.blocks_per_sm);
    const uint64_t per = (units + rounds * resident - 1) / (rounds * resident);
    const uint64_t cap = staged_kid(kid) ? std::min<uint64_t>(lib().item_cap, so_max_sub())
                                        : lib().item_cap;
    return static_cast<uint32_t>(std::max<uint64_t>(1, std::min<uint64_t>(cap, per)));
}

// Units per item for one query given the launch's target `per`: the same
// number of items, but of (nearly) equal size, so that no query ends with a
// short item whose look-back waits for its longer predecessors.
uint32_t balanced_per(uint64_t units, uint32_t per) {
    const uint64_t items = (units + per - 1) / per;
    return static_cast<uint32_t>((units + items - 1) / items);
}

// Units per item of one plan: `per`, lowered for q-gram plans so that a
// warp's share of an item (32 thread ranges of tile_starts / threads starts
// per unit) stays below 2^32 starts (the filter keeps warp-relative 32-bit
// positions).
uint32_t plan_per(const sm_plan *plan, uint32_t per) {
    if (plan->kid != K_QGRAM) return per;
    const uint64_t warp_unit = 32ull * (plan->hdr.tile_starts / qg_kernel_threads());
    const uint64_t most = std::max<uint64_t>(1, 0xFFFFFFFFull / warp_unit);
    return static_cast<uint32_t>(std::min<uint64_t>(per, most));
}

bool query_ok(const uint8_t *text, uint64_t n, const sm_plan *plan, const uint64_t *out_pos,
              uint64_t cap, const uint64_t *out_count) {
    if (!plan || !out_count || !aligned8(out_count)) return false;
    if (n > 0 && !text) return false;
    if (n >= (1ull << 62)) return false;
    if (cap > 0 && (!out_pos || !aligned8(out_pos))) return false;
    return true;
}

}  // namespace

// ---------------------------------------------------------------- kernels

namespace smgpu {

static KernelShape g_shapes[K_COUNT];

cudaError_t kernels_init(int sms) {
    (void)sms;
    for (int k = 0; k < K_COUNT; ++k) {
        KernelShape &s = g_shapes[k];
        if (staged_kid(k)) {
            s.fn = k == K_SOMULTI ? mp_kernel_fn() : so_kernel_fn(k);
            s.threads = so_kernel_threads();
            s.smem = k == K_SOMULTI ? mp_kernel_smem() : so_kernel_smem(k);
            cudaError_t e = cudaFuncSetAttribute(s.fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 static_cast<int>(s.smem));
            if (e != cudaSuccess) return e;
        } else {
            s.fn = qg_kernel_fn(k);
            s.threads = qg_kernel_threads();
            s.smem = 0;
        }
        int bps = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, s.fn, s.threads, s.smem);
        if (e != cudaSuccess) return e;
        s.blocks_per_sm = std::max(1, bps);
    }
    return cudaSuccess;
}

const KernelShape &kernel_shape(int kid) { return g_shapes[kid]; }

uint64_t kernel_tile_starts(int kid, const PlanDev &hdr) {
    return so_kid(kid) ? so_tile_starts() : hdr.tile_starts;
}

uint64_t kernel_ntiles(int kid, const PlanDev &hdr, const uint8_t *text, uint64_t n) {
    if (n < hdr.m) return 0;
    const uint64_t T = kernel_tile_starts(kid, hdr);
    if (so_kid(kid)) {
        const uint64_t o = reinterpret_cast<uintptr_t>(text) & 15u;
        return (o + n + T - 1) / T;  // staged sub-tiles of end positions
    }
    return (n - hdr.m + 1 + T - 1) / T;
}

void count_launches(uint64_t k) { lib().launches.fetch_add(k, std::memory_order_relaxed); }

cudaError_t kernel_launch(int kid, const LaunchArgs &a, int grid, cudaStream_t stream) {
    const KernelShape &s = g_shapes[kid];
    void *args[] = {const_cast<LaunchArgs *>(&a)};
    cudaError_t e = cudaLaunchKernel(s.fn, dim3(grid), dim3(s.threads), args, s.smem, stream);
    if (e == cudaSuccess) lib().launches.fetch_add(1, std::memory_order_relaxed);
    return e;
}

}  // namespace smgpu

// ---------------------------------------------------------------- C ABI

namespace {

sm_status search_plan_impl(const sm_plan *plan, const uint8_t *text, uint64_t n, uint64_t *out_pos,
                           uint64_t cap, uint64_t *out_count, cudaStream_t stream) {
    if (!query_ok(text, n, plan, out_pos, cap, out_count)) return SM_EINVAL;
    sm_status st = ensure_init();
    if (st != SM_OK) return st;
    const uint64_t units = kernel_ntiles(plan->kid, plan->hdr, text, n);
    if (units == 0) {
        SM_TRY_CUDA(cudaMemsetAsync(out_count, 0, sizeof(uint64_t), stream));
        return SM_OK;
    }
    const uint32_t per =
        balanced_per(units, plan_per(plan, std::max(sub_per_item(plan->kid, units, solo_rounds(plan)),
                                                    plan->min_units)));
    const uint64_t ntiles = (units + per - 1) / per;
    const int grid = grid_for(plan->kid, ntiles);
    const size_t reset = align16(kTicketBytes + ntiles * sizeof(uint64_t));
    const size_t spill = so_kid(plan->kid) ? static_cast<size_t>(grid) * so_spill_bytes() : 0;
    uint8_t *ws = nullptr;
    st = get_workspace(stream, reset + spill, &ws);
    if (st != SM_OK) return st;
    SM_TRY_CUDA(cudaMemsetAsync(ws, 0, reset, stream));
    LaunchArgs a{};
    a.nq = 1;
    a.one.text = text;
    a.one.n = n;
    a.one.plan = plan->dev;
    a.one.out_pos = out_pos;
    a.one.cap = cap;
    a.one.out_count = out_count;
    a.one.state = reinterpret_cast<uint64_t *>(ws + kTicketBytes);
    a.one.ntiles = ntiles;
    a.one.first_ticket = 0;
    a.one.nsub = units;
    a.one.sub_per_item = per;
    a.ticket = reinterpret_cast<unsigned long long *>(ws);
    a.total = ntiles;
    a.err = lib().err;
    a.spill = spill ? ws + reset : nullptr;
    SM_TRY_CUDA(kernel_launch(plan->kid, a, grid, stream));
    return SM_OK;
}

// Host-side layout of a batch's device structures at `base` (may be null
// when only the size is wanted): claim counters | look-back words |
// descriptors | zero-count list | flag spill area.  Fills b->groups and the
// host copies of the descriptor and zero arrays.
struct BatchLayout {
    size_t bytes = 0;
    size_t desc_off = 0;
    size_t zero_off = 0;
    size_t pack_off = 0;
    std::vector<QueryDev> desc;
    std::vector<uint64_t *> zero;
    std::vector<uint8_t> packs;  // PackPlan blocks, MP_PLAN_BYTES each
    size_t tmap_off = 0;
    std::vector<uint64_t> tmap;  // ticket maps of the groups that have one, back to back
};

// Texts at least this long are worth reading once for all the queries of
// a launch that scan them (their items interleaved by text position);
// shorter texts stay in L2 across queries anyway.
constexpr uint64_t kShareTextBytes = uint64_t(32) << 20;

// Ticket map of one launch group (LaunchArgs::tmap): appends its entries to
// `out` and returns true, or returns false (plain query-by-query tickets)
// when no long text is shared by two of its queries.  Entry order: by text,
// then by the byte offset where the item starts in the text, then by query;
// each query's items stay in increasing order.  items[i], unit_bytes[i] and
// per[i]: work items, bytes per unit and units per item of the group's
// i-th query.
bool ticket_map(const std::vector<const uint8_t *> &text, const std::vector<uint64_t> &n,
                const std::vector<uint64_t> &items, const std::vector<uint64_t> &unit_bytes,
                const std::vector<uint32_t> &per, std::vector<uint64_t> *out) {
    std::map<std::pair<const uint8_t *, uint64_t>, uint32_t> users;
    bool shared = false;
    for (size_t i = 0; i < text.size(); ++i)
        if (n[i] >= kShareTextBytes && ++users[{text[i], n[i]}] >= 2) shared = true;
    if (!shared || text.size() >= (1u << 24)) return false;
    struct E {
        const uint8_t *t;
        uint64_t start;
        uint32_t q;
        uint64_t item;
    };
    std::vector<E> es;
    for (size_t i = 0; i < text.size(); ++i)
        for (uint64_t k = 0; k < items[i]; ++k)
            es.push_back(E{text[i], k * per[i] * unit_bytes[i], static_cast<uint32_t>(i), k});
    std::stable_sort(es.begin(), es.end(), [](const E &a, const E &b) {
        if (a.t != b.t) return a.t < b.t;
        if (a.start != b.start) return a.start < b.start;
        return a.q < b.q;
    });
    for (const E &e : es) out->push_back((static_cast<uint64_t>(e.q) << 40) | e.item);
    return true;
}

// A pattern can join a multi-pattern pack: Shift-And with a 1- or 2-byte
// mask table (m <= 16) and an alphabet-size hint with sigma^m >= 2^16, so
// that its occurrences are expected sparse (the packed scan rescans the
// 16-byte chunks that hold one).  For skewed texts the hint should be an
// effective alphabet size (see the Python package's hints module).
bool packable(const sm_plan *p) {
    if (p->kid != K_SO4Q && p->kid != K_SO6P && p->kid != K_SO8H && p->kid != K_SO16H) return false;
    if (p->sigma < 2) return false;
    return static_cast<double>(p->hdr.m) * std::log2(static_cast<double>(p->sigma)) >= 16.0;
}

// Lays a batch out at `base` (null: sizes only).  Queries are grouped by
// kernel, keeping input order inside a group.  With `pack`, packable
// queries on the same text (pointer and length) are first grouped into
// multi-pattern packs (first fit by decreasing m: at most 32 bits and
// MP_MAXK patterns a pack); a pack of one pattern stays a plain query.
sm_status batch_layout(const sm_query *qs, uint32_t nq, uint8_t *base, sm_batch *b, BatchLayout *L,
                       bool pack = true) {
    for (uint32_t i = 0; i < nq; ++i)
        if (!query_ok(qs[i].text, qs[i].n, qs[i].plan, qs[i].out_pos, qs[i].cap, qs[i].out_count))
            return SM_EINVAL;
    sm_status st = ensure_init();
    if (st != SM_OK) return st;
    std::vector<std::vector<uint32_t>> by_kid(K_COUNT);
    L->zero.clear();
    L->desc.clear();
    L->packs.clear();
    b->groups.clear();
    std::vector<uint64_t> units(nq), ntiles(nq);
    for (uint32_t i = 0; i < nq; ++i) {
        units[i] = kernel_ntiles(qs[i].plan->kid, qs[i].plan->hdr, qs[i].text, qs[i].n);
        if (units[i] == 0) L->zero.push_back(qs[i].out_count);
    }

    // ---- multi-pattern packs
    std::vector<std::vector<uint32_t>> packs;
    std::vector<char> in_pack(nq, 0);
    if (pack) {
        std::map<std::pair<uintptr_t, uint64_t>, std::vector<uint32_t>> by_text;
        for (uint32_t i = 0; i < nq; ++i)
            if (units[i] && packable(qs[i].plan))
                by_text[{reinterpret_cast<uintptr_t>(qs[i].text), qs[i].n}].push_back(i);
        for (auto &kv : by_text) {
            std::vector<uint32_t> &v = kv.second;
            if (v.size() < 2) continue;
            std::stable_sort(v.begin(), v.end(), [&](uint32_t x, uint32_t y) {
                return qs[x].plan->hdr.m > qs[y].plan->hdr.m;
            });
            std::vector<std::vector<uint32_t>> local;
            std::vector<uint32_t> bits;
            for (uint32_t i : v) {
                const uint32_t m = qs[i].plan->hdr.m;
                size_t j = 0;
                while (j < local.size() && (bits[j] + m > 32 || local[j].size() >= MP_MAXK)) ++j;
                if (j == local.size()) {
                    local.emplace_back();
                    bits.push_back(0);
                }
                local[j].push_back(i);
                bits[j] += m;
            }
            for (auto &pk : local) {
                if (pk.size() < 2) continue;
                for (uint32_t i : pk) in_pack[i] = 1;
                packs.push_back(std::move(pk));
            }
        }
    }

    uint64_t group_units[K_COUNT] = {};
    for (uint32_t i = 0; i < nq; ++i) {
        if (units[i] == 0 || in_pack[i]) continue;
        by_kid[qs[i].plan->kid].push_back(i);
        group_units[qs[i].plan->kid] += units[i];
    }
    for (const auto &pk : packs) group_units[K_SOMULTI] += units[pk[0]];
    uint32_t group_per[K_COUNT];
    for (int k = 0; k < K_COUNT; ++k) group_per[k] = sub_per_item(k, group_units[k]);
    std::vector<uint32_t> per_q(nq, 1);
    for (uint32_t i = 0; i < nq; ++i) {
        if (units[i] == 0 || in_pack[i]) continue;
        per_q[i] = balanced_per(units[i], plan_per(qs[i].plan, std::max(group_per[qs[i].plan->kid],
                                                                        qs[i].plan->min_units)));
        ntiles[i] = (units[i] + per_q[i] - 1) / per_q[i];
    }
    std::vector<uint32_t> per_pack(packs.size());
    std::vector<uint64_t> ntiles_pack(packs.size());
    for (size_t j = 0; j < packs.size(); ++j) {
        // At most 64 work items a pack: every item resolves one prefix per
        // pattern, so short items would spend their time on look-backs.
        const uint64_t u = units[packs[j][0]];
        const uint32_t floor_per = static_cast<uint32_t>(
            std::min<uint64_t>(so_max_sub(), std::max<uint64_t>(8, (u + 63) / 64)));
        per_pack[j] = balanced_per(u, std::max(group_per[K_SOMULTI], floor_per));
        ntiles_pack[j] = (u + per_pack[j] - 1) / per_pack[j];
    }

    uint64_t total_states = 0;
    size_t ndesc = 0;
    for (int k = 0; k < K_COUNT; ++k)
        for (uint32_t i : by_kid[k]) {
            total_states += ntiles[i];
            ++ndesc;
        }
    size_t nmembers = 0;
    for (size_t j = 0; j < packs.size(); ++j) {
        total_states += packs[j].size() * ntiles_pack[j];
        nmembers += packs[j].size();
    }
    ndesc += packs.size() + nmembers;  // pack heads, then the packed patterns' own queries
    const size_t states_off = kTicketBytes;
    L->desc_off = align16(states_off + total_states * sizeof(uint64_t));
    L->zero_off = align16(L->desc_off + ndesc * sizeof(QueryDev));
    L->pack_off = (L->zero_off + L->zero.size() * sizeof(uint64_t *) + 255) & ~size_t(255);
    size_t spill_need = 0;  // staged groups run one after another: they share one area
    for (int k = 0; k < K_COUNT; ++k) {
        if (!staged_kid(k)) continue;
        uint64_t t = 0;
        if (k == K_SOMULTI)
            for (uint64_t x : ntiles_pack) t += x;
        else
            for (uint32_t i : by_kid[k]) t += ntiles[i];
        if (t) spill_need = std::max(spill_need, static_cast<size_t>(grid_for(k, t)) * so_spill_bytes());
    }
    // Ticket maps (sizes first: entries are filled below, group by group).
    std::vector<std::vector<uint64_t>> maps;
    L->tmap.clear();
    {
        auto map_of = [&](const std::vector<uint32_t> &qidx, int k, bool is_pack) {
            std::vector<const uint8_t *> t;
            std::vector<uint64_t> nn, it, ub;
            std::vector<uint32_t> pr;
            for (size_t j = 0; j < qidx.size(); ++j) {
                const uint32_t i = is_pack ? packs[qidx[j]][0] : qidx[j];
                t.push_back(qs[i].text);
                nn.push_back(qs[i].n);
                it.push_back(is_pack ? ntiles_pack[qidx[j]] : ntiles[i]);
                ub.push_back(is_pack ? so_tile_starts() : kernel_tile_starts(k, qs[i].plan->hdr));
                pr.push_back(is_pack ? per_pack[qidx[j]] : per_q[i]);
            }
            std::vector<uint64_t> m;
            if (!ticket_map(t, nn, it, ub, pr, &m)) m.clear();
            return m;
        };
        for (int k = 0; k < K_COUNT; ++k) maps.push_back(by_kid[k].empty() ? std::vector<uint64_t>() : map_of(by_kid[k], k, false));
        std::vector<uint32_t> pk(packs.size());
        for (size_t j = 0; j < packs.size(); ++j) pk[j] = static_cast<uint32_t>(j);
        maps.push_back(packs.empty() ? std::vector<uint64_t>() : map_of(pk, K_SOMULTI, true));
    }
    size_t tmap_entries = 0;
    for (const auto &m : maps) tmap_entries += m.size();
    L->tmap_off = (L->pack_off + packs.size() * MP_PLAN_BYTES + 255) & ~size_t(255);
    const size_t spill_off = (L->tmap_off + tmap_entries * sizeof(uint64_t) + 255) & ~size_t(255);
    L->bytes = spill_off + spill_need + 16;
    L->desc.reserve(ndesc);
    uint64_t state_pos = 0;
    int gi = 0;
    auto add_group = [&](int k, size_t first_desc, uint32_t count, uint64_t tickets,
                         const std::vector<uint64_t> &map) -> sm_status {
        if (gi >= static_cast<int>(kTicketBytes / 8)) return SM_EINVAL;
        sm_batch::Group g{};
        g.kid = k;
        g.args.qs = reinterpret_cast<const QueryDev *>(base + L->desc_off) + first_desc;
        g.args.nq = count;
        if (count == 1) g.args.one = L->desc[first_desc];
        g.args.ticket = reinterpret_cast<unsigned long long *>(base) + gi;
        g.args.total = tickets;
        g.args.err = lib().err;
        g.args.spill = staged_kid(k) ? base + spill_off : nullptr;
        if (!map.empty()) {
            g.args.tmap = reinterpret_cast<const uint64_t *>(base + L->tmap_off) + L->tmap.size();
            L->tmap.insert(L->tmap.end(), map.begin(), map.end());
        }
        g.grid = grid_for(k, tickets);
        b->groups.push_back(g);
        ++gi;
        return SM_OK;
    };
    for (int k = 0; k < K_COUNT; ++k) {
        if (by_kid[k].empty()) continue;
        const size_t first_desc = L->desc.size();
        uint64_t ticket = 0;
        for (uint32_t i : by_kid[k]) {
            QueryDev d{};
            d.text = qs[i].text;
            d.n = qs[i].n;
            d.plan = qs[i].plan->dev;
            d.out_pos = qs[i].out_pos;
            d.cap = qs[i].cap;
            d.out_count = qs[i].out_count;
            d.state = reinterpret_cast<uint64_t *>(base + states_off) + state_pos;
            d.ntiles = ntiles[i];
            d.first_ticket = ticket;
            d.nsub = units[i];
            d.sub_per_item = per_q[i];
            ticket += ntiles[i];
            state_pos += ntiles[i];
            L->desc.push_back(d);
        }
        st = add_group(k, first_desc, static_cast<uint32_t>(by_kid[k].size()), ticket, maps[k]);
        if (st != SM_OK) return st;
    }
    if (!packs.empty()) {
        // Heads first (the kernel's queries), then the members.
        const size_t first_head = L->desc.size();
        const size_t first_member = first_head + packs.size();
        L->packs.assign(packs.size() * MP_PLAN_BYTES, 0);
        uint64_t ticket = 0;
        size_t mi = first_member;
        std::vector<QueryDev> members;
        members.reserve(nmembers);
        for (size_t j = 0; j < packs.size(); ++j) {
            const uint32_t h = packs[j][0];
            QueryDev d{};
            d.text = qs[h].text;
            d.n = qs[h].n;
            d.plan = reinterpret_cast<const PlanDev *>(base + L->pack_off + j * MP_PLAN_BYTES);
            d.ntiles = ntiles_pack[j];
            d.first_ticket = ticket;
            d.nsub = units[h];
            d.sub_per_item = per_pack[j];
            ticket += ntiles_pack[j];
            L->desc.push_back(d);
            PackPlan &P = *reinterpret_cast<PackPlan *>(L->packs.data() + j * MP_PLAN_BYTES);
            P.k = static_cast<uint32_t>(packs[j].size());
            uint32_t shift = 0;
            for (uint32_t t = 0; t < P.k; ++t) {
                const uint32_t i = packs[j][t];
                const sm_plan *pl = qs[i].plan;
                const uint32_t m = pl->hdr.m;
                P.shift[t] = static_cast<uint8_t>(shift);
                P.len[t] = static_cast<uint8_t>(m);
                P.I |= 1u << shift;
                P.F |= 1u << (shift + m - 1);
                P.maxm = std::max(P.maxm, m);
                for (uint32_t q = 0; q < m; ++q) P.table[pl->pattern[q]] |= 1u << (shift + q);
                P.member[t] = reinterpret_cast<const QueryDev *>(base + L->desc_off) + mi;
                QueryDev md{};
                md.text = qs[i].text;
                md.n = qs[i].n;
                md.plan = pl->dev;
                md.out_pos = qs[i].out_pos;
                md.cap = qs[i].cap;
                md.out_count = qs[i].out_count;
                md.state = reinterpret_cast<uint64_t *>(base + states_off) + state_pos;
                md.ntiles = ntiles_pack[j];
                md.nsub = units[h];
                md.sub_per_item = per_pack[j];
                state_pos += ntiles_pack[j];
                members.push_back(md);
                ++mi;
                shift += m;
            }
        }
        L->desc.insert(L->desc.end(), members.begin(), members.end());
        st = add_group(K_SOMULTI, first_head, static_cast<uint32_t>(packs.size()), ticket, maps[K_COUNT]);
        if (st != SM_OK) return st;
    }
    b->base = base;
    b->zero_list = reinterpret_cast<uint64_t **>(base + L->zero_off);
    b->nzero = static_cast<uint32_t>(L->zero.size());
    b->reset_bytes = L->desc_off;
    b->kernels = static_cast<uint32_t>(b->groups.size()) + (b->nzero ? 1u : 0u);
    return SM_OK;
}

// Copies a laid-out batch's descriptors, zero list and packs to `base`
// (pageable sources: each copy returns once its bytes are staged).
// Pinned host ring for batch uploads that must not block the host: a span
// is filled on the host, copied by cudaMemcpyAsync on the caller's stream,
// and reused only once an event recorded behind that copy has completed.
// (A copy from pageable memory may wait for the work already queued on the
// stream, which would keep the host from preparing the next batch while the
// GPU runs this one.)  Spans are handed out in ring order; a request that
// does not fit waits for the oldest spans it overlaps.  Larger requests than
// a quarter of the ring, or a ring that could not be allocated, use a plain
// copy.
class UploadRing {
  public:
    static UploadRing &get() {
        static UploadRing *R = new UploadRing();  // never destroyed: copies may be in flight at exit
        return *R;
    }
    cudaError_t copy(void *dst, const void *src, size_t bytes, cudaStream_t stream) {
        if (bytes == 0) return cudaSuccess;
        std::lock_guard<std::mutex> g(mu_);
        const size_t need = (bytes + 255) & ~size_t(255);
        if (!buf_ && !tried_) {
            tried_ = true;
            if (cudaHostAlloc(reinterpret_cast<void **>(&buf_), kCap, cudaHostAllocDefault) != cudaSuccess) {
                buf_ = nullptr;
                (void)cudaGetLastError();
            }
        }
        if (!buf_ || need > kCap / 4) return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, stream);
        while (!live_.empty() && cudaEventQuery(live_.front().ev) == cudaSuccess) {
            cudaEventDestroy(live_.front().ev);
            live_.pop_front();
        }
        (void)cudaGetLastError();  // cudaErrorNotReady from the query is not an error
        const size_t at = head_ + need <= kCap ? head_ : 0;
        // While any span in flight overlaps [at, at + need), wait for the
        // oldest one and drop it (older spans are waited for first).
        auto overlapped = [&] {
            for (const Span &o : live_)
                if (o.off < at + need && at < o.off + o.bytes) return true;
            return false;
        };
        while (overlapped()) {
            const Span &o = live_.front();
            cudaError_t e = cudaEventSynchronize(o.ev);
            cudaEventDestroy(o.ev);
            live_.pop_front();
            if (e != cudaSuccess) return e;
        }
        std::memcpy(buf_ + at, src, bytes);
        cudaError_t e = cudaMemcpyAsync(dst, buf_ + at, bytes, cudaMemcpyHostToDevice, stream);
        if (e != cudaSuccess) return e;
        cudaEvent_t ev;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(ev, stream);
        if (e != cudaSuccess) {
            cudaStreamSynchronize(stream);  // the span is free once the copy is done
            return e;
        }
        live_.push_back(Span{at, need, ev});
        head_ = at + need;
        return cudaSuccess;
    }

  private:
    static constexpr size_t kCap = size_t(64) << 20;
    struct Span {
        size_t off, bytes;
        cudaEvent_t ev;
    };
    std::mutex mu_;
    uint8_t *buf_ = nullptr;
    bool tried_ = false;
    size_t head_ = 0;
    std::deque<Span> live_;  // copies in flight, oldest first
};

sm_status batch_upload(const BatchLayout &L, uint8_t *base, cudaStream_t stream) {
    UploadRing &R = UploadRing::get();
    if (!L.desc.empty())
        SM_TRY_CUDA(R.copy(base + L.desc_off, L.desc.data(), L.desc.size() * sizeof(QueryDev), stream));
    if (!L.zero.empty())
        SM_TRY_CUDA(R.copy(base + L.zero_off, L.zero.data(), L.zero.size() * sizeof(uint64_t *), stream));
    if (!L.packs.empty()) SM_TRY_CUDA(R.copy(base + L.pack_off, L.packs.data(), L.packs.size(), stream));
    if (!L.tmap.empty())
        SM_TRY_CUDA(R.copy(base + L.tmap_off, L.tmap.data(), L.tmap.size() * sizeof(uint64_t), stream));
    return SM_OK;
}

// Builds a batch in its own device allocation (descriptors copied with
// blocking copies).
sm_status batch_build(const sm_query *qs, uint32_t nq, sm_batch *b, bool pack = true) {
    BatchLayout L;
    sm_status st = batch_layout(qs, nq, nullptr, b, &L, pack);
    if (st != SM_OK) return st;
    auto arena = std::make_shared<DevArena>();
    SM_TRY_CUDA(cudaMalloc(&arena->ptr, L.bytes));
    uint8_t *base = static_cast<uint8_t *>(arena->ptr);
    st = batch_layout(qs, nq, base, b, &L, pack);
    if (st != SM_OK) return st;
    st = batch_upload(L, base, nullptr);
    if (st != SM_OK) return st;
    SM_TRY_CUDA(cudaStreamSynchronize(nullptr));
    b->arena = arena;
    return SM_OK;
}

sm_status batch_enqueue(const sm_batch *b, cudaStream_t stream) {
    SM_TRY_CUDA(cudaMemsetAsync(b->base, 0, b->reset_bytes, stream));
    if (b->nzero) SM_TRY_CUDA(launch_zero_counts(b->zero_list, b->nzero, stream));
    for (const auto &g : b->groups) SM_TRY_CUDA(kernel_launch(g.kid, g.args, g.grid, stream));
    return SM_OK;
}

}  // namespace

extern "C" {

sm_status sm_prepare_ex(const uint8_t *pattern, uint32_t m, uint32_t sigma_hint,
                        const sm_config *config, sm_stream_t stream, sm_plan **out_plan) {
    if (!pattern || !out_plan || m == 0 || m > kMaxM) return SM_EINVAL;
    return prepare_many(pattern, &m, 1, sigma_hint, config, stream, out_plan);
}

sm_status sm_prepare(const uint8_t *pattern, uint32_t m, uint32_t sigma_hint, sm_stream_t stream,
                     sm_plan **out_plan) {
    return sm_prepare_ex(pattern, m, sigma_hint, nullptr, stream, out_plan);
}

sm_status sm_prepare_many(const uint8_t *patterns, const uint32_t *lengths, uint32_t count,
                          uint32_t sigma_hint, const sm_config *config, sm_stream_t stream,
                          sm_plan **out_plans) {
    if (count == 0) return SM_OK;
    if (!patterns || !lengths || !out_plans) return SM_EINVAL;
    return prepare_many(patterns, lengths, count, sigma_hint, config, stream, out_plans);
}

sm_status sm_plan_free(sm_plan *plan) {
    delete plan;  // the shared arena is released with its last plan
    return SM_OK;
}

sm_status sm_plan_free_many(sm_plan *const *plans, uint32_t count) {
    if (count == 0) return SM_OK;
    if (!plans) return SM_EINVAL;
    for (uint32_t i = 0; i < count; ++i) delete plans[i];
    return SM_OK;
}

sm_status sm_plan_info(const sm_plan *plan, sm_plan_desc *out) {
    if (!plan || !out) return SM_EINVAL;
    sm_plan_desc d{};
    d.m = plan->hdr.m;
    d.variant = plan->hdr.variant == VAR_SHIFTOR ? SM_VARIANT_SHIFTOR
                : plan->hdr.variant == VAR_QGRAM ? SM_VARIANT_QGRAM
                : plan->hdr.variant == VAR_DFA   ? SM_VARIANT_DFA
                                                 : SM_VARIANT_LINEAR;
    d.q = plan->hdr.q;
    d.word_bits = plan->hdr.word_bits;
    d.hist = plan->hdr.hist;
    d.tile_starts = static_cast<uint32_t>(kernel_tile_starts(plan->kid, plan->hdr));
    d.device_bytes = plan->hdr.bytes;
    d.kernel = static_cast<uint32_t>(plan->kid);
    *out = d;
    return SM_OK;
}

sm_status sm_plan_image(const uint8_t *pattern, uint32_t m, uint32_t sigma_hint, const sm_config *config,
                        void *image, size_t capacity, sm_plan_layout *layout) {
    if (!pattern || !layout || m == 0 || m > kMaxM) return SM_EINVAL;
    std::vector<uint8_t> blob;
    size_t at = 0;
    PlanDev h{};
    int kid = 0;
    uint32_t min_units = 1;
    const sm_status st = build_blob(pattern, m, sigma_hint, config, nullptr, &blob, &at, &h, &kid, &min_units);
    if (st != SM_OK) return st;
    sm_plan_layout d{};
    d.m = h.m;
    d.variant = h.variant == VAR_SHIFTOR ? SM_VARIANT_SHIFTOR
                : h.variant == VAR_QGRAM ? SM_VARIANT_QGRAM
                : h.variant == VAR_DFA   ? SM_VARIANT_DFA
                                         : SM_VARIANT_LINEAR;
    d.kernel = static_cast<uint32_t>(kid);
    d.bytes = h.bytes;
    d.q = h.q;
    d.s = h.s;
    d.word_bits = h.word_bits;
    d.hist = h.hist;
    d.tile_starts = static_cast<uint32_t>(kernel_tile_starts(kid, h));
    if (h.variant == VAR_SHIFTOR) {
        d.entry_bytes = so_entry_bytes(kid);
        d.off_masks = h.off_tbl;
    }
    d.off_pattern = h.off_pat;
    d.off_border = h.off_fail;
    if (h.variant == VAR_QGRAM) {
        d.off_qgram_bitmap = h.off_bitmap;
        d.bitmap_bits = h.bm_bits;
        d.off_qgram_slots = h.off_slots;
        d.slot_bits = h.slot_bits;
        d.off_qgram_offsets = h.off_offs;
    }
    d.off_classes_tab = h.off_cls;
    d.off_automaton = h.off_dfa;
    d.classes = h.classes;
    *layout = d;
    if (!image) return SM_OK;
    if (capacity < blob.size()) return SM_EINVAL;
    std::memcpy(image, blob.data(), blob.size());
    return SM_OK;
}

sm_status sm_search_plan(const sm_plan *plan, const uint8_t *text, uint64_t n, uint64_t *out_pos,
                         uint64_t cap, uint64_t *out_count, sm_stream_t stream) {
    return search_plan_impl(plan, text, n, out_pos, cap, out_count, stream);
}

sm_status sm_search(const uint8_t *text, uint64_t n, const uint8_t *pattern, uint32_t m,
                    uint64_t *out_pos, uint64_t cap, uint64_t *out_count, sm_stream_t stream) {
    if (!pattern || m == 0 || m > kMaxM) return SM_EINVAL;
    if (!out_count || !aligned8(out_count) || (n > 0 && !text)) return SM_EINVAL;
    if (cap > 0 && (!out_pos || !aligned8(out_pos))) return SM_EINVAL;
    Lib &L = lib();
    const std::string key(reinterpret_cast<const char *>(pattern), m);
    sm_plan *plan = nullptr;
    {
        std::lock_guard<std::mutex> g(L.mu);
        auto it = L.cache.find(key);
        if (it != L.cache.end()) plan = it->second;
    }
    if (!plan) {
        sm_status st = sm_prepare(pattern, m, 0, stream, &plan);
        if (st != SM_OK) return st;
        std::lock_guard<std::mutex> g(L.mu);
        if (L.cache.size() >= 4096) {
            cudaDeviceSynchronize();  // cached plans may be in use
            for (auto &kv : L.cache) delete kv.second;
            L.cache.clear();
        }
        auto ins = L.cache.emplace(key, plan);
        if (!ins.second) {
            delete plan;
            plan = ins.first->second;
        }
    }
    return search_plan_impl(plan, text, n, out_pos, cap, out_count, stream);
}

sm_status sm_search_batch(const sm_query *queries, uint32_t nq, sm_stream_t stream) {
    if (nq == 0) return SM_OK;
    if (!queries) return SM_EINVAL;
    sm_batch b;
    sm_status st = batch_build(queries, nq, &b);
    if (st != SM_OK) return st;
    st = batch_enqueue(&b, stream);
    if (st != SM_OK) return st;
    // The batch's device memory must outlive the enqueued work.
    SM_TRY_CUDA(cudaStreamSynchronize(stream));
    return SM_OK;
}

sm_status sm_batch_workspace_size(const sm_query *queries, uint32_t nq, size_t *bytes) {
    if (!bytes || (nq > 0 && !queries)) return SM_EINVAL;
    if (nq == 0) {
        *bytes = 0;
        return SM_OK;
    }
    sm_batch b;
    BatchLayout L;
    sm_status st = batch_layout(queries, nq, nullptr, &b, &L);
    if (st == SM_OK) *bytes = L.bytes;
    return st;
}

sm_status sm_search_batch_async(const sm_query *queries, uint32_t nq, void *workspace,
                                size_t workspace_bytes, sm_stream_t stream) {
    if (nq == 0) return SM_OK;
    if (!queries || !workspace || (reinterpret_cast<uintptr_t>(workspace) & 255u)) return SM_EINVAL;
    sm_batch b;
    BatchLayout L;
    sm_status st = batch_layout(queries, nq, nullptr, &b, &L);
    if (st != SM_OK) return st;
    if (L.bytes > workspace_bytes) return SM_EINVAL;
    uint8_t *base = static_cast<uint8_t *>(workspace);
    st = batch_layout(queries, nq, base, &b, &L);
    if (st != SM_OK) return st;
    st = batch_upload(L, base, stream);
    if (st != SM_OK) return st;
    return batch_enqueue(&b, stream);
}

sm_status sm_batch_create(const sm_query *queries, uint32_t nq, uint32_t flags, sm_stream_t stream,
                          sm_batch **out_batch) {
    (void)stream;
    if (!out_batch || (nq > 0 && !queries)) return SM_EINVAL;
    sm_batch *b = new sm_batch();
    sm_status st = nq ? batch_build(queries, nq, b, !(flags & 2u)) : SM_OK;
    if (st != SM_OK) {
        delete b;
        return st;
    }
    if (nq && !(flags & 1u)) {
        cudaStream_t cs = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            st = batch_enqueue(b, cs);
            cudaGraph_t graph = nullptr;
            e = cudaStreamEndCapture(cs, &graph);
            if (e == cudaSuccess && st == SM_OK) {
                b->graph = graph;
                e = cudaGraphInstantiate(&b->exec, graph, 0);
            }
            // Capture counted the launches; replays count them again.
            lib().launches.fetch_sub(b->groups.size(), std::memory_order_relaxed);
        }
        if (cs) cudaStreamDestroy(cs);
        if (e != cudaSuccess || st != SM_OK) {
            if (b->exec) cudaGraphExecDestroy(b->exec);
            if (b->graph) cudaGraphDestroy(b->graph);
            delete b;
            return st != SM_OK ? st : from_cuda(e);
        }
    }
    *out_batch = b;
    return SM_OK;
}

sm_status sm_batch_launch(sm_batch *batch, sm_stream_t stream) {
    if (!batch) return SM_EINVAL;
    if (batch->groups.empty() && batch->nzero == 0) return SM_OK;
    if (batch->exec) {
        SM_TRY_CUDA(cudaGraphLaunch(batch->exec, stream));
        lib().launches.fetch_add(batch->groups.size(), std::memory_order_relaxed);
        return SM_OK;
    }
    return batch_enqueue(batch, stream);
}

sm_status sm_batch_free(sm_batch *batch) {
    if (!batch) return SM_OK;
    if (batch->exec) cudaGraphExecDestroy(batch->exec);
    if (batch->graph) cudaGraphDestroy(batch->graph);
    delete batch;
    return SM_OK;
}

sm_status sm_tuning_set(const sm_config *entries, uint32_t count) {
    if (!entries || count != SM_TUNE_M_BUCKETS * SM_TUNE_S_BUCKETS) return SM_EINVAL;
    Lib &L = lib();
    std::lock_guard<std::mutex> g(L.mu);
    std::memcpy(L.tuning, entries, sizeof(L.tuning));
    return SM_OK;
}

sm_status sm_tuning_get(sm_config *entries, uint32_t count) {
    if (!entries || count != SM_TUNE_M_BUCKETS * SM_TUNE_S_BUCKETS) return SM_EINVAL;
    Lib &L = lib();
    std::lock_guard<std::mutex> g(L.mu);
    std::memcpy(entries, L.tuning, sizeof(L.tuning));
    return SM_OK;
}

sm_status sm_tuning_reset(void) {
    Lib &L = lib();
    std::lock_guard<std::mutex> g(L.mu);
    std::memset(L.tuning, 0, sizeof(L.tuning));
    return SM_OK;
}

sm_status sm_sync(sm_stream_t stream) {
    sm_status st = ensure_init();
    if (st != SM_OK) return st;
    SM_TRY_CUDA(cudaStreamSynchronize(stream));
    uint32_t err = 0;
    SM_TRY_CUDA(cudaMemcpy(&err, lib().err, sizeof(err), cudaMemcpyDeviceToHost));
    if (err) {
        SM_TRY_CUDA(cudaMemset(lib().err, 0, sizeof(err)));
        return SM_ETIMEOUT;
    }
    return SM_OK;
}

uint64_t sm_kernel_launches(void) { return lib().launches.load(); }

namespace smgpu {
namespace {

// One warp resolves look-back word 1 whose predecessor (word 0) stays
// empty: the bounded wait runs out, records ERR_TIMEOUT and returns.
__global__ void selftest_wait_kernel(uint64_t *state, uint32_t *err) {
    bool ok = true;
    lookback_resolve(state, 1, 0, err, &ok);
}

}  // namespace
}  // namespace smgpu

sm_status sm_selftest_wait(sm_stream_t stream) {
    sm_status st = ensure_init();
    if (st != SM_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint8_t *ws = nullptr;
    st = get_workspace(s, 256, &ws);
    if (st != SM_OK) return st;
    uint64_t *state = reinterpret_cast<uint64_t *>(ws);
    SM_TRY_CUDA(cudaMemsetAsync(state, 0, 2 * sizeof(uint64_t), s));
    smgpu::selftest_wait_kernel<<<1, 32, 0, s>>>(state, lib().err);
    SM_TRY_CUDA(cudaGetLastError());
    return SM_OK;
}

sm_status sm_shutdown(void) {
    Lib &L = lib();
    std::lock_guard<std::mutex> g(L.mu);
    if (!L.inited) return SM_OK;
    cudaDeviceSynchronize();
    for (auto &kv : L.ws)
        if (kv.second.mem) cudaFree(kv.second.mem);
    L.ws.clear();
    for (auto &kv : L.cache) delete kv.second;
    L.cache.clear();
    return SM_OK;
}

const char *sm_strerror(sm_status status) {
    switch (status) {
        case SM_OK: return "success";
        case SM_EINVAL: return "invalid argument";
        case SM_ENOMEM: return "out of memory";
        case SM_ECUDA: return "CUDA runtime error";
        case SM_ETIMEOUT: return "bounded device wait timed out";
        case SM_ETRUNC: return "more occurrences than output capacity";
    }
    return "unknown status";
}

sm_status sm_gen_text(uint8_t *out, uint64_t start, uint64_t count, uint64_t key, uint32_t sigma,
                      const uint32_t *thresholds, uint32_t nthr, const uint8_t *byte_map,
                      sm_stream_t stream) {
    if (count && !out) return SM_EINVAL;
    if (sigma == 0 && (!thresholds || nthr == 0 || nthr > 255)) return SM_EINVAL;
    if (sigma > 256) return SM_EINVAL;
    sm_status st = ensure_init();
    if (st != SM_OK) return st;
    SM_TRY_CUDA(launch_gen_text(out, start, count, key, sigma, thresholds, nthr, byte_map, stream));
    lib().launches.fetch_add(count ? 1 : 0, std::memory_order_relaxed);
    return SM_OK;
}

}  // extern "C"
