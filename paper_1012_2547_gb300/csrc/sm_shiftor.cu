// Bit-parallel scan for patterns of up to 64 bytes.
//
// The method is the bit-parallel simulation of the nondeterministic
// Morris-Pratt automaton (Shift-Or / Shift-And, Fig. 3 and Section 1: one
// bit per pattern symbol, O(n ceil(m/w)) time for word size w).  This file
// uses the Shift-And polarity: after reading text byte t[e], bit j of the
// state D is 1 iff t[e-j..e] = p[0..j]; the update is
//     D <- ((D << 1) | 1) & B[t[e]],   bit j of B[c] = (p[j] == c),
// and an occurrence ends at e iff bit m-1 of D is 1 (it starts at e-m+1).
//
// GB300 mapping
//   * One warp per block; 20 blocks per SM.  A warp claims work items
//     (query, item) from a device counter; an item is `sub_per_item`
//     consecutive sub-tiles of 32 * 144 end positions whose bytes (plus the
//     64 bytes before them) are staged HBM -> shared memory by one
//     cp.async.bulk (TMA 1-D copy) on an mbarrier, double-buffered so the
//     next sub-tile streams in while this one is scanned.
//   * Lane l scans its own 144-byte segment, one 128-bit shared load per 16
//     bytes (144 is an odd multiple of 16, so the eight lanes of a
//     quarter-warp hit eight different bank groups).  For m <= 16 the start
//     state comes from a warm-up over the 8 or 16 bytes before the segment;
//     otherwise the lane starts from the empty state (its final state is
//     exact, as the segment is at least m bytes long) and lane l+1 takes it
//     (shuffle) to extend only the partial matches it carries across the
//     boundary, which usually die within a byte or two.
//   * Byte tables with m <= 4 (m <= 6) take four (two) text bytes per state
//     update through shifted copies of the table (see so_step4).
//   * When bits m..m+15 of the state are spare (32-bit state and m <= 17,
//     64-bit state and m <= 49), B[c] has ones there, so those bits carry
//     the match flags of the last 16 positions: one shift per 16 bytes
//     yields all 16 flags (variant "H").  Otherwise the state is ORed into
//     an accumulator and a chunk with a match is re-scanned (variant "A").
//   * Per-lane counts -> warp scan -> hits kept per item in a spill area
//     (a position list while sparse, flag and offset words of dense
//     sub-tiles) -> decoupled look-back across the items of the query, one
//     item later -> coalesced copy to the output (capped by `cap`).
//
// Positions are handled in a "virtual" frame shifted by o = text & 15, so
// every staged sub-tile starts on a 16-byte boundary in memory.
#include <type_traits>

#include "sm_internal.h"

namespace smgpu {

namespace {

constexpr int SO_SEGC = 9;                 // 16-byte chunks per lane segment (odd)
constexpr int SO_S = SO_SEGC * 16;          // 144 bytes per lane (>= m for m <= 64)
constexpr uint32_t SO_T = 32 * SO_S;        // end positions per sub-tile (one warp)
constexpr uint32_t SO_LHALO = 64;           // bytes staged before the sub-tile (>= m-1)
constexpr uint32_t SO_BUF = SO_LHALO + SO_T;
// Staging ring: SO_NBUF - 1 sub-tiles in flight while one is scanned.  Two
// slots (9.3 KB a block) leave room for ~21 resident one-warp blocks per
// SM, whose scans hide the copy latency and each other's dependent steps;
// three slots (14 KB) allowed only 15 and scanned 8-16 % fewer bytes/s.
#ifndef SO_NBUF_SLOTS
#define SO_NBUF_SLOTS 2
#endif
constexpr int SO_NBUF = SO_NBUF_SLOTS;
// Hits of one work item kept in shared memory (two buffers).  Zero: every
// hit goes to the spill area (L2-resident), which leaves the shared memory
// to the staging ring and lets 15 one-warp blocks share an SM.
#ifndef SO_HIT_SLOTS
#define SO_HIT_SLOTS 0
#endif
constexpr int SO_HITS = SO_HIT_SLOTS;
constexpr uint32_t SO_MAX_SUB = 64;         // most sub-tiles per work item
// A spilled sub-tile: per lane its flags as 5 words (two chunks each, see
// so_flag_word) and its offset word (exclusive offset | hit count << 16),
// word w of lane l at [w * 32 + l].
constexpr uint32_t SO_SUB_WORDS = 6;
constexpr uint32_t SO_SUB_FLAGS = SO_SUB_WORDS * 32 * 4;
// Spill area of one item: a list of item-relative positions (4 bytes per
// hit: cheaper than a sub-tile's flag and offset words below SO_SUB_FLAGS / 4
// hits), then the flag and offset words of the sub-tiles that follow once
// the list is full or a sub-tile is denser than that.
constexpr uint32_t SO_SPILL_POS = 4096;
// (+256: with an item stride of exactly 64 KiB the packed kernel compiled
// to 111 registers instead of 94.)
constexpr uint32_t SO_SPILL_ITEM = SO_SPILL_POS * 4 + SO_MAX_SUB * SO_SUB_FLAGS + 256;
constexpr uint32_t SO_SPILL_BYTES = 2 * SO_SPILL_ITEM;          // per block (two items)

// Dynamic shared memory of a block: the staging ring, the item hit buffer,
// mbarriers and two run-time constants.  The mask table is a static
// __shared__ array, so a byte value is directly its (immediate-offset)
// address.
template <typename Entry>
struct SOLayout {
    static constexpr uint32_t HITS_OFF = SO_NBUF * SO_BUF;
    static constexpr uint32_t BAR_OFF = HITS_OFF + 2 * SO_HITS * 4;  // two hit buffers
    static constexpr uint32_t CONST_OFF = BAR_OFF + 8 * SO_NBUF;  // multipliers the compiler cannot fold
    static constexpr uint32_t BYTES = CONST_OFF + 16;
};

// Table entry at shared address `addr`, zero-extended by the load itself
// (volatile: never merged across a table reload).
template <typename Entry>
__device__ __forceinline__ typename std::conditional<sizeof(Entry) == 8, uint64_t, uint32_t>::type
lds_entry(uint32_t addr) {
    if constexpr (sizeof(Entry) == 1) {
        uint32_t v;
        asm volatile("ld.shared.u8 %0, [%1];" : "=r"(v) : "r"(addr));
        return v;
    } else if constexpr (sizeof(Entry) == 2) {
        uint32_t v;
        asm volatile("ld.shared.u16 %0, [%1];" : "=r"(v) : "r"(addr));
        return v;
    } else if constexpr (sizeof(Entry) == 4) {
        uint32_t v;
        asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
        return v;
    } else {
        uint64_t v;
        asm volatile("ld.shared.u64 %0, [%1];" : "=l"(v) : "r"(addr));
        return v;
    }
}

// Signed byte at shared address `addr`: bits 8..31 copy bit 7.
__device__ __forceinline__ uint32_t lds_s8(uint32_t addr) {
    int32_t v;
    asm volatile("ld.shared.s8 %0, [%1];" : "=r"(v) : "r"(addr));
    return static_cast<uint32_t>(v);
}

// Run-time constants of the scan steps: values the compiler cannot fold, so
// that the state's shift stays an IMAD on the FMA pipe.
struct SOK {
    uint32_t tb;       // shared address of the mask table B (256-aligned)
    uint32_t tb1;      // multi-byte steps: shifted-mask tables B1, B2, B3
    uint32_t tb2;      //   (B_k[c] = (B[c] << k) | (2^k - 1)), 256-aligned
    uint32_t tb3;
    uint32_t two;      // 2
    uint32_t four;     // 4
    uint32_t sixteen;  // 16
    uint32_t esz;      // bytes per table entry
};

// Table entry of byte b of word x, widened to the state (zero above the
// entry's own bits).  `tb` is the table's shared address, 256-aligned: for
// byte entries one PRMT puts the text byte under tb's upper bytes, which is
// the entry's address; wider entries take c * esz + tb (esz loaded at run
// time, so the multiply-add stays on the FMA pipe).
template <typename Word, typename Entry>
__device__ __forceinline__ Word so_entry_b(uint32_t x, int b, uint32_t tb, uint32_t esz) {
    uint32_t addr;
    if (sizeof(Entry) == 1) addr = __byte_perm(x, tb, 0x7650u | b);
    else addr = __byte_perm(x, 0u, 0x4440u | b) * esz + tb;
    return Word(lds_entry<Entry>(addr));
}

// Mask of byte value c (slow paths): entry plus ones above its own bits.
template <typename Word, typename Entry>
__device__ __forceinline__ Word so_mask(uint32_t tb, uint32_t c, uint32_t esz) {
    constexpr Word HIGH = sizeof(Entry) < sizeof(Word) ? (~Word(0) << (8 * sizeof(Entry))) : Word(0);
    return Word(lds_entry<Entry>(tb + c * esz)) | HIGH;
}

// One Shift-And step D <- ((D << 1) | 1) & B[c] as a single 3-input
// majority: with D2 = D << 1 (bit 0 clear), e the zero-extended entry and
// K = (ones above the entry's bits) | 1,
//   maj(D2, e, K) = (D2 & e) | (K & (D2 | e))
// gives D2 & e on the entry's bits 1.., e on bit 0 (D2 has none) and D2
// above the entry (e has none there) -- exactly the update with the ones
// the table leaves out.  For a 32-bit state the shift is D * two (two
// loaded at run time: an FMA-pipe IMAD next to the ALU's PRMT and LOP3).
template <typename Word, typename Entry>
__device__ __forceinline__ Word so_update(Word D, Word e, uint32_t two) {
    constexpr Word HIGH = sizeof(Entry) < sizeof(Word) ? (~Word(0) << (8 * sizeof(Entry))) : Word(0);
    constexpr Word K = HIGH | Word(1);
    const Word D2 = sizeof(Word) == 4 ? static_cast<Word>(static_cast<uint32_t>(D) * two) : (D << 1);
    return (D2 & e) | (K & (D2 | e));
}

// Four steps on the bytes of x, STEP text bytes per state update (byte
// tables and a 32-bit state for STEP > 1).  Composing k single steps gives
//   D <- ((D << k) | (2^k - 1)) & B_{k-1}[c_1] & ... & B_1[c_{k-1}] & B[c_k],
//   B_j[c] = (B[c] << j) | (2^j - 1),
// where each table holds one byte per entry with every bit >= m of B (so
// >= m + j of B_j) set.  While m + STEP - 1 <= 7, bit 7 of every table
// byte is set, so a sign-extending load supplies the ones above the byte:
//   STEP 2 (m <= 6): per two bytes two PRMT, two loads, one IMAD, one LOP3;
//   STEP 4 (m <= 4): per four bytes four PRMT, four loads, one IMAD and two
//     LOP3, and the chain through D is one IMAD and one LOP3 per four bytes
//     (the tables' AND is off the chain).
template <typename Word, typename Entry, int STEP>
__device__ __forceinline__ void so_step4(Word &D, uint32_t x, const SOK &k) {
    if constexpr (STEP == 4) {
        static_assert(sizeof(Word) == 4 && sizeof(Entry) == 1, "quad steps use byte tables and a 32-bit state");
        const uint32_t e3 = lds_s8(__byte_perm(x, k.tb3, 0x7650u));
        const uint32_t e2 = lds_s8(__byte_perm(x, k.tb2, 0x7651u));
        const uint32_t e1 = lds_s8(__byte_perm(x, k.tb1, 0x7652u));
        const uint32_t e0 = lds_s8(__byte_perm(x, k.tb, 0x7653u));
        const uint32_t t = e3 & e2 & e1;
        D = (static_cast<uint32_t>(D) * k.sixteen + 15u) & t & e0;
    } else if constexpr (STEP == 2) {
        static_assert(sizeof(Word) == 4 && sizeof(Entry) == 1, "pair steps use byte tables and a 32-bit state");
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint32_t e1 = lds_s8(__byte_perm(x, k.tb1, 0x7650u | (2 * h)));
            const uint32_t e2 = lds_s8(__byte_perm(x, k.tb, 0x7650u | (2 * h + 1)));
            D = (static_cast<uint32_t>(D) * k.four + 3u) & e1 & e2;
        }
    } else {
#pragma unroll
        for (int b = 0; b < 4; ++b)
            D = so_update<Word, Entry>(D, so_entry_b<Word, Entry>(x, b, k.tb, k.esz), k.two);
    }
}

// Exact flags of one 16-byte chunk (bit 15-b <=> an occurrence ends at byte
// b of the chunk), re-scanned from the state at the chunk start.
template <typename Word, typename Entry>
__device__ __noinline__ uint32_t so_chunk_flags(Word D, const uint8_t *chunk, uint32_t tb,
                                                uint32_t m, uint32_t esz) {
    uint32_t f = 0;
#pragma unroll 1
    for (int b = 0; b < 16; ++b) {
        D = ((D << 1) | Word(1)) & so_mask<Word, Entry>(tb, chunk[b], esz);
        f |= static_cast<uint32_t>((D >> (m - 1)) & Word(1)) << (15 - b);
    }
    return f;
}

// Bits r of a chunk starting at segment byte cb whose position cb + 15 - r
// lies in [elo, ehi).
__device__ __forceinline__ uint32_t range_mask16(int cb, int elo, int ehi) {
    const int lo = max(cb + 16 - ehi, 0);
    const int hi = min(cb + 15 - elo, 15);
    if (lo > hi) return 0u;
    return ((2u << hi) - 1u) & ~((1u << lo) - 1u);
}

// Local scan of one lane segment from the empty state.  F[c] bit r flags an
// occurrence ending at segment byte 16c + 15 - r; returns the final state,
// which is exact because the segment is at least m bytes long.
template <typename Word, typename Entry, bool HIST, int STEP>
__device__ __forceinline__ Word so_local(const uint8_t *seg, Word D, const SOK &k, uint32_t m,
                                         uint32_t (&F)[SO_SEGC]) {
#pragma unroll
    for (int c = 0; c < SO_SEGC; ++c) {
        const uint4 w = *reinterpret_cast<const uint4 *>(seg + 16 * c);
        if (HIST) {
            so_step4<Word, Entry, STEP>(D, w.x, k);
            so_step4<Word, Entry, STEP>(D, w.y, k);
            so_step4<Word, Entry, STEP>(D, w.z, k);
            so_step4<Word, Entry, STEP>(D, w.w, k);
            F[c] = static_cast<uint32_t>(D >> (m - 1)) & 0xFFFFu;
        } else {
            const Word Ds = D;
            Word A = 0;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint32_t x = q == 0 ? w.x : q == 1 ? w.y : q == 2 ? w.z : w.w;
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    D = so_update<Word, Entry>(D, so_entry_b<Word, Entry>(x, b, k.tb, k.esz), k.two);
                    A |= D;
                }
            }
            F[c] = ((A >> (m - 1)) & Word(1))
                       ? so_chunk_flags<Word, Entry>(Ds, seg + 16 * c, k.tb, m, k.esz)
                       : 0u;
        }
    }
    return D;
}

// State at the segment start from the WARM (8 or 16) bytes before it, run
// from the empty state: exact for every bit below WARM, hence for all bits
// that matter when m - 1 <= WARM.  Replaces the fix-up for short patterns.
template <typename Word, typename Entry, int WARM, int STEP>
__device__ __forceinline__ Word so_warmup(const uint8_t *seg, const SOK &k) {
    Word D = 0;
    if (WARM == 8) {
        const uint2 w = *reinterpret_cast<const uint2 *>(seg - 8);
        so_step4<Word, Entry, STEP>(D, w.x, k);
        so_step4<Word, Entry, STEP>(D, w.y, k);
    } else if (WARM == 16) {
        const uint4 w = *reinterpret_cast<const uint4 *>(seg - 16);
        so_step4<Word, Entry, STEP>(D, w.x, k);
        so_step4<Word, Entry, STEP>(D, w.y, k);
        so_step4<Word, Entry, STEP>(D, w.z, k);
        so_step4<Word, Entry, STEP>(D, w.w, k);
    }
    return D;
}

// Occurrences that start before the segment and end in its first m-1
// bytes.  X holds the partial matches inherited from the true state before
// the segment (bits 0..m-2); they are extended byte by byte until none
// survives.  Flags are merged into F; returns nothing.
template <typename Word, typename Entry>
__device__ __forceinline__ void so_fixup(const uint8_t *seg, uint32_t tb, uint32_t m,
                                         uint32_t esz, Word Dprev, uint32_t (&F)[SO_SEGC]) {
    const Word pm = (Word(1) << (m - 1)) - Word(1);
    Word X = Dprev & pm;
    if (!X) return;
    uint64_t extra = 0;
    for (uint32_t b = 0; X && b + 1 < m; ++b) {
        X = (X << 1) & so_mask<Word, Entry>(tb, seg[b], esz);
        extra |= static_cast<uint64_t>((X >> (m - 1)) & Word(1)) << b;
        X &= pm;
    }
#pragma unroll
    for (int c = 0; c < 4 && c < SO_SEGC; ++c)
        F[c] |= __brev(static_cast<uint32_t>(extra >> (16 * c)) & 0xFFFFu) >> 16;
}

// State after the m-1 bytes that end at `p` (exclusive), from empty.
template <typename Word, typename Entry>
__device__ __forceinline__ Word so_warm(const uint8_t *p, uint32_t tb, uint32_t m, uint32_t esz) {
    Word D = 0;
    for (uint32_t b = 0; b + 1 < m; ++b) D = ((D << 1) | Word(1)) & so_mask<Word, Entry>(tb, p[b], esz);
    return D;
}

// Keep positions e in [elo, ehi) of the segment and count them.
// (Whole warp.)  Lanes whose segment lies wholly inside the valid range --
// all of them except at the two ends of a text -- skip the masking.
__device__ __forceinline__ uint32_t so_mask_count(uint32_t (&F)[SO_SEGC], int elo, int ehi) {
    const bool full = elo == 0 && ehi == SO_S;
    if (!__all_sync(0xffffffffu, full)) {
#pragma unroll
        for (int c = 0; c < SO_SEGC; ++c)
            F[c] &= ehi <= elo ? 0u : range_mask16(16 * c, elo, ehi);
    }
    uint32_t any = 0;
#pragma unroll
    for (int c = 0; c < SO_SEGC; ++c) any |= F[c];
    uint32_t cnt = 0;
    if (any) {
#pragma unroll
        for (int c = 0; c < SO_SEGC; ++c) cnt += __popc(F[c]);
    }
    return cnt;
}

__device__ __forceinline__ uint32_t warp_excl_scan(uint32_t v, uint32_t *total) {
    const int lane = threadIdx.x & 31;
    uint32_t x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    *total = __shfl_sync(0xffffffffu, x, 31);
    return x - v;
}

// Stage sub-tile s (end positions [s*T, (s+1)*T) in the virtual frame) plus
// the 64 bytes before it into buffer `dst`.  Lane 0 only.
__device__ __forceinline__ void so_issue(uint8_t *dst, uint64_t *bar, const uint8_t *text, uint64_t n,
                                         uint64_t s) {
    const uint64_t o = reinterpret_cast<uintptr_t>(text) & 15u;
    const uint8_t *base = text - o;
    const uint64_t a = s * static_cast<uint64_t>(SO_T);
    const uint64_t lo = a >= SO_LHALO ? a - SO_LHALO : 0;
    const uint64_t vlim = (o + n + 15u) & ~uint64_t(15);
    const uint64_t hi = min(a + SO_T, vlim);
    const uint32_t bytes = static_cast<uint32_t>(hi - lo);
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(bar, bytes);
    bulk_g2s(dst + (SO_LHALO - (a - lo)), base + lo, bytes, bar);
}

__device__ __forceinline__ bool so_claim(const LaunchArgs &a, unsigned long long *t, uint32_t *qi,
                                         uint64_t *k) {
    *t = atomicAdd(a.ticket, 1ull);
    if (*t >= a.total) return false;
    resolve_ticket(a, *t, qi, k);
    return true;
}

// A scanned work item whose hits wait in one of the two hit buffers (and
// spill areas) until its prefix is known.  All fields are warp-uniform.
struct SOItem {
    uint32_t qi;
    uint64_t k, sb, se;       // item index, sub-tile range [sb, se)
    uint32_t count;           // hits of the item
    uint32_t buffered;        // hits in the shared buffer
    uint32_t listed;          // hits in the spill area's position list
    uint64_t flag_from;       // first sub-tile whose flag words were spilled (se: none)
};

// Loads plan P's mask table into shared memory unless it is there already.
// Byte tables also get NSHIFTED shifted tables B_j[c] = (B[c] << j) |
// (2^j - 1), j = 1..NSHIFTED, at tbl + 256 j.
template <typename Entry, int NSHIFTED>
__device__ __forceinline__ void so_table(const PlanDev *P, const PlanDev *&cur_plan, uint8_t *tbl,
                                         uint32_t &m) {
    if (P == cur_plan) return;
    __syncwarp();  // no lane still reads the old table
    const uint4 *src = reinterpret_cast<const uint4 *>(reinterpret_cast<const uint8_t *>(P) +
                                                       __ldg(&P->off_tbl));
    const int lane = threadIdx.x & 31;
    for (int c = lane; c < static_cast<int>(256 * sizeof(Entry) / 16); c += 32) {
        const uint4 v = __ldg(&src[c]);
        reinterpret_cast<uint4 *>(tbl)[c] = v;
#pragma unroll
        for (int j = 1; j <= NSHIFTED; ++j) {
            // Per byte (b << j) | (2^j - 1) within each 32-bit word: shift
            // the word, drop the bits carried across bytes, set every byte's
            // low j bits.
            const uint32_t K = 0x01010101u * ((1u << j) - 1u);
            const uint32_t HI = 0x01010101u * ((0xFFu << j) & 0xFFu);
            reinterpret_cast<uint4 *>(tbl + 256 * j)[c] =
                make_uint4(((v.x << j) & HI) | K, ((v.y << j) & HI) | K, ((v.z << j) & HI) | K,
                           ((v.w << j) & HI) | K);
        }
    }
    cur_plan = P;
    m = __ldg(&P->m);
    __syncwarp();
}

// Scan of one sub-tile staged at `buf` (its 64 preceding bytes included):
// flags of the lane's segment, masked to the valid ends.  `carry` is the
// exact state before the sub-tile (fix-up form only).
template <typename Word, typename Entry, bool HIST, int WARM, int STEP>
__device__ __forceinline__ uint32_t so_subtile(const uint8_t *buf, const SOK &k, uint32_t m, Word &carry,
                                               bool warm_carry, int elo, int ehi,
                                               uint32_t (&F)[SO_SEGC]) {
    const int lane = threadIdx.x & 31;
    const uint8_t *seg = buf + lane * SO_S;
    if (WARM) {
        so_local<Word, Entry, HIST, STEP>(seg, so_warmup<Word, Entry, WARM, STEP>(seg, k), k, m, F);
    } else {
        if (warm_carry && lane == 0) carry = so_warm<Word, Entry>(buf - (m - 1), k.tb, m, k.esz);
        const Word Dend = so_local<Word, Entry, HIST, 1>(seg, Word(0), k, m, F);
        Word Dprev = __shfl_up_sync(0xffffffffu, Dend, 1);
        if (lane == 0) Dprev = carry;
        so_fixup<Word, Entry>(seg, k.tb, m, k.esz, Dprev, F);
        carry = __shfl_sync(0xffffffffu, Dend, 31);
    }
    return so_mask_count(F, elo, ehi);
}

// Calls put(b) for every flagged byte b of a lane segment, b increasing.
// F[c] bit r flags byte 16c + 15 - r; one loop per 32 bytes, one iteration
// per hit.  Two forms (both exact; which one compiles better depends on
// the kernel around it, so each kernel takes the one measured faster):
//   MSB_FIRST: g = F[2w] << 16 | F[2w+1] (one PRMT) flags byte 32w + 31 - p
//     at bit p, so taking the highest set bit first (BFIND) yields the
//     bytes in increasing order without bit-reversing the flags;
//   otherwise: the two chunks' flags bit-reversed side by side, lowest set
//     bit first.
static_assert(SO_SEGC == 9, "so_emit packs 9 chunks of flags");
__device__ __forceinline__ uint32_t bfind_u32(uint32_t x) {
    uint32_t p;
    asm("bfind.u32 %0, %1;" : "=r"(p) : "r"(x));
    return p;
}
template <bool MSB_FIRST, typename Put>
__device__ __forceinline__ void so_emit(const uint32_t (&F)[SO_SEGC], Put put) {
#pragma unroll
    for (int w = 0; w < 5; ++w) {
        if constexpr (MSB_FIRST) {
            uint32_t g = 2 * w + 1 < SO_SEGC ? __byte_perm(F[2 * w + 1], F[2 * w], 0x5410u) : F[2 * w] << 16;
            while (g) {
                const uint32_t p = bfind_u32(g);
                g ^= 1u << p;
                put(32u * w + 31u - p);
            }
        } else {
            uint32_t q = (__brev(F[2 * w]) >> 16) | (2 * w + 1 < SO_SEGC ? __brev(F[2 * w + 1]) : 0u);
            while (q) {
                const uint32_t b = static_cast<uint32_t>(__ffs(q)) - 1u;
                q &= q - 1u;
                put(32u * w + b);
            }
        }
    }
}

// Flag word w of a lane segment: chunks 2w and 2w + 1 side by side (bit p
// flags byte 32w + 31 - p).
__device__ __forceinline__ uint32_t so_flag_word(const uint32_t (&F)[SO_SEGC], int w) {
    return 2 * w + 1 < SO_SEGC ? __byte_perm(F[2 * w + 1], F[2 * w], 0x5410u) : F[2 * w] << 16;
}

// so_emit over the 5 flag words of a segment (so_flag_word).
template <bool MSB_FIRST, typename Put>
__device__ __forceinline__ void so_emit_words(const uint32_t (&G)[5], Put put) {
#pragma unroll
    for (int w = 0; w < 5; ++w) {
        if constexpr (MSB_FIRST) {
            uint32_t g = G[w];
            while (g) {
                const uint32_t p = bfind_u32(g);
                g ^= 1u << p;
                put(32u * w + 31u - p);
            }
        } else {
            uint32_t q = __brev(G[w]);
            while (q) {
                const uint32_t b = static_cast<uint32_t>(__ffs(q)) - 1u;
                q &= q - 1u;
                put(32u * w + b);
            }
        }
    }
}

// Writes the flagged positions of a lane segment at out[idx...] (capped):
// idx0 + ex is the lane's first index, start0 the output value of sub-tile
// position 0.
template <bool MSB_FIRST>
__device__ __forceinline__ void so_write_flags(const uint32_t (&F)[SO_SEGC], uint32_t ex, uint64_t idx0,
                                               uint64_t cap, uint64_t *out, int64_t start0) {
    const uint64_t first = idx0 + ex;
    if (first >= cap) return;
    // 32-bit counter against the room left (a segment holds at most 144 hits).
    const uint64_t room64 = cap - first;
    const uint32_t room = room64 < 0xFFFFFFFFull ? static_cast<uint32_t>(room64) : 0xFFFFFFFFu;
    uint64_t *dst = out + first;
    const int64_t lane0 = start0 + static_cast<int64_t>(threadIdx.x & 31) * SO_S;
    uint32_t j = 0;
    so_emit<MSB_FIRST>(F, [&](uint32_t b) {
        if (j < room) dst[j] = static_cast<uint64_t>(lane0 + b);
        ++j;
    });
}

// One warp per block.  The warp claims work items (query, item); an item
// is `sub_per_item` consecutive sub-tiles of 32 * 144 end positions, staged
// by bulk copies through an SO_NBUF-slot ring.  Per sub-tile every lane
// scans its 144 bytes (after a warm-up over the bytes before it, or from
// the empty state plus a fix-up from the previous segment's exact state).
// Hits of an item go to shared memory (up to SO_HITS) and then to a
// per-block spill area, as a position list while they are sparse and as the
// sub-tiles' flag words once the list is full.  The item's count is
// published at once and the warp goes on to the next item; its prefix is
// resolved by decoupled look-back one item later -- by then every earlier
// item has been scanned, so the look-back rarely waits -- and the hits are
// copied out.  Two hit buffers and two spill areas alternate between the
// item being scanned and the item waiting for its prefix.  Without a spill
// area an item whose hits overflow the buffer is rescanned at write time.
template <typename Word, typename Entry, bool HIST, int WARM, int STEP = 1>
__global__ void __launch_bounds__(32) so_kernel(const __grid_constant__ LaunchArgs a) {
    using L = SOLayout<Entry>;
    static_assert(STEP == 1 || STEP == 2 || STEP == 4, "one, two or four text bytes per step");
    static_assert(STEP == 1 || (sizeof(Word) == 4 && sizeof(Entry) == 1 && HIST && WARM != 0),
                  "multi-byte steps need byte tables, a 32-bit state and the warm-up form");
    // Byte tables: B, then the shifted tables the steps use (B1 for STEP 1
    // and 2; B1, B2, B3 for STEP 4).
    constexpr int NSHIFTED = sizeof(Entry) != 1 ? 0 : STEP == 4 ? 3 : 1;
    constexpr bool EMIT_MSB = STEP > 1;  // so_emit form (measured per kernel)
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ __align__(256) uint8_t tbl[256 * sizeof(Entry) + 256 * NSHIFTED];
    const uint32_t tb = smem_addr(tbl);
    uint32_t *hits_base = reinterpret_cast<uint32_t *>(smem + L::HITS_OFF);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + L::BAR_OFF);
    const int lane = threadIdx.x;
    uint8_t *spill_base =
        a.spill ? a.spill + static_cast<size_t>(blockIdx.x) * SO_SPILL_BYTES : nullptr;

    unsigned long long t = 0;
    uint32_t qi = 0;
    uint64_t k = 0;
    volatile uint32_t *consts = reinterpret_cast<volatile uint32_t *>(smem + L::CONST_OFF);
    if (lane == 0) {
        consts[0] = 2u;
        consts[1] = static_cast<uint32_t>(sizeof(Entry));
        consts[2] = 4u;
        consts[3] = 16u;
        for (int b = 0; b < SO_NBUF; ++b) mbar_init(&bar[b], 1);
        fence_mbar_init();
        if (so_claim(a, &t, &qi, &k)) {
            const QueryDev &Q = query_of(a, qi);
            const uint64_t s0 = k * Q.sub_per_item;
            const uint64_t s1 = min(s0 + Q.sub_per_item, Q.nsub);
            for (int i = 0; i < SO_NBUF - 1 && s0 + i < s1; ++i)
                so_issue(smem + i * SO_BUF, &bar[i], Q.text, Q.n, s0 + i);
        } else {
            t = a.total;
        }
    }
    __syncwarp();
    t = __shfl_sync(0xffffffffu, t, 0);
    qi = __shfl_sync(0xffffffffu, qi, 0);
    k = __shfl_sync(0xffffffffu, k, 0);
    const SOK kk{tb, tb + 256u, tb + 512u, tb + 768u, consts[0], consts[2], consts[3], consts[1]};

    const PlanDev *cur_plan = nullptr;
    uint32_t m = 1;
    uint32_t parity = 0;  // bit b: parity of the next phase of bar[b]
    int cur = 0;          // ring slot holding the next sub-tile to scan
    int hb = 0;           // hit buffer / spill area of the item being scanned
    bool have_pending = false;
    SOItem pend{};

    // Prefix of the pending item, then its hits to the output (capped).
    auto write_pending = [&]() {
        const QueryDev &Q = query_of(a, pend.qi);
        bool ok;
        const uint64_t excl = lookback_resolve(Q.state, pend.k, pend.count, a.err, &ok);
        if (!ok) return;
        if (lane == 0 && pend.k + 1 == Q.ntiles) *Q.out_count = excl + pend.count;
        const uint64_t cap = Q.cap;
        if (excl >= cap) return;
        uint64_t *out = Q.out_pos;
        const uint8_t *const qtext = Q.text;
        const uint32_t pm = __ldg(&Q.plan->m);
        const int64_t o = static_cast<int64_t>(reinterpret_cast<uintptr_t>(qtext) & 15u);
        const int64_t shift = static_cast<int64_t>(pm) - 1 + o;  // end -> real start
        const int64_t ivstart = static_cast<int64_t>(pend.sb) * SO_T;
        const uint32_t *hits = hits_base + (hb ^ 1) * SO_HITS;
        const bool direct = pend.buffered + pend.listed == pend.count || pend.flag_from < pend.se;
        if (direct) {
            for (uint32_t r = lane; r < pend.buffered; r += 32) {
                const uint64_t idx = excl + r;
                if (idx < cap) out[idx] = static_cast<uint64_t>(ivstart + hits[r] - shift);
            }
            const uint8_t *spill = spill_base + (hb ^ 1) * SO_SPILL_ITEM;
            const uint32_t *list = reinterpret_cast<const uint32_t *>(spill);
            // Eight loads per lane before their stores: the compiler cannot
            // move a load of the list above a store to the output, so a
            // load-store loop would pay one L2 round trip per 32 hits.
            const uint64_t lbase = excl + pend.buffered;
            for (uint32_t r0 = 0; r0 < pend.listed; r0 += 32 * 8) {
                uint32_t v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const uint32_t r = r0 + 32u * u + lane;
                    v[u] = r < pend.listed ? list[r] : 0u;
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const uint32_t r = r0 + 32u * u + lane;
                    if (r < pend.listed && lbase + r < cap) out[lbase + r] = static_cast<uint64_t>(ivstart + v[u] - shift);
                }
            }
            const uint8_t *flags = spill + SO_SPILL_POS * 4;
            uint64_t run = excl + pend.buffered + pend.listed;
            // Flag-word sub-tiles (dense ones, or past a full list) go out
            // through the ring slot that no prefetch uses: the lanes write
            // their hits there as 16-bit sub-tile positions at their
            // exclusive offsets, and the warp copies them out with
            // consecutive lanes on consecutive output words, so a warp store
            // moves 256 contiguous bytes instead of 32 scattered words.  A
            // sub-tile with more hits than the slot holds as 16-bit words
            // (2,336) goes in two passes of 16 lanes (at most 2,304 hits
            // each).
            uint16_t *stage = reinterpret_cast<uint16_t *>(smem + (cur == 0 ? SO_NBUF - 1 : cur - 1) * SO_BUF);
            const uint32_t half = static_cast<uint32_t>(lane) >> 4;
            // The next sub-tile's flag and offset words are loaded before
            // this one's stores (software pipelining over the L2 latency);
            // the offsets were taken by the scan, so no count or warp scan
            // is redone here.
            uint32_t Gn[SO_SUB_WORDS];
            const uint32_t *fsrc = reinterpret_cast<const uint32_t *>(flags) + lane;
#pragma unroll
            for (int w = 0; w < static_cast<int>(SO_SUB_WORDS); ++w)
                Gn[w] = pend.flag_from < pend.se ? fsrc[w * 32] : 0u;
            for (uint64_t s = pend.flag_from; s < pend.se && run < cap; ++s) {
                uint32_t G[5];
                const bool more = s + 1 < pend.se;
                fsrc += SO_SUB_FLAGS / 4;
                const uint32_t E = Gn[5];
#pragma unroll
                for (int w = 0; w < 5; ++w) G[w] = Gn[w];
#pragma unroll
                for (int w = 0; w < static_cast<int>(SO_SUB_WORDS); ++w) Gn[w] = more ? fsrc[w * 32] : 0u;
                const uint32_t ex = E & 0xFFFFu;
                const uint32_t total = __shfl_sync(0xffffffffu, ex + (E >> 16), 31);
                const bool split = total > SO_BUF / 2;
                // First hit of pass 1: lanes 16..31 when split, else none.
                const uint32_t lo1 = split ? __shfl_sync(0xffffffffu, ex, 16) : total;
                const int64_t base = static_cast<int64_t>(s) * SO_T - shift;
#pragma unroll
                for (uint32_t h = 0; h < 2; ++h) {
                    if (h == 1 && !split) break;
                    const uint32_t lo = h ? lo1 : 0u;
                    const uint32_t cnt_h = h ? total - lo1 : lo1;
                    if (!split || half == h) {
                        uint16_t *d = stage + (ex - lo);
                        const uint32_t r0 = static_cast<uint32_t>(lane) * SO_S;
                        so_emit_words<EMIT_MSB>(G, [&](uint32_t b) { *d++ = static_cast<uint16_t>(r0 + b); });
                    }
                    __syncwarp();
                    const uint64_t at = run + lo;
                    const uint32_t nw = at >= cap ? 0u : cap - at < cnt_h ? static_cast<uint32_t>(cap - at) : cnt_h;
                    if constexpr (EMIT_MSB) {
                        // Four stage loads per lane ahead of their four
                        // stores (the multi-byte-step kernels, which the
                        // dense short patterns use).
                        uint64_t *dst = out + at;
                        uint32_t i = lane;
                        for (; i + 96 < nw; i += 128) {
                            const uint32_t v0 = stage[i], v1 = stage[i + 32], v2 = stage[i + 64],
                                           v3 = stage[i + 96];
                            dst[i] = static_cast<uint64_t>(base + v0);
                            dst[i + 32] = static_cast<uint64_t>(base + v1);
                            dst[i + 64] = static_cast<uint64_t>(base + v2);
                            dst[i + 96] = static_cast<uint64_t>(base + v3);
                        }
                        for (; i < nw; i += 32) dst[i] = static_cast<uint64_t>(base + stage[i]);
                    } else {
                        for (uint32_t i = lane; i < nw; i += 32) out[at + i] = static_cast<uint64_t>(base + stage[i]);
                    }
                    __syncwarp();
                }
                run += total;
            }
            return;
        }
        // Too many hits to buffer and no spill area: rescan the item in the
        // ring slot that no prefetch uses, writing each sub-tile's hits at
        // their final offsets.
        so_table<Entry, NSHIFTED>(Q.plan, cur_plan, tbl, m);
        const uint64_t qn = Q.n;
        const int64_t vlo = o + static_cast<int64_t>(m) - 1;
        const int64_t vhi = o + static_cast<int64_t>(qn);
        const int wb = cur == 0 ? SO_NBUF - 1 : cur - 1;
        uint64_t run = excl;
        Word carry = 0;
        for (uint64_t s = pend.sb; s < pend.se && run < cap; ++s) {
            if (lane == 0) so_issue(smem + wb * SO_BUF, &bar[wb], qtext, qn, s);
            const bool arrived = mbar_wait_bounded(&bar[wb], (parity >> wb) & 1u);
            parity ^= 1u << wb;
            if (!__all_sync(0xffffffffu, arrived)) {
                if (lane == 0) atomicOr(a.err, ERR_COPY);
                break;
            }
            const int64_t x = static_cast<int64_t>(s) * SO_T + lane * SO_S;
            const int elo = static_cast<int>(vlo - x > 0 ? vlo - x : int64_t(0));
            const int ehi = static_cast<int>(vhi - x < SO_S ? vhi - x : int64_t(SO_S));
            uint32_t F[SO_SEGC];
            const uint8_t *buf = smem + wb * SO_BUF + SO_LHALO;
            const bool first = s == pend.sb && s > 0;
            const uint32_t cnt = so_subtile<Word, Entry, HIST, WARM, STEP>(buf, kk, m, carry, first, elo, ehi, F);
            uint32_t total;
            const uint32_t ex = warp_excl_scan(cnt, &total);
            so_write_flags<EMIT_MSB>(F, ex, run, cap, out, static_cast<int64_t>(s) * SO_T - shift);
            run += total;
            __syncwarp();
        }
    };

    while (t < a.total) {
        const QueryDev &Q = query_of(a, qi);
        so_table<Entry, NSHIFTED>(Q.plan, cur_plan, tbl, m);
        // Query fields in registers: the mbarrier waits are compiler
        // barriers, after which descriptor fields would be reloaded.
        const uint8_t *const qtext = Q.text;
        const uint64_t qn = Q.n;
        const uint64_t qnsub = Q.nsub;
        const uint64_t sb = k * Q.sub_per_item;
        const uint64_t se = min(sb + Q.sub_per_item, qnsub);
        const int64_t o = static_cast<int64_t>(reinterpret_cast<uintptr_t>(qtext) & 15u);
        const int64_t vlo = o + static_cast<int64_t>(m) - 1;  // first valid end
        const int64_t vhi = o + static_cast<int64_t>(qn);     // one past the last
        const int64_t ivstart = static_cast<int64_t>(sb) * SO_T;
        uint32_t *hits = hits_base + hb * SO_HITS;
        uint8_t *spill = spill_base ? spill_base + hb * SO_SPILL_ITEM : nullptr;
        uint32_t *list = reinterpret_cast<uint32_t *>(spill);
        uint8_t *flags = spill ? spill + SO_SPILL_POS * 4 : nullptr;

        // ---- pass over the item's sub-tiles: count and keep hits
        uint32_t count = 0;
        Word carry = 0;
        bool failed = false;
        int pending = 0;           // prefetches in flight when the loop stops early
        int mode = 0;              // hits go to: 0 the shared buffer, 1 the list, 2 flag words
        uint32_t buffered = 0;     // hits in the shared buffer when the list began
        uint32_t listed = 0;       // hits in the list when the flag words began
        uint64_t flag_from = se;   // first sub-tile kept as flag words
        for (uint64_t s = sb; s < se; ++s) {
            const int ahead = cur == 0 ? SO_NBUF - 1 : cur - 1;  // (cur + SO_NBUF - 1) mod SO_NBUF
            if (lane == 0 && s + SO_NBUF - 1 < se)
                so_issue(smem + ahead * SO_BUF, &bar[ahead], qtext, qn, s + SO_NBUF - 1);
            const bool arrived = mbar_wait_bounded(&bar[cur], (parity >> cur) & 1u);
            parity ^= 1u << cur;
            if (!__all_sync(0xffffffffu, arrived)) {
                failed = true;
                pending = 0;
                for (int i = 1; i < SO_NBUF; ++i) pending += s + i < se;
                break;
            }
            const int64_t x = static_cast<int64_t>(s) * SO_T + lane * SO_S;
            // Only a text's first and last sub-tiles hold invalid ends.
            const bool edge = s == 0 || s + 1 == qnsub;
            const int elo = edge ? static_cast<int>(vlo - x > 0 ? vlo - x : int64_t(0)) : 0;
            const int ehi = edge ? static_cast<int>(vhi - x < SO_S ? vhi - x : int64_t(SO_S)) : SO_S;
            uint32_t F[SO_SEGC];
            const uint8_t *buf = smem + cur * SO_BUF + SO_LHALO;
            const bool first = s == sb && s > 0;
            const uint32_t cnt = so_subtile<Word, Entry, HIST, WARM, STEP>(buf, kk, m, carry, first, elo, ehi, F);
            uint32_t total = 0, ex = 0;
            if (__any_sync(0xffffffffu, cnt != 0)) ex = warp_excl_scan(cnt, &total);
            if (total != 0 && spill) {
                if (mode == 0 && count + total > SO_HITS) {
                    mode = 1;
                    buffered = count;
                }
                // Flag words cost SO_SUB_FLAGS bytes a sub-tile, the list 4 a
                // hit: a dense sub-tile, or a full list, switches to flags.
                if (mode == 1 && (count - buffered + total > SO_SPILL_POS || 4 * total > SO_SUB_FLAGS)) {
                    mode = 2;
                    listed = count - buffered;
                    flag_from = s;
                }
            }
            if (mode == 2) {
                // Keep this sub-tile's flag words and offsets for the write
                // phase.
                uint32_t *dst = reinterpret_cast<uint32_t *>(flags + (s - flag_from) * SO_SUB_FLAGS);
#pragma unroll
                for (int w = 0; w < 5; ++w) dst[w * 32 + lane] = so_flag_word(F, w);
                dst[5 * 32 + lane] = ex | (cnt << 16);
            } else if (cnt && (mode == 1 || count + total <= SO_HITS)) {
                uint32_t *dst = mode == 0 ? hits + count + ex : list + (count - buffered) + ex;
                const uint32_t rel0 = static_cast<uint32_t>(x - ivstart);
                so_emit<EMIT_MSB>(F, [&](uint32_t b) { *dst++ = rel0 + b; });
            }
            count += total;
            __syncwarp();  // slot `cur` and the hit buffer are settled
            cur = cur == SO_NBUF - 1 ? 0 : cur + 1;
        }
        if (failed) {
            // The copy of sub-tile `cur` never completed; wait (bounded)
            // for the prefetches still in flight, then leave.  The pending
            // item is marked failed too, so no successor waits for it.
            if (lane == 0) {
                atomicOr(a.err, ERR_COPY);
                st_relaxed(&Q.state[k], LB_ERR);
                if (have_pending) st_relaxed(&query_of(a, pend.qi).state[pend.k], LB_ERR);
                for (int i = 1; i <= pending; ++i) {
                    const int b = (cur + i) % SO_NBUF;
                    mbar_wait_bounded(&bar[b], (parity >> b) & 1u);
                }
            }
            return;
        }

        // ---- publish this item's count; claim the next item and start its
        // first sub-tiles; then finish the previous item.
        lookback_publish(Q.state, k, count);
        unsigned long long nt = a.total;
        uint32_t nqi = 0;
        uint64_t nk = 0;
        if (lane == 0 && so_claim(a, &nt, &nqi, &nk)) {
            const QueryDev &Qn = query_of(a, nqi);
            const uint64_t s0 = nk * Qn.sub_per_item;
            const uint64_t s1 = min(s0 + Qn.sub_per_item, Qn.nsub);
            for (int i = 0; i < SO_NBUF - 1 && s0 + i < s1; ++i) {
                const int c = (cur + i) % SO_NBUF;
                so_issue(smem + c * SO_BUF, &bar[c], Qn.text, Qn.n, s0 + i);
            }
        }
        nt = __shfl_sync(0xffffffffu, nt, 0);
        nqi = __shfl_sync(0xffffffffu, nqi, 0);
        nk = __shfl_sync(0xffffffffu, nk, 0);
        if (have_pending) write_pending();
        if (mode == 0) buffered = count <= SO_HITS ? count : 0;
        if (mode == 1) listed = count - buffered;
        pend = SOItem{qi, k, sb, se, count, buffered, listed, flag_from};
        have_pending = true;
        hb ^= 1;
        __syncwarp();
        t = nt;
        qi = nqi;
        k = nk;
    }
    if (have_pending) write_pending();
}

// ---------------------------------------------------------------- multi-pattern packs
//
// Up to MP_MAXK patterns of at most 16 bytes over one text share one 32-bit
// state: pattern p owns bits shift[p] .. shift[p] + m_p - 1.  One step for
// all of them (the Shift-And recurrence of each field side by side):
//     D <- ((D << 1) | I) & B[c],   I = the first bit of every field,
// where B[c] is the OR of the patterns' masks, each shifted to its field (a
// bit carried out of a field's top lands on the next field's first bit,
// which the OR with I sets anyway).  Pattern p has an occurrence ending at
// e iff bit shift[p] + m_p - 1 (a bit of F) of D is set.  The scan ORs the
// states of each 16-byte chunk; a chunk whose OR meets F is rescanned byte
// by byte to name the (pattern, position) pairs.  The segment's start
// state comes from a warm-up over the 16 bytes before it (every field is at
// most 16 bits, so all fields are exact after it).

constexpr int MP_REC = 4;  // (pattern, position) records a lane keeps in registers per sub-tile
constexpr uint32_t MP_LIST = 13312;  // records of a work item (52 KB of its spill area)
static_assert(MP_LIST * 4 <= SO_SPILL_ITEM, "the records of an item fit its spill area");

struct MPLayout {
    static constexpr uint32_t BAR_OFF = SO_NBUF * SO_BUF;
    static constexpr uint32_t CONST_OFF = BAR_OFF + 8 * SO_NBUF;
    static constexpr uint32_t CNT_OFF = CONST_OFF + 16;         // hits per pattern, current item
    static constexpr uint32_t PCNT_OFF = CNT_OFF + 4 * MP_MAXK;  // hits per pattern, pending item
    static constexpr uint32_t FMAP_OFF = PCNT_OFF + 4 * MP_MAXK; // last bit -> pattern
    static constexpr uint32_t BYTES = FMAP_OFF + 32;
};

struct MPItem {
    uint32_t qi;
    uint64_t k, sb, se;
    uint32_t listed;  // records in the spill list
    bool overflow;    // the list filled: the write phase rescans per pattern
};

// Loads a pack's table and constants into shared memory unless loaded.
__device__ __forceinline__ void mp_table(const PackPlan *P, const PackPlan *&cur, uint32_t *tbl,
                                         uint8_t *fmap) {
    if (P == cur) return;
    __syncwarp();
    const int lane = threadIdx.x & 31;
    const uint4 *src = reinterpret_cast<const uint4 *>(P->table);
    for (int c = lane; c < 64; c += 32) reinterpret_cast<uint4 *>(tbl)[c] = __ldg(&src[c]);
    const uint32_t k = __ldg(&P->k);
    fmap[lane] = 0xFF;
    __syncwarp();
    if (lane < static_cast<int>(k)) fmap[__ldg(&P->shift[lane]) + __ldg(&P->len[lane]) - 1] = static_cast<uint8_t>(lane);
    cur = P;
    __syncwarp();
}

// Entry of byte b of word x from the packed table at shared address tb
// (4-byte entries: address c * four + tb on the FMA pipe).
__device__ __forceinline__ uint32_t mp_entry(uint32_t x, int b, uint32_t tb, uint32_t four) {
    const uint32_t addr = __byte_perm(x, 0u, 0x4440u | b) * four + tb;
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}

// Four packed steps on the bytes of x; A collects the states.
__device__ __forceinline__ void mp_step4(uint32_t &D, uint32_t &A, uint32_t x, uint32_t tb, uint32_t two,
                                         uint32_t four, uint32_t I) {
    uint32_t d[4];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        D = ((D * two) | I) & mp_entry(x, b, tb, four);
        d[b] = D;
    }
    A |= d[0] | d[1] | d[2] | d[3];
}

// Byte-by-byte rescan of a flagged chunk from its start state: every valid
// (pattern, end) pair is counted (shared counters and the lane's `ntrue`)
// and the first MP_REC of the lane's sub-tile are kept as records
// (chunk << 12 | byte << 8 | pattern).
__device__ __noinline__ void mp_chunk(uint32_t D, uint4 w, int c, uint32_t tb, uint32_t two, uint32_t four,
                                      uint32_t I, uint32_t F, const uint8_t *fmap, const PackPlan *P,
                                      int64_t x, int64_t vlo0, int64_t vhi, uint32_t *cnt,
                                      uint64_t &rec, uint32_t &ntrue) {
    for (int b = 0; b < 16; ++b) {
        const uint32_t xw = b < 4 ? w.x : b < 8 ? w.y : b < 12 ? w.z : w.w;
        D = ((D * two) | I) & mp_entry(xw, b & 3, tb, four);
        uint32_t h = D & F;
        const int64_t e = x + 16 * c + b;  // end position (virtual frame)
        while (h) {
            const int bit = __ffs(h) - 1;
            h &= h - 1;
            const int p = fmap[bit];
            if (e < vlo0 + __ldg(&P->len[p]) - 1 || e >= vhi) continue;  // not a valid end of p
            atomicAdd(&cnt[p], 1u);
            if (ntrue < MP_REC) rec |= static_cast<uint64_t>((c << 12) | (b << 8) | p) << (16 * ntrue);
            ++ntrue;
        }
    }
}

// All records of a lane segment staged at `seg`, in position order, written
// to out[0..] as (pattern << 19 | item-relative end): the write of a lane
// with more than MP_REC of them in one sub-tile (counted already).
__device__ __noinline__ void mp_segment_records(const uint8_t *seg, uint32_t tb, uint32_t two, uint32_t four,
                                                uint32_t I, uint32_t F, const uint8_t *fmap,
                                                const PackPlan *P, int64_t x, int64_t vlo0, int64_t vhi,
                                                uint32_t rel0, uint32_t *out) {
    uint32_t D = 0, A = 0;
    {
        const uint4 w = *reinterpret_cast<const uint4 *>(seg - 16);
        mp_step4(D, A, w.x, tb, two, four, I);
        mp_step4(D, A, w.y, tb, two, four, I);
        mp_step4(D, A, w.z, tb, two, four, I);
        mp_step4(D, A, w.w, tb, two, four, I);
    }
    for (int c = 0; c < SO_SEGC; ++c) {
        const uint4 w = *reinterpret_cast<const uint4 *>(seg + 16 * c);
        for (int b = 0; b < 16; ++b) {
            const uint32_t xw = b < 4 ? w.x : b < 8 ? w.y : b < 12 ? w.z : w.w;
            D = ((D * two) | I) & mp_entry(xw, b & 3, tb, four);
            uint32_t h = D & F;
            const int64_t e = x + 16 * c + b;
            while (h) {
                const int bit = __ffs(h) - 1;
                h &= h - 1;
                const int p = fmap[bit];
                if (e < vlo0 + __ldg(&P->len[p]) - 1 || e >= vhi) continue;
                *out++ = (static_cast<uint32_t>(p) << 19) | (rel0 + 16 * c + b);
            }
        }
    }
}

// One warp per block, the same work-item scheme, staging ring and one-item
// lag as so_kernel, over packs instead of single patterns.  A work item's
// records go to the block's spill list in position order; at its write
// phase every pattern's prefix is resolved (lane p for pattern p) and the
// records are scattered to the patterns' outputs with their ranks.  A lane
// with more than MP_REC records in a sub-tile extracts them again from its
// staged segment straight into the list; if the list fills, the write
// phase instead rescans the item from global memory once per pattern
// (exact for any input, slow only for dense ones).
__global__ void __launch_bounds__(32) mp_kernel(const __grid_constant__ LaunchArgs a) {
    using L = MPLayout;
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ __align__(256) uint32_t tbl[256];
    const uint32_t tb = smem_addr(tbl);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + L::BAR_OFF);
    uint32_t *cnt = reinterpret_cast<uint32_t *>(smem + L::CNT_OFF);
    uint32_t *pcnt = reinterpret_cast<uint32_t *>(smem + L::PCNT_OFF);
    uint8_t *fmap = smem + L::FMAP_OFF;
    const int lane = threadIdx.x;
    uint8_t *spill_base =
        a.spill ? a.spill + static_cast<size_t>(blockIdx.x) * SO_SPILL_BYTES : nullptr;
    volatile uint32_t *consts = reinterpret_cast<volatile uint32_t *>(smem + L::CONST_OFF);

    unsigned long long t = 0;
    uint32_t qi = 0;
    uint64_t k = 0;
    if (lane == 0) {
        consts[0] = 2u;
        consts[1] = 4u;
        for (int b = 0; b < SO_NBUF; ++b) mbar_init(&bar[b], 1);
        fence_mbar_init();
        if (so_claim(a, &t, &qi, &k)) {
            const QueryDev &Q = query_of(a, qi);
            const uint64_t s0 = k * Q.sub_per_item;
            const uint64_t s1 = min(s0 + Q.sub_per_item, Q.nsub);
            for (int i = 0; i < SO_NBUF - 1 && s0 + i < s1; ++i)
                so_issue(smem + i * SO_BUF, &bar[i], Q.text, Q.n, s0 + i);
        } else {
            t = a.total;
        }
    }
    __syncwarp();
    t = __shfl_sync(0xffffffffu, t, 0);
    qi = __shfl_sync(0xffffffffu, qi, 0);
    k = __shfl_sync(0xffffffffu, k, 0);
    const uint32_t two = consts[0];
    const uint32_t four = consts[1];

    const PackPlan *cur_pack = nullptr;
    uint32_t parity = 0;
    int cur = 0;
    int hb = 0;
    bool have_pending = false;
    MPItem pend{};

    auto write_pending = [&]() {
        const QueryDev &Q = query_of(a, pend.qi);
        const PackPlan *P = reinterpret_cast<const PackPlan *>(Q.plan);
        const uint32_t kk = __ldg(&P->k);
        const int64_t o = static_cast<int64_t>(reinterpret_cast<uintptr_t>(Q.text) & 15u);
        const int64_t ivstart = static_cast<int64_t>(pend.sb) * SO_T;
        // Pattern p's prefix: lane p first reads the previous item's word
        // (usually inclusive already, one item behind the scan); patterns
        // whose predecessor is not resolved yet take a windowed look-back
        // of the whole warp, one after another.  Lane p keeps its prefix
        // and output.
        uint64_t excl = 0, capp = 0;
        uint64_t *outp = nullptr;
        int64_t shiftp = 0;
        bool ok = true;
        bool fast = true;
        if (lane < static_cast<int>(kk)) {
            const QueryDev *M = P->member[lane];
            capp = M->cap;
            outp = M->out_pos;
            shiftp = static_cast<int64_t>(__ldg(&P->len[lane])) - 1 + o;
            if (pend.k > 0) {
                const uint64_t w = ld_relaxed(&M->state[pend.k - 1]);
                fast = (w & ~LB_VAL) == LB_INC;
                excl = w & LB_VAL;
            }
            if (fast) {
                st_relaxed(&M->state[pend.k], LB_INC | ((excl + pcnt[lane]) & LB_VAL));
                if (pend.k + 1 == M->ntiles) *M->out_count = excl + pcnt[lane];
            }
        }
        unsigned slow = __ballot_sync(0xffffffffu, !fast);
        while (slow) {
            const int p = __ffs(slow) - 1;
            slow &= slow - 1;
            const QueryDev *M = P->member[p];
            const uint64_t agg = pcnt[p];
            bool okp;
            const uint64_t ex = lookback_resolve(M->state, pend.k, agg, a.err, &okp);
            ok &= okp;
            if (lane == p) {
                excl = ex;
                if (okp && pend.k + 1 == M->ntiles) *M->out_count = ex + agg;
            }
        }
        if (!ok) return;
        if (!pend.overflow) {
            const uint32_t *list = reinterpret_cast<const uint32_t *>(spill_base + (hb ^ 1) * SO_SPILL_ITEM);
            // Records of each pattern written so far, in the ring slot that
            // no prefetch uses; the first lane of each pattern's group
            // advances its entry by the group's size.
            uint32_t *wbase = reinterpret_cast<uint32_t *>(smem + (cur == 0 ? SO_NBUF - 1 : cur - 1) * SO_BUF);
            if (lane < MP_MAXK) wbase[lane] = 0;
            __syncwarp();
            // The next 32 records are loaded before this chunk's stores (the
            // compiler cannot move a list load above an output store).
            uint32_t e_next = static_cast<uint32_t>(lane) < pend.listed ? list[lane] : 0u;
            for (uint32_t c0 = 0; c0 < pend.listed; c0 += 32) {
                const bool valid = c0 + lane < pend.listed;
                const uint32_t e = e_next;
                e_next = c0 + 32 + lane < pend.listed ? list[c0 + 32 + lane] : 0u;
                const int p = valid ? static_cast<int>(e >> 19) : 31;
                const uint32_t rel = e & 0x7FFFFu;
                const unsigned peers = __match_any_sync(0xffffffffu, p);
                const uint32_t rank = __popc(peers & ((1u << lane) - 1u));
                const uint64_t ex = __shfl_sync(0xffffffffu, excl, p);
                const uint64_t cp = __shfl_sync(0xffffffffu, capp, p);
                uint64_t *op = reinterpret_cast<uint64_t *>(
                    __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(outp), p));
                const int64_t sh = __shfl_sync(0xffffffffu, shiftp, p);
                const uint32_t bp = wbase[p & (MP_MAXK - 1)];
                __syncwarp();
                if (valid && rank == 0) wbase[p] = bp + __popc(peers);
                __syncwarp();
                const uint64_t idx = ex + bp + rank;
                if (valid && idx < cp) op[idx] = static_cast<uint64_t>(ivstart + rel - sh);
            }
            return;
        }
        // Overflow: one pass per pattern over the item's text in global
        // memory, with that pattern's own masks (its field of the table).
        mp_table(P, cur_pack, tbl, fmap);
        const uint8_t *base = Q.text - o;
        const int64_t vhi = o + static_cast<int64_t>(Q.n);
        const int64_t vlim = (vhi + 15) & ~int64_t(15);
        for (uint32_t p = 0; p < kk; ++p) {
            const uint64_t ex = __shfl_sync(0xffffffffu, excl, p);
            const uint64_t cp = __shfl_sync(0xffffffffu, capp, p);
            uint64_t *op = reinterpret_cast<uint64_t *>(
                __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(outp), p));
            const int64_t sh = __shfl_sync(0xffffffffu, shiftp, p);
            const uint32_t sp = __ldg(&P->shift[p]);
            const uint32_t mpl = __ldg(&P->len[p]);
            const uint32_t low = (mpl >= 32 ? 0xFFFFFFFFu : ((1u << mpl) - 1u));
            const int64_t vlo = o + static_cast<int64_t>(mpl) - 1;
            uint64_t run = ex;
            for (uint64_t s = pend.sb; s < pend.se && run < cp; ++s) {
                const int64_t x = static_cast<int64_t>(s) * SO_T + lane * SO_S;
                uint32_t F[SO_SEGC];
                uint32_t D = 0;
                for (int64_t y = x - 16; y < x + SO_S; ++y) {
                    const uint32_t cbyte = (y >= 0 && y < vlim) ? base[y] : 0u;
                    D = ((D << 1) | 1u) & ((tbl[cbyte] >> sp) & low);
                    if (y >= x) {
                        const int r = static_cast<int>(y - x);
                        if ((r & 15) == 0) F[r >> 4] = 0;
                        F[r >> 4] |= ((D >> (mpl - 1)) & 1u) << (15 - (r & 15));
                    }
                }
                const int elo = static_cast<int>(vlo - x > 0 ? vlo - x : int64_t(0));
                const int ehi = static_cast<int>(vhi - x < SO_S ? vhi - x : int64_t(SO_S));
                const uint32_t c = so_mask_count(F, elo, ehi);
                uint32_t total;
                const uint32_t exl = warp_excl_scan(c, &total);
                so_write_flags<false>(F, exl, run, cp, op, static_cast<int64_t>(s) * SO_T - sh);
                run += total;
            }
        }
    };

    while (t < a.total) {
        const QueryDev &Q = query_of(a, qi);
        const PackPlan *P = reinterpret_cast<const PackPlan *>(Q.plan);
        mp_table(P, cur_pack, tbl, fmap);
        const uint32_t I = __ldg(&P->I);
        const uint32_t F = __ldg(&P->F);
        const uint8_t *const qtext = Q.text;
        const uint64_t qn = Q.n;
        const uint64_t qnsub = Q.nsub;
        const uint64_t sb = k * Q.sub_per_item;
        const uint64_t se = min(sb + Q.sub_per_item, qnsub);
        const int64_t o = static_cast<int64_t>(reinterpret_cast<uintptr_t>(qtext) & 15u);
        const int64_t vhi = o + static_cast<int64_t>(qn);
        const int64_t ivstart = static_cast<int64_t>(sb) * SO_T;
        uint32_t *list = spill_base ? reinterpret_cast<uint32_t *>(spill_base + hb * SO_SPILL_ITEM) : nullptr;
        if (lane < MP_MAXK) cnt[lane] = 0;
        __syncwarp();

        uint32_t listed = 0;
        bool overflow = list == nullptr;
        bool failed = false;
        int pending = 0;
        for (uint64_t s = sb; s < se; ++s) {
            const int ahead = cur == 0 ? SO_NBUF - 1 : cur - 1;
            if (lane == 0 && s + SO_NBUF - 1 < se)
                so_issue(smem + ahead * SO_BUF, &bar[ahead], qtext, qn, s + SO_NBUF - 1);
            const bool arrived = mbar_wait_bounded(&bar[cur], (parity >> cur) & 1u);
            parity ^= 1u << cur;
            if (!__all_sync(0xffffffffu, arrived)) {
                failed = true;
                pending = 0;
                for (int i = 1; i < SO_NBUF; ++i) pending += s + i < se;
                break;
            }
            const uint8_t *seg = smem + cur * SO_BUF + SO_LHALO + lane * SO_S;
            const int64_t x = static_cast<int64_t>(s) * SO_T + lane * SO_S;
            uint32_t D = 0, A = 0;
            {
                const uint4 w = *reinterpret_cast<const uint4 *>(seg - 16);
                mp_step4(D, A, w.x, tb, two, four, I);
                mp_step4(D, A, w.y, tb, two, four, I);
                mp_step4(D, A, w.z, tb, two, four, I);
                mp_step4(D, A, w.w, tb, two, four, I);
            }
            uint64_t rec = 0;
            uint32_t ntrue = 0;
#pragma unroll
            for (int c = 0; c < SO_SEGC; ++c) {
                const uint4 w = *reinterpret_cast<const uint4 *>(seg + 16 * c);
                const uint32_t Ds = D;
                A = 0;
                mp_step4(D, A, w.x, tb, two, four, I);
                mp_step4(D, A, w.y, tb, two, four, I);
                mp_step4(D, A, w.z, tb, two, four, I);
                mp_step4(D, A, w.w, tb, two, four, I);
                if (A & F) mp_chunk(Ds, w, c, tb, two, four, I, F, fmap, P, x, o, vhi, cnt, rec, ntrue);
            }
            if (__any_sync(0xffffffffu, ntrue != 0)) {
                uint32_t total;
                const uint32_t ex = warp_excl_scan(ntrue, &total);
                overflow |= listed + total > MP_LIST;
                if (!overflow) {
                    const uint32_t rel0 = static_cast<uint32_t>(x - ivstart);
                    if (ntrue <= static_cast<uint32_t>(MP_REC)) {
                        for (uint32_t r = 0; r < ntrue; ++r) {
                            const uint32_t v = static_cast<uint32_t>(rec >> (16 * r)) & 0xFFFFu;
                            const uint32_t pos = rel0 + 16 * ((v >> 12) & 15u) + ((v >> 8) & 15u);
                            list[listed + ex + r] = ((v & 0xFFu) << 19) | pos;
                        }
                    } else {
                        mp_segment_records(seg, tb, two, four, I, F, fmap, P, x, o, vhi, rel0,
                                           list + listed + ex);
                    }
                }
                listed += total;
            }
            __syncwarp();
            cur = cur == SO_NBUF - 1 ? 0 : cur + 1;
        }
        if (failed) {
            if (lane == 0) {
                atomicOr(a.err, ERR_COPY);
                for (int i = 1; i <= pending; ++i) {
                    const int b = (cur + i) % SO_NBUF;
                    mbar_wait_bounded(&bar[b], (parity >> b) & 1u);
                }
            }
            const uint32_t kk = __ldg(&P->k);
            if (lane < static_cast<int>(kk)) st_relaxed(&P->member[lane]->state[k], LB_ERR);
            if (have_pending) {
                const PackPlan *Pp = reinterpret_cast<const PackPlan *>(query_of(a, pend.qi).plan);
                if (lane < static_cast<int>(__ldg(&Pp->k))) st_relaxed(&Pp->member[lane]->state[pend.k], LB_ERR);
            }
            return;
        }

        // ---- publish every pattern's count; claim and start the next item;
        // finish the previous one.
        __syncwarp();
        const uint32_t kk = __ldg(&P->k);
        if (lane < static_cast<int>(kk))
            st_relaxed(&P->member[lane]->state[k], (k == 0 ? LB_INC : LB_AGG) | cnt[lane]);
        unsigned long long nt = a.total;
        uint32_t nqi = 0;
        uint64_t nk = 0;
        if (lane == 0 && so_claim(a, &nt, &nqi, &nk)) {
            const QueryDev &Qn = query_of(a, nqi);
            const uint64_t s0 = nk * Qn.sub_per_item;
            const uint64_t s1 = min(s0 + Qn.sub_per_item, Qn.nsub);
            for (int i = 0; i < SO_NBUF - 1 && s0 + i < s1; ++i) {
                const int c = (cur + i) % SO_NBUF;
                so_issue(smem + c * SO_BUF, &bar[c], Qn.text, Qn.n, s0 + i);
            }
        }
        nt = __shfl_sync(0xffffffffu, nt, 0);
        nqi = __shfl_sync(0xffffffffu, nqi, 0);
        nk = __shfl_sync(0xffffffffu, nk, 0);
        if (have_pending) write_pending();
        __syncwarp();
        if (lane < MP_MAXK) pcnt[lane] = cnt[lane];
        pend = MPItem{qi, k, sb, se, listed, overflow};
        have_pending = true;
        hb ^= 1;
        __syncwarp();
        t = nt;
        qi = nqi;
        k = nk;
    }
    if (have_pending) write_pending();
}

}  // namespace

// ---------------------------------------------------------------- registry

const void *so_kernel_fn(int kid) {
    switch (kid) {
        case K_SO4Q: return reinterpret_cast<const void *>(&so_kernel<uint32_t, uint8_t, true, 8, 4>);
        case K_SO6P: return reinterpret_cast<const void *>(&so_kernel<uint32_t, uint8_t, true, 8, 2>);
        case K_SO8H: return reinterpret_cast<const void *>(&so_kernel<uint32_t, uint8_t, true, 8>);
        case K_SO16H: return reinterpret_cast<const void *>(&so_kernel<uint32_t, uint16_t, true, 16>);
        case K_SO32H: return reinterpret_cast<const void *>(&so_kernel<uint32_t, uint32_t, true, 16>);
        case K_SO32A: return reinterpret_cast<const void *>(&so_kernel<uint32_t, uint32_t, false, 0>);
        case K_SO64H: return reinterpret_cast<const void *>(&so_kernel<uint64_t, uint64_t, true, 0>);
        case K_SO64A: return reinterpret_cast<const void *>(&so_kernel<uint64_t, uint64_t, false, 0>);
        default: return nullptr;
    }
}

size_t so_kernel_smem(int kid) {
    switch (so_entry_bytes(kid)) {
        case 1: return SOLayout<uint8_t>::BYTES;
        case 2: return SOLayout<uint16_t>::BYTES;
        case 4: return SOLayout<uint32_t>::BYTES;
        default: return SOLayout<uint64_t>::BYTES;
    }
}

int so_kernel_threads() { return 32; }

uint64_t so_tile_starts() { return SO_T; }

uint32_t so_hit_buffer() { return SO_HITS; }

uint32_t so_spill_bytes() { return SO_SPILL_BYTES; }

uint32_t so_max_sub() { return SO_MAX_SUB; }

const void *mp_kernel_fn() { return reinterpret_cast<const void *>(&mp_kernel); }

size_t mp_kernel_smem() { return MPLayout::BYTES; }

}  // namespace smgpu

// ---------------------------------------------------------------- no-allocation search
//
// sm_search_noalloc runs the bit-parallel kernel above without any device
// allocation: the plan (header + Shift-And masks) and the kernel's scratch
// (claim counter, error word and one look-back word per work item) live in
// the file-scope array below, which every GPU that loads this library keeps
// until the process exits.  Host code must not use the array's name as a
// device address; it takes the address from cudaGetSymbolAddress once per
// device (the first call on a device does that set-up).  All calls share
// the array and it keeps the previous call's contents: a small kernel
// rewrites the plan from the pattern passed by value, and the claim counter,
// error word and look-back words are cleared on the stream before every
// launch.  Calls whose GPU work overlaps (e.g. on two streams at once) race
// on the array.

#include <mutex>

#include "smgpu.h"

namespace {

constexpr uint32_t NA_MAX_ITEMS = 65536;                 // look-back words
constexpr size_t NA_CTRL = 256;                          // claim counter, error word
constexpr size_t NA_PLAN = 4096;                         // plan blob
constexpr size_t NA_BYTES = NA_CTRL + NA_PLAN + size_t(NA_MAX_ITEMS) * 8;
constexpr int NA_MAX_DEVICES = 64;
// Longest text: o + n <= NA_MAX_ITEMS * 64 * SO_T for any o = text & 15, so
// at most NA_MAX_ITEMS work items of at most 64 sub-tiles are ever needed.
constexpr uint64_t NA_MAX_N = uint64_t(NA_MAX_ITEMS) * 64 * smgpu::SO_T - 16;

static __device__ __align__(256) uint8_t g_noalloc_scratch[NA_BYTES];

struct NoAllocDevice {
    bool ready = false;
    uint8_t *scratch = nullptr;  // device address of g_noalloc_scratch
    int sms = 0;
    int bps[smgpu::K_COUNT] = {};  // resident blocks per SM of the bit-parallel kernels
};

std::mutex g_noalloc_mu;
NoAllocDevice g_noalloc_dev[NA_MAX_DEVICES];

const void *na_kernel(int kid) { return smgpu::so_kernel_fn(kid); }

// The pattern, passed to the plan kernel by value.
struct NAPattern {
    uint8_t b[64];
};

// Writes a Shift-And plan for pattern p (m <= 64) into `plan`: the header,
// then 256 entries of esz bytes, little-endian, where bit j (j < m) of entry
// c is 1 iff p[j] = c and every bit >= m is 1 (Section 1's one-bit-per-
// symbol masks, with the high bits kept so older match flags survive).
// One thread per byte value c; 256 threads.
__global__ void na_plan_kernel(uint8_t *plan, const __grid_constant__ smgpu::PlanDev hdr,
                               const __grid_constant__ NAPattern pat, uint32_t esz) {
    const uint32_t c = threadIdx.x;
    const uint32_t m = hdr.m;
    uint64_t w = m >= 64 ? 0ull : ~((1ull << m) - 1ull);
    for (uint32_t j = 0; j < m; ++j)
        if (pat.b[j] == c) w |= 1ull << j;
    uint8_t *e = plan + hdr.off_tbl + esz * c;
    for (uint32_t k = 0; k < esz; ++k) e[k] = static_cast<uint8_t>(w >> (8 * k));
    if (c < sizeof(smgpu::PlanDev) / 4)
        reinterpret_cast<uint32_t *>(plan)[c] = reinterpret_cast<const uint32_t *>(&hdr)[c];
}

// Runs after the search on the same stream: if any wait of the search ran
// out (nonzero error word), the count becomes UINT64_MAX whatever the last
// work item wrote, so a partial result is never reported as complete.
__global__ void na_finish_kernel(const uint32_t *err, uint64_t *out_count) {
    if (*reinterpret_cast<const volatile uint32_t *>(err) != 0u) *out_count = ~0ull;
}

sm_status na_setup(NoAllocDevice **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SM_ECUDA;
    if (dev < 0 || dev >= NA_MAX_DEVICES) return SM_EINVAL;
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    NoAllocDevice &d = g_noalloc_dev[dev];
    if (!d.ready) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return SM_ECUDA;
        if (cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return SM_ECUDA;
        for (int k = 0; k < smgpu::K_COUNT; ++k) {
            if (!smgpu::so_kid(k)) continue;
            const size_t smem = smgpu::so_kernel_smem(k);
            if (cudaFuncSetAttribute(na_kernel(k), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     static_cast<int>(smem)) != cudaSuccess)
                return SM_ECUDA;
            int bps = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, na_kernel(k), 32, smem) !=
                cudaSuccess)
                return SM_ECUDA;
            d.bps[k] = bps > 0 ? bps : 1;
        }
        d.scratch = static_cast<uint8_t *>(p);
        d.ready = true;
    }
    *out = &d;
    return SM_OK;
}

}  // namespace

extern "C" sm_status sm_search_noalloc(const uint8_t *text, uint64_t n, const uint8_t *pattern,
                                       uint32_t m, uint64_t *out_pos, uint64_t cap,
                                       uint64_t *out_count, sm_stream_t stream) {
    using namespace smgpu;
    if (!pattern || m == 0 || m > 64) return SM_EINVAL;
    if (!out_count || (reinterpret_cast<uintptr_t>(out_count) & 7u)) return SM_EINVAL;
    if (cap > 0 && (!out_pos || (reinterpret_cast<uintptr_t>(out_pos) & 7u))) return SM_EINVAL;
    if (n > 0 && !text) return SM_EINVAL;
    if (n > NA_MAX_N) return SM_EINVAL;  // checked before any CUDA call
    NoAllocDevice *d = nullptr;
    sm_status st = na_setup(&d);
    if (st != SM_OK) return st;
    cudaStream_t s = stream;
    if (n < m) return cudaMemsetAsync(out_count, 0, sizeof(uint64_t), s) == cudaSuccess ? SM_OK : SM_ECUDA;

    // Work split exactly as sm_search does for this kernel.
    const int kid = so_kid_for(m, 0);
    const uint64_t o = reinterpret_cast<uintptr_t>(text) & 15u;
    const uint64_t units = (o + n + SO_T - 1) / SO_T;
    const uint64_t resident = static_cast<uint64_t>(d->sms) * static_cast<uint64_t>(d->bps[kid]);
    uint64_t per = (units + 4 * resident - 1) / (4 * resident);
    per = per < 1 ? 1 : (per > 64 ? 64 : per);
    const uint64_t items = (units + per - 1) / per;
    if (items > NA_MAX_ITEMS) return SM_EINVAL;  // cannot happen when n <= NA_MAX_N

    PlanDev h{};
    h.m = m;
    h.variant = VAR_SHIFTOR;
    h.word_bits = so_word_bits(kid);
    h.hist = so_hist(kid) ? 1 : 0;
    h.off_tbl = sizeof(PlanDev);
    h.tile_starts = SO_T;
    const uint32_t esz = so_entry_bytes(kid);
    h.bytes = static_cast<uint32_t>(sizeof(PlanDev) + 256 * esz);
    NAPattern pat{};
    memcpy(pat.b, pattern, m);

    uint8_t *ctrl = d->scratch;
    uint8_t *plan = d->scratch + NA_CTRL;
    uint64_t *state = reinterpret_cast<uint64_t *>(d->scratch + NA_CTRL + NA_PLAN);
    uint32_t *err = reinterpret_cast<uint32_t *>(ctrl + 8);
    na_plan_kernel<<<1, 256, 0, s>>>(plan, h, pat, esz);
    if (cudaGetLastError() != cudaSuccess) return SM_ECUDA;
    if (cudaMemsetAsync(ctrl, 0, NA_CTRL, s) != cudaSuccess) return SM_ECUDA;
    if (cudaMemsetAsync(state, 0, items * sizeof(uint64_t), s) != cudaSuccess) return SM_ECUDA;
    // All-ones until the last work item writes the true total: a count of
    // UINT64_MAX after the stream completes means a bounded wait ran out.
    if (cudaMemsetAsync(out_count, 0xFF, sizeof(uint64_t), s) != cudaSuccess) return SM_ECUDA;

    LaunchArgs a{};
    a.nq = 1;
    a.one.text = text;
    a.one.n = n;
    a.one.plan = reinterpret_cast<const PlanDev *>(plan);
    a.one.out_pos = out_pos;
    a.one.cap = cap;
    a.one.out_count = out_count;
    a.one.state = state;
    a.one.ntiles = items;
    a.one.first_ticket = 0;
    a.one.nsub = units;
    a.one.sub_per_item = static_cast<uint32_t>(per);
    a.ticket = reinterpret_cast<unsigned long long *>(ctrl);
    a.total = items;
    a.err = err;
    const uint64_t full = resident;
    const int grid = static_cast<int>(items < full ? items : full);
    void *args[] = {&a};
    if (cudaLaunchKernel(na_kernel(kid), dim3(grid), dim3(32), args, so_kernel_smem(kid), s) !=
        cudaSuccess)
        return SM_ECUDA;
    na_finish_kernel<<<1, 1, 0, s>>>(err, out_count);
    if (cudaGetLastError() != cudaSuccess) return SM_ECUDA;
    count_launches(3);
    return SM_OK;
}
