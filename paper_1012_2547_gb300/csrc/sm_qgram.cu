// Long patterns: exact q-gram stride filter with warp-cooperative
// verification, and two linear-time per-segment scans that serve as its
// fallback and as kernel families of their own: Knuth-Morris-Pratt, and the
// string-matching automaton (the AUT/DFA algorithm of the paper's tables).
//
// Filter (the Hash-q idea of Fig. 1, with q-grams compared exactly).  Let
// s = m - q + 1 and probe k sit at P_k = k*s + s - 1.  Any occurrence
// [i, i+m-1] has its q-gram window [i, i+m-q] = [i, i+s-1], which holds
// exactly one probe position (s consecutive integers hold one value
// = s-1 mod s), that of k = floor(i/s); the q-gram of the text there equals
// p[j..j+q-1] for j = P_k - i in [0, m-q].  So only the text q-grams at the
// probe positions are looked up in the table of the pattern's q-grams; each
// listed offset j gives one candidate i = P_k - j, and every occurrence is
// produced exactly once, by the probe whose start range [k*s, k*s+s) holds
// it.  Offsets are stored in decreasing order, so a probe's candidates come
// out increasing, and consecutive probes cover consecutive start ranges.
//
// Probes are interleaved over the lanes of a warp: in a round, lane l takes
// probe k0 + l, so one warp load touches one contiguous stretch of text (a
// stride of s bytes between lanes: every 32-byte sector when s < 32, about
// one sector in s/32 when s is larger, which is where the filter reads less
// than the whole text), and the warp's hits of a round come out in lane
// order.  The q-grams of several rounds are loaded before the first of them
// is looked up.  A probe first tests a presence bitmap; only rounds where
// some lane passes it look the q-gram up in the hash table of exact keys.
//
// Verification of a round: each lane walks its own candidates in order and
// compares their first bytes; the survivors are checked in lane order, one
// at a time, by all 32 lanes together (lane l compares bytes 16l..16l+15 of
// every 512-byte block) with a ballot deciding the result.  The warp keeps
// its hits in order in shared memory.
//
// Density guard: a warp whose fully checked candidates exceed a fixed number
// per probe
// (periodic patterns on periodic text, e.g. a^m in a^n) flags the work
// item, which is then recomputed with a linear scan per thread over its
// start range plus m-1 bytes, O(range + m): the automaton (read through the
// L1 cache) when the plan carries one -- periodic patterns, the only ones
// that can occur densely -- else Knuth-Morris-Pratt.
//
// Automaton.  delta(q, c) is the length of the longest prefix of p that is a
// suffix of p[0..q-1] c (q = m after a match); the automaton started in
// state 0 at L reaches state m exactly at the ends of the occurrences that
// start at or after L.  Bytes absent from p share one class, whose
// transitions all go to state 0, so the table has (m+1) x C entries for C-1
// distinct pattern bytes.  The DFA kernel keeps it in shared memory; a step
// is two shared loads (class, then transition) and one add, the same for
// every m.
//
// Compaction is the same as in the bit-parallel kernel: per-warp (filter) or
// per-thread (linear scans) counts, block scan, decoupled look-back, ordered
// writes.  Hits are kept in shared memory; a warp or thread with more hits
// than its buffer holds recomputes its range in write mode once its output
// offset is known.
#include "sm_internal.h"

namespace smgpu {

namespace {

constexpr int QG_THREADS = 128;
constexpr int QG_HB = 8;              // buffered hits per thread (linear scans)
constexpr int QG_ROUNDS_PER_PROBE = 4; // density guard budget (candidates per probe)
constexpr int QG_WL = 512;            // hits a warp keeps in shared memory per work item
constexpr int QG_U = 4;               // probe rounds whose q-grams are loaded ahead

// Per-warp shared state of the q-gram filter.
struct QGWarp {
    uint32_t list[QG_WL];  // hits, relative to the warp's first start
};

// Kernel families built from this file.
enum : int { QG_QGRAM = 0, QG_KMP = 1, QG_DFA = 2 };

struct QGCtl {
    unsigned long long ticket;
    uint64_t excl;
    uint32_t qi;
    uint32_t dense;
    uint64_t tile;
    uint32_t warp_ex[32];
    uint32_t ok;
};

__device__ __forceinline__ uint32_t lds_u32(uint32_t addr) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}

// Hash of a packed q-gram for the key table's slots (64-bit golden-ratio
// multiplicative hashing).
__device__ __forceinline__ uint64_t qgram_hash(uint64_t g) { return g * 0x9E3779B97F4A7C15ull; }

// Hash of a packed q-gram (lo: bytes 0..3, hi: bytes 4..7) for the presence
// bitmap, whose bit is its top bm_bits bits: two 32-bit multiplicative
// hashes (the golden-ratio constant 0x9E3779B1 and xxHash32's second prime
// 0x85EBCA77) xored, two IMADs and one LOP in the probe loop.
__device__ __forceinline__ uint32_t qgram_bitmap_hash(uint32_t lo, uint32_t hi) {
    return (lo * 0x9E3779B1u) ^ (hi * 0x85EBCA77u);
}

// Bytes t[pos..pos+q-1] packed little-endian; t[pos+q-1] must be in the text.
__device__ __forceinline__ uint64_t load_qgram(const uint8_t *t, uint64_t pos, uint32_t q) {
    const uintptr_t addr = reinterpret_cast<uintptr_t>(t) + pos;
    const uint64_t *w = reinterpret_cast<const uint64_t *>(addr & ~uintptr_t(7));
    const uint32_t sh = static_cast<uint32_t>(addr & 7u) * 8u;
    uint64_t g = __ldg(w);
    if (sh) {
        g >>= sh;
        if (sh / 8u + q > 8u) g |= __ldg(w + 1) << (64u - sh);
    }
    return q >= 8 ? g : (g & ((1ull << (8u * q)) - 1ull));
}

struct PlanView {
    const uint8_t *pat;
    const uint32_t *bitmap;
    uint32_t bm_smem;  // shared-memory address of the bitmap's copy (q-gram kernel), else 0
    const QSlot *slots;
    const uint32_t *offs;
    const uint32_t *fail;
    uint32_t m, q, s, bm_bits, slot_bits;
    uint32_t off_dfa;  // 0: the plan carries no automaton
};

__device__ __forceinline__ PlanView plan_view(const PlanDev *P) {
    const uint8_t *b = reinterpret_cast<const uint8_t *>(P);
    PlanView v;
    v.m = __ldg(&P->m);
    v.q = __ldg(&P->q);
    v.s = __ldg(&P->s);
    v.bm_bits = __ldg(&P->bm_bits);
    v.slot_bits = __ldg(&P->slot_bits);
    v.pat = b + __ldg(&P->off_pat);
    v.bitmap = reinterpret_cast<const uint32_t *>(b + __ldg(&P->off_bitmap));
    v.bm_smem = 0;
    v.slots = reinterpret_cast<const QSlot *>(b + __ldg(&P->off_slots));
    v.offs = reinterpret_cast<const uint32_t *>(b + __ldg(&P->off_offs));
    v.fail = reinterpret_cast<const uint32_t *>(b + __ldg(&P->off_fail));
    v.off_dfa = __ldg(&P->off_dfa);
    return v;
}

// An automaton: class table (2 x class per byte), transitions (row offsets),
// and the row offset of state m.
struct DfaView {
    const uint16_t *cls;
    const uint8_t *tab;
    uint32_t fin;
    uint32_t m;
};

// Next row offset from row offset r on byte c; SH: tables in shared memory,
// else read-only global loads.
template <bool SH>
__device__ __forceinline__ uint32_t dfa_step(const DfaView &d, uint32_t r, uint32_t c) {
    if (SH) return *reinterpret_cast<const uint16_t *>(d.tab + r + d.cls[c]);
    return __ldg(reinterpret_cast<const uint16_t *>(d.tab + r + __ldg(d.cls + c)));
}

// Looks up q-gram g (whose bitmap bit is set) in the table of exact keys;
// returns the number of offsets and their first index (0: not a key).
__device__ __forceinline__ uint32_t qgram_lookup(const PlanView &v, uint64_t g, uint32_t *first) {
    const uint64_t h = qgram_hash(g);
    const uint32_t mask = (1u << v.slot_bits) - 1u;
    uint32_t sl = static_cast<uint32_t>(h >> (64u - v.slot_bits));
    while (true) {
        const QSlot *S = &v.slots[sl];
        const uint32_t cnt = __ldg(&S->count);
        if (cnt == 0) return 0;
        if (__ldg(&S->key) == g) {
            *first = __ldg(&S->first);
            return cnt;
        }
        sl = (sl + 1u) & mask;
    }
}

// All lanes: does t[0..m-1] equal p[0..m-1]?
__device__ __forceinline__ bool warp_equal(const uint8_t *t, const uint8_t *p, uint32_t m) {
    const uint32_t lane = threadIdx.x & 31u;
    bool bad = false;
    for (uint32_t off = lane * 16u; off < m; off += 512u) {
        const uint32_t e = min(off + 16u, m);
        for (uint32_t b = off; b < e; ++b) bad |= __ldg(t + b) != __ldg(p + b);
    }
    return !__any_sync(0xffffffffu, bad);
}

enum : int { SINK_BUFFER = 0, SINK_WRITE = 1, SINK_DISCARD = 2 };

// Where a thread's hits go: its shared-memory buffer (count pass), the
// output array at its offset (write pass), or nowhere (a lane that only
// helps its warp verify).
struct Sink {
    int mode;
    uint64_t *out;
    uint64_t cap;
    uint64_t idx;
    uint32_t *hb;      // shared buffer, column tid, stride QG_THREADS
    uint32_t cnt;

    __device__ __forceinline__ void put(uint64_t i, uint64_t L) {
        if (mode == SINK_WRITE) {
            if (idx < cap) out[idx] = i;
            ++idx;
        } else if (mode == SINK_BUFFER && cnt < QG_HB) {
            hb[cnt * QG_THREADS] = static_cast<uint32_t>(i - L);
        }
        ++cnt;
    }
};

// Write-mode sink of the automaton scans: a thread's hits are consecutive
// output words, so they are gathered four at a time and written with one
// 32-byte store once the output address is 32-byte aligned (one memory
// request per four hits instead of one per hit on dense inputs).
struct VSink {
    uint64_t *out;
    uint64_t cap;
    uint64_t idx;
    uint64_t b0, b1, b2, b3;  // b[4 - nb .. 3] hold the pending hits
    uint32_t nb;

    __device__ __forceinline__ void put(uint64_t i, uint64_t) {
        if (nb == 0 && (reinterpret_cast<uintptr_t>(out + idx) & 31u)) {
            if (idx < cap) out[idx] = i;
            ++idx;
            return;
        }
        b0 = b1;
        b1 = b2;
        b2 = b3;
        b3 = i;
        if (++nb == 4) {
            if (idx + 4 <= cap) {
                // No memory clobber: nothing in the kernel reads the output,
                // and a clobber would pin the next bytes' table loads behind
                // the store.
                asm volatile("st.global.v4.b64 [%0], {%1, %2, %3, %4};" ::"l"(out + idx), "l"(b0), "l"(b1),
                             "l"(b2), "l"(b3));
            } else {  // the capacity ends inside these four words
                if (idx < cap) out[idx] = b0;
                if (idx + 1 < cap) out[idx + 1] = b1;
                if (idx + 2 < cap) out[idx + 2] = b2;
            }
            idx += 4;
            nb = 0;
        }
    }
    // Writes the hits still pending (idx is the index of the first of them).
    __device__ __forceinline__ void finish() {
        if (nb >= 3) {
            if (idx < cap) out[idx] = b1;
            ++idx;
        }
        if (nb >= 2) {
            if (idx < cap) out[idx] = b2;
            ++idx;
        }
        if (nb >= 1) {
            if (idx < cap) out[idx] = b3;
            ++idx;
        }
        nb = 0;
    }
};

// Filter state a warp carries across its probe rounds.
struct QGRun {
    uint64_t ncand;  // candidates fully checked so far (density guard)
    uint32_t cnt;    // hits so far
    uint32_t ovf;    // 1: more hits than the warp's list holds
};

// Output side of a warp's filter run: the count pass keeps hits in ws.list,
// the write pass stores them at out[base + rank] (ranks below cap).
struct QGOut {
    QGWarp *ws;
    uint64_t *out;
    uint64_t cap;
    uint64_t base;
    uint32_t write;
};

// One probe round that some lane's bitmap test passed.  Each such lane
// looks its q-gram up in the table of exact keys (loading it again, so the
// probe loop keeps no q-gram alive past its bitmap test) and walks its
// candidates in increasing order, comparing the first min(m, 8) bytes; the
// survivors are checked one at a time by the whole warp, the lowest lane's
// first, and only that lane moves on to its next survivor, so hits come out
// in lane order and, within a lane, in increasing order.  Returns false if
// the count pass exceeds the density budget (full checks per probe).
__device__ __forceinline__ bool qgram_round(const PlanView &v, uint64_t patw, const uint8_t *text, uint64_t n,
                                            uint64_t Lw, bool hit, uint64_t P, uint64_t budget,
                                            const QGOut &o, QGRun &run) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t pre = min(v.m, 8u);
    const uint64_t last = n - v.m;  // last valid start
    uint32_t first = 0, c = 0, t = 0;
    if (hit) c = qgram_lookup(v, load_qgram(text, P, v.q), &first);
    uint64_t cand = 0;
    // Next candidate of this lane that passes the prefix comparison.
    auto advance = [&]() -> bool {
        while (t < c) {
            const uint64_t i = P - __ldg(&v.offs[first + t]);
            ++t;
            if (i > last) {  // offsets descend, so every later candidate is past the end too
                t = c;
                break;
            }
            if (load_qgram(text, i, pre) == patw) {
                cand = i;
                return true;
            }
        }
        return false;
    };
    bool have = advance();
    while (true) {
        const unsigned mask = __ballot_sync(0xffffffffu, have);
        if (!mask) break;
        const int src = __ffs(mask) - 1;
        const uint64_t ic = __shfl_sync(0xffffffffu, cand, src);
        if (!o.write && ++run.ncand > budget) return false;
        if (warp_equal(text + ic, v.pat, v.m)) {
            const uint32_t rs = static_cast<uint32_t>(ic - Lw);
            if (o.write) {
                if (lane == 0 && o.base + run.cnt < o.cap) o.out[o.base + run.cnt] = ic;
            } else if (run.cnt < static_cast<uint32_t>(QG_WL)) {
                if (lane == 0) o.ws->list[run.cnt] = rs;
            } else {
                run.ovf = 1u;
            }
            ++run.cnt;
        }
        if (lane == static_cast<uint32_t>(src)) have = advance();
    }
    return true;
}

// The q-gram filter of one warp over the start range [Lw, Lw + span) (Lw
// and span multiples of s; span < 2^32), in probe rounds of 32 probes (lane
// l takes the l-th).  Hits go, in increasing order, to the warp's list
// (count pass; run.ovf set when more than QG_WL were found) or straight to
// the output (write pass).  Returns false if the count pass exceeded the
// density budget: the work item is then recomputed linearly.  Whole warp,
// warp-uniform arguments.
__device__ bool qgram_warp(const PlanView &v, uint64_t patw, const uint8_t *text, uint64_t n, uint64_t Lw,
                           uint64_t span, const QGOut &o, QGRun &run) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t s = v.s;
    const uint64_t k0 = Lw / s;
    const uint64_t kend = min(k0 + span / s, (n - v.m) / s + 1);  // probes [k0, kend) hold valid starts
    // Probe k0 + j sits at first + j * s; j and j * s fit in 32 bits (a
    // warp's span is below 2^32 starts).
    const uint32_t np = kend > k0 ? static_cast<uint32_t>(kend - k0) : 0u;
    const uint32_t nr = (np + 31u) / 32u;
    const uint32_t s32 = static_cast<uint32_t>(s);
    const uintptr_t first = reinterpret_cast<uintptr_t>(text) + k0 * s + (s - 1u);
    const uint32_t q = v.q;
    const uint32_t mlo = q >= 4 ? 0xFFFFFFFFu : ((1u << (8u * q)) - 1u);
    const uint32_t mhi = q >= 8 ? 0xFFFFFFFFu : q <= 4 ? 0u : ((1u << (8u * (q - 4u))) - 1u);
    const uint32_t bshift = 32u - v.bm_bits;
    run = QGRun{0, 0, 0};
    for (uint32_t r0 = 0; r0 < nr; r0 += QG_U) {
        // Every load of the QG_U rounds is issued before any of their words
        // is used: the aligned 32-bit words that hold each probe's q-gram
        // (the second and third only when the q-gram reaches into them),
        // then the bitmap words; one vote decides whether any of the rounds
        // needs the key table.
        uint32_t w0[QG_U], w1[QG_U], w2[QG_U], sh[QG_U];
#pragma unroll
        for (int u = 0; u < QG_U; ++u) {
            const uint32_t j = (r0 + u) * 32u + lane;
            const bool live = j < np;
            const uintptr_t addr = first + (live ? static_cast<uint64_t>(j) * s32 : 0u);
            const uint32_t *w = reinterpret_cast<const uint32_t *>(addr & ~uintptr_t(3));
            const uint32_t b = static_cast<uint32_t>(addr & 3u);
            sh[u] = 8u * b;
            w0[u] = live ? __ldg(w) : 0u;
            w1[u] = live && b + q > 4u ? __ldg(w + 1) : 0u;
            w2[u] = live && b + q > 8u ? __ldg(w + 2) : 0u;
        }
        uint32_t bw[QG_U], bb[QG_U];
#pragma unroll
        for (int u = 0; u < QG_U; ++u) {
            const uint32_t lo = __funnelshift_r(w0[u], w1[u], sh[u]) & mlo;
            const uint32_t hi = __funnelshift_r(w1[u], w2[u], sh[u]) & mhi;
            const uint32_t hb = qgram_bitmap_hash(lo, hi) >> bshift;
            bb[u] = hb & 31u;
            bw[u] = lds_u32(v.bm_smem + 4u * (hb >> 5));
        }
        uint32_t hits = 0;  // bit u: round u passes the bitmap on this lane
#pragma unroll
        for (int u = 0; u < QG_U; ++u) {
            const uint32_t j = (r0 + u) * 32u + lane;
            hits |= (j < np && ((bw[u] >> bb[u]) & 1u)) ? (1u << u) : 0u;
        }
        if (!__any_sync(0xffffffffu, hits != 0)) continue;
#pragma unroll 1
        for (int u = 0; u < QG_U; ++u) {
            const bool hit = (hits >> u) & 1u;
            if (!__any_sync(0xffffffffu, hit)) continue;
            const uint64_t kp = k0 + (r0 + u) * 32u + lane;
            // Density guard, checked as the rounds go: at most
            // QG_ROUNDS_PER_PROBE full checks per probe so far (plus slack),
            // so a dense item is given up within a round or two.
            const uint64_t budget = static_cast<uint64_t>(QG_ROUNDS_PER_PROBE) * 32u * (r0 + u + 1) + 64u;
            if (!qgram_round(v, patw, text, n, Lw, hit, kp * s + s - 1u, budget, o, run)) return false;
        }
    }
    return true;
}

// Knuth-Morris-Pratt from state 0 at L: occurrences starting in
// [L, min(L+R, n-m+1)).  fail[q] = longest proper border of p[0..q-1].
__device__ void linear_range(const PlanView &v, const uint8_t *text, uint64_t n, uint64_t L,
                             uint64_t R, Sink &sink) {
    const uint64_t hi = min(L + R, n - v.m + 1);
    if (L >= hi) return;
    const uint64_t end = hi + v.m - 1;  // bytes [L, end)
    uint32_t q = 0;
    for (uint64_t i = L; i < end; ++i) {
        const uint8_t c = __ldg(text + i);
        while (q > 0 && __ldg(v.pat + q) != c) q = __ldg(&v.fail[q]);
        if (__ldg(v.pat + q) == c) ++q;
        if (q == v.m) {
            sink.put(i + 1 - v.m, L);
            q = __ldg(&v.fail[q]);
        }
    }
}

// The automaton from state 0 at L: occurrences starting in
// [L, min(L+R, n-m+1)).  Bytes are read 16 at a time where aligned.
template <bool SH, typename S>
__device__ __forceinline__ void dfa_range(const DfaView &d, const uint8_t *text, uint64_t n, uint64_t L,
                                          uint64_t R, S &sink) {
    const uint64_t hi = min(L + R, n - d.m + 1);
    if (L >= hi) return;
    const uint64_t end = hi + d.m - 1;  // bytes [L, end)
    const uint64_t back = d.m - 1;      // end -> start
    const uint32_t fin = d.fin;
    uint32_t r = 0;
    uint64_t i = L;
    const uint64_t head = min(end, i + ((16u - (reinterpret_cast<uintptr_t>(text + i) & 15u)) & 15u));
    for (; i < head; ++i) {
        r = dfa_step<SH>(d, r, __ldg(text + i));
        if (r == fin) sink.put(i - back, L);
    }
    // DFA kernel: the next 16 bytes are loaded before these 16 are stepped
    // through, so the load's latency hides behind sixteen dependent table
    // steps.  (The q-gram kernel's rare dense fallback keeps one load at a
    // time: its registers are the filter's.)
    uint4 nx = SH && i + 16 <= end ? __ldg(reinterpret_cast<const uint4 *>(text + i)) : make_uint4(0, 0, 0, 0);
    for (; i + 16 <= end; i += 16) {
        uint4 v;
        if (SH) {
            v = nx;
            if (i + 32 <= end) nx = __ldg(reinterpret_cast<const uint4 *>(text + i + 16));
        } else {
            v = __ldg(reinterpret_cast<const uint4 *>(text + i));
        }
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            r = dfa_step<SH>(d, r, (w[k >> 2] >> (8 * (k & 3))) & 0xffu);
            if (r == fin) sink.put(i + k - back, L);
        }
    }
    for (; i < end; ++i) {
        r = dfa_step<SH>(d, r, __ldg(text + i));
        if (r == fin) sink.put(i - back, L);
    }
}

// Dense fallback of the q-gram kernel through the plan's automaton in
// global memory.  Inlined, with the plain sink and one text load at a time:
// a call frame, the vector sink or a second load in flight would each raise
// the filter kernel's register count or add spills to its hot path.
__device__ __forceinline__ void dfa_range_global(const PlanDev *P, const PlanView &v, const uint8_t *text,
                                              uint64_t n, uint64_t L, uint64_t R, Sink &sink) {
    const uint8_t *b = reinterpret_cast<const uint8_t *>(P);
    const DfaView d{reinterpret_cast<const uint16_t *>(b + __ldg(&P->off_cls)), b + v.off_dfa,
                    __ldg(&P->dfa_final), v.m};
    dfa_range<false>(d, text, n, L, R, sink);
}

// Shared memory of the DFA kernel: class table and transitions.
struct DfaShared {
    uint16_t cls[256];
    uint8_t tab[DFA_MAX_TABLE];
};

template <int MODE>
__global__ void __launch_bounds__(QG_THREADS) qg_kernel(const LaunchArgs a) {
    constexpr int NW = QG_THREADS / 32;
    __shared__ QGCtl ctl;
    __shared__ uint32_t hbuf[QG_HB * QG_THREADS];
    __shared__ __align__(16) uint8_t dfa_raw[MODE == QG_DFA ? sizeof(DfaShared) : 16];
    __shared__ __align__(16) uint8_t qgw_raw[MODE == QG_QGRAM ? sizeof(QGWarp) * (QG_THREADS / 32) : 16];
    QGWarp *qgw = reinterpret_cast<QGWarp *>(qgw_raw);
    __shared__ __align__(16) uint32_t qbm[MODE == QG_QGRAM ? (1u << 16) / 32 : 4];
    DfaShared &dsm = *reinterpret_cast<DfaShared *>(dfa_raw);
    const PlanDev *loaded = nullptr;  // plan whose automaton is in shared memory
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;

    while (true) {
        if (tid == 0) {
            const unsigned long long t = atomicAdd(a.ticket, 1ull);
            ctl.ticket = t;
            if (t < a.total) {
                uint32_t qi;
                uint64_t k;
                resolve_ticket(a, t, &qi, &k);
                ctl.qi = qi;
                ctl.tile = k;
            }
            ctl.dense = MODE == QG_QGRAM ? 0u : 1u;
        }
        __syncthreads();
        if (ctl.ticket >= a.total) break;
        const QueryDev &Q = query_of(a, ctl.qi);
        const uint64_t k = ctl.tile;
        PlanView v = plan_view(Q.plan);
        if (MODE == QG_QGRAM) v.bm_smem = smem_addr(qbm);
        const uint64_t R = static_cast<uint64_t>(__ldg(&Q.plan->tile_starts) / QG_THREADS) *
                           Q.sub_per_item;
        const uint64_t L = k * R * QG_THREADS + static_cast<uint64_t>(tid) * R;
        const uint8_t *text = Q.text;
        const uint64_t n = Q.n;
        if (MODE == QG_QGRAM && Q.plan != loaded) {
            // The plan's presence bitmap (at most 2^16 bits) goes to shared
            // memory: the probe loop's bitmap loads then never compete with
            // the text streaming through L1.  Every thread is past its last
            // use of the previous one (barrier at the end of the item).
            const uint4 *src = reinterpret_cast<const uint4 *>(v.bitmap);
            uint4 *dst = reinterpret_cast<uint4 *>(qbm);
            for (uint32_t i = tid; i < (1u << v.bm_bits) / 128u; i += QG_THREADS) dst[i] = __ldg(src + i);
            loaded = Q.plan;
            __syncthreads();
        }
        if (MODE == QG_DFA && Q.plan != loaded) {
            // Every thread is past its last use of the previous automaton
            // (barrier at the end of the previous item).  Blob offsets and
            // sizes are multiples of 16 within the 256-byte-aligned blob.
            const uint8_t *b = reinterpret_cast<const uint8_t *>(Q.plan);
            const uint4 *src = reinterpret_cast<const uint4 *>(b + __ldg(&Q.plan->off_cls));
            uint4 *dst = reinterpret_cast<uint4 *>(dsm.cls);
            for (int i = tid; i < 512 / 16; i += QG_THREADS) dst[i] = __ldg(src + i);
            const uint32_t tbytes = (v.m + 1) * __ldg(&Q.plan->classes) * 2u;
            src = reinterpret_cast<const uint4 *>(b + v.off_dfa);
            dst = reinterpret_cast<uint4 *>(dsm.tab);
            for (uint32_t i = tid; i < (tbytes + 15u) / 16u; i += QG_THREADS) dst[i] = __ldg(src + i);
            loaded = Q.plan;
            __syncthreads();
        }
        const DfaView dv{dsm.cls, dsm.tab, MODE == QG_DFA ? __ldg(&Q.plan->dfa_final) : 0u, v.m};
        // One linear-time scan of this thread's range (count or write mode).
        auto linear = [&](Sink &sk) {
            if (MODE == QG_DFA) {
                if (sk.mode == SINK_WRITE) {
                    VSink w{sk.out, sk.cap, sk.idx, 0, 0, 0, 0, 0};
                    dfa_range<true>(dv, text, n, L, R, w);
                    w.finish();
                } else {
                    dfa_range<true>(dv, text, n, L, R, sk);
                }
            } else if (MODE == QG_QGRAM && v.off_dfa) dfa_range_global(Q.plan, v, text, n, L, R, sk);
            else linear_range(v, text, n, L, R, sk);
        };

        // ---- count pass (q-gram filter per warp, or linear scan per thread
        // for dense items).  The filter of warp w covers the starts of its
        // 32 threads' ranges, [Lw, Lw + 32 R).
        Sink sink{SINK_BUFFER, nullptr, 0, 0, hbuf + tid, 0};
        const uint64_t Lw = k * R * QG_THREADS + static_cast<uint64_t>(warp) * 32u * R;
        uint64_t patw = 0;
        uint32_t wcnt = 0;
        bool wovf = false;
        if (MODE == QG_QGRAM) {
            const uint32_t pre = min(v.m, 8u);
            patw = *reinterpret_cast<const uint64_t *>(v.pat);  // 16-byte aligned, zero padded
            if (pre < 8) patw &= (1ull << (8u * pre)) - 1ull;
            QGRun run;
            const bool fine = qgram_warp(v, patw, text, n, Lw, 32u * R, QGOut{&qgw[warp], nullptr, 0, 0, 0u}, run);
            wcnt = run.cnt;
            wovf = run.ovf != 0;
            if (!fine && lane == 0) ctl.dense = 1u;
        }
        __syncthreads();
        const bool dense = ctl.dense != 0;
        if (dense) {
            sink.cnt = 0;
            linear(sink);
        }
        // Sparse q-gram items: the warp's total stands on its lane 0, so the
        // block scan below yields the warp's output offset there.
        const uint32_t cnt = dense ? sink.cnt : (lane == 0 ? wcnt : 0u);

        // ---- block scan + look-back
        uint32_t x = cnt;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= d) x += y;
        }
        if (lane == 31) ctl.warp_ex[warp] = x;
        __syncthreads();
        if (warp == 0) {
            const uint32_t val = lane < NW ? ctl.warp_ex[lane] : 0u;
            uint32_t sc = val;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, sc, d);
                if (lane >= d) sc += y;
            }
            const uint32_t total = __shfl_sync(0xffffffffu, sc, 31);
            if (lane < NW) ctl.warp_ex[lane] = sc - val;
            bool ok;
            const uint64_t ex = lookback_exclusive(Q.state, k, total, a.err, &ok);
            if (lane == 0) {
                ctl.excl = ex;
                ctl.ok = ok ? 1u : 0u;
                if (ok && k + 1 == Q.ntiles) *Q.out_count = ex + total;
            }
        }
        __syncthreads();

        // ---- write pass
        if (ctl.ok) {
            const uint64_t base = ctl.excl + ctl.warp_ex[warp] + (x - cnt);
            if (dense) {
                const bool over = cnt > QG_HB;
                if (!over) {
                    for (uint32_t r = 0; r < cnt; ++r) {
                        const uint64_t idx = base + r;
                        if (idx < Q.cap) Q.out_pos[idx] = L + hbuf[r * QG_THREADS + tid];
                    }
                } else {
                    // Threads whose hits did not fit recompute their range
                    // in write mode.
                    Sink w{SINK_WRITE, Q.out_pos, Q.cap, base, nullptr, 0};
                    linear(w);
                }
            } else if (MODE == QG_QGRAM) {
                const uint64_t bw = __shfl_sync(0xffffffffu, base, 0);
                if (!wovf) {
                    const uint64_t cap = Q.cap;
                    uint64_t *out = Q.out_pos;
                    for (uint32_t r = lane; r < wcnt; r += 32) {
                        if (bw + r < cap) out[bw + r] = Lw + qgw[warp].list[r];
                    }
                } else {
                    // More hits than the warp's list holds: run the filter
                    // again, writing at the final offsets.
                    QGRun run;
                    qgram_warp(v, patw, text, n, Lw, 32u * R, QGOut{&qgw[warp], Q.out_pos, Q.cap, bw, 1u}, run);
                }
            }
        }
        __syncthreads();
    }
}

}  // namespace

const void *qg_kernel_fn(int kid) {
    if (kid == K_QGRAM) return reinterpret_cast<const void *>(&qg_kernel<QG_QGRAM>);
    if (kid == K_LINEAR) return reinterpret_cast<const void *>(&qg_kernel<QG_KMP>);
    if (kid == K_DFA) return reinterpret_cast<const void *>(&qg_kernel<QG_DFA>);
    return nullptr;
}

int qg_kernel_threads() { return QG_THREADS; }

}  // namespace smgpu
