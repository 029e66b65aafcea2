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
//   * A persistent block claims work items (query, tile) from a device
//     counter.  A tile is T = THREADS * S start positions; its T + 64 bytes
//     are staged HBM -> shared memory by one cp.async.bulk (TMA 1-D copy)
//     completing on an mbarrier, double-buffered so the next tile streams in
//     while this one is scanned.
//   * Thread `tid` scans its own S = 16 * SEGC bytes plus up to 16*HCMAX
//     bytes of the next segment (the m-1 byte halo), 16 bytes per 128-bit
//     shared load.  S is an odd multiple of 16 bytes, so the eight lanes of
//     each quarter-warp read eight different 16-byte bank groups.
//   * When bits m..m+15 of the state are spare (32-bit state and m <= 17,
//     64-bit state and m <= 49), B[c] has ones there, so those bits carry
//     the match flags of the last 16 positions: one shift per 16 bytes
//     yields all 16 flags (variant "H").  Otherwise the state is ORed into
//     an accumulator and a chunk with a match is re-scanned (variant "A").
//   * Per-thread counts -> warp shuffle scan -> block scan -> decoupled
//     look-back across the tiles of the query -> every thread writes its
//     hits in increasing order at its global offset (capped by `cap`).
//
// Text positions are handled in a "virtual" frame shifted by
// o = text & 15, so every tile starts on a 16-byte boundary in memory.
#include "sm_internal.h"

namespace smgpu {

namespace {

constexpr int SO_THREADS = 128;
constexpr int SO_SEGC = 15;  // chunks of 16 bytes per thread segment (odd)

template <typename Word, int THREADS, int SEGC>
struct SOCfg {
    static constexpr int S = SEGC * 16;
    static constexpr uint32_t T = THREADS * S;
    static constexpr uint32_t HALO = 64;  // >= m-1 for m <= 64, multiple of 16
    static constexpr uint32_t BUF = T + HALO;
    static constexpr uint32_t TBL = 256 * sizeof(Word);
};

struct SOCtl {
    uint64_t bar[2];
    unsigned long long ticket[2];
    uint64_t tile[2];
    uint32_t qi[2];
    uint64_t excl;
    uint32_t warp_ex[32];
    uint32_t tile_total;
    uint32_t ok;
};

template <typename Word, int THREADS, int SEGC>
constexpr size_t so_smem_bytes() {
    return 2 * SOCfg<Word, THREADS, SEGC>::BUF + SOCfg<Word, THREADS, SEGC>::TBL + sizeof(SOCtl);
}

template <typename Word>
__device__ __forceinline__ void so_step4(Word &D, uint32_t x, const Word *__restrict__ tbl) {
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const uint32_t c = __byte_perm(x, 0u, 0x4440u | b);
        D = ((D << 1) | Word(1)) & tbl[c];
    }
}

// Exact flags of one 16-byte chunk (bit 15-b <=> an occurrence ends at byte
// b of the chunk), re-scanned from the state at the chunk start.
template <typename Word>
__device__ __noinline__ uint32_t so_chunk_flags(Word D, const uint8_t *chunk, const Word *tbl,
                                                uint32_t m) {
    uint32_t f = 0;
#pragma unroll 1
    for (int b = 0; b < 16; ++b) {
        D = ((D << 1) | Word(1)) & tbl[chunk[b]];
        f |= static_cast<uint32_t>((D >> (m - 1)) & Word(1)) << (15 - b);
    }
    return f;
}

// Bits r of a chunk starting at segment byte cb whose end e = cb + 15 - r
// lies in [elo, ehi).
__device__ __forceinline__ uint32_t range_mask16(int cb, int elo, int ehi) {
    const int lo = max(cb + 16 - ehi, 0);
    const int hi = min(cb + 15 - elo, 15);
    if (lo > hi) return 0u;
    return ((2u << hi) - 1u) & ~((1u << lo) - 1u);
}

template <typename Word, int THREADS, int SEGC>
__device__ __forceinline__ void so_claim(const LaunchArgs &a, SOCtl &ctl, int b, uint8_t *bufs) {
    using C = SOCfg<Word, THREADS, SEGC>;
    const unsigned long long t = atomicAdd(a.ticket, 1ull);
    ctl.ticket[b] = t;
    if (t >= a.total) return;
    uint32_t qi;
    uint64_t k;
    resolve_ticket(a, t, &qi, &k);
    ctl.qi[b] = qi;
    ctl.tile[b] = k;
    const QueryDev &Q = query_of(a, qi);
    const uint64_t o = reinterpret_cast<uintptr_t>(Q.text) & 15u;
    const uint8_t *base = Q.text - o;
    const uint64_t vstart = k * static_cast<uint64_t>(C::T);
    const uint64_t vlim = (o + Q.n + 15u) & ~uint64_t(15);
    const uint64_t vend = min(vstart + C::BUF, vlim);
    const uint32_t bytes = static_cast<uint32_t>(vend - vstart);
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&ctl.bar[b], bytes);
    bulk_g2s(bufs + b * C::BUF, base + vstart, bytes, &ctl.bar[b]);
}

template <typename Word, bool HIST, int HCMAX, int THREADS, int SEGC>
__global__ void __launch_bounds__(THREADS) so_kernel(const LaunchArgs a) {
    using C = SOCfg<Word, THREADS, SEGC>;
    constexpr int S = C::S;
    constexpr int NCH = SEGC + HCMAX;
    constexpr int NW = THREADS / 32;
    extern __shared__ __align__(128) uint8_t smem[];
    uint8_t *bufs = smem;
    Word *tbl = reinterpret_cast<Word *>(smem + 2 * C::BUF);
    SOCtl &ctl = *reinterpret_cast<SOCtl *>(smem + 2 * C::BUF + C::TBL);
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;

    if (tid == 0) {
        mbar_init(&ctl.bar[0], 1);
        mbar_init(&ctl.bar[1], 1);
        fence_mbar_init();
        so_claim<Word, THREADS, SEGC>(a, ctl, 0, bufs);
    }
    __syncthreads();

    const PlanDev *cur_plan = nullptr;
    uint32_t m = 1;
    uint32_t parity = 0;  // bit b: parity of the next phase of bar[b]
    int cur = 0;
    while (true) {
        const unsigned long long t = ctl.ticket[cur];
        if (t >= a.total) break;
        const uint32_t qi = ctl.qi[cur];
        const uint64_t k = ctl.tile[cur];
        const QueryDev &Q = query_of(a, qi);
        const PlanDev *P = Q.plan;
        if (P != cur_plan) {
            const Word *src = reinterpret_cast<const Word *>(reinterpret_cast<const uint8_t *>(P) +
                                                             __ldg(&P->off_tbl));
            for (int c = tid; c < 256; c += THREADS) tbl[c] = src[c];
            cur_plan = P;
            m = __ldg(&P->m);
        }
        __syncthreads();
        if (tid == 0) so_claim<Word, THREADS, SEGC>(a, ctl, cur ^ 1, bufs);

        const bool arrived = mbar_wait_bounded(&ctl.bar[cur], (parity >> cur) & 1u);
        parity ^= 1u << cur;
        if (!__syncthreads_and(arrived)) {
            // The tile never arrived: fail it and the prefetched one, wait
            // (bounded) for the prefetch copy, and leave.
            if (tid == 0) {
                atomicOr(a.err, ERR_COPY);
                st_relaxed(&Q.state[k], LB_ERR);
                const unsigned long long t2 = ctl.ticket[cur ^ 1];
                if (t2 < a.total) {
                    const QueryDev &Q2 = query_of(a, ctl.qi[cur ^ 1]);
                    st_relaxed(&Q2.state[ctl.tile[cur ^ 1]], LB_ERR);
                    mbar_wait_bounded(&ctl.bar[cur ^ 1], (parity >> (cur ^ 1)) & 1u);
                }
            }
            return;
        }

        // ---- scan this thread's segment
        const uint8_t *seg = bufs + cur * C::BUF + tid * S;
        const int64_t o = static_cast<int64_t>(reinterpret_cast<uintptr_t>(Q.text) & 15u);
        const int64_t V = o + static_cast<int64_t>(Q.n) - static_cast<int64_t>(m) + 1;
        const int64_t base = static_cast<int64_t>(k) * C::T + static_cast<int64_t>(tid) * S;
        const int lo_s = static_cast<int>(o - base > 0 ? o - base : int64_t(0));
        const int hi_s = static_cast<int>(V - base < S ? V - base : int64_t(S));
        const uint32_t hc = (m + 14u) >> 4;  // halo chunks: ceil((m-1)/16)

        uint32_t F[NCH];
        Word D = 0;
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
            if (c < SEGC || static_cast<uint32_t>(c - SEGC) < hc) {
                const uint4 w = *reinterpret_cast<const uint4 *>(seg + 16 * c);
                if (HIST) {
                    so_step4(D, w.x, tbl);
                    so_step4(D, w.y, tbl);
                    so_step4(D, w.z, tbl);
                    so_step4(D, w.w, tbl);
                    F[c] = static_cast<uint32_t>(D >> (m - 1)) & 0xFFFFu;
                } else {
                    const Word Ds = D;
                    Word A = 0;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const uint32_t x = q == 0 ? w.x : q == 1 ? w.y : q == 2 ? w.z : w.w;
#pragma unroll
                        for (int b = 0; b < 4; ++b) {
                            const uint32_t ch = __byte_perm(x, 0u, 0x4440u | b);
                            D = ((D << 1) | Word(1)) & tbl[ch];
                            A |= D;
                        }
                    }
                    F[c] = ((A >> (m - 1)) & Word(1)) ? so_chunk_flags<Word>(Ds, seg + 16 * c, tbl, m)
                                                       : 0u;
                }
            } else {
                F[c] = 0u;
            }
        }

        // ---- keep ends e in [lo_s + m - 1, hi_s + m - 1) and count
        uint32_t cnt = 0;
        if (hi_s <= lo_s) {
#pragma unroll
            for (int c = 0; c < NCH; ++c) F[c] = 0u;
        } else {
            const int elo = lo_s + static_cast<int>(m) - 1;
            const int ehi = hi_s + static_cast<int>(m) - 1;
            const bool full = lo_s == 0 && hi_s == S;
#pragma unroll
            for (int c = 0; c < NCH; ++c) {
                if (!full || c >= SEGC) F[c] &= range_mask16(16 * c, elo, ehi);
                cnt += __popc(F[c]);
            }
        }

        // ---- block scan of counts
        uint32_t x = cnt;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= d) x += y;
        }
        if (lane == 31) ctl.warp_ex[warp] = x;
        __syncthreads();
        if (warp == 0) {
            uint32_t v = lane < NW ? ctl.warp_ex[lane] : 0u;
            uint32_t s = v;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, s, d);
                if (lane >= d) s += y;
            }
            const uint32_t total = __shfl_sync(0xffffffffu, s, 31);
            if (lane < NW) ctl.warp_ex[lane] = s - v;
            bool ok;
            const uint64_t ex = lookback_exclusive(Q.state, k, total, a.err, &ok);
            if (lane == 0) {
                ctl.excl = ex;
                ctl.tile_total = total;
                ctl.ok = ok ? 1u : 0u;
                if (ok && k + 1 == Q.ntiles) *Q.out_count = ex + total;
            }
        }
        __syncthreads();

        // ---- write hits in increasing order
        if (cnt != 0 && ctl.ok) {
            uint64_t idx = ctl.excl + ctl.warp_ex[warp] + (x - cnt);
            const uint64_t cap = Q.cap;
            uint64_t *out = Q.out_pos;
            const int64_t rbase = base - o - static_cast<int64_t>(m) + 1;
#pragma unroll
            for (int c = 0; c < NCH; ++c) {
                uint32_t f = F[c];
                while (f) {
                    const int r = 31 - __clz(f);
                    f ^= 1u << r;
                    const uint64_t pos = static_cast<uint64_t>(rbase + 16 * c + 15 - r);
                    if (idx < cap) out[idx] = pos;
                    ++idx;
                }
            }
        }
        __syncthreads();
        cur ^= 1;
    }
}

}  // namespace

// ---------------------------------------------------------------- registry

#define SO_INST(W, H, HC) so_kernel<W, H, HC, SO_THREADS, SO_SEGC>

const void *so_kernel_fn(int kid) {
    switch (kid) {
        case K_SO32H: return reinterpret_cast<const void *>(&SO_INST(uint32_t, true, 1));
        case K_SO32A: return reinterpret_cast<const void *>(&SO_INST(uint32_t, false, 2));
        case K_SO64H: return reinterpret_cast<const void *>(&SO_INST(uint64_t, true, 3));
        case K_SO64A: return reinterpret_cast<const void *>(&SO_INST(uint64_t, false, 4));
        default: return nullptr;
    }
}

size_t so_kernel_smem(int kid) {
    return (kid == K_SO32H || kid == K_SO32A) ? so_smem_bytes<uint32_t, SO_THREADS, SO_SEGC>()
                                              : so_smem_bytes<uint64_t, SO_THREADS, SO_SEGC>();
}

int so_kernel_threads() { return SO_THREADS; }

uint64_t so_tile_starts() { return SOCfg<uint32_t, SO_THREADS, SO_SEGC>::T; }

}  // namespace smgpu
