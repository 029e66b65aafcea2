/*
 * CPU oracle for the online exact string matching problem.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file: only tests/, __graft_entry__.smoke() and the cpu_baseline /
 * reference leg of bench.py use it.  It shares no code, header, table or
 * helper with the CUDA library.
 *
 * What it computes (Faro & Lecroq, Section 1, problem statement): given a
 * text t of length n and a pattern p of length m over an alphabet Sigma,
 * report ALL occurrences of p in t, i.e. the set
 *
 *     H = { i in [0, n-m] : t[i+j] = p[j] for every 0 <= j < m }
 *
 * as 0-based start positions in increasing order.  Overlapping occurrences
 * are all reported (the abstract stresses "all" occurrences).  Symbols are
 * bytes 0..255.  m = 0 is outside the definition (callers reject it);
 * m > n gives the empty set.
 *
 * Three routines:
 *   oracle_naive    - the definition written out: every alignment i, every
 *                     j, byte by byte, no early library calls (this is the
 *                     Brute-Force algorithm of Fig. 1).
 *   oracle_kmp      - Knuth-Morris-Pratt (Fig. 1), an independent linear
 *                     algorithm, used as a cross-check of the naive routine
 *                     and for inputs where the naive loop is O(n m).
 *   oracle_naive_mt - oracle_naive over text chunks on several POSIX
 *                     threads; chunk c owns the start positions
 *                     [lo_c, hi_c) and reads bytes [lo_c, hi_c + m - 1).
 * and one helper for the exhaustive binary check (oracle_binary_masks).
 *
 * Parity pins (tests/test_oracle.py): exhaustive comparison over every
 * binary (text, pattern) pair with n <= 12 against an integer-window
 * formulation; closed forms (a^m in a^n, m = 1, m > n, absent symbol);
 * Python's bytes.find and re overlapping search as library routines;
 * hand-derived fixtures in tests/golden/; and planted-mutation tests.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Write position i as the next hit; count every hit even past cap. */
static inline void emit(uint64_t *out, uint64_t cap, uint64_t *cnt, uint64_t i) {
    if (*cnt < cap) out[*cnt] = i;
    (*cnt)++;
}

/* Start positions in [lo, hi) only; bytes up to hi + m - 2 are read. */
static uint64_t naive_range(const uint8_t *t, uint64_t lo, uint64_t hi,
                            const uint8_t *p, uint64_t m, uint64_t *out, uint64_t cap) {
    uint64_t cnt = 0;
    for (uint64_t i = lo; i < hi; ++i) {
        uint64_t j = 0;
        while (j < m && t[i + j] == p[j]) ++j;
        if (j == m) emit(out, cap, &cnt, i);
    }
    return cnt;
}

/* Returns |H|; the first min(|H|, cap) positions go to out in order. */
uint64_t oracle_naive(const uint8_t *t, uint64_t n, const uint8_t *p, uint64_t m,
                      uint64_t *out, uint64_t cap) {
    if (m == 0 || m > n) return 0;
    return naive_range(t, 0, n - m + 1, p, m, out, cap);
}

/*
 * Knuth-Morris-Pratt.  fail[q] (q = 1..m) is the length of the longest
 * proper border of p[0..q-1] (a border is a string that is both a prefix and
 * a suffix).  While scanning, q is the length of the longest prefix of p
 * that is a suffix of the text read so far; on a mismatch q falls back along
 * the border chain.
 */
uint64_t oracle_kmp(const uint8_t *t, uint64_t n, const uint8_t *p, uint64_t m,
                    uint64_t *out, uint64_t cap) {
    if (m == 0 || m > n) return 0;
    uint64_t *fail = (uint64_t *)malloc((m + 1) * sizeof(uint64_t));
    if (!fail) return UINT64_MAX;
    fail[0] = 0;
    if (m >= 1) fail[1] = 0;
    uint64_t k = 0;
    for (uint64_t q = 1; q < m; ++q) {
        while (k > 0 && p[k] != p[q]) k = fail[k];
        if (p[k] == p[q]) ++k;
        fail[q + 1] = k;
    }
    uint64_t cnt = 0, q = 0;
    for (uint64_t i = 0; i < n; ++i) {
        while (q > 0 && p[q] != t[i]) q = fail[q];
        if (p[q] == t[i]) ++q;
        if (q == m) {
            emit(out, cap, &cnt, i + 1 - m);
            q = fail[q];
        }
    }
    free(fail);
    return cnt;
}

typedef struct {
    const uint8_t *t;
    const uint8_t *p;
    uint64_t m, lo, hi;
    uint64_t *hits;
    uint64_t count, alloc;
    int failed;
    int want_hits;
} chunk_job;

static void *chunk_main(void *arg) {
    chunk_job *c = (chunk_job *)arg;
    /* First pass counts, second pass writes: no reallocation needed. */
    c->count = naive_range(c->t, c->lo, c->hi, c->p, c->m, NULL, 0);
    if (!c->want_hits) return NULL;
    c->alloc = c->count ? c->count : 1;
    c->hits = (uint64_t *)malloc(c->alloc * sizeof(uint64_t));
    if (!c->hits) { c->failed = 1; return NULL; }
    naive_range(c->t, c->lo, c->hi, c->p, c->m, c->hits, c->count);
    return NULL;
}

/* oracle_naive split over `threads` POSIX threads by start position. */
uint64_t oracle_naive_mt(const uint8_t *t, uint64_t n, const uint8_t *p, uint64_t m,
                         uint64_t *out, uint64_t cap, int threads) {
    if (m == 0 || m > n) return 0;
    if (threads < 1) threads = 1;
    uint64_t starts = n - m + 1;
    if ((uint64_t)threads > starts) threads = (int)starts;
    chunk_job *jobs = (chunk_job *)calloc((size_t)threads, sizeof(chunk_job));
    pthread_t *tid = (pthread_t *)calloc((size_t)threads, sizeof(pthread_t));
    if (!jobs || !tid) { free(jobs); free(tid); return UINT64_MAX; }
    for (int c = 0; c < threads; ++c) {
        jobs[c].t = t; jobs[c].p = p; jobs[c].m = m;
        jobs[c].want_hits = cap > 0;
        jobs[c].lo = starts * (uint64_t)c / (uint64_t)threads;
        jobs[c].hi = starts * (uint64_t)(c + 1) / (uint64_t)threads;
    }
    for (int c = 1; c < threads; ++c) {
        if (pthread_create(&tid[c], NULL, chunk_main, &jobs[c]) != 0) {
            chunk_main(&jobs[c]); /* no thread: run the chunk here */
            tid[c] = 0;
        }
    }
    chunk_main(&jobs[0]);
    for (int c = 1; c < threads; ++c)
        if (tid[c]) pthread_join(tid[c], NULL);
    uint64_t total = 0;
    int failed = 0;
    for (int c = 0; c < threads; ++c) {
        failed |= jobs[c].failed;
        if (!jobs[c].want_hits) {
            total += jobs[c].count;
            continue;
        }
        for (uint64_t k = 0; k < jobs[c].count && !jobs[c].failed; ++k) {
            if (total < cap) out[total] = jobs[c].hits[k];
            total++;
        }
        free(jobs[c].hits);
    }
    free(jobs);
    free(tid);
    return failed ? UINT64_MAX : total;
}

/*
 * Exhaustive binary check helper.  For every text of length n and every
 * pattern of length m over {0,1} (bit j of the integer is symbol j), run
 * the chosen routine (0 = naive, 1 = kmp) and store the set of hits as a
 * bitmask (bit i set <=> i is a hit) at masks[text * 2^m + pattern].
 * Requires n <= 16.
 */
int oracle_binary_masks(int n, int m, int which, uint32_t *masks) {
    if (n < 1 || n > 16 || m < 1 || m > n) return -1;
    uint8_t t[16], p[16];
    uint64_t hits[16];
    uint32_t nt = 1u << n, np_ = 1u << m;
    for (uint32_t tv = 0; tv < nt; ++tv) {
        for (int j = 0; j < n; ++j) t[j] = (uint8_t)((tv >> j) & 1u);
        for (uint32_t pv = 0; pv < np_; ++pv) {
            for (int j = 0; j < m; ++j) p[j] = (uint8_t)((pv >> j) & 1u);
            uint64_t c = which == 0 ? oracle_naive(t, (uint64_t)n, p, (uint64_t)m, hits, 16)
                                    : oracle_kmp(t, (uint64_t)n, p, (uint64_t)m, hits, 16);
            uint32_t mask = 0;
            for (uint64_t k = 0; k < c && k < 16; ++k) mask |= 1u << hits[k];
            masks[(size_t)tv * np_ + pv] = mask;
        }
    }
    return 0;
}
