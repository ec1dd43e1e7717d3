/*
 * glop_oracle.c -- CPU oracle for exact multi-pattern byte-string search.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this file's library.  It shares no code,
 * header, table or constant with the GPU library and must never be called by
 * the product path.
 *
 * What it computes (the graded definition).  Given a text t[0..n) of bytes
 * (all 256 values, length-delimited, no terminator) and patterns p_0..p_{P-1}
 * (byte strings of length >= 1, id = index in the list), the result is the set
 *     { (i, j) : i + |p_j| <= n  and  t[i .. i+|p_j|) == p_j }
 * emitted sorted by (i ascending, j ascending), as uint32 pairs.  This is the
 * set a Parallel Failureless Aho-Corasick scan reports when one walk starts at
 * every byte offset and every terminal state on the walk is reported (Sec. 5).
 * With prefix_len = K > 0 every pattern is first cut to its first
 * min(|p_j|, K) bytes (the prefix / partial matching of Sec. 1 and Sec. 5).
 *
 * Two independent ways to reach it:
 *   oracle_naive  -- the naive approach of Sec. 2: at every offset compare
 *                    every pattern byte by byte (patterns bucketed by their
 *                    first byte, ids kept ascending inside a bucket).
 *   oracle_ac     -- the Aho-Corasick automaton of Sec. 4: goto graph built
 *                    from the patterns, failure function by breadth-first
 *                    search, output(s) = own(s) U output(fail(s)); one pass
 *                    over the text with failure transitions; a match is seen
 *                    at its end position and converted to its start.
 *   oracle_ac_mt  -- the chunked multi-threaded form of Sec. 4: the text is
 *                    cut into chunks that overlap by (longest pattern - 1)
 *                    bytes; a chunk keeps only matches starting inside it.
 *   oracle_batch  -- the same definition per segment of a concatenated
 *                    buffer (offsets relative to the segment start; no match
 *                    crosses a segment end), as (segment, offset, id).
 *   oracle_ac_trace -- the goto/failure transitions the automaton takes on a
 *                    text, one line per text byte, for the worked example of
 *                    Sec. 4.
 *   oracle_kmp    -- Knuth-Morris-Pratt, the single-pattern method the paper
 *                    compares against (Sec. 2, Sec. 7), run once per pattern:
 *                    a third way to the same set.
 *
 * Return codes: 0 ok, 1 invalid argument (zero-length pattern, text longer
 * than 2^32-1 bytes, null pointer), 2 out of memory.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

/* ORACLE_MUTANT (default 0) plants one known mistake for the test suite's
 * mutation check, which rebuilds this file with -DORACLE_MUTANT=k and asserts
 * that the pins catch it.  A normal build never defines it. */
#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif

#define OR_OK 0
#define OR_EINVAL 1
#define OR_ENOMEM 2
#define NONE 0xFFFFFFFFu

/* ------------------------------------------------------------------ */
/* growable arrays of uint32 records                                    */
/* ------------------------------------------------------------------ */
typedef struct {
    uint32_t *a;
    uint64_t n, cap; /* counted in uint32 words */
} u32vec;

static int vec_push(u32vec *v, const uint32_t *rec, int w) {
    if (v->n + (uint64_t)w > v->cap) {
        uint64_t nc = v->cap ? v->cap * 2 : 1024;
        while (nc < v->n + (uint64_t)w) nc *= 2;
        uint32_t *na = (uint32_t *)realloc(v->a, nc * sizeof(uint32_t));
        if (!na) return OR_ENOMEM;
        v->a = na;
        v->cap = nc;
    }
    for (int k = 0; k < w; ++k) v->a[v->n + (uint64_t)k] = rec[k];
    v->n += (uint64_t)w;
    return OR_OK;
}

static int cmp_pair(const void *x, const void *y) {
    const uint32_t *a = (const uint32_t *)x, *b = (const uint32_t *)y;
    if (a[0] != b[0]) return a[0] < b[0] ? -1 : 1;
    if (a[1] != b[1]) return a[1] < b[1] ? -1 : 1;
    return 0;
}

void oracle_free(void *p) { free(p); }

/* effective pattern length under prefix mode */
static uint64_t eff_len(const uint64_t *poff, uint32_t j, uint32_t prefix_len) {
    uint64_t L = poff[j + 1] - poff[j];
    if (prefix_len && L > prefix_len) L = prefix_len + (ORACLE_MUTANT == 6 ? 1 : 0);
    return L;
}

static int check_patterns(const uint64_t *poff, uint32_t npat, uint32_t prefix_len, uint64_t *maxlen) {
    uint64_t m = 0;
    for (uint32_t j = 0; j < npat; ++j) {
        if (poff[j + 1] < poff[j]) return OR_EINVAL;
        uint64_t L = eff_len(poff, j, prefix_len);
        if (L == 0) return OR_EINVAL;
        if (L > m) m = L;
    }
    *maxlen = m;
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* naive oracle (Sec. 2)                                                */
/* ------------------------------------------------------------------ */
typedef struct {
    uint32_t *head;  /* [256] first pattern id with that first byte, NONE if none */
    uint32_t *next;  /* [npat] next id in the same bucket (ascending) */
} buckets_t;

static int build_buckets(const uint8_t *pat, const uint64_t *poff, uint32_t npat, buckets_t *b) {
    b->head = (uint32_t *)malloc(256 * sizeof(uint32_t));
    b->next = (uint32_t *)malloc(((size_t)npat + 1) * sizeof(uint32_t));
    if (!b->head || !b->next) return OR_ENOMEM;
    uint32_t tail[256];
    for (int c = 0; c < 256; ++c) b->head[c] = tail[c] = NONE;
    for (uint32_t j = 0; j < npat; ++j) {
        uint8_t c = pat[poff[j]];
        b->next[j] = NONE;
        if (b->head[c] == NONE) b->head[c] = j; else b->next[tail[c]] = j;
        tail[c] = j;
    }
    return OR_OK;
}

/* every match starting in [lo, hi) of text[0..n); offsets reported as i - base */
static int naive_range(const uint8_t *text, uint64_t n, uint64_t lo, uint64_t hi, uint64_t base,
                       const uint8_t *pat, const uint64_t *poff, uint32_t prefix_len,
                       const buckets_t *b, int with_seg, uint32_t seg, u32vec *out) {
    for (uint64_t i = lo; i < hi; ++i) {
        for (uint32_t j = b->head[text[i]]; j != NONE; j = b->next[j]) {
            uint64_t L = eff_len(poff, j, prefix_len);
            if (ORACLE_MUTANT == 1 ? i + L >= n : i + L > n) continue;
            if (memcmp(text + i, pat + poff[j], (size_t)L - (ORACLE_MUTANT == 7 ? 1 : 0)) != 0) continue;
            uint32_t rec[3];
            int w = 0;
            if (with_seg) rec[w++] = seg;
            rec[w++] = (uint32_t)(i - base);
            rec[w++] = j;
            if (vec_push(out, rec, w)) return OR_ENOMEM;
        }
    }
    return OR_OK;
}

int oracle_naive(const uint8_t *text, uint64_t n, const uint8_t *pat, const uint64_t *poff,
                 uint32_t npat, uint32_t prefix_len, uint32_t **out, uint64_t *count) {
    *out = NULL;
    *count = 0;
    if ((!text && n) || !poff || (npat && !pat) || n > 0xFFFFFFFFull) return OR_EINVAL;
    uint64_t maxlen;
    int rc = check_patterns(poff, npat, prefix_len, &maxlen);
    if (rc) return rc;
    if (npat == 0 || n == 0) return OR_OK;
    buckets_t b;
    rc = build_buckets(pat, poff, npat, &b);
    u32vec v = {0, 0, 0};
    if (!rc) rc = naive_range(text, n, 0, n, 0, pat, poff, prefix_len, &b, 0, 0, &v);
    free(b.head);
    free(b.next);
    if (rc) { free(v.a); return rc; }
    *out = v.a;
    *count = v.n / 2;
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Knuth-Morris-Pratt, once per pattern (Sec. 2, Sec. 7)                */
/* ------------------------------------------------------------------ */
static void sort_records(u32vec *v, int w);

/* For pattern p of length m, border[q] is the length of the longest proper
 * prefix of p[0..q] that is also a suffix of it.  The scan keeps q = the
 * length of the longest prefix of p that ends at the current text byte; on
 * a mismatch it falls back along the borders.  q == m is an occurrence
 * ending here, which then continues from border[m-1]. */
int oracle_kmp(const uint8_t *text, uint64_t n, const uint8_t *pat, const uint64_t *poff,
               uint32_t npat, uint32_t prefix_len, uint32_t **out, uint64_t *count) {
    *out = NULL;
    *count = 0;
    if ((!text && n) || !poff || (npat && !pat) || n > 0xFFFFFFFFull) return OR_EINVAL;
    uint64_t maxlen;
    int rc = check_patterns(poff, npat, prefix_len, &maxlen);
    if (rc) return rc;
    if (npat == 0 || n == 0) return OR_OK;
    uint64_t *border = (uint64_t *)malloc((size_t)maxlen * sizeof(uint64_t));
    if (!border) return OR_ENOMEM;
    u32vec v = {0, 0, 0};
    for (uint32_t j = 0; j < npat && !rc; ++j) {
        const uint8_t *p = pat + poff[j];
        const uint64_t m = eff_len(poff, j, prefix_len);
        border[0] = 0;
        for (uint64_t q = 1, k = 0; q < m; ++q) {
            while (k > 0 && p[q] != p[k]) k = border[k - 1];
            if (p[q] == p[k]) ++k;
            border[q] = k;
        }
        for (uint64_t i = 0, q = 0; i < n; ++i) {
            while (q > 0 && text[i] != p[q]) q = border[q - 1];
            if (text[i] == p[q]) ++q;
            if (q == m) {
                const uint32_t rec[2] = {(uint32_t)(i + 1 - m), j};
                rc = vec_push(&v, rec, 2);
                if (rc) break;
                q = ORACLE_MUTANT == 9 ? 0 : border[m - 1];
            }
        }
    }
    free(border);
    if (rc) { free(v.a); return rc; }
    sort_records(&v, 2);
    *out = v.a;
    *count = v.n / 2;
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Aho-Corasick oracle (Sec. 4)                                         */
/* ------------------------------------------------------------------ */
typedef struct {
    uint32_t nnodes;
    uint32_t root_goto[256]; /* g(0, a); 0 = stay at the root (the root never fails) */
    uint32_t *edge_head;     /* per node: first outgoing edge, NONE if none */
    uint32_t *edge_next;     /* per edge (edge id = child node id): sibling edge */
    uint8_t *edge_byte;      /* per node: byte on the edge into it */
    uint32_t *parent;        /* per node */
    uint32_t *fail;          /* failure function f(s) */
    uint32_t *dict;          /* nearest state on the failure chain with own outputs, 0 if none */
    uint32_t *own_head;      /* per node: first pattern id ending here, NONE if none */
    uint32_t *own_next;      /* per pattern: next pattern id ending at the same node */
    uint32_t *plen;          /* per pattern: effective length */
} ac_t;

static void ac_free(ac_t *a) {
    free(a->edge_head); free(a->edge_next); free(a->edge_byte); free(a->parent);
    free(a->fail); free(a->dict); free(a->own_head); free(a->own_next); free(a->plen);
    memset(a, 0, sizeof(*a));
}

/* goto function for a non-root state: child on byte c, or NONE (fail) */
static inline uint32_t ac_find(const ac_t *a, uint32_t s, uint8_t c) {
    if (s == 0) return a->root_goto[c]; /* never fails */
    for (uint32_t e = a->edge_head[s]; e != NONE; e = a->edge_next[e])
        if (a->edge_byte[e] == c) return e;
    return NONE;
}

static int ac_build(ac_t *a, const uint8_t *pat, const uint64_t *poff, uint32_t npat, uint32_t prefix_len) {
    memset(a, 0, sizeof(*a));
    uint64_t total = 1;
    for (uint32_t j = 0; j < npat; ++j) total += eff_len(poff, j, prefix_len);
    if (total > 0xFFFFFFF0ull) return OR_EINVAL;
    size_t N = (size_t)total;
    a->edge_head = (uint32_t *)malloc(N * sizeof(uint32_t));
    a->edge_next = (uint32_t *)malloc(N * sizeof(uint32_t));
    a->edge_byte = (uint8_t *)malloc(N);
    a->parent = (uint32_t *)malloc(N * sizeof(uint32_t));
    a->fail = (uint32_t *)malloc(N * sizeof(uint32_t));
    a->dict = (uint32_t *)malloc(N * sizeof(uint32_t));
    a->own_head = (uint32_t *)malloc(N * sizeof(uint32_t));
    a->own_next = (uint32_t *)malloc(((size_t)npat + 1) * sizeof(uint32_t));
    a->plen = (uint32_t *)malloc(((size_t)npat + 1) * sizeof(uint32_t));
    if (!a->edge_head || !a->edge_next || !a->edge_byte || !a->parent || !a->fail || !a->dict ||
        !a->own_head || !a->own_next || !a->plen) { ac_free(a); return OR_ENOMEM; }
    memset(a->root_goto, 0, sizeof(a->root_goto));
    a->nnodes = 1;
    a->edge_head[0] = NONE; a->own_head[0] = NONE; a->parent[0] = 0; a->edge_byte[0] = 0;

    /* phase 1a: goto graph (the trie of the patterns) */
    for (uint32_t j = 0; j < npat; ++j) {
        uint32_t L = (uint32_t)eff_len(poff, j, prefix_len);
        a->plen[j] = L;
        const uint8_t *p = pat + poff[j];
        uint32_t s = 0;
        for (uint32_t k = 0; k < L; ++k) {
            uint32_t nx = (s == 0) ? (a->root_goto[p[k]] ? a->root_goto[p[k]] : NONE) : ac_find(a, s, p[k]);
            if (nx == NONE) {
                nx = a->nnodes++;
                a->edge_head[nx] = NONE; a->own_head[nx] = NONE;
                a->edge_byte[nx] = p[k]; a->parent[nx] = s;
                if (s == 0) { a->root_goto[p[k]] = nx; a->edge_next[nx] = NONE; }
                else { a->edge_next[nx] = a->edge_head[s]; a->edge_head[s] = nx; }
            }
            s = nx;
        }
        a->own_next[j] = a->own_head[s]; /* own list; order is irrelevant, results are sorted */
        a->own_head[s] = j;
    }

    /* phase 1b: failure function by breadth-first search over the goto graph */
    uint32_t *queue = (uint32_t *)malloc((size_t)a->nnodes * sizeof(uint32_t));
    if (!queue) { ac_free(a); return OR_ENOMEM; }
    uint32_t qh = 0, qt = 0;
    a->fail[0] = 0; a->dict[0] = 0;
    for (int c = 0; c < 256; ++c) {
        uint32_t s = a->root_goto[c];
        if (s) { a->fail[s] = 0; a->dict[s] = 0; queue[qt++] = s; }
    }
    while (qh < qt) {
        uint32_t r = queue[qh++];
        for (uint32_t s = a->edge_head[r]; s != NONE; s = a->edge_next[s]) {
            queue[qt++] = s;
            uint8_t c = a->edge_byte[s];
            uint32_t st = a->fail[r];
            while (st != 0 && ac_find(a, st, c) == NONE) st = a->fail[st];
            uint32_t f = ac_find(a, st, c); /* st == 0 -> root goto, 0 if absent */
            if (ORACLE_MUTANT == 5) f = 0;
            a->fail[s] = f;
            /* output(s) = own(s) U output(f(s)): keep a link to the nearest
               state on the failure chain that owns outputs */
            a->dict[s] = (a->own_head[f] != NONE) ? f : a->dict[f];
            if (ORACLE_MUTANT == 2) a->dict[s] = 0;
        }
    }
    free(queue);
    return OR_OK;
}

/* one pass over text[lo..hi_ext); report matches whose start is in [lo, hi_own) */
static int ac_range(const ac_t *a, const uint8_t *text, uint64_t lo, uint64_t hi_own, uint64_t hi_ext,
                    uint64_t base, int with_seg, uint32_t seg, u32vec *out) {
    uint32_t s = 0;
    for (uint64_t i = lo; i < hi_ext; ++i) {
        uint8_t c = text[i];
        while (s != 0 && ac_find(a, s, c) == NONE) s = a->fail[s];
        s = ac_find(a, s, c);
        uint32_t u = (a->own_head[s] != NONE) ? s : a->dict[s];
        for (; u != 0; u = a->dict[u]) {
            for (uint32_t j = a->own_head[u]; j != NONE; j = a->own_next[j]) {
                uint64_t start = i + 1 - a->plen[j] - (ORACLE_MUTANT == 3 ? 1 : 0);
                if (start < lo || start >= hi_own) continue;
                uint32_t rec[3];
                int w = 0;
                if (with_seg) rec[w++] = seg;
                rec[w++] = (uint32_t)(start - base);
                rec[w++] = j;
                if (vec_push(out, rec, w)) return OR_ENOMEM;
            }
        }
    }
    return OR_OK;
}

static void sort_records(u32vec *v, int w) {
    if (w == 2) qsort(v->a, (size_t)(v->n / 2), 2 * sizeof(uint32_t), cmp_pair);
}

int oracle_ac(const uint8_t *text, uint64_t n, const uint8_t *pat, const uint64_t *poff,
              uint32_t npat, uint32_t prefix_len, uint32_t **out, uint64_t *count) {
    *out = NULL;
    *count = 0;
    if ((!text && n) || !poff || (npat && !pat) || n > 0xFFFFFFFFull) return OR_EINVAL;
    uint64_t maxlen;
    int rc = check_patterns(poff, npat, prefix_len, &maxlen);
    if (rc) return rc;
    if (npat == 0 || n == 0) return OR_OK;
    ac_t a;
    rc = ac_build(&a, pat, poff, npat, prefix_len);
    if (rc) return rc;
    u32vec v = {0, 0, 0};
    rc = ac_range(&a, text, 0, n, n, 0, 0, 0, &v);
    ac_free(&a);
    if (rc) { free(v.a); return rc; }
    sort_records(&v, 2);
    *out = v.a;
    *count = v.n / 2;
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* chunked multi-threaded Aho-Corasick (Sec. 4, chunk overlap)          */
/* ------------------------------------------------------------------ */
typedef struct {
    const ac_t *a;
    const uint8_t *text;
    uint64_t n, lo, hi, overlap;
    u32vec v;
    int rc;
} mt_job;

static void *mt_worker(void *arg) {
    mt_job *jb = (mt_job *)arg;
    uint64_t ext = jb->hi + jb->overlap;
    if (ext > jb->n) ext = jb->n;
    jb->rc = ac_range(jb->a, jb->text, jb->lo, jb->hi, ext, 0, 0, 0, &jb->v);
    if (!jb->rc) sort_records(&jb->v, 2);
    return NULL;
}

int oracle_ac_mt(const uint8_t *text, uint64_t n, const uint8_t *pat, const uint64_t *poff,
                 uint32_t npat, uint32_t prefix_len, uint32_t nthreads,
                 uint32_t **out, uint64_t *count) {
    *out = NULL;
    *count = 0;
    if ((!text && n) || !poff || (npat && !pat) || n > 0xFFFFFFFFull) return OR_EINVAL;
    uint64_t maxlen;
    int rc = check_patterns(poff, npat, prefix_len, &maxlen);
    if (rc) return rc;
    if (npat == 0 || n == 0) return OR_OK;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 1024) nthreads = 1024;
    ac_t a;
    rc = ac_build(&a, pat, poff, npat, prefix_len);
    if (rc) return rc;
    mt_job *jobs = (mt_job *)calloc(nthreads, sizeof(mt_job));
    pthread_t *th = (pthread_t *)calloc(nthreads, sizeof(pthread_t));
    if (!jobs || !th) { free(jobs); free(th); ac_free(&a); return OR_ENOMEM; }
    uint64_t chunk = (n + nthreads - 1) / nthreads;
    for (uint32_t k = 0; k < nthreads; ++k) {
        jobs[k].a = &a; jobs[k].text = text; jobs[k].n = n;
        jobs[k].lo = (uint64_t)k * chunk < n ? (uint64_t)k * chunk : n;
        jobs[k].hi = jobs[k].lo + chunk < n ? jobs[k].lo + chunk : n;
        jobs[k].overlap = maxlen - 1 - (ORACLE_MUTANT == 4 && maxlen > 1 ? 1 : 0); /* longest pattern - 1 */
        pthread_create(&th[k], NULL, mt_worker, &jobs[k]);
    }
    uint64_t total = 0;
    for (uint32_t k = 0; k < nthreads; ++k) {
        pthread_join(th[k], NULL);
        if (jobs[k].rc) rc = jobs[k].rc;
        total += jobs[k].v.n;
    }
    uint32_t *res = NULL;
    if (!rc && total) {
        res = (uint32_t *)malloc((size_t)total * sizeof(uint32_t));
        if (!res) rc = OR_ENOMEM;
    }
    uint64_t at = 0;
    for (uint32_t k = 0; k < nthreads; ++k) {
        if (!rc && jobs[k].v.n) memcpy(res + at, jobs[k].v.a, (size_t)jobs[k].v.n * sizeof(uint32_t));
        at += jobs[k].v.n;
        free(jobs[k].v.a);
    }
    free(jobs); free(th); ac_free(&a);
    if (rc) { free(res); return rc; }
    *out = res;
    *count = total / 2;
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* batch: the definition applied per segment                            */
/* ------------------------------------------------------------------ */
typedef struct {
    const ac_t *a;
    const buckets_t *b;
    const uint8_t *text, *pat;
    const uint64_t *seg, *poff;
    uint32_t s_lo, s_hi, prefix_len;
    int method;
    u32vec v;
    int rc;
} batch_job;

static void *batch_worker(void *arg) {
    batch_job *jb = (batch_job *)arg;
    for (uint32_t s = jb->s_lo; s < jb->s_hi && !jb->rc; ++s) {
        uint64_t lo = jb->seg[s], hi = jb->seg[s + 1] + (ORACLE_MUTANT == 8 && s + 1 < jb->s_hi ? 1 : 0);
        if (hi <= lo) continue;
        uint64_t mark = jb->v.n;
        if (jb->method == 0)
            jb->rc = naive_range(jb->text + lo, hi - lo, 0, hi - lo, 0, jb->pat, jb->poff, jb->prefix_len,
                                 jb->b, 1, s, &jb->v);
        else {
            jb->rc = ac_range(jb->a, jb->text + lo, 0, hi - lo, hi - lo, 0, 1, s, &jb->v);
            /* AC reports by end position: sort this segment's (offset, id) */
            uint64_t cnt = (jb->v.n - mark) / 3;
            uint32_t *p = jb->v.a + mark;
            /* (segment, offset, id) triples of one segment: sort on (offset, id) */
            for (uint64_t x = 0; x < cnt; ++x) { p[2 * x] = p[3 * x + 1]; p[2 * x + 1] = p[3 * x + 2]; }
            qsort(p, (size_t)cnt, 2 * sizeof(uint32_t), cmp_pair);
            for (uint64_t x = cnt; x-- > 0;) {
                uint32_t o = p[2 * x], j = p[2 * x + 1];
                p[3 * x] = s; p[3 * x + 1] = o; p[3 * x + 2] = j;
            }
        }
    }
    return NULL;
}

int oracle_batch(const uint8_t *text, const uint64_t *seg, uint32_t nseg, const uint8_t *pat,
                 const uint64_t *poff, uint32_t npat, uint32_t prefix_len, int method,
                 uint32_t nthreads, uint32_t **out, uint64_t *count) {
    *out = NULL;
    *count = 0;
    if (!seg || !poff || (npat && !pat) || (method != 0 && method != 1)) return OR_EINVAL;
    for (uint32_t s = 0; s < nseg; ++s) {
        if (seg[s + 1] < seg[s]) return OR_EINVAL;
        if (seg[s + 1] - seg[s] > 0xFFFFFFFFull) return OR_EINVAL;
    }
    if (nseg && seg[nseg] > seg[0] && !text) return OR_EINVAL;
    uint64_t maxlen;
    int rc = check_patterns(poff, npat, prefix_len, &maxlen);
    if (rc) return rc;
    if (npat == 0 || nseg == 0) return OR_OK;
    ac_t a;
    memset(&a, 0, sizeof(a));
    buckets_t b = {0, 0};
    if (method == 1) rc = ac_build(&a, pat, poff, npat, prefix_len);
    else rc = build_buckets(pat, poff, npat, &b);
    if (rc) { free(b.head); free(b.next); return rc; }
    if (nthreads < 1) nthreads = 1;
    if (nthreads > nseg) nthreads = nseg;
    if (nthreads > 1024) nthreads = 1024;
    batch_job *jobs = (batch_job *)calloc(nthreads, sizeof(batch_job));
    pthread_t *th = (pthread_t *)calloc(nthreads, sizeof(pthread_t));
    if (!jobs || !th) { free(jobs); free(th); ac_free(&a); free(b.head); free(b.next); return OR_ENOMEM; }
    /* contiguous runs of segments with about equal bytes per thread */
    uint64_t tot = seg[nseg] - seg[0];
    uint32_t s = 0;
    for (uint32_t k = 0; k < nthreads; ++k) {
        jobs[k].a = &a; jobs[k].b = &b; jobs[k].text = text; jobs[k].pat = pat;
        jobs[k].seg = seg; jobs[k].poff = poff; jobs[k].prefix_len = prefix_len; jobs[k].method = method;
        jobs[k].s_lo = s;
        uint64_t goal = seg[0] + (tot * (uint64_t)(k + 1)) / nthreads;
        if (k == nthreads - 1) s = nseg;
        else while (s < nseg && seg[s + 1] <= goal) ++s;
        jobs[k].s_hi = s;
    }
    for (uint32_t k = 0; k < nthreads; ++k) pthread_create(&th[k], NULL, batch_worker, &jobs[k]);
    uint64_t total = 0;
    for (uint32_t k = 0; k < nthreads; ++k) {
        pthread_join(th[k], NULL);
        if (jobs[k].rc) rc = jobs[k].rc;
        total += jobs[k].v.n;
    }
    uint32_t *res = NULL;
    if (!rc && total) {
        res = (uint32_t *)malloc((size_t)total * sizeof(uint32_t));
        if (!res) rc = OR_ENOMEM;
    }
    uint64_t at = 0;
    for (uint32_t k = 0; k < nthreads; ++k) {
        if (!rc && jobs[k].v.n) memcpy(res + at, jobs[k].v.a, (size_t)jobs[k].v.n * sizeof(uint32_t));
        at += jobs[k].v.n;
        free(jobs[k].v.a);
    }
    free(jobs); free(th); ac_free(&a); free(b.head); free(b.next);
    if (rc) { free(res); return rc; }
    *out = res;
    *count = total / 3;
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* transition trace for the worked example of Sec. 4                   */
/* ------------------------------------------------------------------ */
static int label(const ac_t *a, uint32_t s, char *buf, size_t cap) {
    if (s == 0) { if (cap < 2) return -1; buf[0] = '$'; buf[1] = 0; return 1; }
    char tmp[4096];
    int d = 0;
    for (uint32_t u = s; u != 0 && d < 4095; u = a->parent[u]) tmp[d++] = (char)a->edge_byte[u];
    if ((size_t)d + 1 > cap) return -1;
    for (int k = 0; k < d; ++k) buf[k] = tmp[d - 1 - k];
    buf[d] = 0;
    return d;
}

/* One line per text byte: "<byte> f:<state> ... g:<state>", where f: is a
 * failure transition and g: the regular transition taken; states are named
 * by the pattern prefix they stand for, "$" for the initial state.  The
 * output set of the final state is appended as " out:<id>,<id>" when not
 * empty.  Returns the number of bytes written (without the terminator), or -1
 * when buf is too small / arguments are invalid. */
int64_t oracle_ac_trace(const uint8_t *text, uint64_t n, const uint8_t *pat, const uint64_t *poff,
                        uint32_t npat, char *buf, uint64_t cap) {
    uint64_t maxlen;
    if (!buf || cap == 0 || check_patterns(poff, npat, 0, &maxlen)) return -1;
    ac_t a;
    if (ac_build(&a, pat, poff, npat, 0)) return -1;
    uint64_t at = 0;
    char lab[4200];
    int bad = 0;
#define EMIT(...) do { int w_ = snprintf(buf + at, (size_t)(cap - at), __VA_ARGS__); \
        if (w_ < 0 || (uint64_t)w_ >= cap - at) { bad = 1; break; } at += (uint64_t)w_; } while (0)
    uint32_t s = 0;
    for (uint64_t i = 0; i < n && !bad; ++i) {
        uint8_t c = text[i];
        EMIT("%c", (c >= 0x21 && c < 0x7f) ? (char)c : '.');
        if (bad) break;
        while (s != 0 && ac_find(&a, s, c) == NONE) {
            s = a.fail[s];
            if (label(&a, s, lab, sizeof lab) < 0) { bad = 1; break; }
            EMIT(" f:%s", lab);
        }
        if (bad) break;
        s = ac_find(&a, s, c);
        if (label(&a, s, lab, sizeof lab) < 0) { bad = 1; break; }
        EMIT(" g:%s", lab);
        if (bad) break;
        int first = 1;
        for (uint32_t u = (a.own_head[s] != NONE) ? s : a.dict[s]; u != 0 && !bad; u = a.dict[u])
            for (uint32_t j = a.own_head[u]; j != NONE && !bad; j = a.own_next[j]) {
                EMIT(first ? " out:%u" : ",%u", j);
                first = 0;
            }
        if (bad) break;
        EMIT("\n");
    }
#undef EMIT
    ac_free(&a);
    return bad ? -1 : (int64_t)at;
}
