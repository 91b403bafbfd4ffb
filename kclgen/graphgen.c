/*
 * kclgen — seeded synthetic graph generators shared by the test/benchmark
 * harness, the oracle checks and the GPU path.  This module only builds
 * inputs: it holds none of the k-clique method's arithmetic.
 *
 * Every random draw comes from xoshiro256** (Blackman & Vigna, 2018) seeded
 * through SplitMix64 (Steele, Lea & Flood, OOPSLA 2014).  Sampling decisions
 * are taken in integer arithmetic; the only floating point (Chung-Lu weights)
 * uses +, -, *, / and the project's own exp/log series, compiled with
 * -ffp-contract=off, so the same seed gives the same graph on x86-64 and
 * AArch64 hosts.
 *
 * Output is an undirected simple graph as symmetric CSR: uint64 row offsets,
 * uint32 neighbour ids, every row strictly ascending, no self-loops.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

/* ------------------------------------------------------------------ PRNG */
static uint64_t sm64_next(uint64_t *s) {
    uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

typedef struct { uint64_t s[4]; } xo256;

static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static uint64_t xo_next(xo256 *r) {
    uint64_t *s = r->s;
    uint64_t result = rotl64(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl64(s[3], 45);
    return result;
}

static void xo_seed(xo256 *r, uint64_t seed) {
    uint64_t st = seed;
    for (int i = 0; i < 4; i++) r->s[i] = sm64_next(&st);
}

/* uniform integer in [0, bound) by the high half of a 64x64 product */
static inline uint64_t xo_below(xo256 *r, uint64_t bound) {
    return (uint64_t)(((u128)xo_next(r) * (u128)bound) >> 64);
}

/* Public helper: the i-th SplitMix64 output of a stream seeded with `seed`
 * (used by the harness to derive per-graph parameters deterministically). */
uint64_t kg_splitmix64(uint64_t seed, uint64_t i) {
    uint64_t st = seed + i * 0x9E3779B97F4A7C15ull;
    return sm64_next(&st);
}

/* ------------------------------------------- portable exp / log (x > 0) */
/* ln(x): x = f * 2^e with f in [sqrt(1/2), sqrt(2)); ln f = 2 atanh(t),
 * t = (f-1)/(f+1), |t| < 0.172, series to t^41. */
static double kg_log(double x) {
    int e = 0;
    while (x >= 1.4142135623730951) { x *= 0.5; e++; }
    while (x < 0.7071067811865476) { x *= 2.0; e--; }
    double t = (x - 1.0) / (x + 1.0), t2 = t * t, term = t, sum = 0.0;
    for (int k = 1; k <= 41; k += 2) { sum += term / (double)k; term *= t2; }
    return 2.0 * sum + (double)e * 0.6931471805599453;
}

/* exp(y): y = j ln2 + r, |r| <= ln2/2; Taylor series to r^24. */
static double kg_exp(double y) {
    double jd = y / 0.6931471805599453;
    long j = (long)(jd < 0 ? jd - 0.5 : jd + 0.5);
    double r = y - (double)j * 0.6931471805599453, term = 1.0, sum = 1.0;
    for (int k = 1; k <= 24; k++) { term *= r / (double)k; sum += term; }
    while (j > 0) { sum *= 2.0; j--; }
    while (j < 0) { sum *= 0.5; j++; }
    return sum;
}

/* ------------------------------------------------------------ edge set */
typedef struct {
    uint64_t *slots;   /* open addressing, empty = ~0 */
    uint64_t mask;
    uint64_t *keys;    /* unique keys in insertion order */
    uint64_t count, cap_keys;
} edge_set;

static inline uint64_t es_hash(uint64_t k) {
    k ^= k >> 33; k *= 0xFF51AFD7ED558CCDull; k ^= k >> 33; k *= 0xC4CEB9FE1A85EC53ull; k ^= k >> 33;
    return k;
}

static int es_init(edge_set *s, uint64_t expected) {
    uint64_t cap = 1024;
    while (cap < 2 * expected + 16) cap <<= 1;
    s->slots = (uint64_t *)malloc(cap * sizeof(uint64_t));
    s->keys = (uint64_t *)malloc((expected + 16) * sizeof(uint64_t));
    if (!s->slots || !s->keys) { free(s->slots); free(s->keys); return -1; }
    memset(s->slots, 0xFF, cap * sizeof(uint64_t));
    s->mask = cap - 1; s->count = 0; s->cap_keys = expected + 16;
    return 0;
}

static void es_free(edge_set *s) { free(s->slots); free(s->keys); s->slots = s->keys = 0; }

static int es_grow(edge_set *s) {
    uint64_t ncap = (s->mask + 1) * 2;
    uint64_t *ns = (uint64_t *)malloc(ncap * sizeof(uint64_t));
    uint64_t *nk = (uint64_t *)realloc(s->keys, (ncap / 2) * sizeof(uint64_t));
    if (!ns || !nk) { free(ns); if (nk) s->keys = nk; return -1; }
    s->keys = nk; s->cap_keys = ncap / 2;
    memset(ns, 0xFF, ncap * sizeof(uint64_t));
    for (uint64_t i = 0; i < s->count; i++) {
        uint64_t h = es_hash(s->keys[i]) & (ncap - 1);
        while (ns[h] != ~0ull) h = (h + 1) & (ncap - 1);
        ns[h] = s->keys[i];
    }
    free(s->slots); s->slots = ns; s->mask = ncap - 1;
    return 0;
}

/* insert undirected edge {u,v}, u != v; returns 1 if new, 0 if present, -1 on OOM */
static int es_insert(edge_set *s, uint32_t u, uint32_t v) {
    if (u > v) { uint32_t t = u; u = v; v = t; }
    uint64_t key = ((uint64_t)u << 32) | v;
    if (s->count + 1 > s->cap_keys || 2 * (s->count + 1) > s->mask + 1)
        if (es_grow(s)) return -1;
    uint64_t h = es_hash(key) & s->mask;
    while (s->slots[h] != ~0ull) {
        if (s->slots[h] == key) return 0;
        h = (h + 1) & s->mask;
    }
    s->slots[h] = key;
    s->keys[s->count++] = key;
    return 1;
}

/* --------------------------------------------------------------- output */
typedef struct {
    uint32_t n;
    uint64_t nnz;        /* = 2 * undirected edges */
    uint64_t *row_ptr;   /* n + 1 */
    uint32_t *col;       /* nnz */
} kg_csr;

void kg_free(kg_csr *g) {
    if (!g) return;
    free(g->row_ptr); free(g->col);
    g->row_ptr = 0; g->col = 0; g->n = 0; g->nnz = 0;
}

/* Build symmetric CSR with ascending rows from a unique undirected edge list.
 * Two stable counting sorts: by destination, then by source. */
static int build_csr(uint32_t n, const uint64_t *keys, uint64_t m, const uint32_t *perm, kg_csr *out) {
    uint64_t nnz = 2 * m;
    uint32_t *src = (uint32_t *)malloc((nnz ? nnz : 1) * sizeof(uint32_t));
    uint32_t *dst = (uint32_t *)malloc((nnz ? nnz : 1) * sizeof(uint32_t));
    uint32_t *tsrc = (uint32_t *)malloc((nnz ? nnz : 1) * sizeof(uint32_t));
    uint32_t *tdst = (uint32_t *)malloc((nnz ? nnz : 1) * sizeof(uint32_t));
    uint64_t *cnt = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
    if (!src || !dst || !tsrc || !tdst || !cnt) {
        free(src); free(dst); free(tsrc); free(tdst); free(cnt); return -1;
    }
    for (uint64_t i = 0; i < m; i++) {
        uint32_t u = (uint32_t)(keys[i] >> 32), v = (uint32_t)keys[i];
        if (perm) { u = perm[u]; v = perm[v]; }
        src[2 * i] = u; dst[2 * i] = v;
        src[2 * i + 1] = v; dst[2 * i + 1] = u;
    }
    /* pass 1: by dst */
    for (uint64_t i = 0; i < nnz; i++) cnt[dst[i] + 1]++;
    for (uint32_t i = 0; i < n; i++) cnt[i + 1] += cnt[i];
    for (uint64_t i = 0; i < nnz; i++) {
        uint64_t p = cnt[dst[i]]++;
        tsrc[p] = src[i]; tdst[p] = dst[i];
    }
    /* pass 2: by src, stable */
    memset(cnt, 0, ((size_t)n + 1) * sizeof(uint64_t));
    for (uint64_t i = 0; i < nnz; i++) cnt[tsrc[i] + 1]++;
    for (uint32_t i = 0; i < n; i++) cnt[i + 1] += cnt[i];
    uint64_t *row_ptr = (uint64_t *)malloc(((size_t)n + 1) * sizeof(uint64_t));
    if (!row_ptr) { free(src); free(dst); free(tsrc); free(tdst); free(cnt); return -1; }
    memcpy(row_ptr, cnt, ((size_t)n + 1) * sizeof(uint64_t));
    for (uint64_t i = 0; i < nnz; i++) {
        uint64_t p = cnt[tsrc[i]]++;
        dst[p] = tdst[i];
    }
    free(src); free(tsrc); free(tdst); free(cnt);
    out->n = n; out->nnz = nnz; out->row_ptr = row_ptr; out->col = dst;
    return 0;
}

/* ------------------------------------------------------------- params */
typedef struct {
    int kind;             /* 0 Chung-Lu, 1 R-MAT, 2 no base graph (planted only) */
    uint32_t n;           /* vertices (kinds 0 and 2) */
    uint32_t scale;       /* R-MAT: n = 2^scale */
    uint64_t m;           /* Chung-Lu: endpoint pairs drawn; R-MAT: unique edges wanted */
    double gamma;         /* Chung-Lu degree exponent (> 1) */
    double cap;           /* Chung-Lu expected-degree cap (<= 0: none) */
    double a, b, c;       /* R-MAT quadrant probabilities (d = 1 - a - b - c) */
    uint32_t n_groups;    /* planted groups */
    uint32_t group_lo, group_hi;  /* group size drawn uniformly in [lo, hi] */
    double group_p;       /* edge probability inside a group (1 = clique) */
    int relabel;          /* apply a seeded random permutation of vertex ids */
    uint64_t seed;
} kg_params;

static uint64_t prob_threshold(double p) {
    if (p <= 0.0) return 0;
    if (p >= 1.0) return ~0ull;
    return (uint64_t)(p * 18446744073709551616.0);  /* p * 2^64, exact scaling */
}

/* Walker/Vose alias table over integer weights. */
typedef struct { uint64_t *prob; uint32_t *alias; uint32_t n; uint64_t total; } alias_tab;

static int alias_build(alias_tab *t, const uint64_t *w, uint32_t n) {
    t->n = n; t->total = 0;
    for (uint32_t i = 0; i < n; i++) t->total += w[i];
    t->prob = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
    t->alias = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    uint64_t *p = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
    uint32_t *small = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    uint32_t *large = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    if (!t->prob || !t->alias || !p || !small || !large || t->total == 0) {
        free(t->prob); free(t->alias); free(p); free(small); free(large); return -1;
    }
    uint64_t T = t->total;  /* each bucket has capacity T; bucket mass = w[i] * n */
    uint32_t ns = 0, nl = 0;
    for (uint32_t i = 0; i < n; i++) {
        p[i] = w[i] * (uint64_t)n;
        if (p[i] < T) small[ns++] = i; else large[nl++] = i;
    }
    while (ns && nl) {
        uint32_t s = small[--ns], l = large[--nl];
        t->prob[s] = p[s]; t->alias[s] = l;
        p[l] -= (T - p[s]);
        if (p[l] < T) small[ns++] = l; else large[nl++] = l;
    }
    while (nl) { uint32_t l = large[--nl]; t->prob[l] = T; t->alias[l] = l; }
    while (ns) { uint32_t s = small[--ns]; t->prob[s] = T; t->alias[s] = s; }
    free(p); free(small); free(large);
    return 0;
}

static inline uint32_t alias_draw(const alias_tab *t, xo256 *r) {
    uint32_t i = (uint32_t)xo_below(r, t->n);
    uint64_t x = xo_below(r, t->total);
    return x < t->prob[i] ? i : t->alias[i];
}

/* Returns 0 on success, -1 on bad parameters, -2 on allocation failure,
 * -3 if the R-MAT edge target could not be reached. */
int kg_generate(const kg_params *P, kg_csr *out) {
    memset(out, 0, sizeof(*out));
    xo256 rng;
    xo_seed(&rng, P->seed);
    uint32_t n;
    if (P->kind == 1) {
        if (P->scale < 1 || P->scale > 31) return -1;
        n = 1u << P->scale;
    } else {
        n = P->n;
    }
    if (n == 0) {
        out->row_ptr = (uint64_t *)calloc(1, sizeof(uint64_t));
        out->col = (uint32_t *)malloc(sizeof(uint32_t));
        return (out->row_ptr && out->col) ? 0 : -2;
    }
    edge_set es;
    uint64_t expect = (P->kind == 2 ? 0 : P->m) + 1024;
    if (es_init(&es, expect)) return -2;
    int rc = 0;

    if (P->kind == 0) {
        if (P->gamma <= 1.0) { es_free(&es); return -1; }
        double expo = -1.0 / (P->gamma - 1.0), sum = 0.0;
        double *w = (double *)malloc((size_t)n * sizeof(double));
        uint64_t *wi = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
        if (!w || !wi) { free(w); free(wi); es_free(&es); return -2; }
        for (uint32_t i = 0; i < n; i++) { w[i] = kg_exp(expo * kg_log((double)i + 1.0)); sum += w[i]; }
        double scale = 2.0 * (double)P->m / sum, wsum = 0.0;
        for (uint32_t i = 0; i < n; i++) {
            w[i] *= scale;
            if (P->cap > 0.0 && w[i] > P->cap) w[i] = P->cap;
            wsum += w[i];
        }
        /* integer weights summing to at most 2^40 */
        for (uint32_t i = 0; i < n; i++) {
            double q = w[i] / wsum * 1099511627776.0;
            wi[i] = (uint64_t)q;
            if (wi[i] == 0) wi[i] = 1;
        }
        free(w);
        alias_tab at;
        if (alias_build(&at, wi, n)) { free(wi); es_free(&es); return -2; }
        free(wi);
        for (uint64_t e = 0; e < P->m; e++) {
            uint32_t u = alias_draw(&at, &rng), v = alias_draw(&at, &rng);
            if (u == v) continue;
            if (es_insert(&es, u, v) < 0) { rc = -2; break; }
        }
        free(at.prob); free(at.alias);
    } else if (P->kind == 1) {
        uint64_t ta = prob_threshold(P->a), tab = prob_threshold(P->a + P->b),
                 tabc = prob_threshold(P->a + P->b + P->c);
        uint64_t draws = 0, limit = 64 * P->m + 1024;
        while (es.count < P->m && rc == 0) {
            if (++draws > limit) { rc = -3; break; }
            uint32_t u = 0, v = 0;
            for (uint32_t lvl = 0; lvl < P->scale; lvl++) {
                uint64_t x = xo_next(&rng);
                uint32_t ub, vb;
                if (x < ta) { ub = 0; vb = 0; }
                else if (x < tab) { ub = 0; vb = 1; }
                else if (x < tabc) { ub = 1; vb = 0; }
                else { ub = 1; vb = 1; }
                u = (u << 1) | ub; v = (v << 1) | vb;
            }
            if (u == v) continue;
            if (es_insert(&es, u, v) < 0) rc = -2;
        }
    }

    /* planted groups: s distinct vertices, each pair kept with probability p */
    if (rc == 0 && P->n_groups) {
        uint32_t hi = P->group_hi < P->group_lo ? P->group_lo : P->group_hi;
        if (hi > n) hi = n;
        uint32_t lo = P->group_lo > hi ? hi : P->group_lo;
        uint32_t *mark = (uint32_t *)calloc((size_t)n, sizeof(uint32_t));
        uint32_t *memb = (uint32_t *)malloc(((size_t)hi + 1) * sizeof(uint32_t));
        uint64_t tp = prob_threshold(P->group_p);
        if (!mark || !memb) rc = -2;
        for (uint32_t g = 0; g < P->n_groups && rc == 0; g++) {
            uint32_t s = lo + (uint32_t)xo_below(&rng, (uint64_t)(hi - lo) + 1);
            uint32_t got = 0;
            while (got < s) {
                uint32_t v = (uint32_t)xo_below(&rng, n);
                if (mark[v] == g + 1) continue;
                mark[v] = g + 1; memb[got++] = v;
            }
            for (uint32_t i = 0; i < s && rc == 0; i++)
                for (uint32_t j = i + 1; j < s; j++) {
                    if (tp != ~0ull && xo_next(&rng) >= tp) continue;
                    if (es_insert(&es, memb[i], memb[j]) < 0) { rc = -2; break; }
                }
        }
        free(mark); free(memb);
    }

    uint32_t *perm = 0;
    if (rc == 0 && P->relabel) {
        perm = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
        if (!perm) rc = -2;
        else {
            for (uint32_t i = 0; i < n; i++) perm[i] = i;
            for (uint32_t i = n - 1; i > 0; i--) {
                uint32_t j = (uint32_t)xo_below(&rng, (uint64_t)i + 1);
                uint32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
            }
        }
    }
    if (rc == 0 && build_csr(n, es.keys, es.count, perm, out)) rc = -2;
    free(perm);
    es_free(&es);
    return rc;
}

/* Build symmetric sorted CSR from an arbitrary undirected edge list
 * (duplicates and self-loops dropped).  Used by tests for hand-written graphs. */
int kg_from_edges(uint32_t n, const uint32_t *eu, const uint32_t *ev, uint64_t ne, kg_csr *out) {
    memset(out, 0, sizeof(*out));
    edge_set es;
    if (es_init(&es, ne + 16)) return -2;
    for (uint64_t i = 0; i < ne; i++) {
        if (eu[i] >= n || ev[i] >= n) { es_free(&es); return -1; }
        if (eu[i] == ev[i]) continue;
        if (es_insert(&es, eu[i], ev[i]) < 0) { es_free(&es); return -2; }
    }
    int rc = build_csr(n, es.keys, es.count, 0, out) ? -2 : 0;
    es_free(&es);
    return rc;
}

/* Parameters of graph i of the batched workload: n log-uniform in [50, 20000],
 * average degree uniform in [4, 40], degree exponent 2.3, 0-5 planted cliques
 * of size 8-16, k uniform in 3..9.  All draws derive from SplitMix64(base+i). */
void kg_batch_params(uint64_t base_seed, uint64_t i, kg_params *P, uint32_t *k_out) {
    uint64_t s = kg_splitmix64(base_seed + i, 0);
    double u1 = (double)(kg_splitmix64(s, 1) >> 11) * (1.0 / 9007199254740992.0);
    double u2 = (double)(kg_splitmix64(s, 2) >> 11) * (1.0 / 9007199254740992.0);
    double lo = kg_log(50.0), hi = kg_log(20000.0);
    uint32_t n = (uint32_t)kg_exp(lo + u1 * (hi - lo));
    if (n < 50) n = 50;
    if (n > 20000) n = 20000;
    double d = 4.0 + 36.0 * u2;
    memset(P, 0, sizeof(*P));
    P->kind = 0;
    P->n = n;
    P->m = (uint64_t)((double)n * d * 0.5);
    P->gamma = 2.3;
    P->cap = 0.0;
    P->n_groups = (uint32_t)(kg_splitmix64(s, 3) % 6);
    P->group_lo = 8; P->group_hi = 16; P->group_p = 1.0;
    P->relabel = 1;
    P->seed = s;
    if (k_out) *k_out = 3 + (uint32_t)(kg_splitmix64(s, 4) % 7);
}
