/*
 * kcl_oracle.c — plain, slow, obviously correct CPU oracle for k-clique
 * listing ("Efficient k-clique Listing with Set Intersection Speedup").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file; only the test-suite, the smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no code, header, table or helper with the
 * CUDA library.
 *
 * What it computes
 *   count(G,k)    = number of k-vertex subsets of V that are cliques
 *                   (Definition 2).
 *   checksum(G,k) = sum over those subsets S of H(sorted S) mod 2^64, where
 *                   H(v_1<...<v_k) = mix(...mix(mix(GOLD ^ k) ^ v_1)... ^ v_k),
 *                   mix = the SplitMix64 output finaliser (Steele, Lea &
 *                   Flood, OOPSLA 2014), GOLD = 0x9E3779B97F4A7C15, ids are
 *                   the caller's original vertex ids.  (The paper defines no
 *                   checksum; this one is order independent by construction.)
 *
 * Modes, each written out separately:
 *   oracle_plain    the reference answer: the ordering-based DAG recursion of
 *                   Algorithm 2 (kClist) on the original graph, degree
 *                   orientation, sorted-list merge intersections, no
 *                   preprocessing and no pruning beyond |C| >= 1.
 *   oracle_precore  Algorithm 3 (Pre-Core), queue form.
 *   oracle_prelist  Algorithm 4 (Pre-List), BFS over components.
 *   oracle_sdegree  Algorithm 5 (SDegree) with Pre-Core and Pre-List.
 *   oracle_bitcol   Algorithm 6 (BitCol): degeneracy DAG, per-root colour
 *                   ordering (Section VII-A), BitEncode with an L-bit word
 *                   (Section VII-C), BitColList and BitJoin.
 *   count_only      (SDegree and BitCol) the same recursion and counters, but
 *                   the last level adds |C'| instead of enumerating each
 *                   clique; used to count algorithmic work on large inputs.
 *
 * Readings taken where the paper is silent or inconsistent (each is listed
 * in the design notes):
 *   - Pre-Core keeps the (k-1)-core: remove while degree < k-1 (Algorithm 3,
 *     Example 2), not "at least k".
 *   - Pre-List: m_c is the sum of the component's (current) degrees, i.e. the
 *     directed edge count 2|E(C)|; the component is a clique iff
 *     m_c = n_c (n_c - 1) (Algorithm 4, Example 3).
 *   - Degree ordering (Section VI-B): u -> v iff (d_u, u) < (d_v, v), degrees
 *     taken in the graph left by the preprocessing.
 *   - Degeneracy ordering (Algorithm 6): bulk peel rounds.  t = 0; repeat:
 *     S = remaining vertices of current degree <= t; if S is empty then t++,
 *     else remove S at once and record the round.  eta = (round, id).
 *   - Colouring (Section VII-A, Example 6): vertices of G_u in descending
 *     G_u-degree, ties by ascending id; colours start at 1; each vertex takes
 *     the smallest colour not used by its already coloured neighbours.
 *   - BitColList prunes v iff color(v) < l (Algorithm 6).
 *   - Bit i of the bitmap <-> the i-th out-neighbour of u in ascending id,
 *     least significant bit first (Table II).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

enum { OR_OK = 0, OR_EINVAL = 1, OR_ENOMEM = 2, OR_EOVERFLOW = 3, OR_ETRUNC = 4 };

/* ---------------------------------------------------------------- hash */
uint64_t oracle_mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* ids must already be sorted ascending */
uint64_t oracle_clique_hash(uint32_t k, const uint32_t *ids) {
    uint64_t h = oracle_mix64(0x9E3779B97F4A7C15ull ^ (uint64_t)k);
    for (uint32_t i = 0; i < k; i++) h = oracle_mix64(h ^ (uint64_t)ids[i]);
    return h;
}

/* ------------------------------------------------------------ counters */
typedef struct {
    uint64_t intersections;  /* merge joins (SDegree) or BitJoin calls (BitCol) */
    uint64_t merge_elems;    /* SDegree: sum of (|C| + d+_v) per merge join (Lemma 2) */
    uint64_t bitjoin_words;  /* BitCol: words touched by BitJoin */
    uint64_t build_reads;    /* BitCol: sum over v in N+_u of d+_v (G_u construction) */
    uint64_t roots;          /* roots with d+_u >= k-1 that were expanded */
    uint64_t max_outdeg;     /* maximum out-degree of the DAG (Delta) */
    uint64_t bitrow_words;   /* SDegree: per merge join, ceil(d+_root / 32) -- the words a
                                bitmap over N+_root's index space touches for it */
} oracle_counters;

/* -------------------------------------------------------- clique sink */
/* Collects one clique: sorts a copy of its ids, adds its hash to the
 * checksum and, if room is left, appends it to the caller's buffer. */
typedef struct {
    uint32_t k;
    u128 count;
    uint64_t checksum;
    uint32_t *out;          /* k ids per clique, or NULL */
    uint64_t cap, written;
    uint64_t *per_root;     /* indexed by the root vertex, or NULL */
    uint32_t root;
    int count_only;         /* count without enumerating (no checksum, no output) */
    uint32_t tmp[64];
} sink;

/* Count-only mode: add c cliques found at once (the leaf of a recursion). */
static void sink_add(sink *s, uint64_t c) {
    s->count += c;
    if (s->per_root) s->per_root[s->root] += c;
}

static void sink_emit(sink *s, const uint32_t *ids) {
    uint32_t k = s->k;
    for (uint32_t i = 0; i < k; i++) s->tmp[i] = ids[i];
    for (uint32_t i = 1; i < k; i++) {              /* insertion sort */
        uint32_t x = s->tmp[i], j = i;
        while (j > 0 && s->tmp[j - 1] > x) { s->tmp[j] = s->tmp[j - 1]; j--; }
        s->tmp[j] = x;
    }
    s->checksum += oracle_clique_hash(k, s->tmp);
    s->count += 1;
    if (s->per_root) s->per_root[s->root] += 1;
    if (s->out && s->written < s->cap) {
        memcpy(s->out + s->written * k, s->tmp, k * sizeof(uint32_t));
        s->written++;
    }
}

/* ------------------------------------------------------- small helpers */
static int is_adjacent(const uint64_t *rp, const uint32_t *col, uint32_t a, uint32_t b) {
    uint64_t lo = rp[a], hi = rp[a + 1];
    while (lo < hi) {                                /* binary search, rows sorted */
        uint64_t mid = lo + (hi - lo) / 2;
        if (col[mid] == b) return 1;
        if (col[mid] < b) lo = mid + 1; else hi = mid;
    }
    return 0;
}

/* merge join of two ascending lists; returns |out| */
static uint32_t merge_intersect(const uint32_t *a, uint32_t na, const uint32_t *b, uint32_t nb,
                                uint32_t *out) {
    uint32_t i = 0, j = 0, r = 0;
    while (i < na && j < nb) {
        if (a[i] == b[j]) { out[r++] = a[i]; i++; j++; }
        else if (a[i] < b[j]) i++;
        else j++;
    }
    return r;
}

/* Binomial coefficient C(n, k) in 128 bits; returns 0 on overflow of 128 bits
 * (flagged through *ovf). */
static u128 binom128(uint64_t n, uint64_t k, int *ovf) {
    if (k > n) return 0;
    if (k > n - k) k = n - k;
    u128 r = 1;
    for (uint64_t i = 1; i <= k; i++) {
        u128 f = (u128)(n - k + i);
        if (r > (~(u128)0) / f) { *ovf = 1; return 0; }
        r = r * f / i;  /* exact: r * f / i = C(n-k+i, i) */
    }
    return r;
}

/* Validate the input: symmetric CSR, rows strictly ascending, ids < n,
 * no self-loops. */
int oracle_validate(uint32_t n, const uint64_t *rp, const uint32_t *col) {
    if (rp[0] != 0) return OR_EINVAL;
    for (uint32_t u = 0; u < n; u++) {
        if (rp[u + 1] < rp[u]) return OR_EINVAL;
        for (uint64_t e = rp[u]; e < rp[u + 1]; e++) {
            uint32_t v = col[e];
            if (v >= n || v == u) return OR_EINVAL;
            if (e > rp[u] && col[e - 1] >= v) return OR_EINVAL;
        }
    }
    for (uint32_t u = 0; u < n; u++)
        for (uint64_t e = rp[u]; e < rp[u + 1]; e++)
            if (!is_adjacent(rp, col, col[e], u)) return OR_EINVAL;
    return OR_OK;
}

/* -------------------------------------------------------------- DAG */
/* Out-lists of the DAG over alive vertices for an ordering key (key, id):
 * u -> v iff (key[u], u) < (key[v], v).  Lists keep ascending id order. */
typedef struct {
    uint64_t *optr;
    uint32_t *oadj;
} dag;

static int eta_less(const uint64_t *key, uint32_t a, uint32_t b) {
    if (key[a] != key[b]) return key[a] < key[b];
    return a < b;
}

static int build_dag(uint32_t n, const uint64_t *rp, const uint32_t *col, const uint8_t *alive,
                     const uint64_t *key, dag *D) {
    D->optr = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
    if (!D->optr) return OR_ENOMEM;
    for (uint32_t u = 0; u < n; u++) {
        uint64_t c = 0;
        if (alive[u])
            for (uint64_t e = rp[u]; e < rp[u + 1]; e++) {
                uint32_t v = col[e];
                if (alive[v] && eta_less(key, u, v)) c++;
            }
        D->optr[u + 1] = D->optr[u] + c;
    }
    D->oadj = (uint32_t *)malloc((D->optr[n] ? D->optr[n] : 1) * sizeof(uint32_t));
    if (!D->oadj) { free(D->optr); return OR_ENOMEM; }
    for (uint32_t u = 0; u < n; u++) {
        uint64_t p = D->optr[u];
        if (alive[u])
            for (uint64_t e = rp[u]; e < rp[u + 1]; e++) {
                uint32_t v = col[e];
                if (alive[v] && eta_less(key, u, v)) D->oadj[p++] = v;
            }
    }
    return OR_OK;
}

static void free_dag(dag *D) { free(D->optr); free(D->oadj); }

static uint64_t dag_max_outdeg(uint32_t n, const dag *D) {
    uint64_t mx = 0;
    for (uint32_t u = 0; u < n; u++)
        if (D->optr[u + 1] - D->optr[u] > mx) mx = D->optr[u + 1] - D->optr[u];
    return mx;
}

/* Degrees counted over alive neighbours only. */
static void alive_degrees(uint32_t n, const uint64_t *rp, const uint32_t *col, const uint8_t *alive,
                          uint64_t *deg) {
    for (uint32_t u = 0; u < n; u++) {
        deg[u] = 0;
        if (!alive[u]) continue;
        for (uint64_t e = rp[u]; e < rp[u + 1]; e++)
            if (alive[col[e]]) deg[u]++;
    }
}

/* ============================================================ plain */
/* Algorithm 2 (kClist) with a degree ordering and sorted-list intersections:
 * every k-clique is reached once, along its unique eta-increasing order. */
typedef struct {
    const dag *D;
    sink *S;
    uint32_t k;
    uint32_t R[64];
    uint32_t **buf;  /* one candidate buffer per depth */
} plain_ctx;

static void plain_rec(plain_ctx *c, uint32_t depth, const uint32_t *C, uint32_t nC) {
    /* R[0..depth-1] is a clique; every vertex of C extends it */
    for (uint32_t i = 0; i < nC; i++) {
        uint32_t v = C[i];
        c->R[depth] = v;
        if (depth + 1 == c->k) { sink_emit(c->S, c->R); continue; }
        const uint32_t *Nv = c->D->oadj + c->D->optr[v];
        uint32_t dv = (uint32_t)(c->D->optr[v + 1] - c->D->optr[v]);
        uint32_t nn = merge_intersect(Nv, dv, C, nC, c->buf[depth + 1]);
        if (nn) plain_rec(c, depth + 1, c->buf[depth + 1], nn);
    }
}

int oracle_plain(uint32_t n, const uint64_t *rp, const uint32_t *col, uint32_t k,
                 uint64_t *count, uint64_t *checksum, uint32_t *out, uint64_t cap,
                 uint64_t *written) {
    if (k < 1 || k > 64) return OR_EINVAL;
    uint8_t *alive = (uint8_t *)malloc((size_t)n + 1);
    uint64_t *deg = (uint64_t *)malloc(((size_t)n + 1) * sizeof(uint64_t));
    if (!alive || !deg) { free(alive); free(deg); return OR_ENOMEM; }
    memset(alive, 1, (size_t)n + 1);
    for (uint32_t u = 0; u < n; u++) deg[u] = rp[u + 1] - rp[u];
    dag D;
    int rc = build_dag(n, rp, col, alive, deg, &D);
    if (rc) { free(alive); free(deg); return rc; }
    sink S;
    memset(&S, 0, sizeof(S));
    S.k = k; S.out = out; S.cap = cap;
    plain_ctx c;
    memset(&c, 0, sizeof(c));
    c.D = &D; c.S = &S; c.k = k;
    uint64_t mx = dag_max_outdeg(n, &D) + 1;
    c.buf = (uint32_t **)calloc(k + 1, sizeof(uint32_t *));
    for (uint32_t i = 0; c.buf && i <= k; i++) c.buf[i] = (uint32_t *)malloc(mx * sizeof(uint32_t));
    uint32_t *all = (uint32_t *)malloc(((size_t)n + 1) * sizeof(uint32_t));
    if (c.buf && all) {
        if (k == 1) {
            for (uint32_t u = 0; u < n; u++) all[u] = u;
            plain_rec(&c, 0, all, n);
        } else {
            for (uint32_t u = 0; u < n; u++) {
                c.R[0] = u;
                uint32_t du = (uint32_t)(D.optr[u + 1] - D.optr[u]);
                if (du) plain_rec(&c, 1, D.oadj + D.optr[u], du);
            }
        }
    } else rc = OR_ENOMEM;
    for (uint32_t i = 0; c.buf && i <= k; i++) free(c.buf[i]);
    free(c.buf); free(all);
    free_dag(&D); free(alive); free(deg);
    if (rc) return rc;
    if (S.count >> 64) return OR_EOVERFLOW;
    *count = (uint64_t)S.count;
    *checksum = S.checksum;
    if (written) *written = S.written;
    if (out && S.written < S.count) return OR_ETRUNC;
    return OR_OK;
}

/* ========================================================== Pre-Core */
/* Algorithm 3: a queue of vertices whose degree fell below k-1; each popped
 * vertex lowers its neighbours' degrees; F collects the removed vertices.
 * alive[v] = 1 for the survivors (the (k-1)-core). */
int oracle_precore(uint32_t n, const uint64_t *rp, const uint32_t *col, uint32_t k, uint8_t *alive) {
    if (k < 1) return OR_EINVAL;
    uint64_t *d = (uint64_t *)malloc(((size_t)n + 1) * sizeof(uint64_t));
    uint32_t *Q = (uint32_t *)malloc(((size_t)n + 1) * sizeof(uint32_t));
    uint8_t *F = (uint8_t *)calloc((size_t)n + 1, 1);
    if (!d || !Q || !F) { free(d); free(Q); free(F); return OR_ENOMEM; }
    uint64_t head = 0, tail = 0, thr = (uint64_t)k - 1;
    for (uint32_t u = 0; u < n; u++) {
        d[u] = rp[u + 1] - rp[u];
        if (d[u] < thr) { Q[tail++] = u; F[u] = 1; }
    }
    while (head < tail) {
        uint32_t u = Q[head++];
        for (uint64_t e = rp[u]; e < rp[u + 1]; e++) {
            uint32_t v = col[e];
            d[v] -= 1;
            if (d[v] < thr && !F[v]) { F[v] = 1; Q[tail++] = v; }
        }
    }
    for (uint32_t u = 0; u < n; u++) alive[u] = F[u] ? 0 : 1;
    free(d); free(Q); free(F);
    return OR_OK;
}

/* ========================================================== Pre-List */
/* Algorithm 4: BFS over the connected components of the alive subgraph.  A
 * component with n_c vertices whose degree sum m_c equals n_c (n_c - 1) is a
 * clique: its C(n_c, k) k-cliques are reported (every k-subset, ids sorted)
 * and the component is removed.  `alive` is updated in place. */
int oracle_prelist(uint32_t n, const uint64_t *rp, const uint32_t *col, uint32_t k, uint8_t *alive,
                   uint64_t *count, uint64_t *checksum, uint32_t *ncomp_removed,
                   uint32_t *out, uint64_t cap, uint64_t *written) {
    if (k < 1 || k > 64) return OR_EINVAL;
    uint32_t *comp = (uint32_t *)malloc(((size_t)n + 1) * sizeof(uint32_t));
    uint32_t *Q = (uint32_t *)malloc(((size_t)n + 1) * sizeof(uint32_t));
    uint8_t *seen = (uint8_t *)calloc((size_t)n + 1, 1);
    if (!comp || !Q || !seen) { free(comp); free(Q); free(seen); return OR_ENOMEM; }
    u128 total = 0;
    uint64_t cks = 0, wr = 0;
    uint32_t removed = 0;
    int ovf = 0;
    sink S;
    memset(&S, 0, sizeof(S));
    S.k = k; S.out = out; S.cap = cap;
    for (uint32_t s = 0; s < n; s++) {
        if (!alive[s] || seen[s]) continue;
        uint32_t head = 0, tail = 0;
        uint64_t m_c = 0;
        Q[tail++] = s; seen[s] = 1;
        while (head < tail) {
            uint32_t u = Q[head++];
            for (uint64_t e = rp[u]; e < rp[u + 1]; e++) {
                uint32_t v = col[e];
                if (!alive[v]) continue;
                m_c++;
                if (!seen[v]) { seen[v] = 1; Q[tail++] = v; }
            }
        }
        uint64_t n_c = tail;
        if (m_c == n_c * (n_c - 1)) {
            /* clique component: report its k-subsets */
            u128 b = binom128(n_c, k, &ovf);
            total += b;
            if (total < b) ovf = 1;
            for (uint32_t i = 0; i < tail; i++) comp[i] = Q[i];
            /* sort member ids */
            for (uint32_t i = 1; i < tail; i++) {
                uint32_t x = comp[i], j = i;
                while (j > 0 && comp[j - 1] > x) { comp[j] = comp[j - 1]; j--; }
                comp[j] = x;
            }
            if (k <= n_c && !ovf) {
                /* enumerate index combinations in lexicographic order */
                uint32_t idx[64], ids[64];
                for (uint32_t i = 0; i < k; i++) idx[i] = i;
                for (;;) {
                    for (uint32_t i = 0; i < k; i++) ids[i] = comp[idx[i]];
                    sink_emit(&S, ids);
                    int32_t p = (int32_t)k - 1;
                    while (p >= 0 && idx[p] == (uint32_t)(n_c - k + (uint32_t)p)) p--;
                    if (p < 0) break;
                    idx[p]++;
                    for (uint32_t q = (uint32_t)p + 1; q < k; q++) idx[q] = idx[q - 1] + 1;
                }
            }
            for (uint32_t i = 0; i < tail; i++) alive[Q[i]] = 0;
            removed++;
        }
    }
    cks = S.checksum; wr = S.written;
    free(comp); free(Q); free(seen);
    if (ovf || (total >> 64)) return OR_EOVERFLOW;
    *count = (uint64_t)total;
    *checksum = cks;
    if (ncomp_removed) *ncomp_removed = removed;
    if (written) *written = wr;
    if (out && S.count > S.written) return OR_ETRUNC;
    return OR_OK;
}

/* ======================================================== orderings */
/* Degeneracy ordering by bulk peel rounds over the alive vertices.
 * round[v] receives the round in which v was removed (dead vertices: ~0). */
int oracle_degeneracy_rounds(uint32_t n, const uint64_t *rp, const uint32_t *col,
                             const uint8_t *alive, uint32_t *round, uint32_t *degeneracy) {
    uint64_t *d = (uint64_t *)malloc(((size_t)n + 1) * sizeof(uint64_t));
    uint8_t *gone = (uint8_t *)malloc((size_t)n + 1);
    uint32_t *S = (uint32_t *)malloc(((size_t)n + 1) * sizeof(uint32_t));
    if (!d || !gone || !S) { free(d); free(gone); free(S); return OR_ENOMEM; }
    alive_degrees(n, rp, col, alive, d);
    uint64_t left = 0;
    for (uint32_t u = 0; u < n; u++) {
        gone[u] = alive[u] ? 0 : 1;
        round[u] = 0xFFFFFFFFu;
        if (alive[u]) left++;
    }
    uint64_t t = 0;
    uint32_t r = 0;
    while (left) {
        uint32_t ns = 0;
        for (uint32_t u = 0; u < n; u++)
            if (!gone[u] && d[u] <= t) S[ns++] = u;
        if (ns == 0) { t++; continue; }
        for (uint32_t i = 0; i < ns; i++) { round[S[i]] = r; gone[S[i]] = 1; }
        for (uint32_t i = 0; i < ns; i++) {
            uint32_t u = S[i];
            for (uint64_t e = rp[u]; e < rp[u + 1]; e++)
                if (!gone[col[e]]) d[col[e]] -= 1;
        }
        left -= ns;
        r++;
    }
    if (degeneracy) *degeneracy = (uint32_t)t;
    free(d); free(gone); free(S);
    return OR_OK;
}

/* Out-degrees of the DAG that a mode builds (0 = degree ordering,
 * 1 = degeneracy ordering) over the given alive set. */
int oracle_outdegrees(uint32_t n, const uint64_t *rp, const uint32_t *col, const uint8_t *alive,
                      int mode, uint32_t *outdeg) {
    uint64_t *key = (uint64_t *)malloc(((size_t)n + 1) * sizeof(uint64_t));
    if (!key) return OR_ENOMEM;
    int rc = OR_OK;
    if (mode == 0) alive_degrees(n, rp, col, alive, key);
    else {
        uint32_t *rd = (uint32_t *)malloc(((size_t)n + 1) * sizeof(uint32_t));
        if (!rd) { free(key); return OR_ENOMEM; }
        rc = oracle_degeneracy_rounds(n, rp, col, alive, rd, 0);
        for (uint32_t u = 0; u < n; u++) key[u] = rd[u];
        free(rd);
    }
    if (rc) { free(key); return rc; }
    dag D;
    rc = build_dag(n, rp, col, alive, key, &D);
    if (!rc) {
        for (uint32_t u = 0; u < n; u++) outdeg[u] = (uint32_t)(D.optr[u + 1] - D.optr[u]);
        free_dag(&D);
    }
    free(key);
    return rc;
}

/* ====================================================== preprocessing */
typedef struct {
    uint8_t *alive;
    u128 count;
    uint64_t checksum;
} prep;

static int run_preprocessing(uint32_t n, const uint64_t *rp, const uint32_t *col, uint32_t k,
                             int enable, prep *P, uint32_t *out, uint64_t cap, uint64_t *written) {
    P->alive = (uint8_t *)malloc((size_t)n + 1);
    P->count = 0; P->checksum = 0;
    if (!P->alive) return OR_ENOMEM;
    if (!enable) { memset(P->alive, 1, (size_t)n + 1); if (written) *written = 0; return OR_OK; }
    int rc = oracle_precore(n, rp, col, k, P->alive);
    if (rc) return rc;
    uint64_t c = 0, s = 0;
    rc = oracle_prelist(n, rp, col, k, P->alive, &c, &s, 0, out, cap, written);
    if (rc && rc != OR_ETRUNC) return rc;
    P->count = c; P->checksum = s;
    return OR_OK;
}

/* =========================================================== SDegree */
/* Algorithm 5.  SDegreeList(l, R, C): for each u in C, skip it when
 * d+_u <= l-2; C' = N+_u intersected with C (merge join); at l = 2 report
 * R + {u, v} for every v in C'; otherwise recurse when |C'| > l-2. */
typedef struct {
    const dag *D;
    sink *S;
    oracle_counters *cnt;
    uint32_t k;
    uint32_t R[64];
    uint32_t **buf;
    uint32_t nw_root;      /* ceil(d+_root / 32) of the current root */
    uint32_t *trace;       /* optional call trace: [l, |R|, R..., |C|, C...] per call */
    uint64_t trace_cap, trace_len;
} sdeg_ctx;

static void trace_call(sdeg_ctx *c, uint32_t l, uint32_t nR, const uint32_t *C, uint32_t nC) {
    if (!c->trace) return;
    uint64_t need = 3 + (uint64_t)nR + nC;
    if (c->trace_len + need > c->trace_cap) return;
    uint32_t *t = c->trace + c->trace_len;
    *t++ = l; *t++ = nR;
    for (uint32_t i = 0; i < nR; i++) *t++ = c->R[i];
    *t++ = nC;
    for (uint32_t i = 0; i < nC; i++) *t++ = C[i];
    c->trace_len += need;
}

static void sdegree_list(sdeg_ctx *c, uint32_t l, uint32_t nR, const uint32_t *C, uint32_t nC) {
    trace_call(c, l, nR, C, nC);
    for (uint32_t i = 0; i < nC; i++) {
        uint32_t u = C[i];
        uint32_t du = (uint32_t)(c->D->optr[u + 1] - c->D->optr[u]);
        if (du <= l - 2) continue;                       /* degree prune */
        uint32_t *Cp = c->buf[nR];
        uint32_t np = merge_intersect(c->D->oadj + c->D->optr[u], du, C, nC, Cp);
        c->cnt->intersections++;
        c->cnt->merge_elems += (uint64_t)nC + du;
        c->cnt->bitrow_words += c->nw_root;
        if (l == 2) {
            c->R[nR] = u;
            if (c->S->count_only) sink_add(c->S, np);
            else
                for (uint32_t j = 0; j < np; j++) { c->R[nR + 1] = Cp[j]; sink_emit(c->S, c->R); }
        } else if (np > l - 2) {
            c->R[nR] = u;
            sdegree_list(c, l - 1, nR + 1, Cp, np);
        }
    }
}

int oracle_sdegree(uint32_t n, const uint64_t *rp, const uint32_t *col, uint32_t k, int preprocess,
                   const uint32_t *roots, uint32_t nroots,
                   uint64_t *count, uint64_t *checksum, uint64_t *per_root,
                   oracle_counters *counters, uint32_t *out, uint64_t cap, uint64_t *written,
                   uint32_t *trace, uint64_t trace_cap, uint64_t *trace_len, int count_only) {
    if (k < 3 || k > 64) return OR_EINVAL;
    oracle_counters local;
    if (!counters) counters = &local;
    memset(counters, 0, sizeof(*counters));
    prep P;
    uint64_t wpre = 0;
    int rc = run_preprocessing(n, rp, col, k, preprocess, &P, out, cap, &wpre);
    if (rc) { free(P.alive); return rc; }
    uint64_t *deg = (uint64_t *)malloc(((size_t)n + 1) * sizeof(uint64_t));
    if (!deg) { free(P.alive); return OR_ENOMEM; }
    alive_degrees(n, rp, col, P.alive, deg);     /* degree in the reduced graph */
    dag D;
    rc = build_dag(n, rp, col, P.alive, deg, &D);
    free(deg);
    if (rc) { free(P.alive); return rc; }
    counters->max_outdeg = dag_max_outdeg(n, &D);
    sink S;
    memset(&S, 0, sizeof(S));
    S.k = k; S.per_root = per_root; S.count_only = count_only;
    S.out = out ? out + wpre * k : 0;
    S.cap = out ? cap - wpre : 0;
    sdeg_ctx c;
    memset(&c, 0, sizeof(c));
    c.D = &D; c.S = &S; c.cnt = counters; c.k = k;
    c.trace = trace; c.trace_cap = trace_cap;
    c.buf = (uint32_t **)calloc(k + 1, sizeof(uint32_t *));
    uint64_t mx = counters->max_outdeg + 1;
    for (uint32_t i = 0; c.buf && i <= k; i++) c.buf[i] = (uint32_t *)malloc(mx * sizeof(uint32_t));
    if (!c.buf) rc = OR_ENOMEM;
    for (uint32_t i = 0; !rc && i <= k; i++) if (!c.buf[i]) rc = OR_ENOMEM;
    uint32_t total_roots = roots ? nroots : n;
    for (uint32_t r = 0; !rc && r < total_roots; r++) {
        uint32_t u = roots ? roots[r] : r;
        if (u >= n) { rc = OR_EINVAL; break; }
        uint32_t du = (uint32_t)(D.optr[u + 1] - D.optr[u]);
        if (!P.alive[u] || du < k - 1) continue;
        counters->roots++;
        c.R[0] = u; S.root = u;
        c.nw_root = (du + 31) / 32;
        sdegree_list(&c, k - 1, 1, D.oadj + D.optr[u], du);
    }
    for (uint32_t i = 0; c.buf && i <= k; i++) free(c.buf[i]);
    free(c.buf);
    free_dag(&D);
    free(P.alive);
    if (rc) return rc;
    if (trace_len) *trace_len = c.trace_len;
    u128 tot = S.count + (roots ? 0 : P.count);
    if (tot >> 64) return OR_EOVERFLOW;
    *count = (uint64_t)tot;
    *checksum = S.checksum + (roots ? 0 : P.checksum);
    if (written) *written = wpre + S.written;
    if (out && (S.written < S.count || wpre < P.count)) return OR_ETRUNC;
    return OR_OK;
}

/* ============================================================ BitCol */
/* Colour ordering of an undirected graph H given by an adjacency predicate
 * over indices 0..h-1 (Section VII-A): order by degree descending then index
 * ascending; greedy smallest unused colour, colours from 1.  `order` gets the
 * colouring order, `colour` the colour of each index. */
static void greedy_colouring(uint32_t h, const uint8_t *adj /* h*h */, uint32_t *order,
                             uint32_t *colour) {
    uint32_t *deg = (uint32_t *)malloc(((size_t)h + 1) * sizeof(uint32_t));
    uint8_t *used = (uint8_t *)malloc((size_t)h + 2);
    for (uint32_t i = 0; i < h; i++) {
        deg[i] = 0;
        for (uint32_t j = 0; j < h; j++) deg[i] += adj[(size_t)i * h + j];
        order[i] = i;
        colour[i] = 0;
    }
    for (uint32_t i = 1; i < h; i++) {                   /* stable insertion sort */
        uint32_t x = order[i], j = i;
        while (j > 0 && deg[order[j - 1]] < deg[x]) { order[j] = order[j - 1]; j--; }
        order[j] = x;
    }
    for (uint32_t t = 0; t < h; t++) {
        uint32_t v = order[t];
        memset(used, 0, (size_t)h + 2);
        for (uint32_t j = 0; j < h; j++)
            if (adj[(size_t)v * h + j] && colour[j]) used[colour[j]] = 1;
        uint32_t c = 1;
        while (used[c]) c++;
        colour[v] = c;
    }
    free(deg); free(used);
}

/* Public entry for pinning the colouring on explicit small graphs (CSR). */
int oracle_colour_graph(uint32_t h, const uint64_t *rp, const uint32_t *col, uint32_t *order,
                        uint32_t *colour) {
    uint8_t *adj = (uint8_t *)calloc((size_t)h * h + 1, 1);
    if (!adj) return OR_ENOMEM;
    for (uint32_t u = 0; u < h; u++)
        for (uint64_t e = rp[u]; e < rp[u + 1]; e++) adj[(size_t)u * h + col[e]] = 1;
    greedy_colouring(h, adj, order, colour);
    free(adj);
    return OR_OK;
}

/* BitEncode (Section VII-C): B(v) has bit i set iff the i-th vertex is an
 * out-neighbour of v in the colour-ordered DAG (colour(v) > colour(i)).
 * Words hold L bits each, least significant bit first; nw = ceil(h / L). */
static void bit_encode(uint32_t h, const uint8_t *adj, const uint32_t *colour, uint32_t L,
                       uint32_t nw, uint32_t *B /* h * nw */) {
    memset(B, 0, (size_t)h * nw * sizeof(uint32_t));
    for (uint32_t v = 0; v < h; v++)
        for (uint32_t i = 0; i < h; i++)
            if (adj[(size_t)v * h + i] && colour[v] > colour[i])
                B[(size_t)v * nw + i / L] |= 1u << (i % L);
}

int oracle_bitencode_graph(uint32_t h, const uint64_t *rp, const uint32_t *col, uint32_t L,
                           uint32_t *colour, uint32_t *B) {
    if (L < 1 || L > 32) return OR_EINVAL;
    uint8_t *adj = (uint8_t *)calloc((size_t)h * h + 1, 1);
    uint32_t *order = (uint32_t *)malloc(((size_t)h + 1) * sizeof(uint32_t));
    if (!adj || !order) { free(adj); free(order); return OR_ENOMEM; }
    for (uint32_t u = 0; u < h; u++)
        for (uint64_t e = rp[u]; e < rp[u + 1]; e++) adj[(size_t)u * h + col[e]] = 1;
    greedy_colouring(h, adj, order, colour);
    bit_encode(h, adj, colour, L, (h + L - 1) / L, B);
    free(adj); free(order);
    return OR_OK;
}

typedef struct {
    sink *S;
    oracle_counters *cnt;
    uint32_t k, L, nw, h;
    const uint32_t *B;       /* h * nw */
    const uint32_t *colour;
    const uint32_t *ids;     /* index -> original id */
    uint32_t R[64];
    uint32_t **buf;          /* one candidate bitmap per level */
} bitcol_ctx;

static uint32_t popcount32(uint32_t x) {
    uint32_t c = 0;
    while (x) { c += x & 1u; x >>= 1; }
    return c;
}

/* BitColList(l, R, C_B): for each v decoded from C_B (ascending index), skip
 * it when color(v) < l; C'_B = BitJoin(B(v), C_B); at l = 2 report R + {v, w}
 * for every w decoded from C'_B; otherwise recurse when |C'_B| >= l-1. */
static void bitcol_list(bitcol_ctx *c, uint32_t l, uint32_t nR, const uint32_t *CB) {
    for (uint32_t v = 0; v < c->h; v++) {
        if (!((CB[v / c->L] >> (v % c->L)) & 1u)) continue;       /* BitDecode */
        if (c->colour[v] < l) continue;                             /* colour prune */
        uint32_t *Cp = c->buf[nR];
        uint32_t size = 0;
        for (uint32_t i = 0; i < c->nw; i++) {                       /* BitJoin */
            Cp[i] = c->B[(size_t)v * c->nw + i] & CB[i];
            size += popcount32(Cp[i]);
        }
        c->cnt->intersections++;
        c->cnt->bitjoin_words += c->nw;
        if (l == 2) {
            c->R[nR] = c->ids[v];
            if (c->S->count_only) sink_add(c->S, size);
            else
                for (uint32_t w = 0; w < c->h; w++)
                    if ((Cp[w / c->L] >> (w % c->L)) & 1u) { c->R[nR + 1] = c->ids[w]; sink_emit(c->S, c->R); }
        } else if (size >= l - 1) {
            c->R[nR] = c->ids[v];
            bitcol_list(c, l - 1, nR + 1, Cp);
        }
    }
}

int oracle_bitcol(uint32_t n, const uint64_t *rp, const uint32_t *col, uint32_t k, int preprocess,
                  uint32_t L, const uint32_t *roots, uint32_t nroots,
                  uint64_t *count, uint64_t *checksum, uint64_t *per_root,
                  oracle_counters *counters, uint32_t *out, uint64_t cap, uint64_t *written,
                  int count_only) {
    if (k < 3 || k > 64 || L < 1 || L > 32) return OR_EINVAL;
    oracle_counters local;
    if (!counters) counters = &local;
    memset(counters, 0, sizeof(*counters));
    prep P;
    uint64_t wpre = 0;
    int rc = run_preprocessing(n, rp, col, k, preprocess, &P, out, cap, &wpre);
    if (rc) { free(P.alive); return rc; }
    uint32_t *rd = (uint32_t *)malloc(((size_t)n + 1) * sizeof(uint32_t));
    uint64_t *key = (uint64_t *)malloc(((size_t)n + 1) * sizeof(uint64_t));
    if (!rd || !key) { free(rd); free(key); free(P.alive); return OR_ENOMEM; }
    rc = oracle_degeneracy_rounds(n, rp, col, P.alive, rd, 0);
    for (uint32_t u = 0; u < n; u++) key[u] = rd[u];
    free(rd);
    dag D;
    if (!rc) rc = build_dag(n, rp, col, P.alive, key, &D);
    free(key);
    if (rc) { free(P.alive); return rc; }
    counters->max_outdeg = dag_max_outdeg(n, &D);
    uint32_t hmax = (uint32_t)counters->max_outdeg;
    uint32_t nwmax = (hmax + L - 1) / L + 1;
    sink S;
    memset(&S, 0, sizeof(S));
    S.k = k; S.per_root = per_root; S.count_only = count_only;
    S.out = out ? out + wpre * k : 0;
    S.cap = out ? cap - wpre : 0;
    bitcol_ctx c;
    memset(&c, 0, sizeof(c));
    c.S = &S; c.cnt = counters; c.k = k; c.L = L;
    uint8_t *adj = (uint8_t *)malloc((size_t)hmax * hmax + 1);
    uint32_t *B = (uint32_t *)malloc(((size_t)hmax * nwmax + 1) * sizeof(uint32_t));
    uint32_t *colour = (uint32_t *)malloc(((size_t)hmax + 1) * sizeof(uint32_t));
    uint32_t *order = (uint32_t *)malloc(((size_t)hmax + 1) * sizeof(uint32_t));
    uint32_t *C0 = (uint32_t *)malloc((size_t)nwmax * sizeof(uint32_t));
    uint32_t *pos = (uint32_t *)calloc((size_t)n + 1, sizeof(uint32_t));
    c.buf = (uint32_t **)calloc(k + 1, sizeof(uint32_t *));
    for (uint32_t i = 0; c.buf && i <= k; i++) c.buf[i] = (uint32_t *)malloc((size_t)nwmax * sizeof(uint32_t));
    if (!adj || !B || !colour || !order || !C0 || !pos || !c.buf) rc = OR_ENOMEM;
    for (uint32_t i = 0; !rc && i <= k; i++) if (!c.buf[i]) rc = OR_ENOMEM;
    uint32_t total_roots = roots ? nroots : n;
    for (uint32_t r = 0; !rc && r < total_roots; r++) {
        uint32_t u = roots ? roots[r] : r;
        if (u >= n) { rc = OR_EINVAL; break; }
        uint32_t h = (uint32_t)(D.optr[u + 1] - D.optr[u]);
        if (!P.alive[u] || h < k - 1) continue;
        counters->roots++;
        const uint32_t *Nu = D.oadj + D.optr[u];
        /* G_u: undirected subgraph induced by N+_u (Section VII-B).  Every
         * edge {a, b} of G_u is oriented by the DAG, so it lies in exactly one
         * of the out-lists N+_a, N+_b: scanning the out-lists of the members
         * of N+_u (pos marks membership) finds each edge once. */
        memset(adj, 0, (size_t)h * h);
        for (uint32_t i = 0; i < h; i++) pos[Nu[i]] = i + 1;
        for (uint32_t i = 0; i < h; i++) {
            uint32_t a = Nu[i];
            counters->build_reads += D.optr[a + 1] - D.optr[a];
            for (uint64_t e = D.optr[a]; e < D.optr[a + 1]; e++) {
                uint32_t j = pos[D.oadj[e]];
                if (j) { adj[(size_t)i * h + (j - 1)] = 1; adj[(size_t)(j - 1) * h + i] = 1; }
            }
        }
        for (uint32_t i = 0; i < h; i++) pos[Nu[i]] = 0;
        greedy_colouring(h, adj, order, colour);       /* ColorOrdering(G_u) */
        uint32_t nw = (h + L - 1) / L;
        bit_encode(h, adj, colour, L, nw, B);           /* BitEncode */
        for (uint32_t i = 0; i < nw; i++) C0[i] = 0;    /* B_u(u): all h bits */
        for (uint32_t i = 0; i < h; i++) C0[i / L] |= 1u << (i % L);
        c.h = h; c.nw = nw; c.B = B; c.colour = colour; c.ids = Nu;
        c.R[0] = u; S.root = u;
        bitcol_list(&c, k - 1, 1, C0);
    }
    for (uint32_t i = 0; c.buf && i <= k; i++) free(c.buf[i]);
    free(c.buf); free(adj); free(B); free(colour); free(order); free(C0); free(pos);
    free_dag(&D);
    free(P.alive);
    if (rc) return rc;
    u128 tot = S.count + (roots ? 0 : P.count);
    if (tot >> 64) return OR_EOVERFLOW;
    *count = (uint64_t)tot;
    *checksum = S.checksum + (roots ? 0 : P.checksum);
    if (written) *written = wpre + S.written;
    if (out && (S.written < S.count || wpre < P.count)) return OR_ETRUNC;
    return OR_OK;
}
