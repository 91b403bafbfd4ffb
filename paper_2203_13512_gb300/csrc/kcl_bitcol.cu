// BitCol on the GPU (Algorithm 6, Section VII).  For every root u of the
// degeneracy DAG with d+_u >= k-1 a group of threads (one warp for small
// out-degrees, one CTA for large ones)
//   1. builds G_u, the undirected subgraph induced by N+_u (Section VII-B), as
//      bit-rows over the index space of N+_u (ascending id): each edge of G_u
//      lies in exactly one DAG out-list, so the group streams the out-lists of
//      N+_u once (flattened, load-balanced over lanes) and probes each entry
//      in a hash table of N+_u;
//   2. colours G_u greedily in (degree descending, index ascending) order,
//      colours from 1 (Section VII-A, Example 6);
//   3. re-indexes G_u by colour (colour classes become contiguous index
//      ranges, start[c] = first index of colour c) and encodes the colour-
//      ordered DAG: B'(p) holds the out-neighbours of p, all below
//      start[colour(p)] (BitEncode, Section VII-C);
//   4. runs BitColList as explicit-stack DFS: at level l only candidates of
//      colour >= l are expanded (Lemma 1 pruning, a prefix test after the
//      re-indexing), C' = B'(v) AND C (BitJoin), recursion when |C'| >= l-1,
//      and at l = 2 each w in C' closes a clique.  In the CTA form the
//      first-level children of the root are shared out to the CTA's warps.
// Lanes evaluate candidates in parallel (lane b takes bit b of a candidate
// word) and each lane ANDs + POPCs the words of its candidate's row that can
// be non-zero; rows have an odd word stride so 32 lanes reading 32 rows hit
// 32 different shared-memory banks.  The word size is 32 bits (the paper
// uses 24 on its CPU); results do not depend on it.
#include "kcl_internal.cuh"

namespace kcl {

namespace {

constexpr unsigned kFull = 0xffffffffu;

// ------------------------------------------------------------- layouts
// Subproblem region (words) for at most D = 32 W vertices.  A (undirected
// rows, old index) and B (colour-DAG rows, new index) may live in a global
// arena instead (a_global / b_global), in which case they take no room here.
struct SubLay {
    uint32_t W, D, WP, WPB, NBR, PRE, IDS, HK, HV, U16, META, PEND, A, B, total;
};

// Row strides.  A (build only): odd, so 32 lanes reading 32 rows hit 32
// banks.  B (read by the DFS): for W >= 4 a multiple of 4 words with an odd
// number of 16-byte chunks, so rows are read as 128-bit vectors and 8 lanes
// reading 8 consecutive rows hit 8 different bank quads.
__host__ __device__ inline uint32_t a_stride(uint32_t W) { return (W & 1) ? W : W + 1; }
__host__ __device__ inline uint32_t b_stride(uint32_t W) {
    return W >= 4 ? (((W >> 2) & 1) ? W : W + 4) : a_stride(W);
}

// D: rows (vertices) the layout holds, at most 32 W (0 = 32 W); a class
// whose largest out-degree is below its limit is laid out for that degree.
__host__ __device__ inline SubLay sub_layout(uint32_t W, bool a_global, bool b_global, uint32_t D = 0) {
    SubLay L;
    L.W = W;
    L.D = D ? D : 32 * W;
    L.WP = a_stride(W);
    L.WPB = b_stride(W);
    L.NBR = 0;
    L.PRE = L.NBR + L.D;        // D + 1
    L.IDS = L.PRE + L.D + 1;    // D
    L.HK = L.IDS + L.D;                 // hash keys (hash_cap(D))
    L.HV = L.HK + hash_cap(L.D);        // hash values, u16 (hash_cap(D))
    L.U16 = L.HV + hash_cap(L.D) / 2;   // colour_old, old2new, colp (D each), start (D + 2), u16
    L.META = L.U16 + (4 * L.D + 2 + 1) / 2;
    L.PEND = L.META + 8;        // first-level children (u16, D)
    uint32_t end = L.PEND + (L.D + 1) / 2;
    L.A = a_global ? 0 : end;
    if (!a_global) end += L.D * L.WP;
    end = (end + 3) & ~3u;  // B rows start on a 16-byte boundary
    L.B = b_global ? 0 : end;
    if (!b_global) end += L.D * L.WPB;
    L.total = (end + 3) & ~3u;
    return L;
}

// Per-warp DFS stack: C and pending-children bitmaps per depth, path, cursor.
// C and P per depth (2 k W), path and cursor (2 k), sortedR (32), leaf
// candidate queue (64 u16)
__host__ __device__ inline uint32_t dfs_words(uint32_t W, uint32_t k) {
    return (k * (2 * W + 2) + 32 + 32 + 3) & ~3u;
}

struct Sub {
    uint32_t *nbr, *pre, *ids, *hk, *meta;
    uint16_t *hv, *colour_old, *old2new, *colp, *start, *pend;
    uint32_t *A, *B;
};

__device__ inline Sub sub_ptrs(uint32_t *S, const SubLay &L, uint32_t *Ag, uint32_t *Bg) {
    Sub s;
    s.nbr = S + L.NBR;
    s.pre = S + L.PRE;
    s.ids = S + L.IDS;
    s.hk = S + L.HK;
    s.hv = reinterpret_cast<uint16_t *>(S + L.HV);
    s.colour_old = reinterpret_cast<uint16_t *>(S + L.U16);
    s.old2new = s.colour_old + L.D;
    s.colp = s.old2new + L.D;
    s.start = s.colp + L.D;
    s.meta = S + L.META;
    s.pend = reinterpret_cast<uint16_t *>(S + L.PEND);
    s.A = Ag ? Ag : S + L.A;
    s.B = Bg ? Bg : S + L.B;
    return s;
}

// A group working on one subproblem: NW = 1 is a single warp, NW > 1 the
// whole CTA (blockDim.x threads, at most NW warps).
template <int NW>
struct Grp {
    static __device__ __forceinline__ uint32_t size() { return NW == 1 ? 32u : blockDim.x; }
    static __device__ __forceinline__ uint32_t nwarps() { return NW == 1 ? 1u : (blockDim.x >> 5); }
    static __device__ __forceinline__ uint32_t tid() { return NW == 1 ? lane_id() : threadIdx.x; }
    static __device__ __forceinline__ uint32_t warp() { return NW == 1 ? 0u : (threadIdx.x >> 5); }
    static __device__ __forceinline__ void sync() {
        if (NW == 1) __syncwarp();
        else __syncthreads();
    }
};


// --------------------------------------------------------------- build
// Steps 1-3 above; leaves B', colp, start, ids and meta[0] = ncol.
template <int NW, int WT>
__device__ void build_sub(uint32_t d, uint32_t base, uint32_t Wrt, const uint32_t *__restrict__ optr,
                          const uint32_t *__restrict__ oadj, const Sub &s) {
    using G = Grp<NW>;
    const uint32_t W = WT ? (uint32_t)WT : Wrt;
    const uint32_t WP = a_stride(W), WPB = b_stride(W);
    const uint32_t tid = G::tid(), lane = lane_id(), warp = G::warp();

    // out-list lengths of N+_u (scanned below), row starts, zero rows
    for (uint32_t i = tid; i < d; i += G::size()) {
        uint32_t v = oadj[base + i];
        s.nbr[i] = v;
        uint32_t r0 = optr[v];
        s.ids[i] = r0;
        s.pre[i] = optr[v + 1] - r0;
    }
    for (uint32_t i = tid; i < d * WP; i += G::size()) s.A[i] = 0;
    for (uint32_t i = tid; i < d * WPB; i += G::size()) s.B[i] = 0;
    G::sync();
    if (warp == 0) {
        uint32_t running = 0;
        for (uint32_t c0 = 0; c0 < d; c0 += 32) {
            uint32_t i = c0 + lane;
            uint32_t x = i < d ? s.pre[i] : 0;
            uint32_t incl = warp_incl_scan(x);
            if (i < d) s.pre[i] = running + incl - x;
            running += __shfl_sync(kFull, incl, 31);
        }
        if (lane == 0) s.pre[d] = running;
    }
    uint32_t T, hshift;
    hash_size(d, &T, &hshift);
    for (uint32_t i = tid; i < T; i += G::size()) s.hk[i] = kHashEmpty;
    G::sync();
    for (uint32_t i = tid; i < d; i += G::size()) {
        uint32_t key = s.nbr[i], h = hash_slot(key, hshift);
        while (atomicCAS(&s.hk[h], kHashEmpty, key) != kHashEmpty) h = (h + 1) & (T - 1);
        s.hv[h] = (uint16_t)i;
    }
    G::sync();

    // G_u adjacency: stream the out-lists of N+_u as one flattened sequence
    const uint32_t total = s.pre[d];
    const uint32_t lo_id = s.nbr[0], hi_id = s.nbr[d - 1];
    uint32_t a0 = 0;
    for (uint32_t c = warp * 32; c < total; c += G::size()) {
        if (NW > 1) {  // row holding element c (largest a with pre[a] <= c)
            uint32_t lo = a0, hi = d;
            while (hi - lo > 1) {
                uint32_t m = (lo + hi) >> 1;
                if (s.pre[m] <= c) lo = m; else hi = m;
            }
            a0 = lo;
        }
        const uint32_t e = c + lane;
        uint32_t a = a0;
        if (e < total) {
            while (s.pre[a + 1] <= e) a++;
            uint32_t w = oadj[s.ids[a] + (e - s.pre[a])];
            if (w >= lo_id && w <= hi_id) {
                int x = hash_find(s.hk, s.hv, T, hshift, w);
                if (x >= 0) {
                    atomicOr(&s.A[a * WP + ((uint32_t)x >> 5)], 1u << (x & 31));
                    atomicOr(&s.A[(uint32_t)x * WP + (a >> 5)], 1u << (a & 31));
                }
            }
        }
        if (NW == 1) a0 = __shfl_sync(kFull, a, 31);
    }
    G::sync();

    // colouring order: degree in G_u descending, index ascending (bitonic sort)
    uint32_t P2 = 1;
    while (P2 < d) P2 <<= 1;
    for (uint32_t i = tid; i < P2; i += G::size()) {
        uint32_t key = 0xFFFFFFFFu;
        if (i < d) {
            uint32_t deg = 0;
            for (uint32_t t = 0; t < W; t++) deg += __popc(s.A[i * WP + t]);
            key = ((0xFFFFu - deg) << 16) | i;
        }
        s.pre[i] = key;
    }
    G::sync();
    for (uint32_t size = 2; size <= P2; size <<= 1)
        for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
            for (uint32_t i = tid; i < P2; i += G::size()) {
                uint32_t j = i ^ stride;
                if (j > i) {
                    bool up = (i & size) == 0;
                    uint32_t x = s.pre[i], y = s.pre[j];
                    if ((x > y) == up) { s.pre[i] = y; s.pre[j] = x; }
                }
            }
            G::sync();
        }

    // greedy colouring (one warp); colour class c is kept as row c-1 of B.
    // Vertex v's row of A is staged once in a 16-byte-aligned scratch (the
    // first-level child list, unused until the DFS), the next vertex's row
    // is fetched while v is tested, and lane i tests colour c0 + i + 1 with
    // 128-bit reads of the class row and broadcast reads of v's row.
    if (warp == 0) {
        uint32_t ncol = 0;
        uint32_t *arow = reinterpret_cast<uint32_t *>(
            (reinterpret_cast<uintptr_t>(s.pend) + 15) & ~static_cast<uintptr_t>(15));
        const bool vec = (W & 3u) == 0 && (WPB & 3u) == 0;
        uint32_t pf = lane < W ? s.A[(s.pre[0] & 0xFFFFu) * WP + lane] : 0u;  // next row, first 32 words
        for (uint32_t t = 0; t < d; t++) {
            const uint32_t v = s.pre[t] & 0xFFFFu;
            if (lane < W) arow[lane] = pf;
            for (uint32_t w = lane + 32; w < W; w += 32) arow[w] = s.A[v * WP + w];
            __syncwarp();
            if (t + 1 < d) pf = lane < W ? s.A[(s.pre[t + 1] & 0xFFFFu) * WP + lane] : 0u;
            uint32_t chosen = 0;
            for (uint32_t c0 = 0;; c0 += 32) {
                uint32_t c = c0 + lane + 1;
                bool fits = false;
                if (c <= ncol) {
                    uint32_t acc = 0;
                    const uint32_t *cls = s.B + (c - 1) * WPB;
                    if (vec) {
                        const uint4 *a4 = reinterpret_cast<const uint4 *>(arow);
                        const uint4 *b4 = reinterpret_cast<const uint4 *>(cls);
                        for (uint32_t w = 0; w < (W >> 2) && !acc; w++) {
                            const uint4 a = a4[w], b = b4[w];
                            acc = (a.x & b.x) | (a.y & b.y) | (a.z & b.z) | (a.w & b.w);
                        }
                    } else {
                        for (uint32_t w = 0; w < W; w++) acc |= arow[w] & cls[w];
                    }
                    fits = acc == 0;
                } else if (c == ncol + 1) {
                    fits = true;
                }
                unsigned m = __ballot_sync(kFull, fits);
                if (m) { chosen = c0 + __ffs(m); break; }
            }
            if (chosen > ncol) ncol = chosen;
            if (lane == 0) {
                s.B[(chosen - 1) * WPB + (v >> 5)] |= 1u << (v & 31);
                s.colour_old[v] = (uint16_t)chosen;
            }
            __syncwarp();
        }
        // start[c]: first index of colour c in the colour-sorted order
        uint32_t run = 0;
        for (uint32_t c0 = 0; c0 < ncol; c0 += 32) {
            uint32_t c = c0 + lane + 1;
            uint32_t sz = 0;
            if (c <= ncol)
                for (uint32_t w = 0; w < W; w++) sz += __popc(s.B[(c - 1) * WPB + w]);
            uint32_t incl = warp_incl_scan(sz);
            if (c <= ncol) s.start[c] = (uint16_t)(run + incl - sz);
            run += __shfl_sync(kFull, incl, 31);
        }
        if (lane == 0) {
            s.start[0] = 0;
            s.start[ncol + 1] = (uint16_t)d;
            s.meta[0] = ncol;
        }
    }
    G::sync();
    for (uint32_t i = tid; i < d; i += G::size()) {
        uint32_t c = s.colour_old[i];
        const uint32_t *cls = s.B + (c - 1) * WPB;
        uint32_t r = 0;
        for (uint32_t w = 0; w < (i >> 5); w++) r += __popc(cls[w]);
        r += __popc(cls[i >> 5] & ((1u << (i & 31)) - 1u));
        uint32_t p = s.start[c] + r;
        s.old2new[i] = (uint16_t)p;
        s.colp[p] = (uint16_t)c;
        s.ids[p] = s.nbr[i];
    }
    G::sync();
    for (uint32_t i = tid; i < d * WPB; i += G::size()) s.B[i] = 0;
    G::sync();
    // B'(p): out-neighbours (lower colour = index below start[colour]); one
    // thread per row, so no two threads write the same row
    for (uint32_t i = tid; i < d; i += G::size()) {
        uint32_t p = s.old2new[i];
        uint32_t lim = s.start[s.colour_old[i]];
        uint32_t *row = s.B + p * WPB;
        for (uint32_t w = 0; w < W; w++) {
            uint32_t m = s.A[i * WP + w];
            while (m) {
                uint32_t j = w * 32 + (__ffs(m) - 1);
                m &= m - 1;
                uint32_t q = s.old2new[j];
                if (q < lim) row[q >> 5] |= 1u << (q & 31);
            }
        }
    }
    G::sync();
}

// ----------------------------------------------------------------- DFS
struct Emit {
    uint32_t *ring;
    unsigned long long capacity;
    int wrap;
    unsigned long long *root_cks;  // listing: per-root checksum sums, or null
    const uint32_t *idmap;         // listing: vertex -> output id, or null (identity)
    uint32_t prune;                // 1: Lemma 1 colour prune (0 only for ablations)
    uint32_t dfs_warps;            // CTA form: warps walking the children (0 = all)
    unsigned long long *slots;     // CTA form: work-splitting slots (one per CTA)
    uint32_t split;                // CTA form: help a root with >= split children left (0 = off)
    const uint8_t *kmap;           // batches: k of each root's graph (null: the launch's k)
};

struct View {  // read-only view of a built subproblem, per warp
    const uint32_t *B;
    const uint16_t *colp, *start;
    const uint32_t *ids;
    uint32_t d, W, WP, ncol, u, k;
    uint32_t prune;  // 0: expand every candidate (ablation of Lemma 1)
    unsigned long long deadline;  // time limit (global timer, ns; 0 = none)
};

// First candidate index at level l: the vertices of colour >= l (Lemma 1),
// which the colour-sorted indexing makes a suffix.
__device__ __forceinline__ uint32_t start_of(const View &v, uint32_t l) {
    if (!v.prune) return 0;
    return l <= v.ncol + 1 ? (uint32_t)v.start[l] : v.d;
}

// bits of C[j] at index >= s
__device__ __forceinline__ uint32_t cand_word(const uint32_t *C, uint32_t j, uint32_t s) {
    uint32_t m = C[j];
    uint32_t lo = j * 32;
    if (s >= lo + 32) return 0u;
    if (s > lo) m &= ~((1u << (s - lo)) - 1u);
    return m;
}

// |row & C| over the first wl words.  For W >= 4 both are read as 128-bit
// vectors up to round4(wl) <= W: C is zero beyond its cw words and a row is
// zero beyond ceil(start[colour] / 32) words, so the extra words add nothing.
__device__ __forceinline__ uint32_t and_popc(const uint32_t *row, const uint32_t *C, uint32_t wl,
                                             uint32_t W) {
    uint32_t x = 0;
    if (W >= 4) {
        const uint4 *r4 = reinterpret_cast<const uint4 *>(row);
        const uint4 *c4 = reinterpret_cast<const uint4 *>(C);
        for (uint32_t t = 0; t < (wl + 3) >> 2; t++) {
            const uint4 a = r4[t], b = c4[t];
            x += __popc(a.x & b.x) + __popc(a.y & b.y) + __popc(a.z & b.z) + __popc(a.w & b.w);
        }
    } else {
        for (uint32_t t = 0; t < wl; t++) x += __popc(row[t] & C[t]);
    }
    return x;
}

__device__ __forceinline__ uint32_t row_words(const View &v, uint32_t p, uint32_t cw) {
    uint32_t wl = (v.start[v.colp[p]] + 31) >> 5;
    return wl < cw ? wl : cw;
}

// A lane's run of rlen cliques within a leaf batch: its first clique is set
// bit `rank` of B'(q[o]) & C, and it walks the set bits of the queued
// candidates' rows from there, writing records lane, lane + 32, ... of the
// batch (base slot0).
template <int NR>
__device__ __forceinline__ void leaf_walk(const View &v, const uint32_t *C, uint32_t cw,
                                          const uint16_t *q, uint32_t o, uint32_t rank, uint32_t rlen,
                                          const uint32_t *sortedR, const Emit &em,
                                          unsigned long long slot0, unsigned long long &cks) {
    CliqueOut<NR> co;
    co.init(sortedR, v.k, em.ring, em.capacity, em.wrap, slot0, lane_id());
    uint32_t po = q[o];
    const uint32_t *row = v.B + po * v.WP;
    uint32_t wl = row_words(v, po, cw), a = v.ids[po];
    uint32_t t = 0, mm = 0;
    for (; t < wl; t++) {
        mm = row[t] & C[t];
        const uint32_t c = __popc(mm);
        if (rank < c) break;
        rank -= c;
    }
    for (uint32_t z = 0; z < rank; z++) mm &= mm - 1;
    for (uint32_t r = 0; r < rlen; r++) {
        // mm holds the remaining bits of word t (its lowest is the next clique)
        const uint32_t b = t * 32 + (__ffs(mm) - 1);
        cks += co.put(a, v.ids[b]);
        mm &= mm - 1;
        while (!mm && r + 1 < rlen) {
            if (++t >= wl) {  // next candidate with cliques
                po = q[++o];
                row = v.B + po * v.WP;
                wl = row_words(v, po, cw);
                a = v.ids[po];
                t = 0;
            }
            mm = row[t] & C[t];
        }
    }
}

// A batch of nb <= 32 leaf candidates q[0..nb): lane i takes candidate q[i]
// and closes |B'(q[i]) & C| cliques.
template <bool LIST>
__device__ void leaf_batch(const View &v, const uint32_t *C, uint32_t cw, const uint16_t *q,
                           uint32_t nb, const uint32_t *sortedR, const Emit &em, DevResult *res,
                           unsigned long long &cnt, unsigned long long &cks) {
    const unsigned lane = lane_id();
    uint32_t x = 0;
    if (lane < nb) {
        const uint32_t p = q[lane];
        const uint32_t *row = v.B + p * v.WP;
        x = and_popc(row, C, row_words(v, p, cw), v.W);
    }
    cnt += x;
    if (!LIST) return;
    // the tot cliques of the batch, in (candidate, bit) order, are cut into
    // 32 contiguous runs, one per lane: a lane finds its first clique once
    // (the candidate whose prefix holds it, then its bit) and walks the set
    // bits of B'(q[o]) & C from there, moving on to the next candidates
    const uint32_t incl = warp_incl_scan(x);
    const uint32_t excl = incl - x;
    const uint32_t tot = __shfl_sync(kFull, incl, 31);
    if (!tot) return;
    unsigned long long slot0 = 0;
    if (em.ring) {
        if (lane == 0) slot0 = ring_base(atomicAdd(&res->emitted, (unsigned long long)tot), em.capacity, em.wrap);
        slot0 = __shfl_sync(kFull, slot0, 0);
    }
    // balanced runs: lane i takes tot/32 cliques, one more when i < tot%32;
    // its j-th clique goes to record j * 32 + i of the batch, so the warp's
    // stores at each step are 32 consecutive records
    const uint32_t rq = tot >> 5, rrem = tot & 31u;
    const uint32_t r0 = lane * rq + (lane < rrem ? lane : rrem);
    const uint32_t rlen = rq + (lane < rrem ? 1u : 0u);
    uint32_t o = 0;  // number of lanes whose inclusive prefix is <= r0
#pragma unroll
    for (uint32_t step = 16; step > 0; step >>= 1) {
        const uint32_t vv = __shfl_sync(kFull, incl, o + step - 1);
        if (vv <= r0) o += step;
    }
    const uint32_t eo = __shfl_sync(kFull, excl, o & 31u);
    if (rlen == 0) return;
    switch (v.k) {  // warp-uniform: R in registers for the common k
        case 3: leaf_walk<1>(v, C, cw, q, o, r0 - eo, rlen, sortedR, em, slot0, cks); break;
        case 4: leaf_walk<2>(v, C, cw, q, o, r0 - eo, rlen, sortedR, em, slot0, cks); break;
        case 5: leaf_walk<3>(v, C, cw, q, o, r0 - eo, rlen, sortedR, em, slot0, cks); break;
        case 6: leaf_walk<4>(v, C, cw, q, o, r0 - eo, rlen, sortedR, em, slot0, cks); break;
        default: leaf_walk<0>(v, C, cw, q, o, r0 - eo, rlen, sortedR, em, slot0, cks);
    }
}

// Leaf (l = 2) over candidate words j0, j0+js, ... < cw: each candidate p
// (colour >= 2) closes |B'(p) & C| cliques.  The candidates of consecutive
// words are packed into a per-warp queue (64 entries after sortedR) and
// evaluated 32 at a time, so lanes stay busy when the words are sparse.
// depth = number of path entries below the root.
template <bool LIST>
__device__ void leaf(const View &v, const uint32_t *C, uint32_t cw, uint32_t depth, uint32_t j0,
                     uint32_t js, const uint32_t *path, uint32_t *sortedR, const Emit &em,
                     DevResult *res, unsigned long long &cnt, unsigned long long &cks) {
    const unsigned lane = lane_id();
    const uint32_t s = start_of(v, 2);
    uint16_t *q = reinterpret_cast<uint16_t *>(sortedR + 32);
    if (LIST) {
        if (lane == 0) {
            sortedR[0] = v.u;
            for (uint32_t t = 1; t <= depth; t++) {
                uint32_t x = v.ids[path[t]], j = t;
                while (j > 0 && sortedR[j - 1] > x) { sortedR[j] = sortedR[j - 1]; j--; }
                sortedR[j] = x;
            }
        }
        __syncwarp();
    }
    uint32_t pend = 0;  // queued candidates (< 32 between words)
    for (uint32_t j = j0; j < cw; j += js) {
        const uint32_t m = cand_word(C, j, s);
        if (!m) continue;
        if ((m >> lane) & 1u) q[pend + __popc(m & ((1u << lane) - 1u))] = (uint16_t)(j * 32 + lane);
        pend += __popc(m);
        if (pend >= 32) {
            __syncwarp();
            leaf_batch<LIST>(v, C, cw, q, 32, sortedR, em, res, cnt, cks);
            __syncwarp();
            if (lane < pend - 32) q[lane] = q[32 + lane];
            pend -= 32;
            __syncwarp();
        }
    }
    if (pend) {
        __syncwarp();
        leaf_batch<LIST>(v, C, cw, q, pend, sortedR, em, res, cnt, cks);
        __syncwarp();
    }
}

// |B'(q) & C| for the 32 rows q = 32 j + lane of candidate word j: the rows
// lie below 32 (j + 1), so every lane reads the same number of words (a
// uniform loop; rows and C are zero beyond their extents).
__device__ __forceinline__ uint32_t word_block_popc(const View &v, const uint32_t *C, uint32_t cw,
                                                    uint32_t j) {
    const uint32_t q = j * 32 + lane_id();
    const uint32_t *row = v.B + q * v.WP;
    uint32_t x = 0;
    if (v.W >= 4) {
        const uint32_t nc = min((j >> 2) + 1, (cw + 3) >> 2);
        const uint4 *r4 = reinterpret_cast<const uint4 *>(row);
        const uint4 *c4 = reinterpret_cast<const uint4 *>(C);
        for (uint32_t t = 0; t < nc; t++) {
            const uint4 a = r4[t], b = c4[t];
            x += __popc(a.x & b.x) + __popc(a.y & b.y) + __popc(a.z & b.z) + __popc(a.w & b.w);
        }
    } else {
        const uint32_t nw = min(j + 1, cw);
        for (uint32_t t = 0; t < nw; t++) x += __popc(row[t] & C[t]);
    }
    return x;
}

// Inner node at level l >= 3: pending children = candidates p with
// |B'(p) & C| >= l-1, as a bitmap P[0..W).
__device__ void expand(const View &v, const uint32_t *C, uint32_t cw, uint32_t l, uint32_t *P) {
    const unsigned lane = lane_id();
    const uint32_t s = start_of(v, l);
    for (uint32_t j = 0; j < v.W; j++) {
        const uint32_t m = j < cw ? cand_word(C, j, s) : 0u;
        bool ok = false;
        if (m) {  // all lanes read their rows (uniform); non-candidates are masked
            const uint32_t x = word_block_popc(v, C, cw, j);
            ok = ((m >> lane) & 1u) && x + 1 >= l;
        }
        const unsigned bal = __ballot_sync(kFull, ok);
        if (lane == 0) P[j] = bal;
    }
    __syncwarp();
}

// |B'(q) & B'(p) & C| for lane pairs (p, q) held in registers (has: the lane
// holds one); the rows lie below q, so all lanes read the words up to the
// largest q.
__device__ __forceinline__ void pair_round(const View &v, const uint32_t *C, uint32_t cw, bool has,
                                           uint32_t p, uint32_t q, uint32_t &acc) {
    const uint32_t qmax = __reduce_max_sync(kFull, has ? q : 0u);
    const uint32_t *rq = v.B + q * v.WP, *rp = v.B + p * v.WP;
    uint32_t x = 0;
    if (v.W >= 4) {
        const uint32_t nc = min((qmax >> 7) + 1, (cw + 3) >> 2);
        const uint4 *a4 = reinterpret_cast<const uint4 *>(rq);
        const uint4 *b4 = reinterpret_cast<const uint4 *>(rp);
        const uint4 *c4 = reinterpret_cast<const uint4 *>(C);
#pragma unroll 2
        for (uint32_t t = 0; t < nc; t++) {
            const uint4 a = a4[t], b = b4[t], c = c4[t];
            x += __popc(a.x & b.x & c.x) + __popc(a.y & b.y & c.y) + __popc(a.z & b.z & c.z) +
                 __popc(a.w & b.w & c.w);
        }
    } else {
        const uint32_t nw = min((qmax >> 5) + 1, cw);
        for (uint32_t t = 0; t < nw; t++) x += __popc(rq[t] & rp[t] & C[t]);
    }
    acc += has ? x : 0u;
}

// Counting below a level-3 node with candidate set C and pending children P
// (Algorithm 6 at levels 3 and 2): for every child p and every q in
// B'(p) & C of colour >= 2, |B'(q) & B'(p) & C| cliques close.  The words
// of B'(p) & Cm (Cm: C restricted to colour >= 2, the leaf candidates) for
// all children p form a stream of items (p, t); each lane holds one item's
// remaining bits and, every round, turns its lowest bit q into the pair
// (p, q), so a round is a batch of up to 32 pairs built in registers.  A lane
// whose word runs out takes the next item from a 64-entry ring (ibuf), which
// the warp refills with up to 32 words of the next child at a time.  The
// per-lane sum stays 32-bit within the node: at most d^2 / 32 pairs of at
// most d cliques per lane, below 2^31 for d <= 4096 (the largest class).
__device__ void leaf_pairs(const View &v, const uint32_t *C, uint32_t cw, const uint32_t *P,
                           uint32_t *Cm, uint32_t *ibuf, unsigned long long &cnt) {
    const unsigned lane = lane_id();
    const uint32_t s2 = start_of(v, 2);
    for (uint32_t t = lane; t < v.W; t += 32) Cm[t] = t < cw ? cand_word(C, t, s2) : 0u;
    __syncwarp();
    const unsigned lt = (1u << lane) - 1u;
    // producer (warp-uniform): child word jp / bits pw, current child cp with
    // its next word ct of cn; ring ibuf[head..tail) (indices mod 64)
    uint32_t jp = s2 >> 5, pw = jp < cw ? P[jp] : 0u, cp = 0, ct = 0, cn = 0;
    uint32_t head = 0, tail = 0;
    // lane: remaining bits m of word t (bit offset tb) of child p
    uint32_t m = 0, p = 0, tb = 0, acc = 0;
    bool more = true;  // items may remain
    for (;;) {
        // give every lane without bits a new word while items remain
        while (more) {
            const unsigned need = __ballot_sync(kFull, m == 0);
            if (!need) break;
            const uint32_t nneed = __popc(need);
            while (tail - head < nneed) {
                if (ct >= cn) {  // next child
                    while (!pw && jp + 1 < cw) pw = P[++jp];
                    if (!pw) break;
                    cp = jp * 32 + (__ffs(pw) - 1);
                    pw &= pw - 1;
                    ct = 0;
                    cn = min(cw, (cp >> 5) + 1);  // B'(p) lies below p
                }
                const uint32_t nt = min(cn - ct, 32u);
                if (lane < nt) ibuf[(tail + lane) & 63u] = (cp << 16) | (ct + lane);
                tail += nt;
                ct += nt;
                __syncwarp();
            }
            const uint32_t avail = min(tail - head, nneed);
            if (avail < nneed) more = false;  // the stream is exhausted
            if (m == 0) {
                const uint32_t r = __popc(need & lt);
                if (r < avail) {
                    const uint32_t it = ibuf[(head + r) & 63u];
                    p = it >> 16;
                    const uint32_t t = it & 0xFFFFu;
                    m = v.B[p * v.WP + t] & Cm[t];
                    tb = t * 32;
                }
            }
            head += avail;
            __syncwarp();
        }
        const bool has = m != 0;
        if (!__any_sync(kFull, has)) break;
        uint32_t q = 0;
        if (has) {
            q = tb + (__ffs(m) - 1);
            m &= m - 1;
        }
        pair_round(v, C, cw, has, p, q, acc);
    }
    cnt += acc;
}

// The subtree below first-level child p0 of the root (C1 = B'(p0)), run by
// one warp with its own stack.
template <bool LIST>
__device__ void dfs_child(const View &v, uint32_t p0, uint32_t *stack, const Emit &em,
                          DevResult *res, unsigned long long &cnt, unsigned long long &cks) {
    const unsigned lane = lane_id();
    const uint32_t W = v.W, k = v.k;
    uint32_t *Cst = stack;             // k * W
    uint32_t *Pst = Cst + k * W;       // k * W
    uint32_t *path = Pst + k * W;      // k
    uint32_t *cur = path + k;          // k
    uint32_t *sortedR = cur + k;       // 32
    const uint32_t dw = (v.d + 31) >> 5;
    // depth 1: C1 = B'(p0) (the root's candidate set is all of N+_u)
    uint32_t cw1 = row_words(v, p0, dw);
    for (uint32_t t = lane; t < W; t += 32) Cst[W + t] = t < cw1 ? v.B[p0 * v.WP + t] : 0u;
    if (lane == 0) path[1] = p0;
    __syncwarp();
    uint32_t l = k - 2;
    if (l == 2) {
        leaf<LIST>(v, Cst + W, cw1, 1, 0, 1, path, sortedR, em, res, cnt, cks);
        __syncwarp();
        return;
    }
    expand(v, Cst + W, cw1, l, Pst + W);
    if (!LIST && l == 3) {  // sortedR and the leaf queue (64 words) hold the pair queue
        leaf_pairs(v, Cst + W, cw1, Pst + W, Cst + 2 * W, sortedR, cnt);
        __syncwarp();
        return;
    }
    if (lane == 0) cur[1] = 0;
    uint32_t cwst[KCL_MAX_K];
    cwst[1] = cw1;
    __syncwarp();
    int depth = 1;
    while (depth >= 1) {
        if (warp_past_deadline(v.deadline, res)) return;
        uint32_t *P = Pst + depth * W;
        uint32_t j = cur[depth];
        while (j < W && P[j] == 0) j++;
        if (j >= W) { depth--; continue; }
        uint32_t pw = P[j];
        uint32_t p = j * 32 + (__ffs(pw) - 1);
        __syncwarp();
        if (lane == 0) { P[j] = pw & (pw - 1); cur[depth] = j; }
        const uint32_t *C = Cst + depth * W;
        uint32_t *Cn = Cst + (depth + 1) * W;
        uint32_t ncw = row_words(v, p, cwst[depth]);
        for (uint32_t t = lane; t < W; t += 32) Cn[t] = t < ncw ? (v.B[p * v.WP + t] & C[t]) : 0u;
        if (lane == 0) path[depth + 1] = p;
        __syncwarp();
        uint32_t lc = k - 2 - (uint32_t)depth;  // level of the child
        if (lc == 2) {
            leaf<LIST>(v, Cn, ncw, depth + 1, 0, 1, path, sortedR, em, res, cnt, cks);
            __syncwarp();
        } else if (!LIST && lc == 3) {
            expand(v, Cn, ncw, 3, Pst + (depth + 1) * W);
            leaf_pairs(v, Cn, ncw, Pst + (depth + 1) * W, Cn + W, sortedR, cnt);
            __syncwarp();
        } else {
            expand(v, Cn, ncw, lc, Pst + (depth + 1) * W);
            if (lane == 0) cur[depth + 1] = 0;
            cwst[depth + 1] = ncw;
            __syncwarp();
            depth++;
        }
    }
}

// First-level children of the root: p >= start[k-1] with |B'(p)| >= k-2,
// written to pend in descending index order (heaviest first); returns count.
template <int NW>
__device__ uint32_t root_children(const View &v, const Sub &s) {
    using G = Grp<NW>;
    const uint32_t l0 = v.k - 1;
    const uint32_t st = start_of(v, l0);
    if (G::warp() == 0) {
        const unsigned lane = lane_id();
        const uint32_t dw = (v.d + 31) >> 5;
        uint32_t n = 0;
        for (uint32_t q = st; q < v.d; q += 32) {
            bool ok = false;
            uint32_t p = 0;
            if (q + lane < v.d) {
                p = v.d - 1 - (q - st) - lane;  // descending from d-1 down to st
                const uint32_t *row = v.B + p * v.WP;
                uint32_t wl = row_words(v, p, dw), x = 0;
                for (uint32_t t = 0; t < wl; t++) x += __popc(row[t]);
                ok = x + 2 >= l0;
            }
            unsigned m = __ballot_sync(kFull, ok);
            if (ok) s.pend[n + __popc(m & ((1u << lane) - 1u))] = (uint16_t)p;
            n += __popc(m);
        }
        if (lane == 0) { s.meta[1] = n; s.meta[2] = 0; }
    }
    G::sync();
    return s.meta[1];
}

// --------------------------------------------------------------- kernels
// Warp per root: subproblem and stack in this warp's slice of shared memory.
template <int WT, bool LIST>
__global__ void __launch_bounds__(128, 8) k_bitcol_warp(uint32_t kmax, const uint32_t *__restrict__ optr,
                                                    const uint32_t *__restrict__ oadj,
                                                    const uint32_t *__restrict__ roots,
                                                    uint32_t begin, uint32_t end, unsigned *queue,
                                                    Emit em, unsigned long long *per_root,
                                                    DevResult *res) {
    extern __shared__ uint32_t smem[];
    const unsigned lane = lane_id();
    const SubLay L = sub_layout(WT, false, false);
    const uint32_t per_warp = L.total + dfs_words(WT, kmax);  // stacks for the largest k
    uint32_t *S = smem + (threadIdx.x >> 5) * per_warp;
    const Sub s = sub_ptrs(S, L, nullptr, nullptr);
    uint32_t *stack = S + L.total;
    const unsigned long long deadline = __ldcg(&res->deadline_ns);
    unsigned long long cnt = 0, cks = 0;
    for (;;) {
        if (warp_past_deadline(deadline, res)) break;
        uint32_t idx = 0;
        if (lane == 0) idx = atomicAdd(queue, 1u);
        idx = __shfl_sync(kFull, idx, 0);
        if (idx >= end - begin) break;
        const uint32_t u = roots[begin + idx];
        const uint32_t k = em.kmap ? (uint32_t)em.kmap[u] : kmax;
        const uint32_t base = optr[u], d = optr[u + 1] - base;
        const unsigned long long before = cnt;
        const unsigned long long before_cks = cks;
        build_sub<1, WT>(d, base, WT, optr, oadj, s);
        if (LIST && em.idmap) {  // output ids (batched unions map back to each graph's ids)
            for (uint32_t i = lane; i < d; i += 32) s.ids[i] = em.idmap[s.ids[i]];
            __syncwarp();
        }
        const uint32_t uo = (LIST && em.idmap) ? em.idmap[u] : u;
        View v{s.B, s.colp, s.start, s.ids, d, WT, L.WPB, s.meta[0], uo, k, em.prune, deadline};
        if (k == 3) {
            const uint32_t dw = (d + 31) >> 5;
            for (uint32_t t = lane; t < WT; t += 32)
                stack[t] = t < dw ? (t * 32 + 32 <= d ? kFull : (1u << (d - t * 32)) - 1u) : 0u;
            __syncwarp();
            uint32_t *path = stack + 2 * k * WT, *sortedR = path + 2 * k;
            leaf<LIST>(v, stack, dw, 0, 0, 1, path, sortedR, em, res, cnt, cks);
        } else {
            const uint32_t nch = root_children<1>(v, s);
            for (uint32_t i = 0; i < nch; i++) dfs_child<LIST>(v, s.pend[i], stack, em, res, cnt, cks);
        }
        if (per_root) {
            unsigned long long mine = cnt - before;
            for (int o = 16; o > 0; o >>= 1) mine += __shfl_down_sync(kFull, mine, o);
            if (lane == 0 && mine) atomicAdd(&per_root[u], mine);
        }
        if (LIST && em.root_cks) {
            unsigned long long mine = cks - before_cks;
            for (int o = 16; o > 0; o >>= 1) mine += __shfl_down_sync(kFull, mine, o);
            if (lane == 0 && mine) atomicAdd(&em.root_cks[u], mine);
        }
        __syncwarp();
    }
    for (int o = 16; o > 0; o >>= 1) {
        cnt += __shfl_down_sync(kFull, cnt, o);
        cks += __shfl_down_sync(kFull, cks, o);
    }
    if (lane == 0) {
        add_count(&res->count, &res->count_carry, cnt);
        if (LIST && cks) atomicAdd(&res->checksum, cks);
    }
}

// CTA per root: the subproblem is built once by the whole CTA (A and/or B in
// a global arena slice when they do not fit), then the root's first-level
// children are handed out to the warps, heaviest first.
// At least 1024 threads per SM (two 512-thread CTAs): at most 64 registers.
template <int NW, bool LIST, bool AG, bool BG>
__global__ void __launch_bounds__(NW * 32, (32 / NW > 0 ? 32 / NW : 1)) k_bitcol_cta(uint32_t kmax, uint32_t W, uint32_t D,
                                                       const uint32_t *__restrict__ optr,
                                                       const uint32_t *__restrict__ oadj,
                                                       const uint32_t *__restrict__ roots,
                                                       uint32_t begin, uint32_t end, unsigned *queue,
                                                       uint32_t *arena, Emit em,
                                                       unsigned long long *per_root, DevResult *res) {
    extern __shared__ uint32_t smem[];
    __shared__ uint32_t root_idx;
    const unsigned lane = lane_id();
    const uint32_t warp = threadIdx.x >> 5;
    // warps that walk the root's children: all of them (EdgeParallel units
    // shared out) unless the tuning caps it (1 = one warp per root)
    const uint32_t nd = em.dfs_warps && em.dfs_warps < (blockDim.x >> 5) ? em.dfs_warps : (blockDim.x >> 5);
    const SubLay L = sub_layout(W, AG, BG, D);
    const size_t rows_a = (size_t)L.D * L.WP, rows_b = (size_t)L.D * L.WPB;
    uint32_t *slice = arena + (size_t)blockIdx.x * ((AG ? rows_a : 0) + (BG ? rows_b : 0));
    uint32_t *Ag = AG ? slice : nullptr;
    uint32_t *Bg = BG ? slice + (AG ? rows_a : 0) : nullptr;
    const Sub s = sub_ptrs(smem, L, Ag, Bg);
    uint32_t *stack = smem + L.total + warp * dfs_words(W, kmax);  // stacks for the largest k
    __shared__ int help_slot;  // -1: own root from the queue; else the slot of the root helped
    const unsigned long long deadline = __ldcg(&res->deadline_ns);
    unsigned long long cnt = 0, cks = 0;
    bool queue_done = false;
    for (;;) {
        if (threadIdx.x == 0) {  // thread 0 alone reads the timer
            if (!queue_done && past_deadline(deadline, res)) queue_done = true;
            root_idx = queue_done ? end - begin : atomicAdd(queue, 1u);
            help_slot = (queue_done && deadline && global_ns() > deadline) ? -2 : -1;
        }
        __syncthreads();
        uint32_t idx = root_idx;
        const bool late = help_slot == -2;
        int helping = -1;
        __syncthreads();  // every thread has read root_idx and help_slot before they are rewritten
        if (idx >= end - begin) {
            queue_done = true;
            // no root left: help the root with the most children left
            if (!em.split || kmax == 3 || late) break;
            if (warp == 0) {
                uint32_t pos = 0;
                const int j = split_pick(em.slots, gridDim.x, blockIdx.x, em.split, &pos);
                if (lane == 0) { help_slot = j; root_idx = pos; }
            }
            __syncthreads();
            helping = help_slot;
            idx = root_idx;
            if (helping < 0 || idx >= end - begin) break;
        }
        const uint32_t u = roots[begin + idx];
        const uint32_t k = em.kmap ? (uint32_t)em.kmap[u] : kmax;
        const uint32_t base = optr[u], d = optr[u + 1] - base;
        const unsigned long long before = cnt;
        const unsigned long long before_cks = cks;
        build_sub<NW, 0>(d, base, W, optr, oadj, s);
        if (LIST && em.idmap) {  // output ids (batched unions map back to each graph's ids)
            for (uint32_t i = threadIdx.x; i < d; i += blockDim.x) s.ids[i] = em.idmap[s.ids[i]];
            __syncthreads();
        }
        const uint32_t uo = (LIST && em.idmap) ? em.idmap[u] : u;
        View v{s.B, s.colp, s.start, s.ids, d, W, L.WPB, s.meta[0], uo, k, em.prune, deadline};
        if (k == 3) {
            const uint32_t dw = (d + 31) >> 5;
            for (uint32_t t = lane; t < W; t += 32)
                stack[t] = t < dw ? (t * 32 + 32 <= d ? kFull : (1u << (d - t * 32)) - 1u) : 0u;
            __syncwarp();
            uint32_t *path = stack + 2 * k * W, *sortedR = path + 2 * k;
            if (warp < nd) leaf<LIST>(v, stack, dw, 0, warp, nd, path, sortedR, em, res, cnt, cks);
        } else {
            const uint32_t nch = root_children<NW>(v, s);
            // children are taken from this CTA's slot (own root) or the
            // helped CTA's slot when splitting is on, else from shared memory
            if (em.split && helping < 0 && threadIdx.x == 0) split_publish(em.slots + blockIdx.x, idx, nch);
            __syncthreads();
            for (; warp < nd;) {
                uint32_t i = 0;
                if (lane == 0)
                    i = em.split ? split_claim(em.slots + (helping >= 0 ? (uint32_t)helping : blockIdx.x), idx)
                                 : atomicAdd(&s.meta[2], 1u);
                i = __shfl_sync(kFull, i, 0);
                if (i >= nch) break;
                dfs_child<LIST>(v, s.pend[i], stack, em, res, cnt, cks);
            }
        }
        if (per_root) {
            unsigned long long mine = cnt - before;
            for (int o = 16; o > 0; o >>= 1) mine += __shfl_down_sync(kFull, mine, o);
            if (lane == 0 && mine) atomicAdd(&per_root[u], mine);
        }
        if (LIST && em.root_cks) {
            unsigned long long mine = cks - before_cks;
            for (int o = 16; o > 0; o >>= 1) mine += __shfl_down_sync(kFull, mine, o);
            if (lane == 0 && mine) atomicAdd(&em.root_cks[u], mine);
        }
        __syncthreads();
    }
    for (int o = 16; o > 0; o >>= 1) {
        cnt += __shfl_down_sync(kFull, cnt, o);
        cks += __shfl_down_sync(kFull, cks, o);
    }
    if (lane == 0) {
        add_count(&res->count, &res->count_carry, cnt);
        if (LIST && cks) atomicAdd(&res->checksum, cks);
    }
}

// The colouring of one root's subproblem, for checking it against an
// independent implementation: the same build_sub as the listing kernels (one
// CTA, both row sets in `arena`), then the colour of each out-neighbour of u
// in ascending id order (Section VII-A; Example 6).
template <int NW>
__global__ void __launch_bounds__(NW * 32) k_bitcol_colours(uint32_t W, uint32_t D,
                                                           const uint32_t *__restrict__ optr,
                                                           const uint32_t *__restrict__ oadj,
                                                           uint32_t u, uint32_t *arena,
                                                           uint32_t *out_nbr, uint32_t *out_colour) {
    extern __shared__ uint32_t smem[];
    const SubLay L = sub_layout(W, true, true, D);
    const Sub s = sub_ptrs(smem, L, arena, arena + (size_t)L.D * L.WP);
    const uint32_t base = optr[u], d = optr[u + 1] - base;
    if (d == 0 || d > D) return;
    build_sub<NW, 0>(d, base, W, optr, oadj, s);
    for (uint32_t i = threadIdx.x; i < d; i += blockDim.x) {
        out_nbr[i] = s.nbr[i];
        out_colour[i] = s.colour_old[i];
    }
}

// --------------------------------------------------------------- classes
// d+ <= 32 W.  Warp per root for W <= 4, CTA per root above.
struct ClassCfg {
    uint32_t W;
    int nw;      // warps per CTA (CTA form) or warps per block (warp form)
    bool cta, ag, bg;
};
constexpr ClassCfg kClass[] = {
    {1, 4, false, false, false},  {2, 4, false, false, false},  {4, 4, false, false, false},
    {8, 8, true, false, false},   {16, 16, true, false, false}, {32, 16, true, true, false},
    {64, 4, true, true, true},    {128, 2, true, true, true},
};
constexpr int kNumClasses = 8;

constexpr size_t kSmemCap = 220 * 1024;
constexpr size_t kSmemHalf = 112 * 1024;  // two CTAs per SM

// Warps per CTA for class c at this k: the configured count, reduced until
// the subproblem plus one DFS stack per warp fits in shared memory.
// Layout of CTA class c when its largest out-degree is maxd: rows for
// round32(maxd) vertices and round4(words) words per row (at most the
// class's own W and 32 W).
void class_layout(int c, uint32_t maxd, uint32_t *W, uint32_t *D) {
    const ClassCfg &cc = kClass[c];
    uint32_t d = maxd < 32 * cc.W ? maxd : 32 * cc.W;
    uint32_t dd = (d + 31) & ~31u;
    if (dd < 32) dd = 32;
    uint32_t w = (((dd >> 5) + 3) & ~3u);
    if (w > cc.W) w = cc.W;
    *W = w;
    *D = dd;
}

int class_warps(int c, uint32_t k, uint32_t W, uint32_t D) {
    const ClassCfg &cc = kClass[c];
    if (!cc.cta) return cc.nw;
    size_t sub = (size_t)sub_layout(W, cc.ag, cc.bg, D).total * 4;
    size_t per = (size_t)dfs_words(W, k) * 4;
    int nw = cc.nw;
    // fewer warps when that lets two CTAs share an SM and keeps at least
    // half of them (more resident warps per SM in total)
    const size_t half = kSmemHalf;
    const int nw2 = half > sub ? (int)((half - sub) / per) : 0;
    if (nw2 < nw && 2 * nw2 >= nw) nw = nw2;
    while (nw > 1 && sub + nw * per > kSmemCap) nw--;
    return nw;
}
int class_warps(int c, uint32_t k) { return class_warps(c, k, kClass[c].W, 32 * kClass[c].W); }

size_t class_smem(int c, uint32_t k, uint32_t W, uint32_t D) {
    const ClassCfg &cc = kClass[c];
    if (!cc.cta) return (size_t)cc.nw * (sub_layout(cc.W, false, false).total + dfs_words(cc.W, k)) * 4;
    return ((size_t)sub_layout(W, cc.ag, cc.bg, D).total + (size_t)class_warps(c, k, W, D) * dfs_words(W, k)) * 4;
}
size_t class_smem(int c, uint32_t k) { return class_smem(c, k, kClass[c].W, 32 * kClass[c].W); }

// Arena slices per SM of a class whose rows spill: two for the class that
// keeps B in shared memory (two CTAs may then share an SM), one for the
// largest classes (A and B in the arena).
uint32_t arena_slices_per_sm(int c) { return (kClass[c].ag && !kClass[c].bg) ? 2u : 1u; }

size_t class_arena_per_cta(int c) {
    const ClassCfg &cc = kClass[c];
    const size_t rows_a = (size_t)32 * cc.W * a_stride(cc.W), rows_b = (size_t)32 * cc.W * b_stride(cc.W);
    return (cc.ag ? rows_a : 0) + (cc.bg ? rows_b : 0);
}

template <int WT, bool LIST>
void launch_warp(uint32_t k, Workspace &w, uint32_t begin, uint32_t end, unsigned *q, const Emit &em,
                 unsigned long long *per_root, int wpb, size_t smem, int num_sms, cudaStream_t s) {
    auto kern = k_bitcol_warp<WT, LIST>;
    int occ = 0;
    if (!allow_max_smem(kern) ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, wpb * 32, smem) != cudaSuccess)
        (void)cudaGetLastError();
    if (occ < 1) occ = 1;
    uint32_t blocks = (uint32_t)num_sms * occ;
    uint32_t need = (end - begin + wpb - 1) / wpb;
    if (blocks > need) blocks = need;
    kern<<<blocks, wpb * 32, smem, s>>>(k, w.optr, w.oadj, w.roots, begin, end, q, em, per_root, w.res);
}

template <int NW, bool LIST, bool AG, bool BG>
void launch_cta(uint32_t k, uint32_t W, uint32_t D, int nw, Workspace &w, uint32_t begin, uint32_t end,
                unsigned *q, const Emit &em, unsigned long long *per_root, size_t smem,
                uint32_t blocks, int num_sms, cudaStream_t s) {
    auto kern = k_bitcol_cta<NW, LIST, AG, BG>;
    int occ = 0;
    if (!allow_max_smem(kern) ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, nw * 32, smem) != cudaSuccess)
        (void)cudaGetLastError();
    if (occ < 1) occ = 1;
    uint32_t cap = (uint32_t)num_sms * occ;
    if (blocks > cap) blocks = cap;
    kern<<<blocks, nw * 32, smem, s>>>(k, W, D, w.optr, w.oadj, w.roots, begin, end, q, w.arena, em,
                                       per_root, w.res);
}

}  // namespace

size_t bitcol_colours_arena_words(uint32_t d) {
    const uint32_t W = (((d + 31) >> 5) + 3) & ~3u, D = (d + 31) & ~31u;
    const SubLay L = sub_layout(W, true, true, D);
    return (size_t)L.D * L.WP + (size_t)L.D * L.WPB;
}

int launch_bitcol_colours(const Workspace &w, uint32_t u, uint32_t d, uint32_t *arena,
                          uint32_t *out_nbr, uint32_t *out_colour, cudaStream_t s) {
    const uint32_t W = (((d + 31) >> 5) + 3) & ~3u, D = (d + 31) & ~31u;
    const size_t smem = (size_t)sub_layout(W, true, true, D).total * 4;
    auto kern = k_bitcol_colours<8>;
    if (!allow_max_smem(kern) || smem > (size_t)max_dynamic_smem()) return -1;
    kern<<<1, 256, smem, s>>>(W, D, w.optr, w.oadj, u, arena, out_nbr, out_colour);
    return 1;
}

int bitcol_classes(uint32_t *limits, int max) {
    int n = kNumClasses < max ? kNumClasses : max;
    for (int i = 0; i < n; i++) limits[i] = 32 * kClass[i].W;
    return n;
}

// CTAs that hold an arena slice are capped at one per SM.
size_t bitcol_arena_words(uint32_t k, int num_sms, uint32_t max_outdeg) {
    (void)k;
    size_t need = 0;
    for (int c = 0; c < kNumClasses; c++) {
        if (c > 0 && 32 * kClass[c - 1].W >= max_outdeg) break;
        size_t words = class_arena_per_cta(c) * (size_t)num_sms * arena_slices_per_sm(c);
        if (words > need) need = words;
    }
    return need;
}

int launch_bitcol(const kcl_graph *g, uint32_t k, Workspace &w, const uint32_t *class_begin,
                  int n_classes, const ListArgs &la, cudaStream_t s) {
    // class c covers root positions [class_begin[c], c ? class_begin[c-1] : n_roots)
    Emit em{la.ring, la.capacity, la.wrap, la.per_root_cks, la.idmap,
            (g->options & KCL_OPT_NO_COLOR_PRUNE) ? 0u : 1u, 0u, w.slots, 0u, w.kmap};
    int launches = 0;
    cudaMemsetAsync(w.queue, 0, 64 * sizeof(unsigned), s);
    for (int c = 0; c < n_classes; c++) {
        const uint32_t begin = class_begin[c];
        const uint32_t end = c ? class_begin[c - 1] : class_begin[n_classes];
        if (end <= begin) continue;
        const ClassCfg &cc = kClass[c];
        unsigned *q = w.queue + c;
        em.dfs_warps = g->tuning.bitcol_cta_warps[c];
        em.split = 0;
        if (cc.cta && g->tuning.bitcol_split[c]) {
            em.split = g->tuning.bitcol_split[c];
            cudaMemsetAsync(w.slots, 0xFF, kMaxSplitSlots * sizeof(unsigned long long), s);
        }
        uint32_t Wl = cc.W, Dl = 32 * cc.W;
        if (cc.cta) class_layout(c, la.max_outdeg, &Wl, &Dl);
        const size_t smem = cc.cta ? class_smem(c, k, Wl, Dl) : class_smem(c, k);
        class_mark(la, c, 0, s);
        if (!cc.cta && la.listing) {
            // listing: every clique is hashed one by one, so a root's cost grows
            // with its clique count; a CTA of 4 warps shares each root's
            // first-level children (counting keeps one warp per root)
            const size_t sm4 = ((size_t)sub_layout(cc.W, false, false).total + 4 * dfs_words(cc.W, k)) * 4;
            uint32_t blocks = (uint32_t)g->num_sms * 8;
            if (blocks > end - begin) blocks = end - begin;
            launch_cta<4, true, false, false>(k, cc.W, 32 * cc.W, 4, w, begin, end, q, em, la.per_root,
                                              sm4, blocks, g->num_sms, s);
        } else if (!cc.cta) {
#define KCL_W(WV)                                                                              \
    if (la.listing) launch_warp<WV, true>(k, w, begin, end, q, em, la.per_root, cc.nw, smem, g->num_sms, s); \
    else launch_warp<WV, false>(k, w, begin, end, q, em, la.per_root, cc.nw, smem, g->num_sms, s);
            if (cc.W == 1) { KCL_W(1) }
            else if (cc.W == 2) { KCL_W(2) }
            else { KCL_W(4) }
#undef KCL_W
        } else {
            uint32_t blocks = (cc.ag || cc.bg) ? (uint32_t)g->num_sms * arena_slices_per_sm(c)
                                               : (uint32_t)g->num_sms * 4;
            // without splitting, CTAs beyond the number of roots would idle
            if (!em.split && blocks > end - begin) blocks = end - begin;
            if (blocks > kMaxSplitSlots) blocks = kMaxSplitSlots;
            const int nw = class_warps(c, k, Wl, Dl);
#define KCL_C(NWV, AGV, BGV)                                                                          \
    if (la.listing) launch_cta<NWV, true, AGV, BGV>(k, Wl, Dl, nw, w, begin, end, q, em, la.per_root, smem, blocks, g->num_sms, s); \
    else launch_cta<NWV, false, AGV, BGV>(k, Wl, Dl, nw, w, begin, end, q, em, la.per_root, smem, blocks, g->num_sms, s);
            if (cc.nw == 8) { KCL_C(8, false, false) }
            else if (cc.nw == 16 && !cc.ag) { KCL_C(16, false, false) }
            else if (cc.nw == 16) { KCL_C(16, true, false) }
            else if (cc.nw == 4) { KCL_C(4, true, true) }
            else { KCL_C(2, true, true) }
#undef KCL_C
        }
        class_mark(la, c, 1, s);
        launches++;
    }
    return launches;
}

}  // namespace kcl
