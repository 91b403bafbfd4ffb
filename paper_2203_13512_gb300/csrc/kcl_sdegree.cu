// SDegree on the GPU (Algorithm 5, Section VI): for every root u of the
// degree-ordered DAG with d+_u >= k-1, one warp runs SDegreeList(k-1, {u},
// N+_u) as an explicit-stack DFS over sorted candidate lists:
//   for each v in C: skip v when d+_v <= l-2 (degree prune);
//                    C' = N+_v intersect C;
//                    l = 2: every w in C' closes a clique R + {v, w};
//                    else recurse on C' when |C'| > l-2.
// The intersection is warp-cooperative: the shorter of the two sorted lists
// is streamed 32 elements at a time (coalesced), each lane binary-searches its
// element in the other list, and a ballot compacts the matches in ascending
// order -- the GPU form of the merge join that the paper vectorises with
// 128-bit SIMD compares (Section VI-C).  Candidate lists live on a per-warp
// stack in shared memory (a global arena for very large out-degrees).
#include "kcl_internal.cuh"

namespace kcl {

namespace {

constexpr unsigned kFull = 0xffffffffu;

struct SLay {
    uint32_t D, LISTS, POS, SIZE, PATH, SORTED, total;
};

__host__ __device__ inline SLay make_slayout(uint32_t D, uint32_t k) {
    SLay L;
    L.D = D;
    L.LISTS = 0;
    L.POS = (k - 1) * D;
    L.SIZE = L.POS + k;
    L.PATH = L.SIZE + k;
    L.SORTED = L.PATH + k;
    L.total = (L.SORTED + 32 + 3) & ~3u;
    return L;
}

struct Emit {
    uint32_t *ring;
    unsigned long long capacity;
    int wrap;
    unsigned long long *root_cks;  // listing: per-root checksum sums, or null
    const uint32_t *idmap;         // listing: vertex -> output id, or null (identity)
    unsigned long long *slots;     // CTA form: work-splitting slots (one per CTA)
    uint32_t split;                // CTA form: help a root with >= split children left (0 = off)
    const uint8_t *kmap;           // batches: k of each root's graph (null: the launch's k)
};

// lower_bound of x in a sorted list
__device__ __forceinline__ bool contains(const uint32_t *a, uint32_t n, uint32_t x) {
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        uint32_t m = (lo + hi) >> 1;
        if (a[m] < x) lo = m + 1; else hi = m;
    }
    return lo < n && a[lo] == x;
}

// Emit the cliques R + {v, w} for the lanes holding a match w (listing mode).
// sortedR holds R (k-2 ids, ascending).
__device__ void emit_matches(bool found, uint32_t w, uint32_t v, uint32_t k, const uint32_t *sortedR,
                             const Emit &em, DevResult *res, unsigned long long &cks) {
    const unsigned lane = lane_id();
    unsigned m = __ballot_sync(kFull, found);
    if (!m) return;
    unsigned long long slot0 = 0;
    if (em.ring) {
        if (lane == 0)
            slot0 = ring_base(atomicAdd(&res->emitted, (unsigned long long)__popc(m)), em.capacity, em.wrap);
        slot0 = __shfl_sync(kFull, slot0, 0);
    }
    if (!found) return;
    if (em.idmap) {
        v = em.idmap[v];
        w = em.idmap[w];
    }
    cks += clique_hash2(sortedR, k - 2, v, w, hash_seed(k),
                        ring_rec(em.ring, em.capacity, em.wrap, slot0, __popc(m & ((1u << lane) - 1u)), k));
}

// C' = N+_v intersect C; writes C' (ascending) to `out` when non-null and
// returns |C'|.  In listing mode with `leaf`, emits each clique.
template <bool LIST>
__device__ uint32_t intersect(const uint32_t *C, uint32_t nC, const uint32_t *__restrict__ Nv,
                              uint32_t dv, uint32_t *out, bool leaf, uint32_t v, uint32_t k,
                              const uint32_t *sortedR, const Emit &em, DevResult *res,
                              unsigned long long &cks) {
    const unsigned lane = lane_id();
    uint32_t nout = 0;
    if (nC == 0 || dv == 0) return 0;
    const uint32_t clo = C[0], chi = C[nC - 1];
    if (dv <= nC) {
        // stream N+_v, search in C
        for (uint32_t s = 0; s < dv; s += 32) {
            uint32_t i = s + lane;
            bool f = false;
            uint32_t x = 0;
            if (i < dv) {
                x = Nv[i];
                f = x >= clo && x <= chi && contains(C, nC, x);
            }
            unsigned m = __ballot_sync(kFull, f);
            if (out && f) out[nout + __popc(m & ((1u << lane) - 1u))] = x;
            if (LIST && leaf) emit_matches(f, x, v, k, sortedR, em, res, cks);
            nout += __popc(m);
            if (__shfl_sync(kFull, x, 31) > chi && s + 32 < dv) break;  // past C's range
        }
    } else {
        // stream C, search in N+_v
        const uint32_t nlo = Nv[0], nhi = Nv[dv - 1];
        for (uint32_t s = 0; s < nC; s += 32) {
            uint32_t i = s + lane;
            bool f = false;
            uint32_t x = 0;
            if (i < nC) {
                x = C[i];
                f = x >= nlo && x <= nhi && contains(Nv, dv, x);
            }
            unsigned m = __ballot_sync(kFull, f);
            if (out && f) out[nout + __popc(m & ((1u << lane) - 1u))] = x;
            if (LIST && leaf) emit_matches(f, x, v, k, sortedR, em, res, cks);
            nout += __popc(m);
        }
    }
    return nout;
}

template <bool LIST>
__device__ void sdegree_root(uint32_t u, uint32_t k, uint32_t D, const uint32_t *__restrict__ optr,
                             const uint32_t *__restrict__ oadj, uint32_t *S, const Emit &em,
                             DevResult *res, unsigned long long &cnt, unsigned long long &cks) {
    const SLay L = make_slayout(D, k);
    const unsigned lane = lane_id();
    uint32_t *lists = S + L.LISTS;
    uint32_t *pos = S + L.POS;
    uint32_t *size = S + L.SIZE;
    uint32_t *path = S + L.PATH;
    uint32_t *sortedR = S + L.SORTED;
    const uint32_t base = optr[u];
    const uint32_t d = optr[u + 1] - base;
    for (uint32_t i = lane; i < d; i += 32) lists[i] = oadj[base + i];
    if (lane == 0) { pos[0] = 0; size[0] = d; path[0] = u; }
    __syncwarp();
    const unsigned long long deadline = __ldcg(&res->deadline_ns);
    int depth = 0;
    while (depth >= 0) {
        if (warp_past_deadline(deadline, res)) return;
        const uint32_t l = k - 1 - (uint32_t)depth;
        const uint32_t *C = lists + depth * D;
        const uint32_t nC = size[depth];
        const uint32_t p = pos[depth];
        if (p >= nC) { depth--; continue; }
        const uint32_t v = C[p];
        __syncwarp();
        if (lane == 0) pos[depth] = p + 1;
        const uint32_t vb = optr[v];
        const uint32_t dv = optr[v + 1] - vb;
        if (dv + 2 <= l) { __syncwarp(); continue; }  // d+_v <= l-2
        if (l == 2) {
            if (LIST && lane == 0) {
                // R = path[0..depth] (original ids), sorted
                for (uint32_t t = 0; t <= (uint32_t)depth; t++) {
                    uint32_t x = em.idmap ? em.idmap[path[t]] : path[t], j = t;
                    while (j > 0 && sortedR[j - 1] > x) { sortedR[j] = sortedR[j - 1]; j--; }
                    sortedR[j] = x;
                }
            }
            __syncwarp();
            uint32_t np = intersect<LIST>(C, nC, oadj + vb, dv, nullptr, true, v, k, sortedR, em,
                                          res, cks);
            if (lane == 0) cnt += np;  // |C'| is uniform across the warp
            __syncwarp();
        } else {
            uint32_t *out = lists + (depth + 1) * D;
            uint32_t np = intersect<LIST>(C, nC, oadj + vb, dv, out, false, v, k, sortedR, em, res,
                                          cks);
            __syncwarp();
            if (np + 2 > l) {  // |C'| > l-2
                if (lane == 0) { pos[depth + 1] = 0; size[depth + 1] = np; path[depth + 1] = v; }
                __syncwarp();
                depth++;
            }
        }
    }
}

// ------------------------------------------------------------------------
// SDegreeList on out-lists reduced to N+_u (the out-neighbour reduction of
// Section VII-B, which the paper motivates by the comparisons SDegree wastes
// on vertices outside N+_u).  Vertices of N+_u get local indices in
// ascending id order; L(i) = N+_{v_i} intersect N+_u as a sorted list of local
// indices.  The DFS then intersects short sorted lists:
//   - lanes evaluate the candidates of a node in parallel, each merging its
//     L(w) with C (block merge join, 4 x 4 compares per step, stopping early
//     once the size bound is met);
//   - the chosen child's C' = L(v) intersect C is materialised warp-
//     cooperatively (lanes stream the shorter list, binary-search the other,
//     ballot-compact the matches in order).
// The degree prune uses |L(v)| (the out-degree inside G_u), which is at most
// the global d+_v, so it prunes at least as much and never drops a clique.
// Roots with d+ <= 128 run one warp each with everything in shared memory;
// larger ones one CTA each: the CTA builds the lists once and deals the
// root's first-level children to its warps.

// Every reduced list is stored from an 8-byte boundary and padded with
// 0xFFFF to a multiple of 4 entries, so the merge join can take the paper's
// SIMD form (Section VI-C, Example 5): load a block of 4 entries from each
// list, compare all 16 pairs, and advance the block whose last entry is
// smaller (both when equal).

constexpr uint16_t kPad = 0xFFFF;  // above every local index (< 1024)

__host__ __device__ inline uint32_t round4(uint32_t x) { return (x + 3) & ~3u; }

// Listing: (candidate, match) pairs waiting to be hashed, per warp.
constexpr uint32_t kEmitBuf = 256;

__host__ __device__ inline uint32_t stack_words(uint32_t cap, uint32_t k, bool list) {
    // clist and pend: (k-2) lists of round4(cap) u16 each; csize, npend,
    // ppos, path: k words each; sortedR: 32 words; listing: the pair buffer
    return (2 * ((k - 2) * round4(cap) / 2) + 4 * k + 32 + (list ? kEmitBuf : 0u) + 3) & ~3u;
}

// Warp-per-root layout (words): build scratch, directed bit-rows, lists, one
// DFS stack with list capacity D.
struct LLay {
    uint32_t D, WPD, NBR, LOFS, PRE, RS, HK, HV, LEN, RK, BITS, LADJ, STACK, total;
};

__host__ __device__ inline LLay make_llayout(uint32_t D, uint32_t k, bool list) {
    LLay L;
    L.D = D;
    uint32_t w = D / 32;
    L.WPD = (w & 1) ? w : w + 1;
    uint64_t emax = (uint64_t)D * (D - 1) / 2 + 3 * (uint64_t)D;  // padded lists
    L.NBR = 0;
    L.LOFS = D;
    L.PRE = L.LOFS + D + 1;   // prefix sums of the members' out-degrees
    L.RS = L.PRE + D + 1;     // row starts of the members' out-lists
    L.HK = L.RS + D;                    // hash keys (hash_cap(D))
    L.HV = L.HK + hash_cap(D);          // hash values, u16 (hash_cap(D))
    L.LEN = L.HV + hash_cap(D) / 2;     // list lengths, u16 (D)
    L.RK = L.LEN + D / 2;     // DAG rank of each member, u16 (D)
    L.BITS = L.RK + D / 2;    // directed bit-rows (D x WPD)
    L.LADJ = (L.BITS + D * L.WPD + 3) & ~3u;
    L.STACK = (L.LADJ + (uint32_t)((emax + 1) / 2) + 3) & ~3u;
    L.total = (L.STACK + stack_words(D, k, list) + 3) & ~3u;
    return L;
}

// One block step of a merge join of padded u16 lists: all 16 pairs of the
// 4-entry blocks x (from a) and y (from b) compared.  Entries are distinct
// within a list, so each a_t meets at most one b entry; a padding entry never
// counts (it may meet padding in b).  Returns the matches; *adv_a / *adv_b
// say which block to advance (the one with the smaller last entry, or both).
__device__ __forceinline__ uint32_t block_step4(uint2 x, uint2 y, bool *adv_a, bool *adv_b) {
    const uint32_t a0 = x.x & 0xFFFFu, a1 = x.x >> 16, a2 = x.y & 0xFFFFu, a3 = x.y >> 16;
    const uint32_t b0 = y.x & 0xFFFFu, b1 = y.x >> 16, b2 = y.y & 0xFFFFu, b3 = y.y >> 16;
    uint32_t c = (a0 != kPad) & ((a0 == b0) | (a0 == b1) | (a0 == b2) | (a0 == b3));
    c += (a1 != kPad) & ((a1 == b0) | (a1 == b1) | (a1 == b2) | (a1 == b3));
    c += (a2 != kPad) & ((a2 == b0) | (a2 == b1) | (a2 == b2) | (a2 == b3));
    c += (a3 != kPad) & ((a3 == b0) | (a3 == b1) | (a3 == b2) | (a3 == b3));
    *adv_a = a3 <= b3;
    *adv_b = b3 <= a3;
    return c;
}

// |a intersect b| for padded u16 lists (8-byte aligned, lengths na, nb),
// block form: one 8-byte load per list per step, all 16 pairs compared, the
// block with the smaller last entry advanced; stops once `stop` is met.
__device__ __forceinline__ uint32_t merge_count4(const uint16_t *a, uint32_t na, const uint16_t *b,
                                                 uint32_t nb, uint32_t stop) {
    const uint2 *A = reinterpret_cast<const uint2 *>(a);
    const uint2 *B = reinterpret_cast<const uint2 *>(b);
    const uint32_t na4 = (na + 3) >> 2, nb4 = (nb + 3) >> 2;
    uint32_t i = 0, j = 0, c = 0;
    while (i < na4 && j < nb4 && c < stop) {
        bool ai, bj;
        c += block_step4(A[i], B[j], &ai, &bj);
        i += ai;
        j += bj;
    }
    return c;
}

__device__ __forceinline__ bool contains16(const uint16_t *a, uint32_t n, uint32_t x) {
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        uint32_t m = (lo + hi) >> 1;
        if (a[m] < x) lo = m + 1; else hi = m;
    }
    return lo < n && a[lo] == x;
}

// Warp-cooperative C' = a intersect b (sorted u16 lists) written to out and
// padded to a multiple of 4 entries.
__device__ uint32_t warp_intersect16(const uint16_t *a, uint32_t na, const uint16_t *b, uint32_t nb,
                                     uint16_t *out) {
    const unsigned lane = lane_id();
    if (na > nb) {
        const uint16_t *t = a; a = b; b = t;
        uint32_t tn = na; na = nb; nb = tn;
    }
    uint32_t nout = 0;
    if (na > 0) {
        const uint32_t blo = b[0], bhi = b[nb - 1];
        for (uint32_t s = 0; s < na; s += 32) {
            uint32_t i = s + lane;
            bool f = false;
            uint32_t x = 0;
            if (i < na) {
                x = a[i];
                f = x >= blo && x <= bhi && contains16(b, nb, x);
            }
            unsigned m = __ballot_sync(kFull, f);
            if (f) out[nout + __popc(m & ((1u << lane) - 1u))] = (uint16_t)x;
            nout += __popc(m);
        }
    }
    if (lane < round4(nout) - nout) out[nout + lane] = kPad;
    return nout;
}

// A built reduced subproblem and one warp's DFS stack.
struct LView {
    const uint32_t *nbr;   // local index -> original id
    const uint32_t *lofs;  // list offsets (u16 units, multiples of 4)
    const uint16_t *len;   // list lengths
    const uint16_t *ladj;  // reduced out-lists, ascending local indices, padded
    uint32_t d, u, k;
    uint32_t gallop;       // leaf form threshold (kcl_tuning.sdegree_gallop); 0 = merges
    unsigned long long deadline;  // time limit (global timer, ns; 0 = none)
    __device__ __forceinline__ uint32_t deg(uint32_t i) const { return len[i]; }
    __device__ __forceinline__ const uint16_t *list(uint32_t i) const { return ladj + lofs[i]; }
};

struct LStack {
    uint16_t *clist, *pend;  // (k-2) lists of cap entries each
    uint32_t *csize, *npend, *ppos, *path, *sortedR;
    uint32_t *ebuf;          // listing: kEmitBuf (candidate << 16 | match) pairs
    uint32_t cap;            // a multiple of 4
};

__device__ inline LStack stack_ptrs(uint32_t *S, uint32_t cap, uint32_t k, bool list) {
    LStack st;
    st.cap = round4(cap);
    uint32_t lw = (k - 2) * st.cap / 2;
    st.clist = reinterpret_cast<uint16_t *>(S);
    st.pend = reinterpret_cast<uint16_t *>(S + lw);
    st.csize = S + 2 * lw;
    st.npend = st.csize + k;
    st.ppos = st.npend + k;
    st.path = st.ppos + k;
    st.sortedR = st.path + k;
    st.ebuf = list ? st.sortedR + 32 : nullptr;
    return st;
}

// Lower-bound search of x in the sorted list a[0..n) by power-of-two steps
// (the same number of steps for every x, so lanes searching one list stay
// converged); true when x is present.
__device__ __forceinline__ bool search16(const uint16_t *a, uint32_t n, uint32_t x) {
    uint32_t lo = 0;
    for (uint32_t step = n ? 1u << (31 - __clz(n)) : 0u; step; step >>= 1)
        if (lo + step <= n && a[lo + step - 1] < x) lo += step;
    return lo < n && a[lo] == x;
}

// Pairs lane, lane + 32, ... of st.ebuf, into records of the same offsets
// from slot0.
template <int NR>
__device__ __forceinline__ void flush_walk(const LView &v, uint32_t nb, const LStack &st,
                                           const Emit &em, unsigned long long slot0,
                                           unsigned long long &cks) {
    const unsigned lane = lane_id();
    CliqueOut<NR> co;
    co.init(st.sortedR, v.k, em.ring, em.capacity, em.wrap, slot0, lane);
    for (uint32_t e = lane; e < nb; e += 32) {
        const uint32_t pr = st.ebuf[e];
        cks += co.put(v.nbr[pr >> 16], v.nbr[pr & 0xFFFFu]);
    }
}

// Listing: hash the nb (candidate << 16 | match) pairs of st.ebuf with all
// lanes; each pair closes the clique R + {candidate, match}.
__device__ void flush_pairs(const LView &v, uint32_t nb, const LStack &st, const Emit &em,
                            DevResult *res, unsigned long long &cks) {
    const unsigned lane = lane_id();
    const uint32_t k = v.k;
    __syncwarp();
    unsigned long long slot0 = 0;
    if (em.ring) {
        if (lane == 0) slot0 = ring_base(atomicAdd(&res->emitted, (unsigned long long)nb), em.capacity, em.wrap);
        slot0 = __shfl_sync(kFull, slot0, 0);
    }
    switch (k) {  // warp-uniform: R in registers for the common k
        case 3: flush_walk<1>(v, nb, st, em, slot0, cks); break;
        case 4: flush_walk<2>(v, nb, st, em, slot0, cks); break;
        case 5: flush_walk<3>(v, nb, st, em, slot0, cks); break;
        case 6: flush_walk<4>(v, nb, st, em, slot0, cks); break;
        default: flush_walk<0>(v, nb, st, em, slot0, cks);
    }
    __syncwarp();
}

// Leaf (l = 2): every candidate w = C[i], i in [b0, b1), closes
// |L(w) intersect C| cliques.  Local indices follow the DAG order, so L(w)
// holds only indices above w and only C[i+1..] can meet it.  Two forms of
// the intersections, chosen per leaf by their estimated cost:
//   galloping: the pairs (i, t), t > i, are spread over the lanes 32 at a
//     time and lane (i, t) searches C[t] in L(C[i]) -- every lane busy,
//     |C|^2/2 searches of log |L| steps;
//   merging: lane i merges L(C[i]) with C[i+1..] in 4 x 4 blocks -- sum of
//     (|L| + |C|)/4 steps per lane, lanes of unequal length.
// depth = number of path entries below the root.
template <bool LIST>
__device__ void lleaf(const LView &v, const uint16_t *C, uint32_t nC, uint32_t b0, uint32_t b1,
                      uint32_t depth, const LStack &st, const Emit &em, DevResult *res,
                      unsigned long long &cnt, unsigned long long &cks) {
    const unsigned lane = lane_id();
    const uint32_t jend = b1 < nC ? b1 : (nC ? nC - 1 : 0);  // rows with a non-empty suffix
    if (b0 >= jend) return;
    if (LIST) {
        if (lane == 0) {
            st.sortedR[0] = v.u;
            for (uint32_t t = 1; t <= depth; t++) {
                uint32_t x = v.nbr[st.path[t]], j = t;
                while (j > 0 && st.sortedR[j - 1] > x) { st.sortedR[j] = st.sortedR[j - 1]; j--; }
                st.sortedR[j] = x;
            }
        }
        __syncwarp();
    }
    // cost estimate: merge ~ (sum |L| + pairs) element steps, galloping
    // ~ pairs searches of lg steps; the tuned threshold weighs the two
    bool gallop = false;
    if (v.gallop) {
        uint32_t lsum = 0;
        for (uint32_t i = b0 + lane; i < jend; i += 32) lsum += v.deg(C[i]);
        lsum = __reduce_add_sync(kFull, lsum);
        const uint64_t rows = jend - b0;
        const uint64_t pairs = rows * (2ull * nC - b0 - jend - 1) / 2;
        const uint32_t lg = 32 - __clz((lsum / (uint32_t)rows) | 1u);
        gallop = pairs * (6ull * lg + 10) * 10 < (lsum + pairs) * (uint64_t)v.gallop;
    }
    if (gallop) {
        uint32_t j = b0, t = b0 + 1 + lane;
        while (j < jend && t >= nC) { t = t - nC + j + 2; j++; }
        uint32_t nbuf = 0;
        for (;;) {
            const bool valid = j < jend;
            if (!__any_sync(kFull, valid)) break;
            bool found = false;
            uint32_t w = 0, x = 0;
            if (valid) {
                w = C[j];
                x = C[t];
                found = search16(v.list(w), v.deg(w), x);
            }
            cnt += found;
            if (LIST) {
                const unsigned m = __ballot_sync(kFull, found);
                if (found) st.ebuf[nbuf + __popc(m & ((1u << lane) - 1u))] = (w << 16) | x;
                nbuf += __popc(m);
                if (nbuf > kEmitBuf - 32) {
                    flush_pairs(v, nbuf, st, em, res, cks);
                    nbuf = 0;
                }
            }
            t += 32;
            while (j < jend && t >= nC) { t = t - nC + j + 2; j++; }
        }
        if (LIST && nbuf) flush_pairs(v, nbuf, st, em, res, cks);
        return;
    }
    for (uint32_t s = b0; s < jend; s += 32) {
        const uint32_t i = s + lane;
        uint32_t x = 0, w = 0;
        if (i < jend) {
            w = C[i];
            const uint32_t dw = v.deg(w);
            const uint32_t q = (i + 1) & ~3u;
            if (dw) x = merge_count4(v.list(w), dw, C + q, nC - q, 0xFFFFFFFFu);
        }
        cnt += x;
        if (LIST) {
            // rounds of kEmitBuf cliques: every lane resumes its merge and
            // writes its next matches as (candidate, match) pairs at its
            // prefix position in the round's window; all lanes then hash them
            const uint32_t incl = warp_incl_scan(x);
            const uint32_t excl = incl - x;
            const uint32_t tot = __shfl_sync(kFull, incl, 31);
            const uint16_t *a = v.list(w);
            uint32_t ia = 0, ib = i + 1, m = 0;
            for (uint32_t base = 0; base < tot; base += kEmitBuf) {
                const uint32_t lim = base + kEmitBuf;
                while (m < x && excl + m < lim) {
                    const uint32_t p = a[ia], q = C[ib];
                    if (p == q) st.ebuf[excl + m - base] = (w << 16) | p, m++;
                    ia += p <= q;
                    ib += q <= p;
                }
                const uint32_t nb = tot - base < kEmitBuf ? tot - base : kEmitBuf;
                flush_pairs(v, nb, st, em, res, cks);
            }
        }
    }
}

// Inner node at level l: the positions i of the pending children w = C[i],
// those with |L(w) intersect C[i+1..]| >= l-1 (a child needs l-1 more
// vertices, all after it in the DAG order, so the last l-1 entries of C never
// qualify).
__device__ uint32_t lexpand(const LView &v, const uint16_t *C, uint32_t nC, uint32_t l, uint16_t *P) {
    const unsigned lane = lane_id();
    uint32_t np = 0;
    const uint32_t lim = nC + 1 >= l ? nC + 1 - l : 0;  // positions i with nC - i - 1 >= l - 1
    for (uint32_t s = 0; s < lim; s += 32) {
        uint32_t i = s + lane;
        bool ok = false;
        if (i < lim) {
            const uint32_t w = C[i];
            const uint32_t dw = v.deg(w);
            const uint32_t q = (i + 1) & ~3u;
            ok = dw + 1 >= l && merge_count4(v.list(w), dw, C + q, nC - q, l - 1) + 1 >= l;
        }
        unsigned m = __ballot_sync(kFull, ok);
        if (ok) P[np + __popc(m & ((1u << lane) - 1u))] = (uint16_t)i;
        np += __popc(m);
    }
    return np;
}

// The subtree below first-level child p0 (C1 = L(p0)), run by one warp.
template <bool LIST>
__device__ void ldfs_child(const LView &v, uint32_t p0, const LStack &st, const Emit &em,
                           DevResult *res, unsigned long long &cnt, unsigned long long &cks) {
    const unsigned lane = lane_id();
    const uint32_t k = v.k, cap = st.cap;
    const uint16_t *C1 = v.list(p0);
    const uint32_t n1 = v.deg(p0);
    if (lane == 0) { st.path[1] = p0; st.csize[1] = n1; }
    __syncwarp();
    if (k - 2 == 2) {
        lleaf<LIST>(v, C1, n1, 0, n1, 1, st, em, res, cnt, cks);
        __syncwarp();
        return;
    }
    uint32_t np = lexpand(v, C1, n1, k - 2, st.pend);
    if (lane == 0) { st.npend[1] = np; st.ppos[1] = 0; }
    __syncwarp();
    int depth = 1;
    while (depth >= 1) {
        if (warp_past_deadline(v.deadline, res)) return;
        const uint32_t pp = st.ppos[depth];
        if (pp >= st.npend[depth]) { depth--; continue; }
        const uint32_t pos = st.pend[(depth - 1) * cap + pp];
        const uint16_t *C = depth == 1 ? C1 : st.clist + (depth - 2) * cap;
        const uint32_t w = C[pos];
        __syncwarp();
        if (lane == 0) { st.ppos[depth] = pp + 1; st.path[depth + 1] = w; }
        uint16_t *Cn = st.clist + (depth - 1) * cap;  // list of depth + 1
        const uint32_t nn =
            warp_intersect16(v.list(w), v.deg(w), C + pos + 1, st.csize[depth] - pos - 1, Cn);
        if (lane == 0) st.csize[depth + 1] = nn;
        __syncwarp();
        const uint32_t l = k - 2 - (uint32_t)depth;  // level of the child
        if (l == 2) {
            lleaf<LIST>(v, Cn, nn, 0, nn, depth + 1, st, em, res, cnt, cks);
            __syncwarp();
        } else if (nn + 1 >= l) {
            uint32_t np2 = lexpand(v, Cn, nn, l, st.pend + depth * cap);
            if (lane == 0) { st.npend[depth + 1] = np2; st.ppos[depth + 1] = 0; }
            __syncwarp();
            depth++;
        }
    }
}

// Warp per root (d+ <= 128): bit-row build in shared memory, padded lists,
// then the root's children in turn.
// ------------------------------------- bit-row form of SDegreeList
// For dense subproblems the reduced out-lists take more room than the
// directed bit-rows of the same DAG (16 bits per edge against 1 bit per
// pair), and lists that spill to global memory are slow to merge.  The CTA
// form can then run SDegreeList on the bit-rows instead: C is a bitmap over
// the local indices, C' = N+_v intersect C is one AND per word, |C'| a POPC,
// and the degree prune and size tests are the same as with lists.  Local
// indices follow the DAG order, so row(v) holds only indices above v and the
// AND for candidate v starts at v's 4-word chunk.
struct BView {
    const uint32_t *R;    // bit-rows, stride WP words
    const uint32_t *ids;  // local index -> output id
    uint32_t d, W, WP, u, k;  // W: words per row
    unsigned long long deadline;  // time limit (global timer, ns; 0 = none)
};

__host__ __device__ inline uint32_t bstack_words(uint32_t W, uint32_t k) {
    // C and P per depth (2 k W), path and cursor (2 k), sortedR (32), queue (32)
    return (k * (2 * W + 2) + 64 + 3) & ~3u;
}

// |row(q) & C|; C is zero beyond its W words and row(q) below q's word.
// Rows of a multiple of 4 words on a 16-byte stride are read as 128-bit
// vectors from q's chunk on; narrow rows (the warp form) word by word.
__device__ __forceinline__ uint32_t brow_and(const BView &v, uint32_t q, const uint32_t *C) {
    uint32_t x = 0;
    if (((v.W | v.WP) & 3u) == 0) {
        const uint4 *r4 = reinterpret_cast<const uint4 *>(v.R + q * v.WP);
        const uint4 *c4 = reinterpret_cast<const uint4 *>(C);
        for (uint32_t t = q >> 7; t < (v.W >> 2); t++) {
            const uint4 a = r4[t], b = c4[t];
            x += __popc(a.x & b.x) + __popc(a.y & b.y) + __popc(a.z & b.z) + __popc(a.w & b.w);
        }
    } else {
        const uint32_t *row = v.R + q * v.WP;
        for (uint32_t t = q >> 5; t < v.W; t++) x += __popc(row[t] & C[t]);
    }
    return x;
}

// A lane's run of rlen cliques within a bit-row leaf batch (as BitCol's
// leaf_walk): its first clique is set bit `rank` of row(q[o]) & C.
template <int NR>
__device__ __forceinline__ void bleaf_walk(const BView &v, const uint32_t *C, const uint16_t *q,
                                           uint32_t o, uint32_t rank, uint32_t rlen,
                                           const uint32_t *sortedR, const Emit &em,
                                           unsigned long long slot0, unsigned long long &cks) {
    CliqueOut<NR> co;
    co.init(sortedR, v.k, em.ring, em.capacity, em.wrap, slot0, lane_id());
    uint32_t qo = q[o];
    const uint32_t *row = v.R + qo * v.WP;
    uint32_t a = v.ids[qo];
    uint32_t t = qo >> 5, mm = 0;
    for (; t < v.W; t++) {
        mm = row[t] & C[t];
        const uint32_t c = __popc(mm);
        if (rank < c) break;
        rank -= c;
    }
    for (uint32_t z = 0; z < rank; z++) mm &= mm - 1;
    for (uint32_t r = 0; r < rlen; r++) {
        const uint32_t b = t * 32 + (__ffs(mm) - 1);
        cks += co.put(a, v.ids[b]);
        mm &= mm - 1;
        while (!mm && r + 1 < rlen) {
            if (++t >= v.W) {  // next candidate with cliques
                qo = q[++o];
                row = v.R + qo * v.WP;
                a = v.ids[qo];
                t = qo >> 5;
            }
            mm = row[t] & C[t];
        }
    }
}

// Leaf (l = 2) on bitmap C: every candidate q in C closes |row(q) & C|
// cliques; candidates are packed 32 to a batch (queue of 64 u16).
template <bool LIST>
__device__ void bleaf_batch(const BView &v, const uint32_t *C, const uint16_t *q, uint32_t nb,
                            const uint32_t *sortedR, const Emit &em, DevResult *res,
                            unsigned long long &cnt, unsigned long long &cks) {
    const unsigned lane = lane_id();
    uint32_t x = lane < nb ? brow_and(v, q[lane], C) : 0u;
    cnt += x;
    if (!LIST) return;
    // the tot cliques of the batch, in (candidate, bit) order, are cut into
    // 32 contiguous runs, one per lane; a lane finds its first clique once
    // and walks the set bits from there (as in BitCol's leaf)
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
    uint32_t o = 0;
#pragma unroll
    for (uint32_t step = 16; step > 0; step >>= 1) {
        const uint32_t vv = __shfl_sync(kFull, incl, o + step - 1);
        if (vv <= r0) o += step;
    }
    const uint32_t eo = __shfl_sync(kFull, excl, o & 31u);
    if (rlen == 0) return;
    switch (v.k) {  // warp-uniform: R in registers for the common k
        case 3: bleaf_walk<1>(v, C, q, o, r0 - eo, rlen, sortedR, em, slot0, cks); break;
        case 4: bleaf_walk<2>(v, C, q, o, r0 - eo, rlen, sortedR, em, slot0, cks); break;
        case 5: bleaf_walk<3>(v, C, q, o, r0 - eo, rlen, sortedR, em, slot0, cks); break;
        case 6: bleaf_walk<4>(v, C, q, o, r0 - eo, rlen, sortedR, em, slot0, cks); break;
        default: bleaf_walk<0>(v, C, q, o, r0 - eo, rlen, sortedR, em, slot0, cks);
    }
}

template <bool LIST>
__device__ void bleaf(const BView &v, const uint32_t *C, uint32_t depth, const uint32_t *path,
                      uint32_t *sortedR, const Emit &em, DevResult *res, unsigned long long &cnt,
                      unsigned long long &cks) {
    const unsigned lane = lane_id();
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
    uint32_t pend = 0;
    for (uint32_t j = 0; j < v.W; j++) {
        const uint32_t m = C[j];
        if (!m) continue;
        if ((m >> lane) & 1u) q[pend + __popc(m & ((1u << lane) - 1u))] = (uint16_t)(j * 32 + lane);
        pend += __popc(m);
        if (pend >= 32) {
            __syncwarp();
            bleaf_batch<LIST>(v, C, q, 32, sortedR, em, res, cnt, cks);
            __syncwarp();
            if (lane < pend - 32) q[lane] = q[32 + lane];
            pend -= 32;
            __syncwarp();
        }
    }
    if (pend) {
        __syncwarp();
        bleaf_batch<LIST>(v, C, q, pend, sortedR, em, res, cnt, cks);
        __syncwarp();
    }
}

// Inner node at level l on bitmap C: P = the candidates q with
// |row(q) & C| >= l-1.
__device__ void bexpand(const BView &v, const uint32_t *C, uint32_t l, uint32_t *P) {
    const unsigned lane = lane_id();
    for (uint32_t j = 0; j < v.W; j++) {
        const uint32_t m = C[j];
        bool ok = false;
        if ((m >> lane) & 1u) ok = brow_and(v, j * 32 + lane, C) + 1 >= l;
        const unsigned bal = __ballot_sync(kFull, ok);
        if (lane == 0) P[j] = bal;
    }
    __syncwarp();
}

// A batch of nb <= 32 (child, candidate) pairs of a level-3 node (counting
// on bit-rows): lane i takes pq[i] = (p << 16) | q and closes
// |row(q) & row(p) & C| cliques.  Rows lie above their vertex, so the batch
// reads a uniform range of words from its smallest q on.
__device__ __forceinline__ void bpair_batch(const BView &v, const uint32_t *C, const uint32_t *pq,
                                            uint32_t nb, uint32_t &acc) {
    const unsigned lane = lane_id();
    const uint32_t e = pq[lane < nb ? lane : nb - 1];
    const uint32_t p = e >> 16, q = e & 0xFFFFu;
    const uint32_t qmin = __reduce_min_sync(kFull, q);
    uint32_t x = 0;
    if (((v.W | v.WP) & 3u) == 0) {
        const uint4 *a4 = reinterpret_cast<const uint4 *>(v.R + q * v.WP);
        const uint4 *b4 = reinterpret_cast<const uint4 *>(v.R + p * v.WP);
        const uint4 *c4 = reinterpret_cast<const uint4 *>(C);
#pragma unroll 2
        for (uint32_t t = qmin >> 7; t < (v.W >> 2); t++) {
            const uint4 a = a4[t], b = b4[t], c = c4[t];
            x += __popc(a.x & b.x & c.x) + __popc(a.y & b.y & c.y) + __popc(a.z & b.z & c.z) +
                 __popc(a.w & b.w & c.w);
        }
    } else {
        const uint32_t *rq = v.R + q * v.WP, *rp = v.R + p * v.WP;
        for (uint32_t t = qmin >> 5; t < v.W; t++) x += __popc(rq[t] & rp[t] & C[t]);
    }
    acc += lane < nb ? x : 0u;
}

// Runs full batches while the queue holds 32 pairs or more (pend <= 64).
__device__ __forceinline__ void bpair_drain(const BView &v, const uint32_t *C, uint32_t *pq,
                                            uint32_t &pend, uint32_t &acc) {
    const unsigned lane = lane_id();
    while (pend >= 32) {
        __syncwarp();
        bpair_batch(v, C, pq, 32, acc);
        __syncwarp();
        if (lane < pend - 32) pq[lane] = pq[32 + lane];
        pend -= 32;
        __syncwarp();
    }
}

// Counting below a level-3 node on bit-rows (Algorithm 5 at levels 3 and 2):
// for every pending child p and every q in row(p) & C, |row(q) & row(p) & C|
// cliques close.  All (p, q) pairs go through the per-warp queue pq (64
// entries), 32 to a batch, so no child materialises its C'.  With 16-byte
// rows the scan reads four words at a time (a row is zero below its
// vertex, so the chunk may start below it) and queues their pairs in one
// step when they fit.  The per-lane sum stays 32-bit within the node: at
// most d^2 / 32 pairs of at most d cliques per lane, and the rows (d^2 / 8
// bytes) sit in shared memory, so d < 2048 and the sum stays below 2^28.
__device__ void bleaf_pairs(const BView &v, const uint32_t *C, const uint32_t *P, uint32_t *pq,
                            unsigned long long &cnt) {
    const unsigned lane = lane_id();
    const unsigned lt = (1u << lane) - 1u, me = 1u << lane;
    const bool vec = ((v.W | v.WP) & 3u) == 0;
    uint32_t pend = 0, acc = 0;
    for (uint32_t jp = 0; jp < v.W; jp++) {
        uint32_t pw = P[jp];
        while (pw) {
            const uint32_t p = jp * 32 + (__ffs(pw) - 1);
            pw &= pw - 1;
            const uint32_t *rowp = v.R + p * v.WP;
            for (uint32_t t0 = vec ? ((p >> 5) & ~3u) : (p >> 5); t0 < v.W; t0 += vec ? 4u : 1u) {
                uint32_t mw[4] = {0u, 0u, 0u, 0u};
                if (vec) {
                    const uint4 a = *reinterpret_cast<const uint4 *>(rowp + t0);
                    const uint4 c = *reinterpret_cast<const uint4 *>(C + t0);
                    mw[0] = a.x & c.x; mw[1] = a.y & c.y; mw[2] = a.z & c.z; mw[3] = a.w & c.w;
                } else {
                    mw[0] = rowp[t0] & C[t0];
                }
                const uint32_t c0 = __popc(mw[0]), c1 = __popc(mw[1]), c2 = __popc(mw[2]),
                               c3 = __popc(mw[3]);
                const uint32_t tot = c0 + c1 + c2 + c3;
                const uint32_t b0 = (p << 16) | (t0 * 32 + lane);
                if (pend + tot <= 64) {
                    const uint32_t o1 = pend + c0, o2 = o1 + c1, o3 = o2 + c2;
                    if (mw[0] & me) pq[pend + __popc(mw[0] & lt)] = b0;
                    if (mw[1] & me) pq[o1 + __popc(mw[1] & lt)] = b0 + 32;
                    if (mw[2] & me) pq[o2 + __popc(mw[2] & lt)] = b0 + 64;
                    if (mw[3] & me) pq[o3 + __popc(mw[3] & lt)] = b0 + 96;
                    pend += tot;
                    bpair_drain(v, C, pq, pend, acc);
                } else {  // dense words: one at a time (each adds at most 32)
#pragma unroll 1
                    for (int z = 0; z < 4; z++) {
                        const uint32_t m = mw[z];
                        if (m & me) pq[pend + __popc(m & lt)] = b0 + 32 * z;
                        pend += __popc(m);
                        bpair_drain(v, C, pq, pend, acc);
                    }
                }
            }
        }
    }
    if (pend) {
        __syncwarp();
        bpair_batch(v, C, pq, pend, acc);
        __syncwarp();
    }
    cnt += acc;
}

// The subtree below first-level child p0 (C1 = row(p0)), one warp.
template <bool LIST>
__device__ void bdfs_child(const BView &v, uint32_t p0, uint32_t *stack, const Emit &em,
                           DevResult *res, unsigned long long &cnt, unsigned long long &cks) {
    const unsigned lane = lane_id();
    const uint32_t W = v.W, k = v.k;
    uint32_t *Cst = stack;
    uint32_t *Pst = Cst + k * W;
    uint32_t *path = Pst + k * W;
    uint32_t *cur = path + k;
    uint32_t *sortedR = cur + k;
    for (uint32_t t = lane; t < W; t += 32) Cst[W + t] = v.R[p0 * v.WP + t];
    if (lane == 0) path[1] = p0;
    __syncwarp();
    if (k - 2 == 2) {
        bleaf<LIST>(v, Cst + W, 1, path, sortedR, em, res, cnt, cks);
        return;
    }
    bexpand(v, Cst + W, k - 2, Pst + W);
    if (!LIST && k - 2 == 3) {  // sortedR and the leaf queue (64 words) hold the pair queue
        bleaf_pairs(v, Cst + W, Pst + W, sortedR, cnt);
        __syncwarp();
        return;
    }
    if (lane == 0) cur[1] = 0;
    __syncwarp();
    int depth = 1;
    while (depth >= 1) {
        if (warp_past_deadline(v.deadline, res)) return;
        uint32_t *P = Pst + depth * W;
        uint32_t j = cur[depth];
        while (j < W && P[j] == 0) j++;
        if (j >= W) { depth--; continue; }
        const uint32_t pw = P[j];
        const uint32_t p = j * 32 + (__ffs(pw) - 1);
        __syncwarp();
        if (lane == 0) { P[j] = pw & (pw - 1); cur[depth] = j; path[depth + 1] = p; }
        const uint32_t *C = Cst + depth * W;
        uint32_t *Cn = Cst + (depth + 1) * W;
        for (uint32_t t = lane; t < W; t += 32) Cn[t] = v.R[p * v.WP + t] & C[t];
        __syncwarp();
        const uint32_t lc = k - 2 - (uint32_t)depth;  // level of the child
        if (lc == 2) {
            bleaf<LIST>(v, Cn, depth + 1, path, sortedR, em, res, cnt, cks);
            __syncwarp();
        } else if (!LIST && lc == 3) {
            bexpand(v, Cn, 3, Pst + (depth + 1) * W);
            bleaf_pairs(v, Cn, Pst + (depth + 1) * W, sortedR, cnt);
            __syncwarp();
        } else {
            bexpand(v, Cn, lc, Pst + (depth + 1) * W);
            if (lane == 0) cur[depth + 1] = 0;
            __syncwarp();
            depth++;
        }
    }
}

// Rank of member i of N+_u (ascending ids nbr[]) in the DAG order (key, id):
// members with a smaller key, plus earlier members with the same key.
__device__ __forceinline__ uint32_t dag_rank(const uint32_t *keys, uint32_t d, uint32_t i) {
    const uint32_t ki = keys[i];
    uint32_t r = 0;
    for (uint32_t j = 0; j < d; j++) {
        const uint32_t kj = keys[j];
        r += (kj < ki) | ((kj == ki) & (j < i));
    }
    return r;
}

template <bool LIST>
__device__ void sdegree_root_local(uint32_t u, uint32_t k, uint32_t D, const uint32_t *__restrict__ optr,
                                   const uint32_t *__restrict__ oadj, const uint32_t *__restrict__ key,
                                   uint32_t *S, const Emit &em, DevResult *res, uint32_t gallop,
                                   uint32_t bitmap, unsigned long long &cnt, unsigned long long &cks) {
    const LLay L = make_llayout(D, k, LIST);
    const unsigned lane = lane_id();
    uint32_t *nbr = S + L.NBR;
    uint32_t *lofs = S + L.LOFS;
    uint32_t *pre = S + L.PRE;
    uint32_t *rs = S + L.RS;
    uint32_t *hk = S + L.HK;
    uint16_t *hv = reinterpret_cast<uint16_t *>(S + L.HV);
    uint16_t *len = reinterpret_cast<uint16_t *>(S + L.LEN);
    uint16_t *rk = reinterpret_cast<uint16_t *>(S + L.RK);
    uint32_t *bits = S + L.BITS;
    uint16_t *ladj = reinterpret_cast<uint16_t *>(S + L.LADJ);
    const LStack st = stack_ptrs(S + L.STACK, D, k, LIST);

    const uint32_t base = optr[u];
    const uint32_t d = optr[u + 1] - base;
    uint32_t running = 0;
    for (uint32_t c0 = 0; c0 < d; c0 += 32) {
        uint32_t i = c0 + lane, x = 0;
        if (i < d) {
            uint32_t v = oadj[base + i];
            nbr[i] = v;
            uint32_t r0 = optr[v];
            rs[i] = r0;
            x = optr[v + 1] - r0;
            lofs[i] = key[v];  // keys until the list offsets are laid out
        }
        uint32_t incl = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(kFull, incl, o);
            if (lane >= (unsigned)o) incl += y;
        }
        if (i < d) pre[i] = running + incl - x;
        running += __shfl_sync(kFull, incl, 31);
    }
    for (uint32_t i = lane; i < d * L.WPD; i += 32) bits[i] = 0;
    if (lane == 0) pre[d] = running;
    __syncwarp();
    const uint32_t total = running;
    const uint32_t lo_id = nbr[0], hi_id = nbr[d - 1];
    // local index = rank in the DAG order, so every reduced out-list L(i)
    // holds only indices above i
    for (uint32_t i = lane; i < d; i += 32) rk[i] = (uint16_t)dag_rank(lofs, d, i);
    __syncwarp();

    // directed bit-rows: the members' out-lists are streamed as one flattened
    // sequence; a hash probe into N+_u finds the local index of each entry
    uint32_t T, hshift;
    hash_size(d, &T, &hshift);
    warp_hash_build(nbr, d, hk, hv, T, hshift);
    uint32_t a0 = 0;
    for (uint32_t c = 0; c < total; c += 32) {
        const uint32_t e = c + lane;
        uint32_t a = a0;
        if (e < total) {
            while (pre[a + 1] <= e) a++;
            uint32_t x = oadj[rs[a] + (e - pre[a])];
            if (x >= lo_id && x <= hi_id) {
                int j = hash_find(hk, hv, T, hshift, x);
                if (j >= 0) {
                    const uint32_t jr = rk[j];
                    atomicOr(&bits[rk[a] * L.WPD + (jr >> 5)], 1u << (jr & 31));
                }
            }
        }
        a0 = __shfl_sync(kFull, a, 31);
    }
    __syncwarp();
    // member ids by local index (rs is free after the build)
    for (uint32_t i = lane; i < d; i += 32) rs[rk[i]] = nbr[i];
    __syncwarp();
    // lengths -> padded offsets -> lists in ascending order
    running = 0;
    for (uint32_t c0 = 0; c0 <= d; c0 += 32) {
        uint32_t i = c0 + lane, x = 0;
        if (i < d) {
            uint32_t c = 0;
            for (uint32_t t = 0; t < L.WPD; t++) c += __popc(bits[i * L.WPD + t]);
            len[i] = (uint16_t)c;
            x = round4(c);
        }
        uint32_t incl = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(kFull, incl, o);
            if (lane >= (unsigned)o) incl += y;
        }
        if (i <= d) lofs[i] = running + incl - x;
        running += __shfl_sync(kFull, incl, 31);
    }
    __syncwarp();
    // bit-row form when the lists would take more than threshold/16 of the
    // rows' room (the rows are already built, in shared memory)
    const uint32_t thr = bitmap ? bitmap : 16u;
    const bool bitrows = k > 3 && bitmap != 0xFFFFFFFFu &&
                         16ull * (lofs[d] / 2) > (unsigned long long)thr * (d * L.WPD);
    for (uint32_t i = bitrows ? d : lane; i < d; i += 32) {
        uint32_t o = lofs[i];
        for (uint32_t t = 0; t < L.WPD; t++) {
            uint32_t m = bits[i * L.WPD + t];
            while (m) {
                ladj[o++] = (uint16_t)(t * 32 + (__ffs(m) - 1));
                m &= m - 1;
            }
        }
        while (o < lofs[i + 1]) ladj[o++] = kPad;
    }
    __syncwarp();

    if (LIST && em.idmap) {  // output ids (batched unions map back to each graph's ids)
        for (uint32_t i = lane; i < d; i += 32) rs[i] = em.idmap[rs[i]];
        __syncwarp();
    }
    const LView v{rs, lofs, len, ladj, d, (LIST && em.idmap) ? em.idmap[u] : u, k, gallop,
                  __ldcg(&res->deadline_ns)};
    if (bitrows) {
        const BView bv{bits, rs, d, (d + 31) >> 5, L.WPD, v.u, k, v.deadline};
        for (uint32_t w = 0; w < d; w++)
            if (v.deg(w) + 2 >= k) bdfs_child<LIST>(bv, w, S + L.STACK, em, res, cnt, cks);
        return;
    }
    if (k == 3) {
        // C = all of N+_u: every edge of the reduced DAG closes a triangle
        if (!LIST) {
            uint32_t c = 0;
            for (uint32_t i = lane; i < d; i += 32) c += len[i];
            cnt += c;
            return;
        }
        for (uint32_t i = lane; i < round4(d); i += 32) st.clist[i] = i < d ? (uint16_t)i : kPad;
        __syncwarp();
        lleaf<LIST>(v, st.clist, d, 0, d, 0, st, em, res, cnt, cks);
        return;
    }
    // depth 0: C = all local indices, so |L(w) intersect C| = |L(w)|
    for (uint32_t w = 0; w < d; w++)
        if (v.deg(w) + 2 >= k) ldfs_child<LIST>(v, w, st, em, res, cnt, cks);
}

// ------------------------------------------------ CTA per root (d+ > 128)
// Shared region (words) of the CTA form; the reduced lists and the per-warp
// stacks follow it in shared memory (lists move to the global arena when
// they do not leave room for enough warps).
struct CLay {
    uint32_t D, WPD, NBR, RS, PRE, LOFS, HK, HV, LEN, RK, P0, META, total;
};

// Above 512 vertices the build's hash table lives in the CTA's arena slice
// (it is dead once the rows are built), leaving shared memory to the rows,
// lists and stacks of the DFS.
__host__ __device__ inline bool cta_hash_global(uint32_t D) { return D > 512; }

__host__ __device__ inline CLay make_clayout(uint32_t D) {
    CLay L;
    L.D = D;
    uint32_t w = D / 32;
    L.WPD = (w & 1) ? w : w + 1;
    L.NBR = 0;
    L.RS = L.NBR + D;
    L.PRE = L.RS + D;          // D + 1
    L.LOFS = L.PRE + D + 1;    // D + 1
    const uint32_t hw = cta_hash_global(D) ? 0u : hash_cap(D) + hash_cap(D) / 2;
    L.HK = L.LOFS + D + 1;              // hash_cap(D) (when in shared memory)
    L.HV = L.HK + hash_cap(D);          // hash_cap(D) u16
    L.LEN = L.LOFS + D + 1 + hw;        // D u16: list lengths
    L.RK = L.LEN + D / 2;      // D u16: DAG rank of each member
    L.P0 = L.RK + D / 2;       // D u16: first-level children
    L.META = L.P0 + D / 2;     // 16 words
    L.total = (L.META + 16 + 3) & ~3u;
    return L;
}

// arena slice per CTA: directed bit-rows (D x WPD words) + padded lists
// (+ the hash table above 512 vertices)
__host__ __device__ inline size_t cta_arena_hash_offset(uint32_t D) {
    CLay L = make_clayout(D);
    size_t rows = ((size_t)D * L.WPD + 3) & ~(size_t)3;
    size_t lists = ((size_t)D * (D - 1) / 2 + 3 * (size_t)D + 1) / 2;
    return (rows + lists + 3) & ~(size_t)3;
}

__host__ __device__ inline size_t cta_arena_words(uint32_t D) {
    size_t words = cta_arena_hash_offset(D);
    if (cta_hash_global(D)) words += ((size_t)hash_cap(D) + hash_cap(D) / 2 + 3) & ~(size_t)3;
    return words;
}

template <bool LIST>
__global__ void __launch_bounds__(512) k_sdegree_cta(uint32_t kmax, uint32_t D, const uint32_t *__restrict__ optr,
                                                    const uint32_t *__restrict__ oadj,
                                                    const uint32_t *__restrict__ key,
                                                    const uint32_t *__restrict__ roots, uint32_t begin,
                                                    uint32_t end, unsigned *queue, uint32_t *arena,
                                                    uint32_t smem_words, Emit em, uint32_t gallop,
                                                    uint32_t bitmap, uint32_t dfs_warps,
                                                    unsigned long long *per_root, DevResult *res) {
    extern __shared__ uint32_t smem[];
    const CLay L = make_clayout(D);
    const uint32_t tid = threadIdx.x, nth = blockDim.x, lane = lane_id(), warp = tid >> 5;
    const uint32_t nwarps = nth >> 5;
    uint32_t *nbr = smem + L.NBR;
    uint32_t *rs = smem + L.RS;
    uint32_t *pre = smem + L.PRE;
    uint32_t *lofs = smem + L.LOFS;
    uint16_t *len = reinterpret_cast<uint16_t *>(smem + L.LEN);
    uint16_t *rk = reinterpret_cast<uint16_t *>(smem + L.RK);
    uint16_t *p0 = reinterpret_cast<uint16_t *>(smem + L.P0);
    uint32_t *meta = smem + L.META;
    uint32_t *slice = arena + (size_t)blockIdx.x * cta_arena_words(D);
    uint32_t *hk = cta_hash_global(D) ? slice + cta_arena_hash_offset(D) : smem + L.HK;
    uint16_t *hv = reinterpret_cast<uint16_t *>(cta_hash_global(D) ? hk + hash_cap(D) : smem + L.HV);
    uint32_t *bits = slice;
    uint16_t *ladj_g = reinterpret_cast<uint16_t *>(slice + (((size_t)D * L.WPD + 3) & ~(size_t)3));
    unsigned long long cnt = 0, cks = 0;
    __shared__ int help_slot;  // -1: own root from the queue; else the slot of the root helped
    unsigned long long *my_slot = em.slots + blockIdx.x;
    bool queue_done = false;
    const unsigned long long deadline = __ldcg(&res->deadline_ns);
    for (;;) {
        if (tid == 0) {  // thread 0 alone reads the timer
            if (!queue_done && past_deadline(deadline, res)) queue_done = true;
            meta[15] = queue_done ? end - begin : atomicAdd(queue, 1u);
            help_slot = (queue_done && deadline && global_ns() > deadline) ? -2 : -1;
        }
        __syncthreads();
        uint32_t idx = meta[15];
        const bool late = help_slot == -2;
        int helping = -1;
        __syncthreads();  // every thread has read meta[15] and help_slot before they are rewritten
        if (idx >= end - begin) {
            queue_done = true;
            // no root left: help the root with the most children left
            if (!em.split || kmax == 3 || late) break;
            if (warp == 0) {
                uint32_t pos = 0;
                const int j = split_pick(em.slots, gridDim.x, blockIdx.x, em.split, &pos);
                if (lane == 0) { help_slot = j; meta[15] = pos; }
            }
            __syncthreads();
            helping = help_slot;
            idx = meta[15];
            if (helping < 0 || idx >= end - begin) break;
        }
        unsigned long long *slot = helping >= 0 ? em.slots + helping : my_slot;
        const uint32_t u = roots[begin + idx];
        const uint32_t k = em.kmap ? (uint32_t)em.kmap[u] : kmax;
        const uint32_t base = optr[u], d = optr[u + 1] - base;
        const unsigned long long before = cnt;
        const unsigned long long before_cks = cks;

        // ---- build: members, out-list lengths, hash of N+_u, zero bit-rows
        for (uint32_t i = tid; i < d; i += nth) {
            uint32_t x = oadj[base + i];
            nbr[i] = x;
            uint32_t r0 = optr[x];
            rs[i] = r0;
            pre[i] = optr[x + 1] - r0;
            lofs[i] = key[x];  // keys until the list offsets are laid out
        }
        uint32_t T, hshift;
        hash_size(d, &T, &hshift);
        for (uint32_t i = tid; i < T; i += nth) hk[i] = kHashEmpty;
        for (uint32_t i = tid; i < d * L.WPD; i += nth) bits[i] = 0;
        if (tid < 15) meta[tid] = 0;  // meta[15] holds the root index
        __syncthreads();
        if (warp == 0) {
            uint32_t running = 0;
            for (uint32_t c0 = 0; c0 < d; c0 += 32) {
                uint32_t i = c0 + lane;
                uint32_t x = i < d ? pre[i] : 0;
                uint32_t incl = x;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    uint32_t y = __shfl_up_sync(kFull, incl, o);
                    if (lane >= (unsigned)o) incl += y;
                }
                if (i < d) pre[i] = running + incl - x;
                running += __shfl_sync(kFull, incl, 31);
            }
            if (lane == 0) pre[d] = running;
        }
        // local index = rank in the DAG order, so every reduced out-list L(i)
        // holds only indices above i; the hash maps an id to its rank
        for (uint32_t i = tid; i < d; i += nth) {
            const uint32_t r = dag_rank(lofs, d, i);
            rk[i] = (uint16_t)r;
            uint32_t id = nbr[i], h = hash_slot(id, hshift);
            while (atomicCAS(&hk[h], kHashEmpty, id) != kHashEmpty) h = (h + 1) & (T - 1);
            hv[h] = (uint16_t)r;
        }
        __syncthreads();
        // ---- directed bit-rows: bit j of row i iff member j is in N+_{v_i}
        const uint32_t total = pre[d];
        const uint32_t lo_id = nbr[0], hi_id = nbr[d - 1];
        uint32_t a0 = 0;
        for (uint32_t c = warp * 32; c < total; c += nth) {
            uint32_t lo = a0, hi = d;
            while (hi - lo > 1) {
                uint32_t m = (lo + hi) >> 1;
                if (pre[m] <= c) lo = m; else hi = m;
            }
            a0 = lo;
            const uint32_t e = c + lane;
            if (e < total) {
                uint32_t a = a0;
                while (pre[a + 1] <= e) a++;
                uint32_t x = oadj[rs[a] + (e - pre[a])];
                if (x >= lo_id && x <= hi_id) {
                    int j = hash_find(hk, hv, T, hshift, x);
                    if (j >= 0) atomicOr(&bits[rk[a] * L.WPD + ((uint32_t)j >> 5)], 1u << (j & 31));
                }
            }
        }
        __syncthreads();
        // member ids by local index (rs is free after the build)
        for (uint32_t i = tid; i < d; i += nth) rs[rk[i]] = nbr[i];
        // ---- row lengths, longest row, padded offsets
        for (uint32_t i = tid; i < d; i += nth) {
            uint32_t c = 0;
            for (uint32_t t = 0; t < L.WPD; t++) c += __popc(bits[i * L.WPD + t]);
            len[i] = (uint16_t)c;
            atomicMax(&meta[3], c);
        }
        __syncthreads();
        if (warp == 0) {
            uint32_t running = 0;
            for (uint32_t c0 = 0; c0 <= d; c0 += 32) {
                uint32_t i = c0 + lane;
                uint32_t x = i < d ? round4(len[i]) : 0;
                uint32_t incl = x;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    uint32_t y = __shfl_up_sync(kFull, incl, o);
                    if (lane >= (unsigned)o) incl += y;
                }
                if (i <= d) lofs[i] = running + incl - x;
                running += __shfl_sync(kFull, incl, 31);
            }
            if (lane == 0) {
                // place the lists and size the stacks: lists in shared memory
                // unless that would leave fewer than min(8, possible) warps
                uint32_t cap = meta[3] ? meta[3] : 1;
                uint32_t sw = stack_words(cap, k, LIST);
                uint32_t budget = smem_words - L.total;
                uint32_t lw = (lofs[d] / 2 + 3) & ~3u;
                uint32_t nw_g = budget / sw;
                if (nw_g > nwarps) nw_g = nwarps;
                uint32_t nw_s = lw <= budget ? (budget - lw) / sw : 0;
                if (nw_s > nwarps) nw_s = nwarps;
                uint32_t want = nw_g < 8 ? nw_g : 8;
                bool in_smem = nw_s >= 1 && nw_s >= want;
                meta[4] = in_smem ? 1u : 0u;
                meta[5] = in_smem ? nw_s : nw_g;
                meta[6] = sw;
                meta[7] = in_smem ? lw : 0u;  // stacks start after the lists
                // bit-row form instead, when the rows fit with enough warps
                // and the lists would take more than threshold/16 of their room
                const uint32_t Wb = round4((d + 31) >> 5);
                const uint32_t WPB = ((Wb >> 2) & 1) ? Wb : Wb + 4;
                const uint32_t bw = d * WPB, bsw = bstack_words(Wb, k);
                uint32_t nw_b = bw <= budget ? (budget - bw) / bsw : 0;
                if (nw_b > nwarps) nw_b = nwarps;
                const uint32_t thr = bitmap ? bitmap : 16u;
                if (k > 3 && bitmap != 0xFFFFFFFFu && nw_b >= want && nw_b >= 1 &&
                    16ull * lw > (unsigned long long)thr * bw) {
                    meta[4] = 2u;
                    meta[5] = nw_b;
                    meta[6] = bsw;
                    meta[7] = bw;  // stacks start after the rows
                    meta[10] = Wb;
                    meta[11] = WPB;
                }
            }
        }
        __syncthreads();
        const bool bitrows = meta[4] == 2u;
        uint16_t *ladj = meta[4] == 1u ? reinterpret_cast<uint16_t *>(smem + L.total) : ladj_g;
        if (bitrows) {
            // rows to shared memory, zero beyond the row's words
            const uint32_t Wb = meta[10], WPB = meta[11];
            uint32_t *R = smem + L.total;
            for (uint32_t e = tid; e < d * Wb; e += nth) {
                const uint32_t i = e / Wb, t = e - i * Wb;
                R[i * WPB + t] = t < L.WPD ? bits[i * L.WPD + t] : 0u;
            }
        }
        // ---- extraction: row i's bits in ascending order -> L(i), padded
        for (uint32_t i = bitrows ? d : tid; i < d; i += nth) {
            uint32_t o = lofs[i];
            for (uint32_t t = 0; t < L.WPD; t++) {
                uint32_t m = bits[i * L.WPD + t];
                while (m) {
                    ladj[o++] = (uint16_t)(t * 32 + (__ffs(m) - 1));
                    m &= m - 1;
                }
            }
            while (o < lofs[i + 1]) ladj[o++] = kPad;
        }
        // warps walking the children: as many as fit, unless the tuning caps
        // it (1 = one warp per root)
        const uint32_t nw_dfs = dfs_warps && dfs_warps < meta[5] ? dfs_warps : meta[5];
        const uint32_t sw = meta[6];
        if (nw_dfs == 0 && tid == 0) atomicOr(&res->status, DEV_ERR_INTERNAL);  // no stack fits
        if (LIST && em.idmap)  // output ids (batched unions map back to each graph's ids)
            for (uint32_t i = tid; i < d; i += nth) rs[i] = em.idmap[rs[i]];
        const LView v{rs, lofs, len, ladj, d, (LIST && em.idmap) ? em.idmap[u] : u, k, gallop,
                  __ldcg(&res->deadline_ns)};
        const uint32_t cap = meta[3] ? meta[3] : 1;
        // ---- first-level children (|L(w)| >= k-2), longest lists first
        if (k > 3 && warp == 0) {
            // four passes: |L(w)| in [3/4, inf), [1/2, 3/4), [1/4, 1/2), [0, 1/4) of the longest
            uint32_t n0 = 0, mx = meta[3];
            for (int bucket = 3; bucket >= 0; bucket--) {
                uint32_t lo = bucket == 0 ? 0u : (mx * (uint32_t)bucket) / 4;
                uint32_t hi = bucket == 3 ? 0xFFFFFFFFu : (mx * (uint32_t)(bucket + 1)) / 4;
                for (uint32_t s = 0; s < d; s += 32) {
                    uint32_t w = s + lane;
                    bool ok = false;
                    if (w < d) {
                        uint32_t dw = len[w];
                        ok = dw + 2 >= k && dw >= lo && dw < hi;
                    }
                    unsigned m = __ballot_sync(kFull, ok);
                    if (ok) p0[n0 + __popc(m & ((1u << lane) - 1u))] = (uint16_t)w;
                    n0 += __popc(m);
                }
            }
            if (lane == 0) { meta[8] = n0; meta[9] = 0; }
        }
        if (k == 3 && LIST) {
            for (uint32_t i = tid; i < round4(d); i += nth) p0[i] = i < d ? (uint16_t)i : kPad;
        }
        __syncthreads();
        if (em.split && k > 3) {  // share the children with CTAs that run out of roots
            if (helping < 0 && tid == 0) split_publish(my_slot, idx, meta[8]);
            __syncthreads();
        }
        if (bitrows && warp < nw_dfs) {
            const BView bv{smem + L.total, rs, d, meta[10], meta[11], v.u, k, deadline};
            uint32_t *stack = smem + L.total + meta[7] + warp * sw;
            const uint32_t n0 = meta[8];
            for (;;) {
                uint32_t i = 0;
                if (lane == 0) i = em.split ? split_claim(slot, idx) : atomicAdd(&meta[9], 1u);
                i = __shfl_sync(kFull, i, 0);
                if (i >= n0) break;
                bdfs_child<LIST>(bv, p0[i], stack, em, res, cnt, cks);
            }
        } else if (warp < nw_dfs) {
            const LStack st = stack_ptrs(smem + L.total + meta[7] + warp * sw, cap < d ? cap : d, k, LIST);
            if (k == 3) {
                if (!LIST) {
                    uint32_t c = 0;
                    for (uint32_t i = tid; i < d; i += nw_dfs * 32) c += len[i];
                    cnt += c;
                } else {
                    // identity candidate list, split across the DFS warps
                    uint32_t chunk = (d + nw_dfs - 1) / nw_dfs;
                    uint32_t b0 = warp * chunk, b1 = b0 + chunk < d ? b0 + chunk : d;
                    if (b0 < b1) lleaf<LIST>(v, p0, d, b0, b1, 0, st, em, res, cnt, cks);
                }
            } else {
                const uint32_t n0 = meta[8];
                for (;;) {
                    uint32_t i = 0;
                    if (lane == 0) i = em.split ? split_claim(slot, idx) : atomicAdd(&meta[9], 1u);
                    i = __shfl_sync(kFull, i, 0);
                    if (i >= n0) break;
                    ldfs_child<LIST>(v, p0[i], st, em, res, cnt, cks);
                }
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

template <bool LIST, bool GLOBAL, bool LOCAL>
__global__ void __launch_bounds__(128) k_sdegree(uint32_t kmax, uint32_t D, const uint32_t *__restrict__ optr,
                                                const uint32_t *__restrict__ oadj,
                                                const uint32_t *__restrict__ key,
                                                const uint32_t *__restrict__ roots, uint32_t begin,
                                                uint32_t end, unsigned *queue, uint32_t *arena,
                                                uint32_t words_per_warp, Emit em, uint32_t gallop,
                                                uint32_t bitmap,
                                                unsigned long long *per_root, DevResult *res) {
    extern __shared__ uint32_t smem[];
    const unsigned lane = lane_id();
    const uint32_t wib = threadIdx.x >> 5;
    uint32_t *S = GLOBAL ? arena + (size_t)(blockIdx.x * (blockDim.x >> 5) + wib) * words_per_warp
                         : smem + wib * words_per_warp;
    const unsigned long long deadline = __ldcg(&res->deadline_ns);
    unsigned long long cnt = 0, cks = 0;
    for (;;) {
        if (warp_past_deadline(deadline, res)) break;
        uint32_t idx = 0;
        if (lane == 0) idx = atomicAdd(queue, 1u);
        idx = __shfl_sync(kFull, idx, 0);
        if (idx >= end - begin) break;
        uint32_t u = roots[begin + idx];
        const uint32_t k = em.kmap ? (uint32_t)em.kmap[u] : kmax;
        unsigned long long before = cnt;
        const unsigned long long before_cks = cks;
        if (LOCAL) sdegree_root_local<LIST>(u, k, D, optr, oadj, key, S, em, res, gallop, bitmap, cnt, cks);
        else sdegree_root<LIST>(u, k, D, optr, oadj, S, em, res, cnt, cks);
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

// Out-degree classes: <= 128 warp per root (reduced lists, shared memory);
// <= 1024 CTA per root (reduced lists); above, SDegreeList on the global
// out-lists with a warp per root and its stack in a global arena.
constexpr uint32_t kClassD[] = {32, 64, 128, 256, 512, 1024, 4096, 16384, 65536};
constexpr int kNumClasses = 9;
constexpr int kWarpClasses = 3;
constexpr int kCtaClasses = 6;
constexpr size_t kSmemPerBlock = 96 * 1024;

// Arena slices (resident CTAs) per SM of the CTA form: small subproblems
// (listing mode's small classes) run four CTAs of 128 threads per SM.
uint32_t cta_slices_per_sm(uint32_t D) { return D <= 128 ? 4u : 2u; }

// Shared memory per CTA: up to d+ = 768 two CTAs fit on an SM (dense
// subproblems there take the bit-row form, whose rows are at most 86 KB,
// and above 512 the build's hash table is in the arena); beyond, one CTA
// with room for its rows or lists.
size_t cta_smem_bytes(uint32_t D) {
    return D <= 128 ? 48 * 1024 : D <= 512 ? 100 * 1024 : D <= 768 ? 112 * 1024 : 200 * 1024;
}
int cta_threads(uint32_t D) { return D <= 128 ? 128 : 512; }

template <bool LIST>
void launch_warp_local(uint32_t k, uint32_t D, Workspace &w, uint32_t begin, uint32_t end,
                       unsigned *queue, const Emit &em, unsigned long long *per_root, int num_sms,
                       uint32_t gallop, uint32_t bitmap, cudaStream_t s) {
    uint32_t words = make_llayout(D, k, LIST).total;
    int wpb = (int)(kSmemPerBlock / ((size_t)words * 4));
    if (wpb > 4) wpb = 4;
    if (wpb < 1) wpb = 1;
    size_t smem = (size_t)wpb * words * 4;
    auto kern = k_sdegree<LIST, false, true>;
    int occ = 0;
    if (!allow_max_smem(kern) ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, wpb * 32, smem) != cudaSuccess)
        (void)cudaGetLastError();
    if (occ < 1) occ = 1;
    uint32_t blocks = (uint32_t)num_sms * occ;
    uint32_t need = (end - begin + wpb - 1) / wpb;
    if (blocks > need) blocks = need;
    kern<<<blocks, wpb * 32, smem, s>>>(k, D, w.optr, w.oadj, w.key, w.roots, begin, end, queue,
                                        w.arena, words, em, gallop, bitmap, per_root, w.res);
}

template <bool LIST>
void launch_cta(uint32_t k, uint32_t D, Workspace &w, uint32_t begin, uint32_t end, unsigned *queue,
                const Emit &em, unsigned long long *per_root, int num_sms, uint32_t gallop,
                uint32_t bitmap, uint32_t dfs_warps, cudaStream_t s) {
    size_t smem = cta_smem_bytes(D);
    const int threads = cta_threads(D);
    auto kern = k_sdegree_cta<LIST>;
    int occ = 0;
    if (!allow_max_smem(kern) ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem) != cudaSuccess)
        (void)cudaGetLastError();
    if (occ < 1) occ = 1;
    if (occ > (int)cta_slices_per_sm(D)) occ = (int)cta_slices_per_sm(D);  // arena slices per SM
    uint32_t blocks = (uint32_t)num_sms * occ;
    // without splitting, CTAs beyond the number of roots would idle
    if (!em.split && blocks > end - begin) blocks = end - begin;
    if (blocks > kMaxSplitSlots) blocks = kMaxSplitSlots;
    kern<<<blocks, threads, smem, s>>>(k, D, w.optr, w.oadj, w.key, w.roots, begin, end, queue,
                                       w.arena, (uint32_t)(smem / 4), em, gallop, bitmap, dfs_warps,
                                       per_root, w.res);
}

template <bool LIST>
void launch_global_lists(uint32_t k, uint32_t D, Workspace &w, uint32_t begin, uint32_t end,
                         unsigned *queue, const Emit &em, unsigned long long *per_root, int num_sms,
                         uint32_t gallop, cudaStream_t s) {
    uint32_t words = make_slayout(D, k).total;
    uint32_t blocks = (uint32_t)num_sms;
    if (blocks * 2 > end - begin) blocks = (end - begin + 1) / 2;
    k_sdegree<LIST, true, false><<<blocks, 64, 0, s>>>(k, D, w.optr, w.oadj, w.key, w.roots, begin,
                                                       end, queue, w.arena, words, em, gallop, 0u,
                                                       per_root, w.res);
}

}  // namespace

int sdegree_classes(uint32_t *limits, int max) {
    int n = kNumClasses < max ? kNumClasses : max;
    for (int i = 0; i < n; i++) limits[i] = kClassD[i];
    return n;
}

// Covers every class that may hold roots, including the small classes' CTA
// form used in listing mode.
size_t sdegree_arena_words(uint32_t k, int num_sms, uint32_t max_outdeg) {
    size_t need = 0;
    for (int c = 0; c < kNumClasses; c++) {
        if (c > 0 && kClassD[c - 1] >= max_outdeg) break;
        size_t words = c < kCtaClasses ? (size_t)num_sms * cta_slices_per_sm(kClassD[c]) * cta_arena_words(kClassD[c])
                                       : (size_t)num_sms * 2 * make_slayout(kClassD[c], k).total;
        if (words > need) need = words;
    }
    return need;
}

int launch_sdegree(const kcl_graph *g, uint32_t k, Workspace &w, const uint32_t *class_begin,
                   int n_classes, const ListArgs &la, cudaStream_t s) {
    Emit em{la.ring, la.capacity, la.wrap, la.per_root_cks, la.idmap, w.slots, 0u, w.kmap};
    int launches = 0;
    cudaMemsetAsync(w.queue, 0, 64 * sizeof(unsigned), s);
    for (int c = 0; c < n_classes; c++) {
        uint32_t begin = class_begin[c];
        uint32_t end = c ? class_begin[c - 1] : class_begin[n_classes];
        if (end <= begin) continue;
        // the CTA form is laid out for the class's largest out-degree
        uint32_t D = kClassD[c];
        if (c < kCtaClasses && la.max_outdeg < D) D = (la.max_outdeg + 31) & ~31u;
        if (D < 32) D = 32;
        unsigned *q = w.queue + c;
        const uint32_t gl = la.listing ? g->tuning.sdegree_gallop_list[c] : g->tuning.sdegree_gallop[c];
        const uint32_t bm = g->tuning.sdegree_bitmap[c];
        const uint32_t dw = g->tuning.sdegree_cta_warps[c];
        const int ns = g->num_sms;
        const bool cta_form = c < kCtaClasses && (c >= kWarpClasses || la.listing);
        em.split = cta_form ? g->tuning.sdegree_split[c] : 0u;
        if (em.split) cudaMemsetAsync(w.slots, 0xFF, kMaxSplitSlots * sizeof(unsigned long long), s);
        class_mark(la, c, 0, s);
        if (c < kWarpClasses) {
            // listing hashes every clique: a root's cost grows with its clique
            // count, so listing shares each root's children over a CTA of 4 warps
            if (la.listing) launch_cta<true>(k, D, w, begin, end, q, em, la.per_root, ns, gl, bm, dw, s);
            else launch_warp_local<false>(k, D, w, begin, end, q, em, la.per_root, ns, gl, bm, s);
        } else if (c < kCtaClasses) {
            if (la.listing) launch_cta<true>(k, D, w, begin, end, q, em, la.per_root, ns, gl, bm, dw, s);
            else launch_cta<false>(k, D, w, begin, end, q, em, la.per_root, ns, gl, bm, dw, s);
        } else {
            if (la.listing) launch_global_lists<true>(k, D, w, begin, end, q, em, la.per_root, ns, gl, s);
            else launch_global_lists<false>(k, D, w, begin, end, q, em, la.per_root, ns, gl, s);
        }
        class_mark(la, c, 1, s);
        launches++;
    }
    return launches;
}

}  // namespace kcl
