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
        if (lane == 0) slot0 = atomicAdd(&res->emitted, (unsigned long long)__popc(m));
        slot0 = __shfl_sync(kFull, slot0, 0);
    }
    if (!found) return;
    uint32_t e0 = v < w ? v : w, e1 = v < w ? w : v;
    uint32_t ex[2] = {e0, e1};
    uint32_t rec[KCL_MAX_K];
    uint32_t nr = k - 2, ri = 0, ei = 0, o = 0;
    while (ri < nr || ei < 2) {
        uint32_t r = ri < nr ? sortedR[ri] : 0xFFFFFFFFu;
        if (ei < 2 && ex[ei] < r) rec[o++] = ex[ei++];
        else rec[o++] = sortedR[ri++];
    }
    uint64_t h = hash_seed(k);
    for (uint32_t z = 0; z < k; z++) h = mix64(h ^ (uint64_t)rec[z]);
    cks += h;
    if (em.ring) {
        unsigned long long sl = slot0 + __popc(m & ((1u << lane) - 1u));
        bool ok = true;
        if (em.wrap) sl %= em.capacity;
        else ok = sl < em.capacity;
        if (ok)
            for (uint32_t z = 0; z < k; z++) em.ring[sl * k + z] = rec[z];
    }
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
    int depth = 0;
    while (depth >= 0) {
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
                    uint32_t x = path[t], j = t;
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
// indices.  The DFS then intersects short sorted lists in shared memory:
//   - lanes evaluate the candidates of a node in parallel, each merging its
//     L(w) with C (two-pointer merge join, stopping early once the size
//     bound is met);
//   - the chosen child's C' = L(v) intersect C is materialised warp-
//     cooperatively (lanes stream the shorter list, binary-search the other,
//     ballot-compact the matches in order).
// The degree prune uses |L(v)| (the out-degree inside G_u), which is at most
// the global d+_v, so it prunes at least as much and never drops a clique.
struct LLay {
    uint32_t D, NBR, LOFS, PRE, RS, HK, HV, LADJ, CL, PD, META, SORTED, total;
};

__host__ __device__ inline LLay make_llayout(uint32_t D, uint32_t k) {
    LLay L;
    L.D = D;
    uint64_t emax = (uint64_t)D * (D - 1) / 2;
    L.NBR = 0;
    L.LOFS = D;
    L.PRE = L.LOFS + D + 1;   // prefix sums of the members' out-degrees
    L.RS = L.PRE + D + 1;     // row starts of the members' out-lists
    L.HK = L.RS + D;          // hash keys (2D)
    L.HV = L.HK + 2 * D;      // hash values, u16 (2D)
    L.LADJ = L.HV + D;
    L.CL = L.LADJ + (uint32_t)((emax + 1) / 2);
    L.PD = L.CL + ((k - 1) * D + 1) / 2;
    L.META = L.PD + ((k - 1) * D + 1) / 2;
    L.SORTED = L.META + 4 * k;
    L.total = (L.SORTED + 32 + 3) & ~3u;
    return L;
}

// |a intersect b| for sorted u16 lists, stopping once `stop` is reached.
__device__ __forceinline__ uint32_t merge_count(const uint16_t *a, uint32_t na, const uint16_t *b,
                                                uint32_t nb, uint32_t stop) {
    uint32_t i = 0, j = 0, c = 0;
    while (i < na && j < nb && c < stop) {
        uint32_t x = a[i], y = b[j];
        c += x == y;
        i += x <= y;
        j += y <= x;
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

// Warp-cooperative C' = a intersect b (sorted u16 lists) written to out.
__device__ uint32_t warp_intersect16(const uint16_t *a, uint32_t na, const uint16_t *b, uint32_t nb,
                                     uint16_t *out) {
    const unsigned lane = lane_id();
    if (na > nb) {
        const uint16_t *t = a; a = b; b = t;
        uint32_t tn = na; na = nb; nb = tn;
    }
    uint32_t nout = 0;
    if (na == 0) return 0;
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
    return nout;
}

template <bool LIST>
__device__ void sdegree_root_local(uint32_t u, uint32_t k, uint32_t D, const uint32_t *__restrict__ optr,
                                   const uint32_t *__restrict__ oadj, uint32_t *S, const Emit &em,
                                   DevResult *res, unsigned long long &cnt, unsigned long long &cks) {
    const LLay L = make_llayout(D, k);
    const unsigned lane = lane_id();
    uint32_t *nbr = S + L.NBR;
    uint32_t *lofs = S + L.LOFS;
    uint32_t *pre = S + L.PRE;
    uint32_t *rs = S + L.RS;
    uint32_t *hk = S + L.HK;
    uint16_t *hv = reinterpret_cast<uint16_t *>(S + L.HV);
    uint16_t *ladj = reinterpret_cast<uint16_t *>(S + L.LADJ);
    uint16_t *clist = reinterpret_cast<uint16_t *>(S + L.CL);   // depth t >= 1 at (t-1)*D
    uint16_t *pend = reinterpret_cast<uint16_t *>(S + L.PD);    // depth t at t*D
    uint32_t *csize = S + L.META;
    uint32_t *npend = csize + k;
    uint32_t *ppos = npend + k;
    uint32_t *path = ppos + k;
    uint32_t *sortedR = S + L.SORTED;

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
            lofs[i] = 0;
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
    if (lane == 0) { pre[d] = running; lofs[d] = 0; }
    __syncwarp();
    const uint32_t total = running;
    const uint32_t lo_id = nbr[0], hi_id = nbr[d - 1];

    // ---- reduced out-lists L(i): the members' out-lists are streamed as one
    // flattened sequence; matches (hash probe into N+_u) are ballot-compacted
    // in stream order, so each L(i) is contiguous and ascending.
    uint32_t T, hshift;
    hash_size(d, &T, &hshift);
    warp_hash_build(nbr, d, hk, hv, T, hshift);
    uint32_t run = 0, a0 = 0;
    for (uint32_t c = 0; c < total; c += 32) {
        const uint32_t e = c + lane;
        uint32_t a = a0;
        int j = -1;
        if (e < total) {
            while (pre[a + 1] <= e) a++;
            uint32_t x = oadj[rs[a] + (e - pre[a])];
            if (x >= lo_id && x <= hi_id) j = hash_find(hk, hv, T, hshift, x);
        }
        unsigned m = __ballot_sync(kFull, j >= 0);
        if (j >= 0) {
            ladj[run + __popc(m & ((1u << lane) - 1u))] = (uint16_t)j;
            atomicAdd(&lofs[a], 1u);
        }
        run += __popc(m);
        a0 = __shfl_sync(kFull, a, 31);
    }
    __syncwarp();
    // row counts -> offsets (exclusive scan over d + 1 entries)
    running = 0;
    for (uint32_t c0 = 0; c0 <= d; c0 += 32) {
        uint32_t i = c0 + lane;
        uint32_t x = i <= d ? lofs[i] : 0;
        uint32_t incl = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(kFull, incl, o);
            if (lane >= (unsigned)o) incl += y;
        }
        __syncwarp();
        if (i <= d) lofs[i] = running + incl - x;
        running += __shfl_sync(kFull, incl, 31);
    }
    __syncwarp();

    auto ldeg = [&](uint32_t i) -> uint32_t { return lofs[i + 1] - lofs[i]; };
    auto Lp = [&](uint32_t i) -> const uint16_t * { return ladj + lofs[i]; };

    // leaf (l = 2): every w in C closes |L(w) intersect C| cliques
    auto leaf = [&](const uint16_t *C, uint32_t nC, uint32_t depth) {
        if (LIST && lane == 0) {
            sortedR[0] = u;
            for (uint32_t t = 1; t <= depth; t++) {
                uint32_t x = nbr[path[t]], j = t;
                while (j > 0 && sortedR[j - 1] > x) { sortedR[j] = sortedR[j - 1]; j--; }
                sortedR[j] = x;
            }
        }
        if (LIST) __syncwarp();
        for (uint32_t s = 0; s < nC; s += 32) {
            uint32_t i = s + lane;
            uint32_t x = 0, w = 0;
            if (i < nC) {
                w = C[i];
                uint32_t dw = ldeg(w);
                if (dw) x = merge_count(Lp(w), dw, C, nC, 0xFFFFFFFFu);
            }
            cnt += x;
            if (LIST) {
                // slots for this batch of lanes, then each lane re-merges and emits
                uint32_t incl = x;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    uint32_t y = __shfl_up_sync(kFull, incl, o);
                    if (lane >= (unsigned)o) incl += y;
                }
                uint32_t tot = __shfl_sync(kFull, incl, 31);
                unsigned long long slot0 = 0;
                if (tot && em.ring) {
                    if (lane == 0) slot0 = atomicAdd(&res->emitted, (unsigned long long)tot);
                    slot0 = __shfl_sync(kFull, slot0, 0);
                }
                if (x) {
                    unsigned long long slot = slot0 + (incl - x);
                    const uint16_t *a = Lp(w);
                    uint32_t na = ldeg(w), ia = 0, ib = 0;
                    uint32_t vid = nbr[w];
                    while (ia < na && ib < nC) {
                        uint32_t p = a[ia], q = C[ib];
                        if (p == q) {
                            uint32_t b2 = nbr[p];
                            uint32_t e0 = vid < b2 ? vid : b2, e1 = vid < b2 ? b2 : vid;
                            uint32_t ex[2] = {e0, e1};
                            uint32_t rec[KCL_MAX_K];
                            uint32_t nr = k - 2, ri = 0, ei = 0, o = 0;
                            while (ri < nr || ei < 2) {
                                uint32_t r = ri < nr ? sortedR[ri] : 0xFFFFFFFFu;
                                if (ei < 2 && ex[ei] < r) rec[o++] = ex[ei++];
                                else rec[o++] = sortedR[ri++];
                            }
                            uint64_t h = hash_seed(k);
                            for (uint32_t z = 0; z < k; z++) h = mix64(h ^ (uint64_t)rec[z]);
                            cks += h;
                            if (em.ring) {
                                unsigned long long sl = slot;
                                bool ok = true;
                                if (em.wrap) sl %= em.capacity;
                                else ok = sl < em.capacity;
                                if (ok)
                                    for (uint32_t z = 0; z < k; z++) em.ring[sl * k + z] = rec[z];
                            }
                            slot++;
                        }
                        ia += p <= q;
                        ib += q <= p;
                    }
                }
            }
        }
    };
    // inner node at level l: pending children w with |L(w) intersect C| >= l-1
    auto expand = [&](const uint16_t *C, uint32_t nC, uint32_t l, uint16_t *P) -> uint32_t {
        uint32_t np = 0;
        for (uint32_t s = 0; s < nC; s += 32) {
            uint32_t i = s + lane;
            bool ok = false;
            uint32_t w = 0;
            if (i < nC) {
                w = C[i];
                uint32_t dw = ldeg(w);
                ok = dw + 1 >= l && merge_count(Lp(w), dw, C, nC, l - 1) + 1 >= l;
            }
            unsigned m = __ballot_sync(kFull, ok);
            if (ok) P[np + __popc(m & ((1u << lane) - 1u))] = (uint16_t)w;
            np += __popc(m);
        }
        return np;
    };

    const uint32_t l0 = k - 1;
    if (l0 == 2) {
        // C = all of N+_u: every edge of the reduced DAG closes a triangle
        if (!LIST) {
            if (lane == 0) cnt += lofs[d];
            return;
        }
        // listing: C is the identity list 0..d-1 (built in clist)
        for (uint32_t i = lane; i < d; i += 32) clist[i] = (uint16_t)i;
        __syncwarp();
        leaf(clist, d, 0);
        return;
    }
    // depth 0: C = all local indices, so |L(w) intersect C| = |L(w)|
    {
        uint32_t np = 0;
        for (uint32_t s = 0; s < d; s += 32) {
            uint32_t w = s + lane;
            bool ok = w < d && ldeg(w) + 1 >= l0;
            unsigned m = __ballot_sync(kFull, ok);
            if (ok) pend[np + __popc(m & ((1u << lane) - 1u))] = (uint16_t)w;
            np += __popc(m);
        }
        if (lane == 0) { npend[0] = np; ppos[0] = 0; path[0] = 0; }
        __syncwarp();
    }
    int depth = 0;
    while (depth >= 0) {
        const uint32_t pp = ppos[depth];
        if (pp >= npend[depth]) { depth--; continue; }
        const uint32_t v = pend[depth * D + pp];
        __syncwarp();
        if (lane == 0) { ppos[depth] = pp + 1; path[depth + 1] = v; }
        // child candidate list C' = L(v) intersect C
        uint16_t *Cn = clist + depth * D;  // list of depth + 1
        uint32_t nn;
        if (depth == 0) {
            nn = ldeg(v);
            const uint16_t *a = Lp(v);
            for (uint32_t i = lane; i < nn; i += 32) Cn[i] = a[i];
        } else {
            const uint16_t *C = clist + (depth - 1) * D;
            nn = warp_intersect16(Lp(v), ldeg(v), C, csize[depth], Cn);
        }
        if (lane == 0) csize[depth + 1] = nn;
        __syncwarp();
        const uint32_t l = k - 2 - (uint32_t)depth;  // level of the child
        if (l == 2) {
            leaf(Cn, nn, depth + 1);
            __syncwarp();
        } else if (nn + 1 >= l) {
            uint32_t np = expand(Cn, nn, l, pend + (depth + 1) * D);
            if (lane == 0) { npend[depth + 1] = np; ppos[depth + 1] = 0; }
            __syncwarp();
            depth++;
        }
    }
}

template <bool LIST, bool GLOBAL, bool LOCAL>
__global__ void __launch_bounds__(128) k_sdegree(uint32_t k, uint32_t D, const uint32_t *__restrict__ optr,
                                                const uint32_t *__restrict__ oadj,
                                                const uint32_t *__restrict__ roots, uint32_t begin,
                                                uint32_t end, unsigned *queue, uint32_t *arena,
                                                uint32_t words_per_warp, Emit em,
                                                unsigned long long *per_root, DevResult *res) {
    extern __shared__ uint32_t smem[];
    const unsigned lane = lane_id();
    const uint32_t wib = threadIdx.x >> 5;
    uint32_t *S = GLOBAL ? arena + (size_t)(blockIdx.x * (blockDim.x >> 5) + wib) * words_per_warp
                         : smem + wib * words_per_warp;
    unsigned long long cnt = 0, cks = 0;
    for (;;) {
        uint32_t idx = 0;
        if (lane == 0) idx = atomicAdd(queue, 1u);
        idx = __shfl_sync(kFull, idx, 0);
        if (idx >= end - begin) break;
        uint32_t u = roots[begin + idx];
        unsigned long long before = cnt;
        if (LOCAL) sdegree_root_local<LIST>(u, k, D, optr, oadj, S, em, res, cnt, cks);
        else sdegree_root<LIST>(u, k, D, optr, oadj, S, em, res, cnt, cks);
        if (per_root) {
            unsigned long long mine = cnt - before;
            for (int o = 16; o > 0; o >>= 1) mine += __shfl_down_sync(kFull, mine, o);
            if (lane == 0 && mine) atomicAdd(&per_root[u], mine);
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

// Out-degree classes.  Up to 1024: reduced lists (shared memory up to 128,
// a global arena above); beyond: SDegreeList on the global out-lists.
constexpr uint32_t kClassD[] = {32, 64, 128, 256, 512, 1024, 4096, 16384, 65536};
constexpr int kNumClasses = 9;
constexpr int kSmemClasses = 3;
constexpr int kLocalClasses = 6;
constexpr size_t kSmemPerBlock = 96 * 1024;

uint32_t class_words(int c, uint32_t k) {
    return c < kLocalClasses ? make_llayout(kClassD[c], k).total : make_slayout(kClassD[c], k).total;
}

int arena_warps(int c, int num_sms) { return num_sms * (c < kLocalClasses ? 4 : 2); }

template <bool LIST, bool GLOBAL, bool LOCAL>
void launch_one(uint32_t k, uint32_t D, uint32_t words, Workspace &w, uint32_t begin, uint32_t end,
                unsigned *queue, const Emit &em, unsigned long long *per_root, int wpb, int blocks,
                cudaStream_t s) {
    size_t smem = GLOBAL ? 0 : (size_t)wpb * words * sizeof(uint32_t);
    auto kern = k_sdegree<LIST, GLOBAL, LOCAL>;
    if (!GLOBAL) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<blocks, wpb * 32, smem, s>>>(k, D, w.optr, w.oadj, w.roots, begin, end, queue, w.arena,
                                        words, em, per_root, w.res);
}

}  // namespace

int sdegree_classes(uint32_t *limits, int max) {
    int n = kNumClasses < max ? kNumClasses : max;
    for (int i = 0; i < n; i++) limits[i] = kClassD[i];
    return n;
}

size_t sdegree_arena_words(uint32_t k, int num_sms, uint32_t max_outdeg) {
    size_t need = 0;
    for (int c = kSmemClasses; c < kNumClasses; c++) {
        if (kClassD[c - 1] >= max_outdeg) break;
        size_t words = (size_t)arena_warps(c, num_sms) * class_words(c, k);
        if (words > need) need = words;
    }
    return need;
}

int launch_sdegree(const kcl_graph *g, uint32_t k, Workspace &w, const uint32_t *class_begin,
                   int n_classes, const ListArgs &la, cudaStream_t s) {
    Emit em{la.ring, la.capacity, la.wrap};
    int launches = 0;
    cudaMemsetAsync(w.queue, 0, 64 * sizeof(unsigned), s);
    for (int c = 0; c < n_classes; c++) {
        uint32_t begin = class_begin[c];
        uint32_t end = c ? class_begin[c - 1] : class_begin[n_classes];
        if (end <= begin) continue;
        uint32_t D = kClassD[c];
        unsigned *q = w.queue + c;
        uint32_t nroots = end - begin;
        uint32_t words = class_words(c, k);
        bool global = c >= kSmemClasses;
        int wpb, blocks;
        if (global) {
            wpb = c < kLocalClasses ? 4 : 2;
            blocks = g->num_sms;
        } else {
            wpb = (int)(kSmemPerBlock / ((size_t)words * 4));
            if (wpb > 4) wpb = 4;
            if (wpb < 1) wpb = 1;
            blocks = g->num_sms * (D <= 64 ? 8 : 4);
        }
        uint32_t need = (nroots + wpb - 1) / wpb;
        if ((uint32_t)blocks > need) blocks = (int)need;
#define KCL_SD(LST, GLB, LOC) \
    launch_one<LST, GLB, LOC>(k, D, words, w, begin, end, q, em, la.per_root, wpb, blocks, s)
        if (!global) {
            if (la.listing) KCL_SD(true, false, true); else KCL_SD(false, false, true);
        } else if (c < kLocalClasses) {
            if (la.listing) KCL_SD(true, true, true); else KCL_SD(false, true, true);
        } else {
            if (la.listing) KCL_SD(true, true, false); else KCL_SD(false, true, false);
        }
#undef KCL_SD
        launches++;
    }
    return launches;
}

}  // namespace kcl
