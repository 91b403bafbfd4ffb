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

template <bool LIST, bool GLOBAL>
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
        sdegree_root<LIST>(u, k, D, optr, oadj, S, em, res, cnt, cks);
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

constexpr uint32_t kClassD[] = {32, 64, 128, 256, 512, 1024, 4096, 16384, 65536};
constexpr int kNumClasses = 9;
constexpr int kSmemClasses = 6;
constexpr size_t kSmemPerBlock = 96 * 1024;

int warps_for(uint32_t D, uint32_t k) {
    size_t per = (size_t)make_slayout(D, k).total * 4;
    int w = (int)(kSmemPerBlock / per);
    if (w > 4) w = 4;
    if (w < 1) w = 1;
    return w;
}

template <bool LIST, bool GLOBAL>
void launch_one(uint32_t k, uint32_t D, Workspace &w, uint32_t begin, uint32_t end, unsigned *queue,
                const Emit &em, unsigned long long *per_root, int wpb, int blocks, cudaStream_t s) {
    SLay L = make_slayout(D, k);
    size_t smem = GLOBAL ? 0 : (size_t)wpb * L.total * sizeof(uint32_t);
    auto kern = k_sdegree<LIST, GLOBAL>;
    if (!GLOBAL) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<blocks, wpb * 32, smem, s>>>(k, D, w.optr, w.oadj, w.roots, begin, end, queue, w.arena,
                                        L.total, em, per_root, w.res);
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
        size_t warps = (size_t)num_sms * 2;
        size_t words = warps * make_slayout(kClassD[c], k).total;
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
        bool global = c >= kSmemClasses;
        int wpb = global ? 2 : warps_for(D, k);
        int blocks = global ? g->num_sms : g->num_sms * (D <= 64 ? 8 : 4);
        uint32_t need = (nroots + wpb - 1) / wpb;
        if ((uint32_t)blocks > need) blocks = (int)need;
        if (global) {
            if (la.listing) launch_one<true, true>(k, D, w, begin, end, q, em, la.per_root, wpb, blocks, s);
            else launch_one<false, true>(k, D, w, begin, end, q, em, la.per_root, wpb, blocks, s);
        } else {
            if (la.listing) launch_one<true, false>(k, D, w, begin, end, q, em, la.per_root, wpb, blocks, s);
            else launch_one<false, false>(k, D, w, begin, end, q, em, la.per_root, wpb, blocks, s);
        }
        launches++;
    }
    return launches;
}

}  // namespace kcl
