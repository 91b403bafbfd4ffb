// BitCol on the GPU (Algorithm 6, Section VII): for every root u of the
// degeneracy DAG with d+_u >= k-1, one warp
//   1. builds G_u, the undirected subgraph induced by N+_u (Section VII-B), as
//      bit-rows over the index space of N+_u (ascending id) -- each edge of
//      G_u lies in exactly one DAG out-list, so the warp scans the out-lists
//      of N+_u once and binary-searches each entry in N+_u;
//   2. colours G_u greedily in (degree descending, index ascending) order,
//      colours from 1 (Section VII-A, Example 6);
//   3. re-indexes G_u by colour (colour classes become contiguous index
//      ranges) and encodes the colour-ordered DAG: B'(p) holds the
//      out-neighbours of p, all of which sit below start[colour(p)]
//      (BitEncode, Section VII-C);
//   4. runs BitColList as an explicit-stack DFS: at level l only candidates
//      with colour >= l are expanded (Lemma 1 pruning, which the re-indexing
//      turns into a prefix test), C' = B'(v) AND C (BitJoin), recursion when
//      |C'| >= l-1, and at l = 2 each w in C' closes a clique.
// Lanes evaluate candidates in parallel (lane b takes bit b of a candidate
// word) and each lane ANDs + POPCs the words of its candidate's row; rows
// have an odd word stride so 32 lanes reading 32 different rows hit 32
// different shared-memory banks.  The word size is 32 (the paper's L = 24 on
// its CPU); the results do not depend on it.
#include "kcl_internal.cuh"

namespace kcl {

namespace {

constexpr unsigned kFull = 0xffffffffu;

// Per-warp scratch layout (32-bit words) for subproblems of at most 32*W
// vertices, with a DFS stack for k levels.
struct Lay {
    uint32_t W, D, WP, NBR, PRE, IDS, U16, ROWS_A, ROWS_B, STACK, total;
};

__host__ __device__ inline Lay make_layout(uint32_t W, uint32_t k) {
    Lay L;
    L.W = W;
    L.D = 32 * W;
    L.WP = (W & 1) ? W : W + 1;
    L.NBR = 0;
    L.PRE = L.NBR + L.D;
    L.IDS = L.PRE + L.D + 1;
    L.U16 = L.IDS + L.D;
    uint32_t u16_words = (4 * L.D + 2 + 1) / 2;  // colour_old, old2new, colp, start
    L.ROWS_A = L.U16 + u16_words;
    L.ROWS_B = L.ROWS_A + L.D * L.WP;
    L.STACK = L.ROWS_B + L.D * L.WP;
    L.total = L.STACK + k * (2 * W + 2) + 32;
    L.total = (L.total + 3) & ~3u;
    return L;
}

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x) {
    const unsigned lane = lane_id();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(kFull, x, o);
        if (lane >= (unsigned)o) x += y;
    }
    return x;
}

__device__ void warp_bitonic_sort(uint32_t *a, uint32_t n) {
    const unsigned lane = lane_id();
    for (uint32_t size = 2; size <= n; size <<= 1)
        for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
            for (uint32_t i = lane; i < n; i += 32) {
                uint32_t j = i ^ stride;
                if (j > i) {
                    bool up = (i & size) == 0;
                    uint32_t x = a[i], y = a[j];
                    if ((x > y) == up) { a[i] = y; a[j] = x; }
                }
            }
            __syncwarp();
        }
}

struct Emit {
    uint32_t *ring;
    unsigned long long capacity;
    int wrap;
};

// One root: build, colour, encode, DFS.  Counts accumulate per lane in
// `cnt`; in listing mode hashes accumulate in `cks`.
template <int WT, bool LIST>
__device__ void bitcol_root(uint32_t u, uint32_t k, uint32_t Wrt, const uint32_t *__restrict__ optr,
                            const uint32_t *__restrict__ oadj, uint32_t *S, const Emit &em,
                            DevResult *res, unsigned long long &cnt, unsigned long long &cks) {
    const uint32_t W = WT ? (uint32_t)WT : Wrt;
    const Lay L = make_layout(W, k);
    const uint32_t WP = L.WP;
    const unsigned lane = lane_id();
    const uint32_t base = optr[u];
    const uint32_t d = optr[u + 1] - base;

    uint32_t *nbr = S + L.NBR;
    uint32_t *pre = S + L.PRE;
    uint32_t *ids = S + L.IDS;
    uint16_t *colour_old = reinterpret_cast<uint16_t *>(S + L.U16);
    uint16_t *old2new = colour_old + L.D;
    uint16_t *colp = old2new + L.D;
    uint16_t *start = colp + L.D;  // D + 2 entries
    uint32_t *A = S + L.ROWS_A;
    uint32_t *B = S + L.ROWS_B;
    uint32_t *Cst = S + L.STACK;
    uint32_t *Pst = Cst + k * W;
    uint32_t *path = Pst + k * W;
    uint32_t *cur = path + k;
    uint32_t *sortedR = cur + k;

    // ---- 1. N+_u, prefix sums of the neighbours' out-degrees, zero rows
    uint32_t running = 0;
    for (uint32_t c0 = 0; c0 < d; c0 += 32) {
        uint32_t i = c0 + lane;
        uint32_t x = 0;
        if (i < d) {
            uint32_t v = oadj[base + i];
            nbr[i] = v;
            uint32_t rs = optr[v];
            ids[i] = rs;  // row start, reused below
            x = optr[v + 1] - rs;
        }
        uint32_t incl = warp_incl_scan(x);
        if (i < d) pre[i] = running + incl - x;
        running += __shfl_sync(kFull, incl, 31);
    }
    for (uint32_t i = lane; i < d * WP; i += 32) { A[i] = 0; B[i] = 0; }
    if (lane == 0) pre[d] = running;
    __syncwarp();
    const uint32_t total = running;
    const uint32_t lo_id = nbr[0], hi_id = nbr[d - 1];

    // ---- 2. adjacency of G_u (both directions of every edge)
    for (uint32_t e = lane; e < total; e += 32) {
        uint32_t a = 0, b = d;  // largest a with pre[a] <= e
        while (b - a > 1) {
            uint32_t m = (a + b) >> 1;
            if (pre[m] <= e) a = m; else b = m;
        }
        uint32_t w = oadj[ids[a] + (e - pre[a])];
        if (w < lo_id || w > hi_id) continue;
        uint32_t x = 0, y = d;
        while (x < y) {
            uint32_t m = (x + y) >> 1;
            if (nbr[m] < w) x = m + 1; else y = m;
        }
        if (x < d && nbr[x] == w) {
            atomicOr(&A[a * WP + (x >> 5)], 1u << (x & 31));
            atomicOr(&A[x * WP + (a >> 5)], 1u << (a & 31));
        }
    }
    __syncwarp();

    // ---- 3. colouring order: degree in G_u descending, index ascending
    uint32_t P2 = 1;
    while (P2 < d) P2 <<= 1;
    for (uint32_t i = lane; i < P2; i += 32) {
        uint32_t key = 0xFFFFFFFFu;
        if (i < d) {
            uint32_t deg = 0;
            for (uint32_t t = 0; t < W; t++) deg += __popc(A[i * WP + t]);
            key = ((0xFFFFu - deg) << 16) | i;
        }
        pre[i] = key;
    }
    __syncwarp();
    warp_bitonic_sort(pre, P2);

    // ---- 4. greedy colouring; colour classes as bitmaps (class c in row c-1 of B)
    uint32_t ncol = 0;
    for (uint32_t t = 0; t < d; t++) {
        uint32_t v = pre[t] & 0xFFFFu;
        uint32_t chosen = 0;
        for (uint32_t c0 = 0;; c0 += 32) {
            uint32_t c = c0 + lane + 1;
            bool fits = false;
            if (c <= ncol) {
                uint32_t acc = 0;
                for (uint32_t w = 0; w < W; w++) acc |= A[v * WP + w] & B[(c - 1) * WP + w];
                fits = acc == 0;
            } else if (c == ncol + 1) {
                fits = true;
            }
            unsigned m = __ballot_sync(kFull, fits);
            if (m) { chosen = c0 + __ffs(m); break; }
        }
        if (chosen > ncol) ncol = chosen;
        if (lane == 0) {
            B[(chosen - 1) * WP + (v >> 5)] |= 1u << (v & 31);
            colour_old[v] = (uint16_t)chosen;
        }
        __syncwarp();
    }

    // ---- 5. colour-sorted index: start[c] = first index of colour c
    for (uint32_t c0 = 0, run = 0; c0 < ncol; c0 += 32) {
        uint32_t c = c0 + lane + 1;
        uint32_t sz = 0;
        if (c <= ncol)
            for (uint32_t w = 0; w < W; w++) sz += __popc(B[(c - 1) * WP + w]);
        uint32_t incl = warp_incl_scan(sz);
        if (c <= ncol) start[c] = (uint16_t)(run + incl - sz);
        run += __shfl_sync(kFull, incl, 31);
    }
    if (lane == 0) {
        start[0] = 0;
        start[ncol + 1] = (uint16_t)d;
    }
    __syncwarp();
    for (uint32_t i = lane; i < d; i += 32) {
        uint32_t c = colour_old[i];
        const uint32_t *cls = B + (c - 1) * WP;
        uint32_t r = 0;
        for (uint32_t w = 0; w < (i >> 5); w++) r += __popc(cls[w]);
        r += __popc(cls[i >> 5] & ((1u << (i & 31)) - 1u));
        uint32_t p = start[c] + r;
        old2new[i] = (uint16_t)p;
        colp[p] = (uint16_t)c;
        ids[p] = nbr[i];
    }
    __syncwarp();

    // ---- 6. oriented rows B'(p): out-neighbours = lower colour = index < start[colour]
    for (uint32_t i = lane; i < d * WP; i += 32) B[i] = 0;
    __syncwarp();
    for (uint32_t i = lane; i < d; i += 32) {
        uint32_t p = old2new[i];
        uint32_t lim = start[colour_old[i]];
        uint32_t *row = B + p * WP;
        for (uint32_t w = 0; w < W; w++) {
            uint32_t m = A[i * WP + w];
            while (m) {
                uint32_t j = w * 32 + (__ffs(m) - 1);
                m &= m - 1;
                uint32_t q = old2new[j];
                if (q < lim) row[q >> 5] |= 1u << (q & 31);
            }
        }
    }
    __syncwarp();

    // ---- 7. BitColList as an explicit-stack DFS
    auto start_of = [&](uint32_t l) -> uint32_t { return l <= ncol + 1 ? (uint32_t)start[l] : d; };
    // candidate words: bits of C at index >= s
    auto cand_word = [&](const uint32_t *C, uint32_t j, uint32_t s) -> uint32_t {
        uint32_t m = C[j];
        uint32_t lo = j * 32;
        if (s >= lo + 32) return 0u;
        if (s > lo) m &= ~((1u << (s - lo)) - 1u);
        return m;
    };
    // leaf (l = 2): every candidate v closes |B'(v) & C| cliques
    auto leaf = [&](const uint32_t *C, uint32_t cw, uint32_t depth) {
        const uint32_t s = start_of(2);
        if (LIST && lane == 0) {
            // R = {u} + path[1..depth], sorted ascending (original ids)
            uint32_t nr = depth + 1;
            sortedR[0] = u;
            for (uint32_t t = 1; t < nr; t++) {
                uint32_t x = ids[path[t]], j = t;
                while (j > 0 && sortedR[j - 1] > x) { sortedR[j] = sortedR[j - 1]; j--; }
                sortedR[j] = x;
            }
        }
        if (LIST) __syncwarp();
        for (uint32_t j = 0; j < cw; j++) {
            uint32_t m = cand_word(C, j, s);
            if (!m) continue;
            uint32_t p = j * 32 + lane;
            uint32_t x = 0;
            bool mine = (m >> lane) & 1u;
            if (mine) {
                const uint32_t *row = B + p * WP;
                uint32_t wl = (start[colp[p]] + 31) >> 5;
                if (wl > cw) wl = cw;
                for (uint32_t t = 0; t < wl; t++) x += __popc(row[t] & C[t]);
            }
            cnt += x;
            if (LIST) {
                uint32_t incl = warp_incl_scan(x);
                uint32_t tot = __shfl_sync(kFull, incl, 31);
                unsigned long long slot0 = 0;
                if (tot) {
                    if (lane == 0 && em.ring) slot0 = atomicAdd(&res->emitted, (unsigned long long)tot);
                    slot0 = __shfl_sync(kFull, slot0, 0);
                }
                if (mine && x) {
                    unsigned long long slot = slot0 + (incl - x);
                    const uint32_t *row = B + p * WP;
                    uint32_t a = ids[p];
                    uint32_t wl = (start[colp[p]] + 31) >> 5;
                    if (wl > cw) wl = cw;
                    for (uint32_t t = 0; t < wl; t++) {
                        uint32_t mm = row[t] & C[t];
                        while (mm) {
                            uint32_t q = t * 32 + (__ffs(mm) - 1);
                            mm &= mm - 1;
                            uint32_t b = ids[q];
                            uint32_t e0 = a < b ? a : b, e1 = a < b ? b : a;
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
                    }
                }
            }
        }
    };
    // inner node (l >= 3): pending children = candidates v with |B'(v) & C| >= l-1
    auto expand = [&](const uint32_t *C, uint32_t cw, uint32_t l, uint32_t *P) {
        const uint32_t s = start_of(l);
        for (uint32_t j = 0; j < W; j++) {
            uint32_t m = j < cw ? cand_word(C, j, s) : 0u;
            bool ok = false;
            if ((m >> lane) & 1u) {
                uint32_t p = j * 32 + lane;
                const uint32_t *row = B + p * WP;
                uint32_t wl = (start[colp[p]] + 31) >> 5;
                if (wl > cw) wl = cw;
                uint32_t x = 0;
                for (uint32_t t = 0; t < wl; t++) x += __popc(row[t] & C[t]);
                ok = x + 1 >= l;
            }
            unsigned bal = __ballot_sync(kFull, ok);
            if (lane == 0) P[j] = bal;
        }
        __syncwarp();
    };

    const uint32_t dw = (d + 31) >> 5;
    for (uint32_t w = lane; w < W; w += 32) {
        uint32_t lo = w * 32;
        Cst[w] = lo + 32 <= d ? kFull : (lo < d ? ((1u << (d - lo)) - 1u) : 0u);
    }
    __syncwarp();
    const uint32_t l0 = k - 1;
    if (l0 == 2) {
        leaf(Cst, dw, 0);
        return;
    }
    if (start_of(l0) >= d) return;  // fewer than k-1 colours: no (k-1)-clique in G_u
    expand(Cst, dw, l0, Pst);
    if (lane == 0) { cur[0] = 0; path[0] = 0; }
    uint32_t cwst[KCL_MAX_K];  // words in use per depth (uniform)
    cwst[0] = dw;
    __syncwarp();
    int depth = 0;
    while (depth >= 0) {
        uint32_t *P = Pst + depth * W;
        uint32_t j = cur[depth];
        while (j < W && P[j] == 0) j++;
        if (j >= W) { depth--; continue; }
        uint32_t pw = P[j];
        uint32_t bit = __ffs(pw) - 1;
        uint32_t p = j * 32 + bit;
        __syncwarp();
        if (lane == 0) { P[j] = pw & (pw - 1); cur[depth] = j; }
        const uint32_t *C = Cst + depth * W;
        uint32_t *Cn = Cst + (depth + 1) * W;
        uint32_t cw = cwst[depth];
        uint32_t ncw = (start[colp[p]] + 31) >> 5;
        if (ncw > cw) ncw = cw;
        for (uint32_t t = lane; t < W; t += 32) Cn[t] = t < ncw ? (B[p * WP + t] & C[t]) : 0u;
        if (lane == 0) path[depth + 1] = p;
        __syncwarp();
        uint32_t l = k - 1 - (uint32_t)(depth + 1);
        if (l == 2) {
            leaf(Cn, ncw, depth + 1);
            __syncwarp();
        } else {
            expand(Cn, ncw, l, Pst + (depth + 1) * W);
            if (lane == 0) cur[depth + 1] = 0;
            cwst[depth + 1] = ncw;
            __syncwarp();
            depth++;
        }
    }
}

template <int WT, bool LIST, bool GLOBAL>
__global__ void __launch_bounds__(128) k_bitcol(uint32_t k, uint32_t Wrt, const uint32_t *__restrict__ optr,
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
        bitcol_root<WT, LIST>(u, k, Wrt, optr, oadj, S, em, res, cnt, cks);
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

// Root classes by out-degree: d+ <= 32 W for W = 1, 2, 4, 8 in shared memory,
// then W = 16 .. 128 with the scratch in a global arena (L2-resident).
constexpr uint32_t kClassW[] = {1, 2, 4, 8, 16, 32, 64, 128};
constexpr int kNumClasses = 8;
constexpr int kSmemClasses = 4;

template <int WT, bool LIST, bool GLOBAL>
void launch_one(uint32_t k, uint32_t W, const kcl_graph *g, Workspace &w, uint32_t begin,
                uint32_t end, unsigned *queue, const Emit &em, unsigned long long *per_root,
                int warps_per_block, int blocks, cudaStream_t s) {
    Lay L = make_layout(W, k);
    size_t smem = GLOBAL ? 0 : (size_t)warps_per_block * L.total * sizeof(uint32_t);
    auto kern = k_bitcol<WT, LIST, GLOBAL>;
    if (!GLOBAL) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<blocks, warps_per_block * 32, smem, s>>>(k, W, w.optr, w.oadj, w.roots, begin, end, queue,
                                                    w.arena, L.total, em, per_root, w.res);
}

}  // namespace

int bitcol_classes(uint32_t *limits, int max) {
    int n = kNumClasses < max ? kNumClasses : max;
    for (int i = 0; i < n; i++) limits[i] = 32 * kClassW[i];
    return n;
}

// Words of global arena the GLOBAL classes need (for the caller to size it).
size_t bitcol_arena_words(uint32_t k, int num_sms, uint32_t max_outdeg) {
    size_t need = 0;
    for (int c = kSmemClasses; c < kNumClasses; c++) {
        if (c > 0 && 32 * kClassW[c - 1] >= max_outdeg) break;
        Lay L = make_layout(kClassW[c], k);
        size_t warps = (size_t)num_sms * 4;
        size_t words = warps * L.total;
        if (words > need) need = words;
    }
    return need;
}

int launch_bitcol(const kcl_graph *g, uint32_t k, Workspace &w, const uint32_t *class_begin,
                  int n_classes, const ListArgs &la, cudaStream_t s) {
    // class c covers root positions [class_begin[c], c ? class_begin[c-1] : n_roots)
    Emit em{la.ring, la.capacity, la.wrap};
    int launches = 0;
    cudaMemsetAsync(w.queue, 0, 64 * sizeof(unsigned), s);
    for (int c = 0; c < n_classes; c++) {
        uint32_t begin = class_begin[c];
        uint32_t end = c ? class_begin[c - 1] : class_begin[n_classes];
        if (end <= begin) continue;
        uint32_t W = kClassW[c];
        unsigned *q = w.queue + c;
        uint32_t nroots = end - begin;
        if (c < kSmemClasses) {
            int wpb = W >= 8 ? 2 : 4;
            int per_sm = W == 1 ? 8 : (W == 2 ? 6 : (W == 4 ? 3 : 3));
            int blocks = g->num_sms * per_sm;
            uint32_t need = (nroots + wpb - 1) / wpb;
            if ((uint32_t)blocks > need) blocks = (int)need;
#define KCL_BC(WV)                                                                                   \
    if (la.listing) launch_one<WV, true, false>(k, W, g, w, begin, end, q, em, la.per_root, wpb, blocks, s); \
    else launch_one<WV, false, false>(k, W, g, w, begin, end, q, em, la.per_root, wpb, blocks, s);
            if (W == 1) { KCL_BC(1) }
            else if (W == 2) { KCL_BC(2) }
            else if (W == 4) { KCL_BC(4) }
            else { KCL_BC(8) }
#undef KCL_BC
        } else {
            int wpb = 4;
            int blocks = g->num_sms;
            uint32_t need = (nroots + wpb - 1) / wpb;
            if ((uint32_t)blocks > need) blocks = (int)need;
            if (la.listing) launch_one<0, true, true>(k, W, g, w, begin, end, q, em, la.per_root, wpb, blocks, s);
            else launch_one<0, false, true>(k, W, g, w, begin, end, q, em, la.per_root, wpb, blocks, s);
        }
        launches++;
    }
    return launches;
}

}  // namespace kcl
