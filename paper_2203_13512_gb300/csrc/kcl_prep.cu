// Front end of the k-clique pipeline on the device: input validation,
// Pre-Core (Algorithm 3), Pre-List (Algorithm 4), the two orientations
// (degree ordering of Section VI-B, degeneracy ordering of Algorithm 6) and
// the out-neighbour CSR of the DAG, plus the root list the listing kernels
// consume.  Every pass here streams the CSR once: these kernels are bound by
// HBM bandwidth, so they use warp-per-vertex row scans with coalesced loads.
#include <mutex>

#include "kcl_internal.cuh"

namespace kcl {

namespace {

constexpr int kBlock = 256;

inline int grid_for(uint64_t items, int per_block, int num_sms, int per_sm = 16) {
    uint64_t g = (items + per_block - 1) / per_block;
    uint64_t cap = (uint64_t)num_sms * per_sm;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

__device__ __forceinline__ uint32_t warp_global() {
    return (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
}
__device__ __forceinline__ uint32_t warps_total() { return (gridDim.x * blockDim.x) >> 5; }

// ----------------------------------------------------------- validation
// Row u: strictly ascending, ids < n, no self-loop, and every v in row u has
// u in row v (binary search).  Also records the maximum degree.
__global__ void k_validate(uint32_t n, uint64_t nnz, const uint64_t *__restrict__ rp,
                           const uint32_t *__restrict__ col, DevResult *res) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (rp[0] != 0 || rp[n] != nnz) atomicOr(&res->status, DEV_ERR_INVALID_GRAPH);
    }
    const unsigned lane = lane_id();
    for (uint32_t u = warp_global(); u < n; u += warps_total()) {
        uint64_t b = rp[u], e = rp[u + 1];
        if (e < b || e > nnz) {
            if (lane == 0) atomicOr(&res->status, DEV_ERR_INVALID_GRAPH);
            continue;
        }
        if (lane == 0 && e - b > 0xFFFFFFFFull) atomicOr(&res->status, DEV_ERR_INVALID_GRAPH);
        if (lane == 0) atomicMax(&res->max_outdeg, (unsigned)(e - b));
        bool bad = false;
        for (uint64_t i = b + lane; i < e; i += 32) {
            uint32_t v = col[i];
            if (v >= n || v == u) { bad = true; continue; }
            if (i > b && col[i - 1] >= v) bad = true;
            // symmetric: u must be in row v
            uint64_t lo = rp[v], hi = rp[v + 1];
            if (hi < lo || hi > nnz) { bad = true; continue; }
            bool found = false;
            while (lo < hi) {
                uint64_t mid = lo + ((hi - lo) >> 1);
                uint32_t x = col[mid];
                if (x == u) { found = true; break; }
                if (x < u) lo = mid + 1; else hi = mid;
            }
            if (!found) bad = true;
        }
        if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(&res->status, DEV_ERR_INVALID_GRAPH);
    }
}

// ------------------------------------------------------------- Pre-Core
// Algorithm 3, frontier form: the initial queue is every vertex of degree
// < k-1; each round, every queued vertex lowers the degree of its alive
// neighbours and a neighbour whose degree falls from k-1 to k-2 joins the
// next queue (exactly one thread sees that transition).
// thr = k-1, or per vertex kmap[v] - 1 when a k map is given (batches of
// graphs with different k).
__global__ void k_precore_init(uint32_t n, const uint64_t *__restrict__ rp, uint32_t thr,
                               const uint8_t *__restrict__ kmap, uint8_t *alive, uint32_t *cdeg,
                               uint32_t *fout, unsigned *fcount) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        uint32_t d = (uint32_t)(rp[v + 1] - rp[v]);
        cdeg[v] = d;
        bool keep = d >= (kmap ? kmap[v] - 1u : thr);
        alive[v] = keep ? 1 : 0;
        if (!keep) fout[atomicAdd(fcount, 1u)] = v;
    }
}

__global__ void k_precore_round(const uint64_t *__restrict__ rp, const uint32_t *__restrict__ col,
                                uint32_t thr, const uint8_t *__restrict__ kmap,
                                const uint32_t *__restrict__ fin, uint32_t nin,
                                uint8_t *alive, uint32_t *cdeg, uint32_t *fout, unsigned *fcount) {
    const unsigned lane = lane_id();
    for (uint32_t i = warp_global(); i < nin; i += warps_total()) {
        uint32_t v = fin[i];
        for (uint64_t e = rp[v] + lane; e < rp[v + 1]; e += 32) {
            uint32_t w = col[e];
            if (!alive[w]) continue;
            uint32_t old = atomicSub(&cdeg[w], 1u);
            if (old == (kmap ? kmap[w] - 1u : thr)) {  // fell from k-1 to k-2
                alive[w] = 0;
                fout[atomicAdd(fcount, 1u)] = w;
            }
        }
    }
}

// ------------------------------------------------------------- Pre-List
// Connected components of the alive subgraph by lock-free union-find
// (hooking the larger root under the smaller one), then per component the
// vertex count n_c and degree sum m_c; m_c = n_c (n_c - 1) marks a clique.
__device__ __forceinline__ uint32_t uf_find(uint32_t *parent, uint32_t x) {
    volatile uint32_t *p = parent;
    uint32_t px = p[x];
    while (px != x) {
        uint32_t gp = p[px];
        if (gp != px) p[x] = gp;  // path halving (benign race)
        x = px;
        px = p[x];
    }
    return x;
}

__global__ void k_uf_init(uint32_t n, uint32_t *parent, uint32_t *comp_n,
                          unsigned long long *comp_sdeg, uint32_t *comp_flag) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        parent[v] = v;
        comp_n[v] = 0;
        comp_sdeg[v] = 0;
        comp_flag[v] = 0;
    }
}

__global__ void k_uf_hook(uint32_t n, const uint64_t *__restrict__ rp, const uint32_t *__restrict__ col,
                          const uint8_t *__restrict__ alive, uint32_t *parent) {
    const unsigned lane = lane_id();
    for (uint32_t u = warp_global(); u < n; u += warps_total()) {
        if (!alive[u]) continue;
        for (uint64_t e = rp[u] + lane; e < rp[u + 1]; e += 32) {
            uint32_t w = col[e];
            if (w <= u || !alive[w]) continue;
            uint32_t a = u, b = w;
            for (;;) {
                a = uf_find(parent, a);
                b = uf_find(parent, b);
                if (a == b) break;
                if (a > b) { uint32_t t = a; a = b; b = t; }
                uint32_t old = atomicCAS(&parent[b], b, a);
                if (old == b) break;
                b = old;
            }
        }
    }
}

__global__ void k_uf_stats(uint32_t n, const uint8_t *__restrict__ alive, uint32_t *parent,
                           const uint32_t *__restrict__ cdeg, uint32_t *comp_n,
                           unsigned long long *comp_sdeg) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        if (!alive[v]) continue;
        uint32_t r = uf_find(parent, v);
        parent[v] = r;
        atomicAdd(&comp_n[r], 1u);
        atomicAdd(&comp_sdeg[r], (unsigned long long)cdeg[v]);
    }
}

// C(n, k) in 64 bits; sets *ovf when it does not fit.
__device__ unsigned long long binom64(unsigned long long n, unsigned k, bool *ovf) {
    if (k > n) return 0;
    if (k > n - k) k = (unsigned)(n - k);
    unsigned long long r = 1;
    for (unsigned i = 1; i <= k; i++) {
        unsigned long long f = n - k + i;
        unsigned long long hi = __umul64hi(r, f);
        unsigned long long lo = r * f;
        if (hi >= i) { *ovf = true; return 0; }
        // exact division of the 128-bit product (hi:lo) by i, hi < i
        unsigned long long q = 0, rem = hi;
        for (int bit = 63; bit >= 0; bit--) {
            unsigned long long top = rem >> 63;
            rem = (rem << 1) | ((lo >> bit) & 1ull);
            if (top || rem >= i) { rem -= i; q |= 1ull << bit; }
        }
        r = q;
    }
    return r;
}

__global__ void k_uf_check(uint32_t n, uint32_t k, const uint8_t *__restrict__ kmap,
                           const uint8_t *__restrict__ alive,
                           const uint32_t *__restrict__ parent, const uint32_t *__restrict__ comp_n,
                           const unsigned long long *__restrict__ comp_sdeg, uint32_t *comp_flag,
                           uint32_t *comp_slot, unsigned long long *vcount, DevResult *res) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        if (!alive[v] || parent[v] != v) continue;
        unsigned long long nc = comp_n[v];
        if (comp_sdeg[v] != nc * (nc - 1)) continue;
        bool ovf = false;
        unsigned long long c = binom64(nc, kmap ? kmap[v] : k, &ovf);  // a component lies in one graph
        if (ovf) atomicOr(&res->status, DEV_ERR_OVERFLOW);
        add_count(&res->pre_count, &res->count_carry, c);
        if (vcount && c) atomicAdd(&vcount[v], c);  // attributed to the component's root
        uint32_t slot = atomicAdd(&res->n_clique_comps, 1u);
        comp_flag[v] = 1;
        if (comp_slot) comp_slot[v] = slot;
    }
}

__global__ void k_uf_remove(uint32_t n, uint8_t *alive, const uint32_t *__restrict__ parent,
                            const uint32_t *__restrict__ comp_flag) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        if (alive[v] && comp_flag[parent[v]]) alive[v] = 0;
}

// Listing of Pre-List cliques: gather each clique component's members,
// sort them, then enumerate every k-subset by unranking (combinatorial
// number system) so each k-clique of the component is reported once.
__global__ void k_comp_gather(uint32_t n, const uint32_t *__restrict__ parent,
                              const uint32_t *__restrict__ comp_flag, const uint32_t *__restrict__ comp_slot,
                              const uint8_t *__restrict__ alive_core, const uint32_t *__restrict__ offs,
                              uint32_t *fill, uint32_t *members) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        if (!alive_core[v]) continue;
        uint32_t r = parent[v];
        if (!comp_flag[r]) continue;
        uint32_t s = comp_slot[r];
        members[offs[s] + atomicAdd(&fill[s], 1u)] = v;
    }
}

__global__ void k_comp_sizes(uint32_t n, const uint32_t *__restrict__ comp_flag,
                             const uint32_t *__restrict__ comp_slot, const uint32_t *__restrict__ comp_n,
                             uint32_t *sizes, uint32_t *roots) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        if (!comp_flag[v]) continue;
        sizes[comp_slot[v]] = comp_n[v];
        roots[comp_slot[v]] = v;
    }
}

// One block per component: odd-even transposition sort of its members.
__global__ void k_comp_sort(const uint32_t *__restrict__ offs, const uint32_t *__restrict__ sizes,
                            uint32_t *members) {
    uint32_t s = blockIdx.x;
    uint32_t *m = members + offs[s];
    uint32_t len = sizes[s];
    for (uint32_t phase = 0; phase < len; phase++) {
        for (uint32_t i = 2 * threadIdx.x + (phase & 1); i + 1 < len; i += 2 * blockDim.x) {
            uint32_t a = m[i], b = m[i + 1];
            if (a > b) { m[i] = b; m[i + 1] = a; }
        }
        __syncthreads();
    }
}

// C(n, k) saturated at 2^64 - 1 (used for comparisons while unranking).
__device__ unsigned long long binom_small(unsigned long long n, unsigned k) {
    bool ovf = false;
    unsigned long long r = binom64(n, k, &ovf);
    return ovf ? ~0ull : r;
}

__global__ void k_comp_emit(uint32_t kk, const uint8_t *__restrict__ kmap, const uint32_t *__restrict__ offs,
                            const uint32_t *__restrict__ sizes, const uint32_t *__restrict__ members,
                            uint32_t *ring, unsigned long long capacity, int wrap,
                            const uint32_t *__restrict__ croots, unsigned long long *vcks,
                            const uint32_t *__restrict__ idmap, DevResult *res) {
    uint32_t s = blockIdx.x;
    const uint32_t k = kmap ? kmap[croots[s]] : kk;
    const uint32_t *m = members + offs[s];
    uint32_t nc = sizes[s];
    if (nc < k) return;
    unsigned long long total = binom_small(nc, k);
    unsigned long long local_sum = 0;
    uint32_t ids[KCL_MAX_K];
    for (unsigned long long r = threadIdx.x; r < total; r += blockDim.x) {
        // unrank r: largest c_i with C(c_i, i) <= remaining, i = k..1
        unsigned long long rem = r;
        uint32_t hi = nc;
        for (uint32_t i = k; i >= 1; i--) {
            uint32_t c = i - 1;
            // linear scan upward is fine for the small components this handles
            uint32_t lo = i - 1, up = hi;  // C(c, i) <= rem, c in [i-1, hi-1]
            while (lo + 1 < up) {
                uint32_t mid = (lo + up) >> 1;
                if (binom_small(mid, i) <= rem) lo = mid; else up = mid;
            }
            c = lo;
            rem -= binom_small(c, i);
            ids[i - 1] = idmap ? idmap[m[c]] : m[c];
            hi = c;
        }
        uint64_t h = hash_seed(k);
        for (uint32_t i = 0; i < k; i++) h = mix64(h ^ (uint64_t)ids[i]);
        local_sum += h;
        if (ring) {
            unsigned long long slot = atomicAdd(&res->emitted, 1ull);
            if (wrap) slot %= capacity;
            if (slot < capacity)
                for (uint32_t i = 0; i < k; i++) ring[slot * k + i] = ids[i];
        }
    }
    atomicAdd(&res->pre_checksum, local_sum);
    if (vcks && local_sum) atomicAdd(&vcks[croots[s]], local_sum);
}

// -------------------------------------------------------- orientations
__global__ void k_degree_key(uint32_t n, const uint8_t *__restrict__ alive,
                             const uint32_t *__restrict__ cdeg, uint32_t *key) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        key[v] = alive[v] ? cdeg[v] : 0xFFFFFFFFu;
}

// Degeneracy ordering by bulk peel rounds: each round removes every remaining
// vertex whose current degree is <= t; when none qualifies t rises to the
// minimum remaining degree.  key[v] = the round v leaves in (UINT_MAX while
// it remains).
__global__ void k_peel_init(uint32_t n, const uint8_t *__restrict__ alive,
                            const uint32_t *__restrict__ cdeg, uint32_t *pdeg, uint32_t *key,
                            DevResult *res) {
    uint32_t cnt = 0;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        pdeg[v] = cdeg[v];
        key[v] = 0xFFFFFFFFu;
        cnt += alive[v] ? 1 : 0;
    }
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    if (lane_id() == 0 && cnt) atomicAdd(&res->remaining, cnt);
}

__global__ void k_peel_min(uint32_t n, const uint8_t *__restrict__ alive,
                           const uint32_t *__restrict__ pdeg, const uint32_t *__restrict__ key,
                           DevResult *res) {
    uint32_t mn = 0xFFFFFFFFu;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        if (alive[v] && key[v] == 0xFFFFFFFFu && pdeg[v] < mn) mn = pdeg[v];
    mn = __reduce_min_sync(0xffffffffu, mn);
    if (lane_id() == 0 && mn != 0xFFFFFFFFu) atomicMin(&res->min_deg, mn);
}

__global__ void k_peel_select_all(uint32_t n, const uint8_t *__restrict__ alive,
                                  const uint32_t *__restrict__ pdeg, uint32_t *key, uint32_t t,
                                  uint32_t round, uint32_t *fout, unsigned *fcount) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        if (alive[v] && key[v] == 0xFFFFFFFFu && pdeg[v] <= t) {
            key[v] = round;
            fout[atomicAdd(fcount, 1u)] = v;
        }
    }
}

__global__ void k_peel_update(const uint64_t *__restrict__ rp, const uint32_t *__restrict__ col,
                              const uint8_t *__restrict__ alive, uint32_t *pdeg, uint32_t *key,
                              const uint32_t *__restrict__ fin, uint32_t nin, uint32_t t,
                              uint32_t next_round, uint32_t *fout, unsigned *fcount) {
    const unsigned lane = lane_id();
    for (uint32_t i = warp_global(); i < nin; i += warps_total()) {
        uint32_t v = fin[i];
        for (uint64_t e = rp[v] + lane; e < rp[v + 1]; e += 32) {
            uint32_t w = col[e];
            if (!alive[w] || key[w] != 0xFFFFFFFFu) continue;
            uint32_t nd = atomicSub(&pdeg[w], 1u) - 1u;
            if (nd <= t && atomicCAS(&key[w], 0xFFFFFFFFu, next_round) == 0xFFFFFFFFu)
                fout[atomicAdd(fcount, 1u)] = w;
        }
    }
}

// The same peel in one cooperative launch (every block resident): rounds are
// separated by a grid barrier instead of a kernel boundary and a host round
// trip.  Every block follows the same control flow, derived from counters
// read after a barrier:
//   a round with a non-empty frontier (a cascade) processes it and ends with
//     one barrier; frontier counters rotate over three rounds (round r reads
//     fcnt[r % 3], appends to fcnt[(r+1) % 3] and clears fcnt[(r+2) % 3],
//     which every block read two barriers earlier);
//   a round with an empty frontier raises t: a pass over the remaining
//     vertices finds their minimum degree (barrier), a second pass selects
//     those at or below t into the frontier and, when rl0/rl1 are given,
//     compacts the vertices still remaining into the other list (barrier),
//     so later passes touch only what is left.
// Arrays written during the launch are read with ld.global.cg (L2) so no
// stale L1 line is used.  Every barrier wait is bounded: past kSpinLimit
// polls the block records an error, all blocks leave, and the host reports
// KCL_ETIMEOUT.
constexpr unsigned long long kSpinLimit = 1ull << 25;

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned *p, unsigned x) {
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(x) : "memory");
    return old;
}

// Generation barrier: thread 0 of each block arrives with an acquire-release
// add (publishing the block's writes, which __syncthreads has ordered before
// it); the last arrival clears the count and bumps the generation with a
// release, and the others poll the generation with acquire loads.
__device__ bool grid_barrier(PeelCtl *c, unsigned nblocks) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned g = ld_acquire(&c->bar_gen);
        const unsigned arrived = atom_add_acq_rel(&c->bar_count, 1u);
        int ok = 1;
        if (arrived == nblocks - 1) {
            atomicExch(&c->bar_count, 0u);
            atom_add_acq_rel(&c->bar_gen, 1u);
        } else {
            unsigned long long spins = 0;
            while (ld_acquire(&c->bar_gen) == g) {
                if (ld_acquire(&c->error)) { ok = 0; break; }
                if (++spins > kSpinLimit) { atomicExch(&c->error, 1u); ok = 0; break; }
            }
        }
        ok_s = ok && ld_acquire(&c->error) == 0;
    }
    __syncthreads();
    return ok_s != 0;
}

// A frontier vertex whose row is longer than `big` goes to a separate list
// (bl0/bl1 by round parity) and its row is walked by every thread of the grid
// instead of one warp, so a hub does not stretch its round.
__global__ void __launch_bounds__(1024) k_peel_coop(uint32_t n, const uint64_t *__restrict__ rp,
                                                    const uint32_t *__restrict__ col,
                                                    const uint8_t *__restrict__ alive,
                                                    const uint32_t *__restrict__ cdeg, uint32_t *pdeg,
                                                    uint32_t *key, uint32_t *fa, uint32_t *fb,
                                                    uint32_t *rl0, uint32_t *rl1, uint32_t *bl0,
                                                    uint32_t *bl1, uint64_t big, PeelCtl *c) {
    const unsigned nblocks = gridDim.x;
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t nth = gridDim.x * blockDim.x;
    const unsigned lane = lane_id();
    volatile PeelCtl *vc = c;
    const bool lists = rl0 != nullptr;
    {
        uint32_t cnt = 0;
        for (uint32_t v0 = tid - lane; v0 < n; v0 += nth) {  // warp-uniform trip count
            const uint32_t v = v0 + lane;
            bool a = false;
            if (v < n) {
                pdeg[v] = cdeg[v];
                key[v] = 0xFFFFFFFFu;
                a = alive[v] != 0;
            }
            cnt += a ? 1 : 0;
            if (lists) {  // the first remaining list: every alive vertex
                const unsigned m = __ballot_sync(0xffffffffu, a);
                unsigned base = 0;
                if (lane == 0 && m) base = atomicAdd(&c->rcnt[0], (unsigned)__popc(m));
                base = __shfl_sync(0xffffffffu, base, 0);
                if (a) rl0[base + __popc(m & ((1u << lane) - 1u))] = v;
            }
        }
        cnt = __reduce_add_sync(0xffffffffu, cnt);
        if (lane == 0 && cnt) atomicAdd(&c->remaining, cnt);
    }
    if (!grid_barrier(c, nblocks)) return;
    uint32_t remaining = vc->remaining;
    uint32_t round = 0, t = 0, level = 0;
    while (remaining > 0) {
        const uint32_t fi = round % 3u;
        uint32_t *fin = (round & 1u) ? fb : fa;
        uint32_t *fout = (round & 1u) ? fa : fb;
        uint32_t *bin = (round & 1u) ? bl1 : bl0;
        uint32_t *bout = (round & 1u) ? bl0 : bl1;
        uint32_t nin = vc->fcnt[fi];
        uint32_t nbig = vc->bcnt[fi];
        if (nin + nbig == 0) {
            // t rises to the minimum remaining degree
            const uint32_t lp = level & 1u;
            const uint32_t *rl = lp ? rl1 : rl0;
            uint32_t *rl_next = lp ? rl0 : rl1;
            const uint32_t nr = lists ? vc->rcnt[lp] : n;
            if (tid == 0 && lists) c->rcnt[lp ^ 1u] = 0;  // read at the previous level
            uint32_t mn = 0xFFFFFFFFu;
            for (uint32_t i = tid; i < nr; i += nth) {
                const uint32_t v = lists ? __ldcg(&rl[i]) : i;
                if ((lists || alive[v]) && __ldcg(&key[v]) == 0xFFFFFFFFu) {
                    const uint32_t d = __ldcg(&pdeg[v]);
                    mn = d < mn ? d : mn;
                }
            }
            mn = __reduce_min_sync(0xffffffffu, mn);
            if (lane == 0 && mn != 0xFFFFFFFFu) atomicMin(&c->minv[lp], mn);
            if (!grid_barrier(c, nblocks)) return;
            const uint32_t mv = vc->minv[lp];
            if (mv > t) t = mv;
            if (tid == 0) c->minv[lp ^ 1u] = 0xFFFFFFFFu;  // read at the previous level
            // select the frontier; compact the rest into the other list
            for (uint32_t i0 = tid - lane; i0 < nr; i0 += nth) {
                const uint32_t i = i0 + lane;
                bool sel = false, keep = false, sbig = false;
                uint32_t v = 0;
                if (i < nr) {
                    v = lists ? __ldcg(&rl[i]) : i;
                    if ((lists || alive[v]) && __ldcg(&key[v]) == 0xFFFFFFFFu) {
                        sel = __ldcg(&pdeg[v]) <= t;
                        keep = !sel;
                        sbig = sel && bl0 && rp[v + 1] - rp[v] > big;
                        sel = sel && !sbig;
                    }
                }
                const unsigned ms = __ballot_sync(0xffffffffu, sel);
                unsigned bs = 0;
                if (lane == 0 && ms) bs = atomicAdd(&c->fcnt[fi], (unsigned)__popc(ms));
                bs = __shfl_sync(0xffffffffu, bs, 0);
                if (sel) {
                    key[v] = round;
                    fin[bs + __popc(ms & ((1u << lane) - 1u))] = v;
                }
                if (sbig) {  // rare: one atomic each
                    key[v] = round;
                    bin[atomicAdd(&c->bcnt[fi], 1u)] = v;
                }
                if (lists) {
                    const unsigned mk = __ballot_sync(0xffffffffu, keep);
                    unsigned bk = 0;
                    if (lane == 0 && mk) bk = atomicAdd(&c->rcnt[lp ^ 1u], (unsigned)__popc(mk));
                    bk = __shfl_sync(0xffffffffu, bk, 0);
                    if (keep) rl_next[bk + __popc(mk & ((1u << lane) - 1u))] = v;
                }
            }
            level++;
            if (!grid_barrier(c, nblocks)) return;
            nin = vc->fcnt[fi];
            nbig = vc->bcnt[fi];
            if (nin + nbig == 0) {  // cannot happen while vertices remain
                if (tid == 0) atomicExch(&c->error, 2u);
                return;
            }
        }
        if (tid == 0) {  // every block read these two barriers ago
            c->fcnt[(round + 2u) % 3u] = 0;
            c->bcnt[(round + 2u) % 3u] = 0;
        }
        // remove this round's vertices: lower the degrees of their remaining
        // neighbours; a neighbour reaching <= t joins the next round
        uint32_t *fnext_cnt = &c->fcnt[(round + 1u) % 3u];
        uint32_t *bnext_cnt = &c->bcnt[(round + 1u) % 3u];
        auto relax = [&](uint32_t w) {
            if (!alive[w] || __ldcg(&key[w]) != 0xFFFFFFFFu) return;
            const uint32_t nd = atomicSub(&pdeg[w], 1u) - 1u;
            if (nd <= t && atomicCAS(&key[w], 0xFFFFFFFFu, round + 1) == 0xFFFFFFFFu) {
                if (bl0 && rp[w + 1] - rp[w] > big) bout[atomicAdd(bnext_cnt, 1u)] = w;
                else fout[atomicAdd(fnext_cnt, 1u)] = w;
            }
        };
        for (uint32_t b = 0; b < nbig; b++) {  // big rows: the whole grid, one edge per thread
            const uint32_t v = __ldcg(&bin[b]);
            for (uint64_t e = rp[v] + tid; e < rp[v + 1]; e += nth) relax(col[e]);
        }
        for (uint32_t i = tid >> 5; i < nin; i += nth >> 5) {
            const uint32_t v = __ldcg(&fin[i]);
            for (uint64_t e = rp[v] + lane; e < rp[v + 1]; e += 32) relax(col[e]);
        }
        const uint32_t gone = nin + nbig;
        remaining -= gone < remaining ? gone : remaining;
        round++;
        if (!grid_barrier(c, nblocks)) return;
    }
}

// Out-degree in the DAG u -> w iff (key[u], u) < (key[w], w), both alive.
__device__ __forceinline__ bool eta_less(uint32_t ku, uint32_t u, uint32_t kw, uint32_t w) {
    return ku < kw || (ku == kw && u < w);
}

__global__ void k_outdeg(uint32_t n, const uint64_t *__restrict__ rp, const uint32_t *__restrict__ col,
                         const uint8_t *__restrict__ alive, const uint32_t *__restrict__ key,
                         uint32_t *outdeg, DevResult *res) {
    const unsigned lane = lane_id();
    for (uint32_t u = warp_global(); u < n; u += warps_total()) {
        uint32_t c = 0;
        if (alive[u]) {
            uint32_t ku = key[u];
            for (uint64_t e = rp[u] + lane; e < rp[u + 1]; e += 32) {
                uint32_t w = col[e];
                if (alive[w] && eta_less(ku, u, key[w], w)) c++;
            }
            c = __reduce_add_sync(0xffffffffu, c);
        }
        if (lane == 0) {
            outdeg[u] = c;
            if (c) atomicMax(&res->max_outdeg, c);
        }
    }
}

__global__ void k_outfill(uint32_t n, const uint64_t *__restrict__ rp, const uint32_t *__restrict__ col,
                          const uint8_t *__restrict__ alive, const uint32_t *__restrict__ key,
                          const uint32_t *__restrict__ optr, uint32_t *oadj) {
    const unsigned lane = lane_id();
    for (uint32_t u = warp_global(); u < n; u += warps_total()) {
        if (!alive[u]) continue;
        uint32_t ku = key[u];
        uint32_t base = optr[u];
        uint64_t b = rp[u], e = rp[u + 1];
        for (uint64_t s = b; s < e; s += 32) {
            uint64_t i = s + lane;
            bool take = false;
            uint32_t w = 0;
            if (i < e) {
                w = col[i];
                take = alive[w] && eta_less(ku, u, key[w], w);
            }
            unsigned m = __ballot_sync(0xffffffffu, take);
            if (take) oadj[base + __popc(m & ((1u << lane) - 1u))] = w;
            base += __popc(m);
        }
    }
}

// Roots (alive, d+ >= k-1) counted by out-degree, then placed in descending
// out-degree order by a counting sort: hist index = max_outdeg - d+.
__global__ void k_root_hist(uint32_t n, uint32_t k, const uint8_t *__restrict__ alive,
                            const uint32_t *__restrict__ outdeg, uint32_t max_outdeg, uint32_t *hist,
                            const uint8_t *__restrict__ mask, const uint8_t *__restrict__ kmap,
                            DevResult *res) {
    uint32_t cnt = 0;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        uint32_t d = outdeg[v];
        if (alive[v] && d + 1 >= (kmap ? kmap[v] : k) && (!mask || mask[v])) {
            atomicAdd(&hist[max_outdeg - d], 1u);
            cnt++;
        }
    }
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    if (lane_id() == 0 && cnt) atomicAdd(&res->n_roots, cnt);
}

__global__ void k_root_scatter(uint32_t n, uint32_t k, const uint8_t *__restrict__ alive,
                               const uint32_t *__restrict__ outdeg, uint32_t max_outdeg,
                               const uint32_t *__restrict__ offs, uint32_t *fill,
                               const uint8_t *__restrict__ mask, const uint8_t *__restrict__ kmap,
                               uint32_t *roots) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        uint32_t d = outdeg[v];
        if (alive[v] && d + 1 >= (kmap ? kmap[v] : k) && (!mask || mask[v])) {
            uint32_t h = max_outdeg - d;
            roots[offs[h] + atomicAdd(&fill[h], 1u)] = v;
        }
    }
}

// class_begin[c] = first root position whose d+ <= limits[c] (roots are in
// descending d+), i.e. the number of roots with d+ > limits[c].
__global__ void k_class_bounds(const uint32_t *__restrict__ offs, uint32_t max_outdeg,
                               const uint32_t *__restrict__ limits, int n_classes, uint32_t n_roots,
                               uint32_t *class_begin) {
    int c = threadIdx.x;
    if (c < n_classes) {
        uint32_t lim = limits[c];
        // hist index h = max_outdeg - d; d > lim  <=>  h < max_outdeg - lim
        class_begin[c] = lim >= max_outdeg ? 0u : offs[max_outdeg - lim];
    }
    if (c == 0) class_begin[n_classes] = n_roots;
}

// --------------------------------------------------------------- scans
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ uint32_t block_excl_scan(uint32_t x, uint32_t *smem, uint32_t *total) {
    const unsigned lane = lane_id(), wid = threadIdx.x >> 5;
    uint32_t v = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= (unsigned)o) v += y;
    }
    if (lane == 31) smem[wid] = v;
    __syncthreads();
    if (wid == 0) {
        uint32_t s = lane < (blockDim.x >> 5) ? smem[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= (unsigned)o) s += y;
        }
        smem[lane] = s;
    }
    __syncthreads();
    uint32_t warp_prefix = wid ? smem[wid - 1] : 0;
    *total = smem[(blockDim.x >> 5) - 1];
    __syncthreads();
    return warp_prefix + v - x;
}

__global__ void k_scan_tiles(const uint32_t *__restrict__ in, uint32_t *out, uint32_t n,
                             uint32_t *tile_sums) {
    __shared__ uint32_t smem[32];
    uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        v[i] = base + i < n ? in[base + i] : 0;
        s += v[i];
    }
    uint32_t total;
    uint32_t p = block_excl_scan(s, smem, &total);
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        if (base + i < n) out[base + i] = p;
        p += v[i];
    }
    if (threadIdx.x == 0 && tile_sums) tile_sums[blockIdx.x] = total;
}

__global__ void k_scan_add(uint32_t *out, uint32_t n, const uint32_t *__restrict__ tile_offs) {
    uint64_t base = (uint64_t)blockIdx.x * kScanTile;
    uint32_t add = tile_offs[blockIdx.x];
    for (uint32_t i = threadIdx.x; i < kScanTile; i += blockDim.x)
        if (base + i < n) out[base + i] += add;
}

}  // namespace

// ====================================================== host launchers
// ---------------------------------------------------------- batching
// Disjoint union of a batch of graphs: block b copies graph b's rows and
// columns with its vertex offset voff[b] and edge offset eoff[b].
__global__ void k_union_build(const BatchSrc *__restrict__ src, uint32_t n_total, uint64_t *urp,
                              uint32_t *ucol, uint32_t *graph_of, uint32_t *idmap, uint8_t *kmap) {
    const BatchSrc b = src[blockIdx.x];
    for (uint32_t v = threadIdx.x; v < b.n; v += blockDim.x) {
        urp[b.voff + v] = b.rp[v] + b.eoff;
        graph_of[b.voff + v] = blockIdx.x;
        idmap[b.voff + v] = v;
        kmap[b.voff + v] = (uint8_t)b.k;
    }
    for (uint64_t e = threadIdx.x; e < b.nnz; e += blockDim.x) ucol[b.eoff + e] = b.col[e] + b.voff;
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) urp[n_total] = b.eoff + b.nnz;
}

// Per-graph sums of per-vertex attributions (one block per graph).
__global__ void k_graph_sums(const BatchSrc *__restrict__ src, const unsigned long long *__restrict__ vcount,
                             const unsigned long long *__restrict__ vcks, unsigned long long *out_count,
                             unsigned long long *out_cks) {
    __shared__ unsigned long long sc[32], sk[32];
    const BatchSrc b = src[blockIdx.x];
    unsigned long long c = 0, h = 0;
    for (uint32_t v = threadIdx.x; v < b.n; v += blockDim.x) {
        c += vcount[b.voff + v];
        if (vcks) h += vcks[b.voff + v];
    }
    for (int o = 16; o > 0; o >>= 1) {
        c += __shfl_down_sync(0xffffffffu, c, o);
        h += __shfl_down_sync(0xffffffffu, h, o);
    }
    if (lane_id() == 0) { sc[threadIdx.x >> 5] = c; sk[threadIdx.x >> 5] = h; }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long tc = 0, th = 0;
        for (uint32_t i = 0; i < (blockDim.x >> 5); i++) { tc += sc[i]; th += sk[i]; }
        out_count[blockIdx.x] = tc;
        if (out_cks) out_cks[blockIdx.x] = th;
    }
}

int launch_union_build(const BatchSrc *src, uint32_t G, uint32_t n_total, uint64_t *urp,
                       uint32_t *ucol, uint32_t *graph_of, uint32_t *idmap, uint8_t *kmap,
                       cudaStream_t s) {
    if (G == 0) return 0;
    k_union_build<<<G, 256, 0, s>>>(src, n_total, urp, ucol, graph_of, idmap, kmap);
    return 1;
}

int launch_graph_sums(const BatchSrc *src, uint32_t G, const unsigned long long *vcount,
                      const unsigned long long *vcks, unsigned long long *out_count,
                      unsigned long long *out_cks, cudaStream_t s) {
    if (G == 0) return 0;
    k_graph_sums<<<G, 256, 0, s>>>(src, vcount, vcks, out_count, out_cks);
    return 1;
}

int launch_exclusive_scan(const uint32_t *in, uint32_t *out, uint32_t n, uint32_t *block_tmp,
                          cudaStream_t s) {
    // exclusive scan; out may alias in.  block_tmp needs ceil(n/2048) +
    // ceil(n/2048^2) + ... words.
    if (n == 0) return 0;
    uint32_t tiles = (n + kScanTile - 1) / kScanTile;
    if (tiles == 1) {
        k_scan_tiles<<<1, kScanThreads, 0, s>>>(in, out, n, nullptr);
        return 1;
    }
    k_scan_tiles<<<tiles, kScanThreads, 0, s>>>(in, out, n, block_tmp);
    int l = 1 + launch_exclusive_scan(block_tmp, block_tmp, tiles, block_tmp + tiles, s);
    k_scan_add<<<tiles, kScanThreads, 0, s>>>(out, n, block_tmp);
    return l + 1;
}

__global__ void k_set_deadline(DevResult *res, unsigned long long limit_ns) {
    res->deadline_ns = limit_ns ? global_ns() + limit_ns : 0ull;
}

int launch_set_deadline(DevResult *res, uint64_t limit_ms, cudaStream_t s) {
    k_set_deadline<<<1, 1, 0, s>>>(res, (unsigned long long)limit_ms * 1000000ull);
    return 1;
}

int launch_validate(const kcl_graph *g, DevResult *res, cudaStream_t s) {
    int grid = grid_for((uint64_t)g->n * 32, kBlock, g->num_sms, 32);
    k_validate<<<grid, kBlock, 0, s>>>(g->n, g->nnz, g->rp, g->col, res);
    return 1;
}

int launch_precore_init(const kcl_graph *g, uint32_t k, Workspace &w, cudaStream_t s) {
    int grid = grid_for(g->n, kBlock, g->num_sms);
    // a threshold of 0 (k = 1: Pre-Core switched off) keeps every vertex, whatever the k map says
    k_precore_init<<<grid, kBlock, 0, s>>>(g->n, g->rp, k - 1, k > 1 ? w.kmap : nullptr, w.alive,
                                           w.cdeg, w.frontier_a, &w.res->frontier);
    return 1;
}

int launch_precore_round(const kcl_graph *g, uint32_t k, const uint32_t *fin, uint32_t nin,
                         uint32_t *fout, Workspace &w, cudaStream_t s) {
    int grid = grid_for((uint64_t)nin * 32, kBlock, g->num_sms, 32);
    k_precore_round<<<grid, kBlock, 0, s>>>(g->rp, g->col, k - 1, k > 1 ? w.kmap : nullptr, fin, nin,
                                            w.alive, w.cdeg, fout, &w.res->frontier);
    return 1;
}

int launch_prelist(const kcl_graph *g, uint32_t k, Workspace &w, int listing, cudaStream_t s) {
    int grid = grid_for(g->n, kBlock, g->num_sms);
    int wgrid = grid_for((uint64_t)g->n * 32, kBlock, g->num_sms, 32);
    k_uf_init<<<grid, kBlock, 0, s>>>(g->n, w.parent, w.comp_n, w.comp_sdeg, w.comp_flag);
    k_uf_hook<<<wgrid, kBlock, 0, s>>>(g->n, g->rp, g->col, w.alive, w.parent);
    k_uf_stats<<<grid, kBlock, 0, s>>>(g->n, w.alive, w.parent, w.cdeg, w.comp_n, w.comp_sdeg);
    k_uf_check<<<grid, kBlock, 0, s>>>(g->n, k, w.kmap, w.alive, w.parent, w.comp_n, w.comp_sdeg,
                                       w.comp_flag, listing ? w.comp_slot : nullptr, w.vcount_pre,
                                       w.res);
    k_uf_remove<<<grid, kBlock, 0, s>>>(g->n, w.alive, w.parent, w.comp_flag);
    return 5;
}

int launch_prelist_emit(const kcl_graph *g, uint32_t k, Workspace &w, uint32_t n_comps,
                        const kcl_ring *ring, cudaStream_t s) {
    if (n_comps == 0) return 0;
    int grid = grid_for(g->n, kBlock, g->num_sms);
    // sizes and offsets of the clique components (by slot)
    uint32_t *sizes = w.hist, *offs = w.hist + n_comps, *fill = w.hist + 2 * n_comps;
    uint32_t *croots = w.frontier_b;
    cudaMemsetAsync(fill, 0, n_comps * sizeof(uint32_t), s);
    k_comp_sizes<<<grid, kBlock, 0, s>>>(g->n, w.comp_flag, w.comp_slot, w.comp_n, sizes, croots);
    int l = 2 + launch_exclusive_scan(sizes, offs, n_comps, w.scan_tmp, s);
    k_comp_gather<<<grid, kBlock, 0, s>>>(g->n, w.parent, w.comp_flag, w.comp_slot, w.alive_core,
                                          offs, fill, w.members);
    k_comp_sort<<<n_comps, 256, 0, s>>>(offs, sizes, w.members);
    const bool to_ring = ring && ring->ids && ring->capacity;
    k_comp_emit<<<n_comps, 256, 0, s>>>(k, w.kmap, offs, sizes, w.members, to_ring ? ring->ids : nullptr,
                                        to_ring ? ring->capacity : 0, to_ring ? ring->wrap : 0,
                                        croots, w.vcks_pre, w.idmap, w.res);
    return l + 3;
}

int launch_degree_key(const kcl_graph *g, Workspace &w, cudaStream_t s) {
    int grid = grid_for(g->n, kBlock, g->num_sms);
    k_degree_key<<<grid, kBlock, 0, s>>>(g->n, w.alive, w.cdeg, w.key);
    return 1;
}

int launch_peel_init(const kcl_graph *g, Workspace &w, cudaStream_t s) {
    int grid = grid_for(g->n, kBlock, g->num_sms);
    k_peel_init<<<grid, kBlock, 0, s>>>(g->n, w.alive, w.cdeg, w.peel_deg, w.key, w.res);
    return 1;
}

int launch_peel_min(const kcl_graph *g, Workspace &w, cudaStream_t s) {
    int grid = grid_for(g->n, kBlock, g->num_sms);
    k_peel_min<<<grid, kBlock, 0, s>>>(g->n, w.alive, w.peel_deg, w.key, w.res);
    return 1;
}

int launch_peel_select_all(const kcl_graph *g, Workspace &w, uint32_t t, uint32_t round,
                           uint32_t *fout, cudaStream_t s) {
    int grid = grid_for(g->n, kBlock, g->num_sms);
    k_peel_select_all<<<grid, kBlock, 0, s>>>(g->n, w.alive, w.peel_deg, w.key, t, round, fout,
                                              &w.res->frontier);
    return 1;
}

int launch_peel_update(const kcl_graph *g, Workspace &w, const uint32_t *fin, uint32_t nin,
                       uint32_t t, uint32_t round, uint32_t *fout, cudaStream_t s) {
    int grid = grid_for((uint64_t)nin * 32, kBlock, g->num_sms, 32);
    k_peel_update<<<grid, kBlock, 0, s>>>(g->rp, g->col, w.alive, w.peel_deg, w.key, fin, nin, t,
                                          round + 1, fout, &w.res->frontier);
    return 1;
}

constexpr int kPeelThreads = 1024;

// Blocks of the cooperative peel for n vertices: one per SM (fewer arrivals
// per grid barrier), none beyond what n needs; -1 if it cannot be resident.
int peel_blocks(int num_sms, uint32_t n) {
    static std::atomic<int> cached{-1};  // several host threads (server slots) call this
    int per_sm = cached.load(std::memory_order_relaxed);
    if (per_sm < 0) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_peel_coop, kPeelThreads, 0) != cudaSuccess) {
            (void)cudaGetLastError();
            b = 0;
        }
        per_sm = b;
        cached.store(b, std::memory_order_relaxed);
    }
    if (per_sm <= 0) return -1;
    int blocks = num_sms;
    const uint64_t need = ((uint64_t)n + kPeelThreads - 1) / kPeelThreads;
    if (need < (uint64_t)blocks) blocks = need ? (int)need : 1;
    return blocks;
}

int launch_peel_coop(const kcl_graph *g, Workspace &w, PeelCtl *ctl, uint32_t *rl0, uint32_t *rl1,
                     uint32_t *bl0, uint32_t *bl1, cudaStream_t s) {
    int blocks = peel_blocks(g->num_sms, g->n);
    if (blocks <= 0) return -1;
    uint32_t n = g->n;
    const uint64_t *rp = g->rp;
    const uint32_t *col = g->col;
    const uint8_t *alive = w.alive;
    const uint32_t *cdeg = w.cdeg;
    uint32_t *pdeg = w.peel_deg, *key = w.key, *fa = w.frontier_a, *fb = w.frontier_b;
    // big rows: longer than 2048 and than 4x the mean degree, so there are at
    // most nnz / big <= n / 4 of them (each list holds n / 2)
    const uint64_t mean = n ? (g->nnz + n - 1) / n : 0;
    uint64_t big = 4 * mean > 2048 ? 4 * mean : 2048;
    void *args[] = {&n, (void *)&rp, (void *)&col, (void *)&alive, (void *)&cdeg, &pdeg, &key, &fa,
                    &fb, &rl0, &rl1, &bl0, &bl1, &big, &ctl};
    if (cudaLaunchCooperativeKernel((const void *)k_peel_coop, blocks, kPeelThreads, args, 0, s) !=
        cudaSuccess)
        return -1;
    return 1;
}

int launch_orient(const kcl_graph *g, uint32_t k, Workspace &w, cudaStream_t s) {
    (void)k;
    int wgrid = grid_for((uint64_t)g->n * 32, kBlock, g->num_sms, 32);
    k_outdeg<<<wgrid, kBlock, 0, s>>>(g->n, g->rp, g->col, w.alive, w.key, w.outdeg, w.res);
    // optr = exclusive scan of outdeg (n + 1 entries; outdeg[n] = 0)
    int l = 1 + launch_exclusive_scan(w.outdeg, w.optr, g->n + 1, w.scan_tmp, s);
    k_outfill<<<wgrid, kBlock, 0, s>>>(g->n, g->rp, g->col, w.alive, w.key, w.optr, w.oadj);
    return l + 1;
}

int launch_roots(const kcl_graph *g, uint32_t k, Workspace &w, uint32_t max_outdeg,
                 uint32_t *class_begin, const uint32_t *class_limits, int n_classes,
                 cudaStream_t s) {
    int grid = grid_for(g->n, kBlock, g->num_sms);
    uint32_t H = max_outdeg + 1;
    uint32_t *hist = w.hist, *offs = w.hist + H + 1, *fill = w.hist + 2 * (H + 1);
    uint32_t *limits = w.hist + 3 * (H + 1);
    cudaMemsetAsync(w.hist, 0, 3 * (H + 1) * sizeof(uint32_t), s);
    cudaMemcpyAsync(limits, class_limits, n_classes * sizeof(uint32_t), cudaMemcpyHostToDevice, s);
    k_root_hist<<<grid, kBlock, 0, s>>>(g->n, k, w.alive, w.outdeg, max_outdeg, hist, w.root_mask,
                                        w.kmap, w.res);
    int l = 1 + launch_exclusive_scan(hist, offs, H + 1, w.scan_tmp, s);
    k_root_scatter<<<grid, kBlock, 0, s>>>(g->n, k, w.alive, w.outdeg, max_outdeg, offs, fill,
                                           w.root_mask, w.kmap, w.roots);
    // class bounds into the tail of hist; n_roots = offs[H]
    uint32_t *cb = w.hist + 3 * (H + 1) + 64;
    k_class_bounds<<<1, 64, 0, s>>>(offs, max_outdeg, limits, n_classes, 0, cb);
    // last entry (n_roots) is patched from DevResult by the host
    cudaMemcpyAsync(class_begin, cb, (n_classes + 1) * sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    return l + 3;
}

}  // namespace kcl

// ======================================= allocation-free degeneracy ordering
// Scratch of kcl_degeneracy_order_noalloc: peel degrees, two frontiers and the
// control block of k_peel_coop for up to KCL_NOALLOC_MAX_VERTICES vertices.
// It is a fixed device array, so the call never allocates; in host code the
// array's name is only a stand-in, and its device address is looked up with
// cudaGetSymbolAddress once per device.
static constexpr size_t kNoAllocWords =
    3 * (size_t)KCL_NOALLOC_MAX_VERTICES + sizeof(kcl::PeelCtl) / sizeof(uint32_t);
static __device__ __align__(256) uint32_t kcl_noalloc_scratch[kNoAllocWords];

namespace {
constexpr int kNoAllocMaxDevices = 64;
std::mutex noalloc_mu;
uint32_t *noalloc_ptr[kNoAllocMaxDevices];
int noalloc_blocks[kNoAllocMaxDevices];

// Device address of the scratch array and the cooperative grid size for the
// current device, set up on the first call on that device.
kcl_status noalloc_setup(uint32_t **ptr, int *blocks) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) {
        (void)cudaGetLastError();
        return KCL_ECUDA;
    }
    std::lock_guard<std::mutex> lock(noalloc_mu);
    if (!noalloc_ptr[dev]) {
        uint32_t *p = nullptr;
        if (cudaGetSymbolAddress((void **)&p, kcl_noalloc_scratch) != cudaSuccess || !p) {
            (void)cudaGetLastError();
            return KCL_ECUDA;
        }
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
            (void)cudaGetLastError();
            return KCL_ECUDA;
        }
        const int blocks = kcl::peel_blocks(sms, KCL_NOALLOC_MAX_VERTICES);
        if (blocks <= 0) return KCL_ECUDA;
        noalloc_blocks[dev] = blocks;
        noalloc_ptr[dev] = p;
    }
    *ptr = noalloc_ptr[dev];
    *blocks = noalloc_blocks[dev];
    return KCL_OK;
}
}  // namespace

extern "C" kcl_status kcl_degeneracy_order_noalloc(uint32_t n, const uint64_t *row_ptr,
                                                   const uint32_t *col, const uint8_t *alive,
                                                   const uint32_t *degree, uint32_t *round_out,
                                                   void *stream) {
    if (n > KCL_NOALLOC_MAX_VERTICES) return KCL_ESIZE;
    if (n == 0) return KCL_OK;
    if (!row_ptr || !col || !alive || !degree || !round_out) return KCL_EINVAL;
    uint32_t *S = nullptr;
    int blocks = 0;
    kcl_status st = noalloc_setup(&S, &blocks);
    if (st != KCL_OK) return st;
    uint64_t need = ((uint64_t)n + kcl::kPeelThreads - 1) / kcl::kPeelThreads;
    if (need < (uint64_t)blocks) blocks = (int)need;
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t *pdeg = S;
    uint32_t *fa = S + KCL_NOALLOC_MAX_VERTICES;
    uint32_t *fb = S + 2 * (size_t)KCL_NOALLOC_MAX_VERTICES;
    kcl::PeelCtl *ctl = reinterpret_cast<kcl::PeelCtl *>(S + 3 * (size_t)KCL_NOALLOC_MAX_VERTICES);
    // the control block keeps the previous call's contents: clear it (minv
    // starts at all ones, everything else at zero)
    if (cudaMemsetAsync(ctl, 0, sizeof(kcl::PeelCtl), s) != cudaSuccess ||
        cudaMemsetAsync(ctl->minv, 0xFF, sizeof(ctl->minv), s) != cudaSuccess) {
        (void)cudaGetLastError();
        return KCL_ECUDA;
    }
    uint32_t nn = n;
    const uint64_t *rp = row_ptr;
    const uint32_t *c = col;
    const uint8_t *al = alive;
    const uint32_t *deg = degree;
    uint32_t *key = round_out;
    uint32_t *rl0 = nullptr, *rl1 = nullptr;  // no room for remaining lists: full scans
    uint32_t *bl0 = nullptr, *bl1 = nullptr;  // nor for big-row lists: a warp per frontier vertex
    uint64_t big = ~0ull;
    void *args[] = {&nn, (void *)&rp, (void *)&c, (void *)&al, (void *)&deg, &pdeg, &key, &fa, &fb,
                    &rl0, &rl1, &bl0, &bl1, &big, &ctl};
    if (cudaLaunchCooperativeKernel((const void *)kcl::k_peel_coop, blocks, kcl::kPeelThreads, args, 0, s) !=
        cudaSuccess) {
        (void)cudaGetLastError();
        return KCL_ECUDA;
    }
    unsigned err = 0;
    if (cudaMemcpyAsync(&err, &ctl->error, sizeof(err), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        (void)cudaGetLastError();
        return KCL_ECUDA;
    }
    return err ? KCL_ETIMEOUT : KCL_OK;
}
