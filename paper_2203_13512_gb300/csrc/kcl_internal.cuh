// Internal declarations shared by the library's CUDA translation units.
// Not part of the public ABI (include/kcl.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "../../include/kcl.h"

namespace kcl {

constexpr int kWarp = 32;

// Device status word bits (recorded by kernels, turned into a kcl_status).
enum : uint32_t {
    DEV_ERR_NONE = 0,
    DEV_ERR_INVALID_GRAPH = 1u << 0,
    DEV_ERR_OUTDEG_LIMIT = 1u << 1,
    DEV_ERR_OVERFLOW = 1u << 2,
    DEV_ERR_INTERNAL = 1u << 3,
    DEV_ERR_TIMEOUT = 1u << 4,  // the call's time limit passed (kcl_set_time_limit)
};

// Result words written by the device and read back once per call.
struct DevResult {
    unsigned long long count;        // k-cliques found by the listing kernels
    unsigned long long checksum;     // sum of clique hashes (list mode)
    unsigned long long emitted;      // clique records claimed in the ring
    unsigned long long pre_count;    // k-cliques of Pre-List clique components
    unsigned long long pre_checksum;
    unsigned long long count_carry;  // set when an addition to `count` wrapped
    unsigned int status;             // DEV_ERR_* bits
    unsigned int frontier;           // size of the next peel frontier
    unsigned int max_outdeg;         // Delta of the DAG
    unsigned int n_roots;            // roots with d+ >= k-1
    unsigned int min_deg;            // minimum current degree (degeneracy peel)
    unsigned int remaining;          // vertices not yet peeled
    unsigned int n_clique_comps;     // components removed by Pre-List
    unsigned int pad;
    unsigned long long deadline_ns;  // %globaltimer value after which listing stops (0: none)
};

// Control block of the single-launch degeneracy peel: grid barrier state,
// the number of vertices to peel, frontier sizes (rotating over three rounds),
// remaining-list sizes and minimum degrees (alternating over threshold
// levels).  All zero at launch except minv, all ones.
struct PeelCtl {
    unsigned bar_count, bar_gen, error, remaining;
    unsigned fcnt[3];   // frontier sizes (vertices up to the big-degree threshold)
    unsigned rcnt[2];
    unsigned minv[2];
    unsigned bcnt[3];   // big-vertex frontier sizes (rotating like fcnt)
};

// One graph of a batch: its device CSR and its place in the disjoint union.
struct BatchSrc {
    const uint64_t *rp;
    const uint32_t *col;
    uint32_t n;
    uint32_t voff;
    uint64_t nnz;
    uint64_t eoff;
    uint32_t k;     // the graph's k (written to the union's k map)
    uint32_t pad;
};

// Workspace owned by a graph, grown on demand and reused across calls.
struct Workspace {
    uint8_t *alive = nullptr;        // n
    uint8_t *alive_core = nullptr;   // n (copy after Pre-Core, for stage info)
    uint32_t *cdeg = nullptr;        // n: current degree in the alive subgraph
    uint32_t *key = nullptr;         // n: ordering key (degree or peel round)
    uint32_t *peel_deg = nullptr;    // n: degrees during the degeneracy peel
    uint32_t *frontier_a = nullptr;  // n
    uint32_t *frontier_b = nullptr;  // n
    uint32_t *parent = nullptr;      // n: union-find forest (Pre-List)
    uint32_t *comp_n = nullptr;      // n: component sizes (by root)
    unsigned long long *comp_sdeg = nullptr;  // n: component degree sums
    uint32_t *comp_flag = nullptr;   // n: 1 = clique component root
    uint32_t *outdeg = nullptr;      // n
    uint32_t *optr = nullptr;        // n + 1: out-CSR offsets
    uint32_t *oadj = nullptr;        // nnz/2: out-neighbours, ascending id
    uint32_t *roots = nullptr;       // n: roots sorted by d+ descending
    uint32_t *hist = nullptr;        // histogram / scan scratch
    uint32_t *scan_tmp = nullptr;    // block sums for scans
    unsigned int *queue = nullptr;   // per-class work counters
    uint32_t *members = nullptr;     // n: clique-component members (listing)
    uint32_t *comp_slot = nullptr;   // n: clique-component slot (listing)
    uint32_t *arena = nullptr;       // global scratch for large subproblems
    unsigned long long *slots = nullptr;  // work-splitting slots, one per CTA of a launch
    size_t arena_words = 0;
    DevResult *res = nullptr;
    DevResult *h_res = nullptr;      // pinned host mirror
    PeelCtl *peel = nullptr;         // single-launch peel control block
    unsigned long long *vcount_pre = nullptr;  // batch: Pre-List counts by component root
    unsigned long long *vcks_pre = nullptr;    // batch: Pre-List checksums by component root
    const uint32_t *idmap = nullptr;           // batch: union vertex -> graph's own id
    const uint8_t *root_mask = nullptr;        // kcl_count_roots: only these roots (null: all)
    const uint8_t *kmap = nullptr;             // batch: union vertex -> k of its graph (null: one k)
    uint32_t n_cap = 0;
    uint64_t nnz_cap = 0;
};

struct Timing {
    int enabled = 0;
    cudaEvent_t ev[2 * KCL_NUM_STAGES] = {};
    cudaEvent_t cev[2 * KCL_MAX_CLASSES] = {};  // around each class's listing launch
    float ms[KCL_NUM_STAGES] = {};
    uint32_t launches[KCL_NUM_STAGES] = {};
    uint32_t n_classes = 0;
    uint32_t class_lo[KCL_MAX_CLASSES] = {}, class_hi[KCL_MAX_CLASSES] = {};
    uint32_t class_roots[KCL_MAX_CLASSES] = {};
    float class_ms[KCL_MAX_CLASSES] = {};
};

}  // namespace kcl

struct kcl_graph {
    uint32_t n = 0;
    uint64_t nnz = 0;          // directed entries = 2 |E|
    int device = 0;
    int num_sms = 0;
    cudaStream_t stream = nullptr;
    uint64_t *rp = nullptr;    // device CSR
    uint32_t *col = nullptr;
    uint32_t max_deg = 0;
    bool owns_csr = true;      // false for a view that shares another graph's CSR
    kcl::Workspace ws;
    kcl::Timing timing;
    kcl_tuning tuning = {};  // listing-kernel knobs (results never depend on them)
    uint32_t options = 0;    // KCL_OPT_* ablation switches
    uint64_t time_limit_ms = 0;  // listing-stage time limit (0: none)
};

namespace kcl {

// ------------------------------------------------------------ utilities
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    // SplitMix64 output finaliser (Steele, Lea & Flood 2014)
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t hash_seed(uint32_t k) {
    return mix64(0x9E3779B97F4A7C15ull ^ (uint64_t)k);
}

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// Hash of the clique R + {a, b} (a != b, neither in R): the SplitMix64
// chain over its ids in ascending order, R's k-2 ids ascending in
// sortedR[0..nr).  The ids are merged on the fly in exactly k = nr + 2 steps
// with selects only, so the lanes of a warp stay converged through the k
// mixing rounds and nothing spills to local memory; when out is not null
// the ascending record is written there (k ids).  seed = hash_seed(k).
__device__ __forceinline__ uint64_t clique_hash2(const uint32_t *sortedR, uint32_t nr, uint32_t a,
                                                 uint32_t b, uint64_t seed, uint32_t *out) {
    uint32_t e = a < b ? a : b;        // the smaller extra id first
    const uint32_t hi = a < b ? b : a;
    uint32_t ne = 2, ri = 0;
    uint64_t h = seed;
    for (uint32_t z = 0; z < nr + 2; z++) {
        const uint32_t r = ri < nr ? sortedR[ri] : 0xFFFFFFFFu;
        const bool take_e = ne > 0 && e < r;
        const uint32_t x = take_e ? e : r;
        ri += take_e ? 0u : 1u;
        ne -= take_e ? 1u : 0u;
        e = take_e ? hi : e;
        h = mix64(h ^ (uint64_t)x);
        if (out) out[z] = x;
    }
    return h;
}

// A lane's cliques R + {a, b} within one batch of records (listing mode):
// the lane writes records lane, lane + 32, lane + 64, ... of the batch, so
// the warp's stores at each step are 32 consecutive records.  NR = k - 2 > 0
// holds R's ids in registers and merges each clique with selects in a fully
// unrolled loop (the same k SplitMix64 rounds over the ascending ids as
// clique_hash2, and the same record); NR = 0 is the runtime-k form.
template <int NR>
struct CliqueOut {
    static constexpr int NRR = NR > 0 ? NR : 1;
    uint32_t R[NRR];
    const uint32_t *sortedR;
    uint64_t seed;
    uint32_t *ring;
    unsigned long long cap, s;  // s: this lane's next record index in the ring
    int wrap;
    uint32_t k;
    bool vec;  // records 16-byte (k = 4) or 8-byte (k = 6) aligned

    // slot0: the batch's first record (ring_base); first: this lane's
    // offset from it.
    __device__ __forceinline__ void init(const uint32_t *sR, uint32_t kk, uint32_t *rg,
                                         unsigned long long capacity, int wr,
                                         unsigned long long slot0, uint32_t first) {
        sortedR = sR;
        k = kk;
        seed = hash_seed(kk);
        ring = rg;
        cap = capacity;
        wrap = wr;
        if constexpr (NR > 0) {
#pragma unroll
            for (int i = 0; i < NR; i++) R[i] = sR[i];
        }
        s = slot0 + first;
        if (wrap && s >= cap) s %= cap;
        const uintptr_t al = reinterpret_cast<uintptr_t>(rg);
        vec = (NR == 2 && (al & 15u) == 0) || (NR == 4 && (al & 7u) == 0);
    }

    __device__ __forceinline__ uint32_t *rec() const {
        if (!ring || (!wrap && s >= cap)) return nullptr;
        return ring + s * k;
    }

    __device__ __forceinline__ void advance() {
        s += 32;
        if (wrap && s >= cap) {
            s -= cap;
            if (s >= cap) s %= cap;  // only for rings smaller than 32 records
        }
    }

    // Hash of R + {a, b} (a != b, neither in R), its record written when
    // the ring keeps it; then moves on to the lane's next record.
    __device__ __forceinline__ uint64_t put(uint32_t a, uint32_t b) {
        uint32_t *out = rec();
        uint64_t h;
        if constexpr (NR == 0) {
            h = clique_hash2(sortedR, k - 2, a, b, seed, out);
        } else {
            uint32_t e = a < b ? a : b, e2 = a < b ? b : a;
            uint32_t q[NR], x[NR + 2];
#pragma unroll
            for (int i = 0; i < NR; i++) q[i] = R[i];
            h = seed;
#pragma unroll
            for (int z = 0; z < NR + 2; z++) {
                // ids are < 2^32 - 1, so 0xFFFFFFFF marks an exhausted source
                const bool te = e < q[0];
                x[z] = te ? e : q[0];
                e = te ? e2 : e;
                e2 = te ? 0xFFFFFFFFu : e2;
#pragma unroll
                for (int i = 0; i + 1 < NR; i++) q[i] = te ? q[i] : q[i + 1];
                q[NR - 1] = te ? q[NR - 1] : 0xFFFFFFFFu;
                h = mix64(h ^ (uint64_t)x[z]);
            }
            if (out) {
                if constexpr (NR == 2) {
                    if (vec) {
                        *reinterpret_cast<uint4 *>(out) = make_uint4(x[0], x[1], x[2], x[3]);
                    } else {
#pragma unroll
                        for (int z = 0; z < 4; z++) out[z] = x[z];
                    }
                } else if constexpr (NR == 4) {
                    if (vec) {
#pragma unroll
                        for (int z = 0; z < 6; z += 2)
                            reinterpret_cast<uint2 *>(out)[z >> 1] = make_uint2(x[z], x[z + 1]);
                    } else {
#pragma unroll
                        for (int z = 0; z < 6; z++) out[z] = x[z];
                    }
                } else {
#pragma unroll
                    for (int z = 0; z < NR + 2; z++) out[z] = x[z];
                }
            }
        }
        advance();
        return h;
    }
};

// Ring records of a batch: the batch claims `count` consecutive record
// indices from `emitted` (one atomic), and its first index becomes the base
// of ring_rec -- taken mod capacity once per batch when the ring wraps, so
// no clique pays a 64-bit division.
__device__ __forceinline__ unsigned long long ring_base(unsigned long long first,
                                                        unsigned long long capacity, int wrap) {
    return wrap ? first % capacity : first;
}

// Record `off` of a batch whose base is `base` (null when it does not fit
// and the ring does not wrap).
__device__ __forceinline__ uint32_t *ring_rec(uint32_t *ring, unsigned long long capacity, int wrap,
                                              unsigned long long base, uint32_t off, uint32_t k) {
    if (!ring) return nullptr;
    unsigned long long s = base + off;
    if (wrap) {
        if (s >= capacity) s -= capacity;
        if (s >= capacity) s %= capacity;  // only for rings smaller than a batch
    } else if (s >= capacity) {
        return nullptr;
    }
    return ring + s * k;
}

// ---------------------------------------------------------- work splitting
// Heavy roots are shared between CTAs (the EdgeParallel units of Section
// IX-C: a root's first-level children, the edges <u, v>).  Every CTA of a
// CTA-per-root launch publishes the root it works on in its slot, one 64-bit
// word: (root position << 32) | (first-level children << 16) | next child.
// The CTA's warps take children by advancing `next`; a CTA that finds the
// root queue empty picks the slot with the most children left, rebuilds that
// root's subproblem (the build is deterministic, so the child list is the
// same) and takes children from the same slot.  Claims are single
// compare-and-swaps that fail once the slot holds another root, so no
// child is taken twice or lost, and nothing waits on another CTA.
constexpr unsigned long long kSlotIdle = ~0ull;
constexpr uint32_t kNoChild = 0xFFFFFFFFu;

__device__ __forceinline__ void split_publish(unsigned long long *slot, uint32_t pos, uint32_t nch) {
    atomicExch(slot, ((unsigned long long)pos << 32) | ((unsigned long long)nch << 16));
}

// Next child (its position in the child list) of root position `pos`
// published in `slot`, or kNoChild when none is left or the slot moved on.
__device__ __forceinline__ uint32_t split_claim(unsigned long long *slot, uint32_t pos) {
    unsigned long long old = *reinterpret_cast<volatile unsigned long long *>(slot);
    for (uint32_t tries = 0; tries < (1u << 20); tries++) {  // bounded retries under contention
        if ((uint32_t)(old >> 32) != pos) return kNoChild;
        const uint32_t nch = (uint32_t)(old >> 16) & 0xFFFFu, next = (uint32_t)old & 0xFFFFu;
        if (next >= nch) return kNoChild;
        const unsigned long long got = atomicCAS(slot, old, old + 1);
        if (got == old) return next;
        old = got;
    }
    return kNoChild;
}

// Run by one warp: the slot (other than `me`) with the most children left,
// at least min_left; -1 if none.  *pos receives its root position.
__device__ __forceinline__ int split_pick(unsigned long long *slots, uint32_t nslots, uint32_t me,
                                          uint32_t min_left, uint32_t *pos) {
    const unsigned lane = threadIdx.x & 31u;
    uint32_t best_left = 0, best = 0xFFFFFFFFu, best_pos = 0;
    for (uint32_t j = lane; j < nslots; j += 32) {
        const unsigned long long v = *reinterpret_cast<volatile unsigned long long *>(slots + j);
        if (v == kSlotIdle || j == me) continue;
        const uint32_t nch = (uint32_t)(v >> 16) & 0xFFFFu, next = (uint32_t)v & 0xFFFFu;
        const uint32_t left = nch > next ? nch - next : 0u;
        if (left >= min_left && left > best_left) { best_left = left; best = j; best_pos = (uint32_t)(v >> 32); }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint32_t l2 = __shfl_xor_sync(0xffffffffu, best_left, o);
        const uint32_t b2 = __shfl_xor_sync(0xffffffffu, best, o);
        const uint32_t p2 = __shfl_xor_sync(0xffffffffu, best_pos, o);
        if (l2 > best_left || (l2 == best_left && b2 < best)) { best_left = l2; best = b2; best_pos = p2; }
    }
    *pos = best_pos;
    return best_left ? (int)best : -1;
}

// ------------------------------------------------------------- time limit
// The listing kernels stop taking work once the device's global timer passes
// DevResult::deadline_ns (set when the listing stage starts; 0 = no limit)
// and record DEV_ERR_TIMEOUT; the call then returns KCL_ETIMEOUT.
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool past_deadline(unsigned long long deadline, DevResult *res) {
    if (!deadline || global_ns() <= deadline) return false;
    atomicOr(&res->status, DEV_ERR_TIMEOUT);
    return true;
}

// The same test taken once per warp (lane 0 reads the timer), so the warp
// stays converged.
__device__ __forceinline__ bool warp_past_deadline(unsigned long long deadline, DevResult *res) {
    bool late = false;
    if (deadline && (threadIdx.x & 31u) == 0) late = past_deadline(deadline, res);
    return __shfl_sync(0xffffffffu, late, 0);
}

// Inclusive prefix sum over the 32 lanes of a warp (all lanes active).
__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x) {
    const unsigned lane = lane_id();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= (unsigned)o) x += y;
    }
    return x;
}

// Add to a 64-bit counter and flag a wrap-around in `carry`.
__device__ __forceinline__ void add_count(unsigned long long *dst, unsigned long long *carry,
                                          unsigned long long x) {
    if (x == 0) return;
    unsigned long long old = atomicAdd(dst, x);
    if (old + x < old) atomicExch(carry, 1ull);
}

// Open-addressing hash table (linear probing) of a vertex set held by one
// warp: ids -> local index.  T is a power of two >= 2 * |set|, so every probe
// sequence ends at an empty slot.
constexpr uint32_t kHashEmpty = 0xFFFFFFFFu;

__device__ __forceinline__ uint32_t hash_slot(uint32_t id, uint32_t shift) {
    return (id * 2654435761u) >> shift;  // Knuth multiplicative hashing
}

// Build the table for ids[0..d) (distinct) with the whole warp.
__device__ __forceinline__ void warp_hash_build(const uint32_t *ids, uint32_t d, uint32_t *hk,
                                                uint16_t *hv, uint32_t T, uint32_t shift) {
    for (uint32_t i = lane_id(); i < T; i += 32) hk[i] = kHashEmpty;
    __syncwarp();
    for (uint32_t i = lane_id(); i < d; i += 32) {
        uint32_t key = ids[i], h = hash_slot(key, shift);
        while (atomicCAS(&hk[h], kHashEmpty, key) != kHashEmpty) h = (h + 1) & (T - 1);
        hv[h] = (uint16_t)i;
    }
    __syncwarp();
}

// Local index of `id`, or -1.
__device__ __forceinline__ int hash_find(const uint32_t *hk, const uint16_t *hv, uint32_t T,
                                         uint32_t shift, uint32_t id) {
    uint32_t h = hash_slot(id, shift);
    for (;;) {
        uint32_t k = hk[h];
        if (k == id) return (int)hv[h];
        if (k == kHashEmpty) return -1;
        h = (h + 1) & (T - 1);
    }
}

// Hash table slots a layout for up to D vertices must hold: the smallest
// power of two >= 2 D (hash_size's T for every d <= D).
__host__ __device__ inline uint32_t hash_cap(uint32_t D) {
    uint32_t t = 2;
    while (t < 2 * D) t <<= 1;
    return t;
}

// Smallest power of two >= 2 * d (at least 2) and its hash shift.
__device__ __forceinline__ void hash_size(uint32_t d, uint32_t *T, uint32_t *shift) {
    uint32_t t = 2, lg = 1;
    while (t < 2 * d) { t <<= 1; lg++; }
    *T = t;
    *shift = 32 - lg;
}

// Largest dynamic shared memory a block may opt in to on the current device.
// Kernels get their MaxDynamicSharedMemorySize attribute set to this value
// (never to a call-specific size): the attribute is per-function state, and
// calls running concurrently on several host threads must not shrink it
// under each other.
inline int max_dynamic_smem() {
    static std::atomic<int> cached[64];  // 0 = not yet read (several host threads call this)
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        dev = 0;
    }
    if (dev >= 0 && dev < 64) {
        const int c = cached[dev].load(std::memory_order_relaxed);
        if (c) return c;
    }
    int v = 48 * 1024;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        (void)cudaGetLastError();
        v = 48 * 1024;
    }
    if (dev >= 0 && dev < 64) cached[dev].store(v, std::memory_order_relaxed);
    return v;
}

// Let `kern` use as much dynamic shared memory as the device allows next to
// its static shared memory.  Returns false if the attribute cannot be set.
template <typename K>
inline bool allow_max_smem(K kern) {
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    int lim = max_dynamic_smem() - (int)fa.sharedSizeBytes;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return true;
}

// ------------------------------------------------------ host-side launchers
// Every launcher enqueues on `s` and returns the number of kernel launches.

// kcl_prep.cu
int launch_validate(const kcl_graph *g, DevResult *res, cudaStream_t s);
int launch_degrees(const kcl_graph *g, uint32_t *deg, cudaStream_t s);
int launch_precore_init(const kcl_graph *g, uint32_t k, Workspace &w, cudaStream_t s);
int launch_precore_round(const kcl_graph *g, uint32_t k, const uint32_t *fin, uint32_t nin,
                         uint32_t *fout, Workspace &w, cudaStream_t s);
int launch_prelist(const kcl_graph *g, uint32_t k, Workspace &w, int listing, cudaStream_t s);
int launch_prelist_emit(const kcl_graph *g, uint32_t k, Workspace &w, uint32_t n_comps,
                        const kcl_ring *ring, cudaStream_t s);
int launch_degree_key(const kcl_graph *g, Workspace &w, cudaStream_t s);
int launch_peel_init(const kcl_graph *g, Workspace &w, cudaStream_t s);
int launch_peel_select_all(const kcl_graph *g, Workspace &w, uint32_t t, uint32_t round,
                           uint32_t *fout, cudaStream_t s);
int launch_peel_update(const kcl_graph *g, Workspace &w, const uint32_t *fin, uint32_t nin,
                       uint32_t t, uint32_t round, uint32_t *fout, cudaStream_t s);
int launch_peel_min(const kcl_graph *g, Workspace &w, cudaStream_t s);
// Whole degeneracy peel in one cooperative launch; -1 if it cannot launch.
// rl0/rl1: two n-entry arrays for the compacted remaining-vertex lists (or
// both null: every threshold rise scans all n vertices); bl0/bl1: two
// n/2-entry arrays for the frontier's big-degree vertices, whose rows the
// whole grid walks together (or null: every frontier vertex takes one warp).
int launch_peel_coop(const kcl_graph *g, Workspace &w, PeelCtl *ctl, uint32_t *rl0, uint32_t *rl1,
                     uint32_t *bl0, uint32_t *bl1, cudaStream_t s);
int launch_orient(const kcl_graph *g, uint32_t k, Workspace &w, cudaStream_t s);
int launch_roots(const kcl_graph *g, uint32_t k, Workspace &w, uint32_t max_outdeg,
                 uint32_t *class_begin, const uint32_t *class_limits, int n_classes,
                 cudaStream_t s);
int launch_exclusive_scan(const uint32_t *in, uint32_t *out, uint32_t n, uint32_t *block_tmp,
                          cudaStream_t s);
// res->deadline_ns = now + limit_ms (or 0 when limit_ms is 0).
int launch_set_deadline(DevResult *res, uint64_t limit_ms, cudaStream_t s);
int launch_union_build(const BatchSrc *src, uint32_t G, uint32_t n_total, uint64_t *urp,
                       uint32_t *ucol, uint32_t *graph_of, uint32_t *idmap, uint8_t *kmap,
                       cudaStream_t s);
int launch_graph_sums(const BatchSrc *src, uint32_t G, const unsigned long long *vcount,
                      const unsigned long long *vcks, unsigned long long *out_count,
                      unsigned long long *out_cks, cudaStream_t s);

// kcl_bitcol.cu
struct ListArgs {
    uint32_t *ring = nullptr;
    unsigned long long capacity = 0;
    int wrap = 0;
    int listing = 0;
    unsigned long long *per_root = nullptr;
    unsigned long long *per_root_cks = nullptr;  // listing: checksum per root
    const uint32_t *idmap = nullptr;             // listing: vertex -> output id
    cudaEvent_t *class_ev = nullptr;             // timing: 2 events per class, or null
    uint32_t max_outdeg = 0;                     // largest root out-degree of the call
};
// Slots for the work splitting of one launch (at most this many CTAs).
constexpr uint32_t kMaxSplitSlots = 4096;
// Records class_ev[2c] / [2c+1] (when timing) around the launch of class c.
inline void class_mark(const ListArgs &la, int c, int end, cudaStream_t s) {
    if (la.class_ev) cudaEventRecord(la.class_ev[2 * c + end], s);
}
int bitcol_classes(uint32_t *limits, int max);
// One root's colouring by the listing path's subproblem builder (parity
// checks); arena: bitcol_colours_arena_words(d) words.  -1: cannot launch.
size_t bitcol_colours_arena_words(uint32_t d);
int launch_bitcol_colours(const Workspace &w, uint32_t u, uint32_t d, uint32_t *arena,
                          uint32_t *out_nbr, uint32_t *out_colour, cudaStream_t s);
int launch_bitcol(const kcl_graph *g, uint32_t k, Workspace &w, const uint32_t *class_begin,
                  int n_classes, const ListArgs &la, cudaStream_t s);

// kcl_sdegree.cu
int sdegree_classes(uint32_t *limits, int max);
size_t sdegree_arena_words(uint32_t k, int num_sms, uint32_t max_outdeg);
size_t bitcol_arena_words(uint32_t k, int num_sms, uint32_t max_outdeg);
int launch_sdegree(const kcl_graph *g, uint32_t k, Workspace &w, const uint32_t *class_begin,
                   int n_classes, const ListArgs &la, cudaStream_t s);

}  // namespace kcl
