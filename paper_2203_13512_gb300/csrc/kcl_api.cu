// C ABI of the library (include/kcl.h): graph loading and validation, and the
// host-side orchestration of one k-clique call:
//   stage 0  Pre-Core (Algorithm 3): frontier rounds until no vertex falls
//            below degree k-1;
//   stage 1  Pre-List (Algorithm 4): clique components counted by C(n_c, k)
//            (and enumerated in listing mode), then removed;
//   stage 2  orientation: degree key (Section VI-B) or degeneracy peel rounds
//            (Algorithm 6), out-neighbour CSR, roots sorted by out-degree;
//   stage 3  listing kernels: SDegreeList (Algorithm 5) or subgraph build +
//            colouring + BitColList (Algorithm 6), one launch per out-degree
//            class.
// Every kernel runs on the graph's stream; the host reads back small status
// words between stages (frontier sizes, Delta, class boundaries).
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <new>
#include <utility>
#include <vector>

#include "kcl_internal.cuh"

using namespace kcl;

namespace {

#define KCL_CK(expr)                                                     \
    do {                                                                 \
        cudaError_t e_ = (expr);                                         \
        if (e_ != cudaSuccess) {                                         \
            (void)cudaGetLastError();                                    \
            return KCL_ECUDA;                                            \
        }                                                                \
    } while (0)

#define KCL_TRY(expr)                     \
    do {                                  \
        kcl_status s_ = (expr);           \
        if (s_ != KCL_OK) return s_;      \
    } while (0)

template <typename T>
kcl_status dev_alloc(T **p, size_t count) {
    if (*p) {
        cudaFree(*p);
        *p = nullptr;
    }
    if (count == 0) count = 1;
    if (cudaMalloc((void **)p, count * sizeof(T)) != cudaSuccess) {
        (void)cudaGetLastError();
        *p = nullptr;
        return KCL_ENOMEM;
    }
    return KCL_OK;
}

void free_workspace(Workspace &w) {
    void *ptrs[] = {w.alive, w.alive_core, w.cdeg, w.key, w.peel_deg, w.frontier_a, w.frontier_b,
                    w.parent, w.comp_n, w.comp_sdeg, w.comp_flag, w.outdeg, w.optr, w.oadj,
                    w.roots, w.hist, w.scan_tmp, w.queue, w.members, w.comp_slot, w.arena, w.res,
                    w.peel, w.slots};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (w.h_res) cudaFreeHost(w.h_res);
    w = Workspace();
}

// Grow the workspace to at least g's size.  Capacities only grow (by at least
// half again), so handles that move between graphs of different sizes (batch
// unions, server slots) settle instead of reallocating on every call.
kcl_status ensure_workspace(kcl_graph *g) {
    Workspace &w = g->ws;
    if (w.res && w.n_cap >= g->n && w.nnz_cap >= g->nnz) return KCL_OK;
    uint32_t n_new = g->n;
    uint64_t nnz_new = g->nnz;
    if (w.res) {
        n_new = (uint32_t)std::min<uint64_t>(0xFFFFFFF0ull, std::max<uint64_t>(g->n, w.n_cap + w.n_cap / 2));
        nnz_new = std::max<uint64_t>(g->nnz, w.nnz_cap + w.nnz_cap / 2);
    }
    size_t arena_words = w.arena_words;
    uint32_t *arena = w.arena;
    w.arena = nullptr;
    free_workspace(w);
    w.arena = arena;  // the arena is sized separately (ensure_arena)
    w.arena_words = arena_words;
    size_t n = (size_t)n_new + 1;
    size_t half = nnz_new / 2 + 1;
    KCL_TRY(dev_alloc(&w.alive, n));
    KCL_TRY(dev_alloc(&w.alive_core, n));
    KCL_TRY(dev_alloc(&w.cdeg, n));
    KCL_TRY(dev_alloc(&w.key, n));
    KCL_TRY(dev_alloc(&w.peel_deg, n));
    KCL_TRY(dev_alloc(&w.frontier_a, n));
    KCL_TRY(dev_alloc(&w.frontier_b, n));
    KCL_TRY(dev_alloc(&w.parent, n));
    KCL_TRY(dev_alloc(&w.comp_n, n));
    KCL_TRY(dev_alloc(&w.comp_sdeg, n));
    KCL_TRY(dev_alloc(&w.comp_flag, n));
    KCL_TRY(dev_alloc(&w.outdeg, n + 1));
    KCL_TRY(dev_alloc(&w.optr, n + 1));
    KCL_TRY(dev_alloc(&w.oadj, half));
    KCL_TRY(dev_alloc(&w.roots, n));
    KCL_TRY(dev_alloc(&w.hist, 3 * n + 1024));
    KCL_TRY(dev_alloc(&w.scan_tmp, n / 1024 + 1024));
    KCL_TRY(dev_alloc(&w.queue, 64));
    KCL_TRY(dev_alloc(&w.members, n));
    KCL_TRY(dev_alloc(&w.comp_slot, n));
    KCL_TRY(dev_alloc(&w.res, 1));
    KCL_TRY(dev_alloc(&w.peel, 1));
    KCL_TRY(dev_alloc(&w.slots, kMaxSplitSlots));
    if (cudaMallocHost((void **)&w.h_res, sizeof(DevResult)) != cudaSuccess) {
        (void)cudaGetLastError();
        w.h_res = nullptr;
        return KCL_ENOMEM;
    }
    // on the graph's own stream: a server slot's stream does not wait for
    // the legacy default stream, so a plain cudaMemset could land after
    // this call's kernels have written outdeg
    KCL_CK(cudaMemsetAsync(w.outdeg, 0, (n + 1) * sizeof(uint32_t), g->stream));
    w.n_cap = n_new;
    w.nnz_cap = nnz_new;
    return KCL_OK;
}

kcl_status ensure_arena(kcl_graph *g, size_t words) {
    Workspace &w = g->ws;
    if (words <= w.arena_words) return KCL_OK;
    KCL_TRY(dev_alloc(&w.arena, words));
    w.arena_words = words;
    return KCL_OK;
}

// Read the device result block into the pinned host mirror.
kcl_status read_result(kcl_graph *g) {
    KCL_CK(cudaMemcpyAsync(g->ws.h_res, g->ws.res, sizeof(DevResult), cudaMemcpyDeviceToHost,
                           g->stream));
    KCL_CK(cudaStreamSynchronize(g->stream));
    return KCL_OK;
}

kcl_status read_u32(kcl_graph *g, const unsigned *dev_field, uint32_t *out) {
    unsigned *h = reinterpret_cast<unsigned *>(reinterpret_cast<char *>(g->ws.h_res) +
                                               (reinterpret_cast<const char *>(dev_field) -
                                                reinterpret_cast<const char *>(g->ws.res)));
    KCL_CK(cudaMemcpyAsync(h, dev_field, sizeof(unsigned), cudaMemcpyDeviceToHost, g->stream));
    KCL_CK(cudaStreamSynchronize(g->stream));
    *out = *h;
    return KCL_OK;
}

kcl_status set_u32(kcl_graph *g, unsigned *dev_field, uint32_t value) {
    if (value == 0) {
        KCL_CK(cudaMemsetAsync(dev_field, 0, sizeof(unsigned), g->stream));
    } else {
        KCL_CK(cudaMemsetAsync(dev_field, 0xFF, sizeof(unsigned), g->stream));
        if (value != 0xFFFFFFFFu) return KCL_EINVAL;
    }
    return KCL_OK;
}

struct StageTimer {
    kcl_graph *g;
    explicit StageTimer(kcl_graph *gg) : g(gg) {
        for (int i = 0; i < KCL_NUM_STAGES; i++) {
            g->timing.ms[i] = 0.f;
            g->timing.launches[i] = 0;
        }
        g->timing.n_classes = 0;
    }
    void mark(int idx) {
        if (g->timing.enabled) cudaEventRecord(g->timing.ev[idx], g->stream);
    }
    void begin(int stage) { mark(2 * stage); }
    void end(int stage) { mark(2 * stage + 1); }
    void add(int stage, int launches) { g->timing.launches[stage] += (uint32_t)launches; }
    void collect() {
        if (!g->timing.enabled) return;
        cudaStreamSynchronize(g->stream);
        for (int i = 0; i < KCL_NUM_STAGES; i++) g->timing.ms[i] = elapsed(g->timing.ev + 2 * i);
    }
    // per-class split of the listing stage; class c holds root positions
    // [class_begin[c], class_begin[c-1]) (roots sorted by d+ descending)
    void collect_classes(uint32_t k, const uint32_t *class_begin, const uint32_t *limits, int n,
                         uint32_t max_outdeg) {
        Timing &t = g->timing;
        t.n_classes = 0;
        if (!t.enabled || n > KCL_MAX_CLASSES) return;
        t.n_classes = (uint32_t)n;
        for (int c = 0; c < n; c++) {
            const uint32_t end = c ? class_begin[c - 1] : class_begin[n];
            t.class_lo[c] = c ? limits[c - 1] + 1 : k - 1;
            t.class_hi[c] = std::min(limits[c], max_outdeg);
            t.class_roots[c] = end > class_begin[c] ? end - class_begin[c] : 0;
            t.class_ms[c] = t.class_roots[c] ? elapsed(t.cev + 2 * c) : 0.f;
        }
    }
    static float elapsed(const cudaEvent_t *ev) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ev[0], ev[1]) != cudaSuccess) {
            (void)cudaGetLastError();
            ms = 0.f;
        }
        return ms;
    }
};

struct FrontEnd {
    uint32_t max_outdeg = 0;
    uint32_t n_roots = 0;
    uint32_t class_begin[17] = {};
    uint32_t limits[16] = {};  // class c: d+ <= limits[c]
    int n_classes = 0;
    unsigned long long pre_count = 0;
};

kcl_status status_from_device(uint32_t st) {
    if (st & DEV_ERR_INTERNAL) return KCL_ECUDA;
    if (st & DEV_ERR_TIMEOUT) return KCL_ETIMEOUT;
    if (st & DEV_ERR_OUTDEG_LIMIT) return KCL_ELIMIT;
    if (st & DEV_ERR_OVERFLOW) return KCL_EOVERFLOW;
    if (st & DEV_ERR_INVALID_GRAPH) return KCL_EINVAL;
    return KCL_OK;
}

// Degeneracy peel in one cooperative launch (false: not launchable here, the
// caller falls back to one launch per round).
bool run_peel_coop(kcl_graph *g, StageTimer &T) {
    Workspace &w = g->ws;
    cudaStream_t s = g->stream;
    if (cudaMemsetAsync(w.peel, 0, sizeof(PeelCtl), s) != cudaSuccess ||
        cudaMemsetAsync(w.peel->minv, 0xFF, sizeof(w.peel->minv), s) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    // the remaining-vertex lists (n words each) and the big-row lists (n / 2
    // each) use the root-histogram scratch (3n + 1024 words), which is free
    // until the roots are sorted after the peel
    const size_t n = g->n;
    int l = launch_peel_coop(g, w, w.peel, w.hist, w.hist + n, w.hist + 2 * n, w.hist + 2 * n + n / 2 + 1, s);
    if (l < 0) {
        (void)cudaGetLastError();
        return false;
    }
    T.add(2, l);
    return true;
}

// Stages 0-2.  listing: enumerate Pre-List cliques into the ring.
kcl_status run_front(kcl_graph *g, uint32_t k, kcl_ordering ord, const kcl_ring *ring, bool listing,
                     StageTimer &T, FrontEnd &fe) {
    Workspace &w = g->ws;
    cudaStream_t s = g->stream;
    KCL_TRY(ensure_workspace(g));
    KCL_CK(cudaMemsetAsync(w.res, 0, sizeof(DevResult), s));
    const uint32_t n = g->n;

    // ---- stage 0: Pre-Core
    T.begin(0);
    // without Pre-Core the threshold is 0: every vertex stays
    T.add(0, launch_precore_init(g, (g->options & KCL_OPT_NO_PRECORE) ? 1u : k, w, s));
    uint32_t *fa = w.frontier_a, *fb = w.frontier_b;
    for (;;) {
        uint32_t nin = 0;
        KCL_TRY(read_u32(g, &w.res->frontier, &nin));
        if (nin == 0) break;
        KCL_TRY(set_u32(g, &w.res->frontier, 0));
        T.add(0, launch_precore_round(g, k, fa, nin, fb, w, s));
        std::swap(fa, fb);
    }
    KCL_CK(cudaMemcpyAsync(w.alive_core, w.alive, n, cudaMemcpyDeviceToDevice, s));
    T.end(0);

    // ---- stage 1: Pre-List
    T.begin(1);
    if (!(g->options & KCL_OPT_NO_PRELIST)) T.add(1, launch_prelist(g, k, w, listing ? 1 : 0, s));
    if (listing && !(g->options & KCL_OPT_NO_PRELIST)) {
        uint32_t ncomp = 0;
        KCL_TRY(read_u32(g, &w.res->n_clique_comps, &ncomp));
        T.add(1, launch_prelist_emit(g, k, w, ncomp, ring, s));
    }
    T.end(1);

    // ---- stage 2: orientation
    T.begin(2);
    if (ord == KCL_ORDER_DEGREE) {
        T.add(2, launch_degree_key(g, w, s));
    } else if (run_peel_coop(g, T)) {
        uint32_t err = 0;
        KCL_CK(cudaMemcpyAsync(&err, &w.peel->error, sizeof(err), cudaMemcpyDeviceToHost, s));
        KCL_CK(cudaStreamSynchronize(s));
        if (err) return KCL_ETIMEOUT;
    } else {
        T.add(2, launch_peel_init(g, w, s));
        uint32_t remaining = 0;
        KCL_TRY(read_u32(g, &w.res->remaining, &remaining));
        uint32_t t = 0, round = 0, nin = 0;
        fa = w.frontier_a;
        fb = w.frontier_b;
        while (remaining > 0) {
            if (nin == 0) {
                KCL_TRY(set_u32(g, &w.res->min_deg, 0xFFFFFFFFu));
                T.add(2, launch_peel_min(g, w, s));
                uint32_t mn = 0;
                KCL_TRY(read_u32(g, &w.res->min_deg, &mn));
                if (mn == 0xFFFFFFFFu) break;  // cannot happen while vertices remain
                t = std::max(t, mn);
                KCL_TRY(set_u32(g, &w.res->frontier, 0));
                T.add(2, launch_peel_select_all(g, w, t, round, fa, s));
                KCL_TRY(read_u32(g, &w.res->frontier, &nin));
                if (nin == 0) return KCL_ECUDA;  // inconsistent device state
            }
            remaining -= std::min(remaining, nin);
            KCL_TRY(set_u32(g, &w.res->frontier, 0));
            T.add(2, launch_peel_update(g, w, fa, nin, t, round, fb, s));
            round++;
            KCL_TRY(read_u32(g, &w.res->frontier, &nin));
            std::swap(fa, fb);
        }
    }
    KCL_CK(cudaMemsetAsync(&w.res->max_outdeg, 0, sizeof(unsigned), s));
    T.add(2, launch_orient(g, k, w, s));
    KCL_TRY(read_u32(g, &w.res->max_outdeg, &fe.max_outdeg));
    uint32_t *limits = fe.limits;
    fe.n_classes = ord == KCL_ORDER_DEGREE ? sdegree_classes(limits, 16) : bitcol_classes(limits, 16);
    T.add(2, launch_roots(g, k, w, fe.max_outdeg, fe.class_begin, limits, fe.n_classes, s));
    T.end(2);
    KCL_TRY(read_result(g));
    fe.n_roots = w.h_res->n_roots;
    fe.class_begin[fe.n_classes] = fe.n_roots;
    fe.pre_count = w.h_res->pre_count;
    if (w.h_res->status) return status_from_device(w.h_res->status);
    // roots above the largest class cannot be processed
    if (fe.class_begin[fe.n_classes - 1] > 0) return KCL_ELIMIT;
    (void)listing;
    return KCL_OK;
}

// Largest root out-degree kcl_root_colouring handles (the largest BitCol class).
constexpr uint32_t kColouringMaxOutdeg = 4096;

kcl_status check_args(kcl_graph *g, uint32_t k, kcl_ordering ord) {
    if (!g) return KCL_EINVAL;
    if (k < 3 || k > KCL_MAX_K) return KCL_EINVAL;
    if (ord != KCL_ORDER_DEGREE && ord != KCL_ORDER_COLOR) return KCL_EINVAL;
    return KCL_OK;
}

// Full call: stages 0-3, results left in the pinned mirror.
kcl_status run_call(kcl_graph *g, uint32_t k, kcl_ordering ord, const kcl_ring *ring, bool listing,
                    unsigned long long *per_root, unsigned long long *per_root_cks = nullptr,
                    const uint32_t *idmap = nullptr) {
    KCL_TRY(check_args(g, k, ord));
    if (cudaSetDevice(g->device) != cudaSuccess) return KCL_ECUDA;
    StageTimer T(g);
    T.mark(2 * 4);  // whole call
    FrontEnd fe;
    KCL_TRY(run_front(g, k, ord, ring, listing, T, fe));
    Workspace &w = g->ws;
    ListArgs la;
    la.listing = listing ? 1 : 0;
    la.per_root = per_root;
    la.per_root_cks = listing ? per_root_cks : nullptr;
    la.idmap = idmap;
    la.max_outdeg = fe.max_outdeg;
    if (g->timing.enabled) la.class_ev = g->timing.cev;
    if (listing && ring) {
        la.ring = ring->capacity ? ring->ids : nullptr;
        la.capacity = ring->capacity;
        la.wrap = ring->wrap;
    }
    T.begin(3);
    // the result block is zeroed per call (deadline 0: none); a limit is set on the device
    if (fe.n_roots > 0 && g->time_limit_ms)
        T.add(3, launch_set_deadline(w.res, g->time_limit_ms, g->stream));
    if (fe.n_roots > 0) {
        size_t arena = ord == KCL_ORDER_DEGREE
                           ? sdegree_arena_words(k, g->num_sms, fe.max_outdeg)
                           : bitcol_arena_words(k, g->num_sms, fe.max_outdeg);
        KCL_TRY(ensure_arena(g, arena));
        int l = ord == KCL_ORDER_DEGREE
                    ? launch_sdegree(g, k, w, fe.class_begin, fe.n_classes, la, g->stream)
                    : launch_bitcol(g, k, w, fe.class_begin, fe.n_classes, la, g->stream);
        T.add(3, l);
    }
    T.end(3);
    T.mark(2 * 4 + 1);
    KCL_CK(cudaGetLastError());
    KCL_TRY(read_result(g));
    T.collect();
    if (fe.n_roots > 0) T.collect_classes(k, fe.class_begin, fe.limits, fe.n_classes, fe.max_outdeg);
    if (w.h_res->status) return status_from_device(w.h_res->status);
    return KCL_OK;
}

kcl_status total_count(const DevResult *r, uint64_t *count) {
    unsigned long long c = r->count + r->pre_count;
    if (r->count_carry || c < r->count) return KCL_EOVERFLOW;
    *count = c;
    return KCL_OK;
}

}  // namespace

// Batched form: graphs that share (k, ordering) are joined as a disjoint
// union on the device and counted in one pipeline pass; each root's (and
// each Pre-List component's) count and checksum are attributed to its
// vertex, and a per-graph reduction gives every graph's own result.
struct kcl_batch {
    cudaStream_t stream = nullptr;
    int device = 0;
    kcl_graph *ug = nullptr;  // the union graph (CSR and workspace reused)
    uint32_t n_cap = 0;
    uint64_t nnz_cap = 0;
    uint32_t *graph_of = nullptr, *idmap = nullptr;
    uint8_t *kmap = nullptr;  // union vertex -> k of its graph
    unsigned long long *vcount = nullptr, *vcks = nullptr;
    unsigned long long *gcount = nullptr, *gcks = nullptr;
    BatchSrc *d_src = nullptr;
    uint32_t g_cap = 0;
    std::vector<BatchSrc> h_src;
    std::vector<unsigned long long> h_count, h_cks;
    kcl_timing timing = {};  // stage times summed over the groups of the last call
    uint32_t groups = 0;
};

namespace {

kcl_status batch_reserve(kcl_batch *b, uint32_t n, uint64_t nnz, uint32_t G) {
    kcl_graph *ug = b->ug;
    if (n > b->n_cap || nnz > b->nnz_cap) {
        uint32_t nc = std::max(n, b->n_cap);
        uint64_t ec = std::max(nnz, b->nnz_cap);
        KCL_TRY(dev_alloc(&ug->rp, (size_t)nc + 1));
        KCL_TRY(dev_alloc(&ug->col, ec ? ec : 1));
        KCL_TRY(dev_alloc(&b->graph_of, (size_t)nc + 1));
        KCL_TRY(dev_alloc(&b->idmap, (size_t)nc + 1));
        KCL_TRY(dev_alloc(&b->kmap, (size_t)nc + 1));
        KCL_TRY(dev_alloc(&b->vcount, (size_t)nc + 1));
        KCL_TRY(dev_alloc(&b->vcks, (size_t)nc + 1));
        b->n_cap = nc;
        b->nnz_cap = ec;
    }
    if (G > b->g_cap) {
        KCL_TRY(dev_alloc(&b->d_src, G));
        KCL_TRY(dev_alloc(&b->gcount, G));
        KCL_TRY(dev_alloc(&b->gcks, G));
        b->g_cap = G;
    }
    return KCL_OK;
}

// One ordering's group of a batch: its graphs, each with its own k, joined
// as one disjoint union and run through one pass of the pipeline (the union's
// k map gives every vertex the k of its graph; kernels are laid out for the
// group's largest k).
kcl_status batch_group(kcl_batch *b, kcl_graph *const *gs, const uint32_t *ks,
                       const std::vector<uint32_t> &idx, kcl_ordering ord, bool listing,
                       uint64_t *counts, uint64_t *checksums) {
    const uint32_t G = (uint32_t)idx.size();
    b->h_src.resize(G);
    uint64_t voff = 0, eoff = 0;
    uint32_t kmax = 3;
    for (uint32_t i = 0; i < G; i++) {
        const kcl_graph *g = gs[idx[i]];
        b->h_src[i] = BatchSrc{g->rp, g->col, g->n, (uint32_t)voff, g->nnz, eoff, ks[idx[i]], 0u};
        voff += g->n;
        eoff += g->nnz;
        kmax = std::max(kmax, ks[idx[i]]);
    }
    const uint32_t k = kmax;
    if (voff > 0xFFFFFFF0ull || eoff / 2 > 0xFFFFFFF0ull) return KCL_ELIMIT;
    const uint32_t n = (uint32_t)voff;
    KCL_TRY(batch_reserve(b, n, eoff, G));
    kcl_graph *ug = b->ug;
    cudaStream_t s = b->stream;
    KCL_CK(cudaMemcpyAsync(b->d_src, b->h_src.data(), G * sizeof(BatchSrc), cudaMemcpyHostToDevice, s));
    launch_union_build(b->d_src, G, n, ug->rp, ug->col, b->graph_of, b->idmap, b->kmap, s);
    ug->n = n;
    ug->nnz = eoff;
    ug->stream = s;
    KCL_CK(cudaMemsetAsync(b->vcount, 0, ((size_t)n + 1) * sizeof(unsigned long long), s));
    if (listing) KCL_CK(cudaMemsetAsync(b->vcks, 0, ((size_t)n + 1) * sizeof(unsigned long long), s));
    KCL_TRY(ensure_workspace(ug));
    ug->ws.vcount_pre = b->vcount;
    ug->ws.vcks_pre = listing ? b->vcks : nullptr;
    ug->ws.idmap = b->idmap;
    ug->ws.kmap = b->kmap;
    kcl_status st = n ? run_call(ug, k, ord, nullptr, listing, b->vcount, b->vcks, b->idmap) : KCL_OK;
    ug->ws.vcount_pre = nullptr;
    ug->ws.vcks_pre = nullptr;
    ug->ws.idmap = nullptr;
    ug->ws.kmap = nullptr;
    if (st != KCL_OK) return st;
    if (ug->timing.enabled && n)
        for (int i = 0; i < KCL_NUM_STAGES; i++) {
            b->timing.ms[i] += ug->timing.ms[i];
            b->timing.launches[i] += ug->timing.launches[i];
        }
    b->groups++;
    launch_graph_sums(b->d_src, G, b->vcount, listing ? b->vcks : nullptr, b->gcount,
                      listing ? b->gcks : nullptr, s);
    b->h_count.resize(G);
    b->h_cks.resize(G);
    KCL_CK(cudaMemcpyAsync(b->h_count.data(), b->gcount, G * sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost, s));
    if (listing)
        KCL_CK(cudaMemcpyAsync(b->h_cks.data(), b->gcks, G * sizeof(unsigned long long),
                               cudaMemcpyDeviceToHost, s));
    KCL_CK(cudaStreamSynchronize(s));
    for (uint32_t i = 0; i < G; i++) {
        counts[idx[i]] = b->h_count[i];
        if (listing) checksums[idx[i]] = b->h_cks[i];
    }
    return KCL_OK;
}

}  // namespace

// ============================================================== public ABI
extern "C" {

const char *kcl_strerror(kcl_status s) {
    switch (s) {
        case KCL_OK: return "ok";
        case KCL_EINVAL: return "invalid argument or malformed graph";
        case KCL_ENOMEM: return "out of memory";
        case KCL_EOVERFLOW: return "clique count exceeds 2^64-1";
        case KCL_ETRUNC: return "more cliques than ring capacity (output truncated)";
        case KCL_ETIMEOUT: return "time limit exceeded or device wait timed out";
        case KCL_ECUDA: return "CUDA runtime error";
        case KCL_EABORT: return "aborted";
        case KCL_ELIMIT: return "root out-degree above the supported limit";
        case KCL_ESIZE: return "input larger than the fixed scratch of an allocation-free call";
    }
    return "unknown status";
}

kcl_status kcl_load_csr(uint32_t n, const uint64_t *row_ptr, const uint32_t *col, int on_device,
                        void *stream, kcl_graph **out) {
    if (!out) return KCL_EINVAL;
    *out = nullptr;
    if (!row_ptr) return KCL_EINVAL;
    kcl_graph *g = new (std::nothrow) kcl_graph();
    if (!g) return KCL_ENOMEM;
    g->n = n;
    g->stream = (cudaStream_t)stream;
    auto fail = [&](kcl_status s) {
        kcl_free_graph(g);
        return s;
    };
    if (cudaGetDevice(&g->device) != cudaSuccess) return fail(KCL_ECUDA);
    if (cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device) != cudaSuccess)
        return fail(KCL_ECUDA);
    uint64_t nnz = 0;
    if (on_device) {
        // ordered on the graph's stream, after the caller's work there
        if (cudaMemcpyAsync(&nnz, row_ptr + n, sizeof(uint64_t), cudaMemcpyDeviceToHost,
                            g->stream) != cudaSuccess ||
            cudaStreamSynchronize(g->stream) != cudaSuccess)
            return fail(KCL_ECUDA);
    } else {
        nnz = row_ptr[n];
    }
    if (nnz > 0 && !col) return fail(KCL_EINVAL);
    if (nnz & 1ull) return fail(KCL_EINVAL);           // symmetric CSR has an even entry count
    if (nnz / 2 > 0xFFFFFFFEull) return fail(KCL_ELIMIT);  // out-CSR uses 32-bit offsets
    g->nnz = nnz;
    if (dev_alloc(&g->rp, (size_t)n + 1) != KCL_OK) return fail(KCL_ENOMEM);
    if (dev_alloc(&g->col, nnz ? nnz : 1) != KCL_OK) return fail(KCL_ENOMEM);
    cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (cudaMemcpyAsync(g->rp, row_ptr, ((size_t)n + 1) * sizeof(uint64_t), kind, g->stream) != cudaSuccess)
        return fail(KCL_ECUDA);
    if (nnz && cudaMemcpyAsync(g->col, col, nnz * sizeof(uint32_t), kind, g->stream) != cudaSuccess)
        return fail(KCL_ECUDA);
    kcl_status st = ensure_workspace(g);
    if (st != KCL_OK) return fail(st);
    if (cudaMemsetAsync(g->ws.res, 0, sizeof(DevResult), g->stream) != cudaSuccess) return fail(KCL_ECUDA);
    if (n) launch_validate(g, g->ws.res, g->stream);
    if (cudaGetLastError() != cudaSuccess) return fail(KCL_ECUDA);
    st = read_result(g);
    if (st != KCL_OK) return fail(st);
    if (g->ws.h_res->status) return fail(KCL_EINVAL);
    g->max_deg = g->ws.h_res->max_outdeg;
    *out = g;
    return KCL_OK;
}

void kcl_free_graph(kcl_graph *g) {
    if (!g) return;
    if (g->stream) cudaStreamSynchronize(g->stream);
    else cudaDeviceSynchronize();
    (void)cudaGetLastError();
    free_workspace(g->ws);
    if (g->owns_csr && g->rp) cudaFree(g->rp);
    if (g->owns_csr && g->col) cudaFree(g->col);
    for (int i = 0; i < 2 * KCL_NUM_STAGES; i++)
        if (g->timing.ev[i]) cudaEventDestroy(g->timing.ev[i]);
    for (int i = 0; i < 2 * KCL_MAX_CLASSES; i++)
        if (g->timing.cev[i]) cudaEventDestroy(g->timing.cev[i]);
    (void)cudaGetLastError();
    delete g;
}

kcl_status kcl_graph_view(const kcl_graph *g, void *stream, kcl_graph **out) {
    if (!g || !out) return KCL_EINVAL;
    *out = nullptr;
    kcl_graph *v = new (std::nothrow) kcl_graph();
    if (!v) return KCL_ENOMEM;
    v->n = g->n;
    v->nnz = g->nnz;
    v->device = g->device;
    v->num_sms = g->num_sms;
    v->stream = (cudaStream_t)stream;
    v->rp = g->rp;
    v->col = g->col;
    v->max_deg = g->max_deg;
    v->owns_csr = false;
    *out = v;
    return KCL_OK;
}

kcl_status kcl_set_stream(kcl_graph *g, void *stream) {
    if (!g) return KCL_EINVAL;
    g->stream = (cudaStream_t)stream;
    return KCL_OK;
}

uint32_t kcl_num_vertices(const kcl_graph *g) { return g ? g->n : 0; }
uint64_t kcl_num_edges(const kcl_graph *g) { return g ? g->nnz / 2 : 0; }

kcl_status kcl_count(kcl_graph *g, uint32_t k, kcl_ordering ord, uint64_t *count) {
    if (!count) return KCL_EINVAL;
    KCL_TRY(run_call(g, k, ord, nullptr, false, nullptr));
    return total_count(g->ws.h_res, count);
}

kcl_status kcl_list(kcl_graph *g, uint32_t k, kcl_ordering ord, const kcl_ring *ring,
                    uint64_t *count, uint64_t *checksum, uint64_t *written) {
    if (!count || !checksum) return KCL_EINVAL;
    if (ring && ring->capacity && !ring->ids) return KCL_EINVAL;
    KCL_TRY(run_call(g, k, ord, ring, true, nullptr));
    const DevResult *r = g->ws.h_res;
    KCL_TRY(total_count(r, count));
    *checksum = r->checksum + r->pre_checksum;
    uint64_t cap = ring ? ring->capacity : 0;
    uint64_t wr = r->emitted < cap ? r->emitted : cap;
    if (written) *written = wr;
    if (ring && !ring->wrap && r->emitted > cap) return KCL_ETRUNC;
    return KCL_OK;
}

kcl_status kcl_count_per_root(kcl_graph *g, uint32_t k, kcl_ordering ord, uint64_t *per_root,
                              uint64_t *count, uint64_t *prelist_count) {
    if (!per_root || !count) return KCL_EINVAL;
    KCL_TRY(check_args(g, k, ord));
    if (cudaMemsetAsync(per_root, 0, (size_t)g->n * sizeof(uint64_t), g->stream) != cudaSuccess) {
        (void)cudaGetLastError();
        return KCL_ECUDA;
    }
    KCL_TRY(run_call(g, k, ord, nullptr, false, reinterpret_cast<unsigned long long *>(per_root)));
    if (prelist_count) *prelist_count = g->ws.h_res->pre_count;
    return total_count(g->ws.h_res, count);
}

kcl_status kcl_count_roots(kcl_graph *g, uint32_t k, kcl_ordering ord, const uint32_t *roots,
                           uint32_t n_roots, uint64_t *per_root, uint64_t *count) {
    if (!per_root || !count || (n_roots && !roots)) return KCL_EINVAL;
    KCL_TRY(check_args(g, k, ord));
    for (uint32_t i = 0; i < n_roots; i++)
        if (roots[i] >= g->n) return KCL_EINVAL;
    if (cudaSetDevice(g->device) != cudaSuccess) return KCL_ECUDA;
    std::vector<uint8_t> mask((size_t)g->n + 1, 0);
    for (uint32_t i = 0; i < n_roots; i++) mask[roots[i]] = 1;
    uint8_t *d_mask = nullptr;
    if (cudaMalloc((void **)&d_mask, mask.size()) != cudaSuccess) {
        (void)cudaGetLastError();
        return KCL_ENOMEM;
    }
    kcl_status st = KCL_OK;
    if (cudaMemcpyAsync(d_mask, mask.data(), mask.size(), cudaMemcpyHostToDevice, g->stream) != cudaSuccess ||
        cudaMemsetAsync(per_root, 0, (size_t)g->n * sizeof(uint64_t), g->stream) != cudaSuccess) {
        (void)cudaGetLastError();
        st = KCL_ECUDA;
    }
    if (st == KCL_OK) {
        g->ws.root_mask = d_mask;
        st = run_call(g, k, ord, nullptr, false, reinterpret_cast<unsigned long long *>(per_root));
        g->ws.root_mask = nullptr;
    }
    if (st == KCL_OK) {
        const DevResult *r = g->ws.h_res;
        if (r->count_carry) st = KCL_EOVERFLOW;
        else *count = r->count;
    }
    cudaStreamSynchronize(g->stream);
    (void)cudaGetLastError();
    cudaFree(d_mask);
    return st;
}

kcl_status kcl_stage_info(kcl_graph *g, uint32_t k, kcl_ordering ord, uint8_t *alive_core,
                          uint8_t *alive_final, uint32_t *outdeg, uint32_t *key,
                          uint64_t *prelist_count, uint32_t *max_outdeg) {
    KCL_TRY(check_args(g, k, ord));
    StageTimer T(g);
    FrontEnd fe;
    kcl_status st = run_front(g, k, ord, nullptr, false, T, fe);
    if (st != KCL_OK && st != KCL_ELIMIT) return st;
    Workspace &w = g->ws;
    size_t n = g->n;
    if (alive_core) KCL_CK(cudaMemcpyAsync(alive_core, w.alive_core, n, cudaMemcpyDeviceToHost, g->stream));
    if (alive_final) KCL_CK(cudaMemcpyAsync(alive_final, w.alive, n, cudaMemcpyDeviceToHost, g->stream));
    if (outdeg) KCL_CK(cudaMemcpyAsync(outdeg, w.outdeg, n * 4, cudaMemcpyDeviceToHost, g->stream));
    if (key) KCL_CK(cudaMemcpyAsync(key, w.key, n * 4, cudaMemcpyDeviceToHost, g->stream));
    KCL_CK(cudaStreamSynchronize(g->stream));
    if (prelist_count) *prelist_count = fe.pre_count;
    if (max_outdeg) *max_outdeg = fe.max_outdeg;
    return KCL_OK;
}

kcl_status kcl_root_colouring(kcl_graph *g, uint32_t k, uint32_t root, uint32_t capacity,
                              uint32_t *nbr, uint32_t *colour, uint32_t *outdeg) {
    KCL_TRY(check_args(g, k, KCL_ORDER_COLOR));
    if (!outdeg || root >= g->n) return KCL_EINVAL;
    *outdeg = 0;
    if (cudaSetDevice(g->device) != cudaSuccess) return KCL_ECUDA;
    StageTimer T(g);
    FrontEnd fe;
    kcl_status st = run_front(g, k, KCL_ORDER_COLOR, nullptr, false, T, fe);
    if (st != KCL_OK && st != KCL_ELIMIT) return st;
    Workspace &w = g->ws;
    uint32_t ptr[2] = {0, 0};
    KCL_CK(cudaMemcpyAsync(ptr, w.optr + root, 2 * sizeof(uint32_t), cudaMemcpyDeviceToHost, g->stream));
    KCL_CK(cudaStreamSynchronize(g->stream));
    const uint32_t d = ptr[1] - ptr[0];
    *outdeg = d;
    if (d == 0) return KCL_OK;
    if (d > kColouringMaxOutdeg) return KCL_ELIMIT;
    if (capacity < d || !nbr || !colour) return KCL_EINVAL;
    uint32_t *arena = nullptr, *out = nullptr;
    const size_t words = bitcol_colours_arena_words(d);
    if (cudaMalloc((void **)&arena, words * 4) != cudaSuccess ||
        cudaMalloc((void **)&out, 2 * (size_t)d * 4) != cudaSuccess) {
        (void)cudaGetLastError();
        cudaFree(arena);
        return KCL_ENOMEM;
    }
    st = KCL_OK;
    if (launch_bitcol_colours(w, root, d, arena, out, out + d, g->stream) < 0) st = KCL_ELIMIT;
    if (st == KCL_OK &&
        (cudaMemcpyAsync(nbr, out, (size_t)d * 4, cudaMemcpyDeviceToHost, g->stream) != cudaSuccess ||
         cudaMemcpyAsync(colour, out + d, (size_t)d * 4, cudaMemcpyDeviceToHost, g->stream) != cudaSuccess ||
         cudaStreamSynchronize(g->stream) != cudaSuccess))
        st = KCL_ECUDA;
    (void)cudaGetLastError();
    cudaFree(arena);
    cudaFree(out);
    return st;
}

kcl_status kcl_batch_create(void *stream, kcl_batch **out) {
    if (!out) return KCL_EINVAL;
    *out = nullptr;
    kcl_batch *b = new (std::nothrow) kcl_batch();
    if (!b) return KCL_ENOMEM;
    b->stream = (cudaStream_t)stream;
    b->ug = new (std::nothrow) kcl_graph();
    if (!b->ug || cudaGetDevice(&b->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&b->ug->num_sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess) {
        (void)cudaGetLastError();
        kcl_batch_free(b);
        return KCL_ECUDA;
    }
    b->ug->device = b->device;
    b->ug->stream = b->stream;
    *out = b;
    return KCL_OK;
}

void kcl_batch_free(kcl_batch *b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    else cudaDeviceSynchronize();
    (void)cudaGetLastError();
    void *ptrs[] = {b->graph_of, b->idmap, b->kmap, b->vcount, b->vcks, b->gcount, b->gcks, b->d_src};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    kcl_free_graph(b->ug);
    delete b;
}

kcl_status kcl_count_batch(kcl_batch *b, kcl_graph *const *gs, const uint32_t *ks,
                           const kcl_ordering *ords, uint32_t G, uint64_t *counts,
                           uint64_t *checksums) {
    if (!b || (G && (!gs || !ks || !ords || !counts))) return KCL_EINVAL;
    std::map<int, std::vector<uint32_t>> groups;  // by ordering; k varies within a group
    for (uint32_t i = 0; i < G; i++) {
        if (!gs[i] || gs[i]->device != b->device) return KCL_EINVAL;
        KCL_TRY(check_args(gs[i], ks[i], ords[i]));
        groups[(int)ords[i]].push_back(i);
    }
    if (cudaSetDevice(b->device) != cudaSuccess) return KCL_ECUDA;
    b->timing = kcl_timing{};
    b->groups = 0;
    for (auto &kv : groups)
        KCL_TRY(batch_group(b, gs, ks, kv.second, (kcl_ordering)kv.first, checksums != nullptr, counts,
                            checksums));
    return KCL_OK;
}

kcl_status kcl_batch_set_time_limit(kcl_batch *b, uint64_t ms) {
    if (!b) return KCL_EINVAL;
    return kcl_set_time_limit(b->ug, ms);
}

kcl_status kcl_batch_enable_timing(kcl_batch *b, int enable) {
    if (!b) return KCL_EINVAL;
    return kcl_enable_timing(b->ug, enable);
}

kcl_status kcl_batch_last_timing(const kcl_batch *b, kcl_timing *t, uint32_t *groups) {
    if (!b || !t) return KCL_EINVAL;
    *t = b->timing;
    if (groups) *groups = b->groups;
    return KCL_OK;
}

kcl_status kcl_enable_timing(kcl_graph *g, int enable) {
    if (!g) return KCL_EINVAL;
    if (enable && !g->timing.ev[0]) {
        for (int i = 0; i < 2 * KCL_NUM_STAGES; i++)
            if (cudaEventCreate(&g->timing.ev[i]) != cudaSuccess) {
                (void)cudaGetLastError();
                return KCL_ECUDA;
            }
        for (int i = 0; i < 2 * KCL_MAX_CLASSES; i++)
            if (cudaEventCreate(&g->timing.cev[i]) != cudaSuccess) {
                (void)cudaGetLastError();
                return KCL_ECUDA;
            }
    }
    g->timing.enabled = enable ? 1 : 0;
    return KCL_OK;
}

kcl_status kcl_last_timing(const kcl_graph *g, kcl_timing *t) {
    if (!g || !t) return KCL_EINVAL;
    *t = kcl_timing{};
    for (int i = 0; i < KCL_NUM_STAGES; i++) {
        t->ms[i] = g->timing.ms[i];
        t->launches[i] = g->timing.launches[i];
    }
    t->n_classes = g->timing.n_classes;
    for (uint32_t c = 0; c < g->timing.n_classes; c++) {
        t->class_lo[c] = g->timing.class_lo[c];
        t->class_hi[c] = g->timing.class_hi[c];
        t->class_roots[c] = g->timing.class_roots[c];
        t->class_ms[c] = g->timing.class_ms[c];
    }
    return KCL_OK;
}

kcl_status kcl_set_time_limit(kcl_graph *g, uint64_t ms) {
    if (!g) return KCL_EINVAL;
    g->time_limit_ms = ms;
    return KCL_OK;
}

kcl_status kcl_set_options(kcl_graph *g, uint32_t flags) {
    if (!g || (flags & ~(KCL_OPT_NO_PRECORE | KCL_OPT_NO_PRELIST | KCL_OPT_NO_COLOR_PRUNE)))
        return KCL_EINVAL;
    g->options = flags;
    return KCL_OK;
}

kcl_status kcl_get_options(const kcl_graph *g, uint32_t *flags) {
    if (!g || !flags) return KCL_EINVAL;
    *flags = g->options;
    return KCL_OK;
}

kcl_status kcl_scratch_bytes(const kcl_graph *g, uint64_t *workspace, uint64_t *arena) {
    if (!g || !workspace || !arena) return KCL_EINVAL;
    const Workspace &w = g->ws;
    uint64_t ws = 0;
    if (w.res) {
        // mirrors ensure_workspace's allocations
        const uint64_t n = (uint64_t)w.n_cap + 1, half = w.nnz_cap / 2 + 1;
        ws = 2 * n                                  // alive, alive_core
             + 4 * n * 13 + 8 * n                   // u32 arrays, comp_sdeg
             + 4 * 2                                // outdeg, optr extra entry
             + 4 * half                             // oadj
             + 4 * (3 * n + 1024) + 4 * (n / 1024 + 1024) + 4 * 64
             + sizeof(DevResult) + sizeof(PeelCtl) + 8 * kMaxSplitSlots;
    }
    *workspace = ws;
    *arena = (uint64_t)w.arena_words * 4;
    return KCL_OK;
}

kcl_status kcl_get_tuning(const kcl_graph *g, kcl_tuning *t) {
    if (!g || !t) return KCL_EINVAL;
    *t = g->tuning;
    return KCL_OK;
}

kcl_status kcl_set_tuning(kcl_graph *g, const kcl_tuning *t) {
    if (!g || !t) return KCL_EINVAL;
    g->tuning = *t;
    return KCL_OK;
}

namespace {

// One tuning pass: for every candidate value of knob[] (all classes at once)
// run the call and keep, per class, the fastest value.
kcl_status tune_knob(kcl_graph *g, uint32_t k, kcl_ordering ord, int listing, uint32_t *knob,
                     const uint32_t *cand, int ncand) {
    float best_ms[KCL_MAX_CLASSES];
    uint32_t best[KCL_MAX_CLASSES];
    for (int c = 0; c < KCL_MAX_CLASSES; c++) {
        best_ms[c] = -1.f;
        best[c] = knob[c];
    }
    uint64_t cnt = 0, cks = 0, wr = 0;
    for (int i = 0; i < ncand; i++) {
        for (int c = 0; c < KCL_MAX_CLASSES; c++) knob[c] = cand[i];
        kcl_status st = listing ? kcl_list(g, k, ord, nullptr, &cnt, &cks, &wr) : kcl_count(g, k, ord, &cnt);
        if (st != KCL_OK) {
            for (int c = 0; c < KCL_MAX_CLASSES; c++) knob[c] = best[c];
            return st;
        }
        for (uint32_t c = 0; c < g->timing.n_classes && c < KCL_MAX_CLASSES; c++) {
            if (!g->timing.class_roots[c]) continue;
            const float ms = g->timing.class_ms[c];
            if (best_ms[c] < 0.f || ms < 0.98f * best_ms[c]) {
                best_ms[c] = ms;
                best[c] = cand[i];
            }
        }
    }
    for (int c = 0; c < KCL_MAX_CLASSES; c++) knob[c] = best[c];
    return KCL_OK;
}

}  // namespace

kcl_status kcl_autotune(kcl_graph *g, uint32_t k, kcl_ordering ord, int listing, kcl_tuning *out) {
    if (!g) return KCL_EINVAL;
    KCL_TRY(check_args(g, k, ord));
    const int was_enabled = g->timing.enabled;
    KCL_TRY(kcl_enable_timing(g, 1));
    kcl_status st = KCL_OK;
    if (ord == KCL_ORDER_DEGREE) {
        static const uint32_t bitmap_cand[] = {0, 4, 64, 0xFFFFFFFFu};
        static const uint32_t gallop_cand[] = {0, 40, 80, 160, 400};
        st = tune_knob(g, k, ord, listing, g->tuning.sdegree_bitmap, bitmap_cand, 4);
        if (st == KCL_OK)
            st = tune_knob(g, k, ord, listing,
                           listing ? g->tuning.sdegree_gallop_list : g->tuning.sdegree_gallop,
                           gallop_cand, 5);
    }
    static const uint32_t warps_cand[] = {0, 4, 8};
    if (st == KCL_OK)
        st = tune_knob(g, k, ord, listing,
                       ord == KCL_ORDER_DEGREE ? g->tuning.sdegree_cta_warps : g->tuning.bitcol_cta_warps,
                       warps_cand, 3);
    static const uint32_t split_cand[] = {0, 2, 8, 32};
    if (st == KCL_OK)
        st = tune_knob(g, k, ord, listing,
                       ord == KCL_ORDER_DEGREE ? g->tuning.sdegree_split : g->tuning.bitcol_split,
                       split_cand, 4);
    if (!was_enabled) kcl_enable_timing(g, 0);
    if (st != KCL_OK) return st;
    if (out) *out = g->tuning;
    return KCL_OK;
}

}  // extern "C"
