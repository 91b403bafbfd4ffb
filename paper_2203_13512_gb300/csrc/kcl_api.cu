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
#include <new>

#include "kcl_internal.cuh"

namespace kcl {
size_t bitcol_arena_words(uint32_t k, int num_sms, uint32_t max_outdeg);
size_t sdegree_arena_words(uint32_t k, int num_sms, uint32_t max_outdeg);
}  // namespace kcl

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
                    w.peel};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (w.h_res) cudaFreeHost(w.h_res);
    w = Workspace();
}

kcl_status ensure_workspace(kcl_graph *g) {
    Workspace &w = g->ws;
    if (w.res && w.n_cap >= g->n && w.nnz_cap >= g->nnz) return KCL_OK;
    free_workspace(w);
    size_t n = (size_t)g->n + 1;
    size_t half = g->nnz / 2 + 1;
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
    if (cudaMallocHost((void **)&w.h_res, sizeof(DevResult)) != cudaSuccess) {
        (void)cudaGetLastError();
        w.h_res = nullptr;
        return KCL_ENOMEM;
    }
    KCL_CK(cudaMemset(w.outdeg, 0, (n + 1) * sizeof(uint32_t)));
    w.n_cap = g->n;
    w.nnz_cap = g->nnz;
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
        for (int i = 0; i < KCL_NUM_STAGES; i++) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, g->timing.ev[2 * i], g->timing.ev[2 * i + 1]) == cudaSuccess)
                g->timing.ms[i] = ms;
            else
                (void)cudaGetLastError();
        }
    }
};

struct FrontEnd {
    uint32_t max_outdeg = 0;
    uint32_t n_roots = 0;
    uint32_t class_begin[17] = {};
    int n_classes = 0;
    unsigned long long pre_count = 0;
};

kcl_status status_from_device(uint32_t st) {
    if (st & DEV_ERR_INTERNAL) return KCL_ECUDA;
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
        cudaMemsetAsync(&w.peel->minv, 0xFF, sizeof(unsigned), s) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    int l = launch_peel_coop(g, w, w.peel, s);
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
    T.add(0, launch_precore_init(g, k, w, s));
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
    T.add(1, launch_prelist(g, k, w, listing ? 1 : 0, s));
    if (listing) {
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
    uint32_t limits[16];
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

kcl_status check_args(kcl_graph *g, uint32_t k, kcl_ordering ord) {
    if (!g) return KCL_EINVAL;
    if (k < 3 || k > KCL_MAX_K) return KCL_EINVAL;
    if (ord != KCL_ORDER_DEGREE && ord != KCL_ORDER_COLOR) return KCL_EINVAL;
    return KCL_OK;
}

// Full call: stages 0-3, results left in the pinned mirror.
kcl_status run_call(kcl_graph *g, uint32_t k, kcl_ordering ord, const kcl_ring *ring, bool listing,
                    unsigned long long *per_root) {
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
    if (listing && ring) {
        la.ring = ring->capacity ? ring->ids : nullptr;
        la.capacity = ring->capacity;
        la.wrap = ring->wrap;
    }
    T.begin(3);
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

// ============================================================== public ABI
extern "C" {

const char *kcl_strerror(kcl_status s) {
    switch (s) {
        case KCL_OK: return "ok";
        case KCL_EINVAL: return "invalid argument or malformed graph";
        case KCL_ENOMEM: return "out of memory";
        case KCL_EOVERFLOW: return "clique count exceeds 2^64-1";
        case KCL_ETRUNC: return "more cliques than ring capacity (output truncated)";
        case KCL_ETIMEOUT: return "device wait timed out";
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
        if (cudaMemcpy(&nnz, row_ptr + n, sizeof(uint64_t), cudaMemcpyDeviceToHost) != cudaSuccess)
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
    if (g->rp) cudaFree(g->rp);
    if (g->col) cudaFree(g->col);
    for (int i = 0; i < 2 * KCL_NUM_STAGES; i++)
        if (g->timing.ev[i]) cudaEventDestroy(g->timing.ev[i]);
    (void)cudaGetLastError();
    delete g;
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

kcl_status kcl_enable_timing(kcl_graph *g, int enable) {
    if (!g) return KCL_EINVAL;
    if (enable && !g->timing.ev[0]) {
        for (int i = 0; i < 2 * KCL_NUM_STAGES; i++)
            if (cudaEventCreate(&g->timing.ev[i]) != cudaSuccess) {
                (void)cudaGetLastError();
                return KCL_ECUDA;
            }
    }
    g->timing.enabled = enable ? 1 : 0;
    return KCL_OK;
}

kcl_status kcl_last_timing(const kcl_graph *g, kcl_timing *t) {
    if (!g || !t) return KCL_EINVAL;
    for (int i = 0; i < KCL_NUM_STAGES; i++) {
        t->ms[i] = g->timing.ms[i];
        t->launches[i] = g->timing.launches[i];
    }
    return KCL_OK;
}

}  // extern "C"
