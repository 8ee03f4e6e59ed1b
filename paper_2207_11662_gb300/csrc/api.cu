// The C-ABI (include/homln.h): handle management, argument checking, host/device
// output placement and the Psi / Theta call sequence of the decoupled method.
//
// Psi (Section 3): each layer is analysed once -- all-sources BFS closeness --
// and its partial results (F, R, closeness, sumDist, degree) are cached in the
// handle. Theta (Section 4, Section 5): compositions read only those partial
// results (plus the layer CSRs for CC1). Ground truth (Section 4): the AND
// aggregate of the selected layers, analysed the same way.
#include "common.cuh"

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <tuple>

namespace homln {

std::atomic<long long> g_kernel_launches{0};

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

void fail(homln_status code, const std::string &msg) { throw Error{code, msg}; }

void check_cuda(cudaError_t e, const char *what) {
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw Error{HOMLN_ECUDA, std::string(what) + ": " + cudaGetErrorString(e)};
    }
}

// Without a caller allocator, device memory comes from one stream-ordered pool per device
// owned by the library. The pool keeps up to kPoolKeepBytes of freed memory mapped across
// synchronisations, so the BFS state and the scratch of repeated calls are not unmapped and
// mapped again every call (a pool with the default threshold of 0 returns it at every sync).
constexpr uint64_t kPoolKeepBytes = 8ull << 30;
constexpr int kMaxDevices = 64;
static std::mutex g_pool_mu;
static cudaMemPool_t g_pools[kMaxDevices];

static cudaMemPool_t device_pool() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pools[dev]) {
        cudaMemPoolProps props;
        std::memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        uint64_t keep = kPoolKeepBytes;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        // Memory freed on one stream is reused on another only through an event dependency the
        // program made itself: with many handles and side streams, the CUDA driver's own cross-stream
        // reuse (completion checks, inserted dependencies) made allocations very slow.
        int off = 0;
        cudaMemPoolSetAttribute(pool, cudaMemPoolReuseAllowOpportunistic, &off);
        cudaMemPoolSetAttribute(pool, cudaMemPoolReuseAllowInternalDependencies, &off);
        g_pools[dev] = pool;
    }
    return g_pools[dev];
}

void *Alloc::get(size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (a.alloc) return a.alloc(a.ctx, bytes, (void *)stream);
    void *p = nullptr;
    cudaMemPool_t pool = device_pool();
    if (!pool) return nullptr;
    if (cudaMallocFromPoolAsync(&p, bytes, pool, stream) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void Alloc::put(void *p, size_t bytes) {
    if (!p) return;
    if (a.free) a.free(a.ctx, p, bytes ? bytes : 16, (void *)stream);
    else cudaFreeAsync(p, stream);
}

// CC nodes of one graph under one selection rule: ids in rank order and a membership bitmap.
struct Selection {
    DBuf<int32_t> ranked;
    DBuf<uint32_t> bits;
    int32_t count = 0;
};

// A selection rule as a cache key: mode, percent (TOPK_PERCENT) and k (TOPK_COUNT).
using SelKey = std::tuple<int32_t, double, int64_t>;

// Partial results of one analysed graph (a layer or an AND aggregate).
struct GraphState {
    Csr csr;     // rows = out-edges (all edges if undirected)
    Csr csr_in;  // rows = in-edges; directed graphs only
    bool analysed = false;
    DBuf<uint64_t> F;
    DBuf<uint32_t> R;
    DBuf<double> cc;
    DBuf<uint64_t> sumdist;
    DBuf<int32_t> deg;
    std::map<SelKey, std::unique_ptr<Selection>> selections;
    BfsGraph bfs;          // the graph as the BFS reads it (built once, kept by homln_invalidate)
    bool bfs_ready = false;
    int graph_refs = 0;    // captured graphs that write this graph's results (buffers stay put)
};

}  // namespace homln

using namespace homln;

// Side streams ("lanes") of a handle: independent per-graph work of one call (the layers' CSR
// builds, the BFS graphs' relabellings, the layers' CC-node selections) runs on them side by
// side, forked from and joined back into the handle's stream with events. Declared first in
// the handle, so they are destroyed after every buffer freed on them.
struct Lanes {
    static constexpr int kCount = 4;
    cudaStream_t s[kCount] = {};
    Alloc al[kCount];  // the handle's allocator, bound to each lane
    cudaEvent_t done[kCount] = {};
    cudaEvent_t fork = nullptr;
    ~Lanes() {
        for (int i = 0; i < kCount; ++i) {
            if (s[i]) {
                cudaStreamSynchronize(s[i]);
                cudaStreamDestroy(s[i]);
            }
            if (done[i]) cudaEventDestroy(done[i]);
        }
        if (fork) cudaEventDestroy(fork);
    }
};

struct homln_graph_s;

struct homln_yield_s;

struct homln_s {
    Lanes lanes;
    Alloc al;  // declared before the buffers: destroyed after every buffer that uses it
    int device = 0;
    cudaStream_t stream = nullptr;
    int32_t n = 0, L = 0;
    bool directed = false;
    BfsTuning tuning;
    DBuf<int32_t> err;
    std::vector<std::unique_ptr<GraphState>> layers;
    std::map<uint64_t, std::unique_ptr<GraphState>> ands;
    std::map<uint64_t, std::unique_ptr<GraphState>> ors;
    bool profiling = false;
    bool instrument = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> events;
    long long bfs_launches = 0;
    int live_graphs = 0;  // captured graphs that involve this handle
    homln_yield_s *yield = nullptr;  // the yield flag this handle's BFS watches (homln_set_yield)
    BfsStats stats;
    ~homln_s() {
        for (auto &e : events) {
            cudaEventDestroy(e.first);
            cudaEventDestroy(e.second);
        }
    }
};

namespace {

// Every entry point is an NVTX range named after it (visible in nsys/ncu timelines; a no-op
// when no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

#define API_BEGIN                        \
    const NvtxRange nvtx_range_(__func__); \
    try {
#define API_END                                           \
    }                                                     \
    catch (const homln::Error &e) {                       \
        set_error(e.msg);                                 \
        return e.code;                                    \
    }                                                     \
    catch (const std::bad_alloc &) {                      \
        set_error("host allocation failed");              \
        return HOMLN_ENOMEM;                              \
    }                                                     \
    catch (...) {                                         \
        set_error("unexpected internal error");           \
        return HOMLN_ECUDA;                               \
    }                                                     \
    set_error("");                                        \
    return HOMLN_OK;

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

void use_device(homln_t h) { HCUDA(cudaSetDevice(h->device)); }

void lanes_open(homln_t h) {
    Lanes &L = h->lanes;
    int prio = 0;  // the lanes run at the priority of the handle's stream
    if (cudaStreamGetPriority(h->stream, &prio) != cudaSuccess) {
        cudaGetLastError();
        prio = 0;
    }
    for (int i = 0; i < Lanes::kCount; ++i) {
        HCUDA(cudaStreamCreateWithPriority(&L.s[i], cudaStreamNonBlocking, prio));
        HCUDA(cudaEventCreateWithFlags(&L.done[i], cudaEventDisableTiming));
        L.al[i].a = h->al.a;
        L.al[i].stream = L.s[i];
    }
    HCUDA(cudaEventCreateWithFlags(&L.fork, cudaEventDisableTiming));
}

// When `count` > 0 work items follow: every lane waits for everything queued so far on the
// handle's stream (all lanes, not only the ones the items use: a buffer a lane owns may be
// freed on it by an item, after the handle's stream last used it).
void lanes_fork(homln_t h, int count) {
    Lanes &L = h->lanes;
    if (count <= 0) return;
    HCUDA(cudaEventRecord(L.fork, h->stream));
    for (int i = 0; i < Lanes::kCount; ++i) HCUDA(cudaStreamWaitEvent(L.s[i], L.fork, 0));
}

// After `count` > 0 work items: the handle's stream waits for everything queued on the lanes.
void lanes_join(homln_t h, int count) {
    Lanes &L = h->lanes;
    if (count <= 0) return;
    for (int i = 0; i < Lanes::kCount; ++i) {
        HCUDA(cudaEventRecord(L.done[i], L.s[i]));
        HCUDA(cudaStreamWaitEvent(h->stream, L.done[i], 0));
    }
}

// Lanes forked for `count` work items, joined into the handle's stream by join() or, when an
// error unwinds the call first, by the destructor (which then ignores CUDA errors): the
// handle's stream never runs ahead of lane work that was already queued.
struct LaneScope {
    homln_t h;
    int count;
    LaneScope(homln_t h_, int c) : h(h_), count(c) { lanes_fork(h, count); }
    LaneScope(const LaneScope &) = delete;
    LaneScope &operator=(const LaneScope &) = delete;
    void join() {
        const int c = count;
        count = 0;
        lanes_join(h, c);
    }
    ~LaneScope() {
        if (count <= 0) return;
        for (int i = 0; i < Lanes::kCount; ++i)
            if (cudaEventRecord(h->lanes.done[i], h->lanes.s[i]) == cudaSuccess)
                cudaStreamWaitEvent(h->stream, h->lanes.done[i], 0);
        cudaGetLastError();
    }
};

// The CSR whose rows are the neighbours that reach a vertex: the in-edges of a directed graph.
const Csr &in_csr(homln_t h, const GraphState &g) { return h->directed ? g.csr_in : g.csr; }

int64_t edge_count(homln_t h, const GraphState &g) {
    const int64_t e = csr_nnz(g.csr, h->stream);
    return h->directed ? e : e / 2;
}

// Forget every cached analysis result (closeness, selections); CSRs and BFS graphs stay.
void drop_results(homln_t h) {
    auto drop = [](GraphState &g) {
        g.analysed = false;
        g.selections.clear();
        if (g.graph_refs > 0) return;  // a captured graph writes into these buffers
        g.F.release();
        g.R.release();
        g.cc.release();
        g.sumdist.release();
        g.deg.release();
    };
    for (auto &g : h->layers) drop(*g);
    for (auto &kv : h->ands) drop(*kv.second);
    for (auto &kv : h->ors) drop(*kv.second);
}

// Map a device-side error word to a status (and clear it).
void check_device_error(homln_t h) {
    int32_t e = 0;
    HCUDA(cudaMemcpyAsync(&e, h->err.p, sizeof(e), cudaMemcpyDeviceToHost, h->stream));
    HCUDA(cudaStreamSynchronize(h->stream));
    if (e == DEV_OK) return;
    HCUDA(cudaMemsetAsync(h->err.p, 0, sizeof(int32_t), h->stream));
    drop_results(h);  // what the failed work left in the cached results is not trusted
    switch (e) {
    case DEV_BAD_ID: fail(HOMLN_EINVAL, "node id outside [0, n)");
    case DEV_TIMEOUT: fail(HOMLN_ETIMEOUT, "a bounded device wait gave up");
    case DEV_RANGE: fail(HOMLN_ERANGE, "a value left the exact fixed-point range");
    default: fail(HOMLN_ECUDA, "unknown device error");
    }
}

// Copy `bytes` from device memory to `dst` (host or device). Returns true if dst is host memory.
bool put_out(homln_t h, void *dst, const void *dsrc, size_t bytes) {
    if (!dst || bytes == 0) return false;
    bool dev = is_device_ptr(dst);
    HCUDA(cudaMemcpyAsync(dst, dsrc, bytes, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
    return !dev;
}

// A device view of a caller buffer: the buffer itself if it is device memory, else a staging copy.
template <typename T>
struct DevIn {
    const T *p = nullptr;
    DBuf<T> tmp;
    void from(homln_t h, const T *src, size_t count) {
        if (count == 0 || is_device_ptr(src)) {
            p = src;
            return;
        }
        if (!tmp.alloc(&h->al, count)) fail(HOMLN_ENOMEM, "staging copy");
        HCUDA(cudaMemcpyAsync(tmp.p, src, count * sizeof(T), cudaMemcpyHostToDevice, h->stream));
        p = tmp.p;
    }
};

// A device target for an output: the caller's buffer if device memory, else scratch to copy from.
template <typename T>
struct DevOut {
    T *p = nullptr;
    T *user = nullptr;
    size_t count = 0;
    DBuf<T> tmp;
    void to(homln_t h, T *dst, size_t cnt) {
        user = dst;
        count = cnt;
        if (dst && is_device_ptr(dst)) {
            p = dst;
            return;
        }
        if (!tmp.alloc(&h->al, cnt > 0 ? cnt : 1)) fail(HOMLN_ENOMEM, "output scratch");
        p = tmp.p;
    }
    bool finish(homln_t h, size_t written) {
        if (!user || p == user || written == 0) return false;
        HCUDA(cudaMemcpyAsync(user, p, written * sizeof(T), cudaMemcpyDeviceToHost, h->stream));
        return true;
    }
};

using Items = std::vector<std::pair<homln_t, GraphState *>>;

// Make every graph of `todo` ready for a BFS launch on h's stream: result buffers allocated
// (kept if they exist), BFS graphs built, other handles' streams ordered before h's.
// `overlap`, if given, enqueues work of its own on h's stream while the lanes relabel.
std::vector<BfsJob> prepare_items(homln_t h, const Items &todo, const std::function<void()> &overlap = {}) {
    std::vector<BfsJob> jobs;
    std::vector<homln_t> others;
    std::vector<std::pair<homln_t, GraphState *>> prep;  // graphs whose BFS form must be (re)built
    for (const auto &it : todo) {
        homln_t o = it.first;
        GraphState *g = it.second;
        const int32_t n = o->n;
        if ((!g->F.p && !g->F.alloc(&o->al, n)) || (!g->R.p && !g->R.alloc(&o->al, n)) ||
            (!g->cc.p && !g->cc.alloc(&o->al, n)) || (!g->sumdist.p && !g->sumdist.alloc(&o->al, n)) ||
            (!g->deg.p && !g->deg.alloc(&o->al, n)))
            fail(HOMLN_ENOMEM, "closeness outputs");
        if (!g->bfs_ready || g->bfs.relabeled != (h->tuning.relabel != 0)) prep.push_back(it);
        jobs.push_back(BfsJob{&g->bfs, g->F.p, g->R.p});
        if (o != h && o->stream != h->stream && std::find(others.begin(), others.end(), o) == others.end())
            others.push_back(o);
    }
    // Rebuilding a BFS graph (its relabelling setting changed) frees the old one on the stream
    // that owns it, which need not be ordered after the launches that read it: wait for the
    // device first (a rare path).
    bool rebuild = false;
    for (const auto &it : prep) {
        rebuild |= it.second->bfs_ready;
        if (it.second->bfs_ready && it.second->graph_refs > 0)
            fail(HOMLN_EBUSY, "a captured graph uses this BFS graph; destroy it before changing the relabelling");
    }
    if (rebuild) {
        HCUDA(cudaDeviceSynchronize());
        for (const auto &it : prep) {
            it.second->bfs = BfsGraph();
            it.second->bfs_ready = false;
        }
    }
    // the relabellings of h's graphs run on h's lanes side by side; other handles' on their streams
    int nl = 0;
    for (const auto &it : prep) nl += it.first == h;
    LaneScope lanes(h, nl);
    int k = 0;
    for (const auto &it : prep) {
        homln_t o = it.first;
        GraphState *g = it.second;
        const Csr *gin = o->directed ? &g->csr_in : nullptr;
        if (o == h) {
            const int j = k++ % Lanes::kCount;
            bfs_prepare(g->csr, gin, h->tuning.relabel != 0, g->bfs, &h->lanes.al[j], h->lanes.s[j]);
        } else {
            bfs_prepare(g->csr, gin, h->tuning.relabel != 0, g->bfs, &o->al, o->stream);
        }
        g->bfs_ready = true;
    }
    if (overlap) overlap();
    lanes.join();
    for (homln_t o : others) {  // h's stream waits for the CSRs and outputs queued on the other streams
        cudaEvent_t e;
        HCUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        HCUDA(cudaEventRecord(e, o->stream));
        HCUDA(cudaStreamWaitEvent(h->stream, e, 0));
        cudaEventDestroy(e);
    }
    return jobs;
}

// The other handles' streams of `todo` wait for everything queued so far on h's stream.
void order_after(homln_t h, const Items &todo) {
    std::vector<homln_t> others;
    for (const auto &it : todo)
        if (it.first != h && it.first->stream != h->stream &&
            std::find(others.begin(), others.end(), it.first) == others.end())
            others.push_back(it.first);
    for (homln_t o : others) {
        cudaEvent_t e;
        HCUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        HCUDA(cudaEventRecord(e, h->stream));
        HCUDA(cudaStreamWaitEvent(o->stream, e, 0));
        cudaEventDestroy(e);
    }
}

// Psi for every (handle, graph) item not analysed yet, in one persistent BFS launch on the
// stream of `h` (the other handles' streams are ordered around it with events). Each graph's
// outputs are allocated through its own handle.
void analyse_items(homln_t h, const Items &items) {
    Items todo;
    for (const auto &it : items)
        if (!it.second->analysed &&
            std::find_if(todo.begin(), todo.end(), [&](const auto &x) { return x.second == it.second; }) == todo.end())
            todo.push_back(it);
    if (todo.empty()) return;
    std::vector<BfsJob> jobs = prepare_items(h, todo);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (h->profiling) {
        HCUDA(cudaEventCreate(&e0));
        HCUDA(cudaEventCreate(&e1));
        h->events.push_back({e0, e1});
    }
    BfsStats st;
    msbfs_multi(jobs, h->tuning, h->err.p, &h->al, h->stream, h->instrument ? &st : nullptr, e0, e1);
    if (h->instrument) {
        h->stats.levels += st.levels;
        h->stats.pull_levels += st.pull_levels;
        h->stats.push_levels += st.push_levels;
        h->stats.group_edges += st.group_edges;
        h->stats.lane_words += st.lane_words;
        h->stats.push_edges += st.push_edges;
        h->stats.batches += st.batches;
        h->stats.push_words += st.push_words;
        h->stats.bytes += st.bytes;
        h->stats.visits += st.visits;
        h->stats.words_per_node = st.words_per_node;
        h->stats.teams = st.teams;
    }
    h->bfs_launches += 1;
    for (const auto &it : todo) {
        GraphState *g = it.second;
        closeness_finalize(it.first->n, in_csr(it.first, *g).rowptr.p, g->F.p, g->R.p, g->cc.p, g->sumdist.p, g->deg.p,
                           h->stream);
        g->analysed = true;
    }
    order_after(h, todo);  // and the other streams wait for the results
}

void analyse_many(homln_t h, const std::vector<GraphState *> &gs) {
    std::vector<std::pair<homln_t, GraphState *>> items;
    for (GraphState *g : gs) items.push_back({h, g});
    analyse_items(h, items);
}

void analyse(homln_t h, GraphState &g) { analyse_many(h, {&g}); }

std::vector<int> mask_layers(homln_t h, uint64_t mask) {
    if (mask == 0) fail(HOMLN_EINVAL, "empty layer mask");
    if (h->L < 64 && (mask >> h->L) != 0) fail(HOMLN_EINVAL, "layer mask names a layer that does not exist");
    std::vector<int> out;
    for (int i = 0; i < h->L; ++i)
        if ((mask >> i) & 1ull) out.push_back(i);
    return out;
}

GraphState &and_graph(homln_t h, uint64_t mask) {
    std::vector<int> ids = mask_layers(h, mask);
    auto it = h->ands.find(mask);
    if (it != h->ands.end()) return *it->second;
    auto g = std::make_unique<GraphState>();
    auto copy = [&](const Csr &src, Csr &dst) {
        dst.n = src.n;
        dst.nnz = src.nnz;
        dst.cap = src.cap;
        if (!dst.rowptr.alloc(&h->al, (size_t)h->n + 1) || !dst.col.alloc(&h->al, src.cap > 0 ? src.cap : 1))
            fail(HOMLN_ENOMEM, "and graph");
        HCUDA(cudaMemcpyAsync(dst.rowptr.p, src.rowptr.p, sizeof(int64_t) * (h->n + 1), cudaMemcpyDeviceToDevice,
                              h->stream));
        if (src.cap > 0)
            HCUDA(cudaMemcpyAsync(dst.col.p, src.col.p, sizeof(int32_t) * src.cap, cudaMemcpyDeviceToDevice,
                                  h->stream));
    };
    if (ids.size() == 1) {
        copy(h->layers[ids[0]]->csr, g->csr);
        if (h->directed) copy(h->layers[ids[0]]->csr_in, g->csr_in);
    } else {
        std::vector<const Csr *> ls, lin;
        for (int i : ids) {
            ls.push_back(&h->layers[i]->csr);
            lin.push_back(&h->layers[i]->csr_in);
        }
        and_intersect(h->n, ls, g->csr, &h->al, h->stream);
        if (h->directed) and_intersect(h->n, lin, g->csr_in, &h->al, h->stream);
    }
    GraphState &ref = *g;
    h->ands.emplace(mask, std::move(g));
    return ref;
}

// The graph's CC nodes under `sel`, computed once and cached (the closeness values never change).
SelKey selection_key(const homln_select &sel) {
    return std::make_tuple(sel.mode, sel.mode == HOMLN_TOPK_PERCENT ? sel.percent : 0.0,
                           sel.mode == HOMLN_TOPK_COUNT ? sel.k : (int64_t)0);
}

Selection &selection_of(homln_t h, GraphState &g, const homln_select &sel) {
    const SelKey key = selection_key(sel);
    auto it = g.selections.find(key);
    if (it != g.selections.end()) return *it->second;
    auto s = std::make_unique<Selection>();
    if (!s->ranked.alloc(&h->al, h->n) || !s->bits.alloc(&h->al, ceil_div(h->n, 32)))
        fail(HOMLN_ENOMEM, "selection");
    s->count = select_nodes(h->n, g.cc.p, sel, s->ranked.p, s->bits.p, h->err.p, &h->al, h->stream);
    Selection &ref = *s;
    g.selections.emplace(key, std::move(s));
    return ref;
}

// The CC nodes of several graphs under `sel`: those not cached yet are selected on the lanes
// side by side (their outputs are allocated on the handle's stream first).
void selections_of(homln_t h, const std::vector<GraphState *> &gs, const homln_select &sel) {
    const SelKey key = selection_key(sel);
    std::vector<std::pair<GraphState *, Selection *>> todo;
    for (GraphState *g : gs) {
        if (g->selections.count(key)) continue;
        auto s = std::make_unique<Selection>();
        if (!s->ranked.alloc(&h->al, h->n) || !s->bits.alloc(&h->al, ceil_div(h->n, 32)))
            fail(HOMLN_ENOMEM, "selection");
        todo.push_back({g, s.get()});
        g->selections.emplace(key, std::move(s));
    }
    if (todo.empty()) return;
    LaneScope lanes(h, (int)todo.size());
    for (size_t i = 0; i < todo.size(); ++i) {
        const int j = (int)(i % Lanes::kCount);
        todo[i].second->count = select_nodes(h->n, todo[i].first->cc.p, sel, todo[i].second->ranked.p,
                                             todo[i].second->bits.p, h->err.p, &h->lanes.al[j], h->lanes.s[j]);
    }
    lanes.join();
}

GraphState &or_graph(homln_t h, uint64_t mask) {
    std::vector<int> ids = mask_layers(h, mask);
    auto it = h->ors.find(mask);
    if (it != h->ors.end()) return *it->second;
    auto g = std::make_unique<GraphState>();
    std::vector<const Csr *> ls, lin;
    for (int i : ids) {
        ls.push_back(&h->layers[i]->csr);
        lin.push_back(&h->layers[i]->csr_in);
    }
    or_union(h->n, ls, g->csr, &h->al, h->stream);
    if (h->directed) or_union(h->n, lin, g->csr_in, &h->al, h->stream);
    GraphState &ref = *g;
    h->ors.emplace(mask, std::move(g));
    return ref;
}

void check_select(const homln_select *sel) {
    if (!sel) fail(HOMLN_EINVAL, "selection is NULL");
    if (sel->reserved != 0) fail(HOMLN_EINVAL, "homln_select.reserved must be 0");
    if (sel->mode < HOMLN_TOPK_PERCENT || sel->mode > HOMLN_GT_MEAN) fail(HOMLN_EINVAL, "unknown selection mode");
    if (sel->mode == HOMLN_TOPK_PERCENT && !(sel->percent >= 0.0 && sel->percent <= 100.0))
        fail(HOMLN_EINVAL, "percent must be in [0, 100]");
    if (sel->mode == HOMLN_TOPK_COUNT && sel->k < 0) fail(HOMLN_EINVAL, "k must be >= 0");
    if (!(sel->cc1_overlap >= 0.0 && sel->cc1_overlap <= 1.0)) fail(HOMLN_EINVAL, "cc1_overlap must be in [0, 1]");
}

void write_closeness(homln_t h, GraphState &g, uint64_t *F, uint32_t *R, double *cc) {
    bool host = false;
    host |= put_out(h, F, g.F.p, sizeof(uint64_t) * h->n);
    host |= put_out(h, R, g.R.p, sizeof(uint32_t) * h->n);
    host |= put_out(h, cc, g.cc.p, sizeof(double) * h->n);
    if (host) check_device_error(h);
}

}  // namespace

extern "C" {

const char *homln_last_error(void) { return g_last_error.c_str(); }

const char *homln_version(void) { return "homln-gb300 0.1 (sm_103a)"; }

// One int32 in pinned host memory, mapped into the device's address space.
struct homln_yield_s {
    int32_t *host = nullptr;
    int32_t *dev = nullptr;
    std::atomic<long long> count{0};
    std::atomic<int> watchers{0};  // handles whose BFS watches this flag
    ~homln_yield_s() {
        if (host) cudaFreeHost(host);
    }
};

homln_status homln_yield_create(homln_yield_t *out) {
    API_BEGIN
    if (!out) fail(HOMLN_EINVAL, "out is NULL");
    auto y = std::make_unique<homln_yield_s>();
    void *p = nullptr;
    HCUDA(cudaHostAlloc(&p, 64, cudaHostAllocMapped | cudaHostAllocPortable));
    y->host = static_cast<int32_t *>(p);
    __atomic_store_n(y->host, 0, __ATOMIC_RELEASE);
    void *d = nullptr;
    HCUDA(cudaHostGetDevicePointer(&d, p, 0));
    y->dev = static_cast<int32_t *>(d);
    *out = y.release();
    API_END
}

homln_status homln_yield_destroy(homln_yield_t y) {
    API_BEGIN
    if (y && y->watchers.load() > 0)
        fail(HOMLN_EBUSY, "a handle still watches this yield flag (homln_set_yield(h, NULL) or destroy it first)");
    delete y;
    API_END
}

homln_status homln_yield_set(homln_yield_t y, int32_t raised) {
    API_BEGIN
    if (!y) fail(HOMLN_EINVAL, "yield flag is NULL");
    __atomic_store_n(y->host, raised ? 1 : 0, __ATOMIC_SEQ_CST);
    API_END
}

homln_status homln_yield_count(homln_yield_t y, int64_t *out) {
    API_BEGIN
    if (!y || !out) fail(HOMLN_EINVAL, "yield flag and out are required");
    *out = (int64_t)y->count.load();
    API_END
}

homln_status homln_set_yield(homln_t h, homln_yield_t y) {
    API_BEGIN
    if (!h) fail(HOMLN_EINVAL, "handle is NULL");
    if (h->live_graphs > 0) fail(HOMLN_EBUSY, "a captured graph uses this handle");
    if (h->yield) h->yield->watchers.fetch_sub(1);
    h->yield = y;
    if (y) y->watchers.fetch_add(1);
    h->tuning.yield_host = y ? y->host : nullptr;
    h->tuning.yield_dev = y ? y->dev : nullptr;
    h->tuning.yield_count = y ? &y->count : nullptr;
    API_END
}

homln_status homln_create(int32_t n_nodes, int32_t n_layers, const int64_t *edge_counts, const int32_t *const *src,
                          const int32_t *const *dst, uint32_t flags, const homln_allocator *alloc, void *stream,
                          homln_t *out) {
    API_BEGIN
    if (!out) fail(HOMLN_EINVAL, "out is NULL");
    if (n_nodes < 1 || n_nodes > HOMLN_MAX_NODES) fail(HOMLN_EINVAL, "n_nodes must be in [1, 2^20]");
    if (n_layers < 1 || n_layers > HOMLN_MAX_LAYERS) fail(HOMLN_EINVAL, "n_layers must be in [1, 64]");
    if (!edge_counts || !src || !dst) fail(HOMLN_EINVAL, "edge_counts, src and dst must not be NULL");
    if (flags & ~(HOMLN_PTR_DEVICE | HOMLN_DIRECTED)) fail(HOMLN_EINVAL, "unknown flags");
    for (int i = 0; i < n_layers; ++i) {
        if (edge_counts[i] < 0 || edge_counts[i] > (int64_t(1) << 31)) fail(HOMLN_EINVAL, "edge count out of range");
        if (edge_counts[i] > 0 && (!src[i] || !dst[i])) fail(HOMLN_EINVAL, "edge array is NULL");
    }
    if (alloc && (!alloc->alloc || !alloc->free)) fail(HOMLN_EINVAL, "allocator needs both alloc and free");
    auto h = std::make_unique<homln_s>();
    HCUDA(cudaGetDevice(&h->device));
    h->stream = (cudaStream_t)stream;
    h->al.stream = h->stream;
    if (alloc) h->al.a = *alloc;
    else std::memset(&h->al.a, 0, sizeof(h->al.a));
    h->n = n_nodes;
    h->L = n_layers;
    h->directed = (flags & HOMLN_DIRECTED) != 0;
    lanes_open(h.get());
    if (!h->err.alloc(&h->al, 1)) fail(HOMLN_ENOMEM, "error word");
    HCUDA(cudaMemsetAsync(h->err.p, 0, sizeof(int32_t), h->stream));
    // host edge lists are staged on the handle's stream; then the layers' CSRs are built on the lanes
    std::vector<DBuf<int32_t>> staged(2 * (size_t)n_layers);
    std::vector<const int32_t *> ps(n_layers), pd(n_layers);
    for (int i = 0; i < n_layers; ++i) {
        const int64_t m = edge_counts[i];
        ps[i] = src[i];
        pd[i] = dst[i];
        if (m > 0 && !(flags & HOMLN_PTR_DEVICE)) {
            DBuf<int32_t> &ds = staged[2 * i], &dd = staged[2 * i + 1];
            if (!ds.alloc(&h->al, m) || !dd.alloc(&h->al, m)) fail(HOMLN_ENOMEM, "edge staging");
            HCUDA(cudaMemcpyAsync(ds.p, ps[i], sizeof(int32_t) * m, cudaMemcpyHostToDevice, h->stream));
            HCUDA(cudaMemcpyAsync(dd.p, pd[i], sizeof(int32_t) * m, cudaMemcpyHostToDevice, h->stream));
            ps[i] = ds.p;
            pd[i] = dd.p;
        }
        h->layers.push_back(std::make_unique<GraphState>());
    }
    LaneScope lanes(h.get(), n_layers);
    for (int i = 0; i < n_layers; ++i) {
        const int j = i % Lanes::kCount;
        GraphState &g = *h->layers[i];
        build_csr(n_nodes, ps[i], pd[i], edge_counts[i], g.csr, h->err.p, &h->lanes.al[j], h->lanes.s[j], h->directed);
        if (h->directed)
            build_csr(n_nodes, pd[i], ps[i], edge_counts[i], g.csr_in, h->err.p, &h->lanes.al[j], h->lanes.s[j], true);
    }
    lanes.join();
    check_device_error(h.get());
    *out = h.release();
    API_END
}

homln_status homln_destroy(homln_t h) {
    if (!h) return HOMLN_OK;
    API_BEGIN
    if (h->live_graphs > 0) fail(HOMLN_EBUSY, "a captured graph still uses this handle; destroy it first");
    homln_set_yield(h, nullptr);  // stop watching a yield flag, so that the flag can be destroyed
    cudaSetDevice(h->device);
    cudaStream_t s = h->stream;
    // buffers owned by a lane are freed on it: after everything queued on the handle's stream
    lanes_fork(h, Lanes::kCount);
    delete h;
    HCUDA(cudaStreamSynchronize(s));
    API_END
}

homln_status homln_set_tuning(homln_t h, const homln_tuning *t) {
    API_BEGIN
    if (!h) fail(HOMLN_EINVAL, "null handle");
    BfsTuning bt;
    if (t) {
        if (t->words_per_node) {
            int W = t->words_per_node;
            if (W != 1 && W != 2 && W != 4 && W != 8 && W != 16 && W != 32)
                fail(HOMLN_EINVAL, "words_per_node must be 1, 2, 4, 8, 16 or 32");
            bt.W = W;
        }
        if (t->push_alpha < 0) fail(HOMLN_EINVAL, "push_alpha must be >= 0");
        if (t->push_alpha) bt.push_alpha = t->push_alpha;
        if (t->threads) {
            if (t->threads < 64 || t->threads > 512 || t->threads % 32) fail(HOMLN_EINVAL, "threads must be 64..512, x32");
            bt.threads = t->threads;
        }
        if (t->blocks_per_sm < 0) fail(HOMLN_EINVAL, "blocks_per_sm must be >= 0");
        bt.blocks_per_sm = t->blocks_per_sm;
        if (t->relabel >= 0) bt.relabel = t->relabel ? 1 : 0;
        if (t->teams < 0) fail(HOMLN_EINVAL, "teams must be >= 0");
        bt.teams = t->teams;
        bt.team_mix = t->team_mix ? 1 : 0;
        if (t->schedule < 0 || t->schedule > 1) fail(HOMLN_EINVAL, "schedule must be 0 or 1");
        bt.schedule = t->schedule;
        if (t->wait_limit_ms < 0 || t->wait_limit_ms > 60000) fail(HOMLN_EINVAL, "wait_limit_ms must be in [0, 60000]");
        if (t->wait_limit_ms) bt.wait_limit_ms = t->wait_limit_ms;
        if (t->test_phantom_blocks < 0 || t->test_phantom_blocks > 1024)
            fail(HOMLN_EINVAL, "test_phantom_blocks must be in [0, 1024]");
        bt.phantom = t->test_phantom_blocks;
        if (t->max_tiles_per_launch < 0) fail(HOMLN_EINVAL, "max_tiles_per_launch must be >= 0");
        bt.max_tiles = t->max_tiles_per_launch;
        if (t->sm_count < 0) fail(HOMLN_EINVAL, "sm_count must be >= 0");
        bt.sm_count = t->sm_count;
    }
    bt.yield_host = h->tuning.yield_host;  // the yield flag is set apart (homln_set_yield)
    bt.yield_dev = h->tuning.yield_dev;
    bt.yield_count = h->tuning.yield_count;
    h->tuning = bt;
    API_END
}

homln_status homln_layer_closeness(homln_t h, int32_t layer, uint64_t *farness, uint32_t *reach, double *cc) {
    API_BEGIN
    if (!h) fail(HOMLN_EINVAL, "null handle");
    if (layer < 0 || layer >= h->L) fail(HOMLN_EINVAL, "layer out of range");
    use_device(h);
    GraphState &g = *h->layers[layer];
    analyse(h, g);
    write_closeness(h, g, farness, reach, cc);
    API_END
}

homln_status homln_analyse(homln_t h, uint64_t layer_mask, int32_t with_and) {
    API_BEGIN
    if (!h) fail(HOMLN_EINVAL, "null handle");
    use_device(h);
    std::vector<GraphState *> gs;
    Items layers;
    for (int i : mask_layers(h, layer_mask)) {
        gs.push_back(h->layers[i].get());
        if (!h->layers[i]->analysed) layers.push_back({h, h->layers[i].get()});
    }
    // the AND graph is built, and relabelled, on the handle's stream while the lanes relabel the layers
    GraphState *andg = nullptr;
    prepare_items(h, layers, [&] {
        if (!with_and) return;
        andg = &and_graph(h, layer_mask);
        if (!andg->analysed && !andg->bfs_ready) {  // a rebuild (relabelling changed) is left to analyse_many
            bfs_prepare(andg->csr, h->directed ? &andg->csr_in : nullptr, h->tuning.relabel != 0, andg->bfs,
                        &h->al, h->stream);
            andg->bfs_ready = true;
        }
    });
    if (andg) gs.push_back(andg);
    analyse_many(h, gs);
    API_END
}

homln_status homln_batch_analyse(homln_t *nets, int32_t count, const uint64_t *masks, int32_t with_and) {
    API_BEGIN
    if (!nets || !masks || count < 1) fail(HOMLN_EINVAL, "nets, masks and count >= 1 are required");
    for (int32_t i = 0; i < count; ++i)
        if (!nets[i]) fail(HOMLN_EINVAL, "null handle in nets");
    homln_t h = nets[0];
    for (int32_t i = 1; i < count; ++i)
        if (nets[i]->device != h->device) fail(HOMLN_EINVAL, "all handles must live on one device");
    use_device(h);
    std::vector<std::pair<homln_t, GraphState *>> items;
    for (int32_t i = 0; i < count; ++i) {
        for (int l : mask_layers(nets[i], masks[i])) items.push_back({nets[i], nets[i]->layers[l].get()});
        if (with_and) items.push_back({nets[i], &and_graph(nets[i], masks[i])});
    }
    analyse_items(h, items);
    API_END
}

homln_status homln_batch_closeness(homln_t *nets, int32_t count, void *stream) {
    API_BEGIN
    if (!nets || count < 1) fail(HOMLN_EINVAL, "nets and count >= 1 are required");
    std::vector<uint64_t> masks(count);
    for (int32_t i = 0; i < count; ++i) {
        if (!nets[i]) fail(HOMLN_EINVAL, "null handle in nets");
        masks[i] = nets[i]->L >= 64 ? ~0ull : (1ull << nets[i]->L) - 1;
    }
    homln_t h = nets[0];
    use_device(h);
    cudaStream_t s = (cudaStream_t)stream;
    const bool other = s != h->stream;
    cudaEvent_t e = nullptr;
    if (other) {  // the launch stream waits for `stream`, and `stream` for the results
        HCUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        HCUDA(cudaEventRecord(e, s));
        HCUDA(cudaStreamWaitEvent(h->stream, e, 0));
    }
    homln_status st = homln_batch_analyse(nets, count, masks.data(), 1);
    if (other) {
        HCUDA(cudaEventRecord(e, h->stream));
        HCUDA(cudaStreamWaitEvent(s, e, 0));
        cudaEventDestroy(e);
    }
    if (st != HOMLN_OK) fail(st, homln_last_error());
    API_END
}

}  // extern "C"

// A captured analysis: the plan's buffers, the graphs it writes, and the instantiated graph.
struct homln_graph_s {
    homln_t h = nullptr;  // the launching handle (its stream, tuning and error word)
    Items items;
    std::vector<homln_t> handles;
    BfsPlan *plan = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    ~homln_graph_s() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        bfs_plan_destroy(plan);
        for (auto &it : items) it.second->graph_refs -= 1;
        for (homln_t o : handles) o->live_graphs -= 1;
    }
};

extern "C" {

homln_status homln_graph_capture(homln_t *nets, int32_t count, const uint64_t *masks, int32_t with_and,
                                 homln_graph_t *out) {
    API_BEGIN
    if (!nets || !masks || count < 1 || !out) fail(HOMLN_EINVAL, "nets, masks, count >= 1 and out are required");
    for (int32_t i = 0; i < count; ++i)
        if (!nets[i]) fail(HOMLN_EINVAL, "null handle in nets");
    homln_t h = nets[0];
    for (int32_t i = 1; i < count; ++i)
        if (nets[i]->device != h->device) fail(HOMLN_EINVAL, "all handles must live on one device");
    if (h->tuning.schedule == 1) fail(HOMLN_EINVAL, "the plain schedule cannot be captured (the host drives it)");
    if (h->instrument) fail(HOMLN_EINVAL, "an instrumented handle cannot be captured");
    if (h->tuning.yield_dev) fail(HOMLN_EINVAL, "a handle that watches a yield flag cannot be captured");
    use_device(h);
    Items items;
    for (int32_t i = 0; i < count; ++i) {
        std::vector<GraphState *> gs;
        for (int l : mask_layers(nets[i], masks[i])) gs.push_back(nets[i]->layers[l].get());
        if (with_and) gs.push_back(&and_graph(nets[i], masks[i]));
        for (GraphState *g : gs)
            if (std::find_if(items.begin(), items.end(), [&](const auto &x) { return x.second == g; }) == items.end())
                items.push_back({nets[i], g});
    }
    auto gr = std::make_unique<homln_graph_s>();
    gr->h = h;
    std::vector<BfsJob> jobs = prepare_items(h, items);
    gr->plan = bfs_plan_create(jobs, h->tuning, h->err.p, &h->al, h->stream, false);
    for (int32_t i = 0; i < count; ++i) HCUDA(cudaStreamSynchronize(nets[i]->stream));  // preparation done
    // captured on a private stream (the handle's may be the legacy default stream, which cannot
    // be captured); replays run on the handle's stream
    struct CaptureStream {
        cudaStream_t s = nullptr;
        ~CaptureStream() {
            if (s) cudaStreamDestroy(s);
        }
    } cs;
    HCUDA(cudaStreamCreateWithFlags(&cs.s, cudaStreamNonBlocking));
    HCUDA(cudaStreamBeginCapture(cs.s, cudaStreamCaptureModeThreadLocal));
    try {
        bfs_plan_run(gr->plan, cs.s, nullptr, nullptr);
        for (const auto &it : items) {
            GraphState *g = it.second;
            closeness_finalize(it.first->n, in_csr(it.first, *g).rowptr.p, g->F.p, g->R.p, g->cc.p, g->sumdist.p,
                               g->deg.p, cs.s);
        }
    } catch (...) {
        cudaGraph_t partial = nullptr;
        cudaStreamEndCapture(cs.s, &partial);
        if (partial) cudaGraphDestroy(partial);
        cudaGetLastError();
        throw;
    }
    HCUDA(cudaStreamEndCapture(cs.s, &gr->graph));
    HCUDA(cudaGraphInstantiate(&gr->exec, gr->graph, 0));
    gr->items = items;
    for (auto &it : gr->items) it.second->graph_refs += 1;
    for (const auto &it : items)
        if (std::find(gr->handles.begin(), gr->handles.end(), it.first) == gr->handles.end()) {
            gr->handles.push_back(it.first);
            it.first->live_graphs += 1;
        }
    *out = gr.release();
    API_END
}

homln_status homln_graph_launch(homln_graph_t g) {
    API_BEGIN
    if (!g) fail(HOMLN_EINVAL, "null graph");
    homln_t h = g->h;
    use_device(h);
    // the other handles' streams are ordered before and after the replay on h's stream
    for (homln_t o : g->handles)
        if (o != h && o->stream != h->stream) {
            cudaEvent_t e;
            HCUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            HCUDA(cudaEventRecord(e, o->stream));
            HCUDA(cudaStreamWaitEvent(h->stream, e, 0));
            cudaEventDestroy(e);
        }
    HCUDA(cudaGraphLaunch(g->exec, h->stream));
    h->bfs_launches += 1;
    for (auto &it : g->items) {
        it.second->analysed = true;
        it.second->selections.clear();
    }
    order_after(h, g->items);
    API_END
}

homln_status homln_graph_destroy(homln_graph_t g) {
    if (!g) return HOMLN_OK;
    API_BEGIN
    cudaSetDevice(g->h->device);
    for (homln_t o : g->handles) HCUDA(cudaStreamSynchronize(o->stream));
    delete g;
    API_END
}

homln_status homln_and_aggregate(homln_t h, uint64_t layer_mask, int64_t capacity, int32_t *and_src, int32_t *and_dst,
                                 int64_t *and_edge_count) {
    API_BEGIN
    if (!h) fail(HOMLN_EINVAL, "null handle");
    if (!and_edge_count) fail(HOMLN_EINVAL, "and_edge_count is NULL");
    if ((and_src == nullptr) != (and_dst == nullptr)) fail(HOMLN_EINVAL, "and_src and and_dst must both be given");
    use_device(h);
    GraphState &g = and_graph(h, layer_mask);
    const int64_t m = edge_count(h, g);
    if (and_src) {
        if (capacity < m) {
            *and_edge_count = m;
            fail(HOMLN_ERANGE, "capacity smaller than the AND edge count");
        }
        DevOut<int32_t> os, od;
        os.to(h, and_src, m);
        od.to(h, and_dst, m);
        csr_edge_list(g.csr, os.p, od.p, &h->al, h->stream, h->directed);
        bool host = os.finish(h, m);
        host |= od.finish(h, m);
        if (host) HCUDA(cudaStreamSynchronize(h->stream));
    }
    *and_edge_count = m;
    API_END
}

homln_status homln_or_aggregate(homln_t h, uint64_t layer_mask, int64_t capacity, int32_t *or_src, int32_t *or_dst,
                                int64_t *or_edge_count) {
    API_BEGIN
    if (!h) fail(HOMLN_EINVAL, "null handle");
    if (!or_edge_count) fail(HOMLN_EINVAL, "or_edge_count is NULL");
    if ((or_src == nullptr) != (or_dst == nullptr)) fail(HOMLN_EINVAL, "or_src and or_dst must both be given");
    use_device(h);
    GraphState &g = or_graph(h, layer_mask);
    const int64_t m = edge_count(h, g);
    if (or_src) {
        if (capacity < m) {
            *or_edge_count = m;
            fail(HOMLN_ERANGE, "capacity smaller than the OR edge count");
        }
        DevOut<int32_t> os, od;
        os.to(h, or_src, m);
        od.to(h, or_dst, m);
        csr_edge_list(g.csr, os.p, od.p, &h->al, h->stream, h->directed);
        bool host = os.finish(h, m);
        host |= od.finish(h, m);
        if (host) HCUDA(cudaStreamSynchronize(h->stream));
    }
    *or_edge_count = m;
    API_END
}

homln_status homln_or_closeness(homln_t h, uint64_t layer_mask, uint64_t *farness, uint32_t *reach, double *cc) {
    API_BEGIN
    if (!h) fail(HOMLN_EINVAL, "null handle");
    use_device(h);
    GraphState &g = or_graph(h, layer_mask);
    analyse(h, g);
    write_closeness(h, g, farness, reach, cc);
    API_END
}

homln_status homln_and_closeness(homln_t h, uint64_t layer_mask, uint64_t *farness, uint32_t *reach, double *cc) {
    API_BEGIN
    if (!h) fail(HOMLN_EINVAL, "null handle");
    use_device(h);
    GraphState &g = and_graph(h, layer_mask);
    analyse(h, g);
    write_closeness(h, g, farness, reach, cc);
    API_END
}

namespace {
GraphState &graph_of(homln_t h, int32_t which, uint64_t layer_mask) {
    if (which < -2 || which >= h->L) fail(HOMLN_EINVAL, "which must be -2, -1 or a layer id");
    return which >= 0 ? *h->layers[which] : which == -1 ? and_graph(h, layer_mask) : or_graph(h, layer_mask);
}
}  // namespace

homln_status homln_shard_partials(homln_t h, int32_t which, uint64_t layer_mask, int32_t rank, int32_t world,
                                  uint64_t *farness, uint32_t *reach) {
    API_BEGIN
    if (!h) fail(HOMLN_EINVAL, "null handle");
    if (!farness || !reach) fail(HOMLN_EINVAL, "farness and reach are required");
    if (world < 1 || world > 65536 || rank < 0 || rank >= world) fail(HOMLN_EINVAL, "need 0 <= rank < world");
    if (h->tuning.schedule == 1) fail(HOMLN_EINVAL, "sharded partials use the persistent schedule");
    use_device(h);
    GraphState &g = graph_of(h, which, layer_mask);
    // the graph's BFS form, as an analysis would build it; the partial sums go to scratch
    Items one{{h, &g}};
    prepare_items(h, one);
    const int32_t n = h->n;
    DBuf<uint64_t> F;
    DBuf<uint32_t> R;
    if (!F.alloc(&h->al, n) || !R.alloc(&h->al, n)) fail(HOMLN_ENOMEM, "shard partials");
    BfsTuning t = h->tuning;
    t.shard_rank = rank;
    t.shard_world = world;
    msbfs_multi({BfsJob{&g.bfs, F.p, R.p}}, t, h->err.p, &h->al, h->stream, nullptr, nullptr, nullptr);
    h->bfs_launches += 1;
    bool host = put_out(h, farness, F.p, sizeof(uint64_t) * n);
    host |= put_out(h, reach, R.p, sizeof(uint32_t) * n);
    if (host) check_device_error(h);
    API_END
}

homln_status homln_export_partials(homln_t h, int32_t which, uint64_t layer_mask, uint64_t *farness, uint32_t *reach,
                                   int32_t *degree) {
    API_BEGIN
    if (!h) fail(HOMLN_EINVAL, "null handle");
    if (!farness || !reach) fail(HOMLN_EINVAL, "farness and reach are required");
    use_device(h);
    GraphState &g = graph_of(h, which, layer_mask);
    analyse(h, g);
    bool host = put_out(h, farness, g.F.p, sizeof(uint64_t) * h->n);
    host |= put_out(h, reach, g.R.p, sizeof(uint32_t) * h->n);
    host |= put_out(h, degree, g.deg.p, sizeof(int32_t) * h->n);
    if (host) check_device_error(h);
    API_END
}

homln_status homln_import_partials(homln_t h, int32_t which, uint64_t layer_mask, const uint64_t *farness,
                                   const uint32_t *reach) {
    API_BEGIN
    if (!h) fail(HOMLN_EINVAL, "null handle");
    if (!farness || !reach) fail(HOMLN_EINVAL, "farness and reach are required");
    use_device(h);
    GraphState &g = graph_of(h, which, layer_mask);
    const int32_t n = h->n;
    DevIn<uint64_t> F;
    DevIn<uint32_t> R;
    F.from(h, farness, n);
    R.from(h, reach, n);
    // validated with a flag of its own, so a refusal leaves the handle's error word and results alone
    DBuf<int32_t> bad;
    if (!bad.alloc(&h->al, 1)) fail(HOMLN_ENOMEM, "import flag");
    HCUDA(cudaMemsetAsync(bad.p, 0, sizeof(int32_t), h->stream));
    partials_check(n, F.p, R.p, bad.p, h->stream);
    int32_t hbad = 0;
    HCUDA(cudaMemcpyAsync(&hbad, bad.p, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
    HCUDA(cudaStreamSynchronize(h->stream));
    if (hbad) fail(HOMLN_ERANGE, "imported farness/reach cannot come from a BFS on n nodes");
    DBuf<uint64_t> nF, sd;
    DBuf<uint32_t> nR;
    DBuf<double> cc;
    DBuf<int32_t> deg;
    if (!nF.alloc(&h->al, n) || !nR.alloc(&h->al, n) || !cc.alloc(&h->al, n) || !sd.alloc(&h->al, n) ||
        !deg.alloc(&h->al, n))
        fail(HOMLN_ENOMEM, "imported results");
    HCUDA(cudaMemcpyAsync(nF.p, F.p, sizeof(uint64_t) * n, cudaMemcpyDefault, h->stream));
    HCUDA(cudaMemcpyAsync(nR.p, R.p, sizeof(uint32_t) * n, cudaMemcpyDefault, h->stream));
    closeness_finalize(n, in_csr(h, g).rowptr.p, nF.p, nR.p, cc.p, sd.p, deg.p, h->stream);
    g.selections.clear();
    g.F = std::move(nF);
    g.R = std::move(nR);
    g.cc = std::move(cc);
    g.sumdist = std::move(sd);
    g.deg = std::move(deg);
    g.analysed = true;
    API_END
}

homln_status homln_topk(homln_t h, int32_t which, uint64_t layer_mask, const homln_select *sel, int32_t *nodes_out,
                        int32_t *count_out) {
    API_BEGIN
    if (!h) fail(HOMLN_EINVAL, "null handle");
    check_select(sel);
    if (!count_out) fail(HOMLN_EINVAL, "count_out is NULL");
    if (which < -2 || which >= h->L) fail(HOMLN_EINVAL, "which must be -2, -1 or a layer id");
    use_device(h);
    GraphState &g = which >= 0 ? *h->layers[which] : which == -1 ? and_graph(h, layer_mask) : or_graph(h, layer_mask);
    analyse(h, g);
    Selection &S = selection_of(h, g, *sel);
    const int32_t c = S.count;
    if (nodes_out && put_out(h, nodes_out, S.ranked.p, sizeof(int32_t) * c)) HCUDA(cudaStreamSynchronize(h->stream));
    check_device_error(h);
    *count_out = c;
    API_END
}

homln_status homln_compose(homln_t h, uint64_t layer_mask, int32_t heuristic, const homln_select *sel,
                           int32_t *nodes_out, int32_t *count_out) {
    API_BEGIN
    if (!h) fail(HOMLN_EINVAL, "null handle");
    check_select(sel);
    if (!count_out) fail(HOMLN_EINVAL, "count_out is NULL");
    if (heuristic < HOMLN_NAIVE || heuristic > HOMLN_CC2) fail(HOMLN_EINVAL, "unknown heuristic");
    use_device(h);
    std::vector<int> ids = mask_layers(h, layer_mask);
    for (int i : ids) analyse(h, *h->layers[i]);
    const int32_t n = h->n;
    const int32_t nw = (int32_t)ceil_div(n, 32);
    DevOut<int32_t> o;
    o.to(h, nodes_out, n);
    int32_t c = 0;
    if (heuristic == HOMLN_CC2) {
        std::vector<const uint64_t *> sd;
        for (int i : ids) sd.push_back(h->layers[i]->sumdist.p);
        DBuf<double> scores;
        DBuf<int32_t> ranked;
        DBuf<uint32_t> bits;
        if (!scores.alloc(&h->al, n) || !ranked.alloc(&h->al, n) || !bits.alloc(&h->al, nw))
            fail(HOMLN_ENOMEM, "cc2 scratch");
        cc2_scores(n, sd, scores.p, &h->al, h->stream);
        select_nodes(n, scores.p, *sel, ranked.p, bits.p, h->err.p, &h->al, h->stream);
        c = bits_to_sorted_ids(n, bits.p, o.p, &h->al, h->stream);
    } else {
        // CC-node sets of the layers (cached per selection rule), intersected (naive), then CC1's refinement
        DBuf<uint32_t> common;
        if (!common.alloc(&h->al, nw)) fail(HOMLN_ENOMEM, "compose scratch");
        std::vector<GraphState *> lg;
        for (int i : ids) lg.push_back(h->layers[i].get());
        selections_of(h, lg, *sel);
        for (size_t k = 0; k < ids.size(); ++k) {
            Selection &S = selection_of(h, *h->layers[ids[k]], *sel);
            if (k == 0)
                HCUDA(cudaMemcpyAsync(common.p, S.bits.p, sizeof(uint32_t) * nw, cudaMemcpyDeviceToDevice, h->stream));
            else
                bits_and(nw, common.p, S.bits.p, h->stream);
        }
        if (heuristic == HOMLN_NAIVE) {
            c = bits_to_sorted_ids(n, common.p, o.p, &h->al, h->stream);
        } else {
            std::vector<const Csr *> csrs;
            std::vector<const uint64_t *> sd;
            std::vector<const int32_t *> dg;
            for (int i : ids) {
                csrs.push_back(&in_csr(h, *h->layers[i]));
                sd.push_back(h->layers[i]->sumdist.p);
                dg.push_back(h->layers[i]->deg.p);
            }
            c = cc1_compose(n, csrs, sd, dg, common.p, sel->cc1_overlap, o.p, h->err.p, &h->al, h->stream);
        }
    }
    o.finish(h, c);
    check_device_error(h);
    *count_out = c;
    API_END
}

homln_status homln_subset_sweep(homln_t h, int32_t heuristic, const homln_select *sel, int32_t min_layers,
                                homln_subset_result *out, int32_t capacity, int32_t *count_out) {
    API_BEGIN
    if (!h) fail(HOMLN_EINVAL, "null handle");
    check_select(sel);
    if (!count_out) fail(HOMLN_EINVAL, "count_out is NULL");
    if (heuristic < HOMLN_NAIVE || heuristic > HOMLN_CC2) fail(HOMLN_EINVAL, "unknown heuristic");
    if (h->L > 20) fail(HOMLN_EINVAL, "a sweep covers at most 20 layers (2^20 subsets)");
    use_device(h);
    std::vector<uint64_t> masks;
    for (uint64_t m = 1; m < (1ull << h->L); ++m)
        if (__builtin_popcountll(m) >= std::max(1, min_layers)) masks.push_back(m);
    *count_out = (int32_t)masks.size();
    if (!out) { set_error(""); return HOMLN_OK; }
    if (capacity < (int32_t)masks.size()) fail(HOMLN_ERANGE, "capacity smaller than the number of subsets");
    // Psi once: every layer and every subset's AND graph, one launch
    std::vector<GraphState *> gs;
    for (auto &g : h->layers) gs.push_back(g.get());
    for (uint64_t m : masks) gs.push_back(&and_graph(h, m));
    analyse_many(h, gs);
    const int32_t n = h->n;
    DBuf<int32_t> est;
    if (!est.alloc(&h->al, n)) fail(HOMLN_ENOMEM, "sweep scratch");
    for (size_t i = 0; i < masks.size(); ++i) {
        Selection &T = selection_of(h, and_graph(h, masks[i]), *sel);
        int32_t c = 0;
        homln_status st = homln_compose(h, masks[i], heuristic, sel, est.p, &c);
        if (st != HOMLN_OK) fail(st, homln_last_error());
        homln_accuracy_t acc;
        accuracy_counts(n, est.p, c, T.ranked.p, T.count, &acc, h->err.p, &h->al, h->stream);
        out[i].mask = masks[i];
        out[i].truth_count = T.count;
        out[i].estimate_count = c;
        out[i].acc = acc;
    }
    check_device_error(h);
    API_END
}

homln_status homln_accuracy(homln_t h, const int32_t *pred, int32_t n_pred, const int32_t *truth, int32_t n_truth,
                            homln_accuracy_t *out) {
    API_BEGIN
    if (!h) fail(HOMLN_EINVAL, "null handle");
    if (!out) fail(HOMLN_EINVAL, "out is NULL");
    if (n_pred < 0 || n_truth < 0) fail(HOMLN_EINVAL, "negative list length");
    if ((n_pred > 0 && !pred) || (n_truth > 0 && !truth)) fail(HOMLN_EINVAL, "list is NULL");
    use_device(h);
    DevIn<int32_t> p, t;
    p.from(h, pred, n_pred);
    t.from(h, truth, n_truth);
    homln_accuracy_t r;
    accuracy_counts(h->n, p.p, n_pred, t.p, n_truth, &r, h->err.p, &h->al, h->stream);
    check_device_error(h);
    *out = r;
    API_END
}

homln_status homln_invalidate(homln_t h) {
    API_BEGIN
    if (!h) fail(HOMLN_EINVAL, "null handle");
    use_device(h);
    drop_results(h);
    API_END
}

homln_status homln_sync(homln_t h) {
    API_BEGIN
    if (!h) fail(HOMLN_EINVAL, "null handle");
    use_device(h);
    HCUDA(cudaStreamSynchronize(h->stream));
    check_device_error(h);
    API_END
}

homln_status homln_set_profiling(homln_t h, int32_t timing, int32_t instrument) {
    API_BEGIN
    if (!h) fail(HOMLN_EINVAL, "null handle");
    h->profiling = timing != 0;
    h->instrument = instrument != 0;
    API_END
}

homln_status homln_get_profile(homln_t h, homln_profile_t *out) {
    API_BEGIN
    if (!h || !out) fail(HOMLN_EINVAL, "null argument");
    use_device(h);
    HCUDA(cudaStreamSynchronize(h->stream));
    double ms = 0.0;
    for (auto &e : h->events) {
        float t = 0.f;
        HCUDA(cudaEventElapsedTime(&t, e.first, e.second));
        ms += t;
    }
    out->bfs_launches = h->bfs_launches;
    out->bfs_timed_launches = (int64_t)h->events.size();
    out->bfs_ms = ms;
    out->levels = (int64_t)h->stats.levels;
    out->pull_levels = (int64_t)h->stats.pull_levels;
    out->push_levels = (int64_t)h->stats.push_levels;
    out->batches = (int64_t)h->stats.batches;
    out->edges_scanned = (int64_t)h->stats.group_edges;
    out->words_gathered = (int64_t)h->stats.lane_words;
    out->edges_pushed = (int64_t)h->stats.push_edges;
    out->words_pushed = (int64_t)h->stats.push_words;
    out->bytes = (int64_t)h->stats.bytes;
    out->visits = (int64_t)h->stats.visits;
    out->words_per_node = h->stats.words_per_node;
    out->teams = h->stats.teams;
    API_END
}

homln_status homln_reset_profile(homln_t h) {
    API_BEGIN
    if (!h) fail(HOMLN_EINVAL, "null handle");
    for (auto &e : h->events) {
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
    }
    h->events.clear();
    h->bfs_launches = 0;
    h->stats = BfsStats{};
    API_END
}

int64_t homln_kernel_launches(void) { return (int64_t)g_kernel_launches.load(); }

}  // extern "C"
