// Shared device helpers and host-side plumbing of the homln library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/homln.h"

namespace homln {

// ---------------------------------------------------------------------------
// Device-side error word. Kernels never trap: they record a code and return.
// ---------------------------------------------------------------------------
enum DevErr : int32_t {
    DEV_OK = 0,
    DEV_BAD_ID = 1,       // an edge endpoint outside [0, n)
    DEV_TIMEOUT = 2,      // a bounded grid barrier gave up
    DEV_RANGE = 3,        // an exact fixed-point value left its range
};

__device__ __forceinline__ void dev_fail(int32_t *err, int32_t code) {
    if (err) atomicCAS(err, 0, code);
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(uint32_t *p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid barrier state: arrival counter, generation and the error word.
struct GridBarrier {
    uint32_t *count;
    uint32_t *gen;
    int32_t *err;
};

// Bounded grid-wide barrier for a cooperative launch (all blocks co-resident).
// Every block's thread 0 arrives once; the last arrival bumps the generation.
// A waiter gives up after `limit_ns` of wall time, records DEV_TIMEOUT and the
// caller returns. Returns false when the kernel must stop (timeout or error).
__device__ __forceinline__ bool grid_sync(const GridBarrier &b, uint64_t limit_ns = 2000000000ull) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        uint32_t g = ld_acquire_u32(b.gen);
        __threadfence();
        uint32_t arrived = atomicAdd(b.count, 1u);
        if (arrived == gridDim.x - 1) {
            *b.count = 0;
            __threadfence();
            st_release_u32(b.gen, g + 1);
        } else {
            uint64_t t0 = globaltimer_ns();
            uint32_t spins = 0;
            while (ld_acquire_u32(b.gen) == g) {
                if ((++spins & 255u) == 0) {
                    if (globaltimer_ns() - t0 > limit_ns) {
                        dev_fail(b.err, DEV_TIMEOUT);
                        ok = 0;
                        break;
                    }
                    if (*(volatile int32_t *)b.err != 0) {
                        ok = 0;
                        break;
                    }
                }
            }
        }
        __threadfence();
        if (*(volatile int32_t *)b.err != 0) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Which lanes' candidates v (ascending over the valid lanes [0, nv), distinct) occur in the
// sorted row col[lo, hi) of distinct entries: the warp walks the row 32 entries at a time from
// `lo`, one entry per lane, skips chunks below the candidates, stops at the first chunk above
// them, and each lane looks its candidate up in a chunk by a binary search over the lanes
// (shuffles). `lo` moves past the chunks that no later (larger) candidate can match, so a row
// is walked once across ascending candidate chunks. Every lane of the warp must call it.
__device__ __forceinline__ bool warp_row_has(const int32_t *__restrict__ col, int64_t &lo, int64_t hi, int32_t v,
                                             int nv, int lane) {
    const int32_t vmin = __shfl_sync(0xffffffffu, v, 0), vmax = __shfl_sync(0xffffffffu, v, nv - 1);
    bool hit = false;
    for (int64_t c = lo; c < hi; c += 32) {
        const int64_t j = c + lane;
        const int32_t w = j < hi ? __ldg(col + j) : INT32_MAX;
        const int last = (int)(hi - 1 - c < 31 ? hi - 1 - c : 31);
        const int32_t wmin = __shfl_sync(0xffffffffu, w, 0), wmax = __shfl_sync(0xffffffffu, w, last);
        if (wmax < vmin) {
            lo = c + 32;
            continue;
        }
        if (wmin > vmax) break;
        int a = 0, b = last;  // first entry >= v among lanes [0, last]
#pragma unroll
        for (int step = 0; step < 5; ++step) {
            const int mid = (a + b) >> 1;
            const int32_t wm = __shfl_sync(0xffffffffu, w, mid);
            if (a < b) {
                if (wm < v) a = mid + 1;
                else b = mid;
            }
        }
        hit |= __shfl_sync(0xffffffffu, w, a) == v;
        if (wmax > vmax) break;  // the chunk reaches past the candidates: later ones start here
        lo = c + 32;
    }
    return hit && lane < nv;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
void set_error(const std::string &msg);

struct Ctx;  // per-handle allocation context

// Device memory through the handle's allocator (stream ordered).
struct Alloc {
    homln_allocator a;
    cudaStream_t stream;
    void *get(size_t bytes);
    void put(void *p, size_t bytes);
};

// A device buffer that frees itself through the allocator.
template <typename T>
struct DBuf {
    Alloc *al = nullptr;
    T *p = nullptr;
    size_t n = 0;
    DBuf() = default;
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    DBuf(DBuf &&o) noexcept { *this = std::move(o); }
    DBuf &operator=(DBuf &&o) noexcept {
        if (this != &o) {
            release();
            al = o.al; p = o.p; n = o.n;
            o.p = nullptr; o.n = 0;
        }
        return *this;
    }
    ~DBuf() { release(); }
    bool alloc(Alloc *a, size_t count) {
        release();
        al = a;
        n = count;
        if (count == 0) return true;
        p = static_cast<T *>(a->get(count * sizeof(T)));
        if (!p) n = 0;
        return p != nullptr;
    }
    void release() {
        if (p && al) al->put(p, n * sizeof(T));
        p = nullptr;
        n = 0;
    }
};

// Thrown inside the library, caught at the C-ABI boundary.
struct Error {
    homln_status code;
    std::string msg;
};

[[noreturn]] void fail(homln_status code, const std::string &msg);
void check_cuda(cudaError_t e, const char *what);
#define HCUDA(x) ::homln::check_cuda((x), #x)

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Every kernel launch of the library goes through launch() so it can be counted.
extern std::atomic<long long> g_kernel_launches;
template <typename... KArgs, typename... Args>
inline void launch(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args) {
    g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
    kern<<<grid, block, smem, s>>>(args...);
}

// ---------------------------------------------------------------------------
// Primitives (prims.cu)
// ---------------------------------------------------------------------------
// out[i] = sum_{j<i} in[j] (int64), total written to out[n]. `out` has n+1 entries.
void scan_exclusive_i32(const int32_t *in, int64_t *out, int64_t n, Alloc *al, cudaStream_t s);
void scan_exclusive_i64(const int64_t *in, int64_t *out, int64_t n, Alloc *al, cudaStream_t s);
// Stable LSD radix sort of 64-bit keys on bits [bit0, bit1), optional uint32 payload.
// Result in keys/vals (the alternate buffers are scratch).
void radix_sort_u64(uint64_t *keys, uint32_t *vals, int64_t n, int bit0, int bit1, Alloc *al, cudaStream_t s);
// Sort every CSR row's entries ascending, in place (segmented sort).
// cap: entries allocated in d_col (an upper bound on the longest row).
void sort_rows(int32_t n, const int64_t *d_rowptr, int32_t *d_col, int64_t cap, Alloc *al, cudaStream_t s);

// ---------------------------------------------------------------------------
// Graph building (graph.cu)
// ---------------------------------------------------------------------------
// Rows are built without a host round trip: col is allocated with an upper bound (cap) on
// the entries, and the exact count lives in rowptr[n] on the device until a caller needs it
// on the host (csr_nnz, which synchronises once and caches it).
struct Csr {
    int32_t n = 0;
    int64_t cap = 0;           // entries allocated in col (>= the entries present)
    mutable int64_t nnz = -1;  // entries present (2 x undirected edges); -1 until read
    DBuf<int64_t> rowptr;
    DBuf<int32_t> col;
};
int64_t csr_nnz(const Csr &g, cudaStream_t s);

// Normalise an edge list (device int32 arrays) into a symmetric CSR with sorted rows.
// directed: each edge goes into its source's row only (no symmetrisation).
void build_csr(int32_t n, const int32_t *d_src, const int32_t *d_dst, int64_t m, Csr &out, int32_t *d_err,
               Alloc *al, cudaStream_t s, bool directed = false);
// Edges present in every CSR of `layers` (sorted-row intersection).
void and_intersect(int32_t n, const std::vector<const Csr *> &layers, Csr &out, Alloc *al, cudaStream_t s);
// Edges present in at least one CSR of `layers` (Boolean OR aggregation).
void or_union(int32_t n, const std::vector<const Csr *> &layers, Csr &out, Alloc *al, cudaStream_t s);
// Edge list ascending (u, v) of a CSR: pairs u < v (nnz/2 of them) of an undirected graph, or
// every entry of a directed one.
void csr_edge_list(const Csr &g, int32_t *d_src, int32_t *d_dst, Alloc *al, cudaStream_t s, bool directed = false);
// Relabelling for the BFS: degree descending (degrees of g), then id ascending, except that
// the vertices of small connected components (at most 8 vertices; weakly connected through g
// and `other` when g is one direction of a directed graph) come last. perm[new] = old,
// inv[old] = new; builds the relabelled CSR, and split[0] (on the device) = the number of
// vertices before the small components: vertices 0 .. split[0]-1 form whole components.
void relabel_by_degree(const Csr &g, const Csr *other, Csr &out, DBuf<int32_t> &perm, DBuf<int32_t> &inv,
                       DBuf<int32_t> &split, Alloc *al, cudaStream_t s);
// The same relabelling applied to another CSR over the same vertices.
void relabel_apply(const Csr &g, const int32_t *perm, const int32_t *inv, Csr &out, Alloc *al, cudaStream_t s);

// ---------------------------------------------------------------------------
// Multi-source BFS (msbfs.cu)
// ---------------------------------------------------------------------------
struct BfsTuning {
    int W = 0;           // words per node (0 = auto)
    int teams = 0;       // teams of blocks sharing the grid (0 = auto)
    int team_mix = 0;    // 1: blocks sharing an SM join different teams
    int schedule = 0;    // 0: persistent tile queue; 1: plain, one launch per phase, host-driven levels
    int push_alpha = 16;
    int threads = 512;
    int blocks_per_sm = 0;
    int relabel = 1;
    int wait_limit_ms = 2000;  // device-side waits give up after this long (HOMLN_ETIMEOUT)
    int phantom = 0;           // tests: team barriers also wait for blocks that do not exist
    int max_tiles = 0;         // persistent launches take at most this many tiles each (0 = all)
    int sm_count = 0;          // persistent launches size their grid for this many SMs (0 = all)
    // preemption (homln_set_yield): while *yield_host != 0 the persistent BFS hands out no more
    // tiles (its kernel reads the flag through yield_dev) and stops after the tiles it runs; the
    // host resumes the remaining tiles once the flag is 0 again and counts the stop in yield_count
    const volatile int32_t *yield_host = nullptr;
    const int32_t *yield_dev = nullptr;
    std::atomic<long long> *yield_count = nullptr;
    int shard_rank = 0;        // only source batches shard_rank, shard_rank + shard_world, ...
    int shard_world = 1;       //   (partial F/R of a sharded analysis; 0 / 1 = all sources)
};

struct BfsStats {  // filled by an instrumented run
    uint64_t levels = 0, pull_levels = 0, push_levels = 0;
    uint64_t group_edges = 0;  // edges scanned by pull (per vertex, max over its lanes)
    uint64_t lane_words = 0;   // 8-byte frontier words gathered by pull
    uint64_t push_edges = 0;   // edges pushed
    uint64_t batches = 0;
    uint64_t push_words = 0;   // 8-byte atomic ORs issued by top-down levels
    uint64_t bytes = 0;        // bytes requested by the kernel's loads/stores (broadcast loads once)
    uint64_t visits = 0;       // vertex visits (non-quiet vertices processed per level)
    int words_per_node = 0;    // W of the last launch
    int teams = 0;             // teams of the last launch
};

// The graph the BFS traverses: the CSR itself, or its relabelling (perm[new] = old), in which
// vertices 0 .. split[0]-1 form whole (weakly) connected components and the small components
// follow.
// A directed graph also carries its in-edge CSR (csr_in), which the bottom-up levels read.
struct BfsGraph {
    Csr csr;
    Csr csr_in;
    DBuf<int32_t> perm;
    DBuf<int32_t> split;  // relabelled graphs: [0] = vertices before the small components
    bool relabeled = false;
    bool directed = false;
};
// g_in: the in-edge CSR of a directed graph (nullptr when undirected).
void bfs_prepare(const Csr &g, const Csr *g_in, bool relabel, BfsGraph &out, Alloc *al, cudaStream_t s);

// A BFS over a job list with everything allocated once (msbfs.cu): bfs_plan_run enqueues one
// complete analysis without allocating or copying from the host (capturable in a CUDA graph,
// except the plain schedule and instrumented plans).
struct BfsPlan;
struct BfsJob;
BfsPlan *bfs_plan_create(const std::vector<BfsJob> &jobs, const BfsTuning &t, int32_t *d_err, Alloc *al,
                         cudaStream_t s, bool stats);
void bfs_plan_run(BfsPlan *p, cudaStream_t s, cudaEvent_t ev_start, cudaEvent_t ev_stop);
void bfs_plan_stats(BfsPlan *p, BfsStats *stats, cudaStream_t s);
bool bfs_plan_capturable(const BfsPlan *p);
void bfs_plan_destroy(BfsPlan *p);

struct BfsJob {
    const BfsGraph *g;
    uint64_t *F;  // outputs in the original vertex order
    uint32_t *R;
};

// All-sources BFS of several graphs in one persistent launch (tiles = graph x source batch).
void msbfs_multi(const std::vector<BfsJob> &jobs, const BfsTuning &t, int32_t *d_err, Alloc *al, cudaStream_t s,
                 BfsStats *stats, cudaEvent_t ev_start, cudaEvent_t ev_stop);

int msbfs_pick_words(int32_t n);

// ---------------------------------------------------------------------------
// Finalize / selection / composition / accuracy (select.cu)
// ---------------------------------------------------------------------------
void closeness_finalize(int32_t n, const int64_t *rowptr, const uint64_t *F, const uint32_t *R, double *cc,
                        uint64_t *sumdist, int32_t *deg, cudaStream_t s);
// Device error DEV_RANGE unless every (F, R) pair can come from a BFS on n vertices.
void partials_check(int32_t n, const uint64_t *F, const uint32_t *R, int32_t *d_err, cudaStream_t s);
// Selected ids in rank order into d_out (capacity n); count to host.
int32_t select_nodes(int32_t n, const double *d_scores, const homln_select &sel, int32_t *d_out,
                     uint32_t *d_member_bits, int32_t *d_err, Alloc *al, cudaStream_t s);
void cc2_scores(int32_t n, const std::vector<const uint64_t *> &sumdists, double *d_scores, Alloc *al,
                cudaStream_t s);
int32_t cc1_compose(int32_t n, const std::vector<const Csr *> &csrs, const std::vector<const uint64_t *> &sumdist,
                    const std::vector<const int32_t *> &deg, const uint32_t *d_common_bits, double theta,
                    int32_t *d_out, int32_t *d_err, Alloc *al, cudaStream_t s);
int32_t bits_to_sorted_ids(int32_t n, const uint32_t *d_bits, int32_t *d_out, Alloc *al, cudaStream_t s);
void bits_and(int32_t nwords, uint32_t *d_acc, const uint32_t *d_other, cudaStream_t s);
void accuracy_counts(int32_t n, const int32_t *d_pred, int32_t n_pred, const int32_t *d_truth, int32_t n_truth,
                     homln_accuracy_t *h_out, int32_t *d_err, Alloc *al, cudaStream_t s);
void accuracy_counts_prealloc(int32_t n, const int32_t *d_pred, int32_t n_pred, const int32_t *d_truth,
                              int32_t n_truth, uint32_t *bits_p, uint32_t *bits_t, unsigned long long *c3, double *r4,
                              int32_t *err, homln_accuracy_t *h_out, int32_t *h_err, cudaStream_t s);

}  // namespace homln
