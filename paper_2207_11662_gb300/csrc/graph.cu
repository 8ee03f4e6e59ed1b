// Device graph store: CSR construction, Boolean AND aggregation, edge-list
// export and degree-descending relabelling.
//
// Section 4 treats every layer as a simple undirected graph (NetworkX Graph):
// self loops and repeated edges vanish, each edge is reachable from both ends.
// Section 3.1 / Section 4 define the AND aggregate: an edge survives iff it is
// in every selected layer.
#include "common.cuh"

#include <algorithm>

namespace homln {

namespace {

constexpr int NODE_BITS = 20;  // HOMLN_MAX_NODES = 2^20
constexpr uint64_t NODE_MASK = (1ull << NODE_BITS) - 1;

// Degree of each endpoint of every valid, non-loop edge (both directions; only the source's
// row when the graph is directed).
template <bool SYM>
__global__ void k_count_deg(const int32_t *__restrict__ src, const int32_t *__restrict__ dst, int64_t m, int32_t n,
                            int32_t *__restrict__ deg, int32_t *err) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = src[e], b = dst[e];
        if (a < 0 || a >= n || b < 0 || b >= n) {
            dev_fail(err, DEV_BAD_ID);
            continue;
        }
        if (a == b) continue;
        atomicAdd(&deg[a], 1);
        if (SYM) atomicAdd(&deg[b], 1);
    }
}

// Each edge lands in both endpoints' rows, or only in the source's row when directed
// (row order is fixed later by the row sort).
template <bool SYM>
__global__ void k_scatter_edges(const int32_t *__restrict__ src, const int32_t *__restrict__ dst, int64_t m, int32_t n,
                                unsigned long long *__restrict__ cursor, int32_t *__restrict__ col) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = src[e], b = dst[e];
        if (a < 0 || a >= n || b < 0 || b >= n || a == b) continue;
        col[atomicAdd(&cursor[a], 1ull)] = b;
        if (SYM) col[atomicAdd(&cursor[b], 1ull)] = a;
    }
}

// Warp per row of a row-sorted CSR: count (or write) the entries that differ from their predecessor.
template <bool WRITE>
__global__ void k_row_unique(int32_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                             int32_t *__restrict__ cnt, const int64_t *__restrict__ orp, int32_t *__restrict__ ocol) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = warp; r < n; r += nwarps) {
        const int64_t b = rp[r], e = rp[r + 1];
        const int64_t o = WRITE ? orp[r] : 0;
        int32_t c = 0;
        for (int64_t j0 = b; j0 < e; j0 += 32) {
            const int64_t j = j0 + lane;
            bool keep = false;
            int32_t v = 0;
            if (j < e) {
                v = col[j];
                keep = (j == b) || col[j - 1] != v;
            }
            const uint32_t mk = __ballot_sync(0xffffffffu, keep);
            if (WRITE && keep) ocol[o + c + __popc(mk & ((1u << lane) - 1u))] = v;
            c += __popc(mk);
        }
        if (!WRITE && lane == 0) cnt[r] = c;
    }
}

// Relabelled rows, unsorted: row i of the new graph holds inv[] of old row perm[i].
__global__ void k_relabel_rows(int32_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                               const int32_t *__restrict__ perm, const int32_t *__restrict__ inv,
                               const int64_t *__restrict__ nrp, int32_t *__restrict__ ncol) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < n; i += nwarps) {
        const int32_t old = perm[i];
        const int64_t a = rp[old], len = rp[old + 1] - a, o = nrp[i];
        for (int64_t j = lane; j < len; j += 32) ncol[o + j] = inv[col[a + j]];
    }
}

struct LayerSet {
    const int64_t *rp[HOMLN_MAX_LAYERS];
    const int32_t *col[HOMLN_MAX_LAYERS];
    int r;
};

// One warp per vertex: the lanes take the shortest of its rows 32 entries at a time and keep
// the entries present in every other row; a ballot keeps them in order.
template <bool WRITE>
__global__ void k_and_rows(int32_t n, LayerSet L, int32_t *__restrict__ cnt, const int64_t *__restrict__ out_rp,
                           int32_t *__restrict__ out_col) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = warp; u < n; u += nwarps) {
        int best = 0;
        int64_t best_len = L.rp[0][u + 1] - L.rp[0][u];
        for (int i = 1; i < L.r; ++i) {
            int64_t len = L.rp[i][u + 1] - L.rp[i][u];
            if (len < best_len) { best_len = len; best = i; }
        }
        const int64_t b0 = L.rp[best][u];
        const int64_t o = WRITE ? out_rp[u] : 0;
        int64_t cur[HOMLN_MAX_LAYERS];  // per other layer: where its row walk resumes
        for (int i = 0; i < L.r; ++i) cur[i] = L.rp[i][u];
        int32_t c = 0;
        for (int64_t j0 = 0; j0 < best_len; j0 += 32) {
            const int64_t j = j0 + lane;
            const int nv = (int)(best_len - j0 < 32 ? best_len - j0 : 32);
            const int32_t v = j < best_len ? __ldg(L.col[best] + b0 + j) : -1;
            bool all = lane < nv;
            for (int i = 0; i < L.r; ++i) {
                if (i == best) continue;
                if (!__any_sync(0xffffffffu, all)) break;
                // every lane takes part in the shuffles, so no short-circuit around the call
                const bool has = warp_row_has(L.col[i], cur[i], L.rp[i][u + 1], v, nv, lane);
                all = all && has;
            }
            const uint32_t m = __ballot_sync(0xffffffffu, all);
            if (WRITE && all) out_col[o + c + __popc(m & ((1u << lane) - 1u))] = v;
            c += __popc(m);
        }
        if (!WRITE && lane == 0) cnt[u] = c;
    }
}

// Row u of the concatenation: every selected layer's row u, one after the other.
__global__ void k_sum_degrees(int32_t n, LayerSet L, int32_t *__restrict__ deg) {
    for (int32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        int64_t d = 0;
        for (int i = 0; i < L.r; ++i) d += L.rp[i][u + 1] - L.rp[i][u];
        deg[u] = (int32_t)d;
    }
}

__global__ void k_concat_rows(int32_t n, LayerSet L, const int64_t *__restrict__ orp, int32_t *__restrict__ ocol) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = warp; u < n; u += nwarps) {
        int64_t o = orp[u];
        for (int i = 0; i < L.r; ++i) {
            const int64_t b = L.rp[i][u], len = L.rp[i][u + 1] - b;
            for (int64_t j = lane; j < len; j += 32) ocol[o + j] = L.col[i][b + j];
            o += len;
        }
    }
}

// Length of the part of row u holding neighbours v > u (rows are sorted); the whole row when
// every entry is an edge of its own (directed graphs).
__global__ void k_upper_len(int32_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                            int32_t *__restrict__ len, int64_t *__restrict__ start, int directed) {
    for (int32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        int64_t lo = rp[u], hi = rp[u + 1];
        int64_t a = lo, b = hi;
        while (!directed && a < b) {
            int64_t mid = (a + b) >> 1;
            if (col[mid] <= u) a = mid + 1; else b = mid;
        }
        start[u] = a;
        len[u] = (int32_t)(hi - a);
    }
}

__global__ void k_write_pairs(int32_t n, const int32_t *__restrict__ col, const int64_t *__restrict__ start,
                              const int32_t *__restrict__ len, const int64_t *__restrict__ off, int32_t *__restrict__ s,
                              int32_t *__restrict__ d) {
    for (int32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        int64_t o = off[u], a = start[u];
        for (int32_t j = 0; j < len[u]; ++j) {
            s[o + j] = u;
            d[o + j] = col[a + j];
        }
    }
}

// Sort keys for the BFS order: vertices of small components (at most kSmallComponent vertices)
// last, otherwise degree descending, then id ascending. A thread explores v's component
// breadth-first, along the rows of `a` and (directed: weak components) of `b`, and stops as
// soon as it holds more than kSmallComponent vertices or meets a row that long. The blocks add
// up their small-component vertices; the last block to finish writes split[0] = n - their
// count, the number of vertices placed before them.
constexpr int kSmallComponent = 8;

__device__ __forceinline__ bool small_component(int32_t v, int32_t n, const int64_t *__restrict__ ra,
                                                const int32_t *__restrict__ ca, const int64_t *__restrict__ rb,
                                                const int32_t *__restrict__ cb) {
    constexpr int S = kSmallComponent;
    int32_t vis[S];
#pragma unroll
    for (int k = 0; k < S; ++k) vis[k] = -1;
    vis[0] = v;
    int cnt = 1;
#pragma unroll
    for (int i = 0; i < S; ++i) {
        if (i >= cnt) break;
        int32_t x = -1;
#pragma unroll
        for (int k = 0; k < S; ++k)
            if (k == i) x = vis[k];
        for (int side = 0; side < (rb ? 2 : 1); ++side) {
            const int64_t *rp = side ? rb : ra;
            const int32_t *col = side ? cb : ca;
            const int64_t e0 = rp[x], e1 = rp[x + 1];
            if (e1 - e0 >= S) return false;
            for (int64_t j = e0; j < e1; ++j) {
                const int32_t u = col[j];
                if (u < 0 || u >= n) continue;
                bool seen = false;
#pragma unroll
                for (int k = 0; k < S; ++k) seen |= vis[k] == u;
                if (seen) continue;
                if (cnt == S) return false;
#pragma unroll
                for (int k = 0; k < S; ++k)
                    if (k == cnt) vis[k] = u;
                ++cnt;
            }
        }
    }
    return true;
}

__global__ void k_degree_keys(int32_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                              const int64_t *__restrict__ rp2, const int32_t *__restrict__ col2,
                              unsigned int *__restrict__ ctr, int32_t *__restrict__ split,
                              uint64_t *__restrict__ keys) {
    __shared__ unsigned int block_small;
    if (threadIdx.x == 0) block_small = 0;
    __syncthreads();
    unsigned int mine = 0;
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const uint64_t deg = (uint64_t)(rp[v + 1] - rp[v]);
        const uint64_t small = small_component(v, n, rp, col, rp2, col2) ? 1 : 0;
        mine += (unsigned int)small;
        keys[v] = (small << (2 * NODE_BITS)) | ((NODE_MASK - deg) << NODE_BITS) | (uint64_t)v;
    }
    if (mine) atomicAdd(&block_small, mine);
    __syncthreads();
    if (threadIdx.x != 0) return;
    if (block_small) atomicAdd(ctr, block_small);
    __threadfence();
    if (atomicAdd(ctr + 1, 1u) != gridDim.x - 1) return;
    __threadfence();
    *split = n - (int32_t)atomicAdd(ctr, 0u);
}

__global__ void k_perm_from_keys(int32_t n, const uint64_t *__restrict__ keys, int32_t *__restrict__ perm,
                                 int32_t *__restrict__ inv) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int32_t old = (int32_t)(keys[i] & NODE_MASK);
        perm[i] = old;
        inv[old] = i;
    }
}

__global__ void k_perm_degrees(int32_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ perm,
                               int32_t *__restrict__ newdeg) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int32_t old = perm[i];
        newdeg[i] = (int32_t)(rp[old + 1] - rp[old]);
    }
}

unsigned grid_for(int64_t work, int threads = 256) {
    int64_t b = ceil_div(work > 0 ? work : 1, threads);
    return (unsigned)(b > 65535 * 16 ? 65535 * 16 : b);
}

int64_t read_i64_sync(const int64_t *d, cudaStream_t s) {
    int64_t v = 0;
    HCUDA(cudaMemcpyAsync(&v, d, sizeof(v), cudaMemcpyDeviceToHost, s));
    HCUDA(cudaStreamSynchronize(s));
    return v;
}

}  // namespace

void build_csr(int32_t n, const int32_t *d_src, const int32_t *d_dst, int64_t m, Csr &out, int32_t *d_err, Alloc *al,
               cudaStream_t s, bool directed) {
    // degrees -> row offsets -> scatter both directions of every edge -> sort each row ->
    // drop repeated entries (self loops were dropped at the scatter)
    out.n = n;
    if (!out.rowptr.alloc(al, (size_t)n + 1)) fail(HOMLN_ENOMEM, "csr rowptr");
    if (m == 0) {
        HCUDA(cudaMemsetAsync(out.rowptr.p, 0, sizeof(int64_t) * (n + 1), s));
        out.nnz = 0;
        out.cap = 0;
        out.col.release();
        return;
    }
    const int64_t raw_cap = (directed ? 1 : 2) * m;
    DBuf<int32_t> deg, raw, cnt;
    DBuf<int64_t> rp;
    DBuf<unsigned long long> cursor;
    if (!deg.alloc(al, n) || !rp.alloc(al, (size_t)n + 1) || !cursor.alloc(al, n) || !raw.alloc(al, raw_cap) ||
        !cnt.alloc(al, n))
        fail(HOMLN_ENOMEM, "csr scratch");
    HCUDA(cudaMemsetAsync(deg.p, 0, sizeof(int32_t) * n, s));
    if (directed) launch(k_count_deg<false>, grid_for(m), 256, 0, s, d_src, d_dst, m, n, deg.p, d_err);
    else launch(k_count_deg<true>, grid_for(m), 256, 0, s, d_src, d_dst, m, n, deg.p, d_err);
    scan_exclusive_i32(deg.p, rp.p, n, al, s);
    HCUDA(cudaMemcpyAsync(cursor.p, rp.p, sizeof(int64_t) * n, cudaMemcpyDeviceToDevice, s));
    if (directed) launch(k_scatter_edges<false>, grid_for(m), 256, 0, s, d_src, d_dst, m, n, cursor.p, raw.p);
    else launch(k_scatter_edges<true>, grid_for(m), 256, 0, s, d_src, d_dst, m, n, cursor.p, raw.p);
    sort_rows(n, rp.p, raw.p, raw_cap, al, s);
    launch(k_row_unique<false>, grid_for((int64_t)n * 32), 256, 0, s, n, (const int64_t *)rp.p,
           (const int32_t *)raw.p, cnt.p, (const int64_t *)nullptr, (int32_t *)nullptr);
    scan_exclusive_i32(cnt.p, out.rowptr.p, n, al, s);
    out.cap = raw_cap;
    out.nnz = -1;
    if (!out.col.alloc(al, out.cap)) fail(HOMLN_ENOMEM, "csr col");
    launch(k_row_unique<true>, grid_for((int64_t)n * 32), 256, 0, s, n, (const int64_t *)rp.p,
           (const int32_t *)raw.p, (int32_t *)nullptr, (const int64_t *)out.rowptr.p, out.col.p);
    HCUDA(cudaGetLastError());
}

int64_t csr_nnz(const Csr &g, cudaStream_t s) {
    if (g.nnz < 0) g.nnz = g.cap > 0 ? read_i64_sync(g.rowptr.p + g.n, s) : 0;
    return g.nnz;
}

void and_intersect(int32_t n, const std::vector<const Csr *> &layers, Csr &out, Alloc *al, cudaStream_t s) {
    LayerSet L{};
    L.r = (int)layers.size();
    for (int i = 0; i < L.r; ++i) {
        L.rp[i] = layers[i]->rowptr.p;
        L.col[i] = layers[i]->col.p;
    }
    out.n = n;
    out.cap = layers[0]->cap;  // the intersection is no larger than any of its rows' layers
    for (const Csr *c : layers) out.cap = std::min(out.cap, c->cap);
    out.nnz = out.cap == 0 ? 0 : -1;
    DBuf<int32_t> cnt;
    if (!out.rowptr.alloc(al, (size_t)n + 1) || !cnt.alloc(al, n) || !out.col.alloc(al, out.cap > 0 ? out.cap : 1))
        fail(HOMLN_ENOMEM, "and scratch");
    launch(k_and_rows<false>, grid_for((int64_t)n * 32), 256, 0, s, n, L, cnt.p, nullptr, nullptr);
    scan_exclusive_i32(cnt.p, out.rowptr.p, n, al, s);
    if (out.cap > 0)
        launch(k_and_rows<true>, grid_for((int64_t)n * 32), 256, 0, s, n, L, nullptr, out.rowptr.p, out.col.p);
    HCUDA(cudaGetLastError());
}

void or_union(int32_t n, const std::vector<const Csr *> &layers, Csr &out, Alloc *al, cudaStream_t s) {
    LayerSet L{};
    L.r = (int)layers.size();
    for (int i = 0; i < L.r; ++i) {
        L.rp[i] = layers[i]->rowptr.p;
        L.col[i] = layers[i]->col.p;
    }
    out.n = n;
    DBuf<int32_t> deg, cat, cnt;
    DBuf<int64_t> rp;
    if (!out.rowptr.alloc(al, (size_t)n + 1) || !deg.alloc(al, n) || !rp.alloc(al, (size_t)n + 1) || !cnt.alloc(al, n))
        fail(HOMLN_ENOMEM, "or scratch");
    int64_t total = 0;  // entries of the concatenated rows, at most
    for (const Csr *c : layers) total += c->cap;
    if (!cat.alloc(al, total > 0 ? total : 1)) fail(HOMLN_ENOMEM, "or rows");
    launch(k_sum_degrees, grid_for(n), 256, 0, s, n, L, deg.p);
    scan_exclusive_i32(deg.p, rp.p, n, al, s);
    launch(k_concat_rows, grid_for((int64_t)n * 32), 256, 0, s, n, L, (const int64_t *)rp.p, cat.p);
    sort_rows(n, rp.p, cat.p, total, al, s);
    launch(k_row_unique<false>, grid_for((int64_t)n * 32), 256, 0, s, n, (const int64_t *)rp.p,
           (const int32_t *)cat.p, cnt.p, (const int64_t *)nullptr, (int32_t *)nullptr);
    scan_exclusive_i32(cnt.p, out.rowptr.p, n, al, s);
    out.cap = total;
    out.nnz = total == 0 ? 0 : -1;
    if (!out.col.alloc(al, total > 0 ? total : 1)) fail(HOMLN_ENOMEM, "or col");
    if (total > 0)
        launch(k_row_unique<true>, grid_for((int64_t)n * 32), 256, 0, s, n, (const int64_t *)rp.p,
               (const int32_t *)cat.p, (int32_t *)nullptr, (const int64_t *)out.rowptr.p, out.col.p);
    HCUDA(cudaGetLastError());
}

void csr_edge_list(const Csr &g, int32_t *d_src, int32_t *d_dst, Alloc *al, cudaStream_t s, bool directed) {
    int32_t n = g.n;
    if (g.cap == 0) return;
    DBuf<int32_t> len;
    DBuf<int64_t> start, off;
    if (!len.alloc(al, n) || !start.alloc(al, n) || !off.alloc(al, (size_t)n + 1)) fail(HOMLN_ENOMEM, "edge list");
    launch(k_upper_len, grid_for(n), 256, 0, s, n, g.rowptr.p, g.col.p, len.p, start.p, directed ? 1 : 0);
    scan_exclusive_i32(len.p, off.p, n, al, s);
    launch(k_write_pairs, grid_for(n), 256, 0, s, n, g.col.p, start.p, len.p, off.p, d_src, d_dst);
    HCUDA(cudaGetLastError());
}

void relabel_apply(const Csr &g, const int32_t *perm, const int32_t *inv, Csr &out, Alloc *al, cudaStream_t s) {
    const int32_t n = g.n;
    DBuf<int32_t> newdeg;
    if (!newdeg.alloc(al, n)) fail(HOMLN_ENOMEM, "relabel scratch");
    launch(k_perm_degrees, grid_for(n), 256, 0, s, n, g.rowptr.p, perm, newdeg.p);
    out.n = n;
    out.nnz = g.nnz;
    out.cap = g.cap;
    if (!out.rowptr.alloc(al, (size_t)n + 1) || !out.col.alloc(al, g.cap > 0 ? g.cap : 1))
        fail(HOMLN_ENOMEM, "relabel csr");
    scan_exclusive_i32(newdeg.p, out.rowptr.p, n, al, s);
    if (g.cap > 0) {
        launch(k_relabel_rows, grid_for((int64_t)n * 32), 256, 0, s, n, g.rowptr.p, g.col.p, perm, inv,
               out.rowptr.p, out.col.p);
        sort_rows(n, out.rowptr.p, out.col.p, out.cap, al, s);
    }
    HCUDA(cudaGetLastError());
}

void relabel_by_degree(const Csr &g, const Csr *other, Csr &out, DBuf<int32_t> &perm, DBuf<int32_t> &inv,
                       DBuf<int32_t> &split, Alloc *al, cudaStream_t s) {
    const int32_t n = g.n;
    DBuf<uint64_t> vkeys;
    DBuf<unsigned int> ctr;
    if (!vkeys.alloc(al, n) || !inv.alloc(al, n) || !perm.alloc(al, n) || !split.alloc(al, 1) || !ctr.alloc(al, 2))
        fail(HOMLN_ENOMEM, "relabel scratch");
    HCUDA(cudaMemsetAsync(ctr.p, 0, 2 * sizeof(unsigned int), s));
    launch(k_degree_keys, grid_for(n), 256, 0, s, n, g.rowptr.p, g.col.p, other ? other->rowptr.p : nullptr,
           other ? other->col.p : nullptr, ctr.p, split.p, vkeys.p);
    // the keys are generated in id order, so a stable sort on the small-component bit and the
    // degree bits leaves equal keys in ascending id order
    radix_sort_u64(vkeys.p, nullptr, n, NODE_BITS, 2 * NODE_BITS + 1, al, s);
    launch(k_perm_from_keys, grid_for(n), 256, 0, s, n, vkeys.p, perm.p, inv.p);
    relabel_apply(g, perm.p, inv.p, out, al, s);
}

}  // namespace homln
