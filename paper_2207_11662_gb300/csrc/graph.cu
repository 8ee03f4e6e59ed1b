// Device graph store: CSR construction, Boolean AND aggregation, edge-list
// export and degree-descending relabelling.
//
// Section 4 treats every layer as a simple undirected graph (NetworkX Graph):
// self loops and repeated edges vanish, each edge is reachable from both ends.
// Section 3.1 / Section 4 define the AND aggregate: an edge survives iff it is
// in every selected layer.
#include "common.cuh"

namespace homln {

namespace {

constexpr int NODE_BITS = 20;  // HOMLN_MAX_NODES = 2^20
constexpr uint64_t NODE_MASK = (1ull << NODE_BITS) - 1;
constexpr uint64_t KEY_SENTINEL = (1ull << (2 * NODE_BITS)) - 1;  // sorts after every real key

// Each undirected input edge (a, b) becomes the directed keys a:b and b:a.
__global__ void k_expand_edges(const int32_t *__restrict__ src, const int32_t *__restrict__ dst, int64_t m, int32_t n,
                               uint64_t *__restrict__ keys, int32_t *err) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        int32_t a = src[e], b = dst[e];
        uint64_t k0 = KEY_SENTINEL, k1 = KEY_SENTINEL;
        if (a < 0 || a >= n || b < 0 || b >= n) {
            dev_fail(err, DEV_BAD_ID);
        } else if (a != b) {
            k0 = ((uint64_t)a << NODE_BITS) | (uint64_t)b;
            k1 = ((uint64_t)b << NODE_BITS) | (uint64_t)a;
        }
        keys[2 * e] = k0;
        keys[2 * e + 1] = k1;
    }
}

__global__ void k_unique_flags(const uint64_t *__restrict__ keys, int64_t cnt, int32_t *__restrict__ flag) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t k = keys[i];
        flag[i] = (k != KEY_SENTINEL && (i == 0 || keys[i - 1] != k)) ? 1 : 0;
    }
}

__global__ void k_compact_keys(const uint64_t *__restrict__ keys, const int32_t *__restrict__ flag,
                               const int64_t *__restrict__ pos, int64_t cnt, int32_t *__restrict__ col,
                               int32_t *__restrict__ deg) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x) {
        if (flag[i]) {
            uint64_t k = keys[i];
            col[pos[i]] = (int32_t)(k & NODE_MASK);
            atomicAdd(&deg[k >> NODE_BITS], 1);
        }
    }
}

struct LayerSet {
    const int64_t *rp[HOMLN_MAX_LAYERS];
    const int32_t *col[HOMLN_MAX_LAYERS];
    int r;
};

__device__ __forceinline__ bool row_contains(const int32_t *__restrict__ col, int64_t lo, int64_t hi, int32_t x) {
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        int32_t c = col[mid];
        if (c == x) return true;
        if (c < x) lo = mid + 1; else hi = mid;
    }
    return false;
}

// One warp per vertex: the lanes walk the shortest of its rows 32 entries at a time and keep
// the entries found (binary search) in every other row; a ballot keeps them in order.
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
        int32_t c = 0;
        for (int64_t j0 = 0; j0 < best_len; j0 += 32) {
            const int64_t j = j0 + lane;
            bool all = false;
            int32_t v = 0;
            if (j < best_len) {
                v = L.col[best][b0 + j];
                all = true;
                for (int i = 0; i < L.r && all; ++i)
                    if (i != best) all = row_contains(L.col[i], L.rp[i][u], L.rp[i][u + 1], v);
            }
            const uint32_t m = __ballot_sync(0xffffffffu, all);
            if (WRITE && all) out_col[o + c + __popc(m & ((1u << lane) - 1u))] = v;
            c += __popc(m);
        }
        if (!WRITE && lane == 0) cnt[u] = c;
    }
}

// Length of the part of row u holding neighbours v > u (rows are sorted).
__global__ void k_upper_len(int32_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                            int32_t *__restrict__ len, int64_t *__restrict__ start) {
    for (int32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        int64_t lo = rp[u], hi = rp[u + 1];
        int64_t a = lo, b = hi;
        while (a < b) {
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

__global__ void k_degree_keys(int32_t n, const int64_t *__restrict__ rp, uint64_t *__restrict__ keys) {
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        uint64_t deg = (uint64_t)(rp[v + 1] - rp[v]);
        keys[v] = ((NODE_MASK - deg) << NODE_BITS) | (uint64_t)v;  // degree descending, then id ascending
    }
}

__global__ void k_perm_from_keys(int32_t n, const uint64_t *__restrict__ keys, const int64_t *__restrict__ rp,
                                 int32_t *__restrict__ perm, int32_t *__restrict__ inv, int32_t *__restrict__ newdeg) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int32_t old = (int32_t)(keys[i] & NODE_MASK);
        perm[i] = old;
        inv[old] = i;
        newdeg[i] = (int32_t)(rp[old + 1] - rp[old]);
    }
}

// Relabelled entries as (new row, new col) keys; sorting them sorts every row.
__global__ void k_relabel_entries(int32_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                                  const int32_t *__restrict__ perm, const int32_t *__restrict__ inv,
                                  const int64_t *__restrict__ nrp, uint64_t *__restrict__ keys) {
    // one warp per new row
    int lane = threadIdx.x & 31;
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < n; i += nwarps) {
        int32_t old = perm[i];
        int64_t a = rp[old], len = rp[old + 1] - a, o = nrp[i];
        for (int64_t j = lane; j < len; j += 32)
            keys[o + j] = ((uint64_t)i << NODE_BITS) | (uint64_t)inv[col[a + j]];
    }
}

__global__ void k_keys_to_col(int64_t cnt, const uint64_t *__restrict__ keys, int32_t *__restrict__ col) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x)
        col[i] = (int32_t)(keys[i] & NODE_MASK);
}

unsigned grid_for(int64_t work, int threads = 256) {
    int64_t b = ceil_div(work > 0 ? work : 1, threads);
    return (unsigned)(b > 65535 * 16 ? 65535 * 16 : b);
}

int64_t read_i64(const int64_t *d, cudaStream_t s) {
    int64_t v = 0;
    HCUDA(cudaMemcpyAsync(&v, d, sizeof(v), cudaMemcpyDeviceToHost, s));
    HCUDA(cudaStreamSynchronize(s));
    return v;
}

}  // namespace

void build_csr(int32_t n, const int32_t *d_src, const int32_t *d_dst, int64_t m, Csr &out, int32_t *d_err, Alloc *al,
               cudaStream_t s) {
    out.n = n;
    if (!out.rowptr.alloc(al, (size_t)n + 1)) fail(HOMLN_ENOMEM, "csr rowptr");
    if (m == 0) {
        HCUDA(cudaMemsetAsync(out.rowptr.p, 0, sizeof(int64_t) * (n + 1), s));
        out.nnz = 0;
        out.col.release();
        return;
    }
    const int64_t cnt = 2 * m;
    DBuf<uint64_t> keys;
    DBuf<int32_t> flag, deg;
    DBuf<int64_t> pos;
    if (!keys.alloc(al, cnt) || !flag.alloc(al, cnt) || !pos.alloc(al, cnt + 1) || !deg.alloc(al, n))
        fail(HOMLN_ENOMEM, "csr scratch");
    launch(k_expand_edges, grid_for(m), 256, 0, s, d_src, d_dst, m, n, keys.p, d_err);
    radix_sort_u64(keys.p, nullptr, cnt, 0, 2 * NODE_BITS, al, s);
    launch(k_unique_flags, grid_for(cnt), 256, 0, s, keys.p, cnt, flag.p);
    scan_exclusive_i32(flag.p, pos.p, cnt, al, s);
    out.nnz = read_i64(pos.p + cnt, s);
    if (!out.col.alloc(al, out.nnz > 0 ? out.nnz : 1)) fail(HOMLN_ENOMEM, "csr col");
    HCUDA(cudaMemsetAsync(deg.p, 0, sizeof(int32_t) * n, s));
    launch(k_compact_keys, grid_for(cnt), 256, 0, s, keys.p, flag.p, pos.p, cnt, out.col.p, deg.p);
    scan_exclusive_i32(deg.p, out.rowptr.p, n, al, s);
    HCUDA(cudaGetLastError());
}

void and_intersect(int32_t n, const std::vector<const Csr *> &layers, Csr &out, Alloc *al, cudaStream_t s) {
    LayerSet L{};
    L.r = (int)layers.size();
    for (int i = 0; i < L.r; ++i) {
        L.rp[i] = layers[i]->rowptr.p;
        L.col[i] = layers[i]->col.p;
    }
    out.n = n;
    DBuf<int32_t> cnt;
    if (!out.rowptr.alloc(al, (size_t)n + 1) || !cnt.alloc(al, n)) fail(HOMLN_ENOMEM, "and scratch");
    launch(k_and_rows<false>, grid_for((int64_t)n * 32), 256, 0, s, n, L, cnt.p, nullptr, nullptr);
    scan_exclusive_i32(cnt.p, out.rowptr.p, n, al, s);
    out.nnz = read_i64(out.rowptr.p + n, s);
    if (!out.col.alloc(al, out.nnz > 0 ? out.nnz : 1)) fail(HOMLN_ENOMEM, "and col");
    if (out.nnz > 0)
        launch(k_and_rows<true>, grid_for((int64_t)n * 32), 256, 0, s, n, L, nullptr, out.rowptr.p, out.col.p);
    HCUDA(cudaGetLastError());
}

void csr_edge_list(const Csr &g, int32_t *d_src, int32_t *d_dst, Alloc *al, cudaStream_t s) {
    int32_t n = g.n;
    if (g.nnz == 0) return;
    DBuf<int32_t> len;
    DBuf<int64_t> start, off;
    if (!len.alloc(al, n) || !start.alloc(al, n) || !off.alloc(al, (size_t)n + 1)) fail(HOMLN_ENOMEM, "edge list");
    launch(k_upper_len, grid_for(n), 256, 0, s, n, g.rowptr.p, g.col.p, len.p, start.p);
    scan_exclusive_i32(len.p, off.p, n, al, s);
    launch(k_write_pairs, grid_for(n), 256, 0, s, n, g.col.p, start.p, len.p, off.p, d_src, d_dst);
    HCUDA(cudaGetLastError());
}

void relabel_by_degree(const Csr &g, Csr &out, DBuf<int32_t> &perm, Alloc *al, cudaStream_t s) {
    const int32_t n = g.n;
    DBuf<uint64_t> vkeys;
    DBuf<int32_t> inv, newdeg;
    if (!vkeys.alloc(al, n) || !inv.alloc(al, n) || !newdeg.alloc(al, n) || !perm.alloc(al, n))
        fail(HOMLN_ENOMEM, "relabel scratch");
    launch(k_degree_keys, grid_for(n), 256, 0, s, n, g.rowptr.p, vkeys.p);
    // the keys are generated in id order, so a stable sort on the degree bits alone leaves equal
    // degrees in ascending id order
    radix_sort_u64(vkeys.p, nullptr, n, NODE_BITS, 2 * NODE_BITS, al, s);
    launch(k_perm_from_keys, grid_for(n), 256, 0, s, n, vkeys.p, g.rowptr.p, perm.p, inv.p, newdeg.p);
    out.n = n;
    out.nnz = g.nnz;
    if (!out.rowptr.alloc(al, (size_t)n + 1) || !out.col.alloc(al, g.nnz > 0 ? g.nnz : 1))
        fail(HOMLN_ENOMEM, "relabel csr");
    scan_exclusive_i32(newdeg.p, out.rowptr.p, n, al, s);
    if (g.nnz > 0) {
        DBuf<uint64_t> ekeys;
        if (!ekeys.alloc(al, g.nnz)) fail(HOMLN_ENOMEM, "relabel keys");
        launch(k_relabel_entries, grid_for((int64_t)n * 32), 256, 0, s, n, g.rowptr.p, g.col.p, perm.p, inv.p,
                                                                    out.rowptr.p, ekeys.p);
        radix_sort_u64(ekeys.p, nullptr, g.nnz, 0, 2 * NODE_BITS, al, s);
        launch(k_keys_to_col, grid_for(g.nnz), 256, 0, s, g.nnz, ekeys.p, out.col.p);
    }
    HCUDA(cudaGetLastError());
}

}  // namespace homln
