// All-sources BFS distance sums with a bitset multi-source BFS (MS-BFS).
//
// What it computes (Section 4: closeness by BFS from every vertex; Section 5.1:
// the per-node distance sums CC1/CC2 keep): for every vertex v of an undirected
// unweighted graph,
//     F[v] = sum over vertices u reachable from v of d(v, u),
//     R[v] = number of vertices reachable from v, v excluded.
//
// How: sources are processed in batches of S = 64*W. Every vertex carries three
// S-bit words -- seen, frontier, next -- one bit per source of the batch. A
// level either pulls (bottom-up: next[v] = OR of frontier[u] over neighbours u,
// minus seen[v]) or pushes (top-down: every frontier vertex ORs its word into
// its neighbours' accumulators, then a sweep keeps the bits not yet seen).
// Because the graph is undirected, d(s, v) = d(v, s): a bit of source s that
// first reaches v at level l adds l to F[v] directly, so no per-source scatter
// is needed -- F[v] += l * popc(new[v]), R[v] += popc(new[v]).
//
// The whole BFS of a graph (every batch, every level) runs in one persistent
// cooperative launch; levels are separated by a bounded grid barrier.
#include "common.cuh"

#include <algorithm>

namespace homln {

namespace {

struct BfsArgs {
    int32_t n;
    const int64_t *__restrict__ rowptr;
    const int32_t *__restrict__ col;
    uint64_t *seen;
    uint64_t *fa;
    uint64_t *fb;
    uint64_t *acc;     // top-down accumulator; all zero between phases
    uint8_t *quiet;    // per vertex: levels since its seen word became full (saturates at 2)
    uint64_t *F;
    uint32_t *R;
    unsigned long long *ctr;  // 3 slots x {new bits, frontier edges, unfinished edges, spare}
    GridBarrier bar;
    int32_t nbatches;
    int32_t push_alpha;
    int32_t hub_block_end;  // vertices [0, hub_block_end) are pulled/pushed by a whole block
    int32_t hub_warp_end;   // vertices [hub_block_end, hub_warp_end) by a whole warp
    unsigned long long *stats;
};

// A vertex is "quiet" once its seen word has been full at the start of two levels: both
// frontier buffers then hold zero for it and nothing can change it, so every later level
// of the batch skips it after reading one byte.
constexpr uint8_t QUIET = 2;

enum {
    ST_LEVELS, ST_PULL, ST_PUSH, ST_EDGES, ST_WORDS, ST_PUSHED, ST_BATCHES, ST_PUSHWORDS, ST_BYTES, ST_VISITS, ST_N
};

template <int W>
struct Geo {
    static constexpr int K = W >= 2 ? 2 : 1;  // 64-bit words per lane
    static constexpr int T = W / K;           // lanes per vertex
};

template <int K>
__device__ __forceinline__ void ldw(const uint64_t *p, uint64_t (&x)[K]) {
    if constexpr (K == 2) {
        ulonglong2 t = *reinterpret_cast<const ulonglong2 *>(p);
        x[0] = t.x;
        x[1] = t.y;
    } else {
        x[0] = *p;
    }
}

template <int K>
__device__ __forceinline__ void stw(uint64_t *p, const uint64_t (&x)[K]) {
    if constexpr (K == 2) {
        *reinterpret_cast<ulonglong2 *>(p) = make_ulonglong2(x[0], x[1]);
    } else {
        *p = x[0];
    }
}

template <int T>
__device__ __forceinline__ uint32_t group_sum(uint32_t v) {
#pragma unroll
    for (int o = T / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int T>
__device__ __forceinline__ bool group_any(bool b) {
    uint32_t v = b ? 1u : 0u;
#pragma unroll
    for (int o = T / 2; o > 0; o >>= 1) v |= __shfl_xor_sync(0xffffffffu, v, o);
    return v != 0;
}

template <int T>
__device__ __forceinline__ int64_t group_max(int64_t v) {
#pragma unroll
    for (int o = T / 2; o > 0; o >>= 1) v = max(v, (int64_t)__shfl_xor_sync(0xffffffffu, (long long)v, o));
    return v;
}

template <int K>
__device__ __forceinline__ bool covers(const uint64_t (&acc)[K], const uint64_t (&need)[K]) {
    bool ok = true;
#pragma unroll
    for (int k = 0; k < K; ++k) ok &= ((acc[k] & need[k]) == need[k]);
    return ok;
}

// OR the frontier words (this lane's K of them) of neighbours rb+p, rb+p+S, ... into acc;
// stop once every bit this lane still needs is present. Returns the neighbours visited.
template <int W>
__device__ __forceinline__ int64_t gather_or(const BfsArgs &a, const uint64_t *__restrict__ cur, int64_t rb,
                                             int64_t re, int p, int S, int q,
                                             const uint64_t (&need)[Geo<W>::K], uint64_t (&acc)[Geo<W>::K]) {
    constexpr int K = Geo<W>::K;
    int64_t j = rb + p;
    int64_t it = 0;
    for (; j + 3 * (int64_t)S < re; j += 4 * (int64_t)S) {
        const int32_t u0 = __ldg(a.col + j), u1 = __ldg(a.col + j + S), u2 = __ldg(a.col + j + 2 * S),
                      u3 = __ldg(a.col + j + 3 * S);
        uint64_t f0[K], f1[K], f2[K], f3[K];
        ldw<K>(cur + (int64_t)u0 * W + q * K, f0);
        ldw<K>(cur + (int64_t)u1 * W + q * K, f1);
        ldw<K>(cur + (int64_t)u2 * W + q * K, f2);
        ldw<K>(cur + (int64_t)u3 * W + q * K, f3);
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k] |= f0[k] | f1[k] | f2[k] | f3[k];
        it += 4;
        if (covers<K>(acc, need)) return it;
    }
    for (; j < re; j += S) {
        const int32_t u = __ldg(a.col + j);
        uint64_t f[K];
        ldw<K>(cur + (int64_t)u * W + q * K, f);
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k] |= f[k];
        ++it;
        if (covers<K>(acc, need)) return it;
    }
    return it;
}

struct PhaseCounters {
    unsigned long long newbits = 0, mf = 0, mu = 0;
};

// Block-reduce the phase counters and add them to the slot of this producing phase.
__device__ __forceinline__ void flush_counters(const BfsArgs &a, PhaseCounters &c, uint32_t ps) {
    __shared__ unsigned long long red[3][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned long long x0 = warp_sum(c.newbits), x1 = warp_sum(c.mf), x2 = warp_sum(c.mu);
    if (lane == 0) {
        red[0][warp] = x0;
        red[1][warp] = x1;
        red[2][warp] = x2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long s0 = 0, s1 = 0, s2 = 0;
        for (int w = 0; w < nw; ++w) {
            s0 += red[0][w];
            s1 += red[1][w];
            s2 += red[2][w];
        }
        unsigned long long *slot = a.ctr + 4 * (ps % 3);
        if (s0) atomicAdd(slot + 0, s0);
        if (s1) atomicAdd(slot + 1, s1);
        if (s2) atomicAdd(slot + 2, s2);
    }
    c = PhaseCounters{};
}

__device__ __forceinline__ void reset_next_slot(const BfsArgs &a, uint32_t ps) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        unsigned long long *slot = a.ctr + 4 * ((ps + 1) % 3);
        slot[0] = 0;
        slot[1] = 0;
        slot[2] = 0;
    }
}

// Record the new bits of v (already reduced to this lane's K words) and its counters.
// full0: the vertex's seen word was already full when the level started (its new bits are 0).
template <int W, bool STATS>
__device__ __forceinline__ void commit_vertex(const BfsArgs &a, bool act, bool writer, int64_t v, int q,
                                              const uint64_t (&s)[Geo<W>::K], const uint64_t (&nw)[Geo<W>::K],
                                              uint64_t *nxt, int level, int64_t deg, bool full0, uint8_t qv,
                                              PhaseCounters &c, unsigned long long *st) {
    constexpr int K = Geo<W>::K, T = Geo<W>::T;
    bool any = false, full = true;
    uint32_t cnt = 0;
    uint64_t ns[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        ns[k] = s[k] | nw[k];
        any |= nw[k] != 0;
        full &= ns[k] == ~0ull;
        cnt += __popcll(nw[k]);
    }
    if (act && writer) {
        if (any) stw<K>(a.seen + v * W + q * K, ns);
        stw<K>(nxt + v * W + q * K, nw);
        if (STATS) st[ST_BYTES] += (any ? 16 : 8) * K;
    }
    cnt = group_sum<T>(cnt);
    bool gfull = !group_any<T>(!full);
    if (act && writer && q == 0) {
        if (cnt) {
            a.F[v] += (uint64_t)level * cnt;
            a.R[v] += cnt;
            c.newbits += cnt;
            c.mf += (unsigned long long)deg;
            if (STATS) st[ST_BYTES] += 24;
        }
        if (!gfull) c.mu += (unsigned long long)deg;
        if (full0) a.quiet[v] = qv + 1;
        if (STATS) st[ST_VISITS] += 1;
    }
}

// ---------------------------------------------------------------- phases

// Level 0 and 1 of a batch: seen = own source bit (plus padding bits for a short
// last batch); every source ORs its bit into its neighbours' accumulators.
template <int W, bool STATS>
__device__ void phase_start_batch(const BfsArgs &a, int32_t s0, int32_t ns, unsigned long long *st) {
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t i = gtid; i < (int64_t)a.n * W; i += nthreads) {
        const int64_t v = i / W;
        const int wi = (int)(i % W);
        const int lo = wi * 64;
        uint64_t x = 0;
        if (lo >= ns) x = ~0ull;
        else if (lo + 64 > ns) x = ~0ull << (ns - lo);
        if (v >= s0 && v < (int64_t)s0 + ns) {
            const int b = (int)(v - s0);
            if ((b >> 6) == wi) x |= 1ull << (b & 63);
        }
        a.seen[i] = x;
        if (wi == 0) a.quiet[v] = 0;
        if (STATS) st[ST_BYTES] += 8 + (wi == 0);
    }
    const int64_t e0 = a.rowptr[s0], e1 = a.rowptr[s0 + ns];
    for (int64_t e = e0 + gtid; e < e1; e += nthreads) {
        int lo = 0, hi = ns;  // find the source row holding edge e
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (a.rowptr[s0 + mid] <= e) lo = mid; else hi = mid;
        }
        const int32_t u = __ldg(a.col + e);
        atomicOr(reinterpret_cast<unsigned long long *>(a.acc + (int64_t)u * W + (lo >> 6)), 1ull << (lo & 63));
        if (STATS) { st[ST_BYTES] += 4 + 8; st[ST_PUSHED] += 1; st[ST_PUSHWORDS] += 1; }
    }
}

// Keep the accumulated bits not yet seen: they become the next frontier.
template <int W, bool STATS>
__device__ void phase_finalize(const BfsArgs &a, uint64_t *nxt, int level, uint32_t ps, PhaseCounters &c,
                               unsigned long long *st) {
    constexpr int K = Geo<W>::K, T = Geo<W>::T;
    reset_next_slot(a, ps);
    const int lane = threadIdx.x & 31, q = lane % T;
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t G = ((int64_t)gridDim.x * blockDim.x) / T;
    for (int64_t v = gtid / T; __any_sync(0xffffffffu, v < a.n); v += G) {
        uint8_t qv = 0;
        if (v < a.n) {
            qv = a.quiet[v];
            if (STATS && q == 0) st[ST_BYTES] += 1;
        }
        const bool act = v < a.n && qv < QUIET;
        uint64_t s[K], z[K], nw[K];
        int64_t deg = 0;
        bool lane_full = true;
#pragma unroll
        for (int k = 0; k < K; ++k) s[k] = z[k] = nw[k] = 0;
        if (act) {
            ldw<K>(a.acc + v * W + q * K, z);
            ldw<K>(a.seen + v * W + q * K, s);
            bool nz = false;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                nw[k] = z[k] & ~s[k];
                nz |= z[k] != 0;
                lane_full &= s[k] == ~0ull;
            }
            if (nz) {
                uint64_t zero[K];
#pragma unroll
                for (int k = 0; k < K; ++k) zero[k] = 0;
                stw<K>(a.acc + v * W + q * K, zero);
            }
            deg = a.rowptr[v + 1] - a.rowptr[v];
            if (STATS) st[ST_BYTES] += (nz ? 24 : 16) * K + (q == 0 ? 16 : 0);
        }
        const bool full0 = !group_any<T>(!lane_full);
        commit_vertex<W, STATS>(a, act, true, v, q, s, nw, nxt, level, deg, full0, qv, c, st);
    }
    flush_counters(a, c, ps);
}

// Bottom-up level: each vertex still missing bits gathers its neighbours' frontier words.
template <int W, bool STATS>
__device__ void phase_pull(const BfsArgs &a, const uint64_t *__restrict__ cur, uint64_t *nxt, int level, uint32_t ps,
                           PhaseCounters &c, unsigned long long *st) {
    constexpr int K = Geo<W>::K, T = Geo<W>::T;
    reset_next_slot(a, ps);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int q = lane % T;

    // --- block tier: the largest hubs, all slots of the block share one row
    {
        __shared__ uint64_t red[32][16][2];
        const int S = blockDim.x / T, p = threadIdx.x / T;
        for (int64_t v = blockIdx.x; v < a.hub_block_end; v += gridDim.x) {
            const uint8_t qv = a.quiet[v];
            if (STATS && threadIdx.x == 0) st[ST_BYTES] += 1;
            if (qv >= QUIET) continue;  // uniform over the block
            uint64_t s[K], need[K], acc[K];
            ldw<K>(a.seen + v * W + q * K, s);
            bool lane_need = false;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                need[k] = ~s[k];
                acc[k] = 0;
                lane_need |= need[k] != 0;
            }
            const bool full0 = __syncthreads_or(lane_need ? 1 : 0) == 0;
            const int64_t rb = a.rowptr[v], re = a.rowptr[v + 1];
            int64_t it = 0;
            if (lane_need) it = gather_or<W>(a, cur, rb, re, p, S, q, need, acc);
            if (STATS) {
                st[ST_WORDS] += it * K;
                st[ST_BYTES] += it * 8 * K;
                int64_t gm = group_max<T>(it);
                if (q == 0) { st[ST_EDGES] += gm; st[ST_BYTES] += 4 * gm; }
                if (p == 0) st[ST_BYTES] += 8 * K + (q == 0 ? 16 : 0);
            }
#pragma unroll
            for (int o = T; o < 32; o <<= 1)
#pragma unroll
                for (int k = 0; k < K; ++k) acc[k] |= __shfl_xor_sync(0xffffffffu, acc[k], o);
            if (lane < T)
#pragma unroll
                for (int k = 0; k < K; ++k) red[warp][lane][k] = acc[k];
            __syncthreads();
            if (warp == 0) {
                uint64_t t[K], nw[K];
#pragma unroll
                for (int k = 0; k < K; ++k) t[k] = 0;
                if (lane < T)
                    for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
#pragma unroll
                        for (int k = 0; k < K; ++k) t[k] |= red[w][lane][k];
#pragma unroll
                for (int k = 0; k < K; ++k) nw[k] = t[k] & need[k];
                commit_vertex<W, STATS>(a, true, lane < T, v, q, s, nw, nxt, level, re - rb, full0, qv, c, st);
            }
            __syncthreads();
        }
    }
    // --- warp tier: hubs below the block threshold, all slots of a warp share one row
    {
        const int S = 32 / T, p = lane / T;
        const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        const int64_t NW = ((int64_t)gridDim.x * blockDim.x) >> 5;
        for (int64_t v = a.hub_block_end + gw; v < a.hub_warp_end; v += NW) {
            const uint8_t qv = a.quiet[v];
            if (STATS && lane == 0) st[ST_BYTES] += 1;
            if (qv >= QUIET) continue;  // uniform over the warp
            uint64_t s[K], need[K], acc[K], nw[K];
            ldw<K>(a.seen + v * W + q * K, s);
            bool lane_need = false;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                need[k] = ~s[k];
                acc[k] = 0;
                lane_need |= need[k] != 0;
            }
            const bool full0 = !__any_sync(0xffffffffu, lane_need);
            const int64_t rb = a.rowptr[v], re = a.rowptr[v + 1];
            int64_t it = 0;
            if (lane_need) it = gather_or<W>(a, cur, rb, re, p, S, q, need, acc);
            if (STATS) {
                st[ST_WORDS] += it * K;
                st[ST_BYTES] += it * 8 * K;
                int64_t gm = group_max<T>(it);
                if (q == 0) { st[ST_EDGES] += gm; st[ST_BYTES] += 4 * gm; }
                if (p == 0) st[ST_BYTES] += 8 * K + (q == 0 ? 16 : 0);
            }
#pragma unroll
            for (int o = T; o < 32; o <<= 1)
#pragma unroll
                for (int k = 0; k < K; ++k) acc[k] |= __shfl_xor_sync(0xffffffffu, acc[k], o);
#pragma unroll
            for (int k = 0; k < K; ++k) nw[k] = acc[k] & need[k];
            commit_vertex<W, STATS>(a, true, p == 0, v, q, s, nw, nxt, level, re - rb, full0, qv, c, st);
        }
    }
    // --- group tier: T lanes per vertex
    {
        const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        const int64_t G = ((int64_t)gridDim.x * blockDim.x) / T;
        for (int64_t v = a.hub_warp_end + gtid / T; __any_sync(0xffffffffu, v < a.n); v += G) {
            uint8_t qv = 0;
            if (v < a.n) {
                qv = a.quiet[v];
                if (STATS && q == 0) st[ST_BYTES] += 1;
            }
            const bool act = v < a.n && qv < QUIET;
            uint64_t s[K], need[K], acc[K], nw[K];
            bool lane_need = false;
            int64_t rb = 0, re = 0;
#pragma unroll
            for (int k = 0; k < K; ++k) s[k] = need[k] = acc[k] = 0;
            if (act) {
                ldw<K>(a.seen + v * W + q * K, s);
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    need[k] = ~s[k];
                    lane_need |= need[k] != 0;
                }
                rb = a.rowptr[v];
                re = a.rowptr[v + 1];
            }
            // every lane must take part in the shuffle, so no short-circuit around it
            const bool group_needs = group_any<T>(lane_need);
            const bool full0 = act && !group_needs;
            int64_t it = 0;
            if (lane_need) it = gather_or<W>(a, cur, rb, re, 0, 1, q, need, acc);
            if (STATS) {
                st[ST_WORDS] += it * K;
                st[ST_BYTES] += it * 8 * K;
                int64_t gm = group_max<T>(it);
                if (q == 0) { st[ST_EDGES] += gm; st[ST_BYTES] += 4 * gm; }
                if (act) st[ST_BYTES] += 8 * K + (q == 0 ? 16 : 0);
            }
#pragma unroll
            for (int k = 0; k < K; ++k) nw[k] = acc[k] & need[k];
            commit_vertex<W, STATS>(a, act, true, v, q, s, nw, nxt, level, re - rb, full0, qv, c, st);
        }
    }
    flush_counters(a, c, ps);
}

// Top-down level: frontier vertices OR their words into the neighbours' accumulators
// (quiet neighbours are full and are skipped).
template <int W, bool STATS>
__device__ void phase_push(const BfsArgs &a, const uint64_t *__restrict__ cur, unsigned long long *st) {
    constexpr int K = Geo<W>::K, T = Geo<W>::T;
    const int lane = threadIdx.x & 31;
    const int q = lane % T;
    auto push_row = [&](int64_t v, int p, int S) {
        if (a.quiet[v] >= QUIET) return;  // a quiet vertex has an all-zero frontier word
        uint64_t f[K];
        ldw<K>(cur + v * W + q * K, f);
        if (STATS) st[ST_BYTES] += 8 * K + 1;
        bool any = false;
#pragma unroll
        for (int k = 0; k < K; ++k) any |= f[k] != 0;
        if (!any) return;
        const int64_t rb = a.rowptr[v], re = a.rowptr[v + 1];
        for (int64_t j = rb + p; j < re; j += S) {
            const int64_t u = __ldg(a.col + j);
            if (STATS && q == 0) { st[ST_PUSHED] += 1; st[ST_BYTES] += 5; }
            if (a.quiet[u] >= QUIET) continue;
#pragma unroll
            for (int k = 0; k < K; ++k)
                if (f[k]) {
                    atomicOr(reinterpret_cast<unsigned long long *>(a.acc + u * W + q * K + k), f[k]);
                    if (STATS) { st[ST_PUSHWORDS] += 1; st[ST_BYTES] += 8; }
                }
        }
    };
    for (int64_t v = blockIdx.x; v < a.hub_block_end; v += gridDim.x) push_row(v, threadIdx.x / T, blockDim.x / T);
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t NW = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = a.hub_block_end + gw; v < a.hub_warp_end; v += NW) push_row(v, lane / T, 32 / T);
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t G = ((int64_t)gridDim.x * blockDim.x) / T;
    for (int64_t v = a.hub_warp_end + gtid / T; v < a.n; v += G) push_row(v, 0, 1);
}

template <int W, bool STATS>
__global__ void __launch_bounds__(512, 2) k_msbfs(BfsArgs a) {
    PhaseCounters c;
    unsigned long long st[ST_N];
#pragma unroll
    for (int i = 0; i < ST_N; ++i) st[i] = 0;
    uint32_t ps = 0;  // index of the next counter-producing phase
    for (int32_t b = 0; b < a.nbatches; ++b) {
        const int32_t s0 = b * 64 * W;
        const int32_t ns = min(64 * W, a.n - s0);
        phase_start_batch<W, STATS>(a, s0, ns, st);
        if (!grid_sync(a.bar)) return;
        phase_finalize<W, STATS>(a, a.fa, 1, ps, c, st);
        ++ps;
        if (!grid_sync(a.bar)) return;
        uint64_t *cur = a.fa, *nxt = a.fb;
        if (STATS) { st[ST_BATCHES] += 1; st[ST_LEVELS] += 1; st[ST_PUSH] += 1; }
        for (int level = 2; level <= a.n + 1; ++level) {
            const unsigned long long *slot = a.ctr + 4 * ((ps - 1) % 3);
            const unsigned long long newbits = __ldcg(slot), mf = __ldcg(slot + 1), mu = __ldcg(slot + 2);
            if (newbits == 0) break;
            const bool push = (unsigned long long)a.push_alpha * mf < mu;
            if (push) {
                phase_push<W, STATS>(a, cur, st);
                if (!grid_sync(a.bar)) return;
                phase_finalize<W, STATS>(a, nxt, level, ps, c, st);
            } else {
                phase_pull<W, STATS>(a, cur, nxt, level, ps, c, st);
            }
            ++ps;
            if (!grid_sync(a.bar)) return;
            if (STATS) { st[ST_LEVELS] += 1; st[push ? ST_PUSH : ST_PULL] += 1; }
            uint64_t *t = cur; cur = nxt; nxt = t;
        }
    }
    if (STATS && a.stats) {
        if (threadIdx.x == 0 && blockIdx.x == 0) {
            atomicAdd(a.stats + ST_LEVELS, st[ST_LEVELS]);
            atomicAdd(a.stats + ST_PULL, st[ST_PULL]);
            atomicAdd(a.stats + ST_PUSH, st[ST_PUSH]);
            atomicAdd(a.stats + ST_BATCHES, st[ST_BATCHES]);
        }
        atomicAdd(a.stats + ST_EDGES, st[ST_EDGES]);
        atomicAdd(a.stats + ST_WORDS, st[ST_WORDS]);
        atomicAdd(a.stats + ST_PUSHED, st[ST_PUSHED]);
        atomicAdd(a.stats + ST_PUSHWORDS, st[ST_PUSHWORDS]);
        atomicAdd(a.stats + ST_BYTES, st[ST_BYTES]);
        atomicAdd(a.stats + ST_VISITS, st[ST_VISITS]);
    }
}

__global__ void k_scatter_back(int32_t n, const int32_t *__restrict__ perm, const uint64_t *__restrict__ Fi,
                               const uint32_t *__restrict__ Ri, uint64_t *__restrict__ F, uint32_t *__restrict__ R) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        F[perm[i]] = Fi[i];
        R[perm[i]] = Ri[i];
    }
}

// Since the relabelled rows are sorted by degree (descending), the tier boundaries are
// the first rows whose degree falls below each threshold.
__global__ void k_tier_bounds(int32_t n, const int64_t *__restrict__ rp, int64_t block_deg, int64_t warp_deg,
                              int32_t *out) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int64_t d = rp[i + 1] - rp[i];
        int64_t dn = i + 1 < n ? rp[i + 2] - rp[i + 1] : -1;
        if (d >= block_deg && dn < block_deg) out[0] = i + 1;
        if (d >= warp_deg && dn < warp_deg) out[1] = i + 1;
    }
}

typedef void (*BfsKernel)(BfsArgs);

template <int W>
BfsKernel pick_kernel(bool stats) {
    return stats ? k_msbfs<W, true> : k_msbfs<W, false>;
}

BfsKernel kernel_for(int W, bool stats) {
    switch (W) {
    case 1: return pick_kernel<1>(stats);
    case 2: return pick_kernel<2>(stats);
    case 4: return pick_kernel<4>(stats);
    case 8: return pick_kernel<8>(stats);
    case 16: return pick_kernel<16>(stats);
    case 32: return pick_kernel<32>(stats);
    default: fail(HOMLN_EINVAL, "words_per_node must be 1, 2, 4, 8, 16 or 32");
    }
}

}  // namespace

int msbfs_pick_words(int32_t n, int64_t nnz) {
    (void)nnz;
    // four n x W word arrays should stay well inside L2 (about 48 MB of it)
    int W = 32;
    while (W > 1 && 4.0 * n * 8.0 * W > 48.0e6) W >>= 1;
    while (W > 1 && (int64_t)64 * (W / 2) >= n) W >>= 1;  // no wider than the node count needs
    return W;
}

void msbfs_all_sources(const Csr &g, uint64_t *d_F, uint32_t *d_R, const BfsTuning &t, int32_t *d_err, Alloc *al,
                       cudaStream_t s, BfsStats *stats, float *kernel_ms, cudaEvent_t ev_start, cudaEvent_t ev_stop) {
    const int32_t n = g.n;
    if (n <= 0) return;
    const int W = t.W > 0 ? t.W : msbfs_pick_words(n, g.nnz);
    const int T = W >= 2 ? W / 2 : 1;
    const int threads = t.threads > 0 ? t.threads : 512;
    if (threads % 32 != 0 || threads > 512 || threads < 64) fail(HOMLN_EINVAL, "threads must be 64..512, multiple of 32");

    const Csr *G = &g;
    Csr rl;
    DBuf<int32_t> perm;
    if (t.relabel) {
        relabel_by_degree(g, rl, perm, al, s);
        G = &rl;
    }
    const size_t words = (size_t)n * W;
    DBuf<uint64_t> seen, fa, fb, acc, Fi;
    DBuf<uint8_t> quiet;
    DBuf<uint32_t> Ri;
    DBuf<unsigned long long> ctr, st;
    DBuf<uint32_t> barmem;
    DBuf<int32_t> tiers;
    if (!seen.alloc(al, words) || !fa.alloc(al, words) || !fb.alloc(al, words) || !acc.alloc(al, words) ||
        !quiet.alloc(al, (size_t)n) ||
        !ctr.alloc(al, 12) || !barmem.alloc(al, 2) || !tiers.alloc(al, 2))
        fail(HOMLN_ENOMEM, "bfs state");
    uint64_t *F = d_F;
    uint32_t *R = d_R;
    if (t.relabel) {
        if (!Fi.alloc(al, n) || !Ri.alloc(al, n)) fail(HOMLN_ENOMEM, "bfs relabelled outputs");
        F = Fi.p;
        R = Ri.p;
    }
    if (stats && !st.alloc(al, ST_N)) fail(HOMLN_ENOMEM, "bfs stats");
    HCUDA(cudaMemsetAsync(acc.p, 0, words * sizeof(uint64_t), s));
    HCUDA(cudaMemsetAsync(F, 0, (size_t)n * sizeof(uint64_t), s));
    HCUDA(cudaMemsetAsync(R, 0, (size_t)n * sizeof(uint32_t), s));
    HCUDA(cudaMemsetAsync(ctr.p, 0, 12 * sizeof(unsigned long long), s));
    HCUDA(cudaMemsetAsync(barmem.p, 0, 2 * sizeof(uint32_t), s));
    HCUDA(cudaMemsetAsync(tiers.p, 0, 2 * sizeof(int32_t), s));
    if (stats) HCUDA(cudaMemsetAsync(st.p, 0, ST_N * sizeof(unsigned long long), s));

    int32_t h_tiers[2] = {0, 0};
    if (t.relabel && G->nnz > 0) {
        const int64_t slots_block = threads / T, slots_warp = 32 / T;
        launch(k_tier_bounds, (unsigned)ceil_div(n, 256), 256, 0, s, n, G->rowptr.p, 32 * slots_block, 16 * slots_warp,
                                                               tiers.p);
        HCUDA(cudaMemcpyAsync(h_tiers, tiers.p, sizeof(h_tiers), cudaMemcpyDeviceToHost, s));
        HCUDA(cudaStreamSynchronize(s));
        if (h_tiers[1] < h_tiers[0]) h_tiers[1] = h_tiers[0];
    }

    BfsKernel kern = kernel_for(W, stats != nullptr);
    int dev = 0, nsm = 0, coop = 0, per_sm = 0;
    HCUDA(cudaGetDevice(&dev));
    HCUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    HCUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    if (!coop) fail(HOMLN_ECUDA, "device does not support cooperative launch");
    HCUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0));
    if (per_sm < 1) fail(HOMLN_ECUDA, "bfs kernel does not fit on an SM");
    if (t.blocks_per_sm > 0 && t.blocks_per_sm < per_sm) per_sm = t.blocks_per_sm;

    BfsArgs a{};
    a.n = n;
    a.rowptr = G->rowptr.p;
    a.col = G->col.p;
    a.seen = seen.p;
    a.fa = fa.p;
    a.fb = fb.p;
    a.acc = acc.p;
    a.quiet = quiet.p;
    a.F = F;
    a.R = R;
    a.ctr = ctr.p;
    a.bar = GridBarrier{barmem.p, barmem.p + 1, d_err};
    a.nbatches = (int32_t)ceil_div(n, 64 * W);
    a.push_alpha = t.push_alpha > 0 ? t.push_alpha : 8;
    a.hub_block_end = h_tiers[0];
    a.hub_warp_end = h_tiers[1];
    a.stats = stats ? st.p : nullptr;
    void *args[] = {&a};

    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (kernel_ms) {
        HCUDA(cudaEventCreate(&e0));
        HCUDA(cudaEventCreate(&e1));
        HCUDA(cudaEventRecord(e0, s));
    }
    if (ev_start) HCUDA(cudaEventRecord(ev_start, s));
    g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
    HCUDA(cudaLaunchCooperativeKernel((const void *)kern, dim3(nsm * per_sm), dim3(threads), args, 0, s));
    if (ev_stop) HCUDA(cudaEventRecord(ev_stop, s));
    if (kernel_ms) {
        HCUDA(cudaEventRecord(e1, s));
        HCUDA(cudaEventSynchronize(e1));
        HCUDA(cudaEventElapsedTime(kernel_ms, e0, e1));
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    if (t.relabel)
        launch(k_scatter_back, (unsigned)ceil_div(n, 256), 256, 0, s, n, perm.p, Fi.p, Ri.p, d_F, d_R);
    HCUDA(cudaGetLastError());
    if (stats) {
        unsigned long long h[ST_N];
        HCUDA(cudaMemcpyAsync(h, st.p, sizeof(h), cudaMemcpyDeviceToHost, s));
        HCUDA(cudaStreamSynchronize(s));
        stats->levels += h[ST_LEVELS];
        stats->pull_levels += h[ST_PULL];
        stats->push_levels += h[ST_PUSH];
        stats->group_edges += h[ST_EDGES];
        stats->lane_words += h[ST_WORDS];
        stats->push_edges += h[ST_PUSHED];
        stats->batches += h[ST_BATCHES];
        stats->push_words += h[ST_PUSHWORDS];
        stats->bytes += h[ST_BYTES];
        stats->visits += h[ST_VISITS];
    }
    if (stats) stats->words_per_node = W;
}

}  // namespace homln
