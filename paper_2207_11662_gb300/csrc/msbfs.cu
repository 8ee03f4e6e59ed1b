// All-sources BFS distance sums with a bitset multi-source BFS (MS-BFS).
//
// What it computes (Section 4: closeness by BFS from every vertex; Section 5.1:
// the per-node distance sums CC1/CC2 keep): for every vertex v of an unweighted
// graph,
//     F[v] = sum over vertices u that v reaches (undirected) or that reach v
//            (directed: in-closeness) of the hop distance,
//     R[v] = number of those vertices, v excluded.
//
// How: sources are processed in batches of S = 64*W. Every vertex carries S-bit
// words, one bit per source of the batch, in two snapshots: after level l,
// snapshot l mod 2 holds for every vertex the sources within distance l. A
// level either pulls (bottom-up: the new bits of v are the OR of its
// (in-)neighbours' words in the previous snapshot, minus v's own) or pushes
// (top-down: every vertex with new bits on the previous level ORs its words into
// its (out-)neighbours' words of the next snapshot, then a sweep keeps the bits
// they did not have). A bit of source s that first reaches v at level l means d(s, v) = l,
// which undirected is d(v, s): F[v] += l * popc(new[v]), R[v] += popc(new[v]),
// with no per-source scatter; directed, the same sum is v's in-farness.
//
// Scheduling: one persistent cooperative launch covers every (graph, batch)
// tile of one or many graphs (the layers of a HoMLN and their AND aggregate, or
// many HoMLNs). The grid is split into teams of blocks; a team pops the next
// tile from a device queue and runs its levels, separated by a bounded barrier
// over the team's blocks only. Teams progress independently, so one team's wait
// overlaps another team's work.
#include "common.cuh"

#include <algorithm>
#include <chrono>
#include <memory>
#include <thread>

namespace homln {

namespace {

struct GraphDesc {
    const int64_t *rowptr;  // out-edges: top-down levels push along them
    const int32_t *col;
    const int64_t *prow;    // in-edges: bottom-up levels pull along them (the same CSR if undirected)
    const int32_t *pcol;
    uint64_t *F;
    uint32_t *R;
    int32_t n;
    int32_t nbatches;       // batches of this launch: source batches b0, b0 + bstride, ...
    int32_t tile0;          // index of this graph's first tile
    int32_t by_degree;      // rows are in descending degree order (the hub tiers apply)
    int32_t b0;             // first source batch (a shard's rank; 0 unsharded)
    int32_t bstride;        // batch stride (a shard's world size; 1 unsharded)
    int32_t pad;
    const int32_t *split;   // relabelled graphs: [0] = G, vertices 0 .. G-1 form whole components, so
                            // no other vertex is connected to them (nullptr: G = n, no split)
};

struct TeamArgs {
    const GraphDesc *graphs;
    int32_t ngraphs;
    int32_t ntiles;
    int32_t nteams;
    int32_t push_alpha;
    int64_t maxn;               // per-team state stride in vertices
    uint64_t *state;            // [2 snapshots][nteams][maxn * W]
    uint8_t *quiet;             // [nteams][maxn]
    uint8_t *fresh;             // [nteams][maxn]
    uint8_t *pushed;            // [nteams][maxn]
    unsigned long long *ctr;    // [nteams][16]: 3 counter slots x {new bits, frontier edges, unfinished edges}
    uint32_t *bar;              // [nteams][32]: count, generation, ..., [8] current tile, [9] members
    uint32_t *sm_slots;         // [number of SMs]: blocks registered on each SM so far
    uint32_t *grid_bar;         // whole-grid barrier: count, generation
    int32_t nsm;                // SMs of the device
    int32_t per_sm;             // resident blocks per SM
    int32_t team_mix;           // 1: blocks sharing an SM join different teams; 0: the same team
    int32_t *queue;             // next tile to hand out
    int32_t *err;
    int32_t atomic_fr;          // several teams may update one graph's F/R
    unsigned long long *stats;
    uint64_t wait_ns;           // give-up time of every barrier wait
    int32_t phantom;            // tests: blocks every team barrier waits for in vain
    const int32_t *yield;       // preemption flag in mapped host memory (nullptr: none): while it is
                                // nonzero, teams take no new tile and the launch ends
};

// First vertex of a degree-descending vertex range 0 .. n-1 whose degree is below thr (binary search).
__device__ __forceinline__ int32_t first_below(const int64_t *__restrict__ rp, int32_t n, int64_t thr) {
    int32_t lo = 0, hi = n;
    while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        if (rp[mid + 1] - rp[mid] >= thr) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// One tile as seen by one block: the graph, the team's state, the block's place in the team.
struct Tile {
    const int64_t *__restrict__ rowptr;  // out-edges (push)
    const int32_t *__restrict__ col;
    const int64_t *__restrict__ prow;    // in-edges (pull)
    const int32_t *__restrict__ pcol;
    uint8_t *quiet;
    uint8_t *fresh;
    uint8_t *pushed;  // a top-down level ORed words into the vertex's next frontier words
    int32_t *err;     // device error word (debug builds report bad neighbour ids in it)
    uint64_t *F;
    uint32_t *R;
    unsigned long long *ctr;
    int32_t n;
    int32_t gend;   // vertices 0 .. gend-1 form whole components, disconnected from the rest
    int32_t hub_block_end;
    int32_t hub_warp_end;
    int32_t rank;   // block index within the team
    int32_t tsize;  // blocks in the team
    int32_t push_alpha;
    bool atomic_fr;
};

// Two snapshots per team: level l reads snapshot (l-1) mod 2 and writes snapshot l mod 2.
// Invariant: after level l, snapshot l mod 2 holds state_l(v) -- the sources within distance
// l of v -- for every vertex but the folded leaves (folded_leaf), whose words keep the start
// state: only their one neighbour reads them, and it has their bits from level 1. A vertex
// rewrites its words of the next snapshot only if it finds new bits at level l, or found some
// at level l-1 (then the next snapshot still holds state_{l-2}, which differs); otherwise they
// already hold state_{l-2} = state_{l-1} = state_l. fresh[v] marks the last level at which v
// found new bits. A vertex is "quiet" once both snapshots hold every bit (one level after its
// words became full): every later level of the batch skips it after reading one byte, and
// nobody pushes to it.
constexpr uint8_t QUIET = 1;  // quiet byte of a full vertex

__device__ __forceinline__ uint8_t level_mark(int level) { return (uint8_t)(1 + level % 255); }

// Vertices a warp takes from its team's work counter at a time, in passes of 32/T vertices (the
// bottom-up group tier caps a chunk at 32 vertices). Measured on GB300 (4 BA layers, n = 200,000):
// 8 passes, i.e. 32-vertex chunks at W = 16, 3% faster than 4.
#ifndef HOMLN_CHUNK_PASSES
#define HOMLN_CHUNK_PASSES 8
#endif
constexpr int kChunkPasses = HOMLN_CHUNK_PASSES;
#ifndef HOMLN_WORDS_PER_LANE
#define HOMLN_WORDS_PER_LANE 2
#endif

enum {
    ST_LEVELS, ST_PULL, ST_PUSH, ST_EDGES, ST_WORDS, ST_PUSHED, ST_BATCHES, ST_PUSHWORDS, ST_BYTES, ST_VISITS, ST_N
};

template <int W>
struct Geo {
    static constexpr int K = W >= HOMLN_WORDS_PER_LANE ? HOMLN_WORDS_PER_LANE : W;  // 64-bit words per lane
    static constexpr int T = W / K;           // lanes per vertex
};

template <int K>
__device__ __forceinline__ void ldw(const uint64_t *p, uint64_t (&x)[K]) {
    if constexpr (K == 4) {
        const ulonglong2 t0 = reinterpret_cast<const ulonglong2 *>(p)[0], t1 = reinterpret_cast<const ulonglong2 *>(p)[1];
        x[0] = t0.x;
        x[1] = t0.y;
        x[2] = t1.x;
        x[3] = t1.y;
    } else if constexpr (K == 2) {
        ulonglong2 t = *reinterpret_cast<const ulonglong2 *>(p);
        x[0] = t.x;
        x[1] = t.y;
    } else {
        x[0] = *p;
    }
}

template <int K>
__device__ __forceinline__ void stw(uint64_t *p, const uint64_t (&x)[K]) {
    if constexpr (K == 4) {
        reinterpret_cast<ulonglong2 *>(p)[0] = make_ulonglong2(x[0], x[1]);
        reinterpret_cast<ulonglong2 *>(p)[1] = make_ulonglong2(x[2], x[3]);
    } else if constexpr (K == 2) {
        *reinterpret_cast<ulonglong2 *>(p) = make_ulonglong2(x[0], x[1]);
    } else {
        *p = x[0];
    }
}

// Position of the k-th (0-based) set bit of m; k < popc(m). Chunk loops use it to hand the active
// vertices of a 32-vertex chunk to the lane groups without gaps.
__device__ __forceinline__ int nth_set(uint32_t m, int k) {
    int pos = 0;
#pragma unroll
    for (int w = 16; w > 0; w >>= 1) {
        const int c = __popc(m & ((1u << w) - 1u));
        if (k >= c) {
            k -= c;
            m >>= w;
            pos += w;
        }
    }
    return pos;
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

// Bounded barrier over the blocks of one team (all co-resident in a cooperative launch).
struct TeamBarrier {
    uint32_t *count;
    uint32_t *gen;
    int32_t *err;
    uint32_t size;
    uint64_t limit_ns;  // a waiter gives up after this long: DEV_TIMEOUT
};

__device__ __forceinline__ bool team_sync(const TeamBarrier &b) {
    const uint64_t limit_ns = b.limit_ns;
    if (b.size == 1) {
        __syncthreads();
        return *(volatile int32_t *)b.err == 0;
    }
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        uint32_t g = ld_acquire_u32(b.gen);
        __threadfence();
        uint32_t arrived = atomicAdd(b.count, 1u);
        if (arrived == b.size - 1) {
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

#ifndef HOMLN_GATHER_UNROLL
#define HOMLN_GATHER_UNROLL 4
#endif
#ifndef HOMLN_BFS_MAX_THREADS
#define HOMLN_BFS_MAX_THREADS 512
#endif
#ifndef HOMLN_BFS_MIN_BLOCKS
#define HOMLN_BFS_MIN_BLOCKS 2
#endif
#ifndef HOMLN_WARP_COORD
#define HOMLN_WARP_COORD 1
#endif
#ifndef HOMLN_WARP_TIER_ITERS
#define HOMLN_WARP_TIER_ITERS 8
#endif
#ifndef HOMLN_BLOCK_TIER_ITERS
#define HOMLN_BLOCK_TIER_ITERS 4
#endif
constexpr int kUnroll = HOMLN_GATHER_UNROLL;

// Leaves of undirected graphs are folded out of the BFS. A vertex v whose only neighbour p has
// other neighbours is one hop further than p from every other source, so over all sources
// F(v) = F(p) + R(p) - 1 and R(v) = R(p). Such a vertex is quiet from the start of every batch
// (never swept, gathered for or pushed to); its own source bit still reaches p on level 1, which
// pushes every source's bit to its neighbours. k_fold_leaves fills in F(v) and R(v) afterwards.
#ifndef HOMLN_FOLD_LEAVES
#define HOMLN_FOLD_LEAVES 1
#endif
__host__ __device__ __forceinline__ bool folded_leaf(const int64_t *rowptr, const int32_t *col, int64_t v) {
    const int64_t r = rowptr[v];
    if (rowptr[v + 1] - r != 1) return false;
    const int64_t p = col[r];
    return rowptr[p + 1] - rowptr[p] >= 2;
}

#ifndef HOMLN_DEBUG
#define HOMLN_DEBUG 0
#endif
// Debug builds (-DHOMLN_DEBUG=1) check every neighbour id before it is used: an id outside
// [0, n) records DEV_BAD_ID in the error word and the neighbour is treated as absent. Release
// builds compile the check away.
__device__ __forceinline__ bool id_ok(const Tile &a, int64_t u) {
    if (!HOMLN_DEBUG) return true;
    if (u >= 0 && u < a.n) return true;
    dev_fail(a.err, DEV_BAD_ID);
    return false;
}

// Column indices of the neighbours rb+p, rb+p+S, ... (kUnroll of them; -1 past the row end re).
__device__ __forceinline__ void load_cols(const Tile &a, int64_t j, int64_t re, int S, int32_t (&u)[kUnroll]) {
#pragma unroll
    for (int i = 0; i < kUnroll; ++i) u[i] = (j + (int64_t)i * S < re) ? __ldg(a.pcol + j + (int64_t)i * S) : -1;
}

// OR the frontier words (this lane's K of them) of neighbours rb+p, rb+p+S, ... into acc;
// stop once every bit this lane still needs is present. kUnroll neighbours are gathered per
// step (past the row end the loads are predicated off), and the column indices of the next
// step are loaded while the current frontier words are in flight. u holds the first step's
// column indices (load_cols(a, rb + p, re, S, u)), loaded by the caller so that they can be in
// flight before the caller knows whether the vertex needs any bit. Returns neighbours visited.
template <int W>
__device__ __forceinline__ int64_t gather_or(const Tile &a, const uint64_t *__restrict__ cur, int64_t rb, int64_t re,
                                             int p, int S, int q, int32_t (&u)[kUnroll],
                                             const uint64_t (&need)[Geo<W>::K], uint64_t (&acc)[Geo<W>::K]) {
    constexpr int K = Geo<W>::K, U = kUnroll;
    int64_t j = rb + p;
    if (j >= re) return 0;
    int64_t it = 0;
    while (true) {
        uint64_t f[U][K];
#pragma unroll
        for (int i = 0; i < U; ++i) {
            if (u[i] >= 0 && id_ok(a, u[i])) {
                ldw<K>(cur + (int64_t)u[i] * W + q * K, f[i]);
            } else {
#pragma unroll
                for (int k = 0; k < K; ++k) f[i][k] = 0;
            }
        }
        const int64_t jn = j + (int64_t)U * S;
        const bool more = jn < re;
        const int64_t here = (min(re, jn) - j + S - 1) / S;
        if (more) load_cols(a, jn, re, S, u);
#pragma unroll
        for (int i = 0; i < U; ++i)
#pragma unroll
            for (int k = 0; k < K; ++k) acc[k] |= f[i][k];
        it += here;
        if (covers<K>(acc, need)) return it;
        if (!more) return it;
        j = jn;
    }
}

// The warp-tier gather: the 32/T slots of one warp take every (32/T)-th neighbour of the
// same row; after each step their partial results are OR-ed across the warp, so all slots
// stop as soon as the row as a whole has supplied every missing bit (early exit for the whole
// row, not per slot). Every lane of the warp calls it. Returns the combined OR.
template <int W>
__device__ __forceinline__ int64_t gather_or_warp(const Tile &a, const uint64_t *__restrict__ cur, int64_t rb,
                                                  int64_t re, int q, const uint64_t (&need)[Geo<W>::K],
                                                  uint64_t (&acc)[Geo<W>::K]) {
    constexpr int K = Geo<W>::K, T = Geo<W>::T, S = 32 / T, U = kUnroll;
    const int p = (threadIdx.x & 31) / T;
    int64_t it = 0;
    for (int64_t j = rb + p; __any_sync(0xffffffffu, j < re); j += (int64_t)U * S) {
        uint64_t f[U][K];
#pragma unroll
        for (int i = 0; i < U; ++i) {
            const int64_t jj = j + (int64_t)i * S;
            const int32_t uj = jj < re ? __ldg(a.pcol + jj) : -1;
            if (jj < re && id_ok(a, uj)) {
                ldw<K>(cur + (int64_t)uj * W + q * K, f[i]);
                ++it;
            } else {
#pragma unroll
                for (int k = 0; k < K; ++k) f[i][k] = 0;
            }
        }
#pragma unroll
        for (int i = 0; i < U; ++i)
#pragma unroll
            for (int k = 0; k < K; ++k) acc[k] |= f[i][k];
#pragma unroll
        for (int o = T; o < 32; o <<= 1)
#pragma unroll
            for (int k = 0; k < K; ++k) acc[k] |= __shfl_xor_sync(0xffffffffu, acc[k], o);
        if (__all_sync(0xffffffffu, covers<K>(acc, need))) break;
    }
    return it;
}

struct PhaseCounters {
    unsigned long long newbits = 0, mf = 0, mu = 0;
};

// Block-reduce the phase counters and add them to the team's slot of this producing phase.
__device__ __forceinline__ void flush_counters(const Tile &a, PhaseCounters &c, uint32_t ps) {
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

__device__ __forceinline__ void reset_next_slot(const Tile &a, uint32_t ps) {
    if (a.rank == 0 && threadIdx.x == 0) {
        unsigned long long *slot = a.ctr + 4 * ((ps + 1) % 3);
        slot[0] = 0;
        slot[1] = 0;
        slot[2] = 0;
        slot[3] = 0;  // work counter of the next pull or push phase
    }
}

// Record the new bits nw of v (this lane's K words; s = its words in the previous snapshot)
// in the next snapshot nxt, and its counters. changed_last: v found new bits on the previous
// level, so its words in nxt are out of date and are rewritten even without new bits.
template <int W, bool STATS>
__device__ __forceinline__ void commit_vertex(const Tile &a, bool act, bool writer, int64_t v, int q,
                                              const uint64_t (&s)[Geo<W>::K], const uint64_t (&nw)[Geo<W>::K],
                                              uint64_t *nxt, int level, int64_t deg, bool changed_last,
                                              PhaseCounters &c, unsigned long long *st) {
    constexpr int K = Geo<W>::K, T = Geo<W>::T;
    bool any = false, full = true, sfull = true;
    uint32_t cnt = 0;
    uint64_t ns[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        ns[k] = s[k] | nw[k];
        any |= nw[k] != 0;
        full &= ns[k] == ~0ull;
        sfull &= s[k] == ~0ull;
        cnt += __popcll(nw[k]);
    }
    if (act && writer && (any || changed_last)) {
        stw<K>(nxt + v * W + q * K, ns);
        if (STATS) st[ST_BYTES] += 8 * K;
    }
    cnt = group_sum<T>(cnt);
    const bool gfull = !group_any<T>(!full);
    const bool gsfull = !group_any<T>(!sfull);
    if (act && writer && q == 0) {
        if (cnt) {
            if (a.atomic_fr) {
                atomicAdd(reinterpret_cast<unsigned long long *>(a.F + v), (unsigned long long)level * cnt);
                atomicAdd(a.R + v, cnt);
            } else {
                a.F[v] += (uint64_t)level * cnt;
                a.R[v] += cnt;
            }
            c.newbits += cnt;
            c.mf += (unsigned long long)deg;
            a.fresh[v] = level_mark(level);
            if (STATS) st[ST_BYTES] += 25;
        }
        if (!gfull) c.mu += (unsigned long long)deg;
        // full in the previous snapshot: the next one is full now too (rewritten above, as a vertex
        // becomes full on the level after its last new bits)
        if (gsfull) a.quiet[v] = QUIET;
        if (STATS) st[ST_VISITS] += 1;
    }
}

// ---------------------------------------------------------------- phases

// Level 0 of a batch: both snapshots = the bits of the sources that cannot reach the vertex (the
// padding bits of a short last batch; the batch's sources on the other side of the split at gend)
// and its own source bit; the per-vertex bytes 0, except that a vertex that
// no other source of the batch can reach (none on its side of the split, or no in-edges) is
// quiet from the start. The unreachable bits never arrive, so without them no vertex
// of a batch that mixes the two sides would ever become full.
template <int W, bool STATS>
__device__ void phase_start_batch(const Tile &a, uint64_t *s0buf, uint64_t *s1buf, int32_t s0, int32_t ns,
                                  unsigned long long *st) {
    constexpr int V = W >= 2 ? 2 : 1;  // words per store: 16-byte stores where a node has 2 or more
    const int64_t nthreads = (int64_t)a.tsize * blockDim.x;
    const int64_t gtid = (int64_t)a.rank * blockDim.x + threadIdx.x;
    // the batch's sources below the split are bits 0 .. split-1, the rest split .. ns-1
    const int32_t split = min(max(a.gend - s0, 0), ns);
    for (int64_t i = gtid * V; i < (int64_t)a.n * W; i += nthreads * V) {
        const int64_t v = i / W;
        const int wi0 = (int)(i % W);
        // bits c0 .. c1-1 of the batch can reach v; the rest are set
        const int32_t c0 = v < a.gend ? 0 : split, c1 = v < a.gend ? split : ns;
        const bool source = v >= s0 && v < (int64_t)s0 + ns;
        uint64_t x[V];
#pragma unroll
        for (int k = 0; k < V; ++k) {
            const int wi = wi0 + k, lo = wi * 64;
            const int32_t b0 = max(c0 - lo, 0), b1 = min(c1 - lo, 64);
            x[k] = ~0ull;
            if (b1 > b0) x[k] = ~((b1 - b0 == 64 ? ~0ull : ((1ull << (b1 - b0)) - 1)) << b0);
            if (source) {
                const int b = (int)(v - s0);
                if ((b >> 6) == wi) x[k] |= 1ull << (b & 63);
            }
        }
        if constexpr (V == 2) {  // both snapshots hold state_0
            *reinterpret_cast<ulonglong2 *>(s0buf + i) = make_ulonglong2(x[0], x[1]);
            *reinterpret_cast<ulonglong2 *>(s1buf + i) = make_ulonglong2(x[0], x[1]);
        } else {
            s0buf[i] = x[0];
            s1buf[i] = x[0];
        }
        if (wi0 == 0) {
            const bool lonely = c1 - c0 - (source ? 1 : 0) <= 0 || a.prow[v + 1] == a.prow[v];
            const bool leaf = HOMLN_FOLD_LEAVES && a.prow == a.rowptr && folded_leaf(a.prow, a.pcol, v);
            a.quiet[v] = lonely || leaf ? QUIET : 0;
            a.fresh[v] = 0;
            a.pushed[v] = 0;
        }
        if (STATS) st[ST_BYTES] += 16 * V + (wi0 == 0 ? 3 + 16 : 0);
    }
}

// Level 1, top-down: every source ORs its bit into its neighbours' words of snapshot 1 (which
// holds state_0, written by phase_start_batch before a team barrier).
template <int W, bool STATS>
__device__ void phase_start_push(const Tile &a, uint64_t *fa, int32_t s0, int32_t ns, unsigned long long *st) {
    const int64_t nthreads = (int64_t)a.tsize * blockDim.x;
    const int64_t gtid = (int64_t)a.rank * blockDim.x + threadIdx.x;
    const int64_t e0 = a.rowptr[s0], e1 = a.rowptr[s0 + ns];
    for (int64_t e = e0 + gtid; e < e1; e += nthreads) {
        int lo = 0, hi = ns;  // find the source row holding edge e
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (a.rowptr[s0 + mid] <= e) lo = mid; else hi = mid;
        }
        const int32_t u = __ldg(a.col + e);
        if (!id_ok(a, u)) continue;
        atomicOr(reinterpret_cast<unsigned long long *>(fa + (int64_t)u * W + (lo >> 6)), 1ull << (lo & 63));
        a.pushed[u] = 1;
        if (STATS) { st[ST_BYTES] += 4 + 8 + 1; st[ST_PUSHED] += 1; st[ST_PUSHWORDS] += 1; }
    }
}

// After a top-down level: of the words pushed into a vertex's words of the next snapshot (which
// held state_{l-2}), the bits it did not have after the previous level are its new bits. Warps
// sweep chunks of 32 consecutive vertices: one coalesced load of each per-vertex byte, then only
// the vertices that were pushed to or found bits on the previous level are processed (a top-down
// level has few). Every other live vertex has no new bits, keeps its words, and is not full (a
// full one would have turned quiet): it only adds its edges to the unfinished count.
template <int W, bool STATS>
__device__ void phase_finalize(const Tile &a, const uint64_t *__restrict__ prv, uint64_t *nxt, int level, uint32_t ps,
                               PhaseCounters &c, unsigned long long *st) {
    constexpr int K = Geo<W>::K, T = Geo<W>::T, per_pass = 32 / T;
    reset_next_slot(a, ps);
    const int lane = threadIdx.x & 31, q = lane % T;
    const int64_t gw = ((int64_t)a.rank * blockDim.x + threadIdx.x) >> 5;
    const int64_t NW = ((int64_t)a.tsize * blockDim.x) >> 5;
    const uint8_t last = level_mark(level - 1);
    for (int64_t v0 = gw * 32; v0 < a.n; v0 += NW * 32) {  // uniform over the warp
        const int cnt = (int)min((int64_t)32, (int64_t)a.n - v0);
        const int64_t vl = v0 + lane;
        int qv = QUIET, pv = 0, fv = 0;
        if (lane < cnt) {
            qv = a.quiet[vl];
            pv = a.pushed[vl];
            fv = a.fresh[vl];
            if (STATS) st[ST_BYTES] += 3;
        }
        const bool live = lane < cnt && qv < QUIET;
        const int flags = (pv ? 1 : 0) | (fv == last ? 2 : 0);
        const bool busy = live && flags != 0;
        if (live && !busy) {
            c.mu += (unsigned long long)(a.rowptr[vl + 1] - a.rowptr[vl]);
            if (STATS) st[ST_BYTES] += 16;
        }
        const uint32_t mask = __ballot_sync(0xffffffffu, busy);
        const int nb = __popc(mask);
        for (int pass = 0; pass * per_pass < nb; ++pass) {  // uniform over the warp
            const int slot = pass * per_pass + lane / T;
            const bool act = slot < nb;
            const int src = act ? nth_set(mask, slot) : 0;
            const int fl = __shfl_sync(0xffffffffu, flags, src);
            const int64_t v = v0 + src;
            const bool pushed = act && (fl & 1), chg = act && (fl & 2);
            uint64_t s[K], nw[K];
            int64_t deg = 0;
#pragma unroll
            for (int k = 0; k < K; ++k) s[k] = nw[k] = 0;
            if (act) {
                deg = a.rowptr[v + 1] - a.rowptr[v];
                ldw<K>(prv + v * W + q * K, s);
                if (STATS) st[ST_BYTES] += 8 * K + (q == 0 ? 16 : 0);
                if (pushed) {
                    uint64_t z[K];
                    ldw<K>(nxt + v * W + q * K, z);
#pragma unroll
                    for (int k = 0; k < K; ++k) nw[k] = z[k] & ~s[k];
                    if (STATS) st[ST_BYTES] += 8 * K;
                }
            }
            commit_vertex<W, STATS>(a, act, true, v, q, s, nw, nxt, level, deg, chg, c, st);
            // after the group's shuffles in commit_vertex: every lane of the group has read the flags
            if (pushed && q == 0) a.pushed[v] = 0;
        }
    }
    flush_counters(a, c, ps);
}

// Bottom-up level: each vertex still missing bits gathers its neighbours' frontier words.
template <int W, bool STATS>
__device__ void phase_pull(const Tile &a, const uint64_t *__restrict__ cur, uint64_t *nxt, int level, uint32_t ps,
                           PhaseCounters &c, unsigned long long *st) {
    // cur: the previous snapshot (read: the vertex's own words and its neighbours'); nxt: the next
    constexpr int K = Geo<W>::K, T = Geo<W>::T;
    reset_next_slot(a, ps);
    const uint8_t last = level_mark(level - 1);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int q = lane % T;

    // --- block tier: the largest hubs, all slots of the block share one row
    {
        __shared__ uint64_t red[32][16][Geo<W>::K];
        const int S = blockDim.x / T, p = threadIdx.x / T;
        for (int64_t v = a.rank; v < a.hub_block_end; v += a.tsize) {
            const uint8_t qv = a.quiet[v];
            if (STATS && threadIdx.x == 0) st[ST_BYTES] += 1;
            if (qv >= QUIET) continue;  // uniform over the block
            const bool chg = a.fresh[v] == last;  // read by every thread before warp 0 commits
            uint64_t s[K], need[K], acc[K];
            ldw<K>(cur + v * W + q * K, s);
            bool lane_need = false;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                need[k] = ~s[k];
                acc[k] = 0;
                lane_need |= need[k] != 0;
            }
            const int64_t rb = a.prow[v], re = a.prow[v + 1];
            int64_t it = 0;
            if (lane_need) {
                int32_t u[kUnroll];
                load_cols(a, rb + p, re, S, u);
                it = gather_or<W>(a, cur, rb, re, p, S, q, u, need, acc);
            }
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
                commit_vertex<W, STATS>(a, true, lane < T, v, q, s, nw, nxt, level, re - rb, chg, c, st);
            }
            __syncthreads();
        }
    }
    // --- warp tier: hubs below the block threshold, all slots of a warp share one row
    {
        const int p = lane / T;
#if !HOMLN_WARP_COORD
        const int S = 32 / T;
#endif
        const int64_t gw = ((int64_t)a.rank * blockDim.x + threadIdx.x) >> 5;
        const int64_t NW = ((int64_t)a.tsize * blockDim.x) >> 5;
        for (int64_t v = a.hub_block_end + gw; v < a.hub_warp_end; v += NW) {
            const uint8_t qv = a.quiet[v];
            if (STATS && lane == 0) st[ST_BYTES] += 1;
            if (qv >= QUIET) continue;  // uniform over the warp
            const bool chg = a.fresh[v] == last;
            uint64_t s[K], need[K], acc[K], nw[K];
            ldw<K>(cur + v * W + q * K, s);
            bool lane_need = false;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                need[k] = ~s[k];
                acc[k] = 0;
                lane_need |= need[k] != 0;
            }
            const bool full0 = !__any_sync(0xffffffffu, lane_need);
            const int64_t rb = a.prow[v], re = a.prow[v + 1];
            int64_t it = 0;
#if HOMLN_WARP_COORD
            if (!full0) it = gather_or_warp<W>(a, cur, rb, re, q, need, acc);
#else
            if (lane_need) {
                int32_t u[kUnroll];
                load_cols(a, rb + p, re, S, u);
                it = gather_or<W>(a, cur, rb, re, p, S, q, u, need, acc);
            }
#endif
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
            commit_vertex<W, STATS>(a, true, p == 0, v, q, s, nw, nxt, level, re - rb, chg, c, st);
        }
    }
    // --- group tier: T lanes per vertex. Warps take chunks of consecutive vertices from the
    // team's work counter, so a slow vertex (no early exit, long row) delays only its own chunk.
    // A chunk's row bounds and quiet and fresh bytes are read once, coalesced, and only its live
    // (non-quiet) vertices go to the passes, by shuffles; the warp's next chunk is reserved while
    // the current one runs. A pass then waits for one load (the vertex's words and its first
    // column indices, issued together) before its gathers, instead of three in a row.
    {
        unsigned long long *work = a.ctr + 4 * (ps % 3) + 3;
        constexpr int per_pass = 32 / T;
        constexpr int chunk = per_pass * kChunkPasses < 32 ? per_pass * kChunkPasses : 32;
        const int64_t nrest = a.n - a.hub_warp_end;
        long long next = 0;
        if (lane == 0) next = (long long)atomicAdd(work, (unsigned long long)chunk);
        for (;;) {
            const long long base = __shfl_sync(0xffffffffu, next, 0);
            if (base >= nrest) break;  // uniform over the warp
            if (lane == 0) next = (long long)atomicAdd(work, (unsigned long long)chunk);
            const int64_t v0 = a.hub_warp_end + base;
            const int cnt = (int)min((int64_t)chunk, (int64_t)(nrest - base));  // vertices of this chunk
            // lane i holds vertex v0+i's row bounds and its quiet and fresh bytes (i < cnt)
            const int64_t rb_l = a.prow[v0 + min(lane, cnt)];
            const int64_t re_l = a.prow[v0 + min(lane + 1, cnt)];
            // quiet byte | fresh byte << 8 of vertex v0+lane
            const int qf_l = lane < cnt ? (int)a.quiet[v0 + lane] | ((int)a.fresh[v0 + lane] << 8) : (int)QUIET;
            if (STATS && lane < cnt) st[ST_BYTES] += 2;
            // the chunk's live (non-quiet) vertices, handed to the lane groups without gaps
            const uint32_t live = __ballot_sync(0xffffffffu, lane < cnt && (qf_l & 0xff) < QUIET);
            const int nl = __popc(live);
            for (int pass = 0; pass * per_pass < nl; ++pass) {  // uniform over the warp
                const int slot = pass * per_pass + lane / T;
                const bool act = slot < nl;
                const int i = act ? nth_set(live, slot) : 0;
                const int64_t v = v0 + i;
                const int qf = __shfl_sync(0xffffffffu, qf_l, i);
                const bool chg = act && (qf >> 8) == (int)last;
                const int64_t rb0 = __shfl_sync(0xffffffffu, (long long)rb_l, i);
                const int64_t re0 = __shfl_sync(0xffffffffu, (long long)re_l, i);
                uint64_t s[K], need[K], acc[K], nw[K];
                int32_t u[kUnroll];
                bool lane_need = false;
                int64_t rb = 0, re = 0;
#pragma unroll
                for (int k = 0; k < K; ++k) s[k] = need[k] = acc[k] = 0;
                if (act) {
                    rb = rb0;
                    re = re0;
                    ldw<K>(cur + v * W + q * K, s);
                    load_cols(a, rb, re, 1, u);
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        need[k] = ~s[k];
                        lane_need |= need[k] != 0;
                    }
                }
                int64_t it = 0;
                if (lane_need) it = gather_or<W>(a, cur, rb, re, 0, 1, q, u, need, acc);
                if (STATS) {
                    st[ST_WORDS] += it * K;
                    st[ST_BYTES] += it * 8 * K;
                    int64_t gm = group_max<T>(it);
                    if (q == 0) { st[ST_EDGES] += gm; st[ST_BYTES] += 4 * gm; }
                    if (act) st[ST_BYTES] += 8 * K + (q == 0 ? 16 : 0);
                }
#pragma unroll
                for (int k = 0; k < K; ++k) nw[k] = acc[k] & need[k];
                commit_vertex<W, STATS>(a, act, true, v, q, s, nw, nxt, level, re - rb, chg, c, st);
            }
        }
    }
    flush_counters(a, c, ps);
}

// Top-down level: the vertices with new bits on the previous level OR their words of the previous
// snapshot into their neighbours' words of the next snapshot (quiet neighbours are full and are
// skipped). The whole words are pushed: bits a neighbour already has are masked by the sweep.
template <int W, bool STATS>
__device__ void phase_push(const Tile &a, const uint64_t *__restrict__ cur, uint64_t *nxt, int level, uint32_t ps,
                           unsigned long long *st) {
    constexpr int K = Geo<W>::K, T = Geo<W>::T;
    const int lane = threadIdx.x & 31;
    const int q = lane % T;
    auto push_row = [&](int64_t v, int p, int S, bool known) {
        if (!known && a.fresh[v] != level_mark(level - 1)) return;  // no new bits on the previous level
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
            if (!id_ok(a, u) || a.quiet[u] >= QUIET) continue;
#pragma unroll
            for (int k = 0; k < K; ++k)
                if (f[k]) {
                    atomicOr(reinterpret_cast<unsigned long long *>(nxt + u * W + q * K + k), f[k]);
                    if (STATS) { st[ST_PUSHWORDS] += 1; st[ST_BYTES] += 8; }
                }
            a.pushed[u] = 1;
            if (STATS) st[ST_BYTES] += 1;
        }
    };
    for (int64_t v = a.rank; v < a.hub_block_end; v += a.tsize) push_row(v, threadIdx.x / T, blockDim.x / T, false);
    const int64_t gw = ((int64_t)a.rank * blockDim.x + threadIdx.x) >> 5;
    const int64_t NW = ((int64_t)a.tsize * blockDim.x) >> 5;
    for (int64_t v = a.hub_block_end + gw; v < a.hub_warp_end; v += NW) push_row(v, lane / T, 32 / T, false);
    // group tier: chunks of 32 consecutive vertices from the team's work counter (this phase's slot,
    // cleared beforehand); one coalesced load of their fresh bytes finds the chunk's pushers, which
    // the lane groups then take without gaps
    unsigned long long *work = a.ctr + 4 * (ps % 3) + 3;
    constexpr int per_pass = 32 / T;
    const int64_t nrest = a.n - a.hub_warp_end;
    const uint8_t last = level_mark(level - 1);
    for (;;) {
        long long base = 0;
        if (lane == 0) base = (long long)atomicAdd(work, 32ull);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= nrest) break;  // uniform over the warp
        const int64_t v0 = a.hub_warp_end + base;
        const int cnt = (int)min((int64_t)32, (int64_t)(nrest - base));
        const bool pusher = lane < cnt && a.fresh[v0 + lane] == last;
        if (STATS && lane < cnt) st[ST_BYTES] += 1;
        const uint32_t mask = __ballot_sync(0xffffffffu, pusher);
        const int np = __popc(mask);
        for (int pass = 0; pass * per_pass < np; ++pass) {
            const int slot = pass * per_pass + lane / T;
            if (slot < np) push_row(v0 + nth_set(mask, slot), 0, 1, true);
        }
    }
}

// The levels of one batch (sources s0 .. s0+ns-1) of one graph, run by one team.
// Returns false if a barrier gave up (the kernel must stop).
template <int W, bool STATS>
__device__ bool run_batch(const Tile &a, uint64_t *sa, uint64_t *sb, const TeamBarrier &tb, int32_t s0, int32_t ns,
                          uint32_t &ps, PhaseCounters &c, unsigned long long *st) {
    phase_start_batch<W, STATS>(a, sa, sb, s0, ns, st);
    if (!team_sync(tb)) return false;
    phase_start_push<W, STATS>(a, sb, s0, ns, st);
    if (!team_sync(tb)) return false;
    phase_finalize<W, STATS>(a, sa, sb, 1, ps, c, st);
    ++ps;
    if (!team_sync(tb)) return false;
    uint64_t *cur = sb, *nxt = sa;  // level l reads snapshot (l-1) mod 2, writes l mod 2
    if (STATS) { st[ST_BATCHES] += 1; st[ST_LEVELS] += 1; st[ST_PUSH] += 1; }
    for (int level = 2; level <= a.n + 1; ++level) {
        const unsigned long long *slot = a.ctr + 4 * ((ps - 1) % 3);
        const unsigned long long newbits = __ldcg(slot), mf = __ldcg(slot + 1), mu = __ldcg(slot + 2);
        // done when the last level found nothing, or (undirected) when every vertex that can still
        // change is full: no unfinished edges, and a vertex without edges gets no bits. Later levels
        // would add no bit, and the snapshots need not be brought level once the batch ends. (A
        // directed level counts unfinished edges by out-degree after a top-down level, which says
        // nothing about in-edges.)
        if (newbits == 0 || (mu == 0 && a.prow == a.rowptr)) break;
        const bool push = (unsigned long long)a.push_alpha * mf < mu;
        if (push) {
            phase_push<W, STATS>(a, cur, nxt, level, ps, st);
            if (!team_sync(tb)) return false;
            phase_finalize<W, STATS>(a, cur, nxt, level, ps, c, st);
        } else {
            phase_pull<W, STATS>(a, cur, nxt, level, ps, c, st);
        }
        ++ps;
        if (!team_sync(tb)) return false;
        if (STATS) { st[ST_LEVELS] += 1; st[push ? ST_PUSH : ST_PULL] += 1; }
        uint64_t *t = cur; cur = nxt; nxt = t;
    }
    return true;
}

__device__ __forceinline__ uint32_t sm_id() {
    uint32_t id;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(id));
    return id;
}

template <int W, bool STATS>
__global__ void __launch_bounds__(HOMLN_BFS_MAX_THREADS, HOMLN_BFS_MIN_BLOCKS) k_msbfs(TeamArgs A) {
    PhaseCounters c;
    unsigned long long st[ST_N];
#pragma unroll
    for (int i = 0; i < ST_N; ++i) st[i] = 0;
    // Join a team by SM. By default the blocks that share an SM join the same team (they
    // then share its L1 for the team's frontier gathers: faster on the 50,000-node
    // power-law workload); with team_mix they join different teams instead.
    __shared__ int s_team, s_rank;
    if (threadIdx.x == 0) {
        const uint32_t sm = sm_id() % (uint32_t)A.nsm;
        const uint32_t slot = atomicAdd(A.sm_slots + sm, 1u);
        const uint32_t spread = !A.team_mix ? 0u : A.nteams >= A.per_sm ? (uint32_t)(A.nteams / A.per_sm) : 1u;
        const int tm = (int)((sm + slot * spread) % (uint32_t)A.nteams);
        s_team = tm;
        s_rank = (int)atomicAdd(A.bar + (size_t)tm * 32 + 9, 1u);
    }
    {
        const TeamBarrier all{A.grid_bar, A.grid_bar + 1, A.err, gridDim.x, A.wait_ns};
        if (!team_sync(all)) return;
    }
    const int team = s_team;
    const int rank = s_rank;
    uint32_t *tbar = A.bar + (size_t)team * 32;
    const int tsize = (int)*(volatile uint32_t *)(tbar + 9);
    // (test_phantom_blocks: the barrier also counts blocks that never arrive, so it runs out)
    const TeamBarrier tb{tbar, tbar + 1, A.err, (uint32_t)(tsize + A.phantom), A.wait_ns};
    const size_t stride = (size_t)A.maxn * W;
    const size_t arr = stride * A.nteams;
    uint64_t *sa = A.state + 0 * arr + team * stride;  // snapshot 0
    uint64_t *sb = A.state + 1 * arr + team * stride;  // snapshot 1
    uint8_t *quiet = A.quiet + (size_t)team * A.maxn;
    uint8_t *fresh = A.fresh + (size_t)team * A.maxn;
    uint8_t *pushed = A.pushed + (size_t)team * A.maxn;
    unsigned long long *ctr = A.ctr + (size_t)team * 16;
    volatile int32_t *tile_slot = reinterpret_cast<volatile int32_t *>(tbar + 8);
    uint32_t ps = 0;
    bool ok = true;
    while (ok) {
        if (rank == 0 && threadIdx.x == 0) {
            // a raised yield flag ends the launch before the next tile is taken, so every tile handed
            // out is finished and the queue counter tells the host where to resume
            if (A.yield && *reinterpret_cast<const volatile int32_t *>(A.yield) != 0) *tile_slot = A.ntiles;
            else *tile_slot = atomicAdd(A.queue, 1);
        }
        if (!team_sync(tb)) break;
        const int32_t t = *tile_slot;
        if (t >= A.ntiles) break;
        int lo = 0, hi = A.ngraphs;  // the graph whose tiles contain t
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (A.graphs[mid].tile0 <= t) lo = mid; else hi = mid;
        }
        const GraphDesc &g = A.graphs[lo];
        Tile a;
        a.rowptr = g.rowptr;
        a.col = g.col;
        a.prow = g.prow;
        a.pcol = g.pcol;
        a.quiet = quiet;
        a.fresh = fresh;
        a.pushed = pushed;
        a.err = A.err;
        a.F = g.F;
        a.R = g.R;
        a.ctr = ctr;
        a.n = g.n;
        // hub tiers: rows of at least HOMLN_BLOCK_TIER_ITERS (4) iterations per slot of a block go
        // to a whole block, the rest with at least HOMLN_WARP_TIER_ITERS (8) per slot of a warp to
        // a whole warp (measured on GB300: warp threshold 8 beat 2, 4, 12, 16 and 32)
        a.gend = g.split ? min(max(*g.split, 0), g.n) : g.n;
        a.hub_block_end =
            g.by_degree ? first_below(g.prow, a.gend, HOMLN_BLOCK_TIER_ITERS * (int64_t)(blockDim.x / Geo<W>::T)) : 0;
        a.hub_warp_end = g.by_degree
                             ? max(a.hub_block_end, first_below(g.prow, a.gend, HOMLN_WARP_TIER_ITERS * (32 / Geo<W>::T)))
                             : 0;
        a.rank = rank;
        a.tsize = tsize;
        a.push_alpha = A.push_alpha;
        a.atomic_fr = A.atomic_fr != 0;
        const int32_t b = g.b0 + (t - g.tile0) * g.bstride;
        const int32_t s0 = b * 64 * W;
        const int32_t ns = min(64 * W, g.n - s0);
        ok = run_batch<W, STATS>(a, sa, sb, tb, s0, ns, ps, c, st);
    }
    if (STATS && A.stats) {
        if (threadIdx.x == 0 && rank == 0) {
            atomicAdd(A.stats + ST_LEVELS, st[ST_LEVELS]);
            atomicAdd(A.stats + ST_PULL, st[ST_PULL]);
            atomicAdd(A.stats + ST_PUSH, st[ST_PUSH]);
            atomicAdd(A.stats + ST_BATCHES, st[ST_BATCHES]);
        }
        atomicAdd(A.stats + ST_EDGES, st[ST_EDGES]);
        atomicAdd(A.stats + ST_WORDS, st[ST_WORDS]);
        atomicAdd(A.stats + ST_PUSHED, st[ST_PUSHED]);
        atomicAdd(A.stats + ST_PUSHWORDS, st[ST_PUSHWORDS]);
        atomicAdd(A.stats + ST_BYTES, st[ST_BYTES]);
        atomicAdd(A.stats + ST_VISITS, st[ST_VISITS]);
    }
}

// One phase of one graph as an ordinary (non-cooperative) launch: the plain schedule, in
// which the host drives the levels and kernel boundaries replace the team barrier.
enum PhaseKind { PH_START = 0, PH_FINALIZE = 1, PH_PULL = 2, PH_PUSH = 3, PH_START_PUSH = 4 };

template <int W, bool STATS>
__global__ void __launch_bounds__(HOMLN_BFS_MAX_THREADS, HOMLN_BFS_MIN_BLOCKS) k_phase(TeamArgs A, int32_t gi, int32_t kind, int32_t s0, int32_t ns,
                                                  int32_t level, uint32_t ps, int32_t cur_is_a) {
    PhaseCounters c;
    unsigned long long st[ST_N];
#pragma unroll
    for (int i = 0; i < ST_N; ++i) st[i] = 0;
    const GraphDesc &g = A.graphs[gi];
    const size_t arr = (size_t)A.maxn * W;
    uint64_t *sa = A.state, *sb = A.state + arr;
    Tile a;
    a.rowptr = g.rowptr;
    a.col = g.col;
    a.prow = g.prow;
    a.pcol = g.pcol;
    a.quiet = A.quiet;
    a.fresh = A.fresh;
    a.pushed = A.pushed;
    a.err = A.err;
    a.F = g.F;
    a.R = g.R;
    a.ctr = A.ctr;
    a.n = g.n;
    a.gend = g.split ? min(max(*g.split, 0), g.n) : g.n;
    a.hub_block_end =
            g.by_degree ? first_below(g.prow, a.gend, HOMLN_BLOCK_TIER_ITERS * (int64_t)(blockDim.x / Geo<W>::T)) : 0;
    a.hub_warp_end = g.by_degree
                         ? max(a.hub_block_end, first_below(g.prow, a.gend, HOMLN_WARP_TIER_ITERS * (32 / Geo<W>::T)))
                         : 0;
    a.rank = blockIdx.x;
    a.tsize = gridDim.x;
    a.push_alpha = A.push_alpha;
    a.atomic_fr = false;
    // level 1 (cur_is_a = 0) reads snapshot 0 and writes snapshot 1; the host alternates after
    uint64_t *cur = cur_is_a ? sb : sa, *nxt = cur_is_a ? sa : sb;
    switch (kind) {
    case PH_START: phase_start_batch<W, STATS>(a, sa, sb, s0, ns, st); break;
    case PH_START_PUSH: phase_start_push<W, STATS>(a, sb, s0, ns, st); break;
    case PH_FINALIZE: phase_finalize<W, STATS>(a, cur, nxt, level, ps, c, st); break;
    case PH_PULL: phase_pull<W, STATS>(a, cur, nxt, level, ps, c, st); break;
    default: phase_push<W, STATS>(a, cur, nxt, level, ps, st); break;
    }
    if (STATS && A.stats) {
        if (threadIdx.x == 0 && blockIdx.x == 0) {
            if (kind == PH_START) { atomicAdd(A.stats + ST_BATCHES, 1ull); }
            if (kind == PH_PULL) { atomicAdd(A.stats + ST_LEVELS, 1ull); atomicAdd(A.stats + ST_PULL, 1ull); }
            if (kind == PH_FINALIZE) { atomicAdd(A.stats + ST_LEVELS, 1ull); atomicAdd(A.stats + ST_PUSH, 1ull); }
        }
        atomicAdd(A.stats + ST_EDGES, st[ST_EDGES]);
        atomicAdd(A.stats + ST_WORDS, st[ST_WORDS]);
        atomicAdd(A.stats + ST_PUSHED, st[ST_PUSHED]);
        atomicAdd(A.stats + ST_PUSHWORDS, st[ST_PUSHWORDS]);
        atomicAdd(A.stats + ST_BYTES, st[ST_BYTES]);
        atomicAdd(A.stats + ST_VISITS, st[ST_VISITS]);
    }
}

typedef void (*PhaseKernel)(TeamArgs, int32_t, int32_t, int32_t, int32_t, int32_t, uint32_t, int32_t);

template <int W>
PhaseKernel pick_phase(bool stats) {
    return stats ? k_phase<W, true> : k_phase<W, false>;
}

PhaseKernel phase_kernel_for(int W, bool stats) {
    switch (W) {
    case 1: return pick_phase<1>(stats);
    case 2: return pick_phase<2>(stats);
    case 4: return pick_phase<4>(stats);
    case 8: return pick_phase<8>(stats);
    case 16: return pick_phase<16>(stats);
    case 32: return pick_phase<32>(stats);
    default: fail(HOMLN_EINVAL, "words_per_node must be 1, 2, 4, 8, 16 or 32");
    }
}

__global__ void k_set_i32(int32_t *p, int32_t v) { *p = v; }

// Farness and reach of the folded leaves (see folded_leaf), from their neighbour's. A shard (source
// batches b0, b0 + bstride, ... of spb sources) holds partial sums over its own sources S, and the
// sums over shards must add up: over S, F_S(v) = F_S(p) + R_S(p) + [p in S] - 2 [v in S] and
// R_S(v) = R_S(p) + [p in S] - [v in S] (with one shard of everything: F(p) + R(p) - 1, R(p)).
__global__ void k_fold_leaves(int32_t n, const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                              uint64_t *F, uint32_t *R, int32_t spb, int32_t b0, int32_t bstride) {
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        if (!folded_leaf(rowptr, col, v)) continue;
        const int32_t p = col[rowptr[v]];
        auto in_shard = [&](int32_t x) {
            const int32_t b = x / spb;
            return b >= b0 && (b - b0) % bstride == 0 ? 1u : 0u;
        };
        const uint32_t ip = in_shard(p), iv = in_shard(v);
        F[v] = F[p] + R[p] + ip - 2ull * iv;
        R[v] = R[p] + ip - iv;
    }
}

__global__ void k_scatter_back(int32_t n, const int32_t *__restrict__ perm, const uint64_t *__restrict__ Fi,
                               const uint32_t *__restrict__ Ri, uint64_t *__restrict__ F, uint32_t *__restrict__ R) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        F[perm[i]] = Fi[i];
        R[perm[i]] = Ri[i];
    }
}

typedef void (*BfsKernel)(TeamArgs);

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

// Widest tile: one team's state (2 snapshots of n x W words) stays within this many bytes.
constexpr double kWordsBudget = 104.0e6;
// Default teams: as many as keep the state of all teams near kTeamState bytes (about twice
// L2), at least kDefaultTeams, and never more state than kStateCap bytes. Measured on GB300
// (W = 8, 304 blocks): 24-25 teams at n = 50,000 (power-law: 16 teams 1.3% slower, 12 teams 4%,
// 32 teams 1%), 16 at n = 200,000 (BA: 8-16 equal, 2 teams 24% slower), and for many graphs
// of n <= 20,000 in one launch 60-76 teams (16 teams: 43% slower). The frontier gathers of
// more teams than fit L2 still hit L2 mostly, and smaller teams meet at their barriers sooner.
constexpr int kDefaultTeams = 16;
constexpr double kTeamState = 2.4e8;
constexpr double kStateCap = 2.0e9;

}  // namespace

int msbfs_pick_words(int32_t n) {
    int W = 32;
    while (W > 1 && 2.0 * n * 8.0 * W > kWordsBudget) W >>= 1;
    while (W > 1 && (int64_t)64 * (W / 2) >= n) W >>= 1;  // no wider than the node count needs
    return W;
}

// Everything one BFS over a job list needs, allocated once: the graph descriptors, the
// relabelled graphs' F/R scratch and the teams' state. bfs_plan_run enqueues one complete
// analysis (zeroing, launches, scatter-back) without allocating or copying from the host, so
// it can be captured in a CUDA graph and replayed.
struct BfsPlan {
    std::vector<BfsJob> jobs;
    BfsTuning t;
    bool plain = false, stats = false;
    int W = 8, nteams = 1, threads = 512, grid = 0, nsm = 0, per_sm = 0;
    BfsKernel kern = nullptr;
    PhaseKernel pkern = nullptr;
    std::vector<GraphDesc> desc;
    int32_t tiles = 0, maxn = 0;
    std::vector<DBuf<uint64_t>> Fi;
    std::vector<DBuf<uint32_t>> Ri;
    DBuf<uint64_t> state;
    DBuf<uint8_t> quiet;
    DBuf<unsigned long long> ctr, st;
    DBuf<uint32_t> barmem;
    DBuf<int32_t> queue;
    DBuf<GraphDesc> d_desc;
    size_t bar_words = 0;
    TeamArgs A{};
};

BfsPlan *bfs_plan_create(const std::vector<BfsJob> &jobs, const BfsTuning &t, int32_t *d_err, Alloc *al,
                         cudaStream_t s, bool stats) {
    if (jobs.empty()) return nullptr;
    int32_t maxn = 0;
    for (const BfsJob &j : jobs) maxn = std::max(maxn, j.g->csr.n);
    if (maxn <= 0) return nullptr;
    const int threads = t.threads > 0 ? t.threads : 512;
    if (threads % 32 != 0 || threads > 512 || threads < 64) fail(HOMLN_EINVAL, "threads must be 64..512, multiple of 32");
    std::unique_ptr<BfsPlan> p(new BfsPlan);
    p->jobs = jobs;
    p->t = t;
    p->stats = stats;
    p->threads = threads;
    p->maxn = maxn;
    const bool plain = p->plain = t.schedule == 1;
    // teams and words per node: every team keeps its own state, and all of it should fit the budget
    // Defaults, measured on GB300: 8 words per node (512 sources per tile); teams as above.
    // The plain schedule (one team, the host driving every level) takes the widest tile the
    // budget allows, which needs the fewest launches and host round trips.
    const int W = p->W = t.W > 0 ? t.W : plain ? msbfs_pick_words(maxn) : std::min(8, msbfs_pick_words(maxn));
    int nteams = 1;
    if (!plain) {
        if (t.teams > 0) {
            nteams = t.teams;
        } else {
            const double per_team = 2.0 * maxn * 8.0 * W;  // bytes of one team's state
            nteams = std::max(kDefaultTeams, (int)std::floor(kTeamState / per_team));
            nteams = std::max(1, std::min(nteams, (int)std::floor(kStateCap / per_team)));
            int64_t tiles = 0;  // no more teams than tiles
            for (const BfsJob &j : jobs) tiles += ceil_div(j.g->csr.n, 64 * W);
            tiles = ceil_div(tiles, (int64_t)std::max(1, t.shard_world));
            if (tiles < nteams) nteams = (int)std::max<int64_t>(tiles, 1);
        }
    }
    p->kern = kernel_for(W, stats);
    int dev = 0, nsm = 0, coop = 0, per_sm = 0;
    HCUDA(cudaGetDevice(&dev));
    HCUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    HCUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    if (!coop) fail(HOMLN_ECUDA, "device does not support cooperative launch");
    p->pkern = plain ? phase_kernel_for(W, stats) : nullptr;
    HCUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, p->kern, threads, 0));
    if (per_sm < 1) fail(HOMLN_ECUDA, "bfs kernel does not fit on an SM");
    if (t.blocks_per_sm > 0 && t.blocks_per_sm < per_sm) per_sm = t.blocks_per_sm;
    // sm_count: a grid for that many SMs' worth of blocks leaves the rest of the GPU to other streams
    const int use_sm = t.sm_count > 0 ? std::min(nsm, t.sm_count) : nsm;
    const int grid = p->grid = use_sm * per_sm;
    if (nteams > grid) nteams = grid;
    p->nteams = nteams;
    p->nsm = nsm;
    p->per_sm = per_sm;

    // graph descriptors; relabelled graphs accumulate into scratch and are scattered back after
    const size_t ng = jobs.size();
    p->Fi.resize(ng);
    p->Ri.resize(ng);
    p->desc.resize(ng);
    int32_t tile = 0;
    for (size_t i = 0; i < ng; ++i) {
        const BfsGraph &G = *jobs[i].g;
        GraphDesc &d = p->desc[i];
        d.n = G.csr.n;
        // a shard (rank r of world w) takes the source batches r, r + w, r + 2w, ...
        const int32_t all = (int32_t)ceil_div(d.n, 64 * W);
        d.b0 = t.shard_rank;
        d.bstride = t.shard_world;
        d.nbatches = all > t.shard_rank ? (all - t.shard_rank + t.shard_world - 1) / t.shard_world : 0;
        d.tile0 = tile;
        tile += d.nbatches;
        d.by_degree = G.relabeled ? 1 : 0;
        d.rowptr = G.csr.rowptr.p;
        d.col = G.csr.col.p;
        d.prow = G.directed ? G.csr_in.rowptr.p : G.csr.rowptr.p;
        d.pcol = G.directed ? G.csr_in.col.p : G.csr.col.p;
        d.split = G.relabeled ? G.split.p : nullptr;
        d.pad = 0;
        if (G.relabeled) {
            if (!p->Fi[i].alloc(al, d.n) || !p->Ri[i].alloc(al, d.n)) fail(HOMLN_ENOMEM, "bfs relabelled outputs");
            d.F = p->Fi[i].p;
            d.R = p->Ri[i].p;
        } else {
            d.F = jobs[i].F;
            d.R = jobs[i].R;
        }
    }
    p->tiles = tile;

    const size_t words = (size_t)maxn * W * nteams;
    p->bar_words = 32 * (size_t)nteams + 32 + (size_t)nsm;  // team barriers, grid barrier, SM slots
    if (!p->state.alloc(al, 2 * words) || !p->quiet.alloc(al, 3 * (size_t)maxn * nteams) ||
        !p->ctr.alloc(al, 16 * nteams) || !p->barmem.alloc(al, p->bar_words) || !p->queue.alloc(al, 1) ||
        !p->d_desc.alloc(al, ng))
        fail(HOMLN_ENOMEM, "bfs state");
    if (stats && !p->st.alloc(al, ST_N)) fail(HOMLN_ENOMEM, "bfs stats");
    HCUDA(cudaMemcpyAsync(p->d_desc.p, p->desc.data(), ng * sizeof(GraphDesc), cudaMemcpyHostToDevice, s));

    TeamArgs &A = p->A;
    A.graphs = p->d_desc.p;
    A.ngraphs = (int32_t)ng;
    A.ntiles = tile;
    A.nteams = nteams;
    A.push_alpha = t.push_alpha > 0 ? t.push_alpha : 16;
    A.maxn = maxn;
    A.state = p->state.p;
    A.quiet = p->quiet.p;
    A.fresh = p->quiet.p + (size_t)maxn * nteams;
    A.pushed = p->quiet.p + 2 * (size_t)maxn * nteams;
    A.ctr = p->ctr.p;
    A.bar = p->barmem.p;
    A.grid_bar = p->barmem.p + 32 * (size_t)nteams;
    A.sm_slots = p->barmem.p + 32 * (size_t)nteams + 32;
    A.nsm = nsm;
    A.per_sm = per_sm;
    A.team_mix = t.team_mix;
    A.queue = p->queue.p;
    A.err = d_err;
    A.atomic_fr = nteams > 1 ? 1 : 0;
    A.stats = stats ? p->st.p : nullptr;
    A.wait_ns = (uint64_t)t.wait_limit_ms * 1000000ull;
    A.phantom = t.phantom;
    A.yield = plain ? nullptr : t.yield_dev;
    return p.release();
}

void bfs_plan_destroy(BfsPlan *p) { delete p; }

bool bfs_plan_capturable(const BfsPlan *p) { return p && !p->plain && !p->stats && !p->A.yield; }

// Host side of a yield: block until the flag is 0 again (bounded: HOMLN_ETIMEOUT after 60 s).
static void wait_yield_cleared(const BfsTuning &t) {
    const auto t0 = std::chrono::steady_clock::now();
    while (*t.yield_host != 0) {
        if (std::chrono::steady_clock::now() - t0 > std::chrono::seconds(60))
            fail(HOMLN_ETIMEOUT, "the yield flag stayed raised for 60 s");
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

void bfs_plan_run(BfsPlan *p, cudaStream_t s, cudaEvent_t ev_start, cudaEvent_t ev_stop) {
    if (!p) return;
    const size_t ng = p->jobs.size();
    const int32_t tile = p->tiles;
    const int W = p->W, grid = p->grid, threads = p->threads, nteams = p->nteams;
    for (size_t i = 0; i < ng; ++i) {
        HCUDA(cudaMemsetAsync(p->desc[i].F, 0, (size_t)p->desc[i].n * sizeof(uint64_t), s));
        HCUDA(cudaMemsetAsync(p->desc[i].R, 0, (size_t)p->desc[i].n * sizeof(uint32_t), s));
    }
    HCUDA(cudaMemsetAsync(p->ctr.p, 0, 16 * nteams * sizeof(unsigned long long), s));
    HCUDA(cudaMemsetAsync(p->barmem.p, 0, p->bar_words * sizeof(uint32_t), s));
    HCUDA(cudaMemsetAsync(p->queue.p, 0, sizeof(int32_t), s));
    if (p->stats) HCUDA(cudaMemsetAsync(p->st.p, 0, ST_N * sizeof(unsigned long long), s));
    TeamArgs A = p->A;
    void *args[] = {&A};
    if (ev_start) HCUDA(cudaEventRecord(ev_start, s));
    if (!p->plain) {
        // max_tiles: the tiles go out in several launches of at most that many, so that work of
        // other streams (a higher-priority one, say) can run in between. With a yield flag, a
        // launch that stopped early (the flag was raised) is resumed from the queue counter once
        // the flag is 0 again; the host waits for each launch to end to read the counter.
        const int32_t chunk = p->t.max_tiles > 0 ? p->t.max_tiles : tile;
        int32_t c0 = 0;
        bool first = true;
        while (c0 < tile) {
            if (!first) {  // fresh barriers, counters and team formation; the queue resumes at c0
                HCUDA(cudaMemsetAsync(p->ctr.p, 0, 16 * nteams * sizeof(unsigned long long), s));
                HCUDA(cudaMemsetAsync(p->barmem.p, 0, p->bar_words * sizeof(uint32_t), s));
                launch(k_set_i32, 1, 1, 0, s, p->queue.p, c0);
            }
            first = false;
            A.ntiles = (int32_t)std::min<int64_t>(tile, (int64_t)c0 + chunk);
            g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
            HCUDA(cudaLaunchCooperativeKernel((const void *)p->kern, dim3(grid), dim3(threads), args, 0, s));
            if (A.yield) {
                int32_t handed = 0;  // tiles handed out, all of them finished
                HCUDA(cudaMemcpyAsync(&handed, p->queue.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
                HCUDA(cudaStreamSynchronize(s));
                if (handed < A.ntiles) {
                    if (p->t.yield_count) p->t.yield_count->fetch_add(1, std::memory_order_relaxed);
                    wait_yield_cleared(p->t);
                    c0 = std::max(c0, handed);
                    continue;
                }
            }
            c0 = A.ntiles;
        }
    } else {
        // plain schedule: one launch per phase, the host reads the level counters after every level
        const PhaseKernel pkern = p->pkern;
        uint32_t ps = 0;
        for (size_t gi = 0; gi < ng; ++gi) {
            for (int32_t bi = 0; bi < p->desc[gi].nbatches; ++bi) {
                const int32_t b = p->desc[gi].b0 + bi * p->desc[gi].bstride;
                const int32_t s0 = b * 64 * W, ns = std::min(64 * W, p->desc[gi].n - s0);
                launch(pkern, grid, threads, 0, s, A, (int32_t)gi, (int32_t)PH_START, s0, ns, 0, ps, 0);
                launch(pkern, grid, threads, 0, s, A, (int32_t)gi, (int32_t)PH_START_PUSH, s0, ns, 0, ps, 0);
                launch(pkern, grid, threads, 0, s, A, (int32_t)gi, (int32_t)PH_FINALIZE, s0, ns, 1, ps, 0);
                ++ps;
                int32_t cur_a = 1;
                for (int32_t level = 2; level <= p->desc[gi].n + 1; ++level) {
                    unsigned long long h3[3];
                    HCUDA(cudaMemcpyAsync(h3, p->ctr.p + 4 * ((ps - 1) % 3), sizeof(h3), cudaMemcpyDeviceToHost, s));
                    HCUDA(cudaStreamSynchronize(s));
                    if (h3[0] == 0 || (h3[2] == 0 && !p->jobs[gi].g->directed)) break;
                    if ((unsigned long long)A.push_alpha * h3[1] < h3[2]) {
                        launch(pkern, grid, threads, 0, s, A, (int32_t)gi, (int32_t)PH_PUSH, s0, ns, level, ps, cur_a);
                        launch(pkern, grid, threads, 0, s, A, (int32_t)gi, (int32_t)PH_FINALIZE, s0, ns, level, ps,
                               cur_a);
                    } else {
                        launch(pkern, grid, threads, 0, s, A, (int32_t)gi, (int32_t)PH_PULL, s0, ns, level, ps, cur_a);
                    }
                    ++ps;
                    cur_a ^= 1;
                }
            }
        }
    }
    if (ev_stop) HCUDA(cudaEventRecord(ev_stop, s));
    if (HOMLN_FOLD_LEAVES)
        for (size_t i = 0; i < ng; ++i) {
            const GraphDesc &d = p->desc[i];
            if (d.prow == d.rowptr && d.n > 0)
                launch(k_fold_leaves, (unsigned)std::min<int64_t>(ceil_div(d.n, 256), 4096), 256, 0, s, d.n, d.prow,
                       d.pcol, d.F, d.R, 64 * W, d.b0, d.bstride);
        }
    for (size_t i = 0; i < ng; ++i)
        if (p->jobs[i].g->relabeled)
            launch(k_scatter_back, (unsigned)ceil_div(p->desc[i].n, 256), 256, 0, s, p->desc[i].n,
                   p->jobs[i].g->perm.p, (const uint64_t *)p->Fi[i].p, (const uint32_t *)p->Ri[i].p, p->jobs[i].F,
                   p->jobs[i].R);
    HCUDA(cudaGetLastError());
}

void bfs_plan_stats(BfsPlan *p, BfsStats *stats, cudaStream_t s) {
    if (!p || !p->stats || !stats) return;
    unsigned long long h[ST_N];
    HCUDA(cudaMemcpyAsync(h, p->st.p, sizeof(h), cudaMemcpyDeviceToHost, s));
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
    stats->words_per_node = p->W;
    stats->teams = p->nteams;
}

void msbfs_multi(const std::vector<BfsJob> &jobs, const BfsTuning &t, int32_t *d_err, Alloc *al, cudaStream_t s,
                 BfsStats *stats, cudaEvent_t ev_start, cudaEvent_t ev_stop) {
    std::unique_ptr<BfsPlan> p(bfs_plan_create(jobs, t, d_err, al, s, stats != nullptr));
    bfs_plan_run(p.get(), s, ev_start, ev_stop);
    bfs_plan_stats(p.get(), stats, s);
}

static void copy_csr(const Csr &g, Csr &out, Alloc *al, cudaStream_t s) {
    out.n = g.n;
    out.nnz = g.nnz;
    out.cap = g.cap;
    if (!out.rowptr.alloc(al, (size_t)g.n + 1) || !out.col.alloc(al, g.cap > 0 ? g.cap : 1))
        fail(HOMLN_ENOMEM, "bfs graph");
    HCUDA(cudaMemcpyAsync(out.rowptr.p, g.rowptr.p, sizeof(int64_t) * (g.n + 1), cudaMemcpyDeviceToDevice, s));
    if (g.cap > 0)
        HCUDA(cudaMemcpyAsync(out.col.p, g.col.p, sizeof(int32_t) * g.cap, cudaMemcpyDeviceToDevice, s));
}

void bfs_prepare(const Csr &g, const Csr *g_in, bool relabel, BfsGraph &out, Alloc *al, cudaStream_t s) {
    // the vertex order follows the degrees of the graph the bottom-up levels read (in-edges);
    // a directed graph's small components are the weak ones (in- and out-edges explored)
    out.relabeled = relabel;
    out.directed = g_in != nullptr;
    if (relabel) {
        DBuf<int32_t> inv;
        if (out.directed) {
            relabel_by_degree(*g_in, &g, out.csr_in, out.perm, inv, out.split, al, s);
            relabel_apply(g, out.perm.p, inv.p, out.csr, al, s);
        } else {
            relabel_by_degree(g, nullptr, out.csr, out.perm, inv, out.split, al, s);
        }
    } else {  // the BFS reads the graph as it is
        copy_csr(g, out.csr, al, s);
        if (out.directed) copy_csr(*g_in, out.csr_in, al, s);
    }
}

}  // namespace homln
