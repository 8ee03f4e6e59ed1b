// Device primitives: exclusive prefix sum and a stable LSD radix sort.
// Used by CSR construction (sorting packed edge keys), relabelling and top-k
// selection. Hand-written; no library kernels.
#include "common.cuh"

#include <algorithm>
#include <climits>

namespace homln {

namespace {

constexpr int SCAN_T = 512;
constexpr int SCAN_I = 8;
constexpr int SCAN_TILE = SCAN_T * SCAN_I;

template <typename T>
__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t *total) {
    __shared__ int64_t warp_tot[SCAN_T / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < SCAN_T / 32 ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < SCAN_T / 32) warp_tot[lane] = w;  // inclusive
    }
    __syncthreads();
    int64_t warp_base = warp > 0 ? warp_tot[warp - 1] : 0;
    if (total) *total = warp_tot[SCAN_T / 32 - 1];
    int64_t excl = warp_base + x - v;
    __syncthreads();
    return excl;
}

template <typename T>
__global__ void __launch_bounds__(SCAN_T) k_scan_reduce(const T *__restrict__ in, int64_t n, int64_t *partials) {
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_I;
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_I; ++i)
        if (base + i < n) s += (int64_t)in[base + i];
    int64_t tot;
    block_exclusive_scan<T>(s, &tot);
    if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

// Exclusive scan of the block totals in place; writes the grand total to *total.
__global__ void __launch_bounds__(SCAN_T) k_scan_partials(int64_t *partials, int64_t nb, int64_t *total) {
    int64_t carry = 0;
    for (int64_t base = 0; base < nb; base += SCAN_T) {
        int64_t i = base + threadIdx.x;
        int64_t v = i < nb ? partials[i] : 0;
        int64_t tot;
        int64_t ex = block_exclusive_scan<int64_t>(v, &tot);
        if (i < nb) partials[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) *total = carry;
}

template <typename T>
__global__ void __launch_bounds__(SCAN_T) k_scan_down(const T *__restrict__ in, int64_t *out, int64_t n,
                                                     const int64_t *partials) {
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_I;
    int64_t vals[SCAN_I];
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_I; ++i) {
        vals[i] = (base + i < n) ? (int64_t)in[base + i] : 0;
        s += vals[i];
    }
    int64_t ex = block_exclusive_scan<T>(s, nullptr) + partials[blockIdx.x];
#pragma unroll
    for (int i = 0; i < SCAN_I; ++i) {
        if (base + i < n) out[base + i] = ex;
        ex += vals[i];
    }
}

// A scan that fits one tile: one block, one launch; writes the total to out[n].
template <typename T>
__global__ void __launch_bounds__(SCAN_T) k_scan_single(const T *__restrict__ in, int64_t *out, int64_t n) {
    int64_t base = (int64_t)threadIdx.x * SCAN_I;
    int64_t vals[SCAN_I];
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_I; ++i) {
        vals[i] = (base + i < n) ? (int64_t)in[base + i] : 0;
        s += vals[i];
    }
    int64_t tot;
    int64_t ex = block_exclusive_scan<T>(s, &tot);
#pragma unroll
    for (int i = 0; i < SCAN_I; ++i) {
        if (base + i < n) out[base + i] = ex;
        ex += vals[i];
    }
    if (threadIdx.x == 0) out[n] = tot;
}

template <typename T>
void scan_impl(const T *in, int64_t *out, int64_t n, Alloc *al, cudaStream_t s) {
    if (n <= 0) {
        HCUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
        return;
    }
    if (n <= SCAN_TILE) {
        launch(k_scan_single<T>, 1, SCAN_T, 0, s, in, out, n);
        HCUDA(cudaGetLastError());
        return;
    }
    int64_t nb = ceil_div(n, SCAN_TILE);
    DBuf<int64_t> part;
    if (!part.alloc(al, nb)) fail(HOMLN_ENOMEM, "scan: partials");
    launch(k_scan_reduce<T>, (unsigned)nb, SCAN_T, 0, s, in, n, part.p);
    launch(k_scan_partials, 1, SCAN_T, 0, s, part.p, nb, out + n);
    launch(k_scan_down<T>, (unsigned)nb, SCAN_T, 0, s, in, out, n, part.p);
    HCUDA(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// Radix sort: 8-bit digits, one histogram / offsets / scatter round per digit.
// The scatter ranks each tile's items stably: every warp walks its R*32 items
// in index order, 32 at a time, grouping equal digits with match.any.
// Small inputs (at most kRsFusedTiles tiles) skip the separate scan: every
// scatter block derives its own digit offsets from the per-tile histograms.
// ---------------------------------------------------------------------------
constexpr int RS_T = 256;
constexpr int RS_WARPS = RS_T / 32;
constexpr int kRsFusedTiles = 64;

template <int R>
__global__ void __launch_bounds__(RS_T) k_rs_hist(const uint64_t *__restrict__ keys, int64_t n, int shift,
                                                 uint32_t dmask, int32_t *counts, int64_t nb) {
    __shared__ int32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * (RS_T * R);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int64_t idx = base + r * RS_T + threadIdx.x;
        if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & dmask], 1);
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];
}

// FUSED: offsets[] holds the per-tile histograms (digit-major, counts[d * nb + b]) and each
// block computes its tile's digit offsets from them; otherwise offsets[] is their scan.
template <bool VALS, int R, bool FUSED>
__global__ void __launch_bounds__(RS_T) k_rs_scatter(const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin,
                                                    uint64_t *__restrict__ kout, uint32_t *__restrict__ vout, int64_t n,
                                                    int shift, uint32_t dmask, const int64_t *__restrict__ offsets,
                                                    const int32_t *__restrict__ counts, int64_t nb) {
    __shared__ int32_t wcnt[RS_WARPS][256];
    __shared__ int64_t boff[256];
    __shared__ int64_t wtot[RS_WARPS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < RS_WARPS * 256; i += RS_T) (&wcnt[0][0])[i] = 0;
    if (FUSED) {
        // digit d = threadIdx.x: items of digit d in all tiles, and in the tiles before this one
        const int32_t *row = counts + (int64_t)threadIdx.x * nb;
        int64_t tot = 0, pre = 0;
        for (int64_t b = 0; b < nb; ++b) {
            const int32_t c = row[b];
            tot += c;
            if (b < blockIdx.x) pre += c;
        }
        // exclusive scan of the digit totals over the block
        int64_t x = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wtot[warp] = x;
        __syncthreads();
        int64_t wbase = 0;
        for (int w = 0; w < warp; ++w) wbase += wtot[w];
        boff[threadIdx.x] = wbase + x - tot + pre;
    } else {
        boff[threadIdx.x] = offsets[(int64_t)threadIdx.x * nb + blockIdx.x];
    }
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * (RS_T * R) + (int64_t)warp * (R * 32);
    uint64_t k[R];
    uint32_t v[R];
    int32_t rank[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        int64_t idx = base + r * 32 + lane;
        bool valid = idx < n;
        k[r] = valid ? kin[idx] : 0ull;
        if (VALS) v[r] = valid ? vin[idx] : 0u;
        uint32_t d = valid ? (uint32_t)((k[r] >> shift) & dmask) : 256u;
        uint32_t peers = __match_any_sync(0xffffffffu, d);
        int before = __popc(peers & ((1u << lane) - 1u));
        int leader = __ffs(peers) - 1;
        int cur = valid ? wcnt[warp][d] : 0;
        __syncwarp();
        if (valid && lane == leader) wcnt[warp][d] = cur + __popc(peers);
        __syncwarp();
        rank[r] = cur + before;
    }
    __syncthreads();
    {
        int d = threadIdx.x;
        int32_t run = 0;
#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) {
            int32_t t = wcnt[w][d];
            wcnt[w][d] = run;
            run += t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < R; ++r) {
        int64_t idx = base + r * 32 + lane;
        if (idx < n) {
            uint32_t d = (uint32_t)((k[r] >> shift) & dmask);
            int64_t dest = boff[d] + wcnt[warp][d] + rank[r];
            kout[dest] = k[r];
            if (VALS) vout[dest] = v[r];
        }
    }
}

template <int R, bool FUSED>
void rs_pass(const uint64_t *ka, const uint32_t *va, uint64_t *kb, uint32_t *vb, int64_t n, int shift,
             uint32_t dmask, int32_t *counts, int64_t *offs, int64_t nb, Alloc *al, cudaStream_t s) {
    launch(k_rs_hist<R>, (unsigned)nb, RS_T, 0, s, ka, n, shift, dmask, counts, nb);
    if (!FUSED) scan_impl<int32_t>(counts, offs, 256 * nb, al, s);
    if (va)
        launch(k_rs_scatter<true, R, FUSED>, (unsigned)nb, RS_T, 0, s, ka, va, kb, vb, n, shift, dmask,
               (const int64_t *)offs, (const int32_t *)counts, nb);
    else
        launch(k_rs_scatter<false, R, FUSED>, (unsigned)nb, RS_T, 0, s, ka, (const uint32_t *)nullptr, kb,
               (uint32_t *)nullptr, n, shift, dmask, (const int64_t *)offs, (const int32_t *)counts, nb);
}

// ---------------------------------------------------------------------------
// Segmented sort of CSR rows (each row ascending, in place).
// Rows of <= 32 entries: one warp, a bitonic network in registers. Rows of
// 33 .. kRowSortSmem entries: one block, a bitonic network in shared memory.
// Longer rows (rare: hubs of very large graphs): one block, shared-memory chunks
// merged pairwise through a scratch copy. No host round trip.
// ---------------------------------------------------------------------------
constexpr int kRowSortSmem = 8192;

__device__ __forceinline__ int32_t warp_bitonic_sort(int32_t x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const int32_t y = __shfl_xor_sync(0xffffffffu, x, j);
            const bool up = (lane & k) == 0;
            const bool lower = (lane & j) == 0;
            x = (lower == up) ? min(x, y) : max(x, y);
        }
    }
    return x;
}

// Rows of <= 32 entries are sorted here; longer rows are listed for the block sort (mid[],
// up to kRowSortSmem entries) or the radix fallback (big[]).
__global__ void k_sort_rows_small(int32_t n, const int64_t *__restrict__ rp, int32_t *__restrict__ col,
                                  int32_t *__restrict__ mid, int32_t *__restrict__ big, int32_t *__restrict__ nlist) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = warp; r < n; r += nwarps) {
        const int64_t b = rp[r], d = rp[r + 1] - b;
        if (d > 32) {  // uniform over the warp
            if (lane == 0) {
                if (d <= kRowSortSmem) mid[atomicAdd(&nlist[0], 1)] = (int32_t)r;
                else big[atomicAdd(&nlist[1], 1)] = (int32_t)r;
            }
            continue;
        }
        if (d < 2) continue;
        int32_t x = lane < d ? col[b + lane] : INT32_MAX;
        x = warp_bitonic_sort(x);
        if (lane < d) col[b + lane] = x;
    }
}

// Bitonic sort of col[b, b + len) (len <= kRowSortSmem) in shared memory by one block.
__device__ void block_sort_chunk(int32_t *__restrict__ sh, int32_t *__restrict__ col, int64_t b, int len) {
    int P = 64;
    while (P < len) P <<= 1;
    for (int i = threadIdx.x; i < P; i += blockDim.x) sh[i] = i < len ? col[b + i] : INT32_MAX;
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < P; i += blockDim.x) {
                const int l = i ^ j;
                if (l > i) {
                    const int32_t x = sh[i], y = sh[l];
                    const bool up = (i & k) == 0;
                    if ((x > y) == up) {
                        sh[i] = y;
                        sh[l] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < len; i += blockDim.x) col[b + i] = sh[i];
    __syncthreads();
}

// One block per listed row of 33 .. kRowSortSmem entries.
__global__ void __launch_bounds__(256) k_sort_rows_mid(const int64_t *__restrict__ rp, int32_t *__restrict__ col,
                                                       const int32_t *__restrict__ mid, const int32_t *__restrict__ nlist) {
    __shared__ int32_t sh[kRowSortSmem];
    const int32_t count = nlist[0];
    for (int32_t li = blockIdx.x; li < count; li += gridDim.x) {
        const int32_t r = mid[li];
        block_sort_chunk(sh, col, rp[r], (int)(rp[r + 1] - rp[r]));
    }
}

// One block per listed row longer than kRowSortSmem entries: sort chunks of kRowSortSmem in
// shared memory, then merge runs pairwise (width kRowSortSmem, doubling) between the row and
// its place in tmp[]. Each thread merges an equal share of a run pair's output, its start
// found by a binary search along the merge path; equal keys come from the left run first.
__global__ void __launch_bounds__(256) k_sort_rows_big(const int64_t *__restrict__ rp, int32_t *__restrict__ col,
                                                       int32_t *__restrict__ tmp, const int32_t *__restrict__ big,
                                                       const int32_t *__restrict__ nlist) {
    __shared__ int32_t sh[kRowSortSmem];
    const int32_t count = nlist[1];
    for (int32_t li = blockIdx.x; li < count; li += gridDim.x) {
        const int32_t r = big[li];
        const int64_t b = rp[r], d = rp[r + 1] - b;
        for (int64_t c0 = 0; c0 < d; c0 += kRowSortSmem)
            block_sort_chunk(sh, col, b + c0, (int)(d - c0 < kRowSortSmem ? d - c0 : kRowSortSmem));
        int32_t *src = col + b, *dst = tmp + b;
        for (int64_t w = kRowSortSmem; w < d; w <<= 1) {
            for (int64_t a0 = 0; a0 < d; a0 += 2 * w) {
                const int64_t m1 = a0 + w < d ? a0 + w : d, e = a0 + 2 * w < d ? a0 + 2 * w : d;
                const int32_t *A = src + a0, *B = src + m1;
                const int64_t la = m1 - a0, lb = e - m1, total = e - a0;
                const int64_t share = (total + blockDim.x - 1) / blockDim.x;
                const int64_t k0 = min((int64_t)threadIdx.x * share, total), k1 = min(k0 + share, total);
                int64_t lo = k0 - lb > 0 ? k0 - lb : 0, hi = k0 < la ? k0 : la;
                while (lo < hi) {
                    const int64_t mid = (lo + hi) >> 1;
                    if (A[mid] <= B[k0 - mid - 1]) lo = mid + 1; else hi = mid;
                }
                int64_t i = lo, j = k0 - lo;
                for (int64_t k = k0; k < k1; ++k) {
                    if (j >= lb || (i < la && A[i] <= B[j])) dst[a0 + k] = A[i++];
                    else dst[a0 + k] = B[j++];
                }
            }
            __syncthreads();
            int32_t *x = src; src = dst; dst = x;
        }
        if (src != col + b)
            for (int64_t i = threadIdx.x; i < d; i += blockDim.x) col[b + i] = src[i];
        __syncthreads();
    }
}

unsigned grid_of(int64_t work, int threads) {
    int64_t b = ceil_div(work > 0 ? work : 1, threads);
    return (unsigned)(b > 65535 * 16 ? 65535 * 16 : b);
}

}  // namespace

void scan_exclusive_i32(const int32_t *in, int64_t *out, int64_t n, Alloc *al, cudaStream_t s) {
    scan_impl<int32_t>(in, out, n, al, s);
}

void scan_exclusive_i64(const int64_t *in, int64_t *out, int64_t n, Alloc *al, cudaStream_t s) {
    scan_impl<int64_t>(in, out, n, al, s);
}

void radix_sort_u64(uint64_t *keys, uint32_t *vals, int64_t n, int bit0, int bit1, Alloc *al, cudaStream_t s) {
    if (n <= 1 || bit1 <= bit0) return;
    // tile of 4 items per thread while that keeps the tiles few enough for the fused offsets,
    // else 16 per thread; beyond kRsFusedTiles tiles of 16 a separate scan makes the offsets
    const int R = n <= (int64_t)kRsFusedTiles * RS_T * 4 ? 4 : 16;
    const int64_t nb = ceil_div(n, (int64_t)RS_T * R);
    const bool fused = nb <= kRsFusedTiles;
    DBuf<uint64_t> kalt;
    DBuf<uint32_t> valt;
    DBuf<int32_t> counts;
    DBuf<int64_t> offs;
    if (!kalt.alloc(al, n) || (vals && !valt.alloc(al, n)) || !counts.alloc(al, 256 * nb) ||
        (!fused && !offs.alloc(al, 256 * nb + 1)))
        fail(HOMLN_ENOMEM, "radix sort scratch");
    uint64_t *ka = keys, *kb = kalt.p;
    uint32_t *va = vals, *vb = valt.p;
    for (int shift = bit0; shift < bit1; shift += 8) {
        int bits = bit1 - shift < 8 ? bit1 - shift : 8;
        uint32_t dmask = (1u << bits) - 1u;
        if (R == 4)
            rs_pass<4, true>(ka, va, kb, vb, n, shift, dmask, counts.p, offs.p, nb, al, s);
        else if (fused)
            rs_pass<16, true>(ka, va, kb, vb, n, shift, dmask, counts.p, offs.p, nb, al, s);
        else
            rs_pass<16, false>(ka, va, kb, vb, n, shift, dmask, counts.p, offs.p, nb, al, s);
        HCUDA(cudaGetLastError());
        uint64_t *tk = ka; ka = kb; kb = tk;
        uint32_t *tv = va; va = vb; vb = tv;
    }
    if (ka != keys) {
        HCUDA(cudaMemcpyAsync(keys, ka, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
        if (vals) HCUDA(cudaMemcpyAsync(vals, va, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    }
}

void sort_rows(int32_t n, const int64_t *d_rowptr, int32_t *d_col, int64_t cap, Alloc *al, cudaStream_t s) {
    if (n <= 0 || cap <= 1) return;
    const bool may_be_big = cap > kRowSortSmem;  // a row cannot be longer than all entries together
    DBuf<int32_t> mid, big, nlist, tmp;
    if (!mid.alloc(al, n) || !big.alloc(al, n) || !nlist.alloc(al, 2) || (may_be_big && !tmp.alloc(al, cap)))
        fail(HOMLN_ENOMEM, "row sort scratch");
    HCUDA(cudaMemsetAsync(nlist.p, 0, 2 * sizeof(int32_t), s));
    launch(k_sort_rows_small, grid_of((int64_t)n * 32, 256), 256, 0, s, n, d_rowptr, d_col, mid.p, big.p, nlist.p);
    int dev = 0, nsm = 0;
    HCUDA(cudaGetDevice(&dev));
    HCUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    launch(k_sort_rows_mid, (unsigned)(nsm * 4), 256, 0, s, (const int64_t *)d_rowptr, d_col, (const int32_t *)mid.p,
           (const int32_t *)nlist.p);
    if (may_be_big)
        launch(k_sort_rows_big, (unsigned)nsm, 256, 0, s, (const int64_t *)d_rowptr, d_col, tmp.p,
               (const int32_t *)big.p, (const int32_t *)nlist.p);
    HCUDA(cudaGetLastError());
}

}  // namespace homln
