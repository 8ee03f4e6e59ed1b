// Closeness finalisation, CC-node selection, composition heuristics and accuracy.
//
//   closeness (Section 4): Wasserman-Faust normalised closeness, R^2 / ((n-1) F),
//       which is Eq. 1, (n-1)/F, on a connected graph; one correctly rounded
//       float64 division of exact integers.
//   sumDist (Section 5.1): F + n * (unreachable vertices), i.e. distance n for
//       every vertex that cannot be reached.
//   selection (Section 4, Section 5.2): the top-k, or every node at or above
//       the average score. The average test is exact on the float64 scores:
//       every score is turned into a 256-bit fixed-point integer (LSB 2^-128),
//       so the sum does not depend on the order of the additions.
//   naive (Section 4): intersection of the layers' CC-node sets.
//   CC1 (Section 5.1, Eqs. 2-3): degree-distance ratios, the largest layer
//       average, central one-hop neighbours and their overlap.
//   CC2 (Section 5.2, Algorithm 1): estSumDist = max over layers, scored by Eq. 1.
//   accuracy (Section 5, Section 6.1): tp/fp/fn by popcount of membership bitmaps.
#include "common.cuh"

#include <cmath>

namespace homln {

namespace {

unsigned grid_for(int64_t work, int threads = 256) {
    int64_t b = ceil_div(work > 0 ? work : 1, threads);
    return (unsigned)(b > 65535 * 16 ? 65535 * 16 : b);
}

// ---------------------------------------------------------------- 256-bit fixed point
struct Fix {
    uint64_t w[4];  // little-endian limbs; value = integer / 2^128
};

__device__ __forceinline__ void fix_zero(Fix &a) { a.w[0] = a.w[1] = a.w[2] = a.w[3] = 0; }

__device__ __forceinline__ void fix_add(Fix &a, const Fix &b) {
    unsigned long long c = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        unsigned long long s = a.w[i] + b.w[i];
        unsigned long long c1 = s < a.w[i];
        unsigned long long t = s + c;
        unsigned long long c2 = t < s;
        a.w[i] = t;
        c = c1 | c2;
    }
}

// Exact fixed-point image of a finite double x >= 0; false if it does not fit.
__device__ __forceinline__ bool fix_from_double(double x, Fix &out) {
    fix_zero(out);
    uint64_t bits = (uint64_t)__double_as_longlong(x);
    if (bits >> 63) return x == 0.0;  // -0.0 is zero; negatives do not occur
    int e = (int)((bits >> 52) & 0x7ff);
    uint64_t m = bits & ((1ull << 52) - 1);
    if (e == 0x7ff) return false;
    if (e == 0) {
        if (m == 0) return true;
        e = 1;
    } else {
        m |= 1ull << 52;
    }
    int shift = e - 1075 + 128;  // position of m's lowest bit
    if (shift < 0) {
        if (shift <= -64 || (m & ((1ull << (-shift)) - 1))) return false;
        m >>= -shift;
        shift = 0;
    }
    if (shift + 53 > 255) return false;
    int li = shift >> 6, off = shift & 63;
    out.w[li] = m << off;
    if (off > 11 && li + 1 < 4) out.w[li + 1] = m >> (64 - off);
    return true;
}

// a * small (small < 2^32); false on overflow.
__device__ __forceinline__ bool fix_mul_small(const Fix &a, uint64_t small, Fix &out) {
    unsigned long long carry = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        unsigned long long lo = a.w[i] * small;
        unsigned long long hi = __umul64hi(a.w[i], small);
        unsigned long long t = lo + carry;
        hi += t < lo;
        out.w[i] = t;
        carry = hi;
    }
    return carry == 0;
}

__device__ __forceinline__ int fix_cmp(const Fix &a, const Fix &b) {
#pragma unroll
    for (int i = 3; i >= 0; --i) {
        if (a.w[i] != b.w[i]) return a.w[i] < b.w[i] ? -1 : 1;
    }
    return 0;
}

// Block-level exact sum of fixed-point values; result valid in thread 0.
__device__ Fix block_fix_sum(Fix v) {
    __shared__ Fix sh[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        Fix other;
#pragma unroll
        for (int i = 0; i < 4; ++i) other.w[i] = __shfl_down_sync(0xffffffffu, v.w[i], o);
        if (lane + o < 32) fix_add(v, other);
    }
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    Fix s;
    fix_zero(s);
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) fix_add(s, sh[w]);
    __syncthreads();
    return s;
}

// partials[block] = exact sum of the finite values; cnt[block] = how many were finite.
__global__ void k_fix_sum_blocks(const double *__restrict__ x, int32_t n, Fix *partials, uint32_t *cnt, int32_t *err) {
    Fix acc;
    fix_zero(acc);
    uint32_t c = 0;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double v = x[i];
        if (isinf(v)) continue;
        Fix f;
        if (!fix_from_double(v, f)) dev_fail(err, DEV_RANGE);
        fix_add(acc, f);
        ++c;
    }
    Fix s = block_fix_sum(acc);
    uint32_t cs = (uint32_t)warp_sum((unsigned long long)c);
    __shared__ uint32_t shc[32];
    if ((threadIdx.x & 31) == 0) shc[threadIdx.x >> 5] = cs;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += shc[w];
        partials[blockIdx.x] = s;
        cnt[blockIdx.x] = t;
    }
}

__global__ void k_fix_sum_final(const Fix *partials, const uint32_t *cnt, int nb, Fix *out, uint32_t *out_cnt) {
    Fix acc;
    fix_zero(acc);
    unsigned long long c = 0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        fix_add(acc, partials[i]);
        c += cnt[i];
    }
    Fix s = block_fix_sum(acc);
    __shared__ unsigned long long shc[32];
    unsigned long long cs = warp_sum(c);
    if ((threadIdx.x & 31) == 0) shc[threadIdx.x >> 5] = cs;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += shc[w];
        *out = s;
        *out_cnt = (uint32_t)t;
    }
}

constexpr int SUM_BLOCKS = 304;  // 2 x 152 SMs

// Exact sum (and count) of the finite entries of x into d_sum/d_cnt.
void fix_sum(const double *x, int32_t n, Fix *d_sum, uint32_t *d_cnt, int32_t *d_err, Alloc *al, cudaStream_t s) {
    DBuf<Fix> part;
    DBuf<uint32_t> pc;
    if (!part.alloc(al, SUM_BLOCKS) || !pc.alloc(al, SUM_BLOCKS)) fail(HOMLN_ENOMEM, "exact sum scratch");
    launch(k_fix_sum_blocks, SUM_BLOCKS, 256, 0, s, x, n, part.p, pc.p, d_err);
    launch(k_fix_sum_final, 1, 256, 0, s, part.p, pc.p, SUM_BLOCKS, d_sum, d_cnt);
    HCUDA(cudaGetLastError());
}

// ---------------------------------------------------------------- closeness finalize
__global__ void k_finalize(int32_t n, const int64_t *__restrict__ rp, const uint64_t *__restrict__ F,
                           const uint32_t *__restrict__ R, double *__restrict__ cc, uint64_t *__restrict__ sumdist,
                           int32_t *__restrict__ deg) {
    const uint64_t nm1 = n > 0 ? (uint64_t)(n - 1) : 0;
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        uint64_t f = F[v];
        uint64_t r = R[v];
        if (cc) cc[v] = f > 0 ? __ddiv_rn(__ull2double_rn(r * r), __ull2double_rn(nm1 * f)) : 0.0;
        if (sumdist) sumdist[v] = f + (uint64_t)n * (nm1 - r);
        if (deg) deg[v] = (int32_t)(rp[v + 1] - rp[v]);
    }
}

// Imported partial results must be ones a BFS can produce: R(v) <= n-1 reached vertices, each
// at distance 1 .. n-1 (so R <= F <= R (n-1), and F = 0 exactly when R = 0).
__global__ void k_check_partials(int32_t n, const uint64_t *__restrict__ F, const uint32_t *__restrict__ R,
                                 int32_t *err) {
    const uint64_t nm1 = n > 0 ? (uint64_t)(n - 1) : 0;
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const uint64_t f = F[v], r = R[v];
        if (r > nm1 || f < r || f > r * nm1) dev_fail(err, DEV_RANGE);
    }
}

// ---------------------------------------------------------------- selection
__global__ void k_score_keys(int32_t n, const double *__restrict__ sc, uint64_t *__restrict__ keys,
                             uint32_t *__restrict__ ids) {
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        double x = sc[v];
        uint64_t b = (uint64_t)__double_as_longlong(x == 0.0 ? 0.0 : x);  // scores are >= 0
        keys[v] = ~b;  // ascending key = descending score
        ids[v] = (uint32_t)v;
    }
}

__global__ void k_count_mean(int32_t n, const double *__restrict__ sc, const Fix *sum, bool strict, uint32_t *count,
                             int32_t *err) {
    Fix S = *sum;
    uint32_t c = 0;
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        Fix f, nf;
        if (!fix_from_double(sc[v], f) || !fix_mul_small(f, (uint64_t)n, nf)) {
            dev_fail(err, DEV_RANGE);
            continue;
        }
        int cmp = fix_cmp(nf, S);
        c += strict ? (cmp > 0) : (cmp >= 0);
    }
    c = (uint32_t)warp_sum((unsigned long long)c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

__global__ void k_emit_selected(int32_t count, const uint32_t *__restrict__ ids, int32_t *__restrict__ out,
                                uint32_t *__restrict__ bits) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        uint32_t v = ids[i];
        if (out) out[i] = (int32_t)v;
        if (bits) atomicOr(&bits[v >> 5], 1u << (v & 31));
    }
}

// ---------------------------------------------------------------- CC2
struct PtrSet64 {
    const uint64_t *p[HOMLN_MAX_LAYERS];
    int r;
};

__global__ void k_cc2_scores(int32_t n, PtrSet64 sd, double *__restrict__ out) {
    const double nm1 = (double)(n > 0 ? n - 1 : 0);
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        uint64_t est = sd.p[0][v];
        for (int i = 1; i < sd.r; ++i) est = max(est, sd.p[i][v]);  // Algorithm 1: max of the layer sums
        out[v] = est > 0 ? __ddiv_rn(nm1, __ull2double_rn(est)) : 0.0;  // Eq. 1 on the estimate
    }
}

// ---------------------------------------------------------------- CC1
struct PtrSet32 {
    const int32_t *p[HOMLN_MAX_LAYERS];
    int r;
};

__global__ void k_min_degree(int32_t n, PtrSet32 deg, int32_t *__restrict__ mind) {
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        int32_t m = deg.p[0][v];
        for (int i = 1; i < deg.r; ++i) m = min(m, deg.p[i][v]);
        mind[v] = m;
    }
}

// Eq. 2: sumDist_i(v) / min_j deg_j(v); +inf when the minimum degree is 0.
__global__ void k_cc1_ratio(int32_t n, const uint64_t *__restrict__ sd, const int32_t *__restrict__ mind,
                            double *__restrict__ ratio) {
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        int32_t d = mind[v];
        ratio[v] = d > 0 ? __ddiv_rn(__ull2double_rn(sd[v]), (double)d) : __longlong_as_double(0x7ff0000000000000ll);
    }
}

// Eq. 3: pick the largest of the layer averages S_i / c_i (exact cross multiplication).
__global__ void k_cc1_pick_avg(int r, const Fix *sums, const uint32_t *cnts, Fix *best_sum, uint32_t *best_cnt,
                               int32_t *err) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int b = -1;
    for (int i = 0; i < r; ++i) {
        if (cnts[i] == 0) continue;  // no finite ratio: that layer's average is taken as 0
        if (b < 0) { b = i; continue; }
        Fix x, y;
        if (!fix_mul_small(sums[i], cnts[b], x) || !fix_mul_small(sums[b], cnts[i], y)) dev_fail(err, DEV_RANGE);
        if (fix_cmp(x, y) > 0) b = i;
    }
    if (b < 0) {
        Fix z;
        fix_zero(z);
        *best_sum = z;
        *best_cnt = 1;
    } else {
        *best_sum = sums[b];
        *best_cnt = cnts[b];
    }
}

// central bit of v in one layer: ratio < average, exactly (c * ratio < S).
__global__ void k_cc1_central(int32_t n, const double *__restrict__ ratio, const Fix *avg_sum, const uint32_t *avg_cnt,
                              uint32_t *__restrict__ bits, int32_t *err) {
    const Fix S = *avg_sum;
    const uint64_t c = *avg_cnt;
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        double x = ratio[v];
        if (isinf(x)) continue;
        Fix f, cf;
        if (!fix_from_double(x, f) || !fix_mul_small(f, c, cf)) {
            dev_fail(err, DEV_RANGE);
            continue;
        }
        if (fix_cmp(cf, S) < 0) atomicOr(&bits[v >> 5], 1u << (v & 31));
    }
}

struct Cc1Layers {
    const int64_t *rp[HOMLN_MAX_LAYERS];
    const int32_t *col[HOMLN_MAX_LAYERS];
    const uint32_t *central[HOMLN_MAX_LAYERS];
    int r;
};

__device__ __forceinline__ bool bit_of(const uint32_t *b, int32_t v) { return (b[v >> 5] >> (v & 31)) & 1u; }

// |AND_i C_i(u)| and |OR_i C_i(u)| with C_i(u) the central neighbours of u in layer i; keep u
// iff the union is non-empty and AND >= theta * OR. One warp per common CC node u; the lanes
// walk a row 32 entries at a time and test membership in the other rows with warp_row_has
// (every lane takes part).
__global__ void k_cc1_overlap(int32_t n, Cc1Layers L, const uint32_t *__restrict__ common, double theta,
                              uint32_t *__restrict__ out_bits) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = warp; u < n; u += nwarps) {
        if (!bit_of(common, (int32_t)u)) continue;  // uniform over the warp
        {
            unsigned long long inter = 0, uni = 0;
            for (int i = 0; i < L.r; ++i) {
                const int64_t b0 = L.rp[i][u], len = L.rp[i][u + 1] - b0;
                int64_t cur[HOMLN_MAX_LAYERS];  // per other layer: where its row walk resumes
                for (int k = 0; k < L.r; ++k) cur[k] = L.rp[k][u];
                for (int64_t j0 = 0; j0 < len; j0 += 32) {
                    const int nv = (int)(len - j0 < 32 ? len - j0 : 32);
                    const int32_t v = lane < nv ? L.col[i][b0 + j0 + lane] : -1;
                    const bool cen = lane < nv && bit_of(L.central[i], v);
                    bool earlier = false;  // already counted in the union through a lower layer
                    for (int k = 0; k < i; ++k) {
                        const bool has = warp_row_has(L.col[k], cur[k], L.rp[k][u + 1], v, nv, lane);
                        earlier = earlier || (has && bit_of(L.central[k], v));
                    }
                    if (cen && !earlier) ++uni;
                    if (i == 0) {
                        bool all = cen;
                        for (int k = 1; k < L.r; ++k) {
                            const bool has = warp_row_has(L.col[k], cur[k], L.rp[k][u + 1], v, nv, lane);
                            all = all && has && bit_of(L.central[k], v);
                        }
                        if (all) ++inter;
                    }
                }
            }
            inter = warp_sum(inter);
            uni = warp_sum(uni);
            if (lane == 0 && uni > 0 && (double)inter >= __dmul_rn(theta, (double)uni))
                atomicOr(&out_bits[u >> 5], 1u << (u & 31));
        }
    }
}

// ---------------------------------------------------------------- bitmaps
__global__ void k_bits_and(int32_t nw, uint32_t *acc, const uint32_t *other) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nw; i += gridDim.x * blockDim.x) acc[i] &= other[i];
}

__global__ void k_bits_popc(int32_t nw, const uint32_t *__restrict__ bits, int32_t *__restrict__ cnt) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nw; i += gridDim.x * blockDim.x)
        cnt[i] = __popc(bits[i]);
}

__global__ void k_bits_emit(int32_t nw, const uint32_t *__restrict__ bits, const int64_t *__restrict__ off,
                            int32_t *__restrict__ out) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nw; i += gridDim.x * blockDim.x) {
        uint32_t b = bits[i];
        int64_t o = off[i];
        while (b) {
            int t = __ffs(b) - 1;
            out[o++] = i * 32 + t;
            b &= b - 1;
        }
    }
}

// ---------------------------------------------------------------- accuracy
__global__ void k_list_bits(const int32_t *__restrict__ ids, int32_t cnt, int32_t n, uint32_t *__restrict__ bits,
                            int32_t *err) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) {
        int32_t v = ids[i];
        if (v < 0 || v >= n) {
            dev_fail(err, DEV_BAD_ID);
            continue;
        }
        atomicOr(&bits[v >> 5], 1u << (v & 31));
    }
}

__global__ void k_confusion(int32_t nw, const uint32_t *__restrict__ P, const uint32_t *__restrict__ T,
                            unsigned long long *out3) {
    unsigned long long tp = 0, fp = 0, fn = 0;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nw; i += gridDim.x * blockDim.x) {
        uint32_t p = P[i], t = T[i];
        tp += __popc(p & t);
        fp += __popc(p & ~t);
        fn += __popc(~p & t);
    }
    tp = warp_sum(tp);
    fp = warp_sum(fp);
    fn = warp_sum(fn);
    if ((threadIdx.x & 31) == 0) {
        if (tp) atomicAdd(out3 + 0, tp);
        if (fp) atomicAdd(out3 + 1, fp);
        if (fn) atomicAdd(out3 + 2, fn);
    }
}

// Jaccard, precision, recall, F1 from the counts (zero denominators give 1, 0, 0, 0).
__global__ void k_accuracy_ratios(const unsigned long long *c3, double *out4) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double tp = (double)c3[0], fp = (double)c3[1], fn = (double)c3[2];
    out4[0] = (c3[0] + c3[1] + c3[2]) > 0 ? __ddiv_rn(tp, tp + fp + fn) : 1.0;
    out4[1] = (c3[0] + c3[1]) > 0 ? __ddiv_rn(tp, tp + fp) : 0.0;
    out4[2] = (c3[0] + c3[2]) > 0 ? __ddiv_rn(tp, tp + fn) : 0.0;
    out4[3] = c3[0] > 0 ? __ddiv_rn(2.0 * tp, 2.0 * tp + fp + fn) : 0.0;
}

// Both id lists into their bitmaps in one pass (thread i takes pred[i] and truth[i]).
__global__ void k_lists_bits(const int32_t *__restrict__ pred, int32_t n_pred, const int32_t *__restrict__ truth,
                             int32_t n_truth, int32_t n, uint32_t *__restrict__ P, uint32_t *__restrict__ T, int32_t *err) {
    const int32_t m = n_pred > n_truth ? n_pred : n_truth;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        if (i < n_pred) {
            const int32_t v = pred[i];
            if (v < 0 || v >= n) dev_fail(err, DEV_BAD_ID);
            else atomicOr(&P[v >> 5], 1u << (v & 31));
        }
        if (i < n_truth) {
            const int32_t v = truth[i];
            if (v < 0 || v >= n) dev_fail(err, DEV_BAD_ID);
            else atomicOr(&T[v >> 5], 1u << (v & 31));
        }
    }
}

// Confusion counts of the two bitmaps; the last block to finish turns them into the ratios.
// out: tp, fp, fn (uint64), then jaccard, precision, recall, f1 (double), then a block counter.
struct AccOut {
    unsigned long long c3[3];
    double r4[4];
    unsigned int done;
};

__global__ void k_confusion_ratios(int32_t nw, const uint32_t *__restrict__ P, const uint32_t *__restrict__ T,
                                   AccOut *out) {
    unsigned long long tp = 0, fp = 0, fn = 0;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nw; i += gridDim.x * blockDim.x) {
        const uint32_t p = P[i], t = T[i];
        tp += __popc(p & t);
        fp += __popc(p & ~t);
        fn += __popc(~p & t);
    }
    tp = warp_sum(tp);
    fp = warp_sum(fp);
    fn = warp_sum(fn);
    if ((threadIdx.x & 31) == 0) {
        if (tp) atomicAdd(out->c3 + 0, tp);
        if (fp) atomicAdd(out->c3 + 1, fp);
        if (fn) atomicAdd(out->c3 + 2, fn);
    }
    __threadfence();
    __syncthreads();
    __shared__ bool last;
    if (threadIdx.x == 0) last = atomicAdd(&out->done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    const unsigned long long c0 = atomicAdd(out->c3 + 0, 0ull), c1 = atomicAdd(out->c3 + 1, 0ull),
                             c2 = atomicAdd(out->c3 + 2, 0ull);
    const double dtp = (double)c0, dfp = (double)c1, dfn = (double)c2;
    out->r4[0] = (c0 + c1 + c2) > 0 ? __ddiv_rn(dtp, dtp + dfp + dfn) : 1.0;
    out->r4[1] = (c0 + c1) > 0 ? __ddiv_rn(dtp, dtp + dfp) : 0.0;
    out->r4[2] = (c0 + c2) > 0 ? __ddiv_rn(dtp, dtp + dfn) : 0.0;
    out->r4[3] = c0 > 0 ? __ddiv_rn(2.0 * dtp, 2.0 * dtp + dfp + dfn) : 0.0;
}

}  // namespace

// ============================================================================
void closeness_finalize(int32_t n, const int64_t *rowptr, const uint64_t *F, const uint32_t *R, double *cc,
                        uint64_t *sumdist, int32_t *deg, cudaStream_t s) {
    if (n <= 0) return;
    launch(k_finalize, grid_for(n), 256, 0, s, n, rowptr, F, R, cc, sumdist, deg);
    HCUDA(cudaGetLastError());
}

void partials_check(int32_t n, const uint64_t *F, const uint32_t *R, int32_t *d_err, cudaStream_t s) {
    if (n <= 0) return;
    launch(k_check_partials, grid_for(n), 256, 0, s, n, F, R, d_err);
    HCUDA(cudaGetLastError());
}

int32_t select_nodes(int32_t n, const double *d_scores, const homln_select &sel, int32_t *d_out,
                     uint32_t *d_member_bits, int32_t *d_err, Alloc *al, cudaStream_t s) {
    if (d_member_bits) HCUDA(cudaMemsetAsync(d_member_bits, 0, sizeof(uint32_t) * ceil_div(n, 32), s));
    if (n <= 0) return 0;
    int64_t count = 0;
    if (sel.mode == HOMLN_TOPK_PERCENT) {
        count = (int64_t)std::ceil((sel.percent * (double)n) / 100.0);
    } else if (sel.mode == HOMLN_TOPK_COUNT) {
        count = sel.k;
    }
    DBuf<uint64_t> keys;
    DBuf<uint32_t> ids;
    if (!keys.alloc(al, n) || !ids.alloc(al, n)) fail(HOMLN_ENOMEM, "selection keys");
    launch(k_score_keys, grid_for(n), 256, 0, s, n, d_scores, keys.p, ids.p);
    radix_sort_u64(keys.p, ids.p, n, 0, 64, al, s);
    if (sel.mode == HOMLN_GE_MEAN || sel.mode == HOMLN_GT_MEAN) {
        DBuf<Fix> sum;
        DBuf<uint32_t> cnt;
        if (!sum.alloc(al, 1) || !cnt.alloc(al, 2)) fail(HOMLN_ENOMEM, "mean scratch");
        fix_sum(d_scores, n, sum.p, cnt.p, d_err, al, s);
        HCUDA(cudaMemsetAsync(cnt.p + 1, 0, sizeof(uint32_t), s));
        launch(k_count_mean, SUM_BLOCKS, 256, 0, s, n, d_scores, sum.p, sel.mode == HOMLN_GT_MEAN, cnt.p + 1, d_err);
        uint32_t h = 0;
        HCUDA(cudaMemcpyAsync(&h, cnt.p + 1, sizeof(h), cudaMemcpyDeviceToHost, s));
        HCUDA(cudaStreamSynchronize(s));
        count = h;
    }
    if (count < 0) count = 0;
    if (count > n) count = n;
    if (count > 0) launch(k_emit_selected, grid_for(count), 256, 0, s, (int32_t)count, ids.p, d_out, d_member_bits);
    HCUDA(cudaGetLastError());
    return (int32_t)count;
}

void cc2_scores(int32_t n, const std::vector<const uint64_t *> &sumdists, double *d_scores, Alloc *al, cudaStream_t s) {
    (void)al;
    PtrSet64 p{};
    p.r = (int)sumdists.size();
    for (int i = 0; i < p.r; ++i) p.p[i] = sumdists[i];
    launch(k_cc2_scores, grid_for(n), 256, 0, s, n, p, d_scores);
    HCUDA(cudaGetLastError());
}

int32_t cc1_compose(int32_t n, const std::vector<const Csr *> &csrs, const std::vector<const uint64_t *> &sumdist,
                    const std::vector<const int32_t *> &deg, const uint32_t *d_common_bits, double theta,
                    int32_t *d_out, int32_t *d_err, Alloc *al, cudaStream_t s) {
    const int r = (int)csrs.size();
    const int32_t nw = (int32_t)ceil_div(n, 32);
    DBuf<int32_t> mind;
    DBuf<double> ratio;
    DBuf<Fix> sums, best;
    DBuf<uint32_t> cnts, bestc, central, outbits;
    if (!mind.alloc(al, n) || !ratio.alloc(al, (size_t)n * r) || !sums.alloc(al, r) || !best.alloc(al, 1) ||
        !cnts.alloc(al, r) || !bestc.alloc(al, 1) || !central.alloc(al, (size_t)nw * r) || !outbits.alloc(al, nw))
        fail(HOMLN_ENOMEM, "cc1 scratch");
    PtrSet32 dp{};
    dp.r = r;
    for (int i = 0; i < r; ++i) dp.p[i] = deg[i];
    launch(k_min_degree, grid_for(n), 256, 0, s, n, dp, mind.p);
    for (int i = 0; i < r; ++i) {
        launch(k_cc1_ratio, grid_for(n), 256, 0, s, n, sumdist[i], mind.p, ratio.p + (size_t)i * n);
        fix_sum(ratio.p + (size_t)i * n, n, sums.p + i, cnts.p + i, d_err, al, s);
    }
    launch(k_cc1_pick_avg, 1, 32, 0, s, r, sums.p, cnts.p, best.p, bestc.p, d_err);
    HCUDA(cudaMemsetAsync(central.p, 0, sizeof(uint32_t) * nw * r, s));
    HCUDA(cudaMemsetAsync(outbits.p, 0, sizeof(uint32_t) * nw, s));
    Cc1Layers L{};
    L.r = r;
    for (int i = 0; i < r; ++i) {
        launch(k_cc1_central, grid_for(n), 256, 0, s, n, ratio.p + (size_t)i * n, best.p, bestc.p,
                                                  central.p + (size_t)i * nw, d_err);
        L.rp[i] = csrs[i]->rowptr.p;
        L.col[i] = csrs[i]->col.p;
        L.central[i] = central.p + (size_t)i * nw;
    }
    launch(k_cc1_overlap, grid_for((int64_t)n * 32), 256, 0, s, n, L, d_common_bits, theta, outbits.p);
    HCUDA(cudaGetLastError());
    return bits_to_sorted_ids(n, outbits.p, d_out, al, s);
}

int32_t bits_to_sorted_ids(int32_t n, const uint32_t *d_bits, int32_t *d_out, Alloc *al, cudaStream_t s) {
    const int32_t nw = (int32_t)ceil_div(n, 32);
    if (nw == 0) return 0;
    DBuf<int32_t> cnt;
    DBuf<int64_t> off;
    if (!cnt.alloc(al, nw) || !off.alloc(al, (size_t)nw + 1)) fail(HOMLN_ENOMEM, "bitmap scratch");
    launch(k_bits_popc, grid_for(nw), 256, 0, s, nw, d_bits, cnt.p);
    scan_exclusive_i32(cnt.p, off.p, nw, al, s);
    launch(k_bits_emit, grid_for(nw), 256, 0, s, nw, d_bits, off.p, d_out);
    int64_t total = 0;
    HCUDA(cudaMemcpyAsync(&total, off.p + nw, sizeof(total), cudaMemcpyDeviceToHost, s));
    HCUDA(cudaStreamSynchronize(s));
    return (int32_t)total;
}

void bits_and(int32_t nwords, uint32_t *d_acc, const uint32_t *d_other, cudaStream_t s) {
    launch(k_bits_and, grid_for(nwords), 256, 0, s, nwords, d_acc, d_other);
    HCUDA(cudaGetLastError());
}

void accuracy_counts(int32_t n, const int32_t *d_pred, int32_t n_pred, const int32_t *d_truth, int32_t n_truth,
                     homln_accuracy_t *h_out, int32_t *d_err, Alloc *al, cudaStream_t s) {
    // one scratch block: the two bitmaps, then the counts, ratios and block counter (the even
    // word count 2 * nw keeps AccOut 8-byte aligned)
    const int32_t nw = (int32_t)ceil_div(n, 32);
    static_assert(sizeof(AccOut) % 4 == 0, "AccOut is a whole number of words");
    const size_t words = 2 * (size_t)nw + sizeof(AccOut) / 4;
    DBuf<uint32_t> scratch;
    if (!scratch.alloc(al, words)) fail(HOMLN_ENOMEM, "accuracy scratch");
    uint32_t *P = scratch.p, *T = scratch.p + nw;
    AccOut *out = reinterpret_cast<AccOut *>(scratch.p + 2 * (size_t)nw);
    HCUDA(cudaMemsetAsync(scratch.p, 0, sizeof(uint32_t) * words, s));
    const int32_t m = n_pred > n_truth ? n_pred : n_truth;
    if (m > 0) launch(k_lists_bits, grid_for(m), 256, 0, s, d_pred, n_pred, d_truth, n_truth, n, P, T, d_err);
    launch(k_confusion_ratios, grid_for(nw), 256, 0, s, nw, (const uint32_t *)P, (const uint32_t *)T, out);
    HCUDA(cudaGetLastError());
    AccOut h;
    HCUDA(cudaMemcpyAsync(&h, out, sizeof(h), cudaMemcpyDeviceToHost, s));
    HCUDA(cudaStreamSynchronize(s));
    h_out->tp = (int64_t)h.c3[0];
    h_out->fp = (int64_t)h.c3[1];
    h_out->fn = (int64_t)h.c3[2];
    h_out->jaccard = h.r4[0];
    h_out->precision = h.r4[1];
    h_out->recall = h.r4[2];
    h_out->f1 = h.r4[3];
}

// The accuracy kernels run on scratch the caller provides (no allocation here).
// bits_p/bits_t hold ceil(n/32) words each; c3 three counters; r4 four doubles; err one word.
void accuracy_counts_prealloc(int32_t n, const int32_t *d_pred, int32_t n_pred, const int32_t *d_truth,
                              int32_t n_truth, uint32_t *bits_p, uint32_t *bits_t, unsigned long long *c3, double *r4,
                              int32_t *err, homln_accuracy_t *h_out, int32_t *h_err, cudaStream_t s) {
    const int32_t nw = (int32_t)ceil_div(n, 32);
    HCUDA(cudaMemsetAsync(bits_p, 0, sizeof(uint32_t) * nw, s));
    HCUDA(cudaMemsetAsync(bits_t, 0, sizeof(uint32_t) * nw, s));
    HCUDA(cudaMemsetAsync(c3, 0, sizeof(unsigned long long) * 3, s));
    HCUDA(cudaMemsetAsync(err, 0, sizeof(int32_t), s));
    if (n_pred > 0) launch(k_list_bits, grid_for(n_pred), 256, 0, s, d_pred, n_pred, n, bits_p, err);
    if (n_truth > 0) launch(k_list_bits, grid_for(n_truth), 256, 0, s, d_truth, n_truth, n, bits_t, err);
    launch(k_confusion, grid_for(nw), 256, 0, s, nw, (const uint32_t *)bits_p, (const uint32_t *)bits_t, c3);
    launch(k_accuracy_ratios, 1, 32, 0, s, (const unsigned long long *)c3, r4);
    HCUDA(cudaGetLastError());
    unsigned long long h[3];
    double r[4];
    HCUDA(cudaMemcpyAsync(h, c3, sizeof(h), cudaMemcpyDeviceToHost, s));
    HCUDA(cudaMemcpyAsync(r, r4, sizeof(r), cudaMemcpyDeviceToHost, s));
    HCUDA(cudaMemcpyAsync(h_err, err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    HCUDA(cudaStreamSynchronize(s));
    h_out->tp = (int64_t)h[0];
    h_out->fp = (int64_t)h[1];
    h_out->fn = (int64_t)h[2];
    h_out->jaccard = r[0];
    h_out->precision = r[1];
    h_out->recall = r[2];
    h_out->f1 = r[3];
}

}  // namespace homln
