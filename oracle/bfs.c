/*
 * Oracle: breadth-first search distance sums. TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the CPU-baseline leg of the benchmark may
 * load this library. The GPU product path never calls it.
 *
 * What it computes (Section 4, the NetworkX closeness procedure the paper uses
 * for the layers and the ground truth): for every requested source s, a BFS
 * from s over an undirected unweighted graph gives the hop distance d(s, v) to
 * every vertex it reaches. It returns
 *     F(s) = sum of d(s, v) over all reached v          (unreachable adds 0)
 *     R(s) = number of reached vertices other than s.
 * This is a plain FIFO-queue BFS, one source at a time; nothing is batched,
 * fused or reordered. With n_threads > 1 the independent sources are spread
 * over OpenMP threads, each with its own queue; the per-source arithmetic is
 * unchanged.
 *
 * Graph format: CSR over vertices 0..n-1, rowptr[n+1] (int64), col[rowptr[n]]
 * (int32). Each undirected edge appears in both rows.
 */
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Distances from one source; dist[v] = -1 when v is unreachable. Returns 0 on success. */
int oracle_bfs_dist(int32_t n, const int64_t *rowptr, const int32_t *col, int32_t s, int32_t *dist)
{
    if (n <= 0 || s < 0 || s >= n) return 1;
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!queue) return 2;
    for (int32_t v = 0; v < n; ++v) dist[v] = -1;
    int64_t head = 0, tail = 0;
    dist[s] = 0;
    queue[tail++] = s;
    while (head < tail) {
        int32_t u = queue[head++];
        for (int64_t j = rowptr[u]; j < rowptr[u + 1]; ++j) {
            int32_t v = col[j];
            if (dist[v] < 0) {
                dist[v] = dist[u] + 1;
                queue[tail++] = v;
            }
        }
    }
    free(queue);
    return 0;
}

/* Farness and reach for each of the given sources (sources == NULL means all 0..n-1). */
int oracle_bfs_farness(int32_t n, const int64_t *rowptr, const int32_t *col, int32_t n_sources,
                       const int32_t *sources, uint64_t *farness, uint32_t *reach, int32_t n_threads)
{
    if (n <= 0) return 1;
    if (!sources) n_sources = n;
    for (int32_t i = 0; i < n_sources; ++i) {
        int32_t s = sources ? sources[i] : i;
        if (s < 0 || s >= n) return 1;
    }
    int failed = 0;
#ifdef _OPENMP
    if (n_threads < 1) n_threads = 1;
#pragma omp parallel num_threads(n_threads) reduction(| : failed)
#endif
    {
        int32_t *dist = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
        int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
        if (!dist || !queue) {
            failed = 1;
        } else {
            for (int32_t v = 0; v < n; ++v) dist[v] = -1;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
            for (int32_t i = 0; i < n_sources; ++i) {
                int32_t s = sources ? sources[i] : i;
                int64_t head = 0, tail = 0;
                uint64_t f = 0;
                dist[s] = 0;
                queue[tail++] = s;
                while (head < tail) {
                    int32_t u = queue[head++];
                    for (int64_t j = rowptr[u]; j < rowptr[u + 1]; ++j) {
                        int32_t v = col[j];
                        if (dist[v] < 0) {
                            dist[v] = dist[u] + 1;
                            f += (uint64_t)dist[v];
                            queue[tail++] = v;
                        }
                    }
                }
                farness[i] = f;
                reach[i] = (uint32_t)(tail - 1);
                /* reset only what this BFS touched */
                for (int64_t q = 0; q < tail; ++q) dist[queue[q]] = -1;
            }
        }
        free(dist);
        free(queue);
    }
    return failed ? 2 : 0;
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
