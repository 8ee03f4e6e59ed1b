/*
 * homln.h -- C-ABI of the GB300 library for decoupled closeness centrality on
 * homogeneous multilayer networks (HoMLNs).
 *
 * Method: Pavel, Roy, Santra, Chakravarthy, "Closeness Centrality Detection in
 * Homogeneous Multilayer Networks" (arXiv 2207.11662).
 *   Problem statement (Section 1): given layers G_1(V,E_1) ... G_l(V,E_l) over one
 *   vertex set, find the closeness-centrality (CC) nodes of the Boolean-AND
 *   aggregate of any r <= l layers from partial results of each layer
 *   (analysis step Psi, composition step Theta).
 *
 * Conventions used by every call
 *   - Graphs are unweighted and undirected (or directed with HOMLN_DIRECTED). Node
 *     ids are int32 in [0, n). Self loops and repeated edges in the input are
 *     accepted and dropped (simple-graph semantics, Section 4).
 *   - All GPU work runs on the CUDA stream given to homln_create, on the device
 *     that was current at homln_create.
 *   - Output pointers may be host memory (pageable or pinned) or device memory;
 *     the library asks the CUDA runtime which it is. A call that writes any host
 *     output returns after the data is there (it synchronises the stream). A call
 *     whose outputs are all device memory only enqueues work and returns; errors
 *     raised by that work on the device surface at the next synchronising call or
 *     at homln_sync. Device-side waits are bounded (homln_tuning.wait_limit_ms):
 *     a wait that runs out makes the kernel stop and the call report
 *     HOMLN_ETIMEOUT. When a device-side error is reported, the handle drops its
 *     cached results (as homln_invalidate does) and stays usable; after a failed
 *     homln_batch_analyse, invalidate every handle of the batch.
 *   - Every call returns a homln_status. No C++ exception crosses this boundary.
 *     On error the outputs are left untouched unless stated otherwise, and
 *     homln_last_error() returns a message for the calling thread.
 *   - The caller owns every buffer it passes. The handle owns all device memory
 *     it allocates (CSRs, AND graphs, BFS state, cached results) and frees it
 *     in homln_destroy.
 *   - A handle is not thread safe: one thread at a time may call into it.
 */
#ifndef HOMLN_H
#define HOMLN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define HOMLN_API __attribute__((visibility("default")))
#else
#define HOMLN_API
#endif

/* Opaque handle of a captured analysis (homln_graph_capture). */
typedef struct homln_graph_s *homln_graph_t;
typedef struct homln_yield_s *homln_yield_t;

/* Opaque handle: one HoMLN resident on one GPU. */
typedef struct homln_s *homln_t;

#define HOMLN_MAX_LAYERS 64
#define HOMLN_MAX_NODES 1048576 /* 2^20: (n-1)*farness stays below 2^60 */

typedef enum homln_status {
    HOMLN_OK = 0,
    HOMLN_EINVAL = 1,   /* bad argument: null handle, id out of range, empty mask, n out of range ... */
    HOMLN_ENOMEM = 2,   /* the allocator returned NULL */
    HOMLN_ECUDA = 3,    /* a CUDA runtime call failed (message in homln_last_error) */
    HOMLN_ERANGE = 4,   /* an output capacity is too small, or a value left its exact range */
    HOMLN_ETIMEOUT = 5, /* a bounded device-side wait gave up (the kernel returned early) */
    HOMLN_EBUSY = 6     /* the handle or its results are in use by a captured graph */
} homln_status;

/* homln_create flags */
#define HOMLN_PTR_HOST 0u   /* edge arrays are host memory (flags are a bitwise OR) */
#define HOMLN_PTR_DEVICE 1u /* edge arrays are device memory of the current device */
#define HOMLN_DIRECTED 2u   /* layers are directed: (src, dst) is an arc src -> dst (Section 4 defines
                               closeness for directed graphs too). Closeness is then in-closeness, from
                               the distances d(v, u) of the vertices v that reach u (as NetworkX computes
                               it for directed graphs); reach counts those v; degrees are in-degrees
                               and CC1's one-hop neighbours are in-neighbours; edge lists are arcs. */

/* Composition heuristics: naive (Section 4), CC1 (Section 5.1), CC2 (Section 5.2, Algorithm 1). */
typedef enum homln_heuristic { HOMLN_NAIVE = 0, HOMLN_CC1 = 1, HOMLN_CC2 = 2 } homln_heuristic;

/* CC-node selection rule.
 *   TOPK_PERCENT: the k = ceil(percent * n / 100) highest scores (double arithmetic).
 *   TOPK_COUNT:   the k highest scores (k clamped to [0, n]).
 *   GE_MEAN:      every node whose score is at least the mean score (Section 4),
 *                 decided exactly on the float64 scores.
 *   GT_MEAN:      strictly above the mean.
 * Ranking: score descending, equal scores by ascending node id.
 * cc1_overlap is the threshold theta of CC1's overlap test (Section 5.1 asks for a large
 * overlap of central neighbours without defining it): a common CC node u is kept iff
 * |AND of C_i(u)| >= theta*|OR of C_i(u)| and the union is non-empty. */
typedef enum homln_select_mode {
    HOMLN_TOPK_PERCENT = 0,
    HOMLN_TOPK_COUNT = 1,
    HOMLN_GE_MEAN = 2,
    HOMLN_GT_MEAN = 3
} homln_select_mode;

typedef struct homln_select {
    int32_t mode;       /* homln_select_mode */
    int32_t reserved;   /* must be 0 */
    double percent;     /* TOPK_PERCENT */
    int64_t k;          /* TOPK_COUNT */
    double cc1_overlap; /* CC1 theta in [0, 1] */
} homln_select;

/* Device-memory allocator. alloc returns device memory usable on `stream`
 * (or NULL on failure); free releases it in stream order. NULL for the whole
 * struct selects a stream-ordered memory pool owned by the library, one per
 * device, that keeps up to 8 GiB of freed memory mapped for later calls. The
 * library calls it from the thread that called into the library. */
typedef struct homln_allocator {
    void *ctx;
    void *(*alloc)(void *ctx, size_t bytes, void *stream);
    void (*free)(void *ctx, void *ptr, size_t bytes, void *stream);
} homln_allocator;

/* Accuracy of an estimated CC-node set against ground truth (Section 5,
 * Section 6.1): what the paper calls accuracy is the Jaccard coefficient.
 *   jaccard = tp/(tp+fp+fn) (1 when all three are 0), precision = tp/(tp+fp),
 *   recall = tp/(tp+fn), f1 = 2tp/(2tp+fp+fn) (each 0 when its denominator is 0). */
typedef struct homln_accuracy_t {
    int64_t tp, fp, fn;
    double jaccard, precision, recall, f1;
} homln_accuracy_t;

/* Tuning knobs of the multi-source BFS; zero fields take the built-in defaults. */
typedef struct homln_tuning {
    int32_t words_per_node;  /* W: 64*W sources per BFS batch; 1, 2, 4, 8, 16 or 32 (0 = auto) */
    int32_t push_alpha;      /* go top-down when alpha * frontier_edges < unfinished_edges (0 = default 16) */
    int32_t threads;         /* threads per block of the persistent BFS (0 = 512) */
    int32_t blocks_per_sm;   /* resident blocks per SM (0 = as many as fit) */
    int32_t relabel;         /* 1 = degree-descending relabelling of each graph before BFS, 0 = off, -1 = default */
    int32_t teams;           /* teams of blocks that run (graph, source batch) tiles concurrently (0 = auto:
                                as many as keep the state of all teams near 240 MB, at least 16, at most
                                one per tile and 2 GB of state in all) */
    int32_t team_mix;        /* 1: blocks resident on one SM join different teams; 0 (default): the same team */
    int32_t schedule;        /* 0 (default): one persistent launch over all (graph, batch) tiles;
                                1: plain -- one ordinary launch per BFS phase, levels driven by the host
                                   (the comparison baseline; identical results) */
    int32_t wait_limit_ms;   /* give-up time of every device-side wait of the BFS (team and grid
                                barriers); the call then fails with HOMLN_ETIMEOUT (0 = 2000 ms) */
    int32_t test_phantom_blocks; /* failure-detection tests only: every team barrier of the
                                persistent BFS also waits for this many blocks that do not exist,
                                so its wait runs out after wait_limit_ms (0 = off) */
    int32_t max_tiles_per_launch; /* the persistent BFS takes at most this many (graph, batch) tiles
                                per launch and launches again for the rest, so that work on other
                                streams (e.g. a higher-priority one) can run in between; identical
                                results (0 = all tiles in one launch) */
    int32_t sm_count;        /* the persistent BFS launches blocks_per_sm x sm_count blocks, so that it
                                occupies about sm_count SMs' worth of the GPU and work on other streams
                                (another request's analysis, say) runs beside it on the rest;
                                identical results (0 = every SM; larger than the device: every SM) */
} homln_tuning;

/* Create a handle: copy the layers to the device and build one CSR per layer.
 *   n_nodes      number of shared nodes n, 1 <= n <= HOMLN_MAX_NODES (Section 1: |V| is shared).
 *   n_layers     number of layers l, 1 <= l <= HOMLN_MAX_LAYERS.
 *   edge_counts  host array[n_layers]: edges in layer i (>= 0).
 *   src, dst     host arrays[n_layers] of pointers; layer i's edges are
 *                (src[i][e], dst[i][e]), e < edge_counts[i], int32, host or device
 *                memory according to `flags`.
 *   flags        HOMLN_PTR_HOST or HOMLN_PTR_DEVICE.
 *   alloc        device allocator or NULL (see homln_allocator).
 *   stream       cudaStream_t to run on (NULL = the legacy default stream).
 *   out          receives the handle.
 * Synchronous: returns after the CSRs are built and every id has been checked.
 * Errors: EINVAL (n, l, counts, null pointers, an id outside [0, n)), ENOMEM, ECUDA. */
HOMLN_API homln_status homln_create(int32_t n_nodes, int32_t n_layers, const int64_t *edge_counts,
                          const int32_t *const *src, const int32_t *const *dst, uint32_t flags,
                          const homln_allocator *alloc, void *stream, homln_t *out);

/* Release everything the handle owns (stream-ordered frees, then a stream synchronise). NULL is a no-op. */
HOMLN_API homln_status homln_destroy(homln_t h);

/* Set the BFS tuning of a handle (copied). NULL restores defaults. */
HOMLN_API homln_status homln_set_tuning(homln_t h, const homln_tuning *t);

/* Psi for one layer (Section 3: each layer analysed once; Section 4: BFS from every vertex).
 * Runs the all-sources BFS once per layer and caches the result in the handle.
 *   farness[n] (uint64): F(v) = sum of hop distances from v to the vertices it reaches.
 *   reach[n]   (uint32): R(v) = vertices reachable from v, v excluded.
 *   cc[n]      (double): Wasserman-Faust closeness R^2 / ((n-1) F), 0 when F = 0; on a
 *              connected layer this is Eq. 1, (n-1)/F. One correctly rounded division.
 * Any output may be NULL. Errors: EINVAL (layer out of range), ENOMEM, ECUDA, ETIMEOUT. */
HOMLN_API homln_status homln_layer_closeness(homln_t h, int32_t layer, uint64_t *farness, uint32_t *reach, double *cc);

/* Psi for several graphs in one persistent launch (Section 3: layers are analysed
 * independently and in parallel): every layer in `layer_mask` not analysed yet and, if
 * with_and != 0, the AND aggregate of `layer_mask`. The results are cached exactly as
 * homln_layer_closeness / homln_and_closeness would cache them (and are identical); those
 * calls then only copy them out. Asynchronous on the handle's stream.
 * Errors: EINVAL (mask), ENOMEM, ECUDA; device errors surface at the next synchronising call. */
HOMLN_API homln_status homln_analyse(homln_t h, uint64_t layer_mask, int32_t with_and);

/* Psi for many HoMLNs in one persistent launch: for every handle nets[i], the layers in
 * masks[i] and (with_and != 0) their AND aggregate. The BFS tiles of all these graphs share
 * one device work queue, so small and large graphs balance across the GPU. All handles must
 * live on one device; the launch runs on nets[0]'s stream with nets[0]'s tuning, allocator
 * and error word, and the other handles' streams are ordered before and after it with events.
 * Results are cached in each handle exactly as homln_analyse would cache them.
 * Errors: EINVAL (null handle, masks, devices), ENOMEM, ECUDA. */
HOMLN_API homln_status homln_batch_analyse(homln_t *nets, int32_t count, const uint64_t *masks, int32_t with_and);

/* Capture the analysis that homln_batch_analyse would run (every layer in masks[i] and, with
 * with_and != 0, the AND graph of masks[i], for every handle nets[i]) into a CUDA graph. All
 * preparation happens here, once: CSR and AND builds, relabelling, result buffers and the BFS
 * state. The graph holds the zeroing, the persistent BFS launch(es), the scatter-back and the
 * closeness finalize, so a replay allocates nothing and copies nothing from the host. It runs
 * on nets[0]'s stream with nets[0]'s tuning and error word. While the graph exists, the
 * results of its graphs stay allocated (homln_invalidate only marks them stale), homln_destroy
 * of its handles fails with HOMLN_EBUSY, and changing the relabelling setting fails with
 * HOMLN_EBUSY. Errors: EINVAL (null pointers, masks, devices, the plain schedule or an
 * instrumented handle, neither of which can be captured), ENOMEM, ECUDA (capture refused). */
HOMLN_API homln_status homln_graph_capture(homln_t *nets, int32_t count, const uint64_t *masks, int32_t with_and,
                                           homln_graph_t *out);

/* Replay a captured analysis (asynchronous on nets[0]'s stream; the other handles' streams
 * are ordered around it with events). Afterwards the results are cached exactly as after
 * homln_batch_analyse. Device errors surface at the next synchronising call. */
HOMLN_API homln_status homln_graph_launch(homln_graph_t g);

/* Wait for the graph's replays and release it. NULL is a no-op. */
HOMLN_API homln_status homln_graph_destroy(homln_graph_t g);

/* The batched analysis in one call: every layer of every handle and the AND graph of all its
 * layers (homln_batch_analyse with full masks), ordered after the work queued on `stream`
 * (a cudaStream_t; NULL = the legacy default stream), with `stream` ordered after the results.
 * For repeated runs, homln_graph_capture holds the same analysis as a CUDA graph.
 * Errors: as homln_batch_analyse. */
HOMLN_API homln_status homln_batch_closeness(homln_t *nets, int32_t count, void *stream);

/* Boolean AND aggregation of the layers in `layer_mask` (Section 3.1, Section 4 ground truth):
 * an edge is kept iff it is present in every selected layer. The AND graph is built
 * once per mask and cached. Edges are written as pairs u < v in ascending (u, v) order.
 *   capacity       entries available in and_src/and_dst (ignored when both are NULL).
 *   and_src/dst    int32 outputs (host or device), or NULL to query the count only.
 *   and_edge_count host int64 output: number of undirected AND edges (always written on OK/ERANGE).
 * Errors: EINVAL (empty mask or a bit >= n_layers), ERANGE (capacity < count), ENOMEM, ECUDA. */
HOMLN_API homln_status homln_and_aggregate(homln_t h, uint64_t layer_mask, int64_t capacity, int32_t *and_src,
                                 int32_t *and_dst, int64_t *and_edge_count);

/* Ground truth closeness: all-sources BFS on the AND graph of `layer_mask` (Section 4).
 * Same outputs and rules as homln_layer_closeness. */
HOMLN_API homln_status homln_and_closeness(homln_t h, uint64_t layer_mask, uint64_t *farness, uint32_t *reach, double *cc);

/* Boolean OR aggregation (Section 3.1 names it as the alternative to AND): an edge is kept iff
 * it is present in at least one selected layer. Built once per mask and cached; same output
 * conventions and errors as homln_and_aggregate. */
HOMLN_API homln_status homln_or_aggregate(homln_t h, uint64_t layer_mask, int64_t capacity, int32_t *or_src,
                                          int32_t *or_dst, int64_t *or_edge_count);

/* All-sources BFS closeness of the OR graph of `layer_mask`; same outputs as homln_layer_closeness. */
HOMLN_API homln_status homln_or_closeness(homln_t h, uint64_t layer_mask, uint64_t *farness, uint32_t *reach,
                                          double *cc);

/* CC nodes of one graph: which = layer id, -1 for the AND graph of layer_mask (the ground
 * truth), or -2 for the OR graph of layer_mask. Scores are the closeness values of homln_*_closeness; the selection rule
 * is `sel`. nodes_out (capacity n, host or device) receives the ids in rank order;
 * count_out (host) the number written.
 * Errors: EINVAL (which/mask/sel), ENOMEM, ECUDA, ETIMEOUT. */
HOMLN_API homln_status homln_topk(homln_t h, int32_t which, uint64_t layer_mask, const homln_select *sel,
                        int32_t *nodes_out, int32_t *count_out);

/* Theta: estimated CC nodes of the AND aggregate of `layer_mask` from per-layer partial results.
 *   HOMLN_NAIVE  intersection of the layers' CC-node sets (Section 4).
 *   HOMLN_CC1    Section 5.1: Eq. 2 ratio sumDist_i(u)/min_j deg_j(u), Eq. 3 average = max of the
 *                layers' exact mean ratios, central neighbours (ratio < average), overlap test.
 *   HOMLN_CC2    Section 5.2, Algorithm 1: estSumDist(u) = max_i sumDist_i(u), scored with Eq. 1
 *                as (n-1)/estSumDist(u), then `sel`.
 * sumDist charges n for each unreachable node (Section 5.1). With r > 2 layers the pairwise
 * rules apply across all r (intersection, max, min). Layer CC-node sets use `sel`.
 * nodes_out (capacity n, host or device) receives the ids in ascending order; count_out (host)
 * the number written. Errors: EINVAL, ENOMEM, ECUDA, ETIMEOUT. */
HOMLN_API homln_status homln_compose(homln_t h, uint64_t layer_mask, int32_t heuristic, const homln_select *sel,
                           int32_t *nodes_out, int32_t *count_out);

/* One subset of layers in homln_subset_sweep. */
typedef struct homln_subset_result {
    uint64_t mask;          /* the subset (bit i = layer i) */
    int32_t truth_count;    /* ground-truth CC nodes (AND graph of the subset) */
    int32_t estimate_count; /* CC nodes estimated by the heuristic from the layers' partial results */
    homln_accuracy_t acc;   /* estimate vs ground truth */
} homln_subset_result;

/* Every subset of at least `min_layers` layers (Section 1: any r <= l layers; Section 6.1: the
 * layers are analysed once and reused for every subset). All layers and every subset's AND
 * graph are analysed in one persistent launch (results cached), then for each subset the
 * ground truth, the `heuristic` estimate and their accuracy are computed with `sel`.
 * out (host, capacity entries) receives the subsets in increasing mask order; count_out (host)
 * the number of subsets (2^l - 1 minus the smaller ones). Errors: EINVAL, ERANGE (capacity),
 * ENOMEM, ECUDA. */
HOMLN_API homln_status homln_subset_sweep(homln_t h, int32_t heuristic, const homln_select *sel, int32_t min_layers,
                                          homln_subset_result *out, int32_t capacity, int32_t *count_out);

/* Accuracy of `pred` against `truth` (node-id lists, host or device, duplicates ignored),
 * over the handle's node set. Errors: EINVAL (negative length, id outside [0, n)), ENOMEM, ECUDA. */
HOMLN_API homln_status homln_accuracy(homln_t h, const int32_t *pred, int32_t n_pred, const int32_t *truth,
                            int32_t n_truth, homln_accuracy_t *out);

/* Accuracy without device allocation (the paper has no counterpart: this is an interface
 * for callers that cannot call cudaMalloc, e.g. because another allocator already owns the
 * GPU's memory or because their loop must never enter an allocator; every handle-based call
 * allocates, so this one takes no handle).
 *   n_nodes      node universe, 1 <= n_nodes <= HOMLN_NOALLOC_MAX_NODES (larger: EINVAL).
 *   pred, truth  int32 node-id lists in device memory of the CURRENT device, or managed memory
 *                (host pointers, or another GPU's memory: EINVAL); duplicates ignored.
 *   stream       cudaStream_t to run on (NULL = legacy default stream).
 *   out          host output; the call synchronises `stream` before returning.
 * Same results as homln_accuracy. Scratch is one static device array (two 2^20-bit bitmaps
 * and a few counters, about 256 KB) that every GPU loading the library keeps until exit; it
 * allocates nothing and calls no allocating routine. The first call on a device looks up the
 * array's address (cudaGetSymbolAddress) with that device current, so make that first call
 * before any stream capture. All calls share the array and each clears what it uses: calls
 * that overlap on the GPU (other streams or threads) race -- serialise them. */
#define HOMLN_NOALLOC_MAX_NODES 1048576
HOMLN_API homln_status homln_accuracy_noalloc(int32_t n_nodes, const int32_t *pred, int32_t n_pred,
                                              const int32_t *truth, int32_t n_truth, void *stream,
                                              homln_accuracy_t *out);

/* Measurement support (no counterpart in the paper; used by the benchmark).
 * homln_set_profiling: timing != 0 records CUDA events on the handle's stream right
 * around every BFS kernel launch; instrument != 0 runs the BFS kernels in a
 * counting variant (levels, edges scanned, words gathered) -- slower, for an
 * untimed pass that measures the algorithmic work. Both apply to later analyses.
 * homln_get_profile synchronises the stream and sums what was recorded since
 * the last homln_reset_profile. */
typedef struct homln_profile_t {
    int64_t bfs_launches;       /* all-sources BFS kernels launched */
    int64_t bfs_timed_launches; /* of which event-timed */
    double bfs_ms;              /* summed device time of the timed launches */
    int64_t levels, pull_levels, push_levels, batches; /* instrumented runs only */
    int64_t edges_scanned;      /* bottom-up neighbour visits (per vertex) */
    int64_t words_gathered;     /* 8-byte frontier words read by bottom-up levels */
    int64_t edges_pushed;       /* top-down neighbour visits */
    int64_t words_pushed;       /* 8-byte atomic ORs of top-down levels */
    int64_t bytes;              /* bytes the BFS kernels' loads and stores request (a load shared by the
                                   lanes of one vertex counted once): the algorithmic bytes */
    int64_t visits;             /* vertex visits: non-skipped vertices processed, summed over levels */
    int32_t words_per_node;     /* W of the last instrumented launch */
    int32_t teams;              /* teams of the last instrumented launch */
} homln_profile_t;

/* Preemption of the persistent BFS, for serving (the paper has no counterpart: it concerns how
 * several requests share one GPU). A yield flag is one int32 in pinned host memory that the GPU
 * reads directly.
 *   homln_yield_create   allocate a flag, lowered (0). Errors: EINVAL (out NULL), ECUDA.
 *   homln_yield_destroy  free it (NULL is accepted). Errors: EBUSY while a handle still watches it;
 *                        homln_set_yield(h, NULL) or homln_destroy(h) ends the watching.
 *   homln_yield_set      raise (nonzero) or lower (0) the flag; callable from any host thread.
 *   homln_yield_count    how many times BFS launches watching the flag stopped early for it.
 *   homln_set_yield      the persistent BFS of calls led by handle h (its analyses, and batches
 *                        whose first handle is h) watches flag y (NULL: none). While y is raised
 *                        the BFS hands out no new (graph, batch) tile: the running launch ends
 *                        after the tiles it has started, the calling host thread waits until y
 *                        is lowered (at most 60 s, then HOMLN_ETIMEOUT), and a new launch resumes
 *                        the remaining tiles. Results are identical. Such calls wait for each BFS
 *                        launch to end before returning, and a handle that watches a flag cannot
 *                        be captured in a CUDA graph (EINVAL). homln_set_tuning keeps the flag.
 * Typical use: the worker of large requests watches the flag; the worker of small requests raises
 * it while its own wave runs, so small requests do not wait for a large one to finish. */
HOMLN_API homln_status homln_yield_create(homln_yield_t *out);
HOMLN_API homln_status homln_yield_destroy(homln_yield_t y);
HOMLN_API homln_status homln_yield_set(homln_yield_t y, int32_t raised);
HOMLN_API homln_status homln_yield_count(homln_yield_t y, int64_t *out);
HOMLN_API homln_status homln_set_yield(homln_t h, homln_yield_t y);

HOMLN_API homln_status homln_set_profiling(homln_t h, int32_t timing, int32_t instrument);
HOMLN_API homln_status homln_get_profile(homln_t h, homln_profile_t *out);
HOMLN_API homln_status homln_reset_profile(homln_t h);
/* Number of kernels this library has launched in the process so far. */
HOMLN_API int64_t homln_kernel_launches(void);

/* Checkpoint of the Psi step (Section 3 keeps each layer's analysis results for every later
 * composition): the partial results of one graph -- which = layer id, -1 for the AND graph or
 * -2 for the OR graph of layer_mask -- analysed first if needed.
 *   farness[n] (uint64), reach[n] (uint32): as homln_layer_closeness; degree[n] (int32, may
 *   be NULL): the degree used by CC1 (the in-degree when directed). Host or device memory.
 * Errors: EINVAL, ENOMEM, ECUDA, ETIMEOUT. */
HOMLN_API homln_status homln_export_partials(homln_t h, int32_t which, uint64_t layer_mask, uint64_t *farness,
                                             uint32_t *reach, int32_t *degree);

/* One shard of the analysis of graph `which` (as in homln_export_partials), for splitting it
 * over several GPUs or processes: the BFS from the source batches rank, rank + world,
 * rank + 2 world, ... only (a batch is 64 x words_per_node sources of the graph's BFS order).
 * farness[n] / reach[n] (uint64 / uint32, host or device) receive the partial sums over those
 * sources; summed element-wise over rank = 0 .. world-1 (an all-reduce) they are exactly the
 * graph's farness and reach, which homln_import_partials then takes as its analysis (Section 3
 * keeps analyses apart from compositions; the sum is exact integer arithmetic). The handle's
 * cached results are not touched. Errors: EINVAL (rank/world, which, the plain schedule),
 * ENOMEM, ECUDA, ETIMEOUT. */
HOMLN_API homln_status homln_shard_partials(homln_t h, int32_t which, uint64_t layer_mask, int32_t rank,
                                            int32_t world, uint64_t *farness, uint32_t *reach);

/* Resume from a checkpoint: take farness/reach (host or device, n entries each) as the analysis
 * of graph `which` (as in homln_export_partials) of this handle, which must hold the same layers
 * they were computed on; closeness, sumDist and degrees are derived from them and the handle's
 * CSRs, and later queries on that graph run no BFS. Cached selections of the graph are dropped.
 * Errors: EINVAL; ERANGE (some (F, R) no BFS on n nodes can produce: R > n-1, F < R,
 * F > R (n-1)) -- the graph's previous results are then kept; ENOMEM, ECUDA. */
HOMLN_API homln_status homln_import_partials(homln_t h, int32_t which, uint64_t layer_mask, const uint64_t *farness,
                                             const uint32_t *reach);

/* Drop the cached Psi results (closeness, farness, selections) of every graph of the handle;
 * the CSRs and AND graphs stay. The next query recomputes them (used to re-measure). */
HOMLN_API homln_status homln_invalidate(homln_t h);

/* Wait for all work queued by the handle and report any device-side error it raised. */
HOMLN_API homln_status homln_sync(homln_t h);

/* Message describing the last error on the calling thread ("" if none). */
HOMLN_API const char *homln_last_error(void);

/* Library version string. */
HOMLN_API const char *homln_version(void);

#ifdef __cplusplus
}
#endif

#endif /* HOMLN_H */
