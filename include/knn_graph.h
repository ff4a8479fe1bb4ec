/*
 * knn_graph.h -- C ABI of the online k-nn graph library for one GB300
 * (sm_103a).
 *
 * The method is the online approximate k-nn graph of Debatty, Michiardi and
 * Mees, "Fast Online k-nn Graph Building" (KDD'16): each new point is placed
 * by an iGNNS graph search (Sec. 3) followed by the reverse Update walk
 * (Algorithm 2), as in the sequential build of Algorithm 1.  The initial graph
 * and the ground truth come from a brute-force exact k-nn graph (Sec. 2.1).
 *
 * Conventions shared by every call:
 *   - Similarity is sim(a, b) = 1 / (1 + ||a - b||_2) (the Euclidean distance
 *     of the paper's synthetic data, Sec. 8.1); higher is closer.  Every
 *     neighbour list is sorted best first; equal similarities go to the lower
 *     id.
 *   - Ids are dense insertion indices: the initial points are 0 .. n_init-1,
 *     the i-th inserted point gets the next free id.
 *   - Vectors are row-major float32 [m, dim].  Outputs are row-major.
 *   - Every pointer argument may be host memory (pageable or pinned) or
 *     device memory of the graph's device; the library tells them apart with
 *     cudaPointerGetAttributes and stages host buffers itself.  Pinned host
 *     memory gives asynchronous copies.  The caller owns every buffer it
 *     passes; the library owns the graph.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Work is
 *     ordered on it; device outputs are valid once the stream has reached the
 *     call, host outputs when the call returns (calls that write host memory
 *     synchronise the stream).
 *   - No call aborts.  Each returns a knn_status; on error, knn_last_error()
 *     gives a message for the calling thread.  A graph handle is not
 *     thread-safe: one thread (or external locking) per handle.
 */
#ifndef KNN_GRAPH_H
#define KNN_GRAPH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define KNN_API __attribute__((visibility("default")))
#else
#define KNN_API
#endif

typedef enum knn_status {
    KNN_OK = 0,
    KNN_ERR_INVALID_ARG = -1,    /* a bad size, pointer or parameter           */
    KNN_ERR_OOM = -2,            /* device memory admission refused            */
    KNN_ERR_CAPACITY = -3,       /* the graph or a batch would exceed its size */
    KNN_ERR_CUDA = -4,           /* a CUDA runtime call failed                 */
    KNN_ERR_DEVICE_TIMEOUT = -5, /* reserved: no call returns it.  The only
                                  * device waits are the tensor-core exact
                                  * build's, bounded; one that gives up is
                                  * counted in knn_exact_info.wait_errors and
                                  * its rows are settled on the CUDA cores  */
    KNN_ERR_NOT_FOUND = -6,      /* an id that is not in the graph             */
    KNN_ERR_UNSUPPORTED = -7     /* a size outside the compiled kernels        */
} knn_status;

typedef enum knn_storage {
    KNN_STORAGE_FP32 = 0,     /* searched in FP32                               */
    KNN_STORAGE_BF16 = 1,     /* screened in BF16, best candidates re-scored    */
    KNN_STORAGE_FP8_E4M3 = 2  /* screened in FP8-E4M3 with a per-row scale      */
} knn_storage;

/* Parameters of a graph.  The names follow the paper. */
typedef struct knn_params {
    int32_t dim;          /* vector dimension d, 1 .. 256                         */
    int32_t k;            /* neighbours per node, 1 .. 32 (Sec. 1)                */
    int32_t depth;        /* Update DEPTH (Algorithm 2), 1 .. 5                   */
    int32_t storage;      /* knn_storage of the searched copy                     */
    double speedup;       /* iGNNS budget: B = max(1, floor(n / speedup))
                             similarities per search (Sec. 3); > 0                */
    double expansion;     /* e > 1: a restart r is discarded when
                             sim(q, r) < s_max / e (Sec. 3); <= 0 or +inf
                             disables the test                                   */
    int32_t rescore_mult; /* screening forms: keep rescore_mult * k candidates
                             and re-score them in FP32; ignored for FP32         */
    int32_t max_batch;    /* largest m of one insert or query call, >= 1        */
    uint64_t seed;        /* seed of every restart draw                          */
    int64_t capacity;     /* most nodes the graph will ever hold                 */
} knn_params;

/* Running totals of a graph (Sec. 8.3 counts similarity computations). */
typedef struct knn_stats {
    int64_t n;               /* nodes in the graph                                 */
    int64_t capacity;
    int64_t removed;         /* nodes removed                                      */
    int64_t inserts;         /* points inserted after creation                     */
    int64_t queries;         /* queries answered                                   */
    int64_t search_evals;    /* similarities computed by iGNNS searches            */
    int64_t update_evals;    /* similarities computed by Update beyond level 1     */
    int64_t cross_evals;     /* similarities among the points of one insert batch  */
    int64_t rescore_evals;   /* FP32 re-scores of screening candidates             */
    int64_t restarts;        /* random restart nodes evaluated                     */
    int64_t moves;           /* eager hill-climbing moves                          */
    int64_t adjacency_reads; /* neighbour lists scanned by the climbs              */
    int64_t offers;          /* candidate (node, new) pairs merged by Update        */
    int64_t device_bytes;    /* device memory held by the graph                    */
    int64_t kernel_launches; /* kernels this library launched for the graph        */
} knn_stats;

/* Phases of an insert or query call, in order, for knn_graph_last_timing. */
typedef enum knn_phase {
    KNN_PHASE_STORE = 0,   /* copy in, pad and encode the new rows           */
    KNN_PHASE_SEARCH = 1,  /* iGNNS (Sec. 3), visited sets cleared first      */
    KNN_PHASE_RESCORE = 2, /* FP32 re-score of screening candidates           */
    KNN_PHASE_CROSS = 3,   /* similarities among the points of the batch; in
                              a single graph their top-k runs on a side stream
                              beside the search, so this phase times only the
                              merge with the search results              */
    KNN_PHASE_OFFERS = 4,  /* Update levels 1..DEPTH: candidates per node      */
    KNN_PHASE_MERGE = 5,   /* Update: merge candidates into the lists          */
    KNN_NUM_PHASES = 6
} knn_phase;

typedef struct knn_graph knn_graph; /* opaque, owned by the library */

/* Hill-climbing rule of a search (Sec. 3). */
typedef enum knn_climb {
    KNN_CLIMB_EAGER = 0, /* iGNNS: move to the first neighbour, in list order,
                            strictly more similar than the current node      */
    KNN_CLIMB_BEST = 1   /* GNNS (Sec. 2.2): evaluate every unvisited
                            neighbour, move to the most similar one (ties to
                            the earlier position) if it beats the current node */
} knn_climb;

/*
 * Create a graph from n_init >= k+1 points and build their exact k-nn graph
 * by brute force (Sec. 2.1; the initial graph of Sec. 8.5 is built the same
 * way).  init_vecs: [n_init, dim] float32.  Allocates all device memory the
 * graph will need for `capacity` nodes and `max_batch`-sized calls; returns
 * KNN_ERR_OOM if the device lacks it.  *out receives the handle.
 */
KNN_API knn_status knn_graph_create(const knn_params *params, const float *init_vecs,
                                    int64_t n_init, void *stream, knn_graph **out);

/*
 * Re-create a graph from a snapshot instead of building its exact graph:
 * n points and their adjacency lists, e.g. written by knn_graph_get_edges
 * (checkpoint and resume; not in the paper).  vecs: [n, dim] float32;
 * nbr_ids: [n, k] int64, each row best first, -1 for an empty slot.  Each
 * list keeps the order given; the similarities of its entries are
 * recomputed on the device.  KNN_ERR_INVALID_ARG if an id is outside
 * -1 .. n-1 or a node lists itself.  Sizes and memory as knn_graph_create.
 */
KNN_API knn_status knn_graph_restore(const knn_params *params, const float *vecs, int64_t n,
                                     const int64_t *nbr_ids, void *stream, knn_graph **out);

/*
 * Insert m points (1 <= m <= max_batch), Algorithm 1 for a batch: every point
 * is searched with iGNNS against the graph as it stood before the call, using
 * the restart stream equal to its new id; the exact similarities among the m
 * points are merged into their lists (the batch analogue of each point seeing
 * the ones before it); then Update (Algorithm 2) offers each new point to
 * its neighbours and their neighbours up to DEPTH.  vecs: [m, dim] float32.
 * out_ids (nullable): [m] int64 ids given to the points.
 * out_nbrs (nullable): [m, k] int64, the neighbour list each new point got.
 * KNN_ERR_CAPACITY if n + m > capacity.
 */
KNN_API knn_status knn_graph_insert_batch(knn_graph *g, const float *vecs, int64_t m,
                                          int64_t *out_ids, int64_t *out_nbrs, void *stream);

/*
 * Answer m queries (1 <= m <= max_batch) with iGNNS (Sec. 3) against the
 * current graph, without changing it.  Query i uses restart stream
 * 2^63 + query_id0 + i, so a request's result depends only on the graph, the
 * seed and its id, not on the batch it travels in.  vecs: [m, dim] float32.
 * out_ids: [m, k_out] int64 (-1 where fewer were found); out_sims (nullable):
 * [m, k_out] float32 similarities.  1 <= k_out <= k.
 */
KNN_API knn_status knn_graph_query_batch(knn_graph *g, const float *vecs, int64_t m,
                                         int32_t k_out, uint64_t query_id0,
                                         int64_t *out_ids, float *out_sims, void *stream);

/*
 * knn_graph_query_batch (iGNNS, Sec. 3) with one restart stream per query: query i uses
 * stream 2^63 + query_ids[i] (query_ids: [m] uint64, host or device), so a
 * query's result depends only on the graph it sees, its vector and its id --
 * not on the other queries of the call.  Arguments and errors otherwise as
 * knn_graph_query_batch.
 */
KNN_API knn_status knn_graph_query_ids(knn_graph *g, const float *vecs, int64_t m, int32_t k_out,
                                       const uint64_t *query_ids, int64_t *out_ids, float *out_sims,
                                       void *stream);

/*
 * Partitioned search (Sec. 5, Algorithm 3): every query is searched
 * independently in each of `parts` partitions of the graph, then the k_out
 * most similar of the parts * k_out candidates are kept.  Partition j is
 * the node range part_offsets[j] .. part_offsets[j+1] - 1 (int64, host or
 * device, [parts + 1], nondecreasing from 0 to n: for instance the clusters
 * of knn_balanced_kmedoids after the points were stored in its order); its
 * search is iGNNS (or the climb set by knn_graph_set_search) restricted to
 * the subgraph: restart draws among its nodes, neighbour-list entries
 * outside it not followed, budget max(1, floor(size / speedup)), so that the
 * parts together compute about n / speedup similarities; its restart stream
 * is 2^63 + query_id0 + i + j * 2^56 for query i.  Screening forms keep
 * rescore_mult * k_out candidates per part and re-score the merged best
 * rescore_mult * k_out in FP32.  knn_graph_last_counters then holds per
 * query the sums over its parts.  1 <= parts <= min(KNN_MAX_PARTS,
 * max_batch); other arguments and errors as knn_graph_query_batch.
 */
#define KNN_MAX_PARTS 1024
KNN_API knn_status knn_graph_query_partitioned(knn_graph *g, const float *vecs, int64_t m, int32_t k_out,
                                               uint64_t query_id0, const int64_t *part_offsets,
                                               int32_t parts, int64_t *out_ids, float *out_sims,
                                               void *stream);

/*
 * knn_graph_query_partitioned with one restart stream per query, as
 * knn_graph_query_ids: query i of partition j uses stream
 * 2^63 + query_ids[i] + j * 2^56 (query_ids: [m] uint64, host or device), so
 * a query's result depends only on the graph, its vector, its id and the
 * partitions -- the form the continuous-batching server uses.
 */
KNN_API knn_status knn_graph_query_partitioned_ids(knn_graph *g, const float *vecs, int64_t m, int32_t k_out,
                                                   const uint64_t *query_ids, const int64_t *part_offsets,
                                                   int32_t parts, int64_t *out_ids, float *out_sims,
                                                   void *stream);

/*
 * Distributed online build (Sec. 7, Algorithm 5) on one device.  The graph's
 * n nodes are split in `parts` partitions by labels [n] (int32, 0..parts-1,
 * host or device), each with a medoid (medoids [parts], node ids, host or
 * device): for instance knn_balanced_kmedoids' clusters, in any node order.
 * The state lives on the device with the graph, sized for its capacity.
 * recompute_interval >= 0: the medoids are recomputed (Algorithm 4's update
 * step: in every non-empty partition the member with the smallest sum of
 * Euclidean distances to the other members, ties to the lower id) after each
 * insert batch that leaves the graph at least recompute_interval * n_last
 * nodes larger than it was at the last recompute (n_last: its size at this
 * call, then at each recompute); 0 never recomputes.  Returns
 * KNN_ERR_INVALID_ARG for labels or medoids out of range,
 * KNN_ERR_UNSUPPORTED for parts outside 1..min(KNN_MAX_PARTS, max_batch) or a
 * graph with removed nodes, KNN_ERR_OOM when the state does not fit.
 * Synchronises `stream`.
 */
KNN_API knn_status knn_graph_set_partitions(knn_graph *g, const int32_t *labels, const int64_t *medoids,
                                            int32_t parts, double recompute_interval, void *stream);

/*
 * Algorithm 5 for a batch of m new points (as knn_graph_insert_batch, whose
 * arguments, outputs and errors it shares): the search of every new point is
 * the distributed search (Algorithm 3) over the partitions -- partition j is
 * searched on its own subgraph (its nodes in id order, the entries of their
 * lists inside it; restart draws among its nodes, budget
 * max(1, floor(size / speedup)), restart stream new id + j * 2^56), and the k
 * most similar of all the partitions' candidates are kept, ties to the lower
 * id.  The batch then joins the graph as in knn_graph_insert_batch (its own
 * similarities and Update, Algorithm 2, over the whole graph), every new node
 * is given to the partition of its most similar medoid (ties to the lower
 * partition), and the medoids are recomputed when recompute_interval says
 * so.  With one partition this is knn_graph_insert_batch.  Requires
 * knn_graph_set_partitions; KNN_ERR_UNSUPPORTED once nodes were removed.
 * Synchronises `stream` (the partition sizes are read on the host).
 */
KNN_API knn_status knn_graph_insert_distributed(knn_graph *g, const float *vecs, int64_t m, int64_t *out_ids,
                                                int64_t *out_nbrs, void *stream);

/*
 * The partition state of Algorithm 5 (Sec. 7): labels [n] (int32), medoids [parts] (node ids) and
 * the number of medoid recomputes so far, each nullable, host or device
 * buffers.  KNN_ERR_INVALID_ARG without knn_graph_set_partitions.
 * Synchronises `stream`.
 */
KNN_API knn_status knn_graph_get_partitions(knn_graph *g, int32_t *labels, int64_t *medoids, int64_t *recomputes,
                                            void *stream);

/*
 * Remove m nodes (not in the paper).  Removed nodes are never drawn, climbed
 * to, returned or offered again; lists that still hold them keep the entry.
 * KNN_ERR_NOT_FOUND if an id is outside 0 .. n-1.  ids: [m] int64.
 */
KNN_API knn_status knn_graph_remove(knn_graph *g, const int64_t *ids, int64_t m,
                                    void *stream);

/*
 * Copy out the adjacency lists of nodes 0 .. min(n, n_cap)-1: the k-nn graph
 * the online build maintains (Sec. 1), e.g. to count its correct edges
 * against an exact graph (Sec. 8.5) or to snapshot it for knn_graph_restore.
 * out_ids: [n_cap, k] int64 (-1 for an empty slot); out_sims (nullable):
 * [n_cap, k] float32.  *n_out (host) receives the number of rows written.
 */
KNN_API knn_status knn_graph_get_edges(knn_graph *g, int64_t *out_ids, float *out_sims,
                                       int64_t n_cap, int64_t *n_out, void *stream);

/*
 * Per-item counters of the last insert or query call: for each of its m
 * items, 8 int64 values: search similarities (iGNNS budget spent), Update
 * similarities (levels >= 2), restarts evaluated, restarts discarded by the
 * expansion test, eager moves, neighbour lists scanned, restart draws made
 * (free redraws included), and 0.  out: [m, 8] int64; m <= the last call's m.
 */
KNN_API knn_status knn_graph_last_counters(knn_graph *g, int64_t *out, int64_t m,
                                           void *stream);

/*
 * Per-phase timing with CUDA events recorded on the call's stream around
 * each phase of every later insert and query call (enable = 1), or none
 * (enable = 0, the default).
 */
KNN_API knn_status knn_graph_set_timing(knn_graph *g, int32_t enable);

/*
 * Milliseconds each knn_phase took in the last insert or query call
 * (synchronises that call's stream; phases the call did not run read 0).
 * out_ms: host [n] float, n <= KNN_NUM_PHASES.  KNN_ERR_INVALID_ARG if
 * timing is off.
 */
KNN_API knn_status knn_graph_last_timing(knn_graph *g, float *out_ms, int32_t n);

/*
 * Change the search parameters of a graph for its later inserts and queries
 * (iGNNS, Sec. 3; the GNNS climb it is compared with, Sec. 2.2 and Sec. 8.2):
 * speedup (budget B = max(1, floor(n / speedup))), expansion e (<= 0 or
 * +inf: no expansion test) and climb (knn_climb).  GNNS as the paper
 * compares it with iGNNS is climb = KNN_CLIMB_BEST with expansion = +inf; it
 * keeps iGNNS's budget, restart draws and visited set, so the two compare at
 * equal similarity evaluations.  Errors: KNN_ERR_INVALID_ARG for a
 * non-finite or non-positive speedup, a NaN expansion or an unknown climb.
 */
KNN_API knn_status knn_graph_set_search(knn_graph *g, double speedup, double expansion, int32_t climb);

/* Running totals (synchronises the graph's last stream). */
KNN_API knn_status knn_graph_stats(knn_graph *g, knn_stats *out);

/* Release the graph and all its device memory.  NULL is a no-op. */
KNN_API void knn_graph_destroy(knn_graph *g);

/*
 * Brute-force exact k-nn graph of n points (Sec. 2.1: every pairwise
 * similarity, keep the k best per node, ties to the lower id), without a
 * graph handle: the initial graph and the ground truth of Sec. 8.5.
 * X: [n, dim] float32, n >= k+1, 1 <= k <= 32.  out_ids: [n, k] int64;
 * out_sims (nullable): [n, k] float32.  Allocates its own temporaries.
 */
KNN_API knn_status knn_exact_graph(const float *X, int64_t n, int32_t dim, int32_t k,
                                   int64_t *out_ids, float *out_sims, void *stream);

/*
 * How the brute-force exact graph (knn_exact_graph and the initial graph of
 * knn_graph_create) is computed.  Both give the exact lists up to FP32
 * rounding of the distances.
 *   KNN_EXACT_AUTO          tensor cores when supported (dim <= 128,
 *                           n >= 128), CUDA cores otherwise (default);
 *   KNN_EXACT_CUDA_CORES    FP32 differences on CUDA cores for every pair;
 *   KNN_EXACT_TENSOR_CORES  tensor cores, or KNN_ERR_UNSUPPORTED when the
 *                           call does not qualify.
 * The tensor-core path screens every pair with split-BF16 dot products
 * (hi.hi + hi.lo + lo.hi, FP32 accumulation), keeps 32 candidates per node,
 * re-scores them in FP32 and recomputes by brute force every node for which
 * a proven bound on the screening error cannot exclude a better
 * non-candidate; it reads back three counters and so synchronises the
 * stream before returning.  The setting is process-wide.
 */
typedef enum knn_exact_path {
    KNN_EXACT_AUTO = 0,
    KNN_EXACT_CUDA_CORES = 1,
    KNN_EXACT_TENSOR_CORES = 2
} knn_exact_path;

KNN_API knn_status knn_exact_set_path(int32_t path);

/* What the calling thread's last exact build did. */
typedef struct knn_exact_info {
    int32_t path;          /* KNN_EXACT_CUDA_CORES or KNN_EXACT_TENSOR_CORES          */
    uint32_t wait_errors;  /* tensor-core pipeline waits that gave up (rows redone)  */
    int64_t n;             /* nodes                                                   */
    int64_t rows_redone;   /* nodes settled by the FP32 brute-force pass             */
} knn_exact_info;

KNN_API knn_status knn_exact_last_info(knn_exact_info *out);

/*
 * Failure detection of the tensor-core build: every wait of one of its
 * pipeline roles on another gives up after `ns` nanoseconds (default 2 s;
 * ns < 0 restores it), records the wait in knn_exact_info.wait_errors and
 * sends the rows of that block to the FP32 pass, which keeps the lists
 * exact.  A block always waits for its own copies and MMAs before it exits.
 * Process-wide; meant for tests (ns = 0 makes every pipeline wait that is
 * not already satisfied give up).
 */
KNN_API knn_status knn_exact_set_wait_limit(int64_t ns);

/*
 * Grow a graph to hold `capacity` nodes (nothing happens if it already
 * does), keeping its nodes, lists, removals and counters.  The paper has no
 * counterpart: its graph takes a flow of points without a stated bound
 * (Sec. 1), and this lets the device graph follow that flow as far as
 * device memory allows instead of stopping at the capacity fixed at
 * creation.  The per-node arrays (rows, screening copy, lists, removal bits,
 * Update chain heads, the visited sets of one batch) are allocated anew for
 * `capacity` and the nodes copied over, so the new arrays' bytes must be free
 * on top of the old ones, plus `headroom_bytes` (>= 0) that must stay free
 * afterwards; otherwise KNN_ERR_OOM and the graph is unchanged.  capacity
 * must be below 2^31 (KNN_ERR_CAPACITY).  Waits for every stream the graph
 * used and for `stream`, and returns when the graph is ready.
 */
KNN_API knn_status knn_graph_reserve(knn_graph *g, int64_t capacity, int64_t headroom_bytes, void *stream);

/*
 * The query search of knn_graph_query_batch (iGNNS, Sec. 3; FP32 rows, no removed nodes)
 * over a graph held in the caller's own device buffers, without any device
 * allocation.  The paper has no counterpart: this exists for callers that
 * cannot allocate device memory -- a process whose device memory is owned by
 * another allocator or reserved up front, or a loop that cannot afford the
 * device-wide synchronisation an allocation may cause -- and that therefore
 * cannot create a knn_graph.
 *
 * rows: [n, dim] float32; dim must be 16, 32, 64, 96, 128 or 256 (rows are
 * used as they are, without padding).  nbr_ids: [n, k] int32 lists, best
 * first, -1 for an empty slot; an entry outside 0..n-1 is treated as an
 * empty slot (never followed, never read as a row).  queries: [m, dim]
 * float32.  out_ids: [m, k_out] int64; out_sims (nullable): [m, k_out]
 * float32.  Every buffer must be device memory of the current device
 * (nothing is staged); rows and queries must start on a 16-byte boundary
 * (they are read with 16-byte loads) and the other buffers on a multiple of
 * their element size: anything else returns KNN_ERR_INVALID_ARG before any
 * device work.  Query i uses restart stream 2^63 + query_id0 + i and budget
 * max(1, floor(n / speedup)), so it returns exactly what
 * knn_graph_query_batch returns for the same graph and query id.
 *
 * Temporaries live in a 16 MiB array inside the library (every GPU that
 * loads the library keeps it until the process exits).  A call needs
 * m * (8 * k_out + 64) + n / 8 bytes of it, rounded up per part, and, once
 * n exceeds 225,280 (the visited sets of a block's queries no longer fit in
 * shared memory), about m * n / 8 bytes more; it returns KNN_ERR_CAPACITY,
 * before any device work, when that exceeds 16 MiB.  The
 * first call on a device looks up the array's device address (make that
 * first call before any stream capture).  All calls share the array: calls
 * that overlap on the GPU race; order them on one stream.  Returns after
 * enqueueing; outputs are valid once the stream reaches the call.
 */
KNN_API knn_status knn_search_noalloc(const float *rows, int64_t n, int32_t dim,
                                      const int32_t *nbr_ids, int32_t k, const float *queries,
                                      int64_t m, int32_t k_out, double speedup, double expansion,
                                      uint64_t seed, uint64_t query_id0, int64_t *out_ids,
                                      float *out_sims, void *stream);

/*
 * Balanced k-medoids (Sec. 6, Algorithm 4) of n points, for a node ordering
 * that makes clusters contiguous and for the partitions of the partitioned
 * search (Algorithm 3, knn_graph_query_partitioned).
 *
 * X: [n, dim] float32, host or device; 1 <= dim <= 256.  p clusters,
 * 1 <= p <= 1024, p <= n < 2^31, n * p <= 2^32.  The initial medoids are the
 * first p distinct nodes drawn with the restart generator keyed
 * (seed, 2^62).  The points are split in `chunks` chunks of consecutive ids
 * (the paper's compute nodes, 1 <= chunks <= n); within a chunk, in id
 * order, a point goes to the medoid m maximising sim(m, x) * w(t, m) with
 * w(t, m) = 1 - |C_t(m)| / capacity, capacity = n * imbalance / (p * chunks)
 * and |C_t(m)| the chunk's points given to m so far (ties to the lower
 * cluster); imbalance >= 1, +inf for no penalty.  `iters` rounds of (assign,
 * update) run before the final assign, the update giving every non-empty
 * cluster its member with the smallest sum of Euclidean distances to the
 * others (ties to the lower id).  Decisions are taken in FP32.
 *
 * Outputs (each nullable, host or device): labels [n] int32 (cluster of each
 * point); medoids [p] int64 (those of the final assign); order [n] int64
 * (point ids sorted by (cluster, id): position -> point); offsets [p + 1]
 * int64 (cluster m occupies order[offsets[m] .. offsets[m+1])).  Allocates
 * n * (p + dim + 4) * 4 bytes of temporaries and returns when the outputs
 * are written.
 */
KNN_API knn_status knn_balanced_kmedoids(const float *X, int64_t n, int32_t dim, int32_t p,
                                         double imbalance, int32_t chunks, int32_t iters,
                                         uint64_t seed, int32_t *out_labels, int64_t *out_medoids,
                                         int64_t *out_order, int64_t *out_offsets, void *stream);

/*
 * Continuous-batching server over one graph.  A worker thread owns the
 * graph: it forms device steps from the submitted requests in submission
 * order, admitting requests while their points fit the step's device slots
 * (max_step_points) and, for inserts, the graph's capacity; requests that
 * arrive while steps run join the next step as slots free up.  Two steps
 * are in flight: the host-to-device copy of step t+1 and the device-to-host
 * copy of step t-1 overlap step t's kernels (separate copy streams).
 *
 * A step runs the searches of all its queries and inserts against the graph
 * as it stood before the step (epoch E), then commits its inserts (epoch
 * E+1); searches never overlap an update.  Query point i of request r uses
 * restart stream 2^63 + r * 2^20 + i, so a query's result is a function of
 * (epoch, its vector, r, the graph's seed) alone: the same alone as in any
 * mix.  An insert's search uses its new node id as stream, and its batch
 * shares the intra-batch merge, so an insert's result depends on the mix
 * within the method's recall tolerance.
 */
typedef struct knn_server knn_server;

typedef struct knn_server_params {
    int32_t k_out;           /* neighbours returned per query point, 1..k           */
    int32_t max_step_points; /* points per step, 1..max_batch (0: max_batch)        */
    int64_t grow_headroom_bytes; /* admission by free device memory: when an insert
                                    does not fit the graph's capacity, the worker
                                    grows the graph (knn_graph_reserve, by half its
                                    capacity or to what the insert needs) as long
                                    as this many bytes stay free afterwards; an
                                    insert that cannot be admitted so fails with
                                    KNN_ERR_OOM.  0: the capacity is fixed and
                                    such an insert fails with KNN_ERR_CAPACITY    */
    int32_t query_parts;     /* > 1: queries run the partitioned search
                                (knn_graph_query_partitioned_ids) over the parts
                                given by part_offsets, the last part stretched to
                                the nodes inserted since; a query's result is then
                                a function of (epoch, vector, request, point,
                                parts).  0 or 1: the plain search            */
    int32_t reserved;        /* 0                                                    */
    const int64_t *part_offsets; /* [query_parts + 1] host int64 node offsets of
                                    the graph at server creation, nondecreasing
                                    from 0 to its n (copied at creation)        */
} knn_server_params;

typedef enum knn_request_kind { KNN_REQ_INSERT = 0, KNN_REQ_QUERY = 1 } knn_request_kind;

typedef struct knn_request_info {
    int32_t status;     /* KNN_OK, or the error that failed the request             */
    int32_t kind;       /* knn_request_kind                                          */
    int64_t m;          /* points                                                    */
    int64_t epoch;      /* graph version its searches saw (insert steps before it)  */
    int64_t step;       /* device step that ran it                                   */
    double queue_ms;    /* submission -> admitted into a step                        */
    double latency_ms;  /* submission -> results on the host                         */
} knn_request_info;

typedef struct knn_server_stats {
    int64_t steps, requests, points, inserts, queries;
    int64_t epoch;              /* insert steps committed                             */
    int64_t max_queue;          /* most requests waiting at once                      */
    double busy_ms;             /* device time of all steps (CUDA events)            */
    int64_t grows;              /* times the graph was grown for admission            */
    int64_t capacity;           /* the graph's capacity now                          */
} knn_server_stats;

/* Start a server on g (which it then owns until knn_server_destroy: make no
 * other call on g meanwhile).  Allocates its device slots (two steps of
 * max_step_points points) and pinned host staging. */
KNN_API knn_status knn_server_create(knn_graph *g, const knn_server_params *p, knn_server **out);

/* Enqueue a request of m points (vecs: [m, dim] float32 host memory, copied
 * before returning), 1 <= m <= min(max_step_points, 2^20).  *request_id gets
 * its id: 0, 1, 2, ... in submission order.  Thread-safe. */
KNN_API knn_status knn_server_submit(knn_server *s, int32_t kind, const float *vecs, int64_t m,
                                     uint64_t *request_id);

/* Block until the request has finished, then copy its results to host
 * memory: a query's ids [m, k_out] int64 and sims [m, k_out] float32, an
 * insert's new node ids [m] (sims unused).  Each argument is nullable; a
 * request's results can be taken once.  Thread-safe. */
KNN_API knn_status knn_server_wait(knn_server *s, uint64_t request_id, int64_t *out_ids,
                                   float *out_sims, knn_request_info *info);

KNN_API knn_status knn_server_get_stats(knn_server *s, knn_server_stats *out);

/* Finish every submitted request, stop the worker and free the server (the
 * graph stays alive and usable again). */
KNN_API void knn_server_destroy(knn_server *s);

/*
 * Several independent graphs served together: G graphs of uneven sizes live
 * in one device arena (graph i owns capacity[i] node slots), and a step
 * takes a mixed batch of insert and query items for any of them.  Every
 * item's search runs against its own graph as it stood before the step
 * (budget max(1, floor(n_i / speedup)), restart draws among its nodes), the
 * inserts of one graph meet each other in the intra-batch merge and Update
 * offers them to that graph's older nodes only -- so each graph evolves
 * exactly as a knn_graph given the same items would.  All the step's kernels
 * run with fixed grids and read the step's sizes from device tables, so one
 * launch sequence serves every step; with use_graph it is captured once into
 * a CUDA graph (at the second step) and replayed.
 *
 * knn_multi_create: params as knn_graph_create (max_batch = items per step;
 * capacity is ignored); n_init, capacity: [graphs] with k+1 <= n_init[i] <=
 * capacity[i], sum of capacities < 2^31; init_vecs: [sum n_init, dim] float32
 * host or device, graph after graph; each initial graph is exact.
 *
 * knn_multi_step: m items (1..max_batch), all host memory: vecs [m, dim]
 * float32, graph [m] int32, kind [m] int32 (knn_request_kind), query_ids [m]
 * uint64 (used for queries: stream 2^63 + id).  out_ids [m, k] int64: a
 * query's k best (ids local to its graph), an insert's new local id in
 * column 0 (-1 after); out_sims [m, k] float32 (nullable; 0 for inserts).
 * Returns when the outputs are written.  KNN_ERR_CAPACITY if a graph would
 * overflow (nothing is done).
 */
typedef struct knn_multi knn_multi;

KNN_API knn_status knn_multi_create(const knn_params *params, int32_t graphs, const int64_t *n_init,
                                    const int64_t *capacity, const float *init_vecs, int32_t use_graph,
                                    void *stream, knn_multi **out);
KNN_API knn_status knn_multi_step(knn_multi *mg, const float *vecs, const int32_t *graph,
                                  const int32_t *kind, const uint64_t *query_ids, int64_t m,
                                  int64_t *out_ids, float *out_sims, void *stream);
/* Warps of the search launch of later steps (0: one per item slot, i.e.
 * max_batch).  The search loops over the step's items with that many warps;
 * fewer than the items makes the launch persistent.  For the autotuner. */
KNN_API knn_status knn_multi_set_launch(knn_multi *mg, int32_t search_warps);
/* Order in which the search launch of later steps takes a step's items:
 * largest_first = 0 as packed (inserts grouped by graph, then queries), 1
 * the items of the largest graphs first.  A search's length grows with its
 * graph's size (its budget is n / speedup), so with a persistent launch the
 * longest searches then start in the first round instead of the last.  The
 * results do not depend on it.  For the autotuner; KNN_ERR_INVALID_ARG for a
 * value other than 0 or 1. */
KNN_API knn_status knn_multi_set_order(knn_multi *mg, int32_t largest_first);
/* Nodes and capacity of graph `graph`. */
KNN_API knn_status knn_multi_graph_size(knn_multi *mg, int32_t graph, int64_t *n, int64_t *capacity);
/* Lists of graph `graph`: out_ids [n, k] int64 local ids (host or device). */
KNN_API knn_status knn_multi_get_edges(knn_multi *mg, int32_t graph, int64_t *out_ids, void *stream);
KNN_API void knn_multi_destroy(knn_multi *mg);

/* Message of the last failed call on this thread ("" if none). */
KNN_API const char *knn_last_error(void);

/* Library version string. */
KNN_API const char *knn_version(void);

#ifdef __cplusplus
}
#endif
#endif /* KNN_GRAPH_H */
