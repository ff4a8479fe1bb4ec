// kernels.h -- argument blocks and launchers of the library's CUDA kernels
// (internal; the public interface is include/knn_graph.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "knn_graph.h"

namespace knn {

// Per-item counters written by the search and update kernels.
enum Counter : int {
    CTR_SEARCH_EVALS = 0,  // similarities computed by iGNNS
    CTR_UPDATE_EVALS = 1,  // Update similarities beyond level 1
    CTR_RESTARTS = 2,      // restart nodes evaluated
    CTR_DISCARDED = 3,     // restarts discarded by the expansion test
    CTR_MOVES = 4,         // eager hill-climbing moves
    CTR_ADJ_READS = 5,     // neighbour lists scanned
    CTR_DRAWS = 6,         // restart draws made, free redraws included
    CTR_PAD = 7,
    NCTR = 8
};

// Device-wide running totals (unsigned long long, atomically added).
enum Total : int {
    TOT_SEARCH_EVALS = 0,
    TOT_UPDATE_EVALS,
    TOT_CROSS_EVALS,
    TOT_RESCORE_EVALS,
    TOT_RESTARTS,
    TOT_MOVES,
    TOT_ADJ_READS,
    TOT_OFFERS,
    TOT_SEARCH_ROW_BYTES,  // bytes of stored rows gathered by searches
    NTOT = 16
};

enum ErrorFlag : unsigned {
    ERR_OFFER_OVERFLOW = 1u,
};

// Several graphs in one node arena (knn_multi_*).  Graph s owns the nodes
// lo[s] .. lo[s] + capacity - 1 and has n[s] nodes before a step; the
// step's new points of graph s are insert items first[s] .. first[s+1] - 1
// and take the ids lo[s] + n[s] + (item - first[s]).  A launch given an
// item_seg table reads its item count from *count and loops over its items
// with a fixed grid, so that one captured sequence of launches serves any
// step.
struct Segments {
    const int32_t *item_seg = nullptr;   // [items] graph of each item (nullptr: one graph)
    const uint32_t *lo = nullptr;        // [S] first node of each graph
    const uint32_t *n = nullptr;         // [S] nodes before the step
    const int32_t *first = nullptr;      // [S + 1] insert items of each graph
    const int32_t *count = nullptr;      // device item count of the launch
    const int32_t *order = nullptr;      // nullable: [items] the order the search takes them in
};

__host__ __device__ __forceinline__ uint32_t seg_new_id(const Segments &sg, int32_t s, int32_t item) {
    return sg.lo[s] + sg.n[s] + (uint32_t)(item - sg.first[s]);
}

struct SearchArgs {
    const uint8_t *rows;         // searched copy, row stride = row bytes of the encoding
    const float *row_scale;      // FP8: per-row scale
    const int32_t *nbr;          // adjacency [cap][k]
    const uint32_t *removed;     // bitset
    const float *queries;        // padded FP32 query rows
    int64_t q_stride;            // floats between query rows
    uint32_t *visited;           // [m][vwords] bitsets, zeroed before the launch
    int64_t vwords;
    uint64_t *out_keys;          // [m][KT] sorted (d2 bits << 32 | id)
    long long *counters;         // [m][NCTR]
    unsigned long long *totals;  // [NTOT]
    int32_t m, k, KT;
    uint32_t n;                  // visible nodes
    int64_t n_live;              // visible nodes not removed
    int64_t budget;              // B = max(1, floor(n / speedup))
    uint64_t max_draws;          // 64 n
    uint64_t seed;
    uint64_t stream_base;        // restart stream of item i = stream_base + i
    float expansion;
    int32_t discard;             // expansion test enabled
    int32_t climb;               // KNN_CLIMB_EAGER (iGNNS) or KNN_CLIMB_BEST (GNNS)
    // partitioned search (Algorithm 3): parts > 1 runs m * parts searches,
    // search s = query s / parts over the nodes part_off[p] .. part_off[p+1]-1
    // (p = s % parts) with budget max(1, floor(size / speedup)) and restart
    // stream stream_base + query + p * PART_STREAM_STEP; keys and counters
    // are then per search.  parts == 1: every node, budget and n_live as set.
    int32_t parts = 1;
    const int64_t *part_off = nullptr;   // [parts + 1] device
    const int64_t *part_live = nullptr;  // [parts] live nodes of each partition
    double speedup = 1.0;
    uint32_t vis_n = 0;                  // bits of one visited set (n, or the largest partition)
    const uint64_t *streams = nullptr;   // nullable: restart stream of query i (replaces stream_base + i)
    Segments seg;                        // several graphs: item i searches graph seg.item_seg[i]
    // nullable: with visited sets in global memory, the searches are taken one
    // at a time from this counter (zeroed by the launcher) by a grid of the
    // warps that fit on the GPU at once, so that a warp that ends early takes
    // the next search instead of idling until its block ends
    unsigned *work = nullptr;
};
constexpr uint64_t PART_STREAM_STEP = 1ull << 56;

struct RescoreArgs {
    const float *rows;           // FP32 padded rows
    const float *queries;
    int64_t q_stride;
    const uint64_t *cand_keys;   // [m][KT]
    uint64_t *out_keys;          // [m][k_out]
    unsigned long long *totals;
    int32_t m, KT, k_out;
    const int32_t *m_dev = nullptr;      // nullable: device item count (fixed grid, loop)
};

struct CrossArgs {
    const float *rows;           // FP32 padded rows; the batch is rows n .. n+m-1
    const uint64_t *in_keys;     // [m][k] search result of each new point
    uint64_t *cross_keys;        // [m][k] best k among the batch (split form)
    int32_t *nbr_ids;            // lists; rows n .. n+m-1 are written
    float *nbr_d2;
    unsigned long long *totals;
    int32_t m, k;
    uint32_t n;
    Segments seg;                        // several graphs: only points of one graph meet
};

struct UpdateArgs {
    const float *rows;
    const int32_t *nbr_ids;
    const float *nbr_d2;
    const uint32_t *removed;
    int32_t *head;               // [cap] offer chain heads, -1 = none
    uint64_t *offer_key;
    int32_t *offer_next;
    int32_t *touched;
    unsigned *offer_count;
    unsigned *touched_count;
    unsigned offer_cap;
    unsigned *error_flags;
    long long *counters;         // [m][NCTR]
    unsigned long long *totals;
    int32_t *frontier;           // [m][frontier_cap] nodes of the Update levels
    int64_t frontier_cap;        // min(nodes, k + k^2 + ... + k^DEPTH)
    uint32_t *seen;              // [m][seen_words] global seen bitsets (zeroed), if not on chip
    int64_t seen_words;          // ceil((n + m) / 32)
    int32_t m, k, depth;
    uint32_t n;                  // graph size before the batch
    Segments seg;                // several graphs: seen bits relative to the graph's first node
};

struct MergeArgs {
    int32_t *nbr_ids;
    float *nbr_d2;
    int32_t *head;
    const uint64_t *offer_key;
    const int32_t *offer_next;
    const int32_t *touched;
    const unsigned *touched_count;
    const unsigned *offer_count;
    unsigned long long *totals;
    int32_t k;
};

struct ExactArgs {
    const float *X;              // padded FP32 rows [n][DP]
    const uint32_t *removed;     // nullable
    int32_t *out_ids;            // [n][k]
    float *out_d2;
    int64_t n;
    int32_t k;
    // nullable: compute only the rows rows[0 .. *row_count) (device memory)
    const int32_t *rows = nullptr;
    const unsigned *row_count = nullptr;
    // > 1: the columns are split in this many segments, one block column
    // each; their lists go to `partial` ([row slot][segment][32] packed keys,
    // exact_partial_slots() row slots at most) and are merged afterwards
    int32_t col_segments = 1;
    uint64_t *partial = nullptr;
    // with `rows`: > 0, an upper bound of *row_count known on the host, which
    // sizes the grid (0: n)
    int64_t row_hint = 0;
};
// column segments that let a pass over `rows` listed rows fill the GPU, and
// the row slots x segments of partial lists that choice can need
int exact_col_segments(int64_t rows, int64_t n, int sm_count);
constexpr int64_t EXACT_PARTIAL_SLOTS = 64 * 2 * 2 * 160;

// supported padded dimensions
bool supported_dp(int dp);
int padded_dim(int d);  // smallest supported DP >= d, or -1

cudaError_t launch_search(int storage, int dp, const SearchArgs &a, cudaStream_t s);
// true when the search keeps visited sets in shared memory for a graph of n
// nodes (the global bitsets are then not read and need no clearing)
bool search_visited_on_chip(uint32_t n);
cudaError_t launch_rescore(int dp, const RescoreArgs &a, cudaStream_t s);
cudaError_t launch_cross(int dp, const CrossArgs &a, cudaStream_t s);
// the same lists in two launches (a single graph): the best k among the batch
// into cross_keys (needs no search result), then the merge with in_keys
cudaError_t launch_cross_topk(int dp, const CrossArgs &a, cudaStream_t s);
cudaError_t launch_cross_merge(const CrossArgs &a, cudaStream_t s);
cudaError_t launch_update(int dp, const UpdateArgs &a, cudaStream_t s);
cudaError_t launch_merge(const MergeArgs &a, int sm_count, cudaStream_t s);
// true when Update keeps its seen bitsets (seen_words words each) on chip
bool update_seen_on_chip(int64_t seen_words);
cudaError_t launch_exact(int dp, const ExactArgs &a, cudaStream_t s);
// tensor-core screening + FP32 settling (exact_tc.cu): usable when
// exact_tc_supported(); `scratch` holds exact_tc_scratch_bytes(n, dp) device
// bytes; *counters_out receives the device address of three words
// {largest norm, rows settled by brute force, wait-error bits}.  Reads the
// number of unsettled rows back, so it synchronises the stream once.
bool exact_tc_supported(int dp, int64_t n, int k, const uint32_t *removed);
// pipeline wait limit of the tensor-core build in ns (< 0: the default)
void exact_tc_set_wait(int64_t ns);
size_t exact_tc_scratch_bytes(int64_t n, int dp);
cudaError_t launch_exact_tc(int dp, const ExactArgs &a, void *scratch, unsigned **counters_out, cudaStream_t s);
// snapshot restore: copy int64 lists (checking every id) and recompute their d2
cudaError_t launch_restore_lists(int dp, const float *rows, const int64_t *in_ids, int64_t n, int k,
                                 int32_t *nbr_ids, float *nbr_d2, unsigned *bad, cudaStream_t s);

// several graphs in one arena (misc.cu): staged vectors to query rows and,
// for insert items, to their new nodes; query keys to outputs in caller
// order with graph-local ids; shifting an exact graph's local ids
cudaError_t launch_multi_append(const float *in, const int32_t *count_all, const Segments &ins, int d, int dp,
                                float *q_rows, float *rows, uint16_t *rows_bf16, uint8_t *rows_fp8, float *scale,
                                int grid, cudaStream_t s);
cudaError_t launch_multi_keys_out(const uint64_t *keys, const int32_t *count_q, const int32_t *count_ins, int kk,
                                  int k_out, const int32_t *item_seg, const uint32_t *lo, const int32_t *perm,
                                  int64_t *out_ids, float *out_sims, int grid, cudaStream_t s);
cudaError_t launch_shift_ids(int32_t *ids, int64_t count, int32_t add, cudaStream_t s);

// p[i] += v for i < m (misc.cu)
cudaError_t launch_add_u64(uint64_t *p, uint64_t v, int64_t m, cudaStream_t s);

// partitioned search: per query, the k_keep best of its parts * k_keep
// candidate keys ([m * parts][k_keep] -> [m][k_keep]) and the sums of its
// searches' counters ([m * parts][NCTR] -> [m][NCTR]) (misc.cu)
cudaError_t launch_merge_parts(const uint64_t *keys, int32_t m, int32_t parts, int32_t k_keep, uint64_t *out,
                               const long long *ctr_in, long long *ctr_out, cudaStream_t s);

// balanced k-medoids (kmedoids.cu); X are padded FP32 rows [n][dp]
constexpr int KMED_MAX_P = 1024;
// D[i][m] = squared distance of point i to medoid m ([n][p] floats)
cudaError_t launch_kmed_dist(int dp, const float *X, int64_t n, const int64_t *medoids, int p, float *D,
                             cudaStream_t s);
// the sequential weighted assignment, one warp per chunk of consecutive ids
cudaError_t launch_kmed_assign(const float *D, int64_t n, int p, int chunks, double capacity, int32_t *labels,
                               cudaStream_t s);
// stable counting sort by label: order[position] = id, offsets[p + 1]
size_t kmed_sort_scratch_bytes(int64_t n, int p);
cudaError_t launch_kmed_sort(const int32_t *labels, int64_t n, int p, void *scratch, int64_t *order,
                             int64_t *offsets, cudaStream_t s);
// medoid of every non-empty cluster (members order[offsets[m] .. offsets[m+1]))
cudaError_t launch_kmed_update(int dp, const float *X, const int64_t *order, const int64_t *offsets, int p,
                               int64_t *medoids, cudaStream_t s);

// distributed online build (partition.cu): staged copy of nodes 0..n-1 in
// partition order (pos = inverse of order; rows of row_bytes, a multiple of
// 16; scale nullable; list entries outside a node's partition -> -1)
cudaError_t launch_part_stage(const uint8_t *rows, int64_t row_bytes, const float *scale, const int32_t *nbr, int k,
                              const int32_t *label, const int64_t *order, int64_t *pos, int64_t n, uint8_t *st_rows,
                              float *st_scale, int32_t *st_nbr, cudaStream_t s);
// candidate keys of a staged search: position ids -> node ids (in place)
cudaError_t launch_part_keys_to_nodes(uint64_t *keys, int64_t count, const int64_t *order, cudaStream_t s);
// labels[i] = position of the medoid nearest to rows[i] (ties to the lower)
cudaError_t launch_part_nearest(const float *X, int dp, const float *rows, int64_t m, const int64_t *medoids, int p,
                                int32_t *labels, cudaStream_t s);

// shape of a graph for the server (graph.cu)
struct GraphShape {
    int dim, k, max_batch;
    int64_t n, capacity;
};
GraphShape graph_shape(const knn_graph *g);
// a stream the caller is about to destroy: synchronise it and stop using it
// as the graph's last stream (graph.cu)
void graph_forget_stream(knn_graph *g, cudaStream_t s);

// set the calling thread's knn_last_error() message (graph.cu)
knn_status record_error(knn_status st, const char *msg);

// small helpers (misc.cu)
cudaError_t launch_append(const float *in, int64_t m, int d, int dp, float *rows_fp32,
                          uint16_t *rows_bf16, uint8_t *rows_fp8, float *scale, cudaStream_t s);
cudaError_t launch_keys_to_output(const uint64_t *keys, int64_t m, int kk, int k_out,
                                  int64_t *out_ids, float *out_sims, cudaStream_t s);
cudaError_t launch_lists_to_output(const int32_t *ids, const float *d2, int64_t rows, int k,
                                   int64_t *out_ids, float *out_sims, cudaStream_t s);
cudaError_t launch_fill_ids(int64_t *out, int64_t first, int64_t m, cudaStream_t s);
cudaError_t launch_mark_removed(uint32_t *removed, const int64_t *ids, int64_t m, cudaStream_t s);
cudaError_t launch_fill_i32(int32_t *p, int32_t v, int64_t count, cudaStream_t s);

}  // namespace knn
