// graph.cu -- the C ABI of include/knn_graph.h: graph lifecycle, host/device
// staging, and the kernel pipeline of one insert or query batch.
//
// Device layout of a graph with capacity C, padded dimension DP, k neighbours
// and batches of at most M points:
//   X        [C][DP]  float32 rows (the exact copy; zero padded)
//   Xb / X8  [C][DP]  BF16 / FP8-E4M3 screening copy, scale [C] for FP8
//   nbr_ids  [C][k]   int32 adjacency, best first, -1 = empty slot
//   nbr_d2   [C][k]   float32 squared distances of those entries
//   removed  [C/32]   bitset of removed nodes
//   head     [C]      chain heads of Update candidates (-1 = none)
//   visited  [M][C/32] per-query visited bitsets, cleared per batch
//   plus per-batch keys, counters and the Update candidate pool
//   (M * (k + k^2) entries).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "knn_graph.h"
#include "common.cuh"
#include "kernels.h"

using namespace knn;

struct knn_graph {
    knn_params p;
    int device = 0;
    int sm_count = 0;
    int dp = 0;
    int KT = 0;            // candidates kept by an insert's search
    int64_t frontier_cap = 0;  // Update level entries kept per new point
    int64_t n = 0;
    int64_t n_removed = 0;
    int64_t inserts = 0, queries = 0;
    int64_t last_m = 0;
    int64_t vwords = 0;
    unsigned offer_cap = 0;
    size_t bytes = 0;
    std::vector<void *> allocations;
    std::vector<uint32_t> removed_host;

    float *X = nullptr;
    uint16_t *Xb = nullptr;
    uint8_t *X8 = nullptr;
    float *scale = nullptr;
    int32_t *nbr_ids = nullptr;
    float *nbr_d2 = nullptr;
    uint32_t *removed = nullptr;
    int32_t *head = nullptr;
    uint32_t *visited = nullptr;
    float *qbuf = nullptr;
    float *stage_in = nullptr;
    uint64_t *keys_search = nullptr;
    uint64_t *keys_final = nullptr;
    long long *counters = nullptr;
    uint64_t *keys_merge = nullptr;      // partitioned queries: merged candidates [M][KT]
    uint64_t *qstreams = nullptr;        // per-query restart streams [M] (knn_graph_query_ids)
    long long *counters_q = nullptr;     // partitioned queries: per-query counters [M][NCTR]
    int64_t *part_off = nullptr;         // [KNN_MAX_PARTS + 1]
    int64_t *part_live = nullptr;        // [KNN_MAX_PARTS]
    const long long *last_counters_src = nullptr;
    uint64_t *offer_key = nullptr;
    int32_t *offer_next = nullptr;
    int32_t *touched = nullptr;
    int32_t *frontier = nullptr;
    unsigned *small = nullptr;  // [0] offers, [1] touched, [2] error flags
    unsigned *work = nullptr;   // search counter of the persistent off-chip search
    unsigned long long *totals = nullptr;
    int64_t *out_ids_dev = nullptr;
    float *out_sims_dev = nullptr;
    uint64_t *cross_keys = nullptr;      // best k of each new point among its batch [M][K]
    cudaStream_t side = nullptr;         // the batch's own similarities run here beside the search
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaStream_t last_stream = nullptr;
    int64_t launches = 0;          // kernels launched by this library for the graph
    bool timing = false;           // record events around each phase
    int32_t climb = KNN_CLIMB_EAGER;
    cudaEvent_t ev[KNN_NUM_PHASES + 1] = {};
    bool phase_ran[KNN_NUM_PHASES] = {};

    // distributed online build (Algorithm 5): partitions by label, their
    // medoids, and the staged copy the partitioned search runs on
    int32_t dparts = 0;              // 0: not set
    double d_interval = 0.0;         // medoid recompute interval (fraction of n_last)
    int64_t d_n_last = 0;            // graph size at the last recompute
    int64_t d_recomputes = 0;
    int32_t *d_label = nullptr;      // [cap]
    int64_t *d_medoids = nullptr;    // [KNN_MAX_PARTS]
    int64_t *d_order = nullptr;      // [cap] position -> node
    int64_t *d_pos = nullptr;        // [cap] node -> position
    int64_t *d_offsets = nullptr;    // [KNN_MAX_PARTS + 1]
    uint8_t *d_sort = nullptr;       // counting-sort scratch
    uint8_t *st_rows = nullptr;      // [cap][row bytes] staged searched rows
    float *st_scale = nullptr;       // [cap] staged FP8 scales
    int32_t *st_nbr = nullptr;       // [cap][k] staged lists
};

// Mark the start of phase `ph` (and the end of the previous one).
static void phase_mark(knn_graph *g, int ph, cudaStream_t s) {
    if (!g->timing) return;
    cudaEventRecord(g->ev[ph], s);
}
static void phase_begin_call(knn_graph *g) {
    for (bool &r : g->phase_ran) r = false;
}

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_last_error;

static knn_status fail(knn_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

GraphShape knn::graph_shape(const knn_graph *g) {
    return GraphShape{g->p.dim, g->p.k, g->p.max_batch, g->n, g->p.capacity};
}

void knn::graph_forget_stream(knn_graph *g, cudaStream_t s) {
    cudaStreamSynchronize(s);
    if (g->last_stream == s) g->last_stream = nullptr;
}

knn_status knn::record_error(knn_status st, const char *msg) {
    g_last_error = msg;
    return st;
}

#define CU(call)                                                                      \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess)                                                        \
            return fail(KNN_ERR_CUDA, "%s failed: %s (%s:%d)", #call,                 \
                        cudaGetErrorString(e_), __FILE__, __LINE__);                  \
    } while (0)

// An NVTX range around an ABI call (visible in Nsight tools; free otherwise).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

static bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

// ---------------------------------------------------------------------------
// exact graph: CUDA cores or tensor cores (knn_exact_set_path)
// ---------------------------------------------------------------------------
static std::atomic<int> g_exact_path{KNN_EXACT_AUTO};
static thread_local knn_exact_info g_exact_info{};

// The exact lists of ea.X into ea.out_ids / ea.out_d2.  The tensor-core path
// allocates its scratch on the stream and reads its counters back, so it
// returns with the stream drained.  *launches grows by the kernels launched.
static knn_status run_exact(int dp, const ExactArgs &ea, cudaStream_t s, int64_t *launches) {
    const int mode = g_exact_path.load();
    const bool tc = exact_tc_supported(dp, ea.n, ea.k, ea.removed);
    if (mode == KNN_EXACT_TENSOR_CORES && !tc)
        return fail(KNN_ERR_UNSUPPORTED, "tensor-core exact build needs padded dim <= 128, n >= 128 (dp %d, n %lld)",
                    dp, (long long)ea.n);
    knn_exact_info info{};
    info.n = ea.n;
    if (mode == KNN_EXACT_CUDA_CORES || !tc) {
        CU(launch_exact(dp, ea, s));
        info.path = KNN_EXACT_CUDA_CORES;
        *launches += 1;
        g_exact_info = info;
        return KNN_OK;
    }
    void *scratch = nullptr;
    CU(cudaMallocAsync(&scratch, exact_tc_scratch_bytes(ea.n, dp), s));
    unsigned *counters = nullptr;
    unsigned host[3] = {0, 0, 0};
    cudaError_t e = launch_exact_tc(dp, ea, scratch, &counters, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host, counters, sizeof host, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    const cudaError_t ef = cudaFreeAsync(scratch, s);
    if (e == cudaSuccess) e = ef;
    if (e != cudaSuccess) return fail(KNN_ERR_CUDA, "tensor-core exact build: %s", cudaGetErrorString(e));
    *launches += 4;
    info.path = KNN_EXACT_TENSOR_CORES;
    info.rows_redone = host[1];
    info.wait_errors = host[2];
    g_exact_info = info;
    return KNN_OK;
}

static int64_t budget_of(int64_t n, double speedup) {
    // B = max(1, floor(n / speedup)), the iGNNS similarity budget (Sec. 3)
    double b = std::floor((double)n / speedup);
    return b < 1.0 ? 1 : (int64_t)b;
}

template <class T>
static knn_status dev_alloc(knn_graph *g, T **ptr, size_t count) {
    void *p = nullptr;
    const size_t bytes = std::max<size_t>(count * sizeof(T), 16);
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(KNN_ERR_OOM, "cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    }
    g->allocations.push_back(p);
    g->bytes += bytes;
    *ptr = static_cast<T *>(p);
    return KNN_OK;
}

static void free_graph(knn_graph *g) {
    for (void *p : g->allocations) cudaFree(p);
    for (cudaEvent_t e : g->ev)
        if (e) cudaEventDestroy(e);
    if (g->ev_fork) cudaEventDestroy(g->ev_fork);
    if (g->ev_join) cudaEventDestroy(g->ev_join);
    if (g->side) cudaStreamDestroy(g->side);
    delete g;
}

#define TRY(expr)                               \
    do {                                        \
        knn_status st_ = (expr);                \
        if (st_ != KNN_OK) return st_;          \
    } while (0)

// Copy m rows of `dim` floats (host or device) into the rows starting at
// row `first` of the graph's arrays, with the screening copy if any.
static knn_status append_rows(knn_graph *g, const float *vecs, int64_t m, int64_t first,
                              float *dst_rows, bool screening, cudaStream_t s) {
    const int d = g->p.dim, dp = g->dp;
    const bool dev = is_device_ptr(vecs);
    for (int64_t c0 = 0; c0 < m; c0 += g->p.max_batch) {
        const int64_t cm = std::min<int64_t>(g->p.max_batch, m - c0);
        const float *src = vecs + c0 * d;
        if (!dev) {
            CU(cudaMemcpyAsync(g->stage_in, src, (size_t)cm * d * sizeof(float), cudaMemcpyHostToDevice, s));
            src = g->stage_in;
        }
        const int64_t r = first + c0;
        ++g->launches;
        CU(launch_append(src, cm, d, dp, dst_rows + r * dp,
                         (screening && g->Xb) ? g->Xb + r * dp : nullptr,
                         (screening && g->X8) ? g->X8 + r * dp : nullptr,
                         (screening && g->X8) ? g->scale + r : nullptr, s));
    }
    return KNN_OK;
}

static const uint8_t *searched_rows(const knn_graph *g) {
    switch (g->p.storage) {
        case KNN_STORAGE_BF16: return reinterpret_cast<const uint8_t *>(g->Xb);
        case KNN_STORAGE_FP8_E4M3: return g->X8;
        default: return reinterpret_cast<const uint8_t *>(g->X);
    }
}

// iGNNS for m items whose padded FP32 query rows start at `queries`; leaves
// the best k_out keys of each item in g->keys_final (screening forms) or
// g->keys_search (FP32), and returns which.
static knn_status run_search(knn_graph *g, const float *queries, int64_t m, int k_out,
                             uint64_t stream_base, cudaStream_t s, const uint64_t **keys_out,
                             const uint64_t *streams = nullptr) {
    const bool screening = g->p.storage != KNN_STORAGE_FP32;
    const int KT = screening ? g->p.rescore_mult * k_out : k_out;
    if (!search_visited_on_chip((uint32_t)g->n))
        CU(cudaMemsetAsync(g->visited, 0, (size_t)m * g->vwords * sizeof(uint32_t), s));
    SearchArgs a{};
    a.rows = searched_rows(g);
    a.row_scale = g->scale;
    a.nbr = g->nbr_ids;
    a.removed = g->removed;
    a.queries = queries;
    a.q_stride = g->dp;
    a.visited = g->visited;
    a.vwords = g->vwords;
    a.out_keys = g->keys_search;
    a.counters = g->counters;
    a.totals = g->totals;
    a.m = (int32_t)m;
    a.k = g->p.k;
    a.KT = KT;
    a.n = (uint32_t)g->n;
    a.n_live = g->n - g->n_removed;
    a.budget = budget_of(g->n, g->p.speedup);
    a.max_draws = 64ull * (uint64_t)g->n;
    a.seed = g->p.seed;
    a.stream_base = stream_base;
    const double e = g->p.expansion;
    a.discard = (e > 0.0 && std::isfinite(e)) ? 1 : 0;
    a.expansion = a.discard ? (float)e : 1.0f;
    a.climb = g->climb;
    a.vis_n = (uint32_t)g->n;
    a.speedup = g->p.speedup;
    a.streams = streams;
    a.work = g->work;
    CU(launch_search(g->p.storage, g->dp, a, s));
    g->last_counters_src = g->counters;
    ++g->launches;
    g->phase_ran[KNN_PHASE_SEARCH] = true;
    phase_mark(g, KNN_PHASE_RESCORE, s);
    if (!screening) {
        *keys_out = g->keys_search;
        return KNN_OK;
    }
    RescoreArgs r{};
    r.rows = g->X;
    r.queries = queries;
    r.q_stride = g->dp;
    r.cand_keys = g->keys_search;
    r.out_keys = g->keys_final;
    r.totals = g->totals;
    r.m = (int32_t)m;
    r.KT = KT;
    r.k_out = k_out;
    CU(launch_rescore(g->dp, r, s));
    ++g->launches;
    g->phase_ran[KNN_PHASE_RESCORE] = true;
    *keys_out = g->keys_final;
    return KNN_OK;
}

// Write m*k int64 ids (and optional sims) from keys to a host or device buffer.
static knn_status emit_keys(knn_graph *g, const uint64_t *keys, int64_t m, int kk, int k_out,
                            int64_t *out_ids, float *out_sims, cudaStream_t s, bool *synced) {
    const bool ids_dev = is_device_ptr(out_ids);
    const bool sims_dev = out_sims == nullptr || is_device_ptr(out_sims);
    int64_t *ids_target = ids_dev ? out_ids : g->out_ids_dev;
    float *sims_target = out_sims ? (sims_dev ? out_sims : g->out_sims_dev) : nullptr;
    CU(launch_keys_to_output(keys, m, kk, k_out, ids_target, sims_target, s));
    ++g->launches;
    bool need_sync = false;
    if (!ids_dev) {
        CU(cudaMemcpyAsync(out_ids, g->out_ids_dev, (size_t)m * k_out * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        need_sync = true;
    }
    if (out_sims && !sims_dev) {
        CU(cudaMemcpyAsync(out_sims, g->out_sims_dev, (size_t)m * k_out * sizeof(float), cudaMemcpyDeviceToHost, s));
        need_sync = true;
    }
    if (need_sync) {
        CU(cudaStreamSynchronize(s));
        *synced = true;
    }
    return KNN_OK;
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

KNN_API const char *knn_last_error(void) { return g_last_error.c_str(); }

KNN_API const char *knn_version(void) { return "knn_graph 0.1 (sm_103a)"; }

static knn_status validate_params(const knn_params &p, int64_t n_init) {
    if (p.dim < 1 || p.dim > 256) return fail(KNN_ERR_UNSUPPORTED, "dim %d outside 1..256", p.dim);
    if (p.k < 1 || p.k > 32) return fail(KNN_ERR_UNSUPPORTED, "k %d outside 1..32", p.k);
    if (p.depth < 1 || p.depth > 5) return fail(KNN_ERR_UNSUPPORTED, "depth %d outside 1..5", p.depth);
    if (p.storage < 0 || p.storage > 2) return fail(KNN_ERR_INVALID_ARG, "bad storage %d", p.storage);
    if (!(p.speedup > 0.0) || !std::isfinite(p.speedup))
        return fail(KNN_ERR_INVALID_ARG, "speedup must be finite and > 0");
    if (std::isnan(p.expansion)) return fail(KNN_ERR_INVALID_ARG, "expansion is NaN");
    if (p.storage != KNN_STORAGE_FP32 && (p.rescore_mult < 1 || p.rescore_mult * p.k > 128))
        return fail(KNN_ERR_UNSUPPORTED, "rescore_mult * k must be in 1..128");
    if (p.max_batch < 1) return fail(KNN_ERR_INVALID_ARG, "max_batch must be >= 1");
    if (n_init < p.k + 1) return fail(KNN_ERR_INVALID_ARG, "n_init %lld < k + 1", (long long)n_init);
    if (p.capacity < n_init || p.capacity >= (int64_t)INT32_MAX)
        return fail(KNN_ERR_CAPACITY, "capacity %lld must be >= n_init and < 2^31", (long long)p.capacity);
    return KNN_OK;
}

// Admission and allocation of everything the graph will ever need, then the
// initial fills.  On success *out owns the memory; n is still 0.
static knn_status graph_alloc(const knn_params &p, cudaStream_t s, knn_graph **out) {
    knn_graph *g = new knn_graph();
    g->p = p;
    if (g->p.storage == KNN_STORAGE_FP32) g->p.rescore_mult = 1;
    if (cudaGetDevice(&g->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&g->sm_count, cudaDevAttrMultiProcessorCount, g->device) != cudaSuccess) {
        delete g;
        cudaGetLastError();
        return fail(KNN_ERR_CUDA, "no CUDA device");
    }
    g->dp = padded_dim(p.dim);
    g->KT = g->p.rescore_mult * p.k;
    g->vwords = (p.capacity + 31) / 32;
    const int64_t C = p.capacity, M = p.max_batch, K = p.k, DP = g->dp;
    // Update levels of one new point: k + k^2 + ... + k^DEPTH entries at
    // most, and never more than k plus the nodes of the graph
    int64_t levels = 0, pw = 1;
    for (int t = 1; t <= p.depth; ++t) {
        pw = std::min<int64_t>(pw * K, C + K);
        levels = std::min<int64_t>(levels + pw, C + K);
    }
    g->frontier_cap = levels;
    if ((double)M * (double)(K + levels) >= 4.0e9)
        return fail(KNN_ERR_UNSUPPORTED, "max_batch * (k + Update levels) exceeds 2^32 candidates");
    g->offer_cap = (unsigned)(M * (K + levels));

    size_t need = (size_t)C * DP * 4 + (size_t)C * K * 8 + (size_t)g->vwords * 4 + (size_t)C * 4 +
                  (size_t)M * g->vwords * 4 + (size_t)M * DP * 4 + (size_t)M * p.dim * 4 +
                  (size_t)M * g->KT * 8 + (size_t)M * K * 8 + (size_t)M * NCTR * 8 +
                  (size_t)g->offer_cap * 16 + (size_t)M * K * 12 + (size_t)M * levels * 4 +
                  (size_t)M * g->KT * 8 + (size_t)M * NCTR * 8 + (size_t)(2 * KNN_MAX_PARTS + 1) * 8 +
                  (size_t)M * 8 + (size_t)M * K * 8;
    if (p.storage == KNN_STORAGE_BF16) need += (size_t)C * DP * 2;
    if (p.storage == KNN_STORAGE_FP8_E4M3) need += (size_t)C * DP + (size_t)C * 4;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        delete g;
        cudaGetLastError();
        return fail(KNN_ERR_CUDA, "cudaMemGetInfo failed");
    }
    if (need + (size_t)256 * 1024 * 1024 > free_b) {
        delete g;
        return fail(KNN_ERR_OOM, "graph needs %zu bytes, %zu free", need, free_b);
    }

    knn_status st = KNN_OK;
#define ALLOC(ptr, count)                          \
    if (st == KNN_OK) st = dev_alloc(g, &g->ptr, (size_t)(count));
    ALLOC(X, C * DP)
    if (p.storage == KNN_STORAGE_BF16) { ALLOC(Xb, C * DP) }
    if (p.storage == KNN_STORAGE_FP8_E4M3) { ALLOC(X8, C * DP) ALLOC(scale, C) }
    ALLOC(nbr_ids, C * K)
    ALLOC(nbr_d2, C * K)
    ALLOC(removed, g->vwords)
    ALLOC(head, C)
    ALLOC(visited, M * g->vwords)
    ALLOC(qbuf, M * DP)
    ALLOC(stage_in, M * p.dim)
    ALLOC(keys_search, M * g->KT)
    ALLOC(keys_final, M * K)
    ALLOC(counters, M * NCTR)
    ALLOC(keys_merge, M * g->KT)
    ALLOC(qstreams, M)
    ALLOC(counters_q, M * NCTR)
    ALLOC(part_off, KNN_MAX_PARTS + 1)
    ALLOC(part_live, KNN_MAX_PARTS)
    ALLOC(offer_key, g->offer_cap)
    ALLOC(offer_next, g->offer_cap)
    ALLOC(touched, g->offer_cap)
    ALLOC(frontier, M * levels)
    ALLOC(small, 4)
    ALLOC(work, 4)
    ALLOC(totals, NTOT)
    ALLOC(out_ids_dev, M * K)
    ALLOC(out_sims_dev, M * K)
    ALLOC(cross_keys, M * K)
#undef ALLOC
    if (st == KNN_OK && (cudaStreamCreateWithFlags(&g->side, cudaStreamNonBlocking) != cudaSuccess ||
                         cudaEventCreateWithFlags(&g->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
                         cudaEventCreateWithFlags(&g->ev_join, cudaEventDisableTiming) != cudaSuccess)) {
        cudaGetLastError();
        st = fail(KNN_ERR_CUDA, "creating the graph's side stream failed");
    }
    if (st != KNN_OK) {
        free_graph(g);
        return st;
    }
    g->removed_host.assign((size_t)g->vwords, 0u);
    auto fills = [&]() -> knn_status {
        CU(cudaMemsetAsync(g->X, 0, (size_t)C * DP * 4, s));
        CU(cudaMemsetAsync(g->removed, 0, (size_t)g->vwords * 4, s));
        CU(cudaMemsetAsync(g->small, 0, 16, s));
        CU(cudaMemsetAsync(g->totals, 0, NTOT * 8, s));
        CU(cudaMemsetAsync(g->counters, 0, (size_t)M * NCTR * 8, s));
        CU(launch_fill_i32(g->head, -1, C, s));
        CU(launch_fill_i32(g->nbr_ids, -1, C * K, s));
        // an empty search launch resolves the search kernels of this graph's
        // storage and dimension (both top-list sizes), so that lazy module
        // loading does not land inside the first search
        SearchArgs none{};
        none.KT = 1;
        CU(launch_search(g->p.storage, g->dp, none, s));
        none.KT = 33;
        CU(launch_search(g->p.storage, g->dp, none, s));
        return KNN_OK;
    };
    st = fills();
    if (st != KNN_OK) {
        free_graph(g);
        return st;
    }
    g->last_stream = s;
    *out = g;
    return KNN_OK;
}

KNN_API knn_status knn_graph_create(const knn_params *params, const float *init_vecs, int64_t n_init,
                                    void *stream, knn_graph **out) {
    NvtxRange nvtx_range("knn_graph_create");
    if (!params || !init_vecs || !out) return fail(KNN_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    TRY(validate_params(*params, n_init));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    knn_graph *g = nullptr;
    TRY(graph_alloc(*params, s, &g));
    auto build = [&]() -> knn_status {
        TRY(append_rows(g, init_vecs, n_init, 0, g->X, true, s));
        ExactArgs ea{};
        ea.X = g->X;
        ea.removed = nullptr;
        ea.out_ids = g->nbr_ids;
        ea.out_d2 = g->nbr_d2;
        ea.n = n_init;
        ea.k = g->p.k;
        TRY(run_exact(g->dp, ea, s, &g->launches));
        CU(cudaStreamSynchronize(s));
        return KNN_OK;
    };
    knn_status st = build();
    if (st != KNN_OK) {
        free_graph(g);
        return st;
    }
    g->n = n_init;
    *out = g;
    return KNN_OK;
}

KNN_API knn_status knn_graph_restore(const knn_params *params, const float *vecs, int64_t n,
                                     const int64_t *nbr_ids, void *stream, knn_graph **out) {
    NvtxRange nvtx_range("knn_graph_restore");
    if (!params || !vecs || !nbr_ids || !out) return fail(KNN_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    TRY(validate_params(*params, n));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    knn_graph *g = nullptr;
    TRY(graph_alloc(*params, s, &g));
    auto load = [&]() -> knn_status {
        TRY(append_rows(g, vecs, n, 0, g->X, true, s));
        const int64_t K = g->p.k;
        const int64_t *ids_dev = nbr_ids;
        int64_t *tmp = nullptr;
        if (!is_device_ptr(nbr_ids)) {
            CU(cudaMallocAsync(&tmp, (size_t)n * K * 8, s));
            CU(cudaMemcpyAsync(tmp, nbr_ids, (size_t)n * K * 8, cudaMemcpyHostToDevice, s));
            ids_dev = tmp;
        }
        CU(launch_restore_lists(g->dp, g->X, ids_dev, n, (int)K, g->nbr_ids, g->nbr_d2, g->small + 3, s));
        if (tmp) CU(cudaFreeAsync(tmp, s));
        unsigned bad = 0;
        CU(cudaMemcpyAsync(&bad, g->small + 3, sizeof bad, cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        if (bad) return fail(KNN_ERR_INVALID_ARG, "snapshot lists hold an id outside -1..n-1, a self "
                                                  "edge or an entry after an empty slot");
        return KNN_OK;
    };
    knn_status st = load();
    if (st != KNN_OK) {
        free_graph(g);
        return st;
    }
    g->n = n;
    *out = g;
    return KNN_OK;
}

static knn_status run_search_distributed(knn_graph *g, int64_t n0, int64_t m, cudaStream_t s,
                                         const uint64_t **keys_out);
static knn_status assign_partitions(knn_graph *g, int64_t n0, int64_t m, cudaStream_t s);

// Algorithm 1 for a batch (knn_graph_insert_batch), or Algorithm 5 when
// `distributed` (knn_graph_insert_distributed): the same steps but the search
// and, after it, the new nodes' partitions.
static knn_status insert_impl(knn_graph *g, const float *vecs, int64_t m, int64_t *out_ids, int64_t *out_nbrs,
                              void *stream, bool distributed) {
    if (!g || !vecs) return fail(KNN_ERR_INVALID_ARG, "null argument");
    if (m < 1 || m > g->p.max_batch)
        return fail(KNN_ERR_INVALID_ARG, "m = %lld outside 1..max_batch", (long long)m);
    if (g->n + m > g->p.capacity) return fail(KNN_ERR_CAPACITY, "graph full");
    DeviceGuard dg(g->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    g->last_stream = s;
    const int64_t n0 = g->n;
    const int K = g->p.k;
    phase_begin_call(g);

    // a1: store the new rows (and their screening copy)
    phase_mark(g, KNN_PHASE_STORE, s);
    TRY(append_rows(g, vecs, m, n0, g->X, true, s));
    g->phase_ran[KNN_PHASE_STORE] = true;
    // a6, first half: exact similarities among the batch (the best k of each
    // new point) on the side stream, beside the search: they need only the
    // stored rows, and SMs the search leaves free take them
    CrossArgs ca{};
    ca.rows = g->X;
    ca.cross_keys = g->cross_keys;
    ca.nbr_ids = g->nbr_ids;
    ca.nbr_d2 = g->nbr_d2;
    ca.totals = g->totals;
    ca.m = (int32_t)m;
    ca.k = K;
    ca.n = (uint32_t)n0;
    CU(cudaEventRecord(g->ev_fork, s));
    CU(cudaStreamWaitEvent(g->side, g->ev_fork, 0));
    CU(launch_cross_topk(g->dp, ca, g->side));
    CU(cudaEventRecord(g->ev_join, g->side));
    ++g->launches;
    // a2-a5: iGNNS of every new point against the n0 nodes before the batch
    phase_mark(g, KNN_PHASE_SEARCH, s);
    const uint64_t *keys = nullptr;
    knn_status sst = distributed ? run_search_distributed(g, n0, m, s, &keys)
                                 : run_search(g, g->X + n0 * g->dp, m, K, (uint64_t)n0, s, &keys);
    if (sst != KNN_OK) {
        // the side stream's kernel may still write cross_keys: order it
        // before anything the caller enqueues next on s
        cudaStreamWaitEvent(s, g->ev_join, 0);
        return sst;
    }
    phase_mark(g, KNN_PHASE_CROSS, s);
    // a6, second half: each new list is the best k of the search result and
    // of the batch
    ca.in_keys = keys;
    CU(cudaStreamWaitEvent(s, g->ev_join, 0));
    CU(launch_cross_merge(ca, s));
    ++g->launches;
    g->phase_ran[KNN_PHASE_CROSS] = true;
    // a7-a8: Update (Algorithm 2): collect candidates, then merge them
    phase_mark(g, KNN_PHASE_OFFERS, s);
    CU(cudaMemsetAsync(g->small, 0, 2 * sizeof(unsigned), s));
    UpdateArgs ua{};
    ua.rows = g->X;
    ua.nbr_ids = g->nbr_ids;
    ua.nbr_d2 = g->nbr_d2;
    ua.removed = g->removed;
    ua.head = g->head;
    ua.offer_key = g->offer_key;
    ua.offer_next = g->offer_next;
    ua.touched = g->touched;
    ua.offer_count = g->small + 0;
    ua.touched_count = g->small + 1;
    ua.offer_cap = g->offer_cap;
    ua.error_flags = g->small + 2;
    ua.counters = g->counters;
    ua.totals = g->totals;
    ua.m = (int32_t)m;
    ua.k = K;
    ua.depth = g->p.depth;
    ua.frontier = g->frontier;
    ua.frontier_cap = g->frontier_cap;
    ua.seen = g->visited;
    ua.seen_words = (n0 + m + 31) / 32;
    ua.n = (uint32_t)n0;
    if (ua.depth >= 2 && !update_seen_on_chip(ua.seen_words))
        CU(cudaMemsetAsync(g->visited, 0, (size_t)m * ua.seen_words * sizeof(uint32_t), s));
    CU(launch_update(g->dp, ua, s));
    ++g->launches;
    g->phase_ran[KNN_PHASE_OFFERS] = true;
    phase_mark(g, KNN_PHASE_MERGE, s);
    MergeArgs ma{};
    ma.nbr_ids = g->nbr_ids;
    ma.nbr_d2 = g->nbr_d2;
    ma.head = g->head;
    ma.offer_key = g->offer_key;
    ma.offer_next = g->offer_next;
    ma.touched = g->touched;
    ma.touched_count = g->small + 1;
    ma.offer_count = g->small + 0;
    ma.totals = g->totals;
    ma.k = K;
    CU(launch_merge(ma, g->sm_count, s));
    ++g->launches;
    g->phase_ran[KNN_PHASE_MERGE] = true;
    phase_mark(g, KNN_NUM_PHASES, s);
    // a9: publish
    g->n = n0 + m;
    g->inserts += m;
    g->last_m = m;
    if (distributed) TRY(assign_partitions(g, n0, m, s));

    if (out_ids) {
        if (is_device_ptr(out_ids)) {
            ++g->launches;
            CU(launch_fill_ids(out_ids, n0, m, s));
        } else {
            for (int64_t i = 0; i < m; ++i) out_ids[i] = n0 + i;
        }
    }
    if (out_nbrs) {
        const bool dev = is_device_ptr(out_nbrs);
        int64_t *target = dev ? out_nbrs : g->out_ids_dev;
        ++g->launches;
        CU(launch_lists_to_output(g->nbr_ids + n0 * K, g->nbr_d2 + n0 * K, m, K, target, nullptr, s));
        if (!dev) {
            CU(cudaMemcpyAsync(out_nbrs, g->out_ids_dev, (size_t)m * K * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            CU(cudaStreamSynchronize(s));
        }
    }
    return KNN_OK;
}

KNN_API knn_status knn_graph_insert_batch(knn_graph *g, const float *vecs, int64_t m, int64_t *out_ids,
                                          int64_t *out_nbrs, void *stream) {
    NvtxRange nvtx_range("knn_graph_insert_batch");
    return insert_impl(g, vecs, m, out_ids, out_nbrs, stream, false);
}

KNN_API knn_status knn_graph_insert_distributed(knn_graph *g, const float *vecs, int64_t m, int64_t *out_ids,
                                                int64_t *out_nbrs, void *stream) {
    NvtxRange nvtx_range("knn_graph_insert_distributed");
    if (!g) return fail(KNN_ERR_INVALID_ARG, "null argument");
    if (g->dparts < 1) return fail(KNN_ERR_INVALID_ARG, "no partitions: call knn_graph_set_partitions first");
    if (g->n_removed > 0) return fail(KNN_ERR_UNSUPPORTED, "the distributed build takes no graph with removed nodes");
    return insert_impl(g, vecs, m, out_ids, out_nbrs, stream, true);
}

// Replace the allocation `old` of g by `fresh` (already counted in g->bytes).
static void swap_allocation(knn_graph *g, void *old, void *fresh, size_t old_bytes) {
    for (void *&p : g->allocations)
        if (p == old) {
            p = fresh;
            cudaFree(old);
            g->bytes -= old_bytes;
            return;
        }
}

// Bytes of the per-node arrays of a graph with `capacity` nodes (the rows,
// the screening copy, the lists, the removal bits, the Update chain heads and
// the batch's visited sets).
static size_t node_bytes(const knn_graph *g, int64_t capacity) {
    const size_t C = (size_t)capacity, DP = (size_t)g->dp, K = (size_t)g->p.k;
    const size_t words = (C + 31) / 32;
    size_t b = C * DP * 4 + C * K * 8 + words * 4 + C * 4 + (size_t)g->p.max_batch * words * 4;
    if (g->p.storage == KNN_STORAGE_BF16) b += C * DP * 2;
    if (g->p.storage == KNN_STORAGE_FP8_E4M3) b += C * DP + C * 4;
    return b;
}

KNN_API knn_status knn_graph_reserve(knn_graph *g, int64_t capacity, int64_t headroom_bytes, void *stream) {
    NvtxRange nvtx_range("knn_graph_reserve");
    if (!g) return fail(KNN_ERR_INVALID_ARG, "null argument");
    if (capacity <= g->p.capacity) return KNN_OK;
    if (capacity >= (int64_t)INT32_MAX) return fail(KNN_ERR_CAPACITY, "capacity must stay below 2^31");
    if (headroom_bytes < 0) return fail(KNN_ERR_INVALID_ARG, "headroom_bytes must be >= 0");
    if (g->d_label) return fail(KNN_ERR_UNSUPPORTED, "a graph with partitions set does not grow");
    DeviceGuard dg(g->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // nothing of the graph may be in flight while its arrays move
    CU(cudaStreamSynchronize(g->last_stream));
    CU(cudaStreamSynchronize(g->side));
    CU(cudaStreamSynchronize(s));
    const size_t need = node_bytes(g, capacity);
    size_t free_b = 0, total_b = 0;
    CU(cudaMemGetInfo(&free_b, &total_b));
    if (need + (size_t)headroom_bytes > free_b)
        return fail(KNN_ERR_OOM, "growing to %lld nodes needs %zu bytes with %lld of headroom; %zu free",
                    (long long)capacity, need, (long long)headroom_bytes, free_b);
    const int64_t C0 = g->p.capacity, C = capacity, n = g->n, K = g->p.k, DP = g->dp, M = g->p.max_batch;
    const int64_t w0 = g->vwords, w = (C + 31) / 32;
    // new arrays first, so that a failure leaves the graph as it was
    float *X = nullptr, *nbr_d2 = nullptr, *scale = nullptr;
    uint16_t *Xb = nullptr;
    uint8_t *X8 = nullptr;
    int32_t *nbr_ids = nullptr, *head = nullptr;
    uint32_t *removed = nullptr, *visited = nullptr;
    std::vector<void *> fresh;
    auto get = [&](auto **ptr, size_t count) -> bool {
        void *q = nullptr;
        const size_t bytes = std::max<size_t>(count * sizeof(**ptr), 16);
        if (cudaMalloc(&q, bytes) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        fresh.push_back(q);
        *ptr = static_cast<std::remove_reference_t<decltype(*ptr)>>(q);
        return true;
    };
    bool ok = get(&X, C * DP) && get(&nbr_ids, C * K) && get(&nbr_d2, C * K) && get(&removed, w) &&
              get(&head, C) && get(&visited, M * w);
    if (ok && g->Xb) ok = get(&Xb, C * DP);
    if (ok && g->X8) ok = get(&X8, C * DP) && get(&scale, C);
    // Update's level bound (k + k^2 + ... + k^DEPTH, at most the nodes plus
    // k) grows with the graph while the graph is smaller than it
    int64_t levels = 0, pw = 1;
    for (int t = 1; t <= g->p.depth; ++t) {
        pw = std::min<int64_t>(pw * K, C + K);
        levels = std::min<int64_t>(levels + pw, C + K);
    }
    const bool regrow = levels > g->frontier_cap;
    const unsigned ocap = (unsigned)(M * (K + levels));
    uint64_t *okey = nullptr;
    int32_t *onext = nullptr, *touched = nullptr, *frontier = nullptr;
    if (ok && regrow)
        ok = (double)M * (double)(K + levels) < 4.0e9 && get(&okey, ocap) && get(&onext, ocap) &&
             get(&touched, ocap) && get(&frontier, M * levels);
    if (!ok) {
        for (void *q : fresh) cudaFree(q);
        return fail(KNN_ERR_OOM, "growing to %lld nodes: cudaMalloc failed", (long long)capacity);
    }
    auto moves = [&]() -> knn_status {
        CU(cudaMemcpyAsync(X, g->X, (size_t)n * DP * 4, cudaMemcpyDeviceToDevice, s));
        CU(cudaMemsetAsync(X + n * DP, 0, (size_t)(C - n) * DP * 4, s));
        if (g->Xb) CU(cudaMemcpyAsync(Xb, g->Xb, (size_t)n * DP * 2, cudaMemcpyDeviceToDevice, s));
        if (g->X8) {
            CU(cudaMemcpyAsync(X8, g->X8, (size_t)n * DP, cudaMemcpyDeviceToDevice, s));
            CU(cudaMemcpyAsync(scale, g->scale, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
        }
        CU(cudaMemcpyAsync(nbr_ids, g->nbr_ids, (size_t)n * K * 4, cudaMemcpyDeviceToDevice, s));
        CU(launch_fill_i32(nbr_ids + n * K, -1, (C - n) * K, s));
        CU(cudaMemcpyAsync(nbr_d2, g->nbr_d2, (size_t)n * K * 4, cudaMemcpyDeviceToDevice, s));
        CU(cudaMemsetAsync(removed, 0, (size_t)w * 4, s));
        CU(cudaMemcpyAsync(removed, g->removed, (size_t)w0 * 4, cudaMemcpyDeviceToDevice, s));
        CU(launch_fill_i32(head, -1, C, s));  // every chain is empty between calls
        g->launches += 2;
        CU(cudaStreamSynchronize(s));
        return KNN_OK;
    };
    knn_status st = moves();
    if (st != KNN_OK) {
        for (void *q : fresh) cudaFree(q);
        return st;
    }
    const size_t b_rows = (size_t)C0 * DP * 4, b_list = (size_t)C0 * K * 4, b_bits = (size_t)w0 * 4;
    g->bytes += node_bytes(g, C);
    swap_allocation(g, g->X, X, b_rows);
    swap_allocation(g, g->nbr_ids, nbr_ids, b_list);
    swap_allocation(g, g->nbr_d2, nbr_d2, b_list);
    swap_allocation(g, g->removed, removed, b_bits);
    swap_allocation(g, g->head, head, (size_t)C0 * 4);
    swap_allocation(g, g->visited, visited, (size_t)M * b_bits);
    if (g->Xb) swap_allocation(g, g->Xb, Xb, (size_t)C0 * DP * 2);
    if (g->X8) {
        swap_allocation(g, g->X8, X8, (size_t)C0 * DP);
        swap_allocation(g, g->scale, scale, (size_t)C0 * 4);
    }
    g->X = X;
    g->Xb = Xb ? Xb : g->Xb;
    g->X8 = X8 ? X8 : g->X8;
    g->scale = scale ? scale : g->scale;
    g->nbr_ids = nbr_ids;
    g->nbr_d2 = nbr_d2;
    g->removed = removed;
    g->head = head;
    g->visited = visited;
    if (regrow) {
        g->bytes += (size_t)ocap * 16 + (size_t)M * levels * 4;
        swap_allocation(g, g->offer_key, okey, (size_t)g->offer_cap * 8);
        swap_allocation(g, g->offer_next, onext, (size_t)g->offer_cap * 4);
        swap_allocation(g, g->touched, touched, (size_t)g->offer_cap * 4);
        swap_allocation(g, g->frontier, frontier, (size_t)M * g->frontier_cap * 4);
        g->offer_key = okey;
        g->offer_next = onext;
        g->touched = touched;
        g->frontier = frontier;
        g->offer_cap = ocap;
        g->frontier_cap = levels;
    }
    g->vwords = w;
    g->removed_host.resize((size_t)w, 0u);
    g->p.capacity = C;
    g->last_stream = s;
    return KNN_OK;
}

KNN_API knn_status knn_graph_query_batch(knn_graph *g, const float *vecs, int64_t m, int32_t k_out,
                                         uint64_t query_id0, int64_t *out_ids, float *out_sims,
                                         void *stream) {
    NvtxRange nvtx_range("knn_graph_query_batch");
    if (!g || !vecs || !out_ids) return fail(KNN_ERR_INVALID_ARG, "null argument");
    if (m < 1 || m > g->p.max_batch)
        return fail(KNN_ERR_INVALID_ARG, "m = %lld outside 1..max_batch", (long long)m);
    if (k_out < 1 || k_out > g->p.k) return fail(KNN_ERR_INVALID_ARG, "k_out outside 1..k");
    DeviceGuard dg(g->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    g->last_stream = s;
    phase_begin_call(g);
    phase_mark(g, KNN_PHASE_STORE, s);
    TRY(append_rows(g, vecs, m, 0, g->qbuf, false, s));
    g->phase_ran[KNN_PHASE_STORE] = true;
    phase_mark(g, KNN_PHASE_SEARCH, s);
    const uint64_t *keys = nullptr;
    TRY(run_search(g, g->qbuf, m, k_out, (1ull << 63) + query_id0, s, &keys));
    phase_mark(g, KNN_PHASE_CROSS, s);
    for (int ph = KNN_PHASE_CROSS + 1; ph <= KNN_NUM_PHASES; ++ph) phase_mark(g, ph, s);
    bool synced = false;
    TRY(emit_keys(g, keys, m, k_out, k_out, out_ids, out_sims, s, &synced));
    g->queries += m;
    g->last_m = m;
    return KNN_OK;
}

KNN_API knn_status knn_graph_query_ids(knn_graph *g, const float *vecs, int64_t m, int32_t k_out,
                                       const uint64_t *query_ids, int64_t *out_ids, float *out_sims,
                                       void *stream) {
    NvtxRange nvtx_range("knn_graph_query_ids");
    if (!g || !vecs || !out_ids || !query_ids) return fail(KNN_ERR_INVALID_ARG, "null argument");
    if (m < 1 || m > g->p.max_batch)
        return fail(KNN_ERR_INVALID_ARG, "m = %lld outside 1..max_batch", (long long)m);
    if (k_out < 1 || k_out > g->p.k) return fail(KNN_ERR_INVALID_ARG, "k_out outside 1..k");
    DeviceGuard dg(g->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    g->last_stream = s;
    phase_begin_call(g);
    phase_mark(g, KNN_PHASE_STORE, s);
    TRY(append_rows(g, vecs, m, 0, g->qbuf, false, s));
    // restart stream of query i: 2^63 + query_ids[i], added on the device
    CU(cudaMemcpyAsync(g->qstreams, query_ids, (size_t)m * 8, cudaMemcpyDefault, s));
    CU(launch_add_u64(g->qstreams, 1ull << 63, m, s));
    ++g->launches;
    g->phase_ran[KNN_PHASE_STORE] = true;
    phase_mark(g, KNN_PHASE_SEARCH, s);
    const uint64_t *keys = nullptr;
    TRY(run_search(g, g->qbuf, m, k_out, 0, s, &keys, g->qstreams));
    phase_mark(g, KNN_PHASE_CROSS, s);
    for (int ph = KNN_PHASE_CROSS + 1; ph <= KNN_NUM_PHASES; ++ph) phase_mark(g, ph, s);
    bool synced = false;
    TRY(emit_keys(g, keys, m, k_out, k_out, out_ids, out_sims, s, &synced));
    g->queries += m;
    g->last_m = m;
    return KNN_OK;
}

// Partitioned queries; query i uses restart stream 2^63 + query_id0 + i, or
// 2^63 + query_ids[i] when query_ids is given.
static knn_status query_partitioned(knn_graph *g, const float *vecs, int64_t m, int32_t k_out,
                                    uint64_t query_id0, const uint64_t *query_ids, const int64_t *part_offsets,
                                    int32_t parts, int64_t *out_ids, float *out_sims, void *stream) {
    if (!g || !vecs || !out_ids || !part_offsets) return fail(KNN_ERR_INVALID_ARG, "null argument");
    if (m < 1 || m > g->p.max_batch)
        return fail(KNN_ERR_INVALID_ARG, "m = %lld outside 1..max_batch", (long long)m);
    if (k_out < 1 || k_out > g->p.k) return fail(KNN_ERR_INVALID_ARG, "k_out outside 1..k");
    if (parts < 1 || parts > KNN_MAX_PARTS || parts > g->p.max_batch)
        return fail(KNN_ERR_UNSUPPORTED, "parts %d outside 1..min(%d, max_batch)", parts, KNN_MAX_PARTS);
    DeviceGuard dg(g->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    g->last_stream = s;
    // the partitions: contiguous id ranges covering the graph
    std::vector<int64_t> off((size_t)parts + 1);
    if (is_device_ptr(part_offsets)) {
        CU(cudaMemcpyAsync(off.data(), part_offsets, off.size() * 8, cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
    } else {
        std::memcpy(off.data(), part_offsets, off.size() * 8);
    }
    if (off[0] != 0 || off[(size_t)parts] != g->n)
        return fail(KNN_ERR_INVALID_ARG, "partition offsets must run from 0 to n = %lld", (long long)g->n);
    std::vector<int64_t> live((size_t)parts);
    int64_t largest = 0;
    for (int q = 0; q < parts; ++q) {
        if (off[(size_t)q + 1] < off[(size_t)q]) return fail(KNN_ERR_INVALID_ARG, "partition offsets decrease");
        int64_t rem = 0;
        if (g->n_removed > 0)
            for (int64_t v = off[(size_t)q]; v < off[(size_t)q + 1]; ++v)
                rem += (g->removed_host[(size_t)(v >> 5)] >> (v & 31)) & 1u;
        live[(size_t)q] = off[(size_t)q + 1] - off[(size_t)q] - rem;
        largest = std::max(largest, off[(size_t)q + 1] - off[(size_t)q]);
    }
    CU(cudaMemcpyAsync(g->part_off, off.data(), off.size() * 8, cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(g->part_live, live.data(), live.size() * 8, cudaMemcpyHostToDevice, s));
    phase_begin_call(g);
    phase_mark(g, KNN_PHASE_STORE, s);
    TRY(append_rows(g, vecs, m, 0, g->qbuf, false, s));
    if (query_ids) {
        CU(cudaMemcpyAsync(g->qstreams, query_ids, (size_t)m * 8, cudaMemcpyDefault, s));
        CU(launch_add_u64(g->qstreams, 1ull << 63, m, s));
        ++g->launches;
    }
    g->phase_ran[KNN_PHASE_STORE] = true;
    phase_mark(g, KNN_PHASE_SEARCH, s);
    const bool screening = g->p.storage != KNN_STORAGE_FP32;
    const int KT = screening ? g->p.rescore_mult * k_out : k_out;
    // searches of one launch: parts per query, at most max_batch of them
    const int64_t step = std::max<int64_t>(1, g->p.max_batch / parts);
    const int64_t words = (largest + 31) / 32;
    bool synced = false;
    for (int64_t q0 = 0; q0 < m; q0 += step) {
        const int64_t mq = std::min(step, m - q0);
        if (!search_visited_on_chip((uint32_t)largest))
            CU(cudaMemsetAsync(g->visited, 0, (size_t)mq * parts * words * sizeof(uint32_t), s));
        SearchArgs a{};
        a.rows = searched_rows(g);
        a.row_scale = g->scale;
        a.nbr = g->nbr_ids;
        a.removed = g->removed;
        a.queries = g->qbuf + (size_t)q0 * g->dp;
        a.q_stride = g->dp;
        a.visited = g->visited;
        a.vwords = words;
        a.out_keys = g->keys_search;
        a.counters = g->counters;
        a.totals = g->totals;
        a.m = (int32_t)mq;
        a.k = g->p.k;
        a.KT = KT;
        a.n = (uint32_t)g->n;
        a.n_live = g->n - g->n_removed;
        a.budget = budget_of(g->n, g->p.speedup);
        a.max_draws = 64ull * (uint64_t)g->n;
        a.seed = g->p.seed;
        a.stream_base = (1ull << 63) + query_id0 + (uint64_t)q0;
        a.streams = query_ids ? g->qstreams + q0 : nullptr;
        const double e = g->p.expansion;
        a.discard = (e > 0.0 && std::isfinite(e)) ? 1 : 0;
        a.expansion = a.discard ? (float)e : 1.0f;
        a.climb = g->climb;
        a.parts = parts;
        a.part_off = g->part_off;
        a.part_live = g->part_live;
        a.speedup = g->p.speedup;
        a.vis_n = (uint32_t)largest;
        a.work = g->work;
        CU(launch_search(g->p.storage, g->dp, a, s));
        // the k_out (or KT) best of each query's parts * KT candidates
        CU(launch_merge_parts(g->keys_search, (int32_t)mq, parts, KT, g->keys_merge, g->counters,
                              g->counters_q + (size_t)q0 * NCTR, s));
        g->launches += 2;
        const uint64_t *keys = g->keys_merge;
        if (screening) {
            RescoreArgs r{};
            r.rows = g->X;
            r.queries = a.queries;
            r.q_stride = g->dp;
            r.cand_keys = g->keys_merge;
            r.out_keys = g->keys_final;
            r.totals = g->totals;
            r.m = (int32_t)mq;
            r.KT = KT;
            r.k_out = k_out;
            CU(launch_rescore(g->dp, r, s));
            ++g->launches;
            keys = g->keys_final;
        }
        TRY(emit_keys(g, keys, mq, k_out, k_out, out_ids + q0 * k_out, out_sims ? out_sims + q0 * k_out : nullptr, s,
                      &synced));
    }
    g->phase_ran[KNN_PHASE_SEARCH] = true;
    phase_mark(g, KNN_PHASE_RESCORE, s);
    for (int ph = KNN_PHASE_RESCORE + 1; ph <= KNN_NUM_PHASES; ++ph) phase_mark(g, ph, s);
    g->last_counters_src = g->counters_q;
    g->queries += m;
    g->last_m = m;
    return KNN_OK;
}

KNN_API knn_status knn_graph_query_partitioned(knn_graph *g, const float *vecs, int64_t m, int32_t k_out,
                                               uint64_t query_id0, const int64_t *part_offsets, int32_t parts,
                                               int64_t *out_ids, float *out_sims, void *stream) {
    NvtxRange nvtx_range("knn_graph_query_partitioned");
    return query_partitioned(g, vecs, m, k_out, query_id0, nullptr, part_offsets, parts, out_ids, out_sims,
                             stream);
}

KNN_API knn_status knn_graph_query_partitioned_ids(knn_graph *g, const float *vecs, int64_t m, int32_t k_out,
                                                   const uint64_t *query_ids, const int64_t *part_offsets,
                                                   int32_t parts, int64_t *out_ids, float *out_sims,
                                                   void *stream) {
    NvtxRange nvtx_range("knn_graph_query_partitioned_ids");
    if (!query_ids) return fail(KNN_ERR_INVALID_ARG, "null argument");
    return query_partitioned(g, vecs, m, k_out, 0, query_ids, part_offsets, parts, out_ids, out_sims, stream);
}

// ---------------------------------------------------------------------------
// distributed online build (Sec. 7, Algorithm 5)
// ---------------------------------------------------------------------------
static int64_t searched_row_bytes(const knn_graph *g) {
    switch (g->p.storage) {
        case KNN_STORAGE_BF16: return (int64_t)g->dp * 2;
        case KNN_STORAGE_FP8_E4M3: return (int64_t)g->dp;
        default: return (int64_t)g->dp * 4;
    }
}


KNN_API knn_status knn_graph_set_partitions(knn_graph *g, const int32_t *labels, const int64_t *medoids,
                                            int32_t parts, double recompute_interval, void *stream) {
    NvtxRange nvtx_range("knn_graph_set_partitions");
    if (!g || !labels || !medoids) return fail(KNN_ERR_INVALID_ARG, "null argument");
    if (parts < 1 || parts > KNN_MAX_PARTS || parts > g->p.max_batch)
        return fail(KNN_ERR_UNSUPPORTED, "parts %d outside 1..min(%d, max_batch)", parts, KNN_MAX_PARTS);
    if (!(recompute_interval >= 0.0) || !std::isfinite(recompute_interval))
        return fail(KNN_ERR_INVALID_ARG, "recompute_interval must be finite and >= 0");
    if (g->n_removed > 0) return fail(KNN_ERR_UNSUPPORTED, "the distributed build takes no graph with removed nodes");
    DeviceGuard dg(g->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    g->last_stream = s;
    const int64_t n = g->n;
    // check the labels and medoids on the host
    std::vector<int32_t> lab((size_t)n);
    std::vector<int64_t> med((size_t)parts);
    CU(cudaMemcpyAsync(lab.data(), labels, (size_t)n * 4, cudaMemcpyDefault, s));
    CU(cudaMemcpyAsync(med.data(), medoids, (size_t)parts * 8, cudaMemcpyDefault, s));
    CU(cudaStreamSynchronize(s));
    for (int64_t i = 0; i < n; ++i)
        if (lab[(size_t)i] < 0 || lab[(size_t)i] >= parts)
            return fail(KNN_ERR_INVALID_ARG, "label %d of node %lld outside 0..%d", lab[(size_t)i], (long long)i,
                        parts - 1);
    for (int32_t j = 0; j < parts; ++j)
        if (med[(size_t)j] < 0 || med[(size_t)j] >= n)
            return fail(KNN_ERR_INVALID_ARG, "medoid %d = %lld is not a node", j, (long long)med[(size_t)j]);
    {
        // the state, sized for the capacity (the graph does not grow while
        // set); what an earlier call failed to allocate is tried again
        const int64_t C = g->p.capacity;
        knn_status st = KNN_OK;
#define DALLOC(ptr, count) \
    if (st == KNN_OK && !g->ptr) st = dev_alloc(g, &g->ptr, (size_t)(count));
        DALLOC(d_label, C)
        DALLOC(d_medoids, KNN_MAX_PARTS)
        DALLOC(d_order, C)
        DALLOC(d_pos, C)
        DALLOC(d_offsets, KNN_MAX_PARTS + 1)
        DALLOC(d_sort, kmed_sort_scratch_bytes(C, KNN_MAX_PARTS))
        DALLOC(st_rows, C * searched_row_bytes(g))
        if (g->p.storage == KNN_STORAGE_FP8_E4M3) { DALLOC(st_scale, C) }
        DALLOC(st_nbr, C * g->p.k)
#undef DALLOC
        if (st != KNN_OK) return st;
    }
    CU(cudaMemcpyAsync(g->d_label, lab.data(), (size_t)n * 4, cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(g->d_medoids, med.data(), (size_t)parts * 8, cudaMemcpyHostToDevice, s));
    CU(cudaStreamSynchronize(s));
    g->dparts = parts;
    g->d_interval = recompute_interval;
    g->d_n_last = n;
    g->d_recomputes = 0;
    return KNN_OK;
}

KNN_API knn_status knn_graph_get_partitions(knn_graph *g, int32_t *labels, int64_t *medoids, int64_t *recomputes,
                                            void *stream) {
    if (!g) return fail(KNN_ERR_INVALID_ARG, "null argument");
    if (g->dparts < 1) return fail(KNN_ERR_INVALID_ARG, "no partitions: call knn_graph_set_partitions first");
    DeviceGuard dg(g->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (labels) CU(cudaMemcpyAsync(labels, g->d_label, (size_t)g->n * 4, cudaMemcpyDefault, s));
    if (medoids) CU(cudaMemcpyAsync(medoids, g->d_medoids, (size_t)g->dparts * 8, cudaMemcpyDefault, s));
    if (recomputes) CU(cudaMemcpyAsync(recomputes, &g->d_recomputes, 8, cudaMemcpyDefault, s));
    CU(cudaStreamSynchronize(s));
    return KNN_OK;
}

// The searches of Algorithm 5: Algorithm 3 over the label partitions.  Nodes
// 0..n0-1 are staged in partition order (a stable counting sort by label, so
// a partition keeps id order), each list keeping the entries inside its own
// partition; every new point runs one search per partition on the staged
// copy (the contiguous partitioned search, restart stream new id + j 2^56),
// the candidates' positions become node ids, and the best KT of each point's
// parts * KT candidates are kept (ties to the lower node id).
static knn_status run_search_distributed(knn_graph *g, int64_t n0, int64_t m, cudaStream_t s,
                                         const uint64_t **keys_out) {
    const int P = g->dparts;
    const int K = g->p.k;
    const bool screening = g->p.storage != KNN_STORAGE_FP32;
    const int KT = screening ? g->p.rescore_mult * K : K;
    CU(launch_kmed_sort(g->d_label, n0, P, g->d_sort, g->d_order, g->d_offsets, s));
    std::vector<int64_t> off((size_t)P + 1), live((size_t)P);
    CU(cudaMemcpyAsync(off.data(), g->d_offsets, off.size() * 8, cudaMemcpyDeviceToHost, s));
    CU(launch_part_stage(searched_rows(g), searched_row_bytes(g), g->p.storage == KNN_STORAGE_FP8_E4M3 ? g->scale
                                                                                                       : nullptr,
                         g->nbr_ids, K, g->d_label, g->d_order, g->d_pos, n0, g->st_rows, g->st_scale, g->st_nbr, s));
    g->launches += 5;
    CU(cudaStreamSynchronize(s));
    int64_t largest = 0;
    for (int q = 0; q < P; ++q) {
        live[(size_t)q] = off[(size_t)q + 1] - off[(size_t)q];
        largest = std::max(largest, live[(size_t)q]);
    }
    CU(cudaMemcpyAsync(g->part_live, live.data(), live.size() * 8, cudaMemcpyHostToDevice, s));
    const int64_t step = std::max<int64_t>(1, g->p.max_batch / P);
    const int64_t words = (largest + 31) / 32;
    for (int64_t q0 = 0; q0 < m; q0 += step) {
        const int64_t mq = std::min(step, m - q0);
        if (!search_visited_on_chip((uint32_t)largest))
            CU(cudaMemsetAsync(g->visited, 0, (size_t)mq * P * words * sizeof(uint32_t), s));
        SearchArgs a{};
        a.rows = g->st_rows;
        a.row_scale = g->st_scale;
        a.nbr = g->st_nbr;
        a.removed = g->removed;  // no node is removed
        a.queries = g->X + (size_t)(n0 + q0) * g->dp;
        a.q_stride = g->dp;
        a.visited = g->visited;
        a.vwords = words;
        a.out_keys = g->keys_search;
        a.counters = g->counters;
        a.totals = g->totals;
        a.m = (int32_t)mq;
        a.k = K;
        a.KT = KT;
        a.n = (uint32_t)n0;
        a.n_live = n0;
        a.budget = budget_of(n0, g->p.speedup);
        a.max_draws = 64ull * (uint64_t)n0;
        a.seed = g->p.seed;
        a.stream_base = (uint64_t)(n0 + q0);
        const double e = g->p.expansion;
        a.discard = (e > 0.0 && std::isfinite(e)) ? 1 : 0;
        a.expansion = a.discard ? (float)e : 1.0f;
        a.climb = g->climb;
        a.parts = P;
        a.part_off = g->d_offsets;
        a.part_live = g->part_live;
        a.speedup = g->p.speedup;
        a.vis_n = (uint32_t)largest;
        a.work = g->work;
        CU(launch_search(g->p.storage, g->dp, a, s));
        CU(launch_part_keys_to_nodes(g->keys_search, mq * P * KT, g->d_order, s));
        CU(launch_merge_parts(g->keys_search, (int32_t)mq, P, KT, g->keys_merge + (size_t)q0 * KT, g->counters,
                              g->counters_q + (size_t)q0 * NCTR, s));
        g->launches += 3;
    }
    // per new point, the sums over its parts, where Update adds its own count
    CU(cudaMemcpyAsync(g->counters, g->counters_q, (size_t)m * NCTR * sizeof(long long), cudaMemcpyDeviceToDevice,
                       s));
    g->last_counters_src = g->counters;
    g->phase_ran[KNN_PHASE_SEARCH] = true;
    phase_mark(g, KNN_PHASE_RESCORE, s);
    if (!screening) {
        *keys_out = g->keys_merge;
        return KNN_OK;
    }
    RescoreArgs r{};
    r.rows = g->X;
    r.queries = g->X + (size_t)n0 * g->dp;
    r.q_stride = g->dp;
    r.cand_keys = g->keys_merge;
    r.out_keys = g->keys_final;
    r.totals = g->totals;
    r.m = (int32_t)m;
    r.KT = KT;
    r.k_out = K;
    CU(launch_rescore(g->dp, r, s));
    ++g->launches;
    g->phase_ran[KNN_PHASE_RESCORE] = true;
    *keys_out = g->keys_final;
    return KNN_OK;
}

// After a distributed batch: nodes n0 .. n0+m-1 go to the partition of their
// nearest medoid; then, when the graph has grown by d_interval * d_n_last
// since the last recompute, every non-empty partition takes a new medoid.
static knn_status assign_partitions(knn_graph *g, int64_t n0, int64_t m, cudaStream_t s) {
    CU(launch_part_nearest(g->X, g->dp, g->X + (size_t)n0 * g->dp, m, g->d_medoids, g->dparts, g->d_label + n0, s));
    ++g->launches;
    if (g->d_interval > 0.0 && (double)(g->n - g->d_n_last) >= g->d_interval * (double)g->d_n_last) {
        CU(launch_kmed_sort(g->d_label, g->n, g->dparts, g->d_sort, g->d_order, g->d_offsets, s));
        CU(launch_kmed_update(g->dp, g->X, g->d_order, g->d_offsets, g->dparts, g->d_medoids, s));
        g->launches += 4;
        g->d_n_last = g->n;
        ++g->d_recomputes;
    }
    return KNN_OK;
}

KNN_API knn_status knn_graph_remove(knn_graph *g, const int64_t *ids, int64_t m, void *stream) {
    NvtxRange nvtx_range("knn_graph_remove");
    if (!g || (!ids && m > 0)) return fail(KNN_ERR_INVALID_ARG, "null argument");
    if (m < 0) return fail(KNN_ERR_INVALID_ARG, "negative m");
    if (m == 0) return KNN_OK;
    DeviceGuard dg(g->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    g->last_stream = s;
    std::vector<int64_t> h((size_t)m);
    if (is_device_ptr(ids)) {
        CU(cudaMemcpyAsync(h.data(), ids, (size_t)m * 8, cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
    } else {
        std::memcpy(h.data(), ids, (size_t)m * 8);
    }
    for (int64_t v : h)
        if (v < 0 || v >= g->n) return fail(KNN_ERR_NOT_FOUND, "id %lld not in the graph", (long long)v);
    int64_t newly = 0;
    for (int64_t v : h) {
        uint32_t &w = g->removed_host[(size_t)(v >> 5)];
        const uint32_t b = 1u << (v & 31);
        if (!(w & b)) {
            w |= b;
            ++newly;
        }
    }
    if (g->n - g->n_removed - newly < 1) return fail(KNN_ERR_INVALID_ARG, "cannot remove every node");
    CU(cudaMemcpyAsync(g->removed, g->removed_host.data(), g->removed_host.size() * 4, cudaMemcpyHostToDevice, s));
    CU(cudaStreamSynchronize(s));
    g->n_removed += newly;
    return KNN_OK;
}

KNN_API knn_status knn_graph_get_edges(knn_graph *g, int64_t *out_ids, float *out_sims, int64_t n_cap,
                                       int64_t *n_out, void *stream) {
    NvtxRange nvtx_range("knn_graph_get_edges");
    if (!g || !out_ids || !n_out) return fail(KNN_ERR_INVALID_ARG, "null argument");
    if (n_cap < 0) return fail(KNN_ERR_INVALID_ARG, "negative n_cap");
    DeviceGuard dg(g->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    g->last_stream = s;
    const int64_t rows = std::min(n_cap, g->n);
    const int K = g->p.k;
    const bool ids_dev = is_device_ptr(out_ids);
    const bool sims_dev = out_sims == nullptr || is_device_ptr(out_sims);
    int64_t *tmp_ids = nullptr;
    float *tmp_sims = nullptr;
    if (!ids_dev) CU(cudaMallocAsync(&tmp_ids, std::max<size_t>((size_t)rows * K * 8, 16), s));
    if (out_sims && !sims_dev) CU(cudaMallocAsync(&tmp_sims, std::max<size_t>((size_t)rows * K * 4, 16), s));
    CU(launch_lists_to_output(g->nbr_ids, g->nbr_d2, rows, K, ids_dev ? out_ids : tmp_ids,
                              out_sims ? (sims_dev ? out_sims : tmp_sims) : nullptr, s));
    if (tmp_ids) {
        CU(cudaMemcpyAsync(out_ids, tmp_ids, (size_t)rows * K * 8, cudaMemcpyDeviceToHost, s));
        CU(cudaFreeAsync(tmp_ids, s));
    }
    if (tmp_sims) {
        CU(cudaMemcpyAsync(out_sims, tmp_sims, (size_t)rows * K * 4, cudaMemcpyDeviceToHost, s));
        CU(cudaFreeAsync(tmp_sims, s));
    }
    if (tmp_ids || tmp_sims) CU(cudaStreamSynchronize(s));
    *n_out = rows;
    return KNN_OK;
}

KNN_API knn_status knn_graph_last_counters(knn_graph *g, int64_t *out, int64_t m, void *stream) {
    if (!g || !out) return fail(KNN_ERR_INVALID_ARG, "null argument");
    if (m < 0 || m > g->last_m) return fail(KNN_ERR_INVALID_ARG, "m exceeds the last call's size");
    DeviceGuard dg(g->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool dev = is_device_ptr(out);
    CU(cudaMemcpyAsync(out, g->last_counters_src ? g->last_counters_src : g->counters, (size_t)m * NCTR * 8,
                       dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    if (!dev) CU(cudaStreamSynchronize(s));
    return KNN_OK;
}

KNN_API knn_status knn_graph_stats(knn_graph *g, knn_stats *out) {
    if (!g || !out) return fail(KNN_ERR_INVALID_ARG, "null argument");
    DeviceGuard dg(g->device);
    unsigned long long t[NTOT];
    unsigned flags[4];
    CU(cudaStreamSynchronize(g->last_stream));
    CU(cudaMemcpy(t, g->totals, sizeof t, cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(flags, g->small, sizeof flags, cudaMemcpyDeviceToHost));
    if (flags[2] & ERR_OFFER_OVERFLOW) return fail(KNN_ERR_CAPACITY, "Update candidate pool overflowed");
    std::memset(out, 0, sizeof *out);
    out->n = g->n;
    out->capacity = g->p.capacity;
    out->removed = g->n_removed;
    out->inserts = g->inserts;
    out->queries = g->queries;
    out->search_evals = (int64_t)t[TOT_SEARCH_EVALS];
    out->update_evals = (int64_t)t[TOT_UPDATE_EVALS];
    out->cross_evals = (int64_t)t[TOT_CROSS_EVALS];
    out->rescore_evals = (int64_t)t[TOT_RESCORE_EVALS];
    out->restarts = (int64_t)t[TOT_RESTARTS];
    out->moves = (int64_t)t[TOT_MOVES];
    out->adjacency_reads = (int64_t)t[TOT_ADJ_READS];
    out->offers = (int64_t)t[TOT_OFFERS];
    out->device_bytes = (int64_t)g->bytes;
    out->kernel_launches = g->launches;
    return KNN_OK;
}

KNN_API knn_status knn_graph_set_timing(knn_graph *g, int32_t enable) {
    if (!g) return fail(KNN_ERR_INVALID_ARG, "null argument");
    DeviceGuard dg(g->device);
    if (enable && !g->ev[0])
        for (cudaEvent_t &e : g->ev) CU(cudaEventCreate(&e));
    g->timing = enable != 0;
    return KNN_OK;
}

KNN_API knn_status knn_graph_last_timing(knn_graph *g, float *out_ms, int32_t n) {
    if (!g || !out_ms) return fail(KNN_ERR_INVALID_ARG, "null argument");
    if (!g->timing) return fail(KNN_ERR_INVALID_ARG, "timing is off");
    if (n < 0 || n > KNN_NUM_PHASES) return fail(KNN_ERR_INVALID_ARG, "n outside 0..KNN_NUM_PHASES");
    DeviceGuard dg(g->device);
    CU(cudaEventSynchronize(g->ev[KNN_NUM_PHASES]));
    for (int ph = 0; ph < n; ++ph) {
        out_ms[ph] = 0.f;
        if (g->phase_ran[ph]) CU(cudaEventElapsedTime(&out_ms[ph], g->ev[ph], g->ev[ph + 1]));
    }
    return KNN_OK;
}

KNN_API void knn_graph_destroy(knn_graph *g) {
    if (!g) return;
    DeviceGuard dg(g->device);
    cudaStreamSynchronize(g->last_stream);
    free_graph(g);
}

KNN_API knn_status knn_exact_graph(const float *X, int64_t n, int32_t dim, int32_t k, int64_t *out_ids,
                                   float *out_sims, void *stream) {
    NvtxRange nvtx_range("knn_exact_graph");
    if (!X || !out_ids) return fail(KNN_ERR_INVALID_ARG, "null argument");
    if (dim < 1 || dim > 256) return fail(KNN_ERR_UNSUPPORTED, "dim %d outside 1..256", dim);
    if (k < 1 || k > 32) return fail(KNN_ERR_UNSUPPORTED, "k %d outside 1..32", k);
    if (n < k + 1 || n >= (int64_t)INT32_MAX) return fail(KNN_ERR_INVALID_ARG, "need k+1 <= n < 2^31");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int dp = padded_dim(dim);
    const bool x_dev = is_device_ptr(X);
    const bool ids_dev = is_device_ptr(out_ids);
    const bool sims_dev = out_sims == nullptr || is_device_ptr(out_sims);
    float *rows = nullptr, *d2 = nullptr, *xin = nullptr, *sims_tmp = nullptr;
    int32_t *ids = nullptr;
    int64_t *ids_tmp = nullptr;
    CU(cudaMallocAsync(&rows, (size_t)n * dp * 4, s));
    CU(cudaMallocAsync(&ids, (size_t)n * k * 4, s));
    CU(cudaMallocAsync(&d2, (size_t)n * k * 4, s));
    if (!x_dev) {
        CU(cudaMallocAsync(&xin, (size_t)n * dim * 4, s));
        CU(cudaMemcpyAsync(xin, X, (size_t)n * dim * 4, cudaMemcpyHostToDevice, s));
    }
    CU(launch_append(x_dev ? X : xin, n, dim, dp, rows, nullptr, nullptr, nullptr, s));
    ExactArgs ea{};
    ea.X = rows;
    ea.removed = nullptr;
    ea.out_ids = ids;
    ea.out_d2 = d2;
    ea.n = n;
    ea.k = k;
    int64_t launches = 0;
    TRY(run_exact(dp, ea, s, &launches));
    if (!ids_dev) CU(cudaMallocAsync(&ids_tmp, (size_t)n * k * 8, s));
    if (out_sims && !sims_dev) CU(cudaMallocAsync(&sims_tmp, (size_t)n * k * 4, s));
    CU(launch_lists_to_output(ids, d2, n, k, ids_dev ? out_ids : ids_tmp,
                              out_sims ? (sims_dev ? out_sims : sims_tmp) : nullptr, s));
    if (ids_tmp) CU(cudaMemcpyAsync(out_ids, ids_tmp, (size_t)n * k * 8, cudaMemcpyDeviceToHost, s));
    if (sims_tmp) CU(cudaMemcpyAsync(out_sims, sims_tmp, (size_t)n * k * 4, cudaMemcpyDeviceToHost, s));
    for (void *p : {(void *)rows, (void *)ids, (void *)d2, (void *)xin, (void *)ids_tmp, (void *)sims_tmp})
        if (p) CU(cudaFreeAsync(p, s));
    if (ids_tmp || sims_tmp) CU(cudaStreamSynchronize(s));
    return KNN_OK;
}

KNN_API knn_status knn_graph_set_search(knn_graph *g, double speedup, double expansion, int32_t climb) {
    if (!g) return fail(KNN_ERR_INVALID_ARG, "null graph");
    if (!(speedup > 0.0) || !std::isfinite(speedup))
        return fail(KNN_ERR_INVALID_ARG, "speedup must be finite and > 0");
    if (std::isnan(expansion)) return fail(KNN_ERR_INVALID_ARG, "expansion is NaN");
    if (climb != KNN_CLIMB_EAGER && climb != KNN_CLIMB_BEST)
        return fail(KNN_ERR_INVALID_ARG, "unknown climb %d", climb);
    g->p.speedup = speedup;
    g->p.expansion = expansion;
    g->climb = climb;
    return KNN_OK;
}

KNN_API knn_status knn_balanced_kmedoids(const float *X, int64_t n, int32_t dim, int32_t p,
                                         double imbalance, int32_t chunks, int32_t iters,
                                         uint64_t seed, int32_t *out_labels, int64_t *out_medoids,
                                         int64_t *out_order, int64_t *out_offsets, void *stream) {
    NvtxRange nvtx_range("knn_balanced_kmedoids");
    if (!X) return fail(KNN_ERR_INVALID_ARG, "null argument");
    if (dim < 1 || dim > 256) return fail(KNN_ERR_UNSUPPORTED, "dim %d outside 1..256", dim);
    if (p < 1 || p > KMED_MAX_P) return fail(KNN_ERR_UNSUPPORTED, "p %d outside 1..%d", p, KMED_MAX_P);
    if (n < p || n >= (int64_t)INT32_MAX) return fail(KNN_ERR_INVALID_ARG, "need p <= n < 2^31");
    if ((double)n * (double)p > 4294967296.0)
        return fail(KNN_ERR_UNSUPPORTED, "n * p above 2^32 (the point-medoid distance matrix)");
    if (!(imbalance >= 1.0)) return fail(KNN_ERR_INVALID_ARG, "imbalance must be >= 1");
    if (chunks < 1 || chunks > n) return fail(KNN_ERR_INVALID_ARG, "chunks %d outside 1..n", chunks);
    if (iters < 0 || iters > 1000) return fail(KNN_ERR_INVALID_ARG, "iters %d outside 0..1000", iters);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int dp = padded_dim(dim);
    // initial medoids: the first p distinct draws of the generator keyed (seed, 2^62)
    std::vector<int64_t> med0((size_t)p);
    {
        std::vector<char> taken((size_t)n, 0);
        const uint64_t key = restart_key(seed, 1ull << 62);
        int got = 0;
        for (uint64_t j = 0; got < p; ++j) {
            const uint32_t r = restart_node(key, j, (uint32_t)n);
            if (taken[r]) continue;
            taken[r] = 1;
            med0[(size_t)got++] = r;
        }
    }
    float *rows = nullptr, *D = nullptr, *xin = nullptr;
    int32_t *labels = nullptr;
    int64_t *medoids = nullptr, *order = nullptr, *offsets = nullptr;
    void *sort_scratch = nullptr;
    auto release = [&]() {
        for (void *q : {(void *)rows, (void *)D, (void *)xin, (void *)labels, (void *)medoids, (void *)order,
                        (void *)offsets, sort_scratch})
            if (q) cudaFreeAsync(q, s);
    };
    auto run = [&]() -> knn_status {
        CU(cudaMallocAsync(&rows, (size_t)n * dp * 4, s));
        CU(cudaMallocAsync(&D, (size_t)n * p * 4, s));
        CU(cudaMallocAsync(&labels, (size_t)n * 4, s));
        CU(cudaMallocAsync(&medoids, (size_t)p * 8, s));
        CU(cudaMallocAsync(&order, (size_t)n * 8, s));
        CU(cudaMallocAsync(&offsets, (size_t)(p + 1) * 8, s));
        CU(cudaMallocAsync(&sort_scratch, kmed_sort_scratch_bytes(n, p), s));
        const bool x_dev = is_device_ptr(X);
        if (!x_dev) {
            CU(cudaMallocAsync(&xin, (size_t)n * dim * 4, s));
            CU(cudaMemcpyAsync(xin, X, (size_t)n * dim * 4, cudaMemcpyHostToDevice, s));
        }
        CU(launch_append(x_dev ? X : xin, n, dim, dp, rows, nullptr, nullptr, nullptr, s));
        CU(cudaMemcpyAsync(medoids, med0.data(), (size_t)p * 8, cudaMemcpyHostToDevice, s));
        const double capacity = (double)n * imbalance / ((double)p * (double)chunks);
        for (int it = 0;; ++it) {
            CU(launch_kmed_dist(dp, rows, n, medoids, p, D, s));
            CU(launch_kmed_assign(D, n, p, chunks, capacity, labels, s));
            CU(launch_kmed_sort(labels, n, p, sort_scratch, order, offsets, s));
            if (it == iters) break;
            CU(launch_kmed_update(dp, rows, order, offsets, p, medoids, s));
        }
        auto out = [&](void *dst, const void *src, size_t bytes) -> cudaError_t {
            if (!dst) return cudaSuccess;
            return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s);
        };
        CU(out(out_labels, labels, (size_t)n * 4));
        CU(out(out_medoids, medoids, (size_t)p * 8));
        CU(out(out_order, order, (size_t)n * 8));
        CU(out(out_offsets, offsets, (size_t)(p + 1) * 8));
        return KNN_OK;
    };
    const knn_status st = run();
    release();
    if (st != KNN_OK) return st;
    CU(cudaStreamSynchronize(s));
    return KNN_OK;
}

KNN_API knn_status knn_exact_set_path(int32_t path) {
    if (path != KNN_EXACT_AUTO && path != KNN_EXACT_CUDA_CORES && path != KNN_EXACT_TENSOR_CORES)
        return fail(KNN_ERR_INVALID_ARG, "unknown exact path %d", path);
    g_exact_path.store(path);
    return KNN_OK;
}

KNN_API knn_status knn_exact_set_wait_limit(int64_t ns) {
    exact_tc_set_wait(ns);
    return KNN_OK;
}

KNN_API knn_status knn_exact_last_info(knn_exact_info *out) {
    if (!out) return fail(KNN_ERR_INVALID_ARG, "null argument");
    *out = g_exact_info;
    return KNN_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Several graphs in one arena (knn_multi_*)
// ---------------------------------------------------------------------------
struct knn_multi {
    knn_graph *g = nullptr;  // the arena: every graph's rows, lists and the step buffers
    int G = 0;
    std::vector<uint32_t> lo, cap;
    std::vector<int64_t> n;
    int64_t M = 0;           // items per step
    uint32_t cap_max = 0;
    bool use_graph = false;
    // device tables of a step, uploaded from one pinned block
    uint8_t *h_meta = nullptr, *d_meta = nullptr;
    size_t meta_bytes = 0;
    int32_t *d_counts = nullptr;  // m_all, m_ins, m_q
    int32_t *d_item_seg = nullptr;
    uint32_t *d_lo = nullptr, *d_n = nullptr;
    int32_t *d_first = nullptr, *d_perm = nullptr;
    uint64_t *d_streams = nullptr;
    float *h_vecs = nullptr, *d_vecs = nullptr;
    int64_t *d_out = nullptr, *h_out = nullptr;
    float *d_sims = nullptr, *h_sims = nullptr;
    int32_t search_warps = 0;            // warps of the search launch (0: max_batch)
    bool largest_first = false;          // search order of a step's items
    int32_t *d_order = nullptr;          // [M] that order (step table)
    cudaGraphExec_t exec = nullptr;
    cudaStream_t exec_stream = nullptr;  // a CUDA graph is captured on and replayed from its own stream
    cudaEvent_t joined = nullptr;
    int64_t steps = 0;
};

static size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// The step's kernels, reading every size from the device tables; the same
// sequence serves every step (and is what a CUDA graph captures).
static knn_status multi_launch(knn_multi *mg, cudaStream_t s) {
    knn_graph *g = mg->g;
    const int K = g->p.k, dp = g->dp, M = (int)mg->M;
    const bool screening = g->p.storage != KNN_STORAGE_FP32;
    const int KT = screening ? g->p.rescore_mult * K : K;
    const int64_t vwords = (mg->cap_max + 31) / 32;
    Segments all{mg->d_item_seg, mg->d_lo, mg->d_n, mg->d_first, mg->d_counts};
    Segments ins{mg->d_item_seg, mg->d_lo, mg->d_n, mg->d_first, mg->d_counts + 1};
    const int grid = g->sm_count * 4;
    CU(launch_multi_append(mg->d_vecs, mg->d_counts, ins, g->p.dim, dp, g->qbuf, g->X, g->Xb, g->X8, g->scale, grid,
                           s));
    if (!search_visited_on_chip(mg->cap_max))
        CU(cudaMemsetAsync(g->visited, 0, (size_t)M * vwords * sizeof(uint32_t), s));
    SearchArgs a{};
    a.rows = searched_rows(g);
    a.row_scale = g->scale;
    a.nbr = g->nbr_ids;
    a.removed = g->removed;
    a.queries = g->qbuf;
    a.q_stride = dp;
    a.visited = g->visited;
    a.vwords = vwords;
    a.out_keys = g->keys_search;
    a.counters = g->counters;
    a.totals = g->totals;
    a.m = mg->search_warps > 0 ? mg->search_warps : M;  // warps launched; the items come from the table
    a.k = K;
    a.KT = KT;
    a.seed = g->p.seed;
    const double e = g->p.expansion;
    a.discard = (e > 0.0 && std::isfinite(e)) ? 1 : 0;
    a.expansion = a.discard ? (float)e : 1.0f;
    a.climb = g->climb;
    a.speedup = g->p.speedup;
    a.vis_n = mg->cap_max;
    a.streams = mg->d_streams;
    a.seg = all;
    a.seg.order = mg->d_order;
    CU(launch_search(g->p.storage, dp, a, s));
    const uint64_t *keys = g->keys_search;
    if (screening) {
        RescoreArgs r{};
        r.rows = g->X;
        r.queries = g->qbuf;
        r.q_stride = dp;
        r.cand_keys = g->keys_search;
        r.out_keys = g->keys_final;
        r.totals = g->totals;
        r.m = M;
        r.KT = KT;
        r.k_out = K;
        r.m_dev = mg->d_counts;
        CU(launch_rescore(dp, r, s));
        keys = g->keys_final;
    }
    CrossArgs ca{};
    ca.rows = g->X;
    ca.in_keys = keys;
    ca.nbr_ids = g->nbr_ids;
    ca.nbr_d2 = g->nbr_d2;
    ca.totals = g->totals;
    ca.m = M;
    ca.k = K;
    ca.seg = ins;
    CU(launch_cross(dp, ca, s));
    CU(cudaMemsetAsync(g->small, 0, 2 * sizeof(unsigned), s));
    UpdateArgs ua{};
    ua.rows = g->X;
    ua.nbr_ids = g->nbr_ids;
    ua.nbr_d2 = g->nbr_d2;
    ua.removed = g->removed;
    ua.head = g->head;
    ua.offer_key = g->offer_key;
    ua.offer_next = g->offer_next;
    ua.touched = g->touched;
    ua.offer_count = g->small + 0;
    ua.touched_count = g->small + 1;
    ua.offer_cap = g->offer_cap;
    ua.error_flags = g->small + 2;
    ua.counters = g->counters;
    ua.totals = g->totals;
    ua.m = M;
    ua.k = K;
    ua.depth = g->p.depth;
    ua.frontier = g->frontier;
    ua.frontier_cap = g->frontier_cap;
    ua.seen = g->visited;
    ua.seen_words = vwords;
    ua.seg = ins;
    if (ua.depth >= 2 && !update_seen_on_chip(ua.seen_words))
        CU(cudaMemsetAsync(g->visited, 0, (size_t)M * ua.seen_words * sizeof(uint32_t), s));
    CU(launch_update(dp, ua, s));
    MergeArgs ma{};
    ma.nbr_ids = g->nbr_ids;
    ma.nbr_d2 = g->nbr_d2;
    ma.head = g->head;
    ma.offer_key = g->offer_key;
    ma.offer_next = g->offer_next;
    ma.touched = g->touched;
    ma.touched_count = g->small + 1;
    ma.offer_count = g->small + 0;
    ma.totals = g->totals;
    ma.k = K;
    CU(launch_merge(ma, g->sm_count, s));
    CU(launch_multi_keys_out(keys, mg->d_counts + 2, mg->d_counts + 1, K, K, mg->d_item_seg, mg->d_lo, mg->d_perm,
                             mg->d_out, mg->d_sims, grid, s));
    return KNN_OK;
}

static void free_multi(knn_multi *mg) {
    if (!mg) return;
    if (mg->exec) cudaGraphExecDestroy(mg->exec);
    if (mg->exec_stream) {
        cudaStreamSynchronize(mg->exec_stream);
        if (mg->g && mg->g->last_stream == mg->exec_stream) mg->g->last_stream = nullptr;
        cudaStreamDestroy(mg->exec_stream);
    }
    if (mg->joined) cudaEventDestroy(mg->joined);
    for (void *p : {(void *)mg->h_meta, (void *)mg->h_vecs, (void *)mg->h_out, (void *)mg->h_sims})
        if (p) cudaFreeHost(p);
    for (void *p : {(void *)mg->d_meta, (void *)mg->d_vecs, (void *)mg->d_out, (void *)mg->d_sims})
        if (p) cudaFree(p);
    if (mg->g) free_graph(mg->g);
    delete mg;
}

extern "C" {

KNN_API knn_status knn_multi_create(const knn_params *params, int32_t graphs, const int64_t *n_init,
                                    const int64_t *capacity, const float *init_vecs, int32_t use_graph,
                                    void *stream, knn_multi **out) {
    NvtxRange nvtx_range("knn_multi_create");
    if (!params || !n_init || !capacity || !init_vecs || !out) return fail(KNN_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    if (graphs < 1 || graphs > 65536) return fail(KNN_ERR_INVALID_ARG, "graphs %d outside 1..65536", graphs);
    int64_t total = 0, init_total = 0;
    for (int i = 0; i < graphs; ++i) {
        if (n_init[i] < params->k + 1 || capacity[i] < n_init[i])
            return fail(KNN_ERR_INVALID_ARG, "graph %d: need k+1 <= n_init <= capacity", i);
        total += capacity[i];
        init_total += n_init[i];
    }
    if (total >= (int64_t)INT32_MAX) return fail(KNN_ERR_CAPACITY, "capacities add up past 2^31");
    knn_params p = *params;
    p.capacity = total;
    TRY(validate_params(p, p.k + 1));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    knn_multi *mg = new knn_multi();
    mg->G = graphs;
    mg->use_graph = use_graph != 0;
    mg->M = p.max_batch;
    knn_status st = graph_alloc(p, s, &mg->g);
    if (st != KNN_OK) {
        delete mg;
        return st;
    }
    knn_graph *g = mg->g;
    g->n = total;  // every slot is addressable; each graph's size is its own
    auto build = [&]() -> knn_status {
        // step tables: counts[4] | item_seg[M] | lo[G] | n[G] | first[G+1] | perm[M] | streams[M] |
        // order[M]
        const size_t M = (size_t)mg->M, Gs = (size_t)graphs;
        mg->meta_bytes = align_up(16, 16) + align_up(M * 4, 16) + 2 * align_up(Gs * 4, 16) +
                         align_up((Gs + 1) * 4, 16) + align_up(M * 4, 16) + align_up(M * 8, 16) +
                         align_up(M * 4, 16);
        CU(cudaMallocHost(&mg->h_meta, mg->meta_bytes));
        CU(cudaMalloc(&mg->d_meta, mg->meta_bytes));
        size_t off = 0;
        auto carve = [&](size_t bytes) {
            uint8_t *q = mg->d_meta + off;
            off += align_up(bytes, 16);
            return q;
        };
        mg->d_counts = (int32_t *)carve(16);
        mg->d_item_seg = (int32_t *)carve(M * 4);
        mg->d_lo = (uint32_t *)carve(Gs * 4);
        mg->d_n = (uint32_t *)carve(Gs * 4);
        mg->d_first = (int32_t *)carve((Gs + 1) * 4);
        mg->d_perm = (int32_t *)carve(M * 4);
        mg->d_streams = (uint64_t *)carve(M * 8);
        mg->d_order = (int32_t *)carve(M * 4);
        CU(cudaMallocHost(&mg->h_vecs, M * p.dim * 4));
        CU(cudaMalloc(&mg->d_vecs, M * p.dim * 4));
        CU(cudaMallocHost(&mg->h_out, M * p.k * 8));
        CU(cudaMalloc(&mg->d_out, M * p.k * 8));
        CU(cudaMallocHost(&mg->h_sims, M * p.k * 4));
        CU(cudaMalloc(&mg->d_sims, M * p.k * 4));
        if (mg->use_graph) {
            CU(cudaStreamCreateWithFlags(&mg->exec_stream, cudaStreamNonBlocking));
            CU(cudaEventCreateWithFlags(&mg->joined, cudaEventDisableTiming));
        }
        // the graphs, one after another, each with its exact initial graph
        int64_t base = 0, row = 0;
        for (int i = 0; i < graphs; ++i) {
            mg->lo.push_back((uint32_t)base);
            mg->cap.push_back((uint32_t)capacity[i]);
            mg->n.push_back(n_init[i]);
            mg->cap_max = std::max(mg->cap_max, (uint32_t)capacity[i]);
            TRY(append_rows(g, init_vecs + row * p.dim, n_init[i], base, g->X, true, s));
            ExactArgs ea{};
            ea.X = g->X + base * g->dp;
            ea.out_ids = g->nbr_ids + base * p.k;
            ea.out_d2 = g->nbr_d2 + base * p.k;
            ea.n = n_init[i];
            ea.k = p.k;
            TRY(run_exact(g->dp, ea, s, &g->launches));
            CU(launch_shift_ids(g->nbr_ids + base * p.k, n_init[i] * p.k, (int32_t)base, s));
            base += capacity[i];
            row += n_init[i];
        }
        CU(cudaStreamSynchronize(s));
        return KNN_OK;
    };
    st = build();
    if (st != KNN_OK) {
        free_multi(mg);
        return st;
    }
    (void)init_total;
    *out = mg;
    return KNN_OK;
}

KNN_API knn_status knn_multi_step(knn_multi *mg, const float *vecs, const int32_t *graph, const int32_t *kind,
                                  const uint64_t *query_ids, int64_t m, int64_t *out_ids, float *out_sims,
                                  void *stream) {
    NvtxRange nvtx_range("knn_multi_step");
    if (!mg || !vecs || !graph || !kind || !out_ids) return fail(KNN_ERR_INVALID_ARG, "null argument");
    if (m < 1 || m > mg->M) return fail(KNN_ERR_INVALID_ARG, "m = %lld outside 1..max_batch", (long long)m);
    knn_graph *g = mg->g;
    DeviceGuard dg(g->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (mg->use_graph) {
        // work on the graph's own stream, after what the caller's stream has queued
        CU(cudaEventRecord(mg->joined, s));
        CU(cudaStreamWaitEvent(mg->exec_stream, mg->joined, 0));
        s = mg->exec_stream;
    }
    g->last_stream = s;
    const int G = mg->G, d = g->p.dim, K = g->p.k;
    // order: inserts grouped by graph (in given order), then queries
    std::vector<int64_t> ins_count((size_t)G, 0);
    int64_t m_ins = 0;
    for (int64_t i = 0; i < m; ++i) {
        if (graph[i] < 0 || graph[i] >= G) return fail(KNN_ERR_INVALID_ARG, "item %lld: bad graph", (long long)i);
        if (kind[i] != KNN_REQ_INSERT && kind[i] != KNN_REQ_QUERY)
            return fail(KNN_ERR_INVALID_ARG, "item %lld: bad kind", (long long)i);
        if (kind[i] == KNN_REQ_INSERT) {
            ++ins_count[(size_t)graph[i]];
            ++m_ins;
        } else if (!query_ids) {
            return fail(KNN_ERR_INVALID_ARG, "query items need query_ids");
        }
    }
    for (int i = 0; i < G; ++i)
        if (mg->n[(size_t)i] + ins_count[(size_t)i] > mg->cap[(size_t)i])
            return fail(KNN_ERR_CAPACITY, "graph %d full", i);
    uint8_t *h = mg->h_meta;
    size_t off = 0;
    auto carve = [&](size_t bytes) {
        uint8_t *q = h + off;
        off += align_up(bytes, 16);
        return q;
    };
    const size_t M = (size_t)mg->M, Gs = (size_t)G;
    int32_t *counts = (int32_t *)carve(16);
    int32_t *item_seg = (int32_t *)carve(M * 4);
    uint32_t *lo = (uint32_t *)carve(Gs * 4);
    uint32_t *nn = (uint32_t *)carve(Gs * 4);
    int32_t *first = (int32_t *)carve((Gs + 1) * 4);
    int32_t *perm = (int32_t *)carve(M * 4);
    uint64_t *streams = (uint64_t *)carve(M * 8);
    int32_t *order = (int32_t *)carve(M * 4);
    first[0] = 0;
    for (int i = 0; i < G; ++i) {
        lo[i] = mg->lo[(size_t)i];
        nn[i] = (uint32_t)mg->n[(size_t)i];
        first[i + 1] = first[i] + (int32_t)ins_count[(size_t)i];
    }
    std::vector<int32_t> cursor(first, first + G);
    int32_t qpos = (int32_t)m_ins;
    for (int64_t i = 0; i < m; ++i) {
        int32_t slot;
        if (kind[i] == KNN_REQ_INSERT) {
            const int gi = graph[i];
            slot = cursor[(size_t)gi]++;
            streams[slot] = mg->n[(size_t)gi] + (uint64_t)(slot - first[gi]);  // the new node's local id
        } else {
            slot = qpos++;
            streams[slot] = (1ull << 63) + query_ids[i];
        }
        item_seg[slot] = graph[i];
        perm[slot] = (int32_t)i;
        std::memcpy(mg->h_vecs + (size_t)slot * d, vecs + i * d, (size_t)d * 4);
    }
    // the order the search takes the items in: as packed, or the items of the
    // largest graphs first (a search's length grows with its graph, so the
    // longest ones start in the first round of a persistent launch)
    for (int32_t i = 0; i < (int32_t)m; ++i) order[i] = i;
    if (mg->largest_first) {
        std::stable_sort(order, order + m, [&](int32_t x, int32_t y) {
            return mg->n[(size_t)item_seg[x]] > mg->n[(size_t)item_seg[y]];
        });
    }
    counts[0] = (int32_t)m;
    counts[1] = (int32_t)m_ins;
    counts[2] = (int32_t)(m - m_ins);
    counts[3] = 0;
    CU(cudaMemcpyAsync(mg->d_meta, mg->h_meta, mg->meta_bytes, cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(mg->d_vecs, mg->h_vecs, (size_t)m * d * 4, cudaMemcpyHostToDevice, s));
    if (mg->use_graph && mg->steps >= 1) {
        if (!mg->exec) {
            // capture the launch sequence once (the first step ran it directly)
            cudaGraph_t graph_obj = nullptr;
            CU(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
            const knn_status st = multi_launch(mg, s);
            const cudaError_t ec = cudaStreamEndCapture(s, &graph_obj);
            if (st != KNN_OK) return st;
            CU(ec);
            const cudaError_t ei = cudaGraphInstantiate(&mg->exec, graph_obj, 0);
            cudaGraphDestroy(graph_obj);
            CU(ei);
        }
        CU(cudaGraphLaunch(mg->exec, s));
        g->launches += 1;
    } else {
        TRY(multi_launch(mg, s));
        g->launches += 9;
    }
    CU(cudaMemcpyAsync(mg->h_out, mg->d_out, (size_t)m * K * 8, cudaMemcpyDeviceToHost, s));
    if (out_sims) CU(cudaMemcpyAsync(mg->h_sims, mg->d_sims, (size_t)m * K * 4, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    for (int64_t i = 0; i < m; ++i) {
        if (kind[i] == KNN_REQ_QUERY) {
            std::memcpy(out_ids + i * K, mg->h_out + i * K, (size_t)K * 8);
            if (out_sims) std::memcpy(out_sims + i * K, mg->h_sims + i * K, (size_t)K * 4);
        }
    }
    for (int i = 0; i < G; ++i) {
        for (int32_t slot = first[i]; slot < first[i + 1]; ++slot) {
            const int64_t orig = perm[slot];
            out_ids[orig * K] = mg->n[(size_t)i] + (slot - first[i]);
            for (int c = 1; c < K; ++c) out_ids[orig * K + c] = -1;
            if (out_sims)
                for (int c = 0; c < K; ++c) out_sims[orig * K + c] = 0.f;
        }
        mg->n[(size_t)i] += ins_count[(size_t)i];
    }
    g->inserts += m_ins;
    g->queries += m - m_ins;
    g->last_m = m;
    ++mg->steps;
    return KNN_OK;
}

KNN_API knn_status knn_multi_set_order(knn_multi *mg, int32_t largest_first) {
    if (!mg || (largest_first != 0 && largest_first != 1)) return fail(KNN_ERR_INVALID_ARG, "bad argument");
    mg->largest_first = largest_first != 0;
    return KNN_OK;
}

KNN_API knn_status knn_multi_set_launch(knn_multi *mg, int32_t search_warps) {
    if (!mg || search_warps < 0) return fail(KNN_ERR_INVALID_ARG, "bad argument");
    if (search_warps != mg->search_warps && mg->exec) {
        cudaStreamSynchronize(mg->exec_stream);
        cudaGraphExecDestroy(mg->exec);  // captured with the old launch: capture again
        mg->exec = nullptr;
    }
    mg->search_warps = search_warps;
    return KNN_OK;
}

KNN_API knn_status knn_multi_graph_size(knn_multi *mg, int32_t graph, int64_t *n, int64_t *capacity) {
    if (!mg || graph < 0 || graph >= mg->G) return fail(KNN_ERR_INVALID_ARG, "bad graph");
    if (n) *n = mg->n[(size_t)graph];
    if (capacity) *capacity = mg->cap[(size_t)graph];
    return KNN_OK;
}

KNN_API knn_status knn_multi_get_edges(knn_multi *mg, int32_t graph, int64_t *out_ids, void *stream) {
    if (!mg || !out_ids || graph < 0 || graph >= mg->G) return fail(KNN_ERR_INVALID_ARG, "bad argument");
    knn_graph *g = mg->g;
    DeviceGuard dg(g->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int K = g->p.k;
    const int64_t n = mg->n[(size_t)graph], base = mg->lo[(size_t)graph];
    std::vector<int32_t> ids((size_t)(n * K));
    CU(cudaMemcpyAsync(ids.data(), g->nbr_ids + base * K, ids.size() * 4, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    std::vector<int64_t> local(ids.size());
    for (size_t i = 0; i < ids.size(); ++i) local[i] = ids[i] < 0 ? -1 : (int64_t)ids[i] - base;
    CU(cudaMemcpyAsync(out_ids, local.data(), local.size() * 8, cudaMemcpyDefault, s));
    CU(cudaStreamSynchronize(s));
    return KNN_OK;
}

KNN_API void knn_multi_destroy(knn_multi *mg) {
    if (!mg) return;
    DeviceGuard dg(mg->g->device);
    cudaStreamSynchronize(mg->g->last_stream);
    free_multi(mg);
}

}  // extern "C"
