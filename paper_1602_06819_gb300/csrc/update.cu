// update.cu -- the Update step (Algorithm 2) for a batch of new points, the
// intra-batch cross-merge, and the FP32 re-score of screening candidates.
//
// Algorithm 2 walks from the neighbours found by the search: each node popped
// at depth d has its list read (for depth d+1), gets sim(new, node) computed
// and is offered `new` (it enters when it ranks in the list's best k).  For a
// batch of m new points this runs in three kernels and never waits on a lock:
//
//   cross   one warp per new point: its list = the best k of its search
//           result and the exact similarities to the other m-1 points of the
//           batch (in the sequential build a point sees the ones before it;
//           the batch sees all of them, both ways).
//   offers  one warp per new point: level 1 is its list (similarities known);
//           level 2 is the distinct ids of those nodes' lists minus the ones
//           already seen, minus `new`, minus removed nodes.  Every level reads
//           lists as they stood before the batch, so no read waits on a write.
//           A candidate (node, new) that does not beat the node's current
//           last entry cannot enter its list and is dropped; the others are
//           pushed onto a per-node chain with atomicExch.
//   merge   one warp per node that received candidates: the best k of its
//           list and its chain, written back sorted.  The best k of a set
//           under a strict total order does not depend on the order the
//           candidates arrived in, so the result is the same as any sequence
//           of single offers.
//
// Points of the batch appear in each other's lists through the cross-merge
// only: the offers kernel offers `new` to nodes that existed before the batch.
#include "common.cuh"
#include "kernels.h"

namespace knn {

constexpr int UPD_WARPS = 4;

// ---------------------------------------------------------------------------
// FP32 re-score of screening candidates (best KT by screening distance).
// ---------------------------------------------------------------------------
template <int DP>
__device__ __forceinline__ void rescore_item(const RescoreArgs &a, int item, int lane) {
    using C = RowCfg<ST_FP32, DP>;
    float qv[C::QF];
    load_query<ST_FP32, DP>(a.queries + (size_t)item * a.q_stride, qv);
    const RowSource src{reinterpret_cast<const uint8_t *>(a.rows), nullptr};
    WarpTop<1> top;
    top.init(a.k_out);
    long long n_scored = 0;
    for (int c0 = 0; c0 < a.KT; c0 += 32) {
        const uint64_t ck = (c0 + lane < a.KT) ? a.cand_keys[(size_t)item * a.KT + c0 + lane] : KEY_EMPTY;
        const int nr = __popc(__ballot_sync(FULL, ck != KEY_EMPTY));  // sorted: empties last
        if (nr == 0) break;
        const uint32_t id = key_id(ck);
        const float d2 = gather_d2<ST_FP32, DP>(src, id, nr, qv);
        for (int i = 0; i < nr; ++i) {
            const uint64_t key = pack_key(__shfl_sync(FULL, d2, i), __shfl_sync(FULL, id, i));
            top.offer(key);
        }
        n_scored += nr;
    }
    if (lane < a.k_out) a.out_keys[(size_t)item * a.k_out + lane] = top.e[0];
    if (lane == 0) atomicAdd(a.totals + TOT_RESCORE_EVALS, (unsigned long long)n_scored);
}

template <int DP>
__global__ void __launch_bounds__(UPD_WARPS * 32) rescore_kernel(const RescoreArgs a) {
    const int lane = threadIdx.x & 31;
    const int m = a.m_dev ? *a.m_dev : a.m;
    for (int item = blockIdx.x * UPD_WARPS + (threadIdx.x >> 5); item < m; item += gridDim.x * UPD_WARPS)
        rescore_item<DP>(a, item, lane);
}

// ---------------------------------------------------------------------------
// Cross-merge among the points of one batch.  FUSED: the list of new point i
// is the best k of its search result and of the other points of its batch.
// Split in two for a single graph: cross_topk keeps the best k among the
// batch (it needs no search result and runs beside the search) and
// cross_merge then takes the best k of the two lists.  Keys are unique (a
// search finds old nodes, the batch holds new ones), so both give the same
// list: the best k of a union are the best k of the two lists' best k.
// ---------------------------------------------------------------------------
enum { CROSS_FUSED = 0, CROSS_TOPK = 1 };

template <int DP, int MODE>
__device__ __forceinline__ void cross_item(const CrossArgs &a, int i, int lane) {
    using C = RowCfg<ST_FP32, DP>;
    // the new point's id and the batch points it meets: those of its graph
    uint32_t id0 = a.n;
    int j_lo = 0, j_hi = a.m;
    if (a.seg.item_seg) {
        const int sg = a.seg.item_seg[i];
        j_lo = a.seg.first[sg];
        j_hi = a.seg.first[sg + 1];
        id0 = a.seg.lo[sg] + a.seg.n[sg];
    }
    const uint32_t new_id = id0 + (uint32_t)(i - j_lo);
    float qv[C::QF];
    load_query<ST_FP32, DP>(a.rows + (size_t)new_id * DP, qv);
    const RowSource src{reinterpret_cast<const uint8_t *>(a.rows), nullptr};
    WarpTop<1> top;
    top.init(a.k);
    if (MODE == CROSS_FUSED) {
        top.e[0] = lane < a.k ? a.in_keys[(size_t)i * a.k + lane] : KEY_EMPTY;
        top.worst = top.entry(a.k - 1);
    }
    for (int j0 = j_lo; j0 < j_hi; j0 += 32) {
        const int nr = j_hi - j0 < 32 ? j_hi - j0 : 32;
        const uint32_t id = id0 + (uint32_t)(j0 - j_lo + lane);
        const float d2 = gather_d2<ST_FP32, DP>(src, id, nr, qv);
        for (int t = 0; t < nr; ++t) {
            if (j0 + t == i) continue;
            top.offer(pack_key(__shfl_sync(FULL, d2, t), id0 + (uint32_t)(j0 - j_lo + t)));
        }
    }
    if (MODE == CROSS_TOPK) {
        if (lane < a.k) a.cross_keys[(size_t)i * a.k + lane] = top.e[0];
    } else if (lane < a.k) {
        const uint64_t key = top.e[0];
        a.nbr_ids[(size_t)new_id * a.k + lane] = key == KEY_EMPTY ? -1 : (int32_t)key_id(key);
        a.nbr_d2[(size_t)new_id * a.k + lane] = key == KEY_EMPTY ? __int_as_float(0x7f800000) : key_d2(key);
    }
    if (lane == 0 && j_hi - j_lo > 1) atomicAdd(a.totals + TOT_CROSS_EVALS, (unsigned long long)(j_hi - j_lo - 1));
}

template <int DP, int MODE>
__global__ void __launch_bounds__(UPD_WARPS * 32) cross_kernel(const CrossArgs a) {
    const int lane = threadIdx.x & 31;
    const int m = a.seg.count ? *a.seg.count : a.m;
    for (int i = blockIdx.x * UPD_WARPS + (threadIdx.x >> 5); i < m; i += gridDim.x * UPD_WARPS)
        cross_item<DP, MODE>(a, i, lane);
}

// The list of new point i: the best k of its search result (in_keys) and of
// its best k among the batch (cross_keys); a single graph only.
__global__ void __launch_bounds__(UPD_WARPS * 32) cross_merge_kernel(const CrossArgs a) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * UPD_WARPS + (threadIdx.x >> 5);
    if (i >= a.m) return;  // warp-uniform
    WarpTop<1> top;
    top.init(a.k);
    top.e[0] = lane < a.k ? a.in_keys[(size_t)i * a.k + lane] : KEY_EMPTY;
    top.worst = top.entry(a.k - 1);
    const uint64_t ck = lane < a.k ? a.cross_keys[(size_t)i * a.k + lane] : KEY_EMPTY;
    for (int t = 0; t < a.k; ++t) {
        const uint64_t key = shfl_u64(ck, t);
        if (key == KEY_EMPTY || !top.offer(key)) break;  // the batch list is sorted
    }
    const uint32_t new_id = a.n + (uint32_t)i;
    if (lane < a.k) {
        const uint64_t key = top.e[0];
        a.nbr_ids[(size_t)new_id * a.k + lane] = key == KEY_EMPTY ? -1 : (int32_t)key_id(key);
        a.nbr_d2[(size_t)new_id * a.k + lane] = key == KEY_EMPTY ? __int_as_float(0x7f800000) : key_d2(key);
    }
}

// ---------------------------------------------------------------------------
// Offers: levels 1 and 2 of Algorithm 2.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t list_last_key(const UpdateArgs &a, uint32_t w) {
    const size_t off = (size_t)w * a.k + (a.k - 1);
    const int32_t id = __ldg(a.nbr_ids + off);
    return id < 0 ? KEY_EMPTY : pack_key(__ldg(a.nbr_d2 + off), (uint32_t)id);
}

// Push the lanes' candidates (has: lane holds one) onto their nodes' chains.
__device__ __forceinline__ void push_offers(const UpdateArgs &a, bool has, uint32_t w, uint64_t key) {
    const int lane = threadIdx.x & 31;
    const unsigned bal = __ballot_sync(FULL, has);
    if (bal == 0u) return;
    const int leader = __ffs(bal) - 1;
    unsigned base = 0;
    if (lane == leader) base = atomicAdd(a.offer_count, (unsigned)__popc(bal));
    base = __shfl_sync(FULL, base, leader);
    if (has) {
        const unsigned idx = base + (unsigned)__popc(bal & ((1u << lane) - 1u));
        if (idx < a.offer_cap) {
            a.offer_key[idx] = key;
            const int prev = atomicExch(a.head + w, (int)idx);
            a.offer_next[idx] = prev;
            if (prev < 0) a.touched[atomicAdd(a.touched_count, 1u)] = (int32_t)w;
        } else {
            atomicOr(a.error_flags, (unsigned)ERR_OFFER_OVERFLOW);
        }
    }
}

// Rows of Update levels: while the "seen" bitsets of a block's warps fit
// in 110 KiB of shared memory they live there, otherwise in global memory
// (cleared by the host before the launch).
constexpr size_t UPD_SMEM_SEEN_MAX = 110 * 1024;

template <int DP, bool SMEM_SEEN>
__device__ __forceinline__ void offers_item(const UpdateArgs &a, int i, int lane, int wib, uint32_t *smem_seen) {
    using C = RowCfg<ST_FP32, DP>;
    const unsigned lt_mask = (1u << lane) - 1u;
    // the new point, the end of its graph before the batch (nodes at or past
    // it are points of this batch) and the first node of its graph
    uint32_t new_id = a.n + (uint32_t)i, pre = a.n, base = 0u;
    if (a.seg.item_seg) {
        const int sg = a.seg.item_seg[i];
        base = a.seg.lo[sg];
        pre = base + a.seg.n[sg];
        new_id = pre + (uint32_t)(i - a.seg.first[sg]);
    }
    const RowSource src{reinterpret_cast<const uint8_t *>(a.rows), nullptr};

    // level 1: the new point's list (similarities known from the search)
    const int32_t lid = lane < a.k ? __ldg(a.nbr_ids + (size_t)new_id * a.k + lane) : -1;
    const float ld2 = lane < a.k ? __ldg(a.nbr_d2 + (size_t)new_id * a.k + lane) : 0.0f;
    {
        bool has = false;
        uint64_t key = 0;
        if (lid >= 0 && (uint32_t)lid < pre &&
            !((__ldg(a.removed + (lid >> 5)) >> (lid & 31)) & 1u)) {
            key = pack_key(ld2, new_id);
            has = key < list_last_key(a, (uint32_t)lid);
        }
        push_offers(a, has, (uint32_t)lid, key);
    }

    int upd_evals = 0;
    if (a.depth >= 2) {
        // seen = new, every node of the levels so far; an atomic test-and-set
        // makes each id enter at most one level
        uint32_t *seen;
        if constexpr (SMEM_SEEN) {
            seen = smem_seen + (size_t)wib * a.seen_words;
            for (int64_t w = lane; w < a.seen_words; w += 32) seen[w] = 0u;
        } else {
            seen = a.seen + (size_t)i * a.seen_words;
        }
        __syncwarp();
        if (lane == 0) atomicOr(seen + ((new_id - base) >> 5), 1u << ((new_id - base) & 31));
        if (lid >= 0) atomicOr(seen + (((uint32_t)lid - base) >> 5), 1u << (((uint32_t)lid - base) & 31));
        int32_t *level = a.frontier + (size_t)i * a.frontier_cap;  // the levels, one after another
        if (lane < a.k) level[lane] = lid;
        int lo = 0, hi = a.k;  // the current level is level[lo .. hi)
        __syncwarp();
        float qv[C::QF];
        load_query<ST_FP32, DP>(a.rows + (size_t)new_id * DP, qv);
        const int per = 32 / a.k;  // parents expanded per step
        const int pl = lane / a.k, el = lane % a.k;
        for (int t = 2; t <= a.depth && lo < hi; ++t) {
            // level t = distinct ids of the level t-1 lists, minus seen, minus
            // removed nodes and points of this batch
            int nhi = hi;
            for (int p0 = lo; p0 < hi; p0 += per) {
                int32_t u = -1;
                if (pl < per && p0 + pl < hi) u = level[p0 + pl];
                int32_t w = -1;
                if (u >= 0) w = __ldg(a.nbr_ids + (size_t)u * a.k + el);
                bool keep = false;
                if (w >= 0) {
                    const uint32_t wl = (uint32_t)w - base;
                    const uint32_t bit = 1u << (wl & 31);
                    const uint32_t old = atomicOr(seen + (wl >> 5), bit);
                    keep = !(old & bit) && (uint32_t)w < pre &&
                           !((__ldg(a.removed + (w >> 5)) >> (w & 31)) & 1u);
                }
                const unsigned km = __ballot_sync(FULL, keep);
                if (keep) {
                    const int idx = nhi + __popc(km & lt_mask);
                    if (idx < a.frontier_cap) level[idx] = w;
                    else atomicOr(a.error_flags, (unsigned)ERR_OFFER_OVERFLOW);
                }
                nhi += __popc(km);
            }
            if (nhi > a.frontier_cap) nhi = (int)a.frontier_cap;
            __syncwarp();
            // compute sim(new, node) for the level and offer `new` to the node
            for (int f0 = hi; f0 < nhi; f0 += 32) {
                const int nr = nhi - f0 < 32 ? nhi - f0 : 32;
                const uint32_t w = lane < nr ? (uint32_t)level[f0 + lane] : 0u;
                const float d2 = gather_d2<ST_FP32, DP>(src, w, nr, qv);
                bool has = false;
                uint64_t key = 0;
                if (lane < nr) {
                    key = pack_key(d2, new_id);
                    has = key < list_last_key(a, w);
                }
                push_offers(a, has, w, key);
            }
            upd_evals += nhi - hi;
            lo = hi;
            hi = nhi;
        }
    }
    if (lane == 0) {
        a.counters[(size_t)i * NCTR + CTR_UPDATE_EVALS] = upd_evals;
        atomicAdd(a.totals + TOT_UPDATE_EVALS, (unsigned long long)upd_evals);
    }
}

template <int DP, bool SMEM_SEEN>
__global__ void __launch_bounds__(UPD_WARPS * 32) update_offers_kernel(const UpdateArgs a) {
    extern __shared__ uint32_t smem_seen[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int m = a.seg.count ? *a.seg.count : a.m;
    for (int i = blockIdx.x * UPD_WARPS + wib; i < m; i += gridDim.x * UPD_WARPS) {
        offers_item<DP, SMEM_SEEN>(a, i, lane, wib, smem_seen);
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Merge: best k of each touched node's list and its chain of candidates.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(UPD_WARPS * 32) update_merge_kernel(const MergeArgs a) {
    const int lane = threadIdx.x & 31;
    const unsigned n_touched = *a.touched_count;
    const unsigned n_offers = *a.offer_count;
    const unsigned nwarps = gridDim.x * UPD_WARPS;
    unsigned long long merged = 0;
    for (unsigned t = blockIdx.x * UPD_WARPS + (threadIdx.x >> 5); t < n_touched; t += nwarps) {
        const int32_t w = a.touched[t];
        const size_t off = (size_t)w * a.k;
        WarpTop<1> top;
        top.init(a.k);
        if (lane < a.k) {
            const int32_t id = a.nbr_ids[off + lane];
            top.e[0] = id < 0 ? KEY_EMPTY : pack_key(a.nbr_d2[off + lane], (uint32_t)id);
        }
        top.worst = top.entry(a.k - 1);
        int idx = a.head[w];
        unsigned steps = 0;
        while (idx >= 0 && steps < n_offers) {  // a chain never exceeds the offers made
            top.offer(a.offer_key[idx]);
            idx = a.offer_next[idx];
            ++steps;
        }
        if (lane < a.k) {
            const uint64_t key = top.e[0];
            a.nbr_ids[off + lane] = key == KEY_EMPTY ? -1 : (int32_t)key_id(key);
            a.nbr_d2[off + lane] = key == KEY_EMPTY ? __int_as_float(0x7f800000) : key_d2(key);
        }
        if (lane == 0) a.head[w] = -1;
        merged += steps;
    }
    if (lane == 0 && merged) atomicAdd(a.totals + TOT_OFFERS, merged);
}

// ---------------------------------------------------------------------------
// Snapshot restore: one warp per node copies its list (checking each id) and
// recomputes the squared distances of the entries, keeping the given order.
// ---------------------------------------------------------------------------
template <int DP>
__global__ void __launch_bounds__(UPD_WARPS * 32)
restore_lists_kernel(const float *rows, const int64_t *in_ids, int64_t n, int k, int32_t *nbr_ids,
                     float *nbr_d2, unsigned *bad) {
    using C = RowCfg<ST_FP32, DP>;
    const int lane = threadIdx.x & 31;
    const int64_t u = (int64_t)blockIdx.x * UPD_WARPS + (threadIdx.x >> 5);
    if (u >= n) return;
    int64_t v = lane < k ? in_ids[u * k + lane] : -1;
    if (lane < k && (v < -1 || v >= n || v == u)) {
        atomicOr(bad, 1u);
        v = -1;
    }
    // entries are gathered in list order; empty slots sit at the end
    const unsigned valid = __ballot_sync(FULL, v >= 0);
    const int nv = __popc(valid);
    float qv[C::QF];
    load_query<ST_FP32, DP>(rows + u * DP, qv);
    const RowSource src{reinterpret_cast<const uint8_t *>(rows), nullptr};
    const float d2 = gather_d2<ST_FP32, DP>(src, (uint32_t)(v < 0 ? 0 : v), nv, qv);
    if (lane < k) {
        const bool ok = v >= 0 && lane < nv && ((valid >> lane) & 1u);
        nbr_ids[u * k + lane] = ok ? (int32_t)v : -1;
        nbr_d2[u * k + lane] = ok ? d2 : __int_as_float(0x7f800000);
        if (v >= 0 && !ok) atomicOr(bad, 2u);  // an entry after an empty slot
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <int DP>
static cudaError_t rescore_dp(const RescoreArgs &a, cudaStream_t s) {
    rescore_kernel<DP><<<(a.m + UPD_WARPS - 1) / UPD_WARPS, UPD_WARPS * 32, 0, s>>>(a);
    return cudaGetLastError();
}
template <int DP>
static cudaError_t cross_dp(const CrossArgs &a, cudaStream_t s) {
    cross_kernel<DP, CROSS_FUSED><<<(a.m + UPD_WARPS - 1) / UPD_WARPS, UPD_WARPS * 32, 0, s>>>(a);
    return cudaGetLastError();
}
template <int DP>
static cudaError_t update_dp(const UpdateArgs &a, cudaStream_t s) {
    const int grid = (a.m + UPD_WARPS - 1) / UPD_WARPS;
    const size_t smem = (size_t)UPD_WARPS * a.seen_words * sizeof(uint32_t);
    if (a.depth >= 2 && update_seen_on_chip(a.seen_words)) {
        cudaError_t e = cudaFuncSetAttribute(update_offers_kernel<DP, true>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        update_offers_kernel<DP, true><<<grid, UPD_WARPS * 32, smem, s>>>(a);
    } else {
        update_offers_kernel<DP, false><<<grid, UPD_WARPS * 32, 0, s>>>(a);
    }
    return cudaGetLastError();
}

#define KNN_DP_DISPATCH(FN, DPVAR, ...)                    \
    switch (DPVAR) {                                       \
        case 16: return FN<16>(__VA_ARGS__);               \
        case 32: return FN<32>(__VA_ARGS__);               \
        case 64: return FN<64>(__VA_ARGS__);               \
        case 96: return FN<96>(__VA_ARGS__);               \
        case 128: return FN<128>(__VA_ARGS__);             \
        case 256: return FN<256>(__VA_ARGS__);             \
        default: return cudaErrorInvalidValue;             \
    }

cudaError_t launch_rescore(int dp, const RescoreArgs &a, cudaStream_t s) {
    if (a.m <= 0) return cudaSuccess;
    KNN_DP_DISPATCH(rescore_dp, dp, a, s)
}

cudaError_t launch_cross(int dp, const CrossArgs &a, cudaStream_t s) {
    if (a.m <= 0) return cudaSuccess;
    KNN_DP_DISPATCH(cross_dp, dp, a, s)
}

template <int DP>
static cudaError_t cross_topk_dp(const CrossArgs &a, cudaStream_t s) {
    cross_kernel<DP, CROSS_TOPK><<<(a.m + UPD_WARPS - 1) / UPD_WARPS, UPD_WARPS * 32, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_cross_topk(int dp, const CrossArgs &a, cudaStream_t s) {
    if (a.m <= 0) return cudaSuccess;
    KNN_DP_DISPATCH(cross_topk_dp, dp, a, s)
}

cudaError_t launch_cross_merge(const CrossArgs &a, cudaStream_t s) {
    if (a.m <= 0) return cudaSuccess;
    cross_merge_kernel<<<(a.m + UPD_WARPS - 1) / UPD_WARPS, UPD_WARPS * 32, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_update(int dp, const UpdateArgs &a, cudaStream_t s) {
    if (a.m <= 0) return cudaSuccess;
    KNN_DP_DISPATCH(update_dp, dp, a, s)
}

template <int DP>
static cudaError_t restore_dp(const float *rows, const int64_t *in_ids, int64_t n, int k, int32_t *nbr_ids,
                              float *nbr_d2, unsigned *bad, cudaStream_t s) {
    restore_lists_kernel<DP><<<(unsigned)((n + UPD_WARPS - 1) / UPD_WARPS), UPD_WARPS * 32, 0, s>>>(
        rows, in_ids, n, k, nbr_ids, nbr_d2, bad);
    return cudaGetLastError();
}

cudaError_t launch_restore_lists(int dp, const float *rows, const int64_t *in_ids, int64_t n, int k,
                                 int32_t *nbr_ids, float *nbr_d2, unsigned *bad, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    KNN_DP_DISPATCH(restore_dp, dp, rows, in_ids, n, k, nbr_ids, nbr_d2, bad, s)
}

bool update_seen_on_chip(int64_t seen_words) {
    return (size_t)UPD_WARPS * seen_words * sizeof(uint32_t) <= UPD_SMEM_SEEN_MAX;
}

cudaError_t launch_merge(const MergeArgs &a, int sm_count, cudaStream_t s) {
    update_merge_kernel<<<sm_count * 16, UPD_WARPS * 32, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace knn
