// search.cuh -- iGNNS graph search (Sec. 3), one warp per query.
//
// Each warp runs the sequential search of one query exactly as the paper
// states it: random restarts (draws from the query's own counter-based
// stream), the expansion test that discards a restart r when
// sim(q, r) < s_max / e, eager hill climbing that moves to the first
// neighbour (in list order) strictly more similar than the current node, a
// visited set so that no similarity is computed twice, and a budget of
// B = max(1, floor(n / speedup)) similarity computations.
//
// The decisions are sequential, but the row gathers need not be: the
// similarity of a drawn node does not depend on the search state, so the
// warp draws up to 32 restart candidates ahead, gathers and reduces their
// rows together (16-byte coalesced loads, many rows in flight), and then
// takes the decisions one candidate at a time in draw order.  A candidate
// that became visited in between (an earlier duplicate in the batch, or a
// node reached by a climb) is skipped as the sequential search would skip
// it, at no cost to the budget.  A climb step likewise gathers every
// unvisited neighbour of the current node at once and then scans them in
// list order, stopping at the first improvement.  Rows gathered ahead but
// not reached by the sequential scan are not counted, marked or offered.
#pragma once

#include "common.cuh"
#include "kernels.h"

namespace knn {

constexpr int SEARCH_WARPS = 4;

__device__ __forceinline__ bool test_bit(const uint32_t *bits, uint32_t i) {
    return (bits[i >> 5] >> (i & 31)) & 1u;
}
__device__ __forceinline__ bool test_bit_ro(const uint32_t *bits, uint32_t i) {
    return (__ldg(bits + (i >> 5)) >> (i & 31)) & 1u;
}

template <int STORAGE, int DP, int T>
__global__ void __launch_bounds__(SEARCH_WARPS * 32)
ignns_search_kernel(const SearchArgs a) {
    using C = RowCfg<STORAGE, DP>;
    constexpr int NB = (C::P * C::RPP) < 32 ? (C::P * C::RPP) : 32;  // restart batch
    __shared__ uint32_t s_id[SEARCH_WARPS][32];
    __shared__ uint64_t s_j[SEARCH_WARPS][32];
    __shared__ uint32_t s_nb[SEARCH_WARPS][32];

    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    const RowSource src{a.rows, a.row_scale};
    const int nwarps = gridDim.x * SEARCH_WARPS;
    const float INF = __int_as_float(0x7f800000);

    for (int qi = blockIdx.x * SEARCH_WARPS + wib; qi < a.m; qi += nwarps) {
        float qv[C::QF];
        load_query<STORAGE, DP>(a.queries + (size_t)qi * a.q_stride, qv);
        uint32_t *vis = a.visited + (size_t)qi * a.vwords;
        const uint64_t rkey = restart_key(a.seed, a.stream_base + (uint64_t)qi);

        WarpTop<T> top;
        top.init(a.KT);
        long long evals = 0, nvis = 0, restarts = 0, discarded = 0, moves = 0, adj = 0;
        unsigned long long draws_used = 0;
        uint64_t j = 0;
        float d2min = INF;   // s_max = sim_of_d2(d2min); -inf while no node is known
        float thr = 0.0f;    // s_max / e
        bool done = a.budget <= 0 || a.n_live <= 0;

        while (!done) {
            // ---- draw the next restart candidates (free redraws skipped)
            int nc = 0;
            while (nc < NB && j < a.max_draws && nvis < a.n_live) {
                const uint64_t jj = j + (uint64_t)lane;
                const bool valid = jj < a.max_draws;
                const uint32_t r = valid ? restart_node(rkey, jj, a.n) : 0u;
                const bool good = valid && !test_bit_ro(a.removed, r) && !test_bit(vis, r);
                const unsigned bal = __ballot_sync(FULL, good);
                const int avail = __popc(bal);
                const int take = avail < NB - nc ? avail : NB - nc;
                const int rank = __popc(bal & lt_mask);
                if (good && rank < take) {
                    s_id[wib][nc + rank] = r;
                    s_j[wib][nc + rank] = jj;
                }
                if (take > 0 && take == NB - nc && take < avail) {
                    // batch full: resume after the last draw taken
                    const int last = __ffs(__ballot_sync(FULL, good && rank == take - 1)) - 1;
                    j += (uint64_t)last + 1u;
                } else {
                    j += 32u;
                }
                if (j > a.max_draws) j = a.max_draws;
                nc += take;
            }
            __syncwarp();
            if (nc == 0) break;  // nothing left to draw
            const uint32_t cid = lane < nc ? s_id[wib][lane] : 0u;
            const uint64_t cj = lane < nc ? s_j[wib][lane] : 0ull;
            const float cd2 = gather_d2<STORAGE, DP>(src, cid, nc, qv);

            // ---- decisions in draw order
            unsigned revisited = 0;  // candidates reached by a climb since the draw
            for (int c = 0; c < nc; ++c) {
                if (evals >= a.budget || nvis >= a.n_live) { done = true; break; }
                const uint32_t r = __shfl_sync(FULL, cid, c);
                const bool dup = __ballot_sync(FULL, lane < c && cid == r) != 0u;
                if (dup || ((revisited >> c) & 1u)) continue;  // free redraw
                const float d2 = __shfl_sync(FULL, cd2, c);
                ++evals; ++nvis; ++restarts;
                draws_used = __shfl_sync(FULL, cj, c) + 1ull;
                if (lane == 0) vis[r >> 5] |= 1u << (r & 31);
                top.offer(pack_key(d2, r));
                // expansion test: discard r if sim(q, r) < s_max / e
                if (a.discard && d2min < INF) {
                    if (sim_of_d2(d2) < thr) { ++discarded; continue; }
                }
                if (d2 < d2min) { d2min = d2; thr = sim_of_d2(d2min) / a.expansion; }

                // ---- eager hill climbing from r
                uint32_t cur = r;
                float d2cur = d2;
                while (true) {
                    const int32_t nb = lane < a.k ? __ldg(a.nbr + (size_t)cur * a.k + lane) : -1;
                    ++adj;
                    __syncwarp();
                    const bool unv = nb >= 0 && !test_bit_ro(a.removed, (uint32_t)nb) &&
                                     !test_bit(vis, (uint32_t)nb);
                    const unsigned um = __ballot_sync(FULL, unv);
                    if (um == 0u) break;  // every neighbour visited: local maximum
                    const int nu = __popc(um);
                    if (unv) s_nb[wib][__popc(um & lt_mask)] = (uint32_t)nb;
                    __syncwarp();
                    const uint32_t nid = lane < nu ? s_nb[wib][lane] : 0u;
                    const float nd2 = gather_d2<STORAGE, DP>(src, nid, nu, qv);
                    bool moved = false;
                    for (int i = 0; i < nu; ++i) {
                        if (evals >= a.budget) { done = true; break; }
                        const uint32_t id = __shfl_sync(FULL, nid, i);
                        const float dd = __shfl_sync(FULL, nd2, i);
                        ++evals; ++nvis;
                        if (lane == 0) vis[id >> 5] |= 1u << (id & 31);
                        top.offer(pack_key(dd, id));
                        if (dd < d2min) { d2min = dd; thr = sim_of_d2(d2min) / a.expansion; }
                        if (dd < d2cur) {  // first strict increase of similarity: move
                            cur = id;
                            d2cur = dd;
                            ++moves;
                            moved = true;
                            break;
                        }
                    }
                    if (done || !moved) break;
                }
                if (done) break;
                // the climb may have visited candidates drawn earlier
                __syncwarp();
                const bool rv = lane > c && lane < nc && test_bit(vis, cid);
                revisited |= __ballot_sync(FULL, rv);
            }
        }

        // ---- results and counters
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const int idx = t * 32 + lane;
            if (idx < a.KT) a.out_keys[(size_t)qi * a.KT + idx] = top.e[t];
        }
        if (lane == 0) {
            long long *ctr = a.counters + (size_t)qi * NCTR;
            ctr[CTR_SEARCH_EVALS] = evals;
            ctr[CTR_UPDATE_EVALS] = 0;
            ctr[CTR_RESTARTS] = restarts;
            ctr[CTR_DISCARDED] = discarded;
            ctr[CTR_MOVES] = moves;
            ctr[CTR_ADJ_READS] = adj;
            ctr[CTR_DRAWS] = (long long)draws_used;
            ctr[CTR_PAD] = 0;
            atomicAdd(a.totals + TOT_SEARCH_EVALS, (unsigned long long)evals);
            atomicAdd(a.totals + TOT_RESTARTS, (unsigned long long)restarts);
            atomicAdd(a.totals + TOT_MOVES, (unsigned long long)moves);
            atomicAdd(a.totals + TOT_ADJ_READS, (unsigned long long)adj);
            atomicAdd(a.totals + TOT_SEARCH_ROW_BYTES,
                      (unsigned long long)evals * (unsigned long long)(C::ROW_BYTES + (STORAGE == ST_FP8 ? 4 : 0)));
        }
        __syncwarp();
    }
}

#define KNN_SEARCH_CASE(ST, DPV)                                                          \
    case DPV:                                                                             \
        if (a.KT <= 32)                                                                   \
            ignns_search_kernel<ST, DPV, 1><<<grid, SEARCH_WARPS * 32, 0, s>>>(a);        \
        else                                                                              \
            ignns_search_kernel<ST, DPV, 4><<<grid, SEARCH_WARPS * 32, 0, s>>>(a);        \
        break;

#define KNN_DEFINE_SEARCH_LAUNCHER(NAME, ST)                                              \
    cudaError_t NAME(int dp, const SearchArgs &a, cudaStream_t s) {                       \
        if (a.m <= 0) return cudaSuccess;                                                 \
        const int grid = (a.m + SEARCH_WARPS - 1) / SEARCH_WARPS;                         \
        switch (dp) {                                                                     \
            KNN_SEARCH_CASE(ST, 16)                                                       \
            KNN_SEARCH_CASE(ST, 32)                                                       \
            KNN_SEARCH_CASE(ST, 64)                                                       \
            KNN_SEARCH_CASE(ST, 96)                                                       \
            KNN_SEARCH_CASE(ST, 128)                                                      \
            KNN_SEARCH_CASE(ST, 256)                                                      \
            default:                                                                      \
                return cudaErrorInvalidValue;                                             \
        }                                                                                 \
        return cudaGetLastError();                                                        \
    }

}  // namespace knn
