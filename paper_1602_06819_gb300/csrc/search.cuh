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
// The decisions are sequential, but neither the row gathers nor most of the
// decisions need to be taken one at a time:
//
// * Restarts.  The similarity of a drawn node does not depend on the search
//   state, so the warp draws batches of up to 32 unvisited candidates ahead
//   and gathers a batch's rows together (16-byte coalesced loads, all in
//   flight at once): while one batch is decided the next one loads and the
//   one after it is drawn.  A restart's row is first read in part; most are
//   settled by the partial sum, a lower bound (see the restart loop).
//   Between two accepted restarts the search only counts, marks and offers:
//   one ballot finds the first candidate the expansion test keeps, and every
//   candidate before it is committed at once (a discarded restart cannot
//   change s_max, and the final top list does not depend on the order of the
//   offers).  Duplicates inside a batch are found with one match instruction;
//   candidates a climb has visited since the draw are skipped as free redraws.
// * Climbs.  A step gathers the rows of all neighbours of the current node in
//   the same round trip as their visited bits; one ballot then finds the
//   first unvisited neighbour (in list order) that is strictly more similar,
//   and every unvisited neighbour up to it is committed.  The GNNS climb the
//   paper compares against (Sec. 2.2) commits every unvisited neighbour and
//   moves to the most similar one (a warp minimum) when it beats the
//   current node.
//
// Visited sets.  A query's bitset lives in shared memory when the bitsets of
// a block's warps fit two blocks on an SM (about 220,000 nodes); marks are
// then shared-memory atomics and tests cost a few cycles.  Larger graphs keep
// the bitset in global memory (L2 atomics, L2 reads); there a climb step
// loads its neighbours' visited bits in the same round trip as their rows
// (rows of visited neighbours are loaded too), so that a step waits for one
// memory latency instead of two.
//
// Every similarity computation is thus one the sequential search performs:
// rows gathered ahead but not reached are not counted, marked or offered, and
// the budget cuts a batch exactly where the sequential search would stop.
#pragma once

#include "common.cuh"
#include "kernels.h"

namespace knn {

constexpr int SEARCH_WARPS = 4;

__device__ __forceinline__ bool test_bit_ro(const uint32_t *bits, uint32_t i) {
    return (ld_nc_u32(bits + (i >> 5)) >> (i & 31)) & 1u;
}

// A search's visited set over the nodes base .. base + size - 1: a bitset in
// shared memory or in global memory.
template <bool SMEM>
struct Visited {
    uint32_t *bits;
    uint32_t base;
    __device__ __forceinline__ bool test(uint32_t id) const {
        const uint32_t i = id - base;
        if constexpr (SMEM) return (bits[i >> 5] >> (i & 31)) & 1u;
        // global bits are set with atomics at L2; read them from L2 too
        return (ld_cg_u32(bits + (i >> 5)) >> (i & 31)) & 1u;
    }
    __device__ __forceinline__ void mark(uint32_t id) const {
        const uint32_t i = id - base;
        atomicOr(bits + (i >> 5), 1u << (i & 31));
    }
};

// Shared memory a block may use for visited sets (two blocks per SM); the
// rule is mirrored by search_visited_on_chip().
constexpr size_t SEARCH_SMEM_VIS_MAX = 110 * 1024;
__host__ __device__ constexpr size_t search_smem_bytes(uint32_t n) {
    return (size_t)SEARCH_WARPS * ((n + 31) / 32) * sizeof(uint32_t);
}

// Lanes whose bit is set in `mask`, keeping only the `count` lowest.
__device__ __forceinline__ unsigned lowest_bits(unsigned mask, int count) {
    if (count >= 32) return mask;
    const int lane = threadIdx.x & 31;
    const int rank = __popc(mask & ((1u << lane) - 1u));
    return __ballot_sync(FULL, ((mask >> lane) & 1u) && rank < count);
}

// Bits 0 .. i (i < 32).
__device__ __forceinline__ unsigned upto(int i) { return i >= 31 ? FULL : ((2u << i) - 1u); }

// Offer the keys of the lanes in `lanes` to the warp's top list.  The final
// list does not depend on the order; lanes go in increasing order.
template <int T>
__device__ __forceinline__ void offer_lanes(WarpTop<T> &top, unsigned lanes, uint64_t key) {
    const int lane = threadIdx.x & 31;
    unsigned om = __ballot_sync(FULL, ((lanes >> lane) & 1u) && key < top.worst);
    while (om) {
        const int l = __ffs(om) - 1;
        top.offer(shfl_u64(key, l));
        om &= ~(1u << l);
        om &= __ballot_sync(FULL, key < top.worst);
    }
}

// Two blocks a SM with visited sets in shared memory (their size decides);
// with visited sets in global memory, three where the kernel fits in 168
// registers a thread without large spills (rows up to 96 dimensions, or 128
// in a screening copy): the searches of DRAM-resident graphs wait on memory
// round trips, and more of them in flight finish a batch sooner.
template <int STORAGE, int DP>
constexpr int search_min_blocks(bool smem_vis) {
    return smem_vis ? 8 / SEARCH_WARPS : (DP <= 96 || (STORAGE != ST_FP32 && DP <= 128)) ? 3 : 2;
}
template <int STORAGE, int DP, int T, bool SMEM_VIS>
__global__ void __launch_bounds__(SEARCH_WARPS * 32, search_min_blocks<STORAGE, DP>(SMEM_VIS))
ignns_search_kernel(const SearchArgs a) {
    using C = RowCfg<STORAGE, DP>;
    constexpr int NB = 32;  // restart candidates per batch (one a lane)
    extern __shared__ uint32_t s_visited[];  // SMEM_VIS: one bitset per warp
    __shared__ uint32_t s_id[SEARCH_WARPS][32];
    __shared__ uint64_t s_j[SEARCH_WARPS][32];

    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    const RowSource src{a.rows, a.row_scale};
    const int nwarps = gridDim.x * SEARCH_WARPS;
    const float INF = __int_as_float(0x7f800000);
    const bool multi = a.seg.item_seg != nullptr;
    // no removed node: skip the bitset reads
    const bool any_removed = a.n_live < (int64_t)a.n || a.parts > 1;
    // climb list prefetch: lane l holds entry pf_p of the list of neighbour
    // pf_j, for the first npf = floor(32 / k) neighbours
    const int npf = 32 / a.k;
    const int pf_j = lane / a.k < npf ? lane / a.k : 0, pf_p = lane % a.k;
    const int nsearch = multi ? *a.seg.count : a.m * a.parts;

    // search sw: query sw / parts over partition sw % parts, the nodes
    // lo .. lo + np - 1 (one partition: every node); with several graphs,
    // item sw over its graph's nodes
    // the next search of this warp: the static stride, or the counter
    const bool fetch = !SMEM_VIS && a.work != nullptr;
    auto next_search = [&](int cur) {
        if (!fetch) return cur + nwarps;
        int v = 0;
        if (lane == 0) v = (int)atomicAdd(a.work, 1u);
        return __shfl_sync(FULL, v, 0);
    };
    for (int si = fetch ? next_search(0) : blockIdx.x * SEARCH_WARPS + wib; si < nsearch; si = next_search(si)) {
        // several graphs: the step's tables may give the order the warps take
        // the items in (a search's result does not depend on when it runs)
        const int sw = (multi && a.seg.order) ? a.seg.order[si] : si;
        const int qi = multi ? sw : sw / a.parts, part = multi ? 0 : sw % a.parts;
        uint32_t lo = 0u, np = a.n;
        int64_t live = a.n_live, budget = a.budget;
        uint64_t max_draws = a.max_draws;
        if (multi || a.parts > 1) {
            if (multi) {
                const int sg = a.seg.item_seg[sw];
                lo = a.seg.lo[sg];
                np = a.seg.n[sg];
                live = np;
            } else {
                lo = (uint32_t)a.part_off[part];
                np = (uint32_t)(a.part_off[part + 1] - (int64_t)lo);
                live = a.part_live[part];
            }
            const double b = floor((double)np / a.speedup);  // max(1, floor(n / speedup))
            budget = b < 1.0 ? 1 : (int64_t)b;
            max_draws = 64ull * np;
        }
        // each evaluation visits a new node, so evals also counts visited nodes
        const int limit = (int)(budget < live ? budget : live);
        float qv[C::QF];
        load_query<STORAGE, DP>(a.queries + (size_t)qi * a.q_stride, qv);
        Visited<SMEM_VIS> vis;
        vis.base = lo;
        if constexpr (SMEM_VIS) {
            vis.bits = s_visited + (size_t)wib * ((a.vis_n + 31) / 32);
            for (uint32_t w = lane; w < (np + 31) / 32; w += 32) vis.bits[w] = 0u;
            __syncwarp();
        } else {
            vis.bits = a.visited + (size_t)sw * a.vwords;
        }
        const uint64_t stream = a.streams ? a.streams[qi] : a.stream_base + (uint64_t)qi;
        const uint64_t rkey = restart_key(a.seed, stream + (uint64_t)part * PART_STREAM_STEP);

        WarpTop<T> top;
        top.init(a.KT);
        int evals = 0, restarts = 0, discarded = 0, moves = 0, adj = 0;  // budgets are < 2^31
        unsigned long long jlast = 0;  // this lane's latest committed draw index + 1
        uint64_t j = 0;
        float d2min = INF;  // s_max = sim_of_d2(d2min); none while d2min is +inf
        float thr = 0.0f;   // s_max / e
        // Squared distances below lo2 surely pass the expansion test and
        // those above hi2 surely fail it; only the band between evaluates
        // sim(q, r) < s_max / e itself.  The FP32 similarity errs by a few
        // units of 2^-24 and the band is 2^-12 wide on each side of the
        // boundary ((1 / thr - 1)^2, at least 1 when thr <= 1/2); above 1/2,
        // or past 2^100, every candidate takes the exact test.
        float lo2 = -1.0f, hi2 = INF;
        auto set_best = [&](float d2) {
            d2min = d2;
            thr = sim_of_d2(d2) / a.expansion;
            const float sb = 1.0f / thr - 1.0f;
            if (thr <= 0.5f && sb * sb < 0x1p100f) {
                lo2 = sb * sb * (1.0f - 0x1p-12f);
                hi2 = sb * sb * (1.0f + 0x1p-12f);
            } else {
                lo2 = -1.0f;
                hi2 = INF;
            }
        };
        bool done = limit <= 0;

        // Draw up to `want` candidates after draw j, skipping nodes visited or
        // removed (free redraws); lane c < count receives candidate c, and
        // `same` the lanes holding the same node.  A round looks at 64 draws,
        // two per lane (j + lane and j + 32 + lane).
        auto draw = [&](int want, uint32_t &id, uint64_t &dj, unsigned &same) -> int {
            int nc = 0;
            __syncwarp();  // marks made so far are visible to the bit reads
            while (nc < want && j < max_draws) {
                const uint64_t j0 = j + (uint64_t)lane, j1 = j0 + 32u;
                const bool v0 = j0 < max_draws, v1 = j1 < max_draws;
                const uint32_t r0 = v0 ? lo + restart_node(rkey, j0, np) : lo;
                const uint32_t r1 = v1 ? lo + restart_node(rkey, j1, np) : lo;
                const bool g0 = v0 && !(any_removed && test_bit_ro(a.removed, r0)) && !vis.test(r0);
                const bool g1 = v1 && !(any_removed && test_bit_ro(a.removed, r1)) && !vis.test(r1);
                const unsigned b0 = __ballot_sync(FULL, g0), b1 = __ballot_sync(FULL, g1);
                const int a0 = __popc(b0), avail = a0 + __popc(b1);
                const int take = avail < want - nc ? avail : want - nc;
                const int k0 = __popc(b0 & lt_mask), k1 = a0 + __popc(b1 & lt_mask);
                if (g0 && k0 < take) {
                    s_id[wib][nc + k0] = r0;
                    s_j[wib][nc + k0] = j0;
                }
                if (g1 && k1 < take) {
                    s_id[wib][nc + k1] = r1;
                    s_j[wib][nc + k1] = j1;
                }
                if (take > 0 && take < avail) {
                    // batch full: resume after the last draw taken
                    const unsigned lb = take <= a0 ? __ballot_sync(FULL, g0 && k0 == take - 1)
                                                   : __ballot_sync(FULL, g1 && k1 == take - 1);
                    j += (uint64_t)(__ffs(lb) - 1 + (take <= a0 ? 0 : 32)) + 1u;
                } else {
                    j += 64u;
                }
                if (j > max_draws) j = max_draws;
                nc += take;
            }
            __syncwarp();
            id = lane < nc ? s_id[wib][lane] : 0xffffffffu;
            dj = lane < nc ? s_j[wib][lane] : 0ull;
            same = __match_any_sync(FULL, id);  // used a batch or two later
            return nc;
        };
        auto cap = [&](int room) -> int { return room < NB ? room : NB; };

        // Batch A is decided while the rows of the next batch B load, and the
        // ids of the batch after B (C) are drawn meanwhile: B's loads start
        // as soon as A is settled.
        //
        // A restart's squared distance matters for three things only: the
        // expansion test, the offer to the result list and, when it is kept,
        // the climb.  B first loads the head of each row (its first G * 16
        // bytes); the partial sum over it is a lower bound of the full sum
        // (in FP32 as well: every step adds a nonnegative value, rounding is
        // monotone).  A row whose partial sum is at least hi2 fails the
        // expansion test whatever the rest holds (hi2 only falls as s_max
        // rises) and, above the result list's worst distance (which only
        // falls too), cannot enter it: it is discarded as the full distance
        // would discard it and its distance is recorded as +inf.  The other
        // rows get their full distance, summed exactly as a full gather sums
        // it, in a second round trip.  Every restart still counts as one
        // similarity computation.
        constexpr bool SETTLE = C::CPL >= 2;  // the head is shorter than the row
        RowGatherHead<STORAGE, DP> H;
        auto full_d2 = [&](uint32_t id, int n) -> float {  // lanes < n: rows id
            return n <= 12 ? gather_d2<STORAGE, DP, 12>(src, lane < n ? id : 0u, n, qv)
                           : gather_d2<STORAGE, DP>(src, lane < n ? id : 0u, n, qv);
        };
        auto settle = [&](float part, uint32_t id, int n) -> float {
            if (!SETTLE) return part;  // the head was the whole row
            const bool out = a.discard && part >= hi2 && part > key_d2(top.worst);
            const unsigned need = __ballot_sync(FULL, lane < n && !out);
            float d2 = out ? INF : part;
            if (need) {
                // the rows that need it, compacted to the first lanes
                const int cnt = __popc(need);
                const uint32_t nid = __shfl_sync(FULL, id, lane < cnt ? (int)__fns(need, 0, lane + 1) : 0);
                const float f = full_d2(nid, cnt);
                const float mine = __shfl_sync(FULL, f, __popc(need & lt_mask) & 31);
                if ((need >> lane) & 1u) d2 = mine;
            }
            return d2;
        };
        uint32_t aid = 0xffffffffu, bid = 0xffffffffu;
        uint64_t aj = 0, bj = 0;
        unsigned asame = 0u, bsame = 0u;
        int an = done ? 0 : draw(cap(limit), aid, aj, asame);
        float ad2 = an > 0 ? full_d2(aid, an) : INF;
        int bn = an > 0 && limit - an > 0 ? draw(cap(limit - an), bid, bj, bsame) : 0;
        while (an > 0) {
            // ---- start B's loads, then draw C (filtered by the marks so far).
            // issue and reduce are paired unconditionally, so the row buffer
            // is visibly dead after the reduce
            H.issue(src, lane < bn ? bid : 0u, bn);
            uint32_t cid = 0xffffffffu;
            uint64_t cj = 0;
            unsigned csame = 0u;
            const int room = limit - evals - an - bn;
            const int cn = room > 0 ? draw(cap(room), cid, cj, csame) : 0;

            // ---- decide A, in draw order.  A was filtered before the two
            // batches before it were decided: re-test its candidates; an
            // earlier copy of the same node in A makes a candidate a redraw.
            const uint64_t akey = pack_key(ad2, aid);
            unsigned skip = __ballot_sync(FULL, lane >= an || (asame & lt_mask) != 0u || vis.test(aid));
            // Commit the candidates from `start` up to the first one the
            // expansion test keeps (all are kept while no s_max exists);
            // returns that candidate, or 32 when every candidate left was
            // discarded or skipped.
            auto segment = [&](int start) -> int {
                unsigned ev = ~skip & (FULL << start);
                if (ev == 0u) return 32;
                ev = lowest_bits(ev, limit - evals);
                const bool in = (ev >> lane) & 1u;
                bool keep = in && (!a.discard || !(d2min < INF) || ad2 <= lo2);
                const bool band = in && !keep && !(ad2 >= hi2);
                if (__any_sync(FULL, band))  // rare: the exact test
                    keep |= band && !(sim_of_d2(ad2) < thr);
                const unsigned kept = __ballot_sync(FULL, keep);
                const int ai = kept ? __ffs(kept) - 1 : 32;
                const unsigned evm = ai < 32 ? (ev & upto(ai)) : ev;
                const int ne = __popc(evm);
                evals += ne;
                restarts += ne;
                discarded += ne - (ai < 32 ? 1 : 0);
                if ((evm >> lane) & 1u) {
                    vis.mark(aid);
                    jlast = aj + 1ull;  // draw indexes grow: the last commit is the largest
                }
                offer_lanes(top, evm, akey);
                return ai;
            };
            // the list of a kept restart (lanes < k), loaded as soon as it is kept
            auto list_of = [&](int i) -> int32_t {
                const uint32_t r = __shfl_sync(FULL, aid, i);
                return lane < a.k ? (int32_t)ld_nc_u32(a.nbr + (size_t)r * a.k + lane) : -1;
            };
            int ai = segment(0);
            int32_t nbk = ai < 32 ? list_of(ai) : -1;
            // B's distances, before any climb (one row buffer is live at a time)
            const float bd2 = settle(H.reduce(bn, qv), bid, bn);

            while (ai < 32) {
                const float d2a = __shfl_sync(FULL, ad2, ai);
                if (d2a < d2min) set_best(d2a);
                if (evals >= limit) { done = true; break; }

                // ---- eager hill climbing from the kept restart
                uint32_t cur = __shfl_sync(FULL, aid, ai);
                float d2cur = d2a;
                int32_t nb = nbk;
                while (true) {
                    ++adj;
                    // a partition follows only its own nodes (Algorithm 3)
                    const bool valid = nb >= 0 && (uint32_t)nb - lo < np &&
                                       !(any_removed && test_bit_ro(a.removed, (uint32_t)nb));
                    __syncwarp();
                    unsigned um = 0u;
                    uint32_t bw = 0u;
                    if constexpr (!SMEM_VIS) {
                        // global bits: they load in the round trip of the rows
                        // (the rows of visited neighbours load too)
                        if (valid) {
                            bw = ld_cg_u32(vis.bits + (((uint32_t)nb - lo) >> 5));
                            // and the neighbours' lists start towards L1 for a move
                            const int32_t *l = a.nbr + (size_t)nb * a.k;
                            prefetch_l1(l);
                            prefetch_l1(l + a.k - 1);
                        }
                    } else {
                        const bool seen = valid && vis.test((uint32_t)nb);
                        um = __ballot_sync(FULL, valid && !seen);
                        if (um == 0u) break;  // every neighbour visited: local maximum
                        um = lowest_bits(um, limit - evals);
                    }
                    // the lists of the first 32 / k neighbours load in the same
                    // round trip as their rows (lane l: entry pf_p of neighbour
                    // pf_j), so a move to one of them needs no list load
                    const int32_t nbj = __shfl_sync(FULL, nb, pf_j);
                    // (an entry outside the node range is an empty slot: no list read)
                    const int32_t pfl = (pf_j < npf && (uint32_t)nbj - lo < np)
                                            ? (int32_t)ld_nc_u32(a.nbr + (size_t)nbj * a.k + pf_p) : -1;
                    // only the rows the step can evaluate load; as many passes
                    // as the k rows need (one pass holds 32 / G rows)
                    const bool load = !SMEM_VIS ? valid : ((um >> lane) & 1u) != 0u;
                    const uint32_t nrow = load ? (uint32_t)nb : GATHER_SKIP;
                    const float nd2 = a.k <= 12   ? gather_d2<STORAGE, DP, 12>(src, nrow, a.k, qv)
                                      : a.k <= 24 ? gather_d2<STORAGE, DP, 24>(src, nrow, a.k, qv)
                                                  : gather_d2<STORAGE, DP>(src, nrow, a.k, qv);
                    if constexpr (!SMEM_VIS) {
                        const bool seen = valid && ((bw >> (((uint32_t)nb - lo) & 31u)) & 1u);
                        um = __ballot_sync(FULL, valid && !seen);
                        if (um == 0u) break;  // every neighbour visited: local maximum
                        um = lowest_bits(um, limit - evals);
                    }
                    int mi;
                    unsigned evc;
                    if (a.climb == KNN_CLIMB_BEST) {
                        // GNNS: every unvisited neighbour is evaluated; the
                        // most similar (ties to the earlier position) becomes
                        // cur if it is strictly more similar than cur
                        evc = um;
                        uint64_t pk = ((evc >> lane) & 1u)
                                          ? (((uint64_t)__float_as_uint(nd2) << 32) | (uint32_t)lane)
                                          : ~0ull;
#pragma unroll
                        for (int off = 16; off >= 1; off >>= 1) {
                            const uint64_t o = shfl_u64_xor(pk, off);
                            pk = o < pk ? o : pk;
                        }
                        mi = __uint_as_float((uint32_t)(pk >> 32)) < d2cur ? (int)(uint32_t)pk : 32;
                    } else {
                        const unsigned better = um & __ballot_sync(FULL, nd2 < d2cur);
                        mi = better ? __ffs(better) - 1 : 32;
                        evc = mi < 32 ? (um & upto(mi)) : um;
                    }
                    evals += __popc(evc);
                    const bool mine = (evc >> lane) & 1u;
                    if (mine) vis.mark((uint32_t)nb);
                    offer_lanes(top, evc, pack_key(nd2, (uint32_t)nb));
                    if (__any_sync(FULL, mine && nd2 < d2min)) {  // a new best: s_max rises
                        float mn = mine ? nd2 : INF;
#pragma unroll
                        for (int off = 16; off >= 1; off >>= 1) mn = fminf(mn, __shfl_xor_sync(FULL, mn, off));
                        set_best(mn);
                    }
                    if (mi < 32) ++moves;
                    if (evals >= limit) { done = true; break; }
                    if (mi == 32) break;  // no unvisited neighbour is more similar
                    cur = (uint32_t)__shfl_sync(FULL, nb, mi);  // first strict increase: move
                    d2cur = __shfl_sync(FULL, nd2, mi);
                    if (mi < npf) {  // its list came with the rows
                        const int32_t v = __shfl_sync(FULL, pfl, (mi * a.k + lane) & 31);
                        nb = lane < a.k ? v : -1;
                    } else {
                        nb = lane < a.k ? (int32_t)ld_nc_u32(a.nbr + (size_t)cur * a.k + lane) : -1;
                    }
                }
                if (done) break;
                // the climb may have visited candidates drawn earlier
                __syncwarp();
                skip |= __ballot_sync(FULL, lane > ai && lane < an && vis.test(aid));
                ai = ai + 1 < 32 ? segment(ai + 1) : 32;
                if (ai < 32) nbk = list_of(ai);
            }
            if (evals >= limit) done = true;
            if (done) break;
            if (bn == 0) {
                // B is empty (the budget looked spent when it was drawn): C,
                // else a new draw, becomes A and loads now
                if (cn > 0) {
                    aid = cid;
                    aj = cj;
                    asame = csame;
                    an = cn;
                } else {
                    an = draw(cap(limit - evals), aid, aj, asame);
                    if (an == 0) break;
                }
                ad2 = full_d2(aid, an);
                bn = limit - evals - an > 0 ? draw(cap(limit - evals - an), bid, bj, bsame) : 0;
                continue;
            }
            aid = bid;
            aj = bj;
            asame = bsame;
            an = bn;
            ad2 = bd2;
            bid = cid;
            bj = cj;
            bsame = csame;
            bn = cn;
        }

        // ---- results and counters
        unsigned long long draws_used = jlast;
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) {
            const unsigned long long o = shfl_u64_xor(draws_used, off);
            draws_used = o > draws_used ? o : draws_used;
        }
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const int idx = t * 32 + lane;
            if (idx < a.KT) a.out_keys[(size_t)sw * a.KT + idx] = top.e[t];
        }
        if (lane == 0) {
            long long *ctr = a.counters + (size_t)sw * NCTR;
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

template <int ST, int DPV, int T>
static cudaError_t launch_search_t(const SearchArgs &a, cudaStream_t s) {
    if (a.m <= 0) {
        // nothing to search: resolve both kernels, which loads their code now
        // (with lazy module loading) rather than inside the first search
        cudaFuncAttributes fa;
        cudaError_t e = cudaFuncGetAttributes(&fa, ignns_search_kernel<ST, DPV, T, true>);
        return e == cudaSuccess ? cudaFuncGetAttributes(&fa, ignns_search_kernel<ST, DPV, T, false>) : e;
    }
    const int grid = (a.m * a.parts + SEARCH_WARPS - 1) / SEARCH_WARPS;
    const size_t smem = search_smem_bytes(a.vis_n);
    if (smem <= SEARCH_SMEM_VIS_MAX) {
        cudaError_t e = cudaFuncSetAttribute(ignns_search_kernel<ST, DPV, T, true>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        ignns_search_kernel<ST, DPV, T, true><<<grid, SEARCH_WARPS * 32, smem, s>>>(a);
    } else if (a.work) {
        // persistent: as many blocks as fit at once, the searches taken from
        // the counter
        int dev = 0, sms = 0, per_sm = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ignns_search_kernel<ST, DPV, T, false>,
                                                              SEARCH_WARPS * 32, 0);
        if (e == cudaSuccess) e = cudaMemsetAsync(a.work, 0, sizeof(unsigned), s);
        if (e != cudaSuccess) return e;
        const int cap = (per_sm > 0 ? per_sm : 1) * sms;
        ignns_search_kernel<ST, DPV, T, false><<<grid < cap ? grid : cap, SEARCH_WARPS * 32, 0, s>>>(a);
    } else {
        ignns_search_kernel<ST, DPV, T, false><<<grid, SEARCH_WARPS * 32, 0, s>>>(a);
    }
    return cudaGetLastError();
}

#define KNN_SEARCH_CASE(ST, DPV)                                                          \
    case DPV:                                                                             \
        return a.KT <= 32 ? launch_search_t<ST, DPV, 1>(a, s) : launch_search_t<ST, DPV, 4>(a, s);

#define KNN_DEFINE_SEARCH_LAUNCHER(NAME, ST)                                              \
    cudaError_t NAME(int dp, const SearchArgs &a, cudaStream_t s) {                       \
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
    }

}  // namespace knn
