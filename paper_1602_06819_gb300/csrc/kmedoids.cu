// kmedoids.cu -- balanced k-medoids (Sec. 6, Algorithm 4) on the device: the
// node ordering that makes clusters contiguous, and the partitions of the
// partitioned search (Algorithm 3).
//
// Assign step: the points are split in c chunks of consecutive ids (the
// paper's compute nodes); within a chunk the points are assigned one after
// the other to the medoid m maximising sim(m, x) * w(t, m),
// w(t, m) = 1 - |C_t(m)| / capacity, capacity = n * imbalance / (p * c),
// |C_t(m)| counting the chunk's points given to m so far; ties go to the
// lower cluster position.  The distances do not depend on that sequence, so
// they are computed first for every (point, medoid) pair by a tiled kernel
// over the whole GPU; one warp per chunk then takes the sequential
// decisions, reading each point's row of distances.
//
// Update step: every cluster takes as medoid its member with the smallest
// sum of Euclidean distances to the other members (ties to the lower id); an
// empty cluster keeps its medoid.  Members are grouped by a stable counting
// sort on the labels, which also yields the node ordering.
//
// FP32 throughout: squared distances by fused multiply-adds in dimension
// order, sim = 1/(1 + sqrt(d2)) and the weighted score correctly rounded, the
// distance sums in tile order.
#include "common.cuh"
#include "kernels.h"

namespace knn {

constexpr int KD_TILE = 64;   // points and medoids per distance tile
constexpr int KD_LD = 68;     // padded leading dimension of the k-major tiles
constexpr int KD_THREADS = 256;
constexpr int KS_BLOCK = 1024;  // points per block of the counting sort

// D[i][m] = ||x_i - x_{medoids[m]}||^2 for i < n, m < p.  A block owns 64
// points x 64 medoids; 4 x 4 pairs per thread from k-major shared tiles.
template <int DP>
__global__ void __launch_bounds__(KD_THREADS) kmed_dist_kernel(const float *X, int64_t n, const int64_t *medoids,
                                                               int p, float *D) {
    extern __shared__ float kd_smem[];
    float(*As)[KD_LD] = reinterpret_cast<float(*)[KD_LD]>(kd_smem);            // [DP][KD_LD] points
    float(*Bs)[KD_LD] = reinterpret_cast<float(*)[KD_LD]>(kd_smem + DP * KD_LD);  // [DP][KD_LD] medoids
    const int tid = threadIdx.x;
    const int64_t i0 = (int64_t)blockIdx.x * KD_TILE;
    const int m0 = blockIdx.y * KD_TILE;
    for (int idx = tid; idx < KD_TILE * (DP / 4); idx += KD_THREADS) {
        const int r = idx % KD_TILE, ch = idx / KD_TILE;
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
        if (i0 + r < n) a = *reinterpret_cast<const float4 *>(X + (i0 + r) * DP + ch * 4);
        if (m0 + r < p) b = *reinterpret_cast<const float4 *>(X + medoids[m0 + r] * DP + ch * 4);
        As[ch * 4 + 0][r] = a.x;
        As[ch * 4 + 1][r] = a.y;
        As[ch * 4 + 2][r] = a.z;
        As[ch * 4 + 3][r] = a.w;
        Bs[ch * 4 + 0][r] = b.x;
        Bs[ch * 4 + 1][r] = b.y;
        Bs[ch * 4 + 2][r] = b.z;
        Bs[ch * 4 + 3][r] = b.w;
    }
    __syncthreads();
    const int tr = tid >> 4, tc = tid & 15;  // points tr*4.., medoids tc*4..
    float acc[4][4] = {};
#pragma unroll 4
    for (int kk = 0; kk < DP; ++kk) {
        const float4 av = *reinterpret_cast<const float4 *>(&As[kk][tr * 4]);
        const float4 bv = *reinterpret_cast<const float4 *>(&Bs[kk][tc * 4]);
        const float ar[4] = {av.x, av.y, av.z, av.w};
        const float br[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float d = ar[i] - br[j];
                acc[i][j] = fmaf(d, d, acc[i][j]);
            }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t row = i0 + tr * 4 + i;
        if (row >= n) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int m = m0 + tc * 4 + j;
            if (m < p) D[row * p + m] = acc[i][j];
        }
    }
}

// Sortable bits of a float (unsigned order = float order, -0 < +0).
__device__ __forceinline__ uint32_t float_order(float f) {
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// One warp per chunk: the sequential weighted assignment.  counts lives in
// shared memory (KMED_MAX_P per warp); a point's row of distances is loaded
// while the previous point is decided.
constexpr int KA_WARPS = 4;
__global__ void __launch_bounds__(KA_WARPS * 32) kmed_assign_kernel(const float *D, int64_t n, int p, int chunks,
                                                                    float capacity, int32_t *labels) {
    __shared__ int s_count[KA_WARPS][KMED_MAX_P];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int c = blockIdx.x * KA_WARPS + wib;
    if (c >= chunks) return;  // warp-uniform
    int *count = s_count[wib];
    for (int m = lane; m < p; m += 32) count[m] = 0;
    __syncwarp();
    const int64_t lo = (int64_t)((__int128)c * n / chunks), hi = (int64_t)((__int128)(c + 1) * n / chunks);
    constexpr int PER = KMED_MAX_P / 32;
    float cur[PER], nxt[PER];
    auto load = [&](int64_t i, float(&v)[PER]) {
#pragma unroll
        for (int t = 0; t < PER; ++t) {
            const int m = t * 32 + lane;
            v[t] = (i < hi && m < p) ? __ldcs(D + i * p + m) : 0.f;
        }
    };
    load(lo, cur);
    for (int64_t i = lo; i < hi; ++i) {
        load(i + 1, nxt);
        uint64_t best = 0;
#pragma unroll
        for (int t = 0; t < PER; ++t) {
            const int m = t * 32 + lane;
            if (m < p) {
                const float sim = 1.0f / (1.0f + sqrtf(cur[t]));
                const float w = 1.0f - (float)count[m] / capacity;
                const uint64_t key = ((uint64_t)float_order(sim * w) << 32) | (uint32_t)(0xffffffffu - (uint32_t)m);
                best = key > best ? key : best;
            }
        }
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) {
            const uint64_t o = shfl_u64_xor(best, off);
            best = o > best ? o : best;
        }
        const int m = (int)(0xffffffffu - (uint32_t)best);
        if (lane == 0) {
            count[m] += 1;
            labels[i] = m;
        }
        __syncwarp();
#pragma unroll
        for (int t = 0; t < PER; ++t) cur[t] = nxt[t];
    }
}

// ---- stable counting sort of the points by label ---------------------------
// hist[b][m]: points of block b (KS_BLOCK consecutive ids) with label m.
__global__ void kmed_hist_kernel(const int32_t *labels, int64_t n, int p, int32_t *hist) {
    __shared__ int32_t h[KMED_MAX_P];
    for (int m = threadIdx.x; m < p; m += blockDim.x) h[m] = 0;
    __syncthreads();
    const int64_t i0 = (int64_t)blockIdx.x * KS_BLOCK;
    for (int64_t i = i0 + threadIdx.x; i < n && i < i0 + KS_BLOCK; i += blockDim.x) atomicAdd(&h[labels[i]], 1);
    __syncthreads();
    for (int m = threadIdx.x; m < p; m += blockDim.x) hist[(int64_t)blockIdx.x * p + m] = h[m];
}

// One block: offsets[m] = first position of cluster m (offsets[p] = n), and
// pos[b][m] = first position of block b's points of cluster m.
__global__ void __launch_bounds__(KMED_MAX_P) kmed_offsets_kernel(const int32_t *hist, int nblk, int p, int64_t n,
                                                                  int64_t *offsets, int64_t *pos) {
    __shared__ int64_t s_tot[KMED_MAX_P];
    const int m = threadIdx.x;
    int64_t tot = 0;
    if (m < p)
        for (int b = 0; b < nblk; ++b) tot += hist[(int64_t)b * p + m];
    s_tot[m] = m < p ? tot : 0;
    __syncthreads();
    // exclusive scan over clusters (Hillis-Steele over the block)
    for (int off = 1; off < KMED_MAX_P; off <<= 1) {
        const int64_t v = m >= off ? s_tot[m - off] : 0;
        __syncthreads();
        s_tot[m] += v;
        __syncthreads();
    }
    if (m < p) {
        int64_t run = s_tot[m] - tot;  // exclusive
        offsets[m] = run;
        for (int b = 0; b < nblk; ++b) {
            pos[(int64_t)b * p + m] = run;
            run += hist[(int64_t)b * p + m];
        }
    }
    if (m == 0) offsets[p] = n;
}

// order[position] = point id, stable by id within a cluster: the block's
// points are placed 32 at a time, in id order, by one warp.
__global__ void kmed_scatter_kernel(const int32_t *labels, int64_t n, int p, const int64_t *pos, int64_t *order) {
    __shared__ int64_t cursor[KMED_MAX_P];
    for (int m = threadIdx.x; m < p; m += blockDim.x) cursor[m] = pos[(int64_t)blockIdx.x * p + m];
    __syncthreads();
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    const int64_t i0 = (int64_t)blockIdx.x * KS_BLOCK;
    for (int64_t g = i0; g < n && g < i0 + KS_BLOCK; g += 32) {
        const int64_t i = g + lane;
        const bool valid = i < n && i < i0 + KS_BLOCK;
        const int l = valid ? labels[i] : -1 - lane;  // invalid lanes match nobody
        const unsigned peers = __match_any_sync(FULL, l);
        if (valid) {
            const int rank = __popc(peers & ((1u << lane) - 1u));
            order[cursor[l] + rank] = i;
        }
        __syncwarp();
        if (valid && lane == 31 - __clz(peers)) cursor[l] += __popc(peers);
        __syncwarp();
    }
}

// ---- update: the medoid of each cluster --------------------------------------
// One block per cluster: row sums of distances over 64 x 64 member tiles,
// then the member with the smallest sum (ties to the lower id).
template <int DP>
__global__ void __launch_bounds__(KD_THREADS) kmed_update_kernel(const float *X, const int64_t *order,
                                                                 const int64_t *offsets, int64_t *medoids) {
    extern __shared__ float kd_smem[];
    float(*As)[KD_LD] = reinterpret_cast<float(*)[KD_LD]>(kd_smem);            // [DP][KD_LD] row members
    float(*Bs)[KD_LD] = reinterpret_cast<float(*)[KD_LD]>(kd_smem + DP * KD_LD);  // [DP][KD_LD] column members
    __shared__ uint64_t s_best[KD_THREADS / 32];
    const int m = blockIdx.x;
    const int64_t b0 = offsets[m], cnt = offsets[m + 1] - offsets[m];
    if (cnt == 0) return;  // an empty cluster keeps its medoid
    const int tid = threadIdx.x, lane = tid & 31;
    const int tr = tid >> 4, tc = tid & 15;
    uint64_t best = ~0ull;  // (float_order(sum) << 32 | position) of the smallest sum
    for (int64_t r0 = 0; r0 < cnt; r0 += KD_TILE) {
        __syncthreads();
        for (int idx = tid; idx < KD_TILE * (DP / 4); idx += KD_THREADS) {
            const int r = idx % KD_TILE, ch = idx / KD_TILE;
            float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
            if (r0 + r < cnt) a = *reinterpret_cast<const float4 *>(X + order[b0 + r0 + r] * DP + ch * 4);
            As[ch * 4 + 0][r] = a.x;
            As[ch * 4 + 1][r] = a.y;
            As[ch * 4 + 2][r] = a.z;
            As[ch * 4 + 3][r] = a.w;
        }
        float rs[4] = {0.f, 0.f, 0.f, 0.f};
        for (int64_t c0 = 0; c0 < cnt; c0 += KD_TILE) {
            __syncthreads();
            for (int idx = tid; idx < KD_TILE * (DP / 4); idx += KD_THREADS) {
                const int r = idx % KD_TILE, ch = idx / KD_TILE;
                float4 b = make_float4(0.f, 0.f, 0.f, 0.f);
                if (c0 + r < cnt) b = *reinterpret_cast<const float4 *>(X + order[b0 + c0 + r] * DP + ch * 4);
                Bs[ch * 4 + 0][r] = b.x;
                Bs[ch * 4 + 1][r] = b.y;
                Bs[ch * 4 + 2][r] = b.z;
                Bs[ch * 4 + 3][r] = b.w;
            }
            __syncthreads();
            float acc[4][4] = {};
#pragma unroll 4
            for (int kk = 0; kk < DP; ++kk) {
                const float4 av = *reinterpret_cast<const float4 *>(&As[kk][tr * 4]);
                const float4 bv = *reinterpret_cast<const float4 *>(&Bs[kk][tc * 4]);
                const float ar[4] = {av.x, av.y, av.z, av.w};
                const float br[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const float d = ar[i] - br[j];
                        acc[i][j] = fmaf(d, d, acc[i][j]);
                    }
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (c0 + tc * 4 + j < cnt) rs[i] += sqrtf(acc[i][j]);
        }
        // the 16 threads of a row group hold partial sums of the same rows
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int off = 8; off >= 1; off >>= 1) rs[i] += __shfl_xor_sync(FULL, rs[i], off);
        if (tc == 0) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int64_t r = r0 + tr * 4 + i;
                if (r < cnt) {
                    // members are in id order, so the position breaks ties by id
                    const uint64_t key = ((uint64_t)float_order(rs[i]) << 32) | (uint32_t)r;
                    best = key < best ? key : best;
                }
            }
        }
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        const uint64_t o = shfl_u64_xor(best, off);
        best = o < best ? o : best;
    }
    if (lane == 0) s_best[tid >> 5] = best;
    __syncthreads();
    if (tid == 0) {
        uint64_t b = s_best[0];
        for (int w = 1; w < KD_THREADS / 32; ++w) b = s_best[w] < b ? s_best[w] : b;
        medoids[m] = order[b0 + (uint32_t)b];
    }
}

// ---- launchers -----------------------------------------------------------------
template <int DP>
static cudaError_t kmed_dist(const float *X, int64_t n, const int64_t *medoids, int p, float *D, cudaStream_t s) {
    constexpr size_t smem = 2 * (size_t)DP * KD_LD * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(kmed_dist_kernel<DP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((n + KD_TILE - 1) / KD_TILE), (unsigned)((p + KD_TILE - 1) / KD_TILE));
    kmed_dist_kernel<DP><<<grid, KD_THREADS, smem, s>>>(X, n, medoids, p, D);
    return cudaGetLastError();
}

template <int DP>
static cudaError_t kmed_update(const float *X, const int64_t *order, const int64_t *offsets, int p,
                               int64_t *medoids, cudaStream_t s) {
    constexpr size_t smem = 2 * (size_t)DP * KD_LD * sizeof(float);
    cudaError_t e =
        cudaFuncSetAttribute(kmed_update_kernel<DP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kmed_update_kernel<DP><<<p, KD_THREADS, smem, s>>>(X, order, offsets, medoids);
    return cudaGetLastError();
}

#define KMED_DP_SWITCH(dp, CALL)             \
    switch (dp) {                            \
        case 16: return CALL(16);            \
        case 32: return CALL(32);            \
        case 64: return CALL(64);            \
        case 96: return CALL(96);            \
        case 128: return CALL(128);          \
        case 256: return CALL(256);          \
        default: return cudaErrorInvalidValue; \
    }

cudaError_t launch_kmed_dist(int dp, const float *X, int64_t n, const int64_t *medoids, int p, float *D,
                             cudaStream_t s) {
#define KMED_DIST_CALL(V) kmed_dist<V>(X, n, medoids, p, D, s)
    KMED_DP_SWITCH(dp, KMED_DIST_CALL)
#undef KMED_DIST_CALL
}

cudaError_t launch_kmed_assign(const float *D, int64_t n, int p, int chunks, double capacity, int32_t *labels,
                               cudaStream_t s) {
    kmed_assign_kernel<<<(chunks + KA_WARPS - 1) / KA_WARPS, KA_WARPS * 32, 0, s>>>(D, n, p, chunks,
                                                                                    (float)capacity, labels);
    return cudaGetLastError();
}

size_t kmed_sort_scratch_bytes(int64_t n, int p) {
    const int64_t nblk = (n + KS_BLOCK - 1) / KS_BLOCK;
    return (size_t)nblk * p * (4 + 8) + 16;
}

cudaError_t launch_kmed_sort(const int32_t *labels, int64_t n, int p, void *scratch, int64_t *order,
                             int64_t *offsets, cudaStream_t s) {
    const int64_t nblk = (n + KS_BLOCK - 1) / KS_BLOCK;
    int32_t *hist = static_cast<int32_t *>(scratch);
    int64_t *pos = reinterpret_cast<int64_t *>(hist + ((nblk * p + 1) & ~(int64_t)1));
    kmed_hist_kernel<<<(unsigned)nblk, 256, 0, s>>>(labels, n, p, hist);
    kmed_offsets_kernel<<<1, KMED_MAX_P, 0, s>>>(hist, (int)nblk, p, n, offsets, pos);
    kmed_scatter_kernel<<<(unsigned)nblk, 256, 0, s>>>(labels, n, p, pos, order);
    return cudaGetLastError();
}

cudaError_t launch_kmed_update(int dp, const float *X, const int64_t *order, const int64_t *offsets, int p,
                               int64_t *medoids, cudaStream_t s) {
#define KMED_UPDATE_CALL(V) kmed_update<V>(X, order, offsets, p, medoids, s)
    KMED_DP_SWITCH(dp, KMED_UPDATE_CALL)
#undef KMED_UPDATE_CALL
}

}  // namespace knn
