// partition.cu -- kernels of the distributed online build (Sec. 7,
// Algorithm 5) run on one device: the graph split in P partitions given by a
// label per node, each partition searched on its own subgraph (Algorithm 3),
// every new node given to the partition of its most similar medoid.
//
// The partitioned search kernel searches contiguous node ranges, so before a
// batch the nodes are staged in partition order: position i of the staged
// copy holds node order[i] (a stable counting sort by label, so a partition
// keeps its nodes in id order), its searched row, and its list with the
// entries inside its own partition renumbered to positions and the others
// dropped (-1): the subgraph of each partition, as the distributed search
// sees it.  The staged search's candidate ids are positions; they are mapped
// back to node ids before the partitions' candidates are merged, so the
// merge breaks ties between partitions by node id.
#include "common.cuh"
#include "kernels.h"

namespace knn {

// pos[order[i]] = i for i < n
__global__ void part_positions_kernel(const int64_t *order, int64_t n, int64_t *pos) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) pos[order[i]] = i;
}

// One warp per position i < n: node v = order[i]; its searched row
// (row_bytes, a multiple of 16), its FP8 scale and its list, each entry
// inside v's partition as that node's position, the others -1.
__global__ void part_stage_kernel(const uint8_t *rows, int64_t row_bytes, const float *scale, const int32_t *nbr,
                                  int k, const int32_t *label, const int64_t *order, const int64_t *pos, int64_t n,
                                  uint8_t *st_rows, float *st_scale, int32_t *st_nbr) {
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= n) return;  // warp-uniform
    const int64_t v = order[i];
    const uint4 *src = reinterpret_cast<const uint4 *>(rows + v * row_bytes);
    uint4 *dst = reinterpret_cast<uint4 *>(st_rows + i * row_bytes);
    for (int64_t c = lane; c < row_bytes / 16; c += 32) dst[c] = src[c];
    if (scale && lane == 0) st_scale[i] = scale[v];
    const int32_t own = label[v];
    for (int j = lane; j < k; j += 32) {
        const int32_t nb = nbr[v * k + j];
        st_nbr[i * k + j] = (nb >= 0 && (int64_t)nb < n && label[nb] == own) ? (int32_t)pos[nb] : -1;
    }
}

// Candidate keys of the staged search: position -> node id, in place; empty
// keys stay empty.  The squared distance (the high half) is unchanged.
__global__ void part_keys_to_nodes_kernel(uint64_t *keys, int64_t count, const int64_t *order) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const uint64_t key = keys[i];
    if (key == KEY_EMPTY) return;
    keys[i] = (key & 0xffffffff00000000ull) | (uint64_t)(uint32_t)order[key_id(key)];
}

// Algorithm 5's assignment: one warp per new point x_i (padded FP32 rows,
// i < m), the position of its most similar medoid, i.e. the smallest squared
// distance (FP32, lanes over dimensions, then a butterfly sum); ties to the
// lower position.
__global__ void part_nearest_kernel(const float *X, int dp, const float *rows, int64_t m,
                                    const int64_t *medoids, int p, int32_t *labels) {
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= m) return;  // warp-uniform
    const float *x = rows + i * dp;
    float best = __int_as_float(0x7f800000);
    int best_j = 0;
    for (int j = 0; j < p; ++j) {
        const float *y = X + medoids[j] * dp;
        float s = 0.f;
        for (int c = lane; c < dp; c += 32) {
            const float d = x[c] - y[c];
            s = fmaf(d, d, s);
        }
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) s += __shfl_xor_sync(FULL, s, off);
        if (s < best) {  // the same value in every lane
            best = s;
            best_j = j;
        }
    }
    if (lane == 0) labels[i] = best_j;
}

cudaError_t launch_part_stage(const uint8_t *rows, int64_t row_bytes, const float *scale, const int32_t *nbr, int k,
                              const int32_t *label, const int64_t *order, int64_t *pos, int64_t n, uint8_t *st_rows,
                              float *st_scale, int32_t *st_nbr, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    part_positions_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(order, n, pos);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    part_stage_kernel<<<(unsigned)((n * 32 + 255) / 256), 256, 0, s>>>(rows, row_bytes, scale, nbr, k, label, order,
                                                                        pos, n, st_rows, st_scale, st_nbr);
    return cudaGetLastError();
}

cudaError_t launch_part_keys_to_nodes(uint64_t *keys, int64_t count, const int64_t *order, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    part_keys_to_nodes_kernel<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(keys, count, order);
    return cudaGetLastError();
}

cudaError_t launch_part_nearest(const float *X, int dp, const float *rows, int64_t m, const int64_t *medoids, int p,
                                int32_t *labels, cudaStream_t s) {
    if (m <= 0) return cudaSuccess;
    part_nearest_kernel<<<(unsigned)((m * 32 + 255) / 256), 256, 0, s>>>(X, dp, rows, m, medoids, p, labels);
    return cudaGetLastError();
}

}  // namespace knn
