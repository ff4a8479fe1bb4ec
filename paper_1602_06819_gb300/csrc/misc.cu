// misc.cu -- storing new rows (with their screening encodings), turning
// packed keys into the public (id, similarity) form, and small fills.
#include "common.cuh"
#include "kernels.h"

namespace knn {

cudaError_t launch_search_fp32(int dp, const SearchArgs &a, cudaStream_t s);
cudaError_t launch_search_bf16(int dp, const SearchArgs &a, cudaStream_t s);
cudaError_t launch_search_fp8(int dp, const SearchArgs &a, cudaStream_t s);

bool supported_dp(int dp) {
    return dp == 16 || dp == 32 || dp == 64 || dp == 96 || dp == 128 || dp == 256;
}

int padded_dim(int d) {
    static const int dps[] = {16, 32, 64, 96, 128, 256};
    for (int dp : dps)
        if (d <= dp) return dp;
    return -1;
}

bool search_visited_on_chip(uint32_t n) {
    // the same rule as the search launcher: 4 warps' bitsets within 110 KiB
    return (size_t)4 * ((n + 31) / 32) * sizeof(uint32_t) <= (size_t)110 * 1024;
}

cudaError_t launch_search(int storage, int dp, const SearchArgs &a, cudaStream_t s) {
    switch (storage) {
        case ST_FP32: return launch_search_fp32(dp, a, s);
        case ST_BF16: return launch_search_bf16(dp, a, s);
        case ST_FP8: return launch_search_fp8(dp, a, s);
        default: return cudaErrorInvalidValue;
    }
}

// One warp per row: copy d floats into a DP-wide FP32 row (zero padded) and,
// when asked, the BF16 copy (round to nearest even) or the FP8-E4M3 copy with
// a per-row scale amax / 448 (code = e4m3(x / scale), round to nearest even,
// saturating; a zero row gets scale 1).
// One warp: row `x` (d floats) to row r of the stored copies.
__device__ __forceinline__ void encode_row(const float *x, int d, int dp, int64_t r, float *rows,
                                           uint16_t *rows_bf16, uint8_t *rows_fp8, float *scale) {
    const int lane = threadIdx.x & 31;
    float amax = 0.f;
    for (int c = lane; c < dp; c += 32) {
        const float v = c < d ? x[c] : 0.f;
        rows[r * dp + c] = v;
        amax = fmaxf(amax, fabsf(v));
        if (rows_bf16) rows_bf16[r * dp + c] = __bfloat16_as_ushort(__float2bfloat16_rn(v));
    }
    if (rows_fp8) {
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) amax = fmaxf(amax, __shfl_xor_sync(FULL, amax, off));
        const float sc = amax > 0.f ? __fdiv_rn(amax, 448.0f) : 1.0f;
        if (lane == 0) scale[r] = sc;
        for (int c = lane; c < dp; c += 32) {
            const float v = c < d ? x[c] : 0.f;
            rows_fp8[r * dp + c] = (uint8_t)__nv_cvt_float_to_fp8(__fdiv_rn(v, sc), __NV_SATFINITE, __NV_E4M3);
        }
    }
}

__global__ void append_kernel(const float *in, int64_t m, int d, int dp, float *rows,
                              uint16_t *rows_bf16, uint8_t *rows_fp8, float *scale) {
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (r >= m) return;
    encode_row(in + r * d, d, dp, r, rows, rows_bf16, rows_fp8, scale);
}

// A step over several graphs: item i of the staged vectors (inserts first)
// becomes query row i; an insert item is also stored at its new node.
__global__ void multi_append_kernel(const float *in, const int32_t *count_all, Segments ins, int d, int dp,
                                    float *q_rows, float *rows, uint16_t *rows_bf16, uint8_t *rows_fp8,
                                    float *scale) {
    const int m_all = *count_all, m_ins = *ins.count;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < m_all; i += nw) {
        encode_row(in + i * d, d, dp, i, q_rows, nullptr, nullptr, nullptr);
        if (i < m_ins) {
            const uint32_t node = seg_new_id(ins, ins.item_seg[i], (int32_t)i);
            encode_row(in + i * d, d, dp, node, rows, rows_bf16, rows_fp8, scale);
        }
    }
}

cudaError_t launch_multi_append(const float *in, const int32_t *count_all, const Segments &ins, int d, int dp,
                                float *q_rows, float *rows, uint16_t *rows_bf16, uint8_t *rows_fp8, float *scale,
                                int grid, cudaStream_t s) {
    multi_append_kernel<<<grid, 256, 0, s>>>(in, count_all, ins, d, dp, q_rows, rows, rows_bf16, rows_fp8, scale);
    return cudaGetLastError();
}

// Query results of a step over several graphs: the m_q query items follow
// the m_ins insert items; item i's k_out best keys go to output row perm[i]
// with ids local to its graph.
__global__ void multi_keys_out_kernel(const uint64_t *keys, const int32_t *count_q, const int32_t *count_ins,
                                      int kk, int k_out, const int32_t *item_seg, const uint32_t *lo,
                                      const int32_t *perm, int64_t *out_ids, float *out_sims) {
    const int m_q = *count_q, m_ins = *count_ins;
    const int64_t total = (int64_t)m_q * k_out;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(t / k_out), c = (int)(t % k_out);
        const int i = m_ins + j;
        const uint64_t key = keys[(size_t)i * kk + c];
        const int64_t o = (int64_t)perm[i] * k_out + c;
        out_ids[o] = key == KEY_EMPTY ? -1 : (int64_t)key_id(key) - (int64_t)lo[item_seg[i]];
        if (out_sims) out_sims[o] = key == KEY_EMPTY ? 0.f : sim_of_d2(key_d2(key));
    }
}

cudaError_t launch_multi_keys_out(const uint64_t *keys, const int32_t *count_q, const int32_t *count_ins, int kk,
                                  int k_out, const int32_t *item_seg, const uint32_t *lo, const int32_t *perm,
                                  int64_t *out_ids, float *out_sims, int grid, cudaStream_t s) {
    multi_keys_out_kernel<<<grid, 256, 0, s>>>(keys, count_q, count_ins, kk, k_out, item_seg, lo, perm, out_ids,
                                               out_sims);
    return cudaGetLastError();
}

// ids[i] += add for the i < count entries that are >= 0
__global__ void shift_ids_kernel(int32_t *ids, int64_t count, int32_t add) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < count && ids[t] >= 0) ids[t] += add;
}

cudaError_t launch_shift_ids(int32_t *ids, int64_t count, int32_t add, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    shift_ids_kernel<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(ids, count, add);
    return cudaGetLastError();
}

cudaError_t launch_append(const float *in, int64_t m, int d, int dp, float *rows_fp32,
                          uint16_t *rows_bf16, uint8_t *rows_fp8, float *scale, cudaStream_t s) {
    if (m <= 0) return cudaSuccess;
    const int64_t threads = m * 32;
    append_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(in, m, d, dp, rows_fp32, rows_bf16,
                                                                   rows_fp8, scale);
    return cudaGetLastError();
}

__global__ void keys_to_output_kernel(const uint64_t *keys, int64_t m, int kk, int k_out,
                                      int64_t *out_ids, float *out_sims) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m * k_out) return;
    const int64_t row = t / k_out, col = t % k_out;
    const uint64_t key = keys[row * kk + col];
    out_ids[t] = key == KEY_EMPTY ? -1 : (int64_t)key_id(key);
    if (out_sims) out_sims[t] = key == KEY_EMPTY ? 0.f : sim_of_d2(key_d2(key));
}

cudaError_t launch_keys_to_output(const uint64_t *keys, int64_t m, int kk, int k_out,
                                  int64_t *out_ids, float *out_sims, cudaStream_t s) {
    const int64_t total = m * k_out;
    if (total <= 0) return cudaSuccess;
    keys_to_output_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(keys, m, kk, k_out, out_ids, out_sims);
    return cudaGetLastError();
}

__global__ void lists_to_output_kernel(const int32_t *ids, const float *d2, int64_t total,
                                       int64_t *out_ids, float *out_sims) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    const int32_t id = ids[t];
    out_ids[t] = id;
    if (out_sims) out_sims[t] = id < 0 ? 0.f : sim_of_d2(d2[t]);
}

cudaError_t launch_lists_to_output(const int32_t *ids, const float *d2, int64_t rows, int k,
                                   int64_t *out_ids, float *out_sims, cudaStream_t s) {
    const int64_t total = rows * k;
    if (total <= 0) return cudaSuccess;
    lists_to_output_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(ids, d2, total, out_ids, out_sims);
    return cudaGetLastError();
}

// One warp per query (Algorithm 3, "keep k most similar nodes"): the keys of
// its searches are distinct nodes, so the best k_keep of their union is the
// merged list; counters add up.
template <int T>
__global__ void merge_parts_kernel(const uint64_t *keys, int32_t m, int32_t parts, int32_t k_keep, uint64_t *out,
                                   const long long *ctr_in, long long *ctr_out) {
    const int lane = threadIdx.x & 31;
    const int64_t qi = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (qi >= m) return;  // warp-uniform
    WarpTop<T> top;
    top.init(k_keep);
    for (int p = 0; p < parts; ++p) {
        const uint64_t *src = keys + ((size_t)qi * parts + p) * k_keep;
        for (int i0 = 0; i0 < k_keep; i0 += 32) {
            const uint64_t key = i0 + lane < k_keep ? src[i0 + lane] : KEY_EMPTY;
            unsigned om = __ballot_sync(FULL, key < top.worst);
            while (om) {
                const int l = __ffs(om) - 1;
                top.offer(shfl_u64(key, l));
                om &= ~(1u << l);
                om &= __ballot_sync(FULL, key < top.worst);
            }
        }
    }
#pragma unroll
    for (int t = 0; t < T; ++t) {
        const int idx = t * 32 + lane;
        if (idx < k_keep) out[(size_t)qi * k_keep + idx] = top.e[t];
    }
    if (lane < NCTR) {
        long long sum = 0;
        for (int p = 0; p < parts; ++p) sum += ctr_in[((size_t)qi * parts + p) * NCTR + lane];
        ctr_out[(size_t)qi * NCTR + lane] = sum;
    }
}

cudaError_t launch_merge_parts(const uint64_t *keys, int32_t m, int32_t parts, int32_t k_keep, uint64_t *out,
                               const long long *ctr_in, long long *ctr_out, cudaStream_t s) {
    if (m <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((m * 32 + 127) / 128);
    if (k_keep <= 32)
        merge_parts_kernel<1><<<blocks, 128, 0, s>>>(keys, m, parts, k_keep, out, ctr_in, ctr_out);
    else
        merge_parts_kernel<4><<<blocks, 128, 0, s>>>(keys, m, parts, k_keep, out, ctr_in, ctr_out);
    return cudaGetLastError();
}

__global__ void add_u64_kernel(uint64_t *p, uint64_t v, int64_t m) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < m) p[t] += v;
}

cudaError_t launch_add_u64(uint64_t *p, uint64_t v, int64_t m, cudaStream_t s) {
    if (m <= 0) return cudaSuccess;
    add_u64_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(p, v, m);
    return cudaGetLastError();
}

__global__ void fill_ids_kernel(int64_t *out, int64_t first, int64_t m) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < m) out[t] = first + t;
}

cudaError_t launch_fill_ids(int64_t *out, int64_t first, int64_t m, cudaStream_t s) {
    if (m <= 0) return cudaSuccess;
    fill_ids_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(out, first, m);
    return cudaGetLastError();
}

__global__ void mark_removed_kernel(uint32_t *removed, const int64_t *ids, int64_t m) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < m) atomicOr(removed + (ids[t] >> 5), 1u << (ids[t] & 31));
}

cudaError_t launch_mark_removed(uint32_t *removed, const int64_t *ids, int64_t m, cudaStream_t s) {
    if (m <= 0) return cudaSuccess;
    mark_removed_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(removed, ids, m);
    return cudaGetLastError();
}

__global__ void fill_i32_kernel(int32_t *p, int32_t v, int64_t count) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < count) p[t] = v;
}

cudaError_t launch_fill_i32(int32_t *p, int32_t v, int64_t count, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    fill_i32_kernel<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(p, v, count);
    return cudaGetLastError();
}

}  // namespace knn
