// exact.cu -- brute-force exact k-nn graph (Sec. 2.1: every pairwise
// similarity, keep the k most similar per node), with the per-row selection
// fused into the distance loop so that the n x n distance matrix never
// leaves the chip.
//
// A block owns 64 rows and streams all columns in tiles of 64.  Squared
// distances are accumulated directly as sum (x - y)^2 in FP32 (no
// |x|^2 + |y|^2 - 2xy cancellation), 4 rows x 8 columns per thread from
// k-major shared-memory tiles.  Each tile is staged through shared memory
// and every row keeps its best KM keys (d2 bits << 32 | column) in the
// registers of two threads, each scanning half of the tile; a key that does
// not beat the thread's current last entry costs one compare.  The two
// halves are merged at the end.  Ties go to the lower id because the key
// compares the id after the distance.
//
// Relative error of a squared distance: the DP products of a pair are added
// in dimension order by fused multiply-adds, at most about (DP + 1) units of
// 2^-24.
//
// With a row list (ExactArgs::rows) the blocks take their rows from the list
// instead, so that a subset of the rows can be recomputed against every
// column; blocks past the list's length return at once.  When the list is
// short the columns are split in segments over a second grid dimension, so
// that enough blocks run; each segment's lists are merged by a warp per row.
#include "common.cuh"
#include "kernels.h"

namespace knn {

constexpr int EX_ROWS = 64;
constexpr int EX_COLS = 64;
constexpr int EX_THREADS = 128;
constexpr int EX_LD = 68;  // padded leading dimension of the k-major tiles

template <int KM>
__device__ __forceinline__ void list_insert(uint64_t (&list)[KM], uint64_t key) {
    if (!(key < list[KM - 1])) return;
#pragma unroll
    for (int i = KM - 1; i > 0; --i)
        list[i] = key < list[i - 1] ? list[i - 1] : (key < list[i] ? key : list[i]);
    list[0] = key < list[0] ? key : list[0];
}

template <int DP, int KM>
__global__ void __launch_bounds__(EX_THREADS) exact_knn_kernel(const ExactArgs a) {
    extern __shared__ float ex_smem[];
    float *As = ex_smem;                      // [DP][EX_LD]  rows of this block, k-major
    float *Bs = ex_smem + DP * EX_LD;         // [DP][EX_LD]  current column tile, k-major
    float *Cs = Bs;                           // [EX_ROWS][EX_COLS + 1], reuses Bs after compute

    const int tid = threadIdx.x;
    const int tr = tid >> 3;   // rows tr*4 .. tr*4+3
    const int tc = tid & 7;    // cols tc*8 .. tc*8+7
    const int64_t r0 = (int64_t)blockIdx.x * EX_ROWS;
    const int64_t nrows = a.rows ? (int64_t)*a.row_count : a.n;
    if (r0 >= nrows) return;  // block-uniform
    auto row_of = [&](int64_t i) -> int64_t { return i < nrows ? (a.rows ? (int64_t)a.rows[i] : i) : -1; };
    const int sel_row = tid >> 1, sel_half = tid & 1;
    const int64_t grow = row_of(r0 + sel_row);  // -1: no row
    // this block's columns [c_begin, c_end)
    const int64_t seg_len = ((a.n + gridDim.y - 1) / gridDim.y + EX_COLS - 1) / EX_COLS * EX_COLS;
    const int64_t c_begin = (int64_t)blockIdx.y * seg_len;
    const int64_t c_end = c_begin + seg_len < a.n ? c_begin + seg_len : a.n;

    // stage this block's rows (transposed)
    for (int idx = tid; idx < EX_ROWS * (DP / 4); idx += EX_THREADS) {
        const int row = idx % EX_ROWS, ch = idx / EX_ROWS;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        const int64_t src = row_of(r0 + row);
        if (src >= 0) v = *reinterpret_cast<const float4 *>(a.X + src * DP + ch * 4);
        As[(ch * 4 + 0) * EX_LD + row] = v.x;
        As[(ch * 4 + 1) * EX_LD + row] = v.y;
        As[(ch * 4 + 2) * EX_LD + row] = v.z;
        As[(ch * 4 + 3) * EX_LD + row] = v.w;
    }

    uint64_t list[KM];
#pragma unroll
    for (int i = 0; i < KM; ++i) list[i] = KEY_EMPTY;

    for (int64_t c0 = c_begin; c0 < c_end; c0 += EX_COLS) {
        __syncthreads();  // previous tile's selection done with Cs/Bs
        for (int idx = tid; idx < EX_COLS * (DP / 4); idx += EX_THREADS) {
            const int col = idx % EX_COLS, ch = idx / EX_COLS;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (c0 + col < c_end) v = *reinterpret_cast<const float4 *>(a.X + (c0 + col) * DP + ch * 4);
            Bs[(ch * 4 + 0) * EX_LD + col] = v.x;
            Bs[(ch * 4 + 1) * EX_LD + col] = v.y;
            Bs[(ch * 4 + 2) * EX_LD + col] = v.z;
            Bs[(ch * 4 + 3) * EX_LD + col] = v.w;
        }
        __syncthreads();
        float acc[4][8];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
#pragma unroll 4
        for (int kk = 0; kk < DP; ++kk) {
            const float4 av = *reinterpret_cast<const float4 *>(As + kk * EX_LD + tr * 4);
            const float4 b0 = *reinterpret_cast<const float4 *>(Bs + kk * EX_LD + tc * 8);
            const float4 b1 = *reinterpret_cast<const float4 *>(Bs + kk * EX_LD + tc * 8 + 4);
            const float ar[4] = {av.x, av.y, av.z, av.w};
            const float br[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float d = ar[i] - br[j];
                    acc[i][j] = fmaf(d, d, acc[i][j]);
                }
        }
        __syncthreads();  // everyone done reading Bs
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) Cs[(tr * 4 + i) * (EX_COLS + 1) + tc * 8 + j] = acc[i][j];
        __syncthreads();
        // selection: two threads per row, 32 columns each
        if (grow >= 0) {
#pragma unroll 4
            for (int c = 0; c < EX_COLS / 2; ++c) {
                const int col = sel_half * (EX_COLS / 2) + c;
                const int64_t gcol = c0 + col;
                if (gcol >= c_end || gcol == grow) continue;
                if (a.removed && ((a.removed[gcol >> 5] >> (gcol & 31)) & 1u)) continue;
                list_insert<KM>(list, pack_key(Cs[sel_row * (EX_COLS + 1) + col], (uint32_t)gcol));
            }
        }
    }

    // merge the two halves of each row (partner lane = tid ^ 1)
#pragma unroll
    for (int i = 0; i < KM; ++i) {
        const uint64_t other = shfl_u64_xor(list[i]);
        if (sel_half == 0) list_insert<KM>(list, other);
    }
    if (gridDim.y > 1) {
        if (sel_half == 0 && grow >= 0) {
            uint64_t *part = a.partial + ((r0 + sel_row) * gridDim.y + blockIdx.y) * 32;
#pragma unroll
            for (int i = 0; i < KM; ++i) part[i] = list[i];
            for (int i = KM; i < 32; ++i) part[i] = KEY_EMPTY;
        }
        return;
    }
    if (sel_half == 0 && grow >= 0) {
#pragma unroll
        for (int i = 0; i < KM; ++i) {
            if (i < a.k) {
                a.out_ids[grow * a.k + i] = list[i] == KEY_EMPTY ? -1 : (int32_t)key_id(list[i]);
                a.out_d2[grow * a.k + i] = list[i] == KEY_EMPTY ? __int_as_float(0x7f800000) : key_d2(list[i]);
            }
        }
    }
}

// One warp per listed row: the k best of its segments' partial lists.
__global__ void exact_merge_kernel(const ExactArgs a) {
    const int lane = threadIdx.x & 31;
    const int64_t slot = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (slot >= (int64_t)*a.row_count) return;  // warp-uniform
    const int64_t u = a.rows[slot];
    const uint64_t *part = a.partial + slot * a.col_segments * 32;
    WarpTop<1> top;
    top.init(a.k);
    for (int s = 0; s < a.col_segments; ++s) {
        const uint64_t key = part[s * 32 + lane];
        unsigned m = __ballot_sync(FULL, key < top.worst);
        while (m) {
            const int l = __ffs(m) - 1;
            top.offer(shfl_u64(key, l));
            m &= m - 1;
        }
    }
    if (lane < a.k) {
        const uint64_t key = top.e[0];
        a.out_ids[u * a.k + lane] = key == KEY_EMPTY ? -1 : (int32_t)key_id(key);
        a.out_d2[u * a.k + lane] = key == KEY_EMPTY ? __int_as_float(0x7f800000) : key_d2(key);
    }
}

int exact_col_segments(int64_t rows, int64_t n, int sm_count) {
    const int64_t row_blocks = (rows + EX_ROWS - 1) / EX_ROWS;
    const int64_t want = 2 * (int64_t)sm_count;
    if (rows <= 0 || row_blocks >= want) return 1;
    int64_t seg = (want + row_blocks - 1) / row_blocks;
    const int64_t max_seg = (n + 4 * EX_COLS - 1) / (4 * EX_COLS);  // at least 4 tiles a segment
    if (seg > max_seg) seg = max_seg;
    while (seg > 1 && row_blocks * EX_ROWS * seg > EXACT_PARTIAL_SLOTS) --seg;
    return seg < 1 ? 1 : (int)seg;
}

template <int DP, int KM>
static cudaError_t exact_dp(const ExactArgs &a, cudaStream_t s) {
    constexpr size_t b_floats = (size_t)DP * EX_LD > (size_t)EX_ROWS * (EX_COLS + 1)
                                    ? (size_t)DP * EX_LD : (size_t)EX_ROWS * (EX_COLS + 1);
    const size_t smem = ((size_t)DP * EX_LD + b_floats) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(exact_knn_kernel<DP, KM>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t rows = a.rows && a.row_hint > 0 && a.row_hint < a.n ? a.row_hint : a.n;
    const int64_t blocks = (rows + EX_ROWS - 1) / EX_ROWS;
    const unsigned segs = a.col_segments > 1 && a.rows && a.partial ? (unsigned)a.col_segments : 1u;
    exact_knn_kernel<DP, KM><<<dim3((unsigned)blocks, segs), EX_THREADS, smem, s>>>(a);
    if (segs > 1) {
        // listed rows fill the partial buffer's slots only up to its bound
        int64_t warps = EXACT_PARTIAL_SLOTS / segs;
        if (a.row_hint > 0 && a.row_hint < warps) warps = a.row_hint;
        exact_merge_kernel<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, s>>>(a);
    }
    return cudaGetLastError();
}

template <int DP>
static cudaError_t exact_k(const ExactArgs &a, cudaStream_t s) {
    if (a.k <= 16) return exact_dp<DP, 16>(a, s);
    return exact_dp<DP, 32>(a, s);
}

cudaError_t launch_exact(int dp, const ExactArgs &a, cudaStream_t s) {
    if (a.n <= 0) return cudaSuccess;
    if (a.k < 1 || a.k > 32) return cudaErrorInvalidValue;
    switch (dp) {
        case 16: return exact_k<16>(a, s);
        case 32: return exact_k<32>(a, s);
        case 64: return exact_k<64>(a, s);
        case 96: return exact_k<96>(a, s);
        case 128: return exact_k<128>(a, s);
        case 256: return exact_k<256>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace knn
