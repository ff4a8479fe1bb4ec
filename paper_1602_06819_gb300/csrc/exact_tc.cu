// exact_tc.cu -- brute-force exact k-nn graph (Sec. 2.1) screened on the
// tensor cores and settled in FP32.
//
// Ranking key of column v for row u: ||y_v||^2 - 2 x_u . y_v (the row
// constant ||x_u||^2 is dropped).  The dot products run on tcgen05 with BF16
// operands and FP32 accumulation, made nearly FP32-accurate by splitting each
// value in two BF16 parts, x = hi + lo (hi = bf16(x), lo = bf16(x - hi)), and
// accumulating hi.hi + hi.lo + lo.hi.
//
// One CTA owns 128 rows and streams every column in 192-column tiles (16 warps):
//   warp 0      TMA: the CTA's rows (hi and lo) once, then the column tiles,
//               one 64-element K slice (hi and lo) per ring stage;
//   warp 1      owns the TMEM allocation; one thread issues the MMAs of a
//               192-column tile into one of two FP32 accumulators (256 TMEM
//               columns apart, all 512 allocated), so it runs a tile ahead
//               of the epilogue;
//   warp 2      copies each tile's column norms beside its accumulator;
//   warps 4..15 epilogue, three warpgroups: thread r of warpgroup h reads
//               accumulator lane r (its row), columns 64h .. 64h+63 of each
//               tile, forms their keys and keeps the 24 smallest it sees
//               (20 when k <= 10).
// The three lists of a row share a threshold: each publishes its 24th key in
// shared memory when it changes, and a thread appends only keys below the
// smallest of the three (published keys only fall, so a stale one is merely
// looser).  A key below that threshold is only appended to a per-thread
// buffer in shared memory; when some lane's buffer may not hold 16 more the warp
// merges all buffers into the sorted lists in lockstep, so the costly
// insertions of the 32 rows of a warp run together instead of one lane at
// a time.
//
// The screening is then made exact.  The 72 (60) candidates of a row (24, or
// 20, per warpgroup) are re-scored as FP32 squared differences and the k best
// kept.
// Every other column has a screened key at least the smallest of the three
// lists' last keys (+inf for a list that never filled): it was either not
// appended, so at least some list's 24th at that time, or pushed out of its
// own list; the row is accepted only if a proven bound on the
// screening error shows that no such column can beat its k-th neighbour,
// otherwise it is recomputed against every column in FP32 by the CUDA-core
// kernel.  The lists therefore equal the exact ones up to FP32 rounding of
// the distances.
//
// Every mbarrier wait is bounded.  A pipeline wait (one role waiting for
// another) that gives up after wait_ns sets a bit of the error word and the
// rows of that CTA are marked for the FP32 pass, so the result stays exact;
// before the CTA exits, every copy and MMA it issued is waited for (drain
// waits, on work that completes by itself) so that nothing is left in flight.
#include <algorithm>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "kernels.h"
#include "tc_sm100.cuh"

namespace knn {

using namespace tc;

constexpr int TC_ROWS = 128;            // rows per CTA (MMA M)
constexpr int TC_COLS = 192;            // columns per tile (MMA N)
constexpr int TC_NWG = 3;               // epilogue warpgroups, each with its own columns of a tile
constexpr int TC_WG_COLS = TC_COLS / TC_NWG;  // columns of a tile per epilogue thread
constexpr int TC_ACC_STRIDE = TC_COLS <= 128 ? 128 : 256;  // TMEM columns from one accumulator to the next
constexpr int TC_NACC = 512 / TC_ACC_STRIDE;  // TMEM accumulators: the MMAs run up to TC_NACC - 1 tiles ahead
constexpr int TC_CAND = TC_NWG == 2 ? 32 : 24;  // candidates kept per row and warpgroup, at most
constexpr int TC_CAND_SMALL_K = 20;     // the list of a warpgroup when k <= TC_SMALL_K
constexpr int TC_SMALL_K = 10;
constexpr int TC_NCAND = TC_NWG * TC_CAND;  // candidates per row
constexpr int TC_EPI = TC_NWG * 128;    // epilogue threads
constexpr int TC_THREADS = 128 + TC_EPI;  // 4 warps for the copies, the MMAs and the norms, then the epilogue
constexpr int TC_BUF = TC_NWG == 2 ? 31 : 20;  // buffered keys per epilogue thread
constexpr uint32_t TC_BOX = 128 * 128;  // bytes of one 128-row x 64-element BF16 box (the CTA's rows)
constexpr uint32_t TC_UNIT = 2 * TC_BOX;  // hi and lo boxes of one K slice of the rows
constexpr uint32_t TC_BOX_B = TC_COLS * 128;  // the hi or the lo box of one K slice of a column tile
constexpr uint32_t TC_STAGE = 2 * TC_BOX_B;     // a ring stage: both boxes of one K slice
static_assert(TC_WG_COLS % 32 == 0, "an epilogue thread reads its columns 32 at a time");
static_assert(TC_COLS % 16 == 0 && TC_COLS <= TC_ACC_STRIDE, "MMA N and accumulators in TMEM");
constexpr uint64_t TC_WAIT = 2000000000ull;  // ns before a drain wait gives up (the default pipeline limit too)

// NBOX 64-element K slices per row (padded width 64 * NBOX); the ring takes
// as many stages as the shared memory left holds
template <int NBOX>
struct TcCfg {
    static constexpr uint32_t A_BYTES = NBOX * TC_UNIT;
    static constexpr uint32_t BUF_BYTES = TC_BUF * TC_EPI * 8;
    static constexpr uint32_t FIXED =
        1024 + A_BYTES + BUF_BYTES + TC_NACC * TC_COLS * 4 + TC_NWG * TC_ROWS * 4 + (3 * TC_NACC + 2) * 8 + 16;
    static constexpr int STAGES = (232448 - FIXED) / (TC_STAGE + 16) < 8 ? (232448 - FIXED) / (TC_STAGE + 16) : 8;
    static constexpr int NBAR = 1 + 2 * STAGES + 3 * TC_NACC + 1;  // a_full, b_full/empty, acc full/empty, yn_full, drain
    static constexpr uint32_t SMEM = FIXED + STAGES * (TC_STAGE + 16);
    static_assert(STAGES >= 2 && SMEM <= 232448, "shared memory of one CTA");
};

// x -> (hi, lo) BF16 rows of width dpt (zero padded) and FP32 squared norms;
// the largest norm goes to *norm_max (bit pattern of a non-negative float,
// so that unsigned order is float order).  Rows n .. n_pad-1 get the norm
// +inf, so that a column tile copied past the last row yields keys that are
// never kept.
__global__ void tc_split_kernel(const float *X, int64_t n, int64_t n_pad, int dp, int dpt, __nv_bfloat16 *hi,
                                __nv_bfloat16 *lo, float *norm2, unsigned *norm_max) {
    const int lane = threadIdx.x & 31;
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (r >= n) {
        if (r < n_pad && lane == 0) norm2[r] = __int_as_float(0x7f800000);
        return;
    }
    float s = 0.f;
    for (int c = lane; c < dpt; c += 32) {
        const float x = c < dp ? X[r * dp + c] : 0.f;
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        hi[r * dpt + c] = h;
        lo[r * dpt + c] = __float2bfloat16_rn(x - __bfloat162float(h));
        s = fmaf(x, x, s);
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) s += __shfl_xor_sync(FULL, s, off);
    if (lane == 0) {
        norm2[r] = s;
        atomicMax(norm_max, __float_as_uint(sqrtf(s)));
    }
}

// insert (k, v) into the ascending list of the TC_CAND smallest keys
template <int L>
__device__ __forceinline__ void cand_insert(float (&key)[L], int (&id)[L], float k, int v) {
#pragma unroll
    for (int i = L - 1; i > 0; --i) {
        const bool shift = k < key[i - 1];
        const bool here = !shift && k < key[i];
        key[i] = shift ? key[i - 1] : (here ? k : key[i]);
        id[i] = shift ? id[i - 1] : (here ? v : id[i]);
    }
    if (k < key[0]) {
        key[0] = k;
        id[0] = v;
    }
}

// L: the length of a warpgroup's candidate list (the rest of its TC_CAND
// slots are written empty)
template <int NBOX, int L>
__global__ void __launch_bounds__(TC_THREADS, 1)
exact_tc_kernel(const __grid_constant__ CUtensorMap t_hi, const __grid_constant__ CUtensorMap t_lo,
                const __grid_constant__ CUtensorMap t_bhi, const __grid_constant__ CUtensorMap t_blo,
                const float *__restrict__ norm2, int64_t n, int64_t full_blocks, int parts,
                int32_t *cand_id, float *cand_key, int32_t *part_id, float *part_key, unsigned *err,
                uint64_t wait_ns) {
    using Cfg = TcCfg<NBOX>;
    constexpr int S = Cfg::STAGES;
    extern __shared__ uint8_t tc_raw[];
    // 128-byte swizzled tiles want 1024-byte aligned shared memory
    uint8_t *sm = (uint8_t *)(((uintptr_t)tc_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *As = sm;                                   // NBOX x [hi box][lo box]
    uint8_t *Bs = As + Cfg::A_BYTES;                    // S ring stages
    uint64_t *sbuf = (uint64_t *)(Bs + S * TC_STAGE);   // [TC_BUF][TC_EPI] buffered (column, key bits)
    float *s_yn = (float *)(sbuf + TC_BUF * TC_EPI);    // [TC_NACC][TC_COLS] column norms
    volatile float *s_thr = s_yn + TC_NACC * TC_COLS;       // [TC_NWG][TC_ROWS] each list's last key
    uint64_t *bars = (uint64_t *)(s_yn + TC_NACC * TC_COLS + TC_NWG * TC_ROWS);
    uint64_t *a_full = bars, *b_full = bars + 1, *b_empty = bars + 1 + S;
    uint64_t *acc_full = bars + 1 + 2 * S, *acc_empty = acc_full + TC_NACC, *yn_full = acc_empty + TC_NACC;
    uint64_t *drain = yn_full + TC_NACC;
    uint32_t *tmem_slot = (uint32_t *)(bars + Cfg::NBAR);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        mbar_init(a_full, 1);
        for (int s = 0; s < S; ++s) {
            mbar_init(b_full + s, 1);
            mbar_init(b_empty + s, 1);
        }
        for (int b = 0; b < TC_NACC; ++b) {
            mbar_init(acc_full + b, 1);
            mbar_init(acc_empty + b, TC_EPI / 32);
            mbar_init(yn_full + b, 1);
        }
        mbar_init(drain, 1);
        fence_barrier_init();
    }
    for (int i = threadIdx.x; i < TC_NWG * TC_ROWS; i += blockDim.x) s_thr[i] = __int_as_float(0x7f800000);
    if (warp == 1) {
        tmem_alloc(tmem_slot, TC_NACC * TC_ACC_STRIDE);
        tmem_relinquish();
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    // CTAs below full_blocks take every column tile of their row block; the
    // rest split the row blocks after those into `parts` runs of tiles each
    const int all_tiles = (int)((n + TC_COLS - 1) / TC_COLS);
    int64_t rb = blockIdx.x;
    int part = -1, t0 = 0, ntiles = all_tiles;
    if (rb >= full_blocks) {
        const int64_t j = rb - full_blocks;
        rb = full_blocks + j / parts;
        part = (int)(j % parts);
        t0 = (int)((int64_t)all_tiles * part / parts);
        ntiles = (int)((int64_t)all_tiles * (part + 1) / parts) - t0;
    }
    const int64_t row0 = rb * TC_ROWS;

    if (warp == 0 && lane == 0) {
        // ---- TMA producer
        prefetch_tensormap(&t_hi);
        prefetch_tensormap(&t_lo);
        prefetch_tensormap(&t_bhi);
        prefetch_tensormap(&t_blo);
        mbar_arrive_expect_tx(a_full, Cfg::A_BYTES);
        for (int kb = 0; kb < NBOX; ++kb) {
            tma_load_2d(As + kb * TC_UNIT, &t_hi, a_full, kb * 64, (int)row0);
            tma_load_2d(As + kb * TC_UNIT + TC_BOX, &t_lo, a_full, kb * 64, (int)row0);
        }
        // unit u: K slice u % NBOX of column tile u / NBOX
        const int units = ntiles * NBOX;
        int issued = 0;
        for (int u = 0; u < units; ++u) {
            const int s = u % S;
            if (u >= S && !mbar_wait(b_empty + s, ((u / S) - 1) & 1, wait_ns)) {
                atomicOr(err, 1u);
                break;
            }
            const int t = t0 + u / NBOX, kb = u % NBOX;
            mbar_arrive_expect_tx(b_full + s, TC_STAGE);
            tma_load_2d(Bs + s * TC_STAGE, &t_bhi, b_full + s, kb * 64, t * TC_COLS);
            tma_load_2d(Bs + s * TC_STAGE + TC_BOX_B, &t_blo, b_full + s, kb * 64, t * TC_COLS);
            issued = u + 1;
        }
        // no copy may still be in flight when the CTA exits
        bool landed = mbar_wait(a_full, 0, TC_WAIT);
        for (int u = issued > S ? issued - S : 0; u < issued; ++u)
            landed = mbar_wait(b_full + u % S, (u / S) & 1, TC_WAIT) && landed;
        if (!landed) atomicOr(err, 32u);
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer: acc = A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T
        constexpr uint32_t idesc = idesc_bf16_f32(TC_ROWS, TC_COLS);
        bool ok = mbar_wait(a_full, 0, wait_ns);
        if (!ok) atomicOr(err, 2u);
        for (int t = 0; ok && t < ntiles; ++t) {
            const int buf = t % TC_NACC;
            if (t >= TC_NACC && !mbar_wait(acc_empty + buf, ((t / TC_NACC) - 1) & 1, wait_ns)) {
                atomicOr(err, 8u);
                break;
            }
            const uint32_t d = tmem + buf * TC_ACC_STRIDE;
            for (int kb = 0; kb < NBOX; ++kb) {
                const int u = t * NBOX + kb, s = u % S;
                if (!mbar_wait(b_full + s, (u / S) & 1, wait_ns)) {
                    atomicOr(err, 4u);
                    ok = false;
                    break;
                }
                fence_after_sync();
                const uint64_t ah = sdesc_k_sw128(smem_u32(As + kb * TC_UNIT));
                const uint64_t al = sdesc_k_sw128(smem_u32(As + kb * TC_UNIT + TC_BOX));
                const uint64_t bh = sdesc_k_sw128(smem_u32(Bs + s * TC_STAGE));
                const uint64_t bl = sdesc_k_sw128(smem_u32(Bs + s * TC_STAGE + TC_BOX_B));
                for (int kk = 0; kk < 4; ++kk) {  // K step of 16 BF16 = 32 bytes = 2 descriptor units
                    mma_bf16(d, ah + 2 * kk, bh + 2 * kk, idesc, (kb | kk) != 0);
                    mma_bf16(d, ah + 2 * kk, bl + 2 * kk, idesc, 1u);
                    mma_bf16(d, al + 2 * kk, bh + 2 * kk, idesc, 1u);
                }
                mma_commit(b_empty + s);
            }
            if (ok) mma_commit(acc_full + buf);
        }
        // every MMA issued has finished before TMEM is released
        mma_commit(drain);
        if (!mbar_wait(drain, 0, TC_WAIT)) atomicOr(err, 64u);
    } else if (warp == 2 && lane == 0) {
        // ---- column norms of tile t into s_yn[t % TC_NACC], once the epilogue has
        // released that buffer (with the accumulator of tile t - 2)
        int issued = 0;
        for (int t = 0; t < ntiles; ++t) {
            const int buf = t % TC_NACC;
            if (t >= TC_NACC && !mbar_wait(acc_empty + buf, ((t / TC_NACC) - 1) & 1, wait_ns)) {
                atomicOr(err, 128u);
                break;
            }
            mbar_arrive_expect_tx(yn_full + buf, TC_COLS * 4);
            bulk_load(s_yn + buf * TC_COLS, norm2 + (int64_t)(t0 + t) * TC_COLS, TC_COLS * 4, yn_full + buf);
            issued = t + 1;
        }
        bool landed = true;
        for (int t = issued > TC_NACC ? issued - TC_NACC : 0; t < issued; ++t)
            landed = mbar_wait(yn_full + (t % TC_NACC), (t / TC_NACC) & 1, TC_WAIT) && landed;
        if (!landed) atomicOr(err, 256u);
    } else if (warp >= 4) {
        // ---- epilogue: thread r of warpgroup h owns row row0 + r (TMEM lane r)
        const int te = threadIdx.x - 128;
        const int h = te >> 7, r = te & 127;
        const uint32_t row = (uint32_t)(row0 + r);  // rows and columns are below 2^31
        const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
        uint64_t *mybuf = sbuf + te;  // entry e at mybuf[e * TC_EPI]
        float key[L];
        int id[L];
#pragma unroll
        for (int i = 0; i < L; ++i) {
            key[i] = __int_as_float(0x7f800000);
            id[i] = -1;
        }
        float thr = __int_as_float(0x7f800000);  // current TC_CAND-th key
        int cnt = 0;                              // buffered entries
        auto flush = [&]() {
            const int m = __reduce_max_sync(FULL, cnt);
#pragma unroll 1
            for (int e = 0; e < m; ++e) {
                if (e < cnt) {
                    const uint2 ent = reinterpret_cast<const uint2 *>(mybuf)[e * TC_EPI];
                    const float kk = __uint_as_float(ent.y);
                    if (kk < key[L - 1] && ent.x != row) cand_insert(key, id, kk, (int)ent.x);
                }
            }
            cnt = 0;
            s_thr[h * TC_ROWS + r] = key[L - 1];
            thr = key[L - 1];
#pragma unroll
            for (int j = 1; j < TC_NWG; ++j) thr = fminf(thr, s_thr[((h + j) % TC_NWG) * TC_ROWS + r]);
        };
        bool ok = true;
        uint32_t c_base = (uint32_t)t0 * TC_COLS;  // first column of tile t0 + t
        for (int t = 0; t < ntiles; ++t, c_base += TC_COLS) {
            const int buf = t % TC_NACC;
            if (ok)
                ok = __all_sync(FULL, mbar_wait(acc_full + buf, (t / TC_NACC) & 1, wait_ns) &&
                                          mbar_wait(yn_full + buf, (t / TC_NACC) & 1, wait_ns));
            if (!ok && lane == 0) atomicOr(err, 16u);
            fence_after_sync();
            if (ok) {
                // the other lists of this row may have tightened theirs
#pragma unroll
                for (int j = 1; j < TC_NWG; ++j) thr = fminf(thr, s_thr[((h + j) % TC_NWG) * TC_ROWS + r]);
                const uint32_t ta = tmem + lane_base + buf * TC_ACC_STRIDE + TC_WG_COLS * h;
                const float *yn = s_yn + buf * TC_COLS + TC_WG_COLS * h;
                const uint32_t col0 = (uint32_t)c_base + TC_WG_COLS * h;
                // 16 columns: keys, then per group of 4 their minimum; only
                // the groups where some lane of the warp has a key below its
                // threshold run the appends, so that the common case takes no
                // divergent branch
                auto scan16 = [&](const uint32_t(&v)[16], int c) {
                    float kv[16];
                    const unsigned long long m2 = f32x2_pack(-2.0f, -2.0f);
#pragma unroll
                    for (int j4 = 0; j4 < 4; ++j4) {
                        const float4 y = *reinterpret_cast<const float4 *>(yn + c + 4 * j4);
                        // two keys an instruction, each rounded as fmaf would
                        unsigned long long k01, k23;
                        asm("fma.rn.f32x2 %0, %1, %2, %3;"
                            : "=l"(k01)
                            : "l"(f32x2_pack(__uint_as_float(v[4 * j4]), __uint_as_float(v[4 * j4 + 1]))), "l"(m2),
                              "l"(f32x2_pack(y.x, y.y)));
                        asm("fma.rn.f32x2 %0, %1, %2, %3;"
                            : "=l"(k23)
                            : "l"(f32x2_pack(__uint_as_float(v[4 * j4 + 2]), __uint_as_float(v[4 * j4 + 3]))),
                              "l"(m2), "l"(f32x2_pack(y.z, y.w)));
                        asm("mov.b64 {%0, %1}, %2;" : "=f"(kv[4 * j4]), "=f"(kv[4 * j4 + 1]) : "l"(k01));
                        asm("mov.b64 {%0, %1}, %2;" : "=f"(kv[4 * j4 + 2]), "=f"(kv[4 * j4 + 3]) : "l"(k23));
                    }
                    unsigned g = 0;
#pragma unroll
                    for (int j4 = 0; j4 < 4; ++j4) {
                        float m3, mn;
                        asm("min.f32 %0, %1, %2, %3;" : "=f"(m3) : "f"(kv[4 * j4]), "f"(kv[4 * j4 + 1]), "f"(kv[4 * j4 + 2]));
                        mn = fminf(m3, kv[4 * j4 + 3]);
                        g |= (unsigned)(mn < thr) << j4;
                    }
                    g = __reduce_or_sync(FULL, g);
                    if (g) {
#pragma unroll
                        for (int j4 = 0; j4 < 4; ++j4) {
                            if ((g >> j4) & 1u) {
#pragma unroll
                                for (int jj = 0; jj < 4; ++jj) {
                                    const int j = 4 * j4 + jj;
                                    const bool p = kv[j] < thr;
                                    if (p)
                                        reinterpret_cast<uint2 *>(mybuf)[cnt * TC_EPI] =
                                            make_uint2(col0 + c + j, __float_as_uint(kv[j]));
                                    cnt += p;
                                }
                            }
                        }
                        if (__any_sync(FULL, cnt > TC_BUF - 16)) flush();
                    }
                };
#pragma unroll 1
                for (int c = 0; c < TC_WG_COLS; c += 32) {
                    uint32_t v[32];
                    tmem_ld32_async(ta + c, v);
                    tmem_wait_ld(v);
                    scan16(reinterpret_cast<const uint32_t(&)[16]>(v[0]), c);
                    scan16(reinterpret_cast<const uint32_t(&)[16]>(v[16]), c + 16);
                }
            }
            fence_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(acc_empty + buf);
        }
        flush();
        // (the block's place is recomputed here rather than kept in registers
        // through the scan)
        const int64_t orow = (int64_t)blockIdx.x < full_blocks
                                 ? (int64_t)blockIdx.x * TC_ROWS + r
                                 : (full_blocks + ((int64_t)blockIdx.x - full_blocks) / parts) * TC_ROWS + r;
        if (orow < n) {
            // a part's lists go to the part area, to be merged per row
            const bool split = (int64_t)blockIdx.x >= full_blocks;
            const int64_t at = !split ? orow * TC_NCAND
                                      : ((orow - full_blocks * TC_ROWS) * parts +
                                         ((int64_t)blockIdx.x - full_blocks) % parts) * TC_NCAND;
            int32_t *ci = (split ? part_id : cand_id) + at + h * TC_CAND;
            float *ck = (split ? part_key : cand_key) + at + h * TC_CAND;
#pragma unroll
            for (int i = 0; i < TC_CAND; ++i) {
                // no candidates (and -inf keys): the FP32 pass takes the row
                ci[i] = ok && i < L ? id[i < L ? i : 0] : -1;
                ck[i] = !ok ? -__int_as_float(0x7f800000) : i < L ? key[i < L ? i : 0] : __int_as_float(0x7f800000);
            }
        }
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        fence_after_sync();
        tmem_dealloc(tmem, TC_NACC * TC_ACC_STRIDE);
    }
}

// The row blocks split into parts: one warp per (row, warpgroup list) merges
// the parts' sorted lists into the TC_CAND smallest keys, written where an
// unsplit row keeps its list.  Parts cover disjoint columns; a column left
// out has a key at least the merged last key (it lost the merge) or its own
// part's last key, which is at least the merged last key.  A part that gave
// up (ids -1, first key -inf) empties the row's list, so the FP32 pass takes
// the row.
__global__ void tc_merge_parts_kernel(int64_t n, int64_t row_begin, int parts, const int32_t *part_id,
                                      const float *part_key, int32_t *cand_id, float *cand_key) {
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t row = row_begin + w / TC_NWG;
    const int h = (int)(w % TC_NWG);
    if (row >= n) return;  // warp-uniform
    const float INF = __int_as_float(0x7f800000);
    const int64_t base = (row - row_begin) * parts;
    const int32_t *pid = part_id + (base + lane) * TC_NCAND + h * TC_CAND;
    const float *pkey = part_key + (base + lane) * TC_NCAND + h * TC_CAND;
    int pos = 0;
    int32_t hid = -1;
    float hkey = INF;
    bool failed = false;
    if (lane < parts) {
        hid = pid[0];
        hkey = pkey[0];
        failed = hid < 0 && hkey == -INF;
        if (hid < 0) hkey = INF;
    }
    failed = __any_sync(FULL, failed);
    int32_t my_id = -1;
    float my_key = INF;
#pragma unroll 1
    for (int i = 0; i < TC_CAND; ++i) {
        float m = hkey;
        int who = lane;
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) {
            const float om = __shfl_xor_sync(FULL, m, off);
            const int ow = __shfl_xor_sync(FULL, who, off);
            if (om < m || (om == m && ow < who)) {
                m = om;
                who = ow;
            }
        }
        const int32_t wid = __shfl_sync(FULL, hid, who);
        if (lane == i) {
            my_id = m < INF ? wid : -1;
            my_key = m;
        }
        if (lane == who && m < INF) {
            ++pos;
            hid = pos < TC_CAND ? pid[pos] : -1;
            hkey = hid >= 0 ? pkey[pos] : INF;
        }
    }
    if (lane < TC_CAND) {
        cand_id[row * TC_NCAND + h * TC_CAND + lane] = failed ? -1 : my_id;
        cand_key[row * TC_NCAND + h * TC_CAND + lane] = failed ? -INF : my_key;
    }
}

// Bound on |screened key - true key| for a row of norm xnorm (and FP32
// squared norm xn) against any column, whose norm is at most ymax:
// * split: x = hi + lo + e with |e| <= 2^-18 |x|, and the dropped lo.lo term,
//   leave at most 3 * 2^-18 |x_i| |y_i| per product; 4 * 2^-18 covers the
//   second-order terms;
// * accumulation: the BF16 products are exact in FP32; each of the 3 dpt
//   additions is taken to lose up to 2^-23 (truncation) of the running sum,
//   itself at most sum |x_i y_i| <= xnorm * ymax;
// * the key is -2 times the dot product plus a column norm with an FP32
//   error of (dpt + 2) 2^-24 ymax^2; the fma rounds once more.
// A factor of 2 on the whole covers the FP32 evaluation of the test itself.
__device__ __forceinline__ float screening_error(float xnorm, float xn, float ymax, int dpt) {
    const float dot = (4.0f * 0x1p-18f + 3.0f * dpt * 0x1p-23f) * xnorm * ymax;
    const float rest = (dpt + 4) * 0x1p-24f * (xn + 3.0f * ymax * ymax);
    return 2.0f * (2.0f * dot + rest);
}

// One warp per row: FP32 re-score of the 72 candidates, the k best written
// as the row's list, and the exactness test of the screening.  Rows that
// fail are appended to `redo`.
template <int DP>
__global__ void tc_rescore_kernel(const float *X, const float *norm2, const unsigned *norm_max, int64_t n, int k,
                                  int dpt, int lc, const int32_t *cand_id, const float *cand_key, int32_t *out_ids,
                                  float *out_d2, int32_t *redo, unsigned *redo_count) {
    using C = RowCfg<ST_FP32, DP>;
    const int lane = threadIdx.x & 31;
    const int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (u >= n) return;  // warp-uniform
    float qv[C::QF];
    load_query<ST_FP32, DP>(X + u * DP, qv);
    const RowSource src{reinterpret_cast<const uint8_t *>(X), nullptr};
    WarpTop<1> top;
    top.init(k);
    float thr = __int_as_float(0x7f800000);
#pragma unroll 1
    for (int h = 0; h < TC_NWG; ++h) {
        const int32_t cid = lane < TC_CAND ? cand_id[u * TC_NCAND + h * TC_CAND + lane] : -1;
        const int nc = __popc(__ballot_sync(FULL, cid >= 0));  // candidates fill a prefix
        const float d2 = gather_d2<ST_FP32, DP>(src, cid >= 0 ? (uint32_t)cid : 0u, nc, qv);
        for (int i = 0; i < nc; ++i)
            top.offer(pack_key(__shfl_sync(FULL, d2, i), (uint32_t)__shfl_sync(FULL, cid, i)));
        // a list's lc-th key: the screened keys of the columns left out are
        // at least the smallest of these (also for merged lists, which hold
        // every entry of their parts' lists of lc)
        thr = fminf(thr, cand_key[u * TC_NCAND + h * TC_CAND + lc - 1]);
    }
    if (lane < k) {
        const uint64_t key = top.e[0];
        out_ids[u * k + lane] = key == KEY_EMPTY ? -1 : (int32_t)key_id(key);
        out_d2[u * k + lane] = key == KEY_EMPTY ? __int_as_float(0x7f800000) : key_d2(key);
    }
    // Every column outside the candidates has a screened key >= thr, so a
    // true squared distance >= thr + ||x||^2 - E.  The k-th re-scored
    // distance (FP32, relative error below (DP + 2) 2^-24) must lie below.
    // A list whose screening gave up carries -inf: the row is redone.
    bool exact = false;
    if (thr > -__int_as_float(0x7f800000)) {
        const float dk = key_d2(top.entry(k - 1));
        const float xn = norm2[u];
        const float E = screening_error(sqrtf(xn), xn, __uint_as_float(*norm_max), dpt);
        exact = dk * (1.0f + (DP + 2) * 0x1p-23f) < thr + xn - E;
    }
    if (!exact && lane == 0) redo[atomicAdd(redo_count, 1u)] = (int32_t)u;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }();
    return fn;
}

// rows x dpt BF16 matrix, boxes of box_rows rows x 64 elements, 128-byte
// swizzle; rows past the end read as zeros
static bool bf16_rows_map(CUtensorMap *m, const void *ptr, int64_t rows, int dpt, int box_rows) {
    auto enc = tensor_map_encoder();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)dpt, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)dpt * 2};
    cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static int tc_width(int dp) { return dp <= 64 ? 64 : 128; }
static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

bool exact_tc_supported(int dp, int64_t n, int k, const uint32_t *removed) {
    return removed == nullptr && dp <= 128 && n >= TC_ROWS && n < (int64_t)INT32_MAX && k >= 1 &&
           k <= 32 && tensor_map_encoder() != nullptr;
}

// One CTA fits on an SM, so the row blocks run in waves of `sms` CTAs.  The
// row blocks of a last, partly filled wave are split into runs of column
// tiles, `parts` CTAs each, so that this wave ends about when a whole-row
// CTA would have done 1 / parts of its work.
constexpr int TC_SPLIT_MAX = 8;     // parts of one row block at most
constexpr int TC_SPLIT_CTAS = 256;  // CTAs of the split wave at most
struct TcPlan {
    int64_t full_blocks;  // row blocks taken whole, by CTAs 0 .. full_blocks-1
    int parts;            // CTAs per row block after those
    int64_t grid;
};
static TcPlan tc_plan(int64_t n, int sms) {
    const int64_t blocks = (n + TC_ROWS - 1) / TC_ROWS, tiles = (n + TC_COLS - 1) / TC_COLS;
    const int64_t rem = sms > 0 ? blocks % sms : 0;
    const int64_t parts =
        rem ? std::min(std::min<int64_t>(sms / rem, tiles), std::min<int64_t>(TC_SPLIT_MAX, TC_SPLIT_CTAS / rem)) : 1;
    if (parts < 2) return {blocks, 1, blocks};
    return {blocks - rem, (int)parts, blocks - rem + rem * parts};
}
// rows x parts of the split wave's lists, at most
static size_t tc_part_slots(int64_t n) {
    const int64_t blocks = (n + TC_ROWS - 1) / TC_ROWS;
    return (size_t)std::min<int64_t>(TC_SPLIT_CTAS, blocks * TC_SPLIT_MAX) * TC_ROWS;
}

// scratch, each part 256-byte aligned: hi, lo, norm2, cand_id, cand_key,
// redo, counters[16] = {norm max, redo count, wait error, ...}, partial
// lists of the FP32 pass, the split wave's part_id and part_key
size_t exact_tc_scratch_bytes(int64_t n, int dp) {
    const size_t dpt = tc_width(dp);
    const size_t n_pad = (size_t)(n + TC_COLS - 1) / TC_COLS * TC_COLS;
    return 2 * align256((size_t)n * dpt * 2) + align256(n_pad * 4) + 2 * align256((size_t)n * TC_NCAND * 4) +
           align256((size_t)n * 4) + 256 + align256((size_t)EXACT_PARTIAL_SLOTS * 32 * 8) +
           2 * align256(tc_part_slots(n) * TC_NCAND * 4);
}

static uint64_t g_tc_wait_ns = TC_WAIT;

void exact_tc_set_wait(int64_t ns) { g_tc_wait_ns = ns < 0 ? TC_WAIT : (uint64_t)ns; }

template <int NBOX, int L>
static cudaError_t tc_screen(const CUtensorMap &th, const CUtensorMap &tl, const CUtensorMap &tbh,
                             const CUtensorMap &tbl, const float *norm2, int64_t n, const TcPlan &plan,
                             int32_t *cid, float *ckey, int32_t *pid, float *pkey, unsigned *err, cudaStream_t s) {
    const size_t smem = TcCfg<NBOX>::SMEM;
    cudaError_t e =
        cudaFuncSetAttribute(exact_tc_kernel<NBOX, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    exact_tc_kernel<NBOX, L><<<(unsigned)plan.grid, TC_THREADS, smem, s>>>(
        th, tl, tbh, tbl, norm2, n, plan.full_blocks, plan.parts, cid, ckey, pid, pkey, err, g_tc_wait_ns);
    if ((e = cudaGetLastError()) != cudaSuccess || plan.parts < 2) return e;
    const int64_t row_begin = plan.full_blocks * TC_ROWS;
    const int64_t threads = (n - row_begin) * TC_NWG * 32;
    tc_merge_parts_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(n, row_begin, plan.parts, pid, pkey,
                                                                             cid, ckey);
    return cudaGetLastError();
}

template <int DP>
static cudaError_t tc_rescore(const ExactArgs &a, int dpt, int lc, const float *norm2, unsigned *counters,
                              const int32_t *cid, const float *ckey, int32_t *redo, cudaStream_t s) {
    const int64_t threads = a.n * 32;
    tc_rescore_kernel<DP><<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(
        a.X, norm2, counters, a.n, a.k, dpt, lc, cid, ckey, a.out_ids, a.out_d2, redo, counters + 1);
    return cudaGetLastError();
}

cudaError_t launch_exact_tc(int dp, const ExactArgs &a, void *scratch, unsigned **counters_out, cudaStream_t s) {
    const int dpt = tc_width(dp);
    uint8_t *p = static_cast<uint8_t *>(scratch);
    auto take = [&](size_t bytes) {
        uint8_t *q = p;
        p += align256(bytes);
        return q;
    };
    auto *hi = (__nv_bfloat16 *)take((size_t)a.n * dpt * 2);
    auto *lo = (__nv_bfloat16 *)take((size_t)a.n * dpt * 2);
    const int64_t n_pad = (a.n + TC_COLS - 1) / TC_COLS * TC_COLS;
    auto *norm2 = (float *)take((size_t)n_pad * 4);
    auto *cid = (int32_t *)take((size_t)a.n * TC_NCAND * 4);
    auto *ckey = (float *)take((size_t)a.n * TC_NCAND * 4);
    auto *redo = (int32_t *)take((size_t)a.n * 4);
    auto *counters = (unsigned *)take(64);
    auto *partial = (uint64_t *)take((size_t)EXACT_PARTIAL_SLOTS * 32 * 8);
    auto *pid = (int32_t *)take(tc_part_slots(a.n) * TC_NCAND * 4);
    auto *pkey = (float *)take(tc_part_slots(a.n) * TC_NCAND * 4);
    *counters_out = counters;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const TcPlan plan = tc_plan(a.n, sms);
    // the CTA's rows in 128-row boxes, the column tiles in TC_COLS-row boxes
    CUtensorMap th, tl, tbh, tbl;
    if (!bf16_rows_map(&th, hi, a.n, dpt, TC_ROWS) || !bf16_rows_map(&tl, lo, a.n, dpt, TC_ROWS) ||
        !bf16_rows_map(&tbh, hi, a.n, dpt, TC_COLS) || !bf16_rows_map(&tbl, lo, a.n, dpt, TC_COLS))
        return cudaErrorNotSupported;
    e = cudaMemsetAsync(counters, 0, 64, s);
    if (e != cudaSuccess) return e;
    tc_split_kernel<<<(unsigned)((n_pad * 32 + 255) / 256), 256, 0, s>>>(a.X, a.n, n_pad, dp, dpt, hi, lo,
                                                                          norm2, counters);
    // shorter lists for small k: fewer appends and cheaper merges, while the
    // k-th distance still lies well inside the candidates
    const int lc = a.k <= TC_SMALL_K ? TC_CAND_SMALL_K : TC_CAND;
    if (dpt == 64)
        e = lc == TC_CAND ? tc_screen<1, TC_CAND>(th, tl, tbh, tbl, norm2, a.n, plan, cid, ckey, pid, pkey,
                                                  counters + 2, s)
                          : tc_screen<1, TC_CAND_SMALL_K>(th, tl, tbh, tbl, norm2, a.n, plan, cid, ckey, pid, pkey,
                                                          counters + 2, s);
    else
        e = lc == TC_CAND ? tc_screen<2, TC_CAND>(th, tl, tbh, tbl, norm2, a.n, plan, cid, ckey, pid, pkey,
                                                  counters + 2, s)
                          : tc_screen<2, TC_CAND_SMALL_K>(th, tl, tbh, tbl, norm2, a.n, plan, cid, ckey, pid, pkey,
                                                          counters + 2, s);
    if (e != cudaSuccess) return e;
    switch (dp) {
        case 16: e = tc_rescore<16>(a, dpt, lc, norm2, counters, cid, ckey, redo, s); break;
        case 32: e = tc_rescore<32>(a, dpt, lc, norm2, counters, cid, ckey, redo, s); break;
        case 64: e = tc_rescore<64>(a, dpt, lc, norm2, counters, cid, ckey, redo, s); break;
        case 96: e = tc_rescore<96>(a, dpt, lc, norm2, counters, cid, ckey, redo, s); break;
        case 128: e = tc_rescore<128>(a, dpt, lc, norm2, counters, cid, ckey, redo, s); break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    // the rows the screening could not settle, against every column in FP32;
    // their number decides how the columns are split
    unsigned nredo = 0;
    e = cudaMemcpyAsync(&nredo, counters + 1, sizeof nredo, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess || nredo == 0) return e;
    ExactArgs rest = a;
    rest.rows = redo;
    rest.row_count = counters + 1;
    rest.col_segments = exact_col_segments(nredo, a.n, sms);
    rest.row_hint = nredo;
    rest.partial = partial;
    return launch_exact(dp, rest, s);
}

}  // namespace knn
