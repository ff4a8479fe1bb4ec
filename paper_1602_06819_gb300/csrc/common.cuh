// common.cuh -- device helpers shared by the kernels of the online k-nn graph
// library: the restart generator, the packed (distance, id) order, warp-level
// top lists, and the row-gather distance engine used by every kernel that
// compares a query with stored rows.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <stdint.h>

namespace knn {

constexpr unsigned FULL = 0xffffffffu;
constexpr uint64_t KEY_EMPTY = ~0ull;

enum Storage : int { ST_FP32 = 0, ST_BF16 = 1, ST_FP8 = 2 };

// ---------------------------------------------------------------------------
// Restart draws (Sec. 3: "selects a random node").  SplitMix64 (Steele, Lea
// and Flood, OOPSLA 2014): output j of the generator seeded with s is
// fin(s + (j+1) * gamma).  A search keyed by (seed, stream) uses the
// generator seeded with h = mix(seed ^ mix(stream)), mix(v) = output 0 of
// the generator seeded with v; draw j picks node floor(x_j * n / 2^64)
// (Lemire's multiply-shift range reduction).
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint64_t splitmix_fin(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ uint64_t splitmix_out(uint64_t seed, uint64_t j) {
    return splitmix_fin(seed + (j + 1ull) * 0x9E3779B97F4A7C15ull);
}
__host__ __device__ __forceinline__ uint64_t restart_key(uint64_t seed, uint64_t stream) {
    return splitmix_out(seed ^ splitmix_out(stream, 0), 0);
}
__host__ __device__ __forceinline__ uint32_t restart_node(uint64_t key, uint64_t j, uint32_t n) {
#ifdef __CUDA_ARCH__
    return (uint32_t)__umul64hi(splitmix_out(key, j), (uint64_t)n);
#else
    return (uint32_t)(((unsigned __int128)splitmix_out(key, j) * (uint64_t)n) >> 64);
#endif
}

// ---------------------------------------------------------------------------
// Order of candidates.  sim = 1/(1+dist) is decreasing in the squared
// distance, so "higher similarity, then lower id" is "smaller squared
// distance, then lower id": one unsigned compare of
// (float bits of d2) << 32 | id, since d2 >= 0.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t pack_key(float d2, uint32_t id) {
    return ((uint64_t)__float_as_uint(d2) << 32) | (uint64_t)id;
}
__device__ __forceinline__ uint32_t key_id(uint64_t key) { return (uint32_t)key; }
__device__ __forceinline__ float key_d2(uint64_t key) { return __uint_as_float((uint32_t)(key >> 32)); }

__device__ __forceinline__ float sim_of_d2(float d2) { return 1.0f / (1.0f + sqrtf(d2)); }

__device__ __forceinline__ uint64_t shfl_u64(uint64_t v, int src) {
    uint32_t lo = __shfl_sync(FULL, (uint32_t)v, src);
    uint32_t hi = __shfl_sync(FULL, (uint32_t)(v >> 32), src);
    return ((uint64_t)hi << 32) | lo;
}
__device__ __forceinline__ uint64_t shfl_u64_xor(uint64_t v, int mask = 1) {
    uint32_t lo = __shfl_xor_sync(FULL, (uint32_t)v, mask);
    uint32_t hi = __shfl_xor_sync(FULL, (uint32_t)(v >> 32), mask);
    return ((uint64_t)hi << 32) | lo;
}
__device__ __forceinline__ uint64_t shfl_up_u64(uint64_t v, int delta) {
    uint32_t lo = __shfl_up_sync(FULL, (uint32_t)v, delta);
    uint32_t hi = __shfl_up_sync(FULL, (uint32_t)(v >> 32), delta);
    return ((uint64_t)hi << 32) | lo;
}

// ---------------------------------------------------------------------------
// A sorted list of the best T*32 keys held by one warp: entry t*32 + lane in
// register e[t].  `limit` entries are meaningful; the threshold a candidate
// must beat is entry limit-1.  Every lane calls every method (warp-uniform).
// ---------------------------------------------------------------------------
template <int T>
struct WarpTop {
    uint64_t e[T];
    uint64_t worst;  // entry limit-1 (KEY_EMPTY while the list is short)
    int limit;

    __device__ __forceinline__ void init(int lim) {
#pragma unroll
        for (int t = 0; t < T; ++t) e[t] = KEY_EMPTY;
        worst = KEY_EMPTY;
        limit = lim;
    }
    __device__ __forceinline__ uint64_t entry(int idx) const {  // warp-uniform idx
        uint64_t v = KEY_EMPTY;
#pragma unroll
        for (int t = 0; t < T; ++t)
            if (t == (idx >> 5)) v = e[t];
        return shfl_u64(v, idx & 31);
    }
    // Insert `key` (warp-uniform) if it beats the threshold.  Keys are unique.
    __device__ __forceinline__ bool offer(uint64_t key) {
        if (!(key < worst)) return false;
        const int lane = threadIdx.x & 31;
        int pos = 0;
#pragma unroll
        for (int t = 0; t < T; ++t) pos += __popc(__ballot_sync(FULL, e[t] < key));
        uint64_t prev[T];
#pragma unroll
        for (int t = 0; t < T; ++t) {
            uint64_t up = shfl_up_u64(e[t], 1);
            if (t > 0) {
                uint64_t carry = shfl_u64(e[t - 1], 31);
                if (lane == 0) up = carry;
            }
            prev[t] = up;
        }
#pragma unroll
        for (int t = 0; t < T; ++t) {
            int idx = t * 32 + lane;
            if (idx == pos) e[t] = key;
            else if (idx > pos) e[t] = prev[t];
        }
        worst = entry(limit - 1);
        return true;
    }
};

// ---------------------------------------------------------------------------
// Row gathers.  A stored row is DP elements (the dimension padded with zeros
// to a multiple of 16) in one of three encodings.  A group of G lanes reads
// one row with 16-byte loads: lane i of the group takes chunks i, i+G, ...,
// so each load instruction of the group covers G*16 contiguous bytes.  RPP =
// 32/G rows are read per pass and P passes are kept in flight.
//
// FP32 arithmetic: FP32 and BF16 rows keep four running sums per lane (two
// packed FP32 pairs), each adding every fourth of the lane's e = CPL*E
// squared differences with fused multiply-adds; the lane then adds its four
// sums in two levels and the group adds its partial sums in a log2(G)-level
// butterfly.  With the rounding of each difference, the relative error of a
// squared distance is at most about (e/4 + log2(G) + 4) units of 2^-24.  FP8
// rows keep one running sum in element order: (e + log2(G) + 5) units, the
// product with the row scale included.
// ---------------------------------------------------------------------------
template <int STORAGE, int DP>
struct RowCfg {
    static constexpr int E = STORAGE == ST_FP32 ? 4 : STORAGE == ST_BF16 ? 8 : 16;
    static constexpr int NC = DP / E;  // 16-byte chunks per row
    static constexpr int G = (NC % 8 == 0) ? 8 : (NC % 4 == 0) ? 4 : (NC % 2 == 0) ? 2 : 1;
    static constexpr int CPL = NC / G;
    static constexpr int RPP = 32 / G;
    static constexpr int QF = CPL * E;  // query floats held by a lane
    // passes in flight: up to 32 chunk loads per lane, at most 32 rows
    static constexpr int P_LOADS = 32 / CPL > 1 ? 32 / CPL : 1;
    static constexpr int P = P_LOADS < 32 / RPP ? P_LOADS : 32 / RPP;
    static constexpr int ROW_BYTES = STORAGE == ST_FP32 ? DP * 4 : STORAGE == ST_BF16 ? DP * 2 : DP;
    static_assert(DP % 16 == 0, "rows are padded to 16 elements");
    static_assert(NC % G == 0, "bad lane grouping");
};

struct RowSource {
    const uint8_t *rows;     // row r starts at rows + r * row_bytes
    const float *scale;      // FP8 rows: per-row scale (else unused)
};

// Load this lane's slice of the query (a padded FP32 row) into registers.
template <int STORAGE, int DP>
__device__ __forceinline__ void load_query(const float *q, float (&qv)[RowCfg<STORAGE, DP>::QF]) {
    using C = RowCfg<STORAGE, DP>;
    const int gi = (threadIdx.x & 31) % C::G;
#pragma unroll
    for (int c = 0; c < C::CPL; ++c) {
        const int ch = gi + c * C::G;  // chunk index within the row
#pragma unroll
        for (int v = 0; v < C::E / 4; ++v) {
            float4 f = *reinterpret_cast<const float4 *>(q + ch * C::E + v * 4);
            qv[c * C::E + v * 4 + 0] = f.x;
            qv[c * C::E + v * 4 + 1] = f.y;
            qv[c * C::E + v * 4 + 2] = f.z;
            qv[c * C::E + v * 4 + 3] = f.w;
        }
    }
}

// Global loads as volatile asm: volatile asm statements keep their program
// order, so loads placed early are issued early even under register
// pressure, and the round trips of independent loads overlap.
__device__ __forceinline__ uint4 ld_nc_v4(const void *p) {
    uint4 v;
    asm volatile("ld.global.nc.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
    return v;
}
__device__ __forceinline__ uint32_t ld_nc_u32(const void *p) {
    uint32_t v;
    asm volatile("ld.global.nc.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
// L2-coherent load (bypasses L1): sees atomics other lanes made at L2
__device__ __forceinline__ uint32_t ld_cg_u32(const void *p) {
    uint32_t v;
    asm volatile("ld.global.cg.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

__device__ __forceinline__ float bf16_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }

__device__ __forceinline__ float2 e4m3x2_to_float2(uint16_t pair) {
    __half2_raw h = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)pair, __NV_E4M3);
    return __half22float2(*reinterpret_cast<__half2 *>(&h));
}

// Partial squared distance of one 16-byte chunk against query floats qv[0..E).
template <int STORAGE>
__device__ __forceinline__ float chunk_d2(uint4 w, const float *qv, float scale, float acc) {
    if constexpr (STORAGE == ST_FP32) {
        float d;
        d = qv[0] - __uint_as_float(w.x); acc = fmaf(d, d, acc);
        d = qv[1] - __uint_as_float(w.y); acc = fmaf(d, d, acc);
        d = qv[2] - __uint_as_float(w.z); acc = fmaf(d, d, acc);
        d = qv[3] - __uint_as_float(w.w); acc = fmaf(d, d, acc);
    } else if constexpr (STORAGE == ST_BF16) {
        const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float d;
            d = qv[2 * i] - bf16_lo(ws[i]); acc = fmaf(d, d, acc);
            d = qv[2 * i + 1] - bf16_hi(ws[i]); acc = fmaf(d, d, acc);
        }
    } else {
        const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float2 a = e4m3x2_to_float2((uint16_t)(ws[i] & 0xffffu));
            float2 b = e4m3x2_to_float2((uint16_t)(ws[i] >> 16));
            // the stored value is binary32(code * scale): round the product
            // before the difference so that no fused operation skips it
            float d;
            d = qv[4 * i + 0] - __fmul_rn(a.x, scale); acc = fmaf(d, d, acc);
            d = qv[4 * i + 1] - __fmul_rn(a.y, scale); acc = fmaf(d, d, acc);
            d = qv[4 * i + 2] - __fmul_rn(b.x, scale); acc = fmaf(d, d, acc);
            d = qv[4 * i + 3] - __fmul_rn(b.y, scale); acc = fmaf(d, d, acc);
        }
    }
    return acc;
}

// Packed FP32 pairs (sm_100 and later): each half is an IEEE binary32
// operation rounded to nearest, two per instruction.
__device__ __forceinline__ unsigned long long f32x2_pack(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
// acc + (q - x)^2 on both halves, the difference rounded before the fma
__device__ __forceinline__ unsigned long long f32x2_sqdiff_acc(unsigned long long q, unsigned long long x,
                                                               unsigned long long acc) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(q), "l"(x));
    asm("fma.rn.f32x2 %0, %1, %1, %2;" : "=l"(acc) : "l"(d), "l"(acc));
    return acc;
}
// (a.lo + b.lo) + (a.hi + b.hi)
__device__ __forceinline__ float f32x2_total(unsigned long long a, unsigned long long b) {
    unsigned long long s;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(s) : "l"(a), "l"(b));
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(s));
    return lo + hi;
}

// A lane's partial squared distance over its chunks of one row.
template <int STORAGE>
struct RowAcc {
    float acc = 0.0f;
    __device__ __forceinline__ void add(uint4 w, const float *qv, float scale) {
        acc = chunk_d2<STORAGE>(w, qv, scale, acc);
    }
    __device__ __forceinline__ float total() const { return acc; }
};
template <>
struct RowAcc<ST_FP32> {
    unsigned long long a = 0ull, b = 0ull;  // +0.0f in both halves
    __device__ __forceinline__ void add(uint4 w, const float *qv, float) {
        a = f32x2_sqdiff_acc(f32x2_pack(qv[0], qv[1]), f32x2_pack(__uint_as_float(w.x), __uint_as_float(w.y)), a);
        b = f32x2_sqdiff_acc(f32x2_pack(qv[2], qv[3]), f32x2_pack(__uint_as_float(w.z), __uint_as_float(w.w)), b);
    }
    __device__ __forceinline__ float total() const { return f32x2_total(a, b); }
};
template <>
struct RowAcc<ST_BF16> {
    unsigned long long a = 0ull, b = 0ull;
    __device__ __forceinline__ void add(uint4 w, const float *qv, float) {
        a = f32x2_sqdiff_acc(f32x2_pack(qv[0], qv[1]), f32x2_pack(bf16_lo(w.x), bf16_hi(w.x)), a);
        b = f32x2_sqdiff_acc(f32x2_pack(qv[2], qv[3]), f32x2_pack(bf16_lo(w.y), bf16_hi(w.y)), b);
        a = f32x2_sqdiff_acc(f32x2_pack(qv[4], qv[5]), f32x2_pack(bf16_lo(w.z), bf16_hi(w.z)), a);
        b = f32x2_sqdiff_acc(f32x2_pack(qv[6], qv[7]), f32x2_pack(bf16_lo(w.w), bf16_hi(w.w)), b);
    }
    __device__ __forceinline__ float total() const { return f32x2_total(a, b); }
};

// A row gather split in two: issue() starts the loads of the first chunk of
// every lane's share of up to 32 rows (the first G * 16 bytes of each row;
// lane c < nrows holds row id rid) and reduce() waits for them, leaving in
// lane c the sum of row c's squared differences over those elements,
// accumulated as gather_d2 starts its sum.  Work placed between the two calls
// overlaps with the loads.  Every step of that sum adds a nonnegative value
// and FP32 rounding is monotone, so the partial sum never exceeds the full
// squared distance gather_d2 computes for the same row.
template <int STORAGE, int DP>
struct RowGatherHead {
    using C = RowCfg<STORAGE, DP>;
    static constexpr int P = 32 / C::RPP;
    uint4 buf[P];
    float scl[P];

    // Every pass loads (a group past the last row re-reads the row of lane
    // 0, whose rid must be a valid row even for nrows = 0; the result is
    // dropped), so that reduce() runs straight through and the arithmetic of
    // the passes interleaves.
    __device__ __forceinline__ void issue(const RowSource &src, uint32_t rid, int nrows) {
        const int lane = threadIdx.x & 31;
        const int gl = lane / C::G, gi = lane % C::G;
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const int c = p * C::RPP + gl;
            const uint32_t row = __shfl_sync(FULL, rid, c < nrows ? (c & 31) : 0);
            buf[p] = ld_nc_v4(reinterpret_cast<const uint4 *>(src.rows + (size_t)row * C::ROW_BYTES) + gi);
            scl[p] = STORAGE == ST_FP8 ? __uint_as_float(ld_nc_u32(src.scale + row)) : 1.0f;
        }
    }

    __device__ __forceinline__ float reduce(int nrows, const float (&qv)[C::QF]) const {
        const int lane = threadIdx.x & 31;
        float result = __int_as_float(0x7f800000);
#pragma unroll
        for (int p = 0; p < P; ++p) {
            RowAcc<STORAGE> ra;
            ra.add(buf[p], qv, scl[p]);
            float acc = ra.total();
#pragma unroll
            for (int off = C::G / 2; off >= 1; off >>= 1) acc += __shfl_xor_sync(FULL, acc, off);
            const int c = lane - p * C::RPP;
            const float got = __shfl_sync(FULL, acc, ((lane % C::RPP) * C::G) & 31);
            if (c >= 0 && c < C::RPP && lane < nrows) result = got;
        }
        return result;
    }
};

__device__ __forceinline__ void prefetch_l1(const void *p) {
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// The row layout with passes for MAX_ROWS rows (rounded up to whole passes)
// in flight.
template <int STORAGE, int DP, int MAX_ROWS>
struct GatherCfg : RowCfg<STORAGE, DP> {
    using C0 = RowCfg<STORAGE, DP>;
    static constexpr int NEED = (MAX_ROWS + C0::RPP - 1) / C0::RPP;
    static constexpr int P = NEED < C0::P ? NEED : C0::P;
};

// MAX_ROWS bounds the rows in flight at once (and the registers they take).
// Lane c < nrows holds the id of row c, or GATHER_SKIP for a row that is not
// loaded (its result is meaningless).
constexpr uint32_t GATHER_SKIP = 0xffffffffu;
template <int STORAGE, int DP, int MAX_ROWS = 32>
__device__ __forceinline__ float gather_d2(const RowSource &src, uint32_t rid, int nrows,
                                           const float (&qv)[RowCfg<STORAGE, DP>::QF]) {
    using C = GatherCfg<STORAGE, DP, MAX_ROWS>;
    const int lane = threadIdx.x & 31;
    const int gl = lane / C::G, gi = lane % C::G;
    float result = __int_as_float(0x7f800000);
    for (int p0 = 0; p0 * C::RPP < nrows; p0 += C::P) {
        uint4 buf[C::P][C::CPL];
        float scl[C::P];
#pragma unroll
        for (int p = 0; p < C::P; ++p) {
            const int c = (p0 + p) * C::RPP + gl;
            const uint32_t row = __shfl_sync(FULL, rid, c & 31);
            const bool act = c < nrows && row != GATHER_SKIP;
            const uint4 *base = reinterpret_cast<const uint4 *>(src.rows + (size_t)row * C::ROW_BYTES);
#pragma unroll
            for (int k = 0; k < C::CPL; ++k) {
                buf[p][k] = make_uint4(0, 0, 0, 0);
                if (act) buf[p][k] = ld_nc_v4(base + gi + k * C::G);
            }
            scl[p] = 1.0f;
            if (STORAGE == ST_FP8 && act) scl[p] = __uint_as_float(ld_nc_u32(src.scale + row));
        }
#pragma unroll
        for (int p = 0; p < C::P; ++p) {
            // a gather sized to its rows (MAX_ROWS < 32) reduces every pass,
            // straight through (passes without rows hold zeros)
            if (MAX_ROWS >= 32 && (p0 + p) * C::RPP >= nrows) break;  // warp-uniform
            RowAcc<STORAGE> ra;
#pragma unroll
            for (int k = 0; k < C::CPL; ++k) ra.add(buf[p][k], qv + k * C::E, scl[p]);
            float acc = ra.total();
#pragma unroll
            for (int off = C::G / 2; off >= 1; off >>= 1) acc += __shfl_xor_sync(FULL, acc, off);
            // row c = (p0+p)*RPP + g is held by the lanes of group g
            const int c = lane - (p0 + p) * C::RPP;
            const float got = __shfl_sync(FULL, acc, ((lane % C::RPP) * C::G) & 31);
            if (c >= 0 && c < C::RPP && lane < nrows) result = got;
        }
    }
    return result;
}

}  // namespace knn
