// noalloc.cu -- knn_search_noalloc: the iGNNS query search over a graph the
// caller holds in its own device buffers, with every temporary taken from a
// fixed array that is part of the library image instead of from cudaMalloc.
//
// Who needs it: a caller whose device memory is already owned by another
// allocator (a framework's caching pool, a serving process that reserves
// its whole memory budget up front) cannot ask the driver for more, and a
// caller on a latency-critical loop may not afford the device-wide
// synchronisation a cudaMalloc/cudaFree pair can cause.  Such callers can
// hold the graph themselves and still run the search.
//
// The scratch array below is the only memory the call uses besides the
// caller's buffers.  Every GPU that loads this library keeps the array for
// the life of the process.  All calls share it, so two calls whose work
// overlaps on a GPU (different streams, or different host threads without
// ordering) race on it; a call clears the parts that must start at zero
// (visited sets, removal bits, totals) and overwrites the rest.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <mutex>

#include "knn_graph.h"
#include "kernels.h"

using namespace knn;

namespace {

constexpr size_t kScratchBytes = (size_t)16 << 20;  // 16 MiB per GPU
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char knn_noalloc_scratch[kScratchBytes];

std::mutex g_setup_mutex;
void *g_scratch_addr[kMaxDevices] = {};

size_t round_up(size_t v) { return (v + 255) & ~(size_t)255; }

// Device (or managed) memory of `device`: another GPU's memory would be read
// over the interconnect, or fault, so it is refused like host memory.
bool on_device(const void *p, int device) {
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged) &&
           attr.device == device;
}

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

knn_status reject(knn_status st, const char *fmt, ...) {
    char buf[400];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return knn::record_error(st, buf);
}

// Device address of the scratch array on the current device.  The name of a
// __device__ array in host code is only a host-side stand-in, so the address
// is asked from the runtime once per device, with that device current.
knn_status scratch_on(int device, unsigned char **out) {
    if (device < 0 || device >= kMaxDevices) return reject(KNN_ERR_UNSUPPORTED, "device %d", device);
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, knn_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return reject(KNN_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed: %s",
                          cudaGetErrorString(e));
        g_scratch_addr[device] = p;
    }
    *out = static_cast<unsigned char *>(g_scratch_addr[device]);
    return KNN_OK;
}

}  // namespace

extern "C" KNN_API knn_status knn_search_noalloc(const float *rows, int64_t n, int32_t dim,
                                                 const int32_t *nbr_ids, int32_t k,
                                                 const float *queries, int64_t m, int32_t k_out,
                                                 double speedup, double expansion, uint64_t seed,
                                                 uint64_t query_id0, int64_t *out_ids,
                                                 float *out_sims, void *stream) {
    if (!rows || !nbr_ids || !queries || !out_ids) return reject(KNN_ERR_INVALID_ARG, "null argument");
    if (!(dim == 16 || dim == 32 || dim == 64 || dim == 96 || dim == 128 || dim == 256))
        return reject(KNN_ERR_UNSUPPORTED, "dim %d: must be 16, 32, 64, 96, 128 or 256", dim);
    if (k < 1 || k > 32) return reject(KNN_ERR_UNSUPPORTED, "k %d outside 1..32", k);
    if (k_out < 1 || k_out > k) return reject(KNN_ERR_INVALID_ARG, "k_out outside 1..k");
    if (n < k + 1 || n >= (int64_t)INT32_MAX) return reject(KNN_ERR_INVALID_ARG, "need k+1 <= n < 2^31");
    if (m < 1 || m > INT32_MAX) return reject(KNN_ERR_INVALID_ARG, "m must be >= 1");
    if (!(speedup > 0.0) || !std::isfinite(speedup)) return reject(KNN_ERR_INVALID_ARG, "bad speedup");
    if (std::isnan(expansion)) return reject(KNN_ERR_INVALID_ARG, "expansion is NaN");
    // rows and queries are read with 16-byte vector loads, lists and outputs
    // with loads and stores of their element size (checked before any CUDA
    // call: a misaligned vector load would fault the kernel)
    if (!aligned(rows, 16) || !aligned(queries, 16))
        return reject(KNN_ERR_INVALID_ARG, "rows and queries must start on a 16-byte boundary");
    if (!aligned(nbr_ids, 4) || !aligned(out_ids, 8) || (out_sims && !aligned(out_sims, 4)))
        return reject(KNN_ERR_INVALID_ARG, "nbr_ids, out_ids and out_sims must be aligned to "
                                           "their element size");
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) {
        cudaGetLastError();
        return reject(KNN_ERR_CUDA, "no CUDA device");
    }
    if (!on_device(rows, device) || !on_device(nbr_ids, device) || !on_device(queries, device) ||
        !on_device(out_ids, device) || (out_sims && !on_device(out_sims, device)))
        return reject(KNN_ERR_INVALID_ARG,
                      "every buffer must be device memory of the current device (nothing is staged)");

    // scratch layout: result keys, counters, totals, removal bits, visited
    // sets (these only when they do not fit in shared memory)
    const size_t words = (size_t)((n + 31) / 32);
    const bool vis_off_chip = !search_visited_on_chip((uint32_t)n);
    const size_t off_keys = 0;
    const size_t off_ctr = off_keys + round_up((size_t)m * k_out * sizeof(uint64_t));
    const size_t off_tot = off_ctr + round_up((size_t)m * NCTR * sizeof(long long));
    const size_t off_rem = off_tot + round_up(NTOT * sizeof(unsigned long long));
    const size_t off_vis = off_rem + round_up(words * sizeof(uint32_t));
    const size_t need = off_vis + (vis_off_chip ? round_up((size_t)m * words * sizeof(uint32_t)) : 0);
    if (need > kScratchBytes)
        return reject(KNN_ERR_CAPACITY,
                      "m = %lld queries over n = %lld nodes need %zu bytes of scratch; the fixed "
                      "array holds %zu (about m * n / 8 bytes are needed once n exceeds the "
                      "on-chip visited sets): use fewer queries per call",
                      (long long)m, (long long)n, need, kScratchBytes);

    unsigned char *scratch = nullptr;
    knn_status st = scratch_on(device, &scratch);
    if (st != KNN_OK) return st;

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint64_t *keys = reinterpret_cast<uint64_t *>(scratch + off_keys);
    long long *counters = reinterpret_cast<long long *>(scratch + off_ctr);
    unsigned long long *totals = reinterpret_cast<unsigned long long *>(scratch + off_tot);
    uint32_t *removed = reinterpret_cast<uint32_t *>(scratch + off_rem);
    uint32_t *visited = vis_off_chip ? reinterpret_cast<uint32_t *>(scratch + off_vis) : nullptr;
    cudaError_t e = cudaMemsetAsync(scratch + off_tot, 0, need - off_tot, s);
    if (e != cudaSuccess) return reject(KNN_ERR_CUDA, "clearing the scratch failed: %s", cudaGetErrorString(e));

    SearchArgs a{};
    a.rows = reinterpret_cast<const uint8_t *>(rows);
    a.row_scale = nullptr;
    a.nbr = nbr_ids;
    a.removed = removed;
    a.queries = queries;
    a.q_stride = dim;
    a.visited = visited;
    a.vwords = (int64_t)words;
    a.out_keys = keys;
    a.counters = counters;
    a.totals = totals;
    a.m = (int32_t)m;
    a.k = k;
    a.KT = k_out;
    a.n = (uint32_t)n;
    a.n_live = n;
    const double b = std::floor((double)n / speedup);
    a.budget = b < 1.0 ? 1 : (int64_t)b;
    a.max_draws = 64ull * (uint64_t)n;
    a.seed = seed;
    a.stream_base = (1ull << 63) + query_id0;
    a.discard = (expansion > 0.0 && std::isfinite(expansion)) ? 1 : 0;
    a.expansion = a.discard ? (float)expansion : 1.0f;
    a.vis_n = (uint32_t)n;
    a.speedup = speedup;
    e = launch_search(KNN_STORAGE_FP32, dim, a, s);
    if (e == cudaSuccess) e = launch_keys_to_output(keys, m, k_out, k_out, out_ids, out_sims, s);
    if (e != cudaSuccess) return reject(KNN_ERR_CUDA, "launch failed: %s", cudaGetErrorString(e));
    return KNN_OK;
}
