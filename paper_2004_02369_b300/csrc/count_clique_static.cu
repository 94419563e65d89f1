// k-clique counting without any device allocation.
//
// For callers that must not allocate device memory while they count: a
// process whose device memory is reserved up front by another allocator (a
// framework's caching allocator or a fixed pool), where a cudaMalloc at query
// time can fail or fragment that pool, and latency-bound callers that cannot
// afford the implicit device synchronisation of cudaMalloc / cudaFree.  The
// regular entry points grow a graph-owned scratch arena with cudaMalloc; this
// one runs the same clique kernel on a fixed scratch array that is part of
// the library image instead.
#include <mutex>

#include "pg_internal.h"

// Every device that loads libpg holds this array until the process exits.
static __device__ __align__(256) unsigned char g_pg_static_scratch[PG_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
constexpr size_t kQueueBytes = 256; // work-queue counters, padded to keep slabs aligned

std::mutex g_mu;
void *g_base[kMaxDevices] = {};

// Device address of the array on the current device, resolved once per device.
int static_scratch_base(int dev, void **out) {
    if (dev < 0 || dev >= kMaxDevices) return pg_set_error(PG_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_base[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_pg_static_scratch);
        if (e != cudaSuccess) return pg_cuda_error(e, "cudaGetSymbolAddress(static scratch)");
        g_base[dev] = p;
    }
    *out = g_base[dev];
    return PG_OK;
}

}  // namespace

extern "C" int pg_count_cliques_noalloc(pg_graph *g, int32_t kmin, int32_t kmax, uint64_t *counts_dev,
                                        void *stream) {
    if (!g || !counts_dev) return pg_set_error(PG_EINVAL, "NULL argument");
    if (kmin < 3 || kmax > PG_MAX_PATTERN || kmin > kmax)
        return pg_set_error(PG_EINVAL, "clique sizes must satisfy 3 <= kmin <= kmax <= 8");
    int dev = -1;
    PG_CUDA(cudaGetDevice(&dev));
    if (dev != g->device) return pg_set_error(PG_EINVAL, "the graph lives on another device than the current one");
    const size_t slab = pg_clique_slab_bytes(g, kmax);
    const size_t room = PG_STATIC_SCRATCH_BYTES - kQueueBytes;
    long long max_slabs = slab ? (long long)(room / slab) : (1ll << 40);
    if (slab && max_slabs < g->num_sms)
        return pg_set_error(PG_EINVAL,
                            "graph too large for the static scratch: its maximum out-degree " +
                                std::to_string(g->max_out) + " needs " + std::to_string(slab) +
                                " bytes per block, and the " + std::to_string(PG_STATIC_SCRATCH_BYTES >> 20) +
                                " MiB array holds fewer than one block per SM");
    void *base = nullptr;
    int rc = static_scratch_base(dev, &base);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    // the output and the queue counters (zeroed by the launcher) start at
    // zero; slab contents left by an earlier call are overwritten before
    // they are read
    PG_CUDA(cudaMemsetAsync(counts_dev, 0, 2 * sizeof(uint64_t) * (size_t)(kmax - kmin + 1), s));
    return pg_launch_clique_on(g, kmin, kmax, (unsigned long long *)counts_dev, (unsigned long long *)base,
                               (unsigned char *)base + kQueueBytes, max_slabs, s);
}
