// Graph residency: validation, degree ranking and CSR rewrite on the device.
//
// Section 5.5: the data graph is kept as sorted adjacency lists.
// Section 5.2: vertices are ordered by degree so that, matched high-to-low,
// a high-degree start vertex only extends to its few higher-ranked
// neighbours.  Rank = position in (degree descending, original id
// ascending); a smaller rank means a higher degree.
//
// Sorting uses CUB (header library shipped with the CUDA toolkit) radix sort
// and scan: this runs once per graph load, outside the matching path.
#include <cub/cub.cuh>

#include <vector>

#include "pg_internal.h"

namespace {

constexpr int kBlock = 256;

// Per-vertex validation before the build: ids in range, no loop, strictly
// ascending lists, labels >= 0.  err bit 1: range, 2: loop, 4: order,
// 16: negative label.  Symmetry is checked by k_symmetric on the ranked
// lists.
__global__ void k_validate(const int64_t *off, const int32_t *adj, const int32_t *labels, int64_t n,
                           unsigned *err) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (gridDim.x * (int64_t)blockDim.x) >> 5;
    for (int64_t u = warp; u < n; u += nwarps) {
        const int64_t b = off[u], e = off[u + 1];
        unsigned bad = 0;
        if (lane == 0 && labels && labels[u] < 0) bad |= 16;
        for (int64_t i = b + lane; i < e; i += 32) {
            const int32_t x = adj[i];
            if (x < 0 || x >= n) { bad |= 1; continue; }
            if (x == u) bad |= 2;
            if (i > b && adj[i - 1] >= x) bad |= 4;
        }
        if (bad) atomicOr(err, bad);
    }
}

// Symmetry on the ranked lists: every entry s of adj(r) ranked above r
// (an upward entry) must have r in adj(s), where r lies in the out-prefix of
// s (its neighbours ranked below it: at most max out-degree entries, a
// short search); and upward entries must be half of all entries.  Lists
// hold no duplicates, so the reverses of the upward entries are distinct
// downward entries, and equal counts leave no other downward entry: every
// edge is present in both directions.  err bit 8: asymmetric; *up: upward
// entries.
__global__ void k_symmetric(const int4 *vinfo, const int *adj, int64_t n, unsigned *err, unsigned long long *up) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (gridDim.x * (int64_t)blockDim.x) >> 5;
    bool bad = false;
    unsigned long long cnt = 0;
    for (int64_t r = warp; r < n; r += nwarps) {
        const int4 vr = vinfo[r];
        if (lane == 0) cnt += (unsigned long long)(vr.y - vr.z);
        const int *ar = adj + ((size_t)(unsigned)vr.x << 2);
        for (int i = vr.z + lane; i < vr.y; i += 32) {
            const int4 vs = vinfo[ar[i]];
            const int *as = adj + ((size_t)(unsigned)vs.x << 2);
            int lo = 0, hi = vs.z;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (as[mid] < (int)r) lo = mid + 1; else hi = mid;
            }
            bad |= lo >= vs.z || as[lo] != (int)r;
        }
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(err, 8u);
    if (lane == 0 && cnt) atomicAdd(up, cnt);
}

// First rank whose degree is at most d (degrees fall with rank): binary
// search by one thread.
__global__ void k_first_at_most(const int4 *vinfo, int64_t n, int d, long long *out) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (vinfo[mid].y > d) lo = mid + 1; else hi = mid;
    }
    *out = (long long)lo;
}

__global__ void k_check_offsets(const int64_t *off, int64_t n, int64_t nnz, unsigned *err) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i == 0 && (off[0] != 0 || off[n] != nnz)) atomicOr(err, 32u);
    if (i < n && off[i + 1] < off[i]) atomicOr(err, 32u);
}

__global__ void k_degree_keys(const int64_t *off, int64_t n, unsigned long long *keys) {
    const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= n) return;
    const unsigned long long deg = (unsigned long long)(off[v + 1] - off[v]);
    keys[v] = ((0xffffffffull - deg) << 32) | (unsigned long long)v;
}

// rank[orig] = r ; orig_of[r] = orig ; pdeg[r] = padded degree ; udeg[r] = degree
__global__ void k_rank(const unsigned long long *sorted, const int64_t *off, int64_t n, int *rank, int *orig_of,
                       int64_t *pdeg, int64_t *udeg) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int v = (int)(sorted[r] & 0xffffffffull);
    rank[v] = (int)r;
    orig_of[r] = v;
    const int64_t d = off[v + 1] - off[v];
    udeg[r] = d;
    pdeg[r] = (d + 3) & ~3ll;
}

__global__ void k_edge_keys(const int64_t *off, const int32_t *adj, int64_t n, const int *rank,
                            unsigned long long *keys) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (gridDim.x * (int64_t)blockDim.x) >> 5;
    for (int64_t u = warp; u < n; u += nwarps) {
        const unsigned long long ru = (unsigned long long)rank[u] << 32;
        for (int64_t i = off[u] + lane; i < off[u + 1]; i += 32)
            keys[i] = ru | (unsigned long long)(unsigned)rank[adj[i]];
    }
}

// Sorted (rank_u, rank_w) keys -> padded lists.  ustart[r] = first key of r.
__global__ void k_scatter(const unsigned long long *keys, int64_t nnz, const int64_t *ustart,
                          const int64_t *pstart, int *adj_out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nnz) return;
    const unsigned long long k = keys[i];
    const int r = (int)(k >> 32);
    adj_out[pstart[r] + (i - ustart[r])] = (int)(k & 0xffffffffull);
}

__global__ void k_finish(int *adj, const int64_t *pstart, const int64_t *udeg, const int64_t *pdeg,
                         const unsigned long long *sorted, const int32_t *labels, int64_t n,
                         int4 *vinfo, int *maxes) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int64_t s = pstart[r], d = udeg[r];
    for (int64_t j = d; j < pdeg[r]; ++j) adj[s + j] = PG_PAD;
    // out-degree: neighbours with rank < r
    int lo = 0, hi = (int)d;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (adj[s + mid] < r) lo = mid + 1; else hi = mid;
    }
    const int orig = (int)(sorted[r] & 0xffffffffull);
    const int lab = labels ? labels[orig] : 0;
    vinfo[r] = make_int4((int)(unsigned)(s >> 2), (int)d, lo, lab);
    atomicMax(maxes + 0, (int)d);
    atomicMax(maxes + 1, lo);
    atomicMax(maxes + 2, lab);
}

// heavy clique start vertices: out-degree > heavy_min, keyed by
// (out-degree descending, rank ascending); others get the largest key
__global__ void k_heavy_keys(const int4 *vinfo, int64_t n, int heavy_min, unsigned long long *keys, unsigned *count) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int dplus = vinfo[r].z;
    if (dplus > heavy_min) {
        keys[r] = ((0xffffffffull - (unsigned long long)dplus) << 32) | (unsigned long long)r;
        atomicAdd(count, 1u);
    } else {
        keys[r] = ~0ull;
    }
}

__global__ void k_heavy_ids(const unsigned long long *sorted, int64_t count, int *out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < count) out[i] = (int)(sorted[i] & 0xffffffffull);
}

// hub bitmaps: one warp per hub row, bits of its neighbours
__global__ void k_hub_bits(const int4 *vinfo, const int *adj, int n_hubs, int stride, unsigned *bits) {
    const int lane = threadIdx.x & 31;
    const int r = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    if (r >= n_hubs) return;
    const int4 vi = vinfo[r];
    const int *a = adj + ((size_t)(unsigned)vi.x << 2);
    unsigned *row = bits + (size_t)r * stride;
    for (int i = lane; i < vi.y; i += 32) {
        const int x = a[i];
        atomicOr(row + (x >> 5), 1u << (x & 31));
    }
}

inline unsigned grid_for(int64_t n, int block) {
    int64_t g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > 0x7fffffff) g = 0x7fffffff;
    return (unsigned)g;
}

// Load temporaries: stream-ordered from the library pool, freed on the same
// stream when they go out of scope.
struct DevBuf {
    void *p = nullptr;
    cudaStream_t s = nullptr;
    int alloc(size_t bytes, cudaStream_t st) {
        s = st;
        return pg_dalloc(&p, bytes, st);
    }
    ~DevBuf() { if (p) pg_dfree(p, s); }
};

}  // namespace

int pg_graph_build(pg_graph *g, const int64_t *d_off, const int32_t *d_adj, int64_t nnz,
                   const int32_t *d_labels, cudaStream_t s) {
    const int64_t n = g->n;
    DevBuf err_b, vkeys, vkeys2, tmp, udeg, pdeg, ustart, pstart, ekeys, ekeys2, maxes_b;
    PG_TRY(err_b.alloc(4 * sizeof(unsigned long long), s));
    unsigned *err = (unsigned *)err_b.p;
    unsigned long long *up = (unsigned long long *)err_b.p + 2;
    PG_CUDA(cudaMemsetAsync(err_b.p, 0, 4 * sizeof(unsigned long long), s));
    k_check_offsets<<<grid_for(n + 1, kBlock), kBlock, 0, s>>>(d_off, n, nnz, err);
    unsigned herr = 0;
    PG_CUDA(cudaMemcpyAsync(&herr, err, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    PG_CUDA(cudaStreamSynchronize(s));
    if (herr) return pg_set_error(PG_EINVAL, "offsets must start at 0, end at nnz and be non-decreasing");
    if (n > 0) {
        k_validate<<<grid_for(n * 32, kBlock), kBlock, 0, s>>>(d_off, d_adj, d_labels, n, err);
        PG_CUDA(cudaGetLastError());
        PG_CUDA(cudaMemcpyAsync(&herr, err, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
        PG_CUDA(cudaStreamSynchronize(s));
    }
    if (herr & 1) return pg_set_error(PG_EINVAL, "adjacency entry out of range");
    if (herr & 2) return pg_set_error(PG_EINVAL, "self loop in data graph");
    if (herr & 4) return pg_set_error(PG_EINVAL, "adjacency list not strictly ascending (unsorted or duplicate)");
    if (herr & 16) return pg_set_error(PG_EINVAL, "negative vertex label");

    const int64_t nn = n > 0 ? n : 1;
    PG_TRY(vkeys.alloc(nn * sizeof(unsigned long long), s));
    PG_TRY(vkeys2.alloc(nn * sizeof(unsigned long long), s));
    PG_TRY(udeg.alloc(nn * sizeof(int64_t), s));
    PG_TRY(pdeg.alloc(nn * sizeof(int64_t), s));
    PG_TRY(ustart.alloc(nn * sizeof(int64_t), s));
    PG_TRY(pstart.alloc(nn * sizeof(int64_t), s));
    PG_TRY(pg_dalloc((void **)&g->rank, nn * sizeof(int), s));
    PG_TRY(pg_dalloc((void **)&g->orig, nn * sizeof(int), s));
    PG_TRY(pg_dalloc((void **)&g->vinfo, nn * sizeof(int4), s));
    PG_TRY(maxes_b.alloc(3 * sizeof(int), s));
    int *maxes = (int *)maxes_b.p;
    PG_CUDA(cudaMemsetAsync(maxes, 0, 3 * sizeof(int), s));

    // rank by (degree desc, id asc)
    k_degree_keys<<<grid_for(n, kBlock), kBlock, 0, s>>>(d_off, n, (unsigned long long *)vkeys.p);
    size_t tmp_bytes = 0, need = 0;
    cub::DeviceRadixSort::SortKeys(nullptr, need, (unsigned long long *)vkeys.p,
                                   (unsigned long long *)vkeys2.p, (int64_t)n, 0, 64, s);
    tmp_bytes = need;
    cub::DeviceScan::ExclusiveSum(nullptr, need, (int64_t *)pdeg.p, (int64_t *)pstart.p, (int64_t)n, s);
    tmp_bytes = std::max(tmp_bytes, need);
    const int64_t ne = nnz > 0 ? nnz : 1;
    int bits_n = 1;
    while ((1ll << bits_n) < n) ++bits_n;
    cub::DeviceRadixSort::SortKeys(nullptr, need, (unsigned long long *)nullptr,
                                   (unsigned long long *)nullptr, (int64_t)nnz, 0, 32 + bits_n, s);
    tmp_bytes = std::max(tmp_bytes, need);
    PG_TRY(tmp.alloc(tmp_bytes + 16, s));

    need = tmp_bytes;
    PG_CUDA(cub::DeviceRadixSort::SortKeys(tmp.p, need, (unsigned long long *)vkeys.p,
                                           (unsigned long long *)vkeys2.p, (int64_t)n, 0, 64, s));
    const unsigned long long *sorted = (const unsigned long long *)vkeys2.p;
    k_rank<<<grid_for(n, kBlock), kBlock, 0, s>>>(sorted, d_off, n, g->rank, g->orig, (int64_t *)pdeg.p,
                                                  (int64_t *)udeg.p);
    need = tmp_bytes;
    PG_CUDA(cub::DeviceScan::ExclusiveSum(tmp.p, need, (int64_t *)pdeg.p, (int64_t *)pstart.p, (int64_t)n, s));
    need = tmp_bytes;
    PG_CUDA(cub::DeviceScan::ExclusiveSum(tmp.p, need, (int64_t *)udeg.p, (int64_t *)ustart.p, (int64_t)n, s));

    // padded size = last start + last padded degree
    int64_t last_start = 0, last_pdeg = 0;
    if (n > 0) {
        PG_CUDA(cudaMemcpyAsync(&last_start, (int64_t *)pstart.p + (n - 1), sizeof(int64_t),
                                cudaMemcpyDeviceToHost, s));
        PG_CUDA(cudaMemcpyAsync(&last_pdeg, (int64_t *)pdeg.p + (n - 1), sizeof(int64_t),
                                cudaMemcpyDeviceToHost, s));
        PG_CUDA(cudaStreamSynchronize(s));
    }
    g->adj_entries = last_start + last_pdeg;
    if (g->adj_entries / 4 > 0xffffffffll) return pg_set_error(PG_EINVAL, "graph too large for 32-bit list starts");
    PG_TRY(pg_dalloc((void **)&g->adj, (g->adj_entries > 0 ? g->adj_entries : 4) * sizeof(int), s));

    // rewrite adjacency in ranks, sort by (rank_u, rank_w)
    PG_TRY(ekeys.alloc(ne * sizeof(unsigned long long), s));
    PG_TRY(ekeys2.alloc(ne * sizeof(unsigned long long), s));
    if (nnz > 0) {
        k_edge_keys<<<grid_for(n * 32, kBlock), kBlock, 0, s>>>(d_off, d_adj, n, g->rank,
                                                                (unsigned long long *)ekeys.p);
        need = tmp_bytes;
        PG_CUDA(cub::DeviceRadixSort::SortKeys(tmp.p, need, (unsigned long long *)ekeys.p,
                                               (unsigned long long *)ekeys2.p, (int64_t)nnz, 0, 32 + bits_n, s));
        k_scatter<<<grid_for(nnz, kBlock), kBlock, 0, s>>>((unsigned long long *)ekeys2.p, nnz,
                                                           (int64_t *)ustart.p, (int64_t *)pstart.p, g->adj);
    }
    if (n > 0) {
        k_finish<<<grid_for(n, kBlock), kBlock, 0, s>>>(g->adj, (int64_t *)pstart.p, (int64_t *)udeg.p,
                                                        (int64_t *)pdeg.p, sorted, d_labels, n, g->vinfo, maxes);
        PG_CUDA(cudaGetLastError());
        k_symmetric<<<grid_for(n * 32, kBlock), kBlock, 0, s>>>(g->vinfo, g->adj, n, err, up);
    }
    PG_CUDA(cudaGetLastError());
    int hm[3] = {0, 0, 0};
    unsigned long long hup = 0;
    PG_CUDA(cudaMemcpyAsync(hm, maxes, sizeof(hm), cudaMemcpyDeviceToHost, s));
    PG_CUDA(cudaMemcpyAsync(&herr, err, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    PG_CUDA(cudaMemcpyAsync(&hup, up, sizeof(hup), cudaMemcpyDeviceToHost, s));
    PG_CUDA(cudaStreamSynchronize(s));
    if ((herr & 8) || 2 * hup != (unsigned long long)nnz)
        return pg_set_error(PG_EINVAL, "asymmetric edge: graph must be undirected");
    g->max_deg = hm[0];
    g->max_out = hm[1];
    g->n_labels = d_labels ? hm[2] + 1 : 0;

    int rc = pg_graph_build_hubs(g, g->tune.hub_min_degree, g->tune.hub_max, s);
    if (rc) return rc;
    rc = pg_graph_build_heavy(g, g->tune.clique_heavy_min, s);
    if (rc) return rc;
    rc = pg_graph_build_split(g, g->tune.batched_split_grain, s);
    if (rc) return rc;
    g->bytes_device = (int64_t)(nn * (2 * sizeof(int) + sizeof(int4)) + g->adj_entries * sizeof(int));
    return PG_OK;
}

int64_t pg_graph_bytes(const pg_graph *g) {
    return g->bytes_device + (int64_t)g->n_hubs * g->hub_stride * 4 + g->n_heavy * 4 +
           (g->split_prefix ? (int64_t)(g->n_split + 1) * 8 : 0);
}

// Task split of the batched kernel: ranks r < n_split (degree > grain) own
// ceil(degree / grain) tasks each (at most 1024), laid out by the prefix
// array split_prefix[0..n_split].  Degrees fall with rank, so n_split is
// found by binary search over single vinfo reads.
int pg_graph_build_split(pg_graph *g, int grain, cudaStream_t s) {
    if (g->split_prefix) {
        PG_CUDA(cudaDeviceSynchronize());
        pg_dfree(g->split_prefix, s);
        g->split_prefix = nullptr;
    }
    g->n_split = 0;
    g->n_split_tasks = 0;
    g->split_grain_built = grain;
    if (grain <= 0 || g->n == 0) return PG_OK;
    // first rank with degree <= grain (one device search, one copy)
    DevBuf first_b;
    PG_TRY(first_b.alloc(sizeof(long long), s));
    k_first_at_most<<<1, 1, 0, s>>>(g->vinfo, g->n, grain, (long long *)first_b.p);
    PG_CUDA(cudaGetLastError());
    long long h = 0;
    PG_CUDA(cudaMemcpyAsync(&h, first_b.p, sizeof(long long), cudaMemcpyDeviceToHost, s));
    PG_CUDA(cudaStreamSynchronize(s));
    if (h == 0) return PG_OK;
    std::vector<int4> head(h);
    PG_CUDA(cudaMemcpyAsync(head.data(), g->vinfo, h * sizeof(int4), cudaMemcpyDeviceToHost, s));
    PG_CUDA(cudaStreamSynchronize(s));
    std::vector<long long> prefix(h + 1, 0);
    for (int64_t r = 0; r < h; ++r)
        prefix[r + 1] = prefix[r] + std::min<long long>(1024, ((long long)head[r].y + grain - 1) / grain);
    PG_TRY(pg_dalloc((void **)&g->split_prefix, (h + 1) * sizeof(long long), s));
    PG_CUDA(cudaMemcpyAsync(g->split_prefix, prefix.data(), (h + 1) * sizeof(long long), cudaMemcpyHostToDevice, s));
    PG_CUDA(cudaStreamSynchronize(s));
    g->n_split = (int)h;
    g->n_split_tasks = prefix[h];
    return PG_OK;
}

// Hub bitmaps for the highest-degree ranks: ranks 0..h-1 of degree >=
// min_degree, h <= max_hubs, at most 2 GiB.  Replaces earlier rows.
int pg_graph_build_hubs(pg_graph *g, int min_degree, int max_hubs, cudaStream_t s) {
    const int64_t n = g->n;
    if (g->hubbits) {
        PG_CUDA(cudaDeviceSynchronize()); // launches may still read the old rows
        pg_dfree(g->hubbits, s);
        g->hubbits = nullptr;
    }
    g->n_hubs = 0;
    g->hub_stride = (int)((n + 31) / 32);
    if (n > 0 && max_hubs > 0) {
        std::vector<int4> head(std::min<int64_t>(n, max_hubs));
        PG_CUDA(cudaMemcpyAsync(head.data(), g->vinfo, head.size() * sizeof(int4), cudaMemcpyDeviceToHost, s));
        PG_CUDA(cudaStreamSynchronize(s));
        int h = 0;
        while (h < (int)head.size() && head[h].y >= min_degree) ++h;
        const int stride = g->hub_stride;
        while (h > 0 && (int64_t)h * stride * 4 > (2ll << 30)) --h; // at most 2 GiB
        if (h > 0) {
            PG_TRY(pg_dalloc((void **)&g->hubbits, (size_t)h * stride * sizeof(unsigned), s));
            PG_CUDA(cudaMemsetAsync(g->hubbits, 0, (size_t)h * stride * sizeof(unsigned), s));
            k_hub_bits<<<grid_for((int64_t)h * 32, kBlock), kBlock, 0, s>>>(g->vinfo, g->adj, h, stride, g->hubbits);
            PG_CUDA(cudaGetLastError());
            PG_CUDA(cudaStreamSynchronize(s));
        }
        g->n_hubs = h;
    }
    g->d.hubbits = g->hubbits;
    g->d.n_hubs = g->n_hubs;
    g->d.hub_stride = g->hub_stride;
    return PG_OK;
}

// Heavy clique start vertices: out-degree > heavy_min, by out-degree
// descending (rank ascending on ties).  Replaces the earlier list.
int pg_graph_build_heavy(pg_graph *g, int heavy_min, cudaStream_t s) {
    const int64_t n = g->n;
    if (g->heavy) {
        PG_CUDA(cudaDeviceSynchronize());
        pg_dfree(g->heavy, s);
        g->heavy = nullptr;
    }
    g->n_heavy = 0;
    const int64_t nn = n > 0 ? n : 1;
    PG_TRY(pg_dalloc((void **)&g->heavy, nn * sizeof(int), s));
    if (n == 0) return PG_OK;
    DevBuf k1, k2, cnt, tmp;
    PG_TRY(k1.alloc(nn * sizeof(unsigned long long), s));
    PG_TRY(k2.alloc(nn * sizeof(unsigned long long), s));
    PG_TRY(cnt.alloc(sizeof(unsigned), s));
    size_t tmp_bytes = 0;
    PG_CUDA(cub::DeviceRadixSort::SortKeys(nullptr, tmp_bytes, (unsigned long long *)k1.p,
                                           (unsigned long long *)k2.p, (int64_t)n, 0, 64, s));
    PG_TRY(tmp.alloc(tmp_bytes + 16, s));
    PG_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(unsigned), s));
    k_heavy_keys<<<grid_for(n, kBlock), kBlock, 0, s>>>(g->vinfo, n, heavy_min, (unsigned long long *)k1.p,
                                                        (unsigned *)cnt.p);
    PG_CUDA(cudaGetLastError());
    PG_CUDA(cub::DeviceRadixSort::SortKeys(tmp.p, tmp_bytes, (unsigned long long *)k1.p,
                                           (unsigned long long *)k2.p, (int64_t)n, 0, 64, s));
    unsigned nh = 0;
    PG_CUDA(cudaMemcpyAsync(&nh, cnt.p, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    PG_CUDA(cudaStreamSynchronize(s));
    g->n_heavy = nh;
    g->heavy_min_built = heavy_min;
    if (nh > 0) k_heavy_ids<<<grid_for(nh, kBlock), kBlock, 0, s>>>((unsigned long long *)k2.p, nh, g->heavy);
    PG_CUDA(cudaGetLastError());
    PG_CUDA(cudaStreamSynchronize(s));
    return PG_OK;
}
