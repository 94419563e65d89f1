// Labeled 3-motifs with label discovery (Section 6 workloads: "labeled 3-
// motifs"; Section 3.2.1: the labels of a pattern are discovered from its
// matches).  Every vertex-induced 3-vertex match is aggregated by its labels:
//
//   triangle (a, b, c), a <= b <= c        T[a, b, c]
//   wedge    centre c, leaves x <= y       W[c; x, y]
//
// Wedges are not enumerated: a centre v with h[l] neighbours labeled l has
// h[x] h[y] (x < y) or C(h[x], 2) (x = y) edge-induced wedges with those leaf
// labels (the non-core completion by cardinality of Section 5.1).  Triangles
// are enumerated once each, from their largest rank: for c, every b in
// N+(c) and every a in N+(c) below b that lies in N+(b).  A triangle with
// label multiset M contains, for each of its vertices, one edge-induced
// wedge centred there, so the vertex-induced wedges are
//
//   W[c; x, y] = Wn[c; x, y] - mult_c({c, x, y}) * T[{c, x, y}]
//
// with mult_c the number of c's in the multiset.  Per-block tables in shared
// memory absorb the many small additions; blocks flush them into 128-bit
// global counters.
#include "device_sets.cuh"

namespace {

constexpr int kWarps = 8;
constexpr int kBlock = kWarps * 32;
constexpr int kMaxLabels = 32;

// index of the pair x <= y among C(L + 1, 2)
__host__ __device__ __forceinline__ int pair_index(int x, int y) { return y * (y + 1) / 2 + x; }
// index of the sorted triple a <= b <= c among C(L + 2, 3)
__host__ __device__ __forceinline__ int triple_index(int a, int b, int c) {
    return c * (c + 1) * (c + 2) / 6 + b * (b + 1) / 2 + a;
}

__device__ __forceinline__ void sort3(int &a, int &b, int &c) {
    int t;
    if (a > b) { t = a; a = b; b = t; }
    if (b > c) { t = b; b = c; c = t; }
    if (a > b) { t = a; a = b; b = t; }
}

// edge-induced wedges per (centre label, leaf-label pair): Wn[c * P + p]
__global__ void __launch_bounds__(kBlock) k_lm_wedges(DevGraph g, int L, unsigned long long *wn) {
    extern __shared__ __align__(16) unsigned long long smem[];
    const int P = L * (L + 1) / 2;
    unsigned long long *tab = smem;                         // L * P
    int *hist = (int *)(tab + (size_t)L * P) + (threadIdx.x >> 5) * L;
    const int lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < L * P; i += blockDim.x) tab[i] = 0;
    __syncthreads();
    const long long nw = (gridDim.x * (long long)blockDim.x) >> 5;
    for (long long v = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; v < g.n; v += nw) {
        for (int l = lane; l < L; l += 32) hist[l] = 0;
        __syncwarp();
        const int4 vi = __ldg(&g.vinfo[v]);
        const int *a = adj_of(g, vi);
        for (int i = lane; i < vi.y; i += 32) atomicAdd(&hist[__ldg(&g.vinfo[__ldg(a + i)].w)], 1);
        __syncwarp();
        unsigned long long *row = tab + (size_t)vi.w * P;
        for (int y = 0; y < L; ++y) {
            const unsigned long long hy = (unsigned)hist[y];
            if (!hy) continue;
            for (int x = lane; x <= y; x += 32) {
                const unsigned long long hx = (unsigned)hist[x];
                const unsigned long long c = x == y ? hx * (hx - 1) / 2 : hx * hy;
                if (c) atomicAdd(row + pair_index(x, y), c);
            }
        }
        __syncwarp();
    }
    __syncthreads();
    for (int i = threadIdx.x; i < L * P; i += blockDim.x)
        if (tab[i]) atomic_add_u128(wn + 2 * i, tab[i]);
}

// triangles per sorted label triple: T[triple_index]
__global__ void __launch_bounds__(kBlock) k_lm_triangles(DevGraph g, int L, unsigned long long *tri) {
    extern __shared__ __align__(16) unsigned long long smem[];
    const int Q = L * (L + 1) * (L + 2) / 6;
    unsigned long long *tab = smem;
    const int lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < Q; i += blockDim.x) tab[i] = 0;
    __syncthreads();
    const long long nw = (gridDim.x * (long long)blockDim.x) >> 5;
    for (long long c = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; c < g.n; c += nw) {
        const int4 ci = __ldg(&g.vinfo[c]);
        const int *nc = adj_of(g, ci); // N+(c) = first ci.z entries (smaller ranks)
        for (int j = 1; j < ci.z; ++j) {
            const int b = __ldg(nc + j);
            const int4 bi = __ldg(&g.vinfo[b]);
            const int *nb = adj_of(g, bi);
            for (int i = lane; i < j; i += 32) {
                const int a = __ldg(nc + i);
                if (contains_g(nb, bi.z, a)) {
                    int la = __ldg(&g.vinfo[a].w), lb = bi.w, lc = ci.w;
                    sort3(la, lb, lc);
                    atomicAdd(tab + triple_index(la, lb, lc), 1ull);
                }
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < Q; i += blockDim.x)
        if (tab[i]) atomic_add_u128(tri + 2 * i, tab[i]);
}

__device__ __forceinline__ unsigned __int128 u128(const unsigned long long *p) {
    return ((unsigned __int128)p[1] << 64) | p[0];
}

// induced wedges and triangles -> nonzero records
__global__ void k_lm_emit(int L, const unsigned long long *wn, const unsigned long long *tri, pg_labeled_count *out,
                          long long capacity, unsigned long long *n_out) {
    const int P = L * (L + 1) / 2, Q = L * (L + 1) * (L + 2) / 6;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    pg_labeled_count r;
    unsigned __int128 cnt = 0;
    if (i < (long long)L * P) {
        const int c = (int)(i / P), p = (int)(i % P);
        int y = 0;
        while ((y + 1) * (y + 2) / 2 <= p) ++y;
        const int x = p - y * (y + 1) / 2;
        int a = c, b = x, d = y;
        sort3(a, b, d);
        const int mult = (a == c) + (b == c) + (d == c);
        cnt = u128(wn + 2 * i) - (unsigned __int128)mult * u128(tri + 2 * triple_index(a, b, d));
        r.shape = PG_FSM_WEDGE;
        r.labels[0] = c;
        r.labels[1] = x;
        r.labels[2] = y;
    } else if (i < (long long)L * P + Q) {
        const int t = (int)(i - (long long)L * P);
        int cc = 0;
        while ((cc + 1) * (cc + 2) * (cc + 3) / 6 <= t) ++cc;
        const int rest = t - cc * (cc + 1) * (cc + 2) / 6;
        int bb = 0;
        while ((bb + 1) * (bb + 2) / 2 <= rest) ++bb;
        const int aa = rest - bb * (bb + 1) / 2;
        cnt = u128(tri + 2 * t);
        r.shape = PG_FSM_TRIANGLE;
        r.labels[0] = aa;
        r.labels[1] = bb;
        r.labels[2] = cc;
    } else {
        return;
    }
    if (!cnt) return;
    r.count_lo = (unsigned long long)cnt;
    r.count_hi = (unsigned long long)(cnt >> 64);
    const unsigned long long slot = atomicAdd(n_out, 1ull);
    if ((long long)slot < capacity) out[slot] = r;
}

// Temporaries from the library pool, freed on their stream.
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

int pg_labeled_motif3_run(pg_graph *g, pg_labeled_count *out, int64_t capacity, int64_t *n_out, cudaStream_t s) {
    *n_out = 0;
    if (!g->labeled) return pg_set_error(PG_EINVAL, "labeled motifs need a labeled graph");
    const int L = std::max(1, (int)g->n_labels);
    if (L > kMaxLabels) return pg_set_error(PG_EUNSUPPORTED, "labeled motifs support labels 0..31");
    const int P = L * (L + 1) / 2, Q = L * (L + 1) * (L + 2) / 6;
    const size_t wn_words = 2 * (size_t)L * P, tri_words = 2 * (size_t)Q;
    DevBuf tabs, recs;
    PG_TRY(tabs.alloc((wn_words + tri_words + 1) * sizeof(unsigned long long), s));
    unsigned long long *wn = (unsigned long long *)tabs.p, *tri = wn + wn_words, *cnt = tri + tri_words;
    PG_CUDA(cudaMemsetAsync(tabs.p, 0, (wn_words + tri_words + 1) * sizeof(unsigned long long), s));
    const size_t smem_w = (size_t)L * P * sizeof(unsigned long long) + (size_t)kWarps * L * sizeof(int);
    const size_t smem_t = (size_t)Q * sizeof(unsigned long long);
    PG_CUDA(cudaFuncSetAttribute(k_lm_wedges, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_w));
    PG_CUDA(cudaFuncSetAttribute(k_lm_triangles, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_t));
    int per_sm = 0;
    PG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lm_wedges, kBlock, smem_w));
    if (g->n > 0) {
        k_lm_wedges<<<std::max(1, per_sm) * g->num_sms, kBlock, smem_w, s>>>(g->d, L, wn);
        PG_CUDA(cudaGetLastError());
        PG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lm_triangles, kBlock, smem_t));
        k_lm_triangles<<<std::max(1, per_sm) * g->num_sms, kBlock, smem_t, s>>>(g->d, L, tri);
        PG_CUDA(cudaGetLastError());
    }
    const long long total = (long long)L * P + Q;
    const long long cap = std::max<long long>(capacity, 0);
    PG_TRY(recs.alloc(std::max<long long>(cap, 1) * sizeof(pg_labeled_count), s));
    k_lm_emit<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(L, wn, tri, (pg_labeled_count *)recs.p, cap, cnt);
    PG_CUDA(cudaGetLastError());
    unsigned long long n = 0;
    PG_CUDA(cudaMemcpyAsync(&n, cnt, sizeof(n), cudaMemcpyDeviceToHost, s));
    PG_CUDA(cudaStreamSynchronize(s));
    *n_out = (int64_t)n;
    const long long copy = std::min<long long>((long long)n, cap);
    if (copy > 0) {
        PG_CUDA(cudaMemcpyAsync(out, recs.p, copy * sizeof(pg_labeled_count), cudaMemcpyDeviceToHost, s));
        PG_CUDA(cudaStreamSynchronize(s));
    }
    if ((long long)n > cap) return pg_set_error(PG_ETRUNC, "more labeled motifs than capacity; *n_out is exact");
    return PG_OK;
}
