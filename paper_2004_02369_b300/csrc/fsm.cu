// Labeled frequent subgraph mining with MNI support, patterns of 1..3 edges
// (Section 2.1: FSM, MNI support; Section 3.2.1: label discovery; Section 5.5:
// domains kept as bitmaps of the data vertices each pattern vertex maps to).
//
// The MNI support of a labeled pattern is the smallest of its pattern
// vertices' domains, D(u) = { phi(u) : phi a valid edge-induced map }.  A data
// vertex v lies in D(u) iff some match puts v at u, so the kernels decide,
// for every vertex v, which (shape, position, label tuple) domains contain v:
// the vertices next to v on the shape (its core) are scanned, and the last,
// leaf vertex of the shape is never enumerated -- its existence follows from
// label-partitioned neighbour counts of an already bound vertex, with the
// vertices already used subtracted (the non-core completion by set
// cardinality of Section 5.1, applied to domains).  Each vertex's answers
// form one row of membership bits (its column of every domain bitmap); rows
// are grouped by the vertex's label, and a column reduction per label gives
// every domain size.  Support = min over positions; the frequent set is the
// patterns with support >= threshold (equal to the extend-by-edge loop's
// result because MNI support is anti-monotone).
//
// Row layout (one 32-bit mask over the last label index per word), v's own
// label being l:
//   E          y      v has a neighbour labeled y                     edge end
//   WC[x]      y      distinct neighbours labeled x and y             wedge centre
//   WL[c]      y      v - w(c) - u(y), u != v                         wedge leaf
//   T[c]       y      v, w(c), u(y) pairwise adjacent                 triangle
//   SC[x][y]   z      distinct neighbours labeled x, y, z             star centre
//   SL[c][y]   z      v - w(c), w has two more neighbours y, z        star leaf
//   PE[b][c]   d      v - w(b) - u(c) - x(d), all distinct            path end
//   PI[a][c]   d      a'(a) - v - w(c) - x(d), all distinct           path inner
#include <algorithm>
#include <vector>

#include "device_sets.cuh"

namespace {

constexpr int kWarps = 4;
constexpr int kBlock = kWarps * 32;

struct FsmLayout {
    int nl;
    int oE, oWC, oWL, oT, oSC, oSL, oPE, oPI, words;
};

FsmLayout fsm_layout(int nl) {
    FsmLayout L;
    L.nl = nl;
    L.oE = 0;
    L.oWC = 1;
    L.oWL = L.oWC + nl;
    L.oT = L.oWL + nl;
    L.oSC = L.oT + nl;
    L.oSL = L.oSC + nl * nl;
    L.oPE = L.oSL + nl * nl;
    L.oPI = L.oPE + nl * nl;
    L.words = L.oPI + nl * nl;
    return L;
}

__device__ __forceinline__ unsigned bit(int l) { return 1u << l; }

// per vertex: label counts saturated at 3, as masks {l : count >= 1, 2, 3}
__global__ void k_label_masks(DevGraph g, int4 *info) {
    const int lane = threadIdx.x & 31;
    const long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nw = (gridDim.x * (long long)blockDim.x) >> 5;
    for (long long v = w; v < g.n; v += nw) {
        const int4 vi = __ldg(&g.vinfo[v]);
        const int *a = adj_of(g, vi);
        unsigned m1 = 0, m2 = 0, m3 = 0;
        for (int i = lane; i < vi.y; i += 32) {
            const unsigned b = bit(__ldg(&g.vinfo[__ldg(a + i)].w));
            // saturating count per label across the lane's own elements
            m3 |= m2 & b;
            m2 |= m1 & b;
            m1 |= b;
        }
        // combine lanes: count >= 2 if two lanes have it, etc.
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned a1 = __shfl_xor_sync(PG_FULL, m1, o), a2 = __shfl_xor_sync(PG_FULL, m2, o),
                           a3 = __shfl_xor_sync(PG_FULL, m3, o);
            const unsigned n1 = m1 | a1, n2 = m2 | a2 | (m1 & a1), n3 = m3 | a3 | (m2 & a1) | (m1 & a2);
            m1 = n1;
            m2 = n2;
            m3 = n3;
        }
        if (lane == 0) info[v] = make_int4((int)m1, (int)m2, (int)m3, vi.w);
    }
}

// bucket position of every vertex in label order
__global__ void k_label_hist(DevGraph g, unsigned *hist) {
    const long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v < g.n) atomicAdd(hist + __ldg(&g.vinfo[v].w), 1u);
}

__global__ void k_label_slot(DevGraph g, unsigned *cursor, int *row_of) {
    const long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v < g.n) row_of[v] = (int)atomicAdd(cursor + __ldg(&g.vinfo[v].w), 1u);
}

struct FlagArgs {
    DevGraph g;
    FsmLayout L;
    const int4 *info;
    const int *row_of;
    unsigned *rows; // [n][L.words]
    unsigned long long *queue;
};

// mask of labels l with (count(l) - [l == drop]) >= 1
__device__ __forceinline__ unsigned avail1(int4 in, int drop) {
    return ((unsigned)in.x & ~bit(drop)) | ((unsigned)in.y & bit(drop));
}
// ... >= 2
__device__ __forceinline__ unsigned avail2(int4 in, int drop) {
    return ((unsigned)in.y & ~bit(drop)) | ((unsigned)in.z & bit(drop));
}
// ... == 1
__device__ __forceinline__ unsigned exact1(int4 in, int drop) {
    return (((unsigned)in.x & ~(unsigned)in.y) & ~bit(drop)) | (((unsigned)in.y & ~(unsigned)in.z) & bit(drop));
}
__device__ __forceinline__ bool has(int4 in, int l, int c) {
    const unsigned m = c == 1 ? (unsigned)in.x : c == 2 ? (unsigned)in.y : (unsigned)in.z;
    return (m >> l) & 1u;
}

__global__ void __launch_bounds__(kBlock) k_fsm_rows(FlagArgs a) {
    extern __shared__ unsigned s_rows[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const FsmLayout L = a.L;
    const int nl = L.nl;
    unsigned *R = s_rows + (size_t)wib * L.words;
    const DevGraph &g = a.g;
    for (;;) {
        int v = 0;
        if (lane == 0) v = (int)atomicAdd(a.queue, 1ull);
        v = __shfl_sync(PG_FULL, v, 0);
        if (v >= g.n) break;
        for (int i = lane; i < L.words; i += 32) R[i] = 0;
        __syncwarp();
        const int4 vi = __ldg(&g.vinfo[v]);
        const int4 iv = a.info[v];
        const int lv = iv.w;
        const int *av = adj_of(g, vi);
        // ---- v's own counts: edge end, wedge centre, star centre ----------
        if (lane == 0) R[L.oE] = (unsigned)iv.x;
        for (int x = lane; x < nl; x += 32)
            R[L.oWC + x] = has(iv, x, 1) ? (avail1(iv, x) & ~bit(x)) | ((unsigned)iv.y & bit(x)) : 0u;
        for (int p = lane; p < nl * nl; p += 32) {
            const int x = p / nl, y = p % nl;
            unsigned mz = 0;
            for (int z = 0; z < nl; ++z) {
                const int cx = 1 + (y == x) + (z == x);
                bool ok = has(iv, x, cx);
                if (y != x) ok = ok && has(iv, y, 1 + (z == y));
                if (z != x && z != y) ok = ok && has(iv, z, 1);
                if (ok) mz |= bit(z);
            }
            R[L.oSC + p] = mz;
        }
        __syncwarp();
        // ---- neighbours w ----------------------------------------------------
        for (int e = 0; e < vi.y; ++e) {
            const int w = __ldg(av + e);
            const int4 wi = __ldg(&g.vinfo[w]);
            const int4 iw = a.info[w];
            const int lw = iw.w;
            const unsigned a1 = avail1(iw, lv); // labels among adj(w) \ {v}
            // wedge leaf, star leaf (centre w)
            if (lane == 0) atomicOr(&R[L.oWL + lw], a1);
            if (lane < nl && ((a1 >> lane) & 1u)) {
                const unsigned a2 = avail2(iw, lv);
                atomicOr(&R[L.oSL + lw * nl + lane], (a1 & ~bit(lane)) | (a2 & bit(lane)));
            }
            // triangle: labels of common neighbours of v and w
            const int *aw = adj_of(g, wi);
            unsigned tri = 0;
            {
                const bool v_small = vi.y <= wi.y;
                const int *sp = v_small ? av : aw;
                const int sl = v_small ? vi.y : wi.y;
                const Slice big = v_small ? Slice{aw, wi.y, w} : Slice{av, vi.y, v};
                for (int i = lane; i < sl; i += 32) {
                    const int u = __ldg(sp + i);
                    if (in_slice(g, big, u)) tri |= bit(__ldg(&g.vinfo[u].w));
                }
                tri = __reduce_or_sync(PG_FULL, tri);
            }
            if (lane == 0) atomicOr(&R[L.oT + lw], tri);
            // path inner: a'(a) in adj(v) \ {w}, d'(d) in adj(w) \ {v}, a' != d'
            {
                const unsigned amask = avail1(iv, lw);
                const unsigned corner = exact1(iv, lw) & exact1(iw, lv) & tri;
                if (lane < nl && ((amask >> lane) & 1u)) {
                    unsigned dm = a1;
                    if ((corner >> lane) & 1u) dm &= ~bit(lane); // single a' == single d'
                    atomicOr(&R[L.oPI + lane * nl + lw], dm);
                }
            }
            // path end: u in adj(w) \ {v}, x(d) in adj(u) \ {w, v}
            for (int i = lane; i < wi.y; i += 32) {
                const int u = __ldg(aw + i);
                if (u == v) continue;
                const int4 iu = a.info[u];
                unsigned dm = avail1(iu, lw);
                if (((dm & exact1(iu, lw)) >> lv) & 1u) {
                    // the single candidate labeled lv may be v itself
                    if (in_slice(g, Slice{av, vi.y, v}, u)) dm &= ~bit(lv);
                }
                atomicOr(&R[L.oPE + lw * nl + iu.w], dm);
            }
        }
        __syncwarp();
        unsigned *out = a.rows + (size_t)a.row_of[v] * L.words;
        for (int i = lane; i < L.words; i += 32) out[i] = R[i];
        __syncwarp();
    }
}

// counts[label][word][bit] += number of rows of that label with the bit set
__global__ void k_fsm_reduce(const unsigned *rows, FsmLayout L, const unsigned *label_start, int chunk,
                             unsigned *counts) {
    const int lane = threadIdx.x & 31;
    const long long task = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const int groups = (L.words + 31) / 32;
    // task = (label, chunk, word group)
    long long t = task;
    int lab = 0;
    const int nl = L.nl;
    for (; lab < nl; ++lab) {
        const unsigned rows_l = label_start[lab + 1] - label_start[lab];
        const long long chunks = (rows_l + chunk - 1) / chunk;
        if (t < chunks * groups) break;
        t -= chunks * groups;
    }
    if (lab >= nl) return;
    const int c = (int)(t / groups), wg = (int)(t % groups);
    const int word = wg * 32 + lane;
    const unsigned r0 = label_start[lab] + (unsigned)c * chunk;
    const unsigned r1 = min(label_start[lab + 1], r0 + chunk);
    if (word >= L.words) return;
    unsigned cnt[32];
    for (int b = 0; b < nl; ++b) cnt[b] = 0;
    for (unsigned r = r0; r < r1; ++r) {
        const unsigned x = rows[(size_t)r * L.words + word];
        if (!x) continue;
        for (int b = 0; b < nl; ++b) cnt[b] += (x >> b) & 1u;
    }
    unsigned *dst = counts + ((size_t)lab * L.words + word) * nl;
    for (int b = 0; b < nl; ++b)
        if (cnt[b]) atomicAdd(dst + b, cnt[b]);
}

struct Found {
    int shape;
    int l[4];
    unsigned long long support;
};

__device__ __forceinline__ unsigned cnt_at(const unsigned *counts, const FsmLayout &L, int lab, int word, int b) {
    return counts[((size_t)lab * L.words + word) * L.nl + b];
}

// supports of canonical tuples of one shape; frequent ones appended
__global__ void k_fsm_support(const unsigned *counts, FsmLayout L, int shape, unsigned long long threshold,
                              Found *out, unsigned long long *n_out, unsigned long long cap) {
    const int nl = L.nl;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long total = shape == 1 ? (long long)nl * nl : (shape <= 3) ? (long long)nl * nl * nl : (long long)nl * nl * nl * nl;
    if (t >= total) return;
    int l0 = (int)(t % nl), l1 = (int)((t / nl) % nl), l2 = (int)((t / nl / nl) % nl), l3 = (int)(t / nl / nl / nl);
    unsigned long long s = 0;
    Found f;
    f.shape = shape;
    f.l[0] = f.l[1] = f.l[2] = f.l[3] = -1;
    if (shape == 1) { // edge (x <= y)
        const int x = l1, y = l0;
        if (x > y) return;
        s = min(cnt_at(counts, L, x, L.oE, y), cnt_at(counts, L, y, L.oE, x));
        f.l[0] = x; f.l[1] = y;
    } else if (shape == 2) { // wedge (c; x <= y)
        const int c = l2, x = l1, y = l0;
        if (x > y) return;
        s = cnt_at(counts, L, c, L.oWC + x, y);
        s = min(s, (unsigned long long)cnt_at(counts, L, x, L.oWL + c, y));
        s = min(s, (unsigned long long)cnt_at(counts, L, y, L.oWL + c, x));
        f.l[0] = c; f.l[1] = x; f.l[2] = y;
    } else if (shape == 3) { // triangle x <= y <= z
        const int x = l2, y = l1, z = l0;
        if (x > y || y > z) return;
        s = cnt_at(counts, L, x, L.oT + y, z);
        s = min(s, (unsigned long long)cnt_at(counts, L, y, L.oT + x, z));
        s = min(s, (unsigned long long)cnt_at(counts, L, z, L.oT + x, y));
        f.l[0] = x; f.l[1] = y; f.l[2] = z;
    } else if (shape == 4) { // path a-b-c-d, canonical = min(tuple, reverse)
        const int a = l3, b = l2, c = l1, d = l0;
        // lexicographic (a,b,c,d) <= (d,c,b,a)
        const bool canon = a < d || (a == d && (b < c || b == c));
        if (!canon) return;
        s = cnt_at(counts, L, a, L.oPE + b * nl + c, d);
        s = min(s, (unsigned long long)cnt_at(counts, L, d, L.oPE + c * nl + b, a));
        s = min(s, (unsigned long long)cnt_at(counts, L, b, L.oPI + a * nl + c, d));
        s = min(s, (unsigned long long)cnt_at(counts, L, c, L.oPI + d * nl + b, a));
        f.l[0] = a; f.l[1] = b; f.l[2] = c; f.l[3] = d;
    } else { // star (c; x <= y <= z)
        const int c = l3, x = l2, y = l1, z = l0;
        if (x > y || y > z) return;
        s = cnt_at(counts, L, c, L.oSC + x * nl + y, z);
        s = min(s, (unsigned long long)cnt_at(counts, L, x, L.oSL + c * nl + y, z));
        s = min(s, (unsigned long long)cnt_at(counts, L, y, L.oSL + c * nl + x, z));
        s = min(s, (unsigned long long)cnt_at(counts, L, z, L.oSL + c * nl + x, y));
        f.l[0] = c; f.l[1] = x; f.l[2] = y; f.l[3] = z;
    }
    if (s < threshold || s == 0) return;
    f.support = s;
    const unsigned long long i = atomicAdd(n_out, 1ull);
    if (i < cap) out[i] = f;
}

struct DevMem {
    void *p = nullptr;
    ~DevMem() { if (p) cudaFree(p); }
};

}  // namespace

int pg_fsm_run(pg_graph *g, int max_edges, unsigned long long threshold, pg_fsm_pattern *out, int64_t capacity,
               int64_t *n_frequent, cudaStream_t s) {
    if (!g->labeled) return pg_set_error(PG_EINVAL, "frequent subgraph mining needs a labeled graph");
    if (max_edges < 1 || max_edges > 3) return pg_set_error(PG_EINVAL, "max_edges must be 1..3");
    const int nl = std::max(1, g->n_labels);
    if (nl > 32) return pg_set_error(PG_EUNSUPPORTED, "at most 32 labels");
    *n_frequent = 0;
    if (g->n == 0) return PG_OK;
    const FsmLayout L = fsm_layout(nl);
    const long long n = g->n;
    DevMem info, hist, row_of, rows, counts, found, nfound, queue;
    PG_CUDA(cudaMalloc(&info.p, n * sizeof(int4)));
    PG_CUDA(cudaMalloc(&hist.p, 2 * (nl + 1) * sizeof(unsigned)));
    PG_CUDA(cudaMalloc(&row_of.p, n * sizeof(int)));
    PG_CUDA(cudaMalloc(&rows.p, (size_t)n * L.words * sizeof(unsigned)));
    const size_t n_counts = (size_t)nl * L.words * nl;
    PG_CUDA(cudaMalloc(&counts.p, n_counts * sizeof(unsigned)));
    const unsigned long long cap = (unsigned long long)nl * nl * nl * nl * 2 + (unsigned long long)nl * nl * nl * 2 +
                                   (unsigned long long)nl * nl;
    PG_CUDA(cudaMalloc(&found.p, cap * sizeof(Found)));
    PG_CUDA(cudaMalloc(&nfound.p, sizeof(unsigned long long)));
    PG_CUDA(cudaMalloc(&queue.p, sizeof(unsigned long long)));
    unsigned *h = (unsigned *)hist.p, *cursor = h + (nl + 1);
    PG_CUDA(cudaMemsetAsync(hist.p, 0, 2 * (nl + 1) * sizeof(unsigned), s));
    PG_CUDA(cudaMemsetAsync(counts.p, 0, n_counts * sizeof(unsigned), s));
    PG_CUDA(cudaMemsetAsync(nfound.p, 0, sizeof(unsigned long long), s));
    PG_CUDA(cudaMemsetAsync(queue.p, 0, sizeof(unsigned long long), s));
    const unsigned nb = (unsigned)((n + 255) / 256);
    k_label_masks<<<(unsigned)std::min<long long>((n * 32 + 255) / 256, 1 << 20), 256, 0, s>>>(g->d, (int4 *)info.p);
    k_label_hist<<<nb, 256, 0, s>>>(g->d, h);
    // exclusive scan of the label histogram (host: nl <= 32 values)
    std::vector<unsigned> hh(nl + 1, 0), start(nl + 1, 0);
    PG_CUDA(cudaMemcpyAsync(hh.data(), h, nl * sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    PG_CUDA(cudaStreamSynchronize(s));
    for (int l = 0; l < nl; ++l) start[l + 1] = start[l] + hh[l];
    PG_CUDA(cudaMemcpyAsync(cursor, start.data(), (nl + 1) * sizeof(unsigned), cudaMemcpyHostToDevice, s));
    k_label_slot<<<nb, 256, 0, s>>>(g->d, cursor, (int *)row_of.p);
    PG_CUDA(cudaMemcpyAsync(h, start.data(), (nl + 1) * sizeof(unsigned), cudaMemcpyHostToDevice, s));
    FlagArgs fa;
    fa.g = g->d;
    fa.L = L;
    fa.info = (const int4 *)info.p;
    fa.row_of = (const int *)row_of.p;
    fa.rows = (unsigned *)rows.p;
    fa.queue = (unsigned long long *)queue.p;
    const size_t smem = (size_t)kWarps * L.words * sizeof(unsigned);
    PG_CUDA(cudaFuncSetAttribute(k_fsm_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fsm_rows, kBlock, smem);
    k_fsm_rows<<<std::max(1, per_sm) * g->num_sms, kBlock, smem, s>>>(fa);
    PG_CUDA(cudaGetLastError());
    const int chunk = 2048, groups = (L.words + 31) / 32;
    long long tasks = 0;
    for (int l = 0; l < nl; ++l) tasks += (long long)((hh[l] + chunk - 1) / chunk) * groups;
    if (tasks > 0) {
        k_fsm_reduce<<<(unsigned)((tasks * 32 + 255) / 256), 256, 0, s>>>((const unsigned *)rows.p, L, h, chunk,
                                                                         (unsigned *)counts.p);
        PG_CUDA(cudaGetLastError());
    }
    const int shapes_for[4] = {0, 1, 2, 5};
    for (int shape = 1; shape <= shapes_for[max_edges]; ++shape) {
        const long long total = shape == 1 ? (long long)nl * nl : shape <= 3 ? (long long)nl * nl * nl
                                                                               : (long long)nl * nl * nl * nl;
        if (max_edges == 2 && shape > 2) break;
        k_fsm_support<<<(unsigned)((total + 255) / 256), 256, 0, s>>>((const unsigned *)counts.p, L, shape,
                                                                     threshold, (Found *)found.p,
                                                                     (unsigned long long *)nfound.p, cap);
        PG_CUDA(cudaGetLastError());
    }
    unsigned long long nf = 0;
    PG_CUDA(cudaMemcpyAsync(&nf, nfound.p, sizeof(nf), cudaMemcpyDeviceToHost, s));
    PG_CUDA(cudaStreamSynchronize(s));
    std::vector<Found> hf((size_t)std::min(nf, cap));
    if (!hf.empty()) {
        PG_CUDA(cudaMemcpyAsync(hf.data(), found.p, hf.size() * sizeof(Found), cudaMemcpyDeviceToHost, s));
        PG_CUDA(cudaStreamSynchronize(s));
    }
    std::sort(hf.begin(), hf.end(), [](const Found &x, const Found &y) {
        if (x.shape != y.shape) return x.shape < y.shape;
        for (int i = 0; i < 4; ++i)
            if (x.l[i] != y.l[i]) return x.l[i] < y.l[i];
        return false;
    });
    *n_frequent = (int64_t)hf.size();
    for (size_t i = 0; i < hf.size() && (int64_t)i < capacity; ++i) {
        out[i].shape = hf[i].shape;
        for (int j = 0; j < 4; ++j) out[i].labels[j] = hf[i].l[j];
        out[i].support = hf[i].support;
    }
    if ((int64_t)hf.size() > capacity) return pg_set_error(PG_ETRUNC, "output capacity smaller than the frequent set");
    return PG_OK;
}
