// Level operations of the plan interpreter, shared by the single-plan and
// the batched (trie) kernels.  A level's candidate set is
//   S = (/\ adj(m[int_src])) \ (\/ adj(m[diff_src])) within (max m[lo_src],
//       min m[hi_src]), label-filtered, without m[excl_src]
// (Section 4.1 matching orders with partial-order bounds; Section 4.2
// anti-edges as set differences; Section 5.1 sorted-list set operations).
#pragma once
#include "device_sets.cuh"

namespace pgk {

struct LevelRange {
    int lo, hi; // open interval (lo, hi); lo = -1 / hi = INT_MAX when unbounded
};

__device__ __forceinline__ LevelRange level_range(const PgLevel &L, const int *m) {
    LevelRange r{-1, 0x7fffffff};
    for (int i = 0; i < L.n_lo; ++i) r.lo = max(r.lo, m[L.lo_src[i]]);
    for (int i = 0; i < L.n_hi; ++i) r.hi = min(r.hi, m[L.hi_src[i]]);
    return r;
}

// x passes label and exclusion tests of level L
__device__ __forceinline__ bool pass_label_excl(const DevGraph &g, const PgLevel &L, const int *m, int x) {
    bool ok = true;
    for (int i = 0; i < L.n_excl; ++i) ok &= (x != m[L.excl_src[i]]);
    if (ok && L.label >= 0) ok = (__ldg(&g.vinfo[x].w) == L.label);
    return ok;
}

// x[j] pass label and exclusion tests of level L (ANDed into ok[j]).
__device__ __forceinline__ void label_excl4(const DevGraph &g, const PgLevel &L, const int *m, const int (&x)[4],
                                            bool (&ok)[4]) {
    for (int i = 0; i < L.n_excl; ++i) {
        const int e = m[L.excl_src[i]];
#pragma unroll
        for (int j = 0; j < 4; ++j) ok[j] = ok[j] && x[j] != e;
    }
    if (L.label >= 0) {
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (ok[j]) ok[j] = __ldg(&g.vinfo[x[j]].w) == L.label;
    }
}

// Materialise the candidate set of (non-last) level L into buf, in
// ascending order; returns its size.  Each lane takes four driver elements
// per step (one 16-byte load) and tests them against the other lists four
// searches at a time; a warp prefix sum compacts the survivors.
static __device__ __noinline__ int fill_level(const DevGraph &g, const PgLevel &L, const int *m, int *buf, int lane) {
    const LevelRange r = level_range(L, m);
    if (r.lo + 1 >= r.hi) return 0;
    Slice s[PGP_MAXK];
    int drv = 0;
    for (int i = 0; i < L.n_int; ++i) {
        const int w = m[L.int_src[i]];
        const int4 vi = __ldg(&g.vinfo[w]);
        s[i] = bound_slice(adj_of(g, vi), vi.y, r.lo, r.hi, w);
        if (s[i].len < s[drv].len) drv = i;
    }
    const Driver4 dv = driver4(s[drv]);
    int n_out = 0;
    for (int base = 0; base < dv.total; base += 128) {
        int x[4];
        bool ok[4];
        driver4_load(dv, base, lane, x, ok);
        for (int i = 0; i < L.n_int; ++i)
            if (i != drv) in_slice4(g, s[i], x, ok, false);
        for (int i = 0; i < L.n_diff; ++i) {
            const int w = m[L.diff_src[i]];
            const int4 vi = __ldg(&g.vinfo[w]);
            in_slice4(g, Slice{adj_of(g, vi), vi.y, w}, x, ok, true);
        }
        label_excl4(g, L, m, x, ok);
        const int c = (int)ok[0] + (int)ok[1] + (int)ok[2] + (int)ok[3];
        int step_total;
        int pos = n_out + warp_excl_scan(c, lane, &step_total);
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (ok[j]) buf[pos++] = x[j];
        n_out += step_total;
    }
    __syncwarp();
    return n_out;
}

// Number of elements of slice d that lie in every slice of s[0, n) other
// than index `skip`, in none of s[n, n + nd), and carry `label` (>= 0).
__device__ __forceinline__ unsigned long long count_filtered(const DevGraph &g, const Slice &d, const Slice *s,
                                                              int n, int skip, int nd, int label, int lane) {
    const Driver4 dv = driver4(d);
    unsigned c = 0;
    for (int base = 0; base < dv.total; base += 128) {
        int x[4];
        bool ok[4];
        driver4_load(dv, base, lane, x, ok);
        for (int i = 0; i < n; ++i)
            if (i != skip) in_slice4(g, s[i], x, ok, false);
        for (int i = 0; i < nd; ++i) in_slice4(g, s[n + i], x, ok, true);
        if (label >= 0) {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (ok[j]) ok[j] = __ldg(&g.vinfo[x[j]].w) == label;
        }
        c += (unsigned)ok[0] + (unsigned)ok[1] + (unsigned)ok[2] + (unsigned)ok[3];
    }
    return (unsigned long long)__reduce_add_sync(PG_FULL, c);
}

// |S| of the last level (before C(|S|, g)).
static __device__ __noinline__ unsigned long long count_last(const DevGraph &g, const PgLevel &L, const int *m, int lane) {
    const LevelRange r = level_range(L, m);
    if (r.lo + 1 >= r.hi) return 0;
    Slice s[2 * PGP_MAXK];
    const int ni = L.n_int, nd = L.n_diff;
    int drv = 0;
    for (int i = 0; i < ni; ++i) {
        const int w = m[L.int_src[i]];
        const int4 vi = __ldg(&g.vinfo[w]);
        s[i] = bound_slice(adj_of(g, vi), vi.y, r.lo, r.hi, w);
        if (s[i].len < s[drv].len) drv = i;
    }
    for (int j = 0; j < nd; ++j) {
        const int w = m[L.diff_src[j]];
        const int4 vi = __ldg(&g.vinfo[w]);
        s[ni + j] = bound_slice(adj_of(g, vi), vi.y, r.lo, r.hi, w);
    }
    const bool labeled = L.label >= 0;
    // cost of filtering the driver directly vs inclusion-exclusion
    long long direct = (long long)s[drv].len * (ni - 1 + nd + (labeled ? 1 : 0));
    long long ie = 0;
    for (unsigned T = 1; T < (1u << nd); ++T) {
        int mn = s[drv].len, terms = ni - 1 + (labeled ? 1 : 0);
        for (int j = 0; j < nd; ++j)
            if (T >> j & 1) { mn = min(mn, s[ni + j].len); ++terms; }
        ie += (long long)mn * terms;
    }
    if (labeled || ni > 1) ie += (long long)s[drv].len * (ni - 1 + (labeled ? 1 : 0));
    long long total = 0;
    if (ni == 1 && nd == 0 && !labeled) {
        // a plain bounded slice of one list: its length (the excluded
        // images inside it are removed below), no pass over its elements
        total = s[0].len;
    } else if (nd == 0 || direct <= ie) {
        total = (long long)count_filtered(g, s[drv], s, ni, drv, nd, L.label, lane);
    } else {
        // |A \ (B1 u ... u Bd)| = sum over T subset of diffs of (-1)^|T| |A n B_T|
        for (unsigned T = 0; T < (1u << nd); ++T) {
            int dd = drv;
            for (int j = 0; j < nd; ++j)
                if ((T >> j & 1) && s[ni + j].len < s[dd].len) dd = ni + j;
            long long term;
            if (ni == 1 && T == 0 && !labeled) {
                term = s[dd].len;
            } else {
                // the intersected lists: the regular ones and the differences in T
                Slice t[2 * PGP_MAXK];
                int nt = 0, skip = -1;
                for (int i = 0; i < ni; ++i) {
                    if (i == dd) skip = nt;
                    t[nt++] = s[i];
                }
                for (int j = 0; j < nd; ++j)
                    if (T >> j & 1) {
                        if (ni + j == dd) skip = nt;
                        t[nt++] = s[ni + j];
                    }
                term = (long long)count_filtered(g, s[dd], t, nt, skip, 0, L.label, lane);
            }
            total += (__popc(T) & 1) ? -term : term;
        }
    }
    // injectivity: remove earlier images that fall inside S
    // (earlier images are pairwise distinct, so each is removed at most once)
    bool in = false;
    if (lane < L.n_excl) {
        const int x = m[L.excl_src[lane]];
        in = x > r.lo && x < r.hi;
        for (int i = 0; i < ni && in; ++i) in = in_slice(g, s[i], x);
        for (int j = 0; j < nd && in; ++j) in = !in_slice(g, s[ni + j], x);
        if (in && labeled) in = (__ldg(&g.vinfo[x].w) == L.label);
    }
    total -= (long long)__popc(__ballot_sync(PG_FULL, in));
    return (unsigned long long)total;
}

// Anti-vertex check C on the bound images m (Section 3.1.2): true iff no
// data vertex lies in every adj(m[int_src]) other than the images
// m[excl_src].  The warp walks the shortest list and stops at the first
// witness.
static __device__ __noinline__ bool anti_ok(const DevGraph &g, const PgAntiCheck &C, const int *m, int lane) {
    Slice s[PGP_MAXK];
    int drv = 0;
    for (int i = 0; i < C.n_int; ++i) {
        const int w = m[C.int_src[i]];
        const int4 vi = __ldg(&g.vinfo[w]);
        s[i] = Slice{adj_of(g, vi), vi.y, w};
        if (s[i].len < s[drv].len) drv = i;
    }
    const Slice d = s[drv];
    for (int base = 0; base < d.len; base += 32) {
        const int idx = base + lane;
        bool hit = idx < d.len;
        if (hit) {
            const int x = __ldg(d.p + idx);
            for (int i = 0; i < C.n_int && hit; ++i)
                if (i != drv) hit = in_slice(g, s[i], x);
            for (int i = 0; i < C.n_excl && hit; ++i) hit = x != m[C.excl_src[i]];
        }
        if (__any_sync(PG_FULL, hit)) return false;
    }
    return true;
}

// Every anti-vertex check attached to level l passes for the images m.
__device__ __forceinline__ bool checks_ok(const DevGraph &g, const PgOrder &ord, int l, const int *m, int lane) {
    bool ok = true;
    for (int c = 0; c < ord.n_checks && ok; ++c)
        if (ord.chk[c].level == l) ok = anti_ok(g, ord.chk[c], m, lane);
    return ok;
}

// Keep the candidates buf[0, n) of level l that pass its anti-vertex checks
// (m[l] takes each candidate in turn); returns how many are kept, in order.
static __device__ __noinline__ int filter_anti(const DevGraph &g, const PgOrder &ord, int l, int *m, int *buf, int n,
                                               int lane) {
    int kept = 0;
    for (int i = 0; i < n; ++i) {
        const int x = buf[i];
        m[l] = x;
        if (checks_ok(g, ord, l, m, lane)) {
            if (lane == 0) buf[kept] = x; // kept <= i: never a slot still to be read
            ++kept;
        }
    }
    __syncwarp();
    return kept;
}

// x lies in the candidate set of level spec L (bounds, lists, differences,
// label, excluded images): one lane's test.
__device__ __forceinline__ bool in_level_set(const DevGraph &g, const PgLevel &L, const int *m, int x) {
    const LevelRange r = level_range(L, m);
    if (!(x > r.lo && x < r.hi)) return false;
    for (int i = 0; i < L.n_excl; ++i)
        if (x == m[L.excl_src[i]]) return false;
    for (int i = 0; i < L.n_int; ++i) {
        const int w = m[L.int_src[i]];
        const int4 vi = __ldg(&g.vinfo[w]);
        if (!in_slice(g, Slice{adj_of(g, vi), vi.y, w}, x)) return false;
    }
    for (int i = 0; i < L.n_diff; ++i) {
        const int w = m[L.diff_src[i]];
        const int4 vi = __ldg(&g.vinfo[w]);
        if (in_slice(g, Slice{adj_of(g, vi), vi.y, w}, x)) return false;
    }
    return L.label < 0 || __ldg(&g.vinfo[x].w) == L.label;
}

// A set given by a level spec is a plain bounded slice of one adjacency list
// (minus excluded images) when it has one intersected list, no differences
// and no label: its elements and ranks are read off the list directly.
__device__ __forceinline__ bool is_slice(const PgLevel &L) {
    return L.n_int == 1 && L.n_diff == 0 && L.label < 0;
}

__device__ __forceinline__ Slice level_slice(const DevGraph &g, const PgLevel &L, const int *m) {
    const LevelRange r = level_range(L, m);
    const int w = m[L.int_src[0]];
    const int4 vi = __ldg(&g.vinfo[w]);
    if (r.lo + 1 >= r.hi) return Slice{adj_of(g, vi), 0, w};
    return bound_slice(adj_of(g, vi), vi.y, r.lo, r.hi, w);
}

// Joint count of the last two levels: X (single non-core vertex x at level
// xl) and Y (single non-core vertex y whose spec refers to x only through
// the partial order or injectivity).  With Y' = Y without those references:
//   no order between x, y:  |SX| |SY'| - |SX n SY'|   (x != y)
//   y > x (or y < x):       sum over x in SX of |SY' above (below) x|
// computed by walking the smaller set and rank queries in the larger one
// (binary search in the list slice, or in the materialised set).
static __device__ __noinline__ unsigned long long count_joint(const DevGraph &g, const PgLevel &X, const PgLevel &Y,
                                                              int xl, const int *m, int *bufA, int *bufB, int lane) {
    PgLevel Yp = Y;
    int rel = 0;
    bool excl_xy = false;
    {
        int n = 0;
        for (int i = 0; i < Y.n_lo; ++i)
            if (Y.lo_src[i] == xl) rel = 1; else Yp.lo_src[n++] = Y.lo_src[i];
        Yp.n_lo = (int8_t)n;
        n = 0;
        for (int i = 0; i < Y.n_hi; ++i)
            if (Y.hi_src[i] == xl) rel = -1; else Yp.hi_src[n++] = Y.hi_src[i];
        Yp.n_hi = (int8_t)n;
        n = 0;
        for (int i = 0; i < Y.n_excl; ++i)
            if (Y.excl_src[i] == xl) excl_xy = true; else Yp.excl_src[n++] = Y.excl_src[i];
        Yp.n_excl = (int8_t)n;
    }
    const unsigned long long nX = count_last(g, X, m, lane);
    if (nX == 0) return 0;
    const unsigned long long nY = count_last(g, Yp, m, lane);
    if (nY == 0) return 0;
    if (rel == 0 && !excl_xy) return nX * nY;
    if (rel == 0) {
        // one set inside the other's list: when A is a plain unbounded slice
        // of adj(w) and B intersects adj(w) too, B lies in adj(w), so
        // |A n B| = |B| minus A's excluded images that lie in B
        auto sub = [&](const PgLevel &A, const PgLevel &B, unsigned long long nB, unsigned long long *inter) {
            if (!(is_slice(A) && A.n_lo == 0 && A.n_hi == 0)) return false;
            bool in_b = false;
            for (int i = 0; i < B.n_int; ++i) in_b |= B.int_src[i] == A.int_src[0];
            if (!in_b) return false;
            bool hit = false;
            if (lane < A.n_excl) hit = in_level_set(g, B, m, m[A.excl_src[lane]]);
            *inter = nB - (unsigned long long)__popc(__ballot_sync(PG_FULL, hit));
            return true;
        };
        unsigned long long inter;
        if (sub(X, Yp, nY, &inter) || sub(Yp, X, nX, &inter)) return nX * nY - inter;
    }
    const bool iterX = nX <= nY;
    const PgLevel &I = iterX ? X : Yp;
    const PgLevel &Q = iterX ? Yp : X;
    // elements of I
    Slice is;
    const bool islice = is_slice(I);
    if (islice) is = level_slice(g, I, m);
    else is = Slice{bufA, fill_level(g, I, m, bufA, lane), -1};
    // query structure of Q, and Q's excluded images that sit in its slice
    Slice qs;
    const bool qslice = is_slice(Q);
    int qx[PGP_MAXK];
    int nqx = 0;
    if (qslice) {
        qs = level_slice(g, Q, m);
        const LevelRange r = level_range(Q, m);
        for (int i = 0; i < Q.n_excl; ++i) {
            const int v = m[Q.excl_src[i]];
            if (v > r.lo && v < r.hi && contains_g(qs.p, qs.len, v)) qx[nqx++] = v;
        }
    } else {
        qs = Slice{bufB, fill_level(g, Q, m, bufB, lane), -1};
    }
    // side: count Q elements greater than e, or smaller than e.  Lanes take
    // four elements of I per step (one 16-byte load; a list slice may start
    // mid-group, a scratch set starts aligned) and run four searches at once.
    const bool greater = (iterX && rel > 0) || (!iterX && rel < 0);
    const int off = islice ? (int)(((uintptr_t)is.p >> 2) & 3u) : 0;
    const int4 *v4 = (const int4 *)(is.p - off);
    const int total = is.len + off;
    unsigned long long acc = 0;
    for (int base = 0; base < total; base += 128) {
        const int q = base + 4 * lane;
        int4 t = make_int4(0x7fffffff, 0x7fffffff, 0x7fffffff, 0x7fffffff);
        if (q < total) t = islice ? __ldg(v4 + (q >> 2)) : v4[q >> 2];
        const int e[4] = {t.x, t.y, t.z, t.w};
        bool ok[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) ok[j] = q + j >= off && q + j < total;
        if (islice)
            for (int i = 0; i < I.n_excl; ++i) {
                const int x = m[I.excl_src[i]];
#pragma unroll
                for (int j = 0; j < 4; ++j) ok[j] = ok[j] && e[j] != x;
            }
        if (rel == 0) {
            bool in[4] = {ok[0], ok[1], ok[2], ok[3]};
            if (qslice) {
                in_slice4(g, qs, e, in, false);
            } else {
                int pos[4];
                lower_bound4<false>(qs.p, qs.len, e, pos);
#pragma unroll
                for (int j = 0; j < 4; ++j) in[j] = in[j] && pos[j] < qs.len && qs.p[pos[j]] == e[j];
            }
            for (int i = 0; i < nqx; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) in[j] = in[j] && e[j] != qx[i];
            acc += (unsigned)in[0] + (unsigned)in[1] + (unsigned)in[2] + (unsigned)in[3];
        } else {
            int pos[4];
            if (qslice) lower_bound4<true>(qs.p, qs.len, e, pos);
            else lower_bound4<false>(qs.p, qs.len, e, pos);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (!ok[j]) continue;
                const bool has = pos[j] < qs.len && (qslice ? __ldg(qs.p + pos[j]) : qs.p[pos[j]]) == e[j];
                long long c = greater ? (long long)(qs.len - pos[j] - (has ? 1 : 0)) : (long long)pos[j];
                for (int i = 0; i < nqx; ++i) c -= greater ? (qx[i] > e[j]) : (qx[i] < e[j]);
                acc += (unsigned long long)c;
            }
        }
    }
    acc = warp_sum_u64(acc);
    return rel == 0 ? nX * nY - acc : acc;
}

}  // namespace pgk
