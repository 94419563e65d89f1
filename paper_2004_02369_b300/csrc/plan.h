// Exploration plan: host compiler output and the plain-old-data level
// program the kernels interpret.
//
// A plan holds one "order program" per matching order (Section 4.1: one
// matching order per valid sequence of core vertices).  An order program is a
// list of levels; level 0 binds the start vertex (the task of Section 5.1),
// every later level binds one more pattern vertex, and the last level is not
// enumerated but counted from a set cardinality (non-core completion,
// Section 5.1; counted as C(|S|, g) for a chain of g interchangeable non-core
// vertices).  The candidate set of a level is
//
//   S = ( /\ adj(m[int_src]) ) \ ( \/ adj(m[diff_src]) )
//       restricted to  max(m[lo_src]) < x < min(m[hi_src]),
//       label(x) == label (if label >= 0),  x != m[excl_src]
//
// where m[j] is the data vertex bound at level j.
//
// An anti-vertex check (Section 3.1.2, Section 4.3 "Checking Anti-Vertices")
// runs at the level that binds the last of the vertices it reads: a
// candidate x of that level survives iff
//
//   ( /\ adj(m[int_src]) ) \ { m[excl_src] }  is empty,
//
// int_src being the anti-vertex's neighbours and excl_src the pattern
// neighbours of those neighbours (their images are not witnesses).
//
// A last level marked `joint` belongs to a single non-core vertex y whose
// only ties to the previous level's single non-core vertex x are the
// partial order and injectivity (non-core vertices share no edge or
// anti-edge).  A kernel may then count the pairs (x, y) from the two sets'
// cardinalities and ranks instead of enumerating x; enumerating x and
// counting y level by level gives the same number.  Intersections implement
// true edges and differences anti-edges (Section 4.2); the bounds implement
// the symmetry-breaking partial order on degree-ranked ids (Section 5.2).
#pragma once
#include <stdint.h>

#define PGP_MAXK 8
#define PGP_MAX_ORDERS 5040

struct PgLevel {
    int8_t n_int, n_diff, n_lo, n_hi, n_excl;
    int8_t group;          // last level: the counted chain length g; else 1
    int8_t pattern_vertex; // pattern vertex bound here
    int8_t is_core;
    int8_t out_bounded;    // candidates lie in N+(start): at most max out-degree
    int8_t joint;          // last level only: counted jointly with the previous
                           // level (two single non-core vertices, see plan.cpp)
    int8_t n_anti;         // anti-vertex checks attached to this level
    int8_t int_src[PGP_MAXK];
    int8_t diff_src[PGP_MAXK];
    int8_t lo_src[PGP_MAXK];
    int8_t hi_src[PGP_MAXK];
    int8_t excl_src[PGP_MAXK];
    int32_t label; // -1: any
};

struct PgAntiCheck {
    int8_t level; // checked when this level binds its candidate
    int8_t n_int, n_excl, pad;
    int8_t int_src[PGP_MAXK];
    int8_t excl_src[PGP_MAXK];
};

struct PgOrder {
    int32_t n_levels;
    int32_t n_core;
    PgLevel lv[PGP_MAXK];
    int32_t n_checks;
    int32_t pad;
    PgAntiCheck chk[PGP_MAXK];
};

#ifdef __cplusplus
#include <string>
#include <vector>

struct PgPattern {
    int k = 0;
    uint8_t rel[PGP_MAXK][PGP_MAXK] = {}; // 0 none, 1 edge, 2 anti-edge
    int32_t label[PGP_MAXK] = {-1, -1, -1, -1, -1, -1, -1, -1};
    uint8_t anti_vertex[PGP_MAXK] = {};
};

struct PgPlanHost {
    PgPattern pat;                        // after the vertex-induced expansion
    uint64_t aut = 1;                     // |Aut| restricted to regular vertices
    std::vector<std::pair<int, int>> po;  // symmetry-breaking pairs a < b
    uint32_t core_mask = 0;
    int n_regular = 0;
    int counted_group = 1;
    bool is_clique = false;               // k-clique (edge- or vertex-induced), unlabeled
    int clique_k = 0;                     // k of a k-clique plan (any size), else 0
    bool big_clique = false;              // k-clique with k > PGP_MAXK: no level program,
                                          // counted by the k-clique kernel only (pat unused)
    bool labeled = false;
    bool anti_vertices = false;           // pattern has anti-vertices (checks in the orders)
    std::vector<PgOrder> orders;          // counting program: last level counted
    std::vector<PgOrder> list_orders;     // listing program: every vertex its own level
    double compile_ms = 0.0;
};

// Returns 0 or a PG_E* code; on error `err` holds a message.
int pg_plan_compile(const PgPattern &in, bool vertex_induced, PgPlanHost &out, std::string &err);
#endif
