// CPU oracle for stratified k-bisimulation by signature refinement.
//
// TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
// restatement of what the GPU library computes.  Only the tests, the smoke
// check and the benchmark's CPU-baseline leg may load it; the library never
// does.  It shares no code, header, table or constant with the CUDA path: no
// hashing, no device-style table, its own transpose.
//
// What it computes (paper Section 3.2-3.3 and Section 4.1):
//   * Level 0 (Def. "vertex-labeled-bw-bisimulation", first bullet; Alg. 1
//     initialisation): P_0 groups vertices by vertex label when vertex labels
//     are used, otherwise P_0 = {V}.
//   * Level i >= 1 (Defs. "edge-labeled-fw-bisimulation" and
//     "vertex-labeled-bw-bisimulation", second bullet; Def. "signature"):
//     u and v share a block of P_i iff they share a block of P_{i-1} and their
//     signatures w.r.t. P_{i-1} are equal, where the signature of x is the SET
//     { (d, l(e), B_{i-1}(y)) : e an edge of x in direction d, y its other end }.
//     d is 0 for out-edges and 1 for in-edges; l(e) is 0 when edge labels are
//     not used.
//   * Block numbering is canonical: the blocks of each level are numbered
//     0, 1, 2, ... in increasing order of their smallest member vertex.
//     Visiting vertices in increasing id order and numbering keys at first
//     sight gives exactly that numbering.
//   * Early stop (Alg. 1, the block-count test and its footnote: blocks only
//     split): when count_i == count_{i-1} the partition is stable; levels
//     i+1..k are copies of level i.
//   * Summary graph (Sec. "Graph Summaries for Bisimulation"): the distinct
//     (block, label, block) triples over the edges, see oracle_summary.
//
// Readings where the paper is silent or ambiguous (each is also listed in the
// design notes): the key includes the vertex's own previous block (needed once
// P_0 is the label partition); one label per vertex and per edge; duplicate
// pairs count once (set semantics); the BOTH direction is the union of the
// out- and in-signature tagged by direction; k = 0 returns level 0 only.

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <set>
#include <tuple>
#include <utility>
#include <vector>

namespace {

typedef std::tuple<int32_t, int32_t, int32_t> Pair;            // (d, label, block)
typedef std::pair<int32_t, std::vector<Pair> > Key;             // (own block, signature set)

struct EdgeLists {
    // For each vertex, the (other end, label) of its edges in one direction.
    std::vector<std::vector<std::pair<int32_t, int32_t> > > adj;
};

EdgeLists out_lists(int64_t n, const int64_t* row, const int32_t* col, const int32_t* lab) {
    EdgeLists L;
    L.adj.resize((size_t)n);
    for (int64_t v = 0; v < n; ++v)
        for (int64_t e = row[v]; e < row[v + 1]; ++e)
            L.adj[(size_t)v].push_back(std::make_pair(col[e], lab ? lab[e] : 0));
    return L;
}

EdgeLists in_lists(int64_t n, const int64_t* row, const int32_t* col, const int32_t* lab) {
    EdgeLists L;
    L.adj.resize((size_t)n);
    for (int64_t v = 0; v < n; ++v)
        for (int64_t e = row[v]; e < row[v + 1]; ++e)
            L.adj[(size_t)col[e]].push_back(std::make_pair((int32_t)v, lab ? lab[e] : 0));
    return L;
}

}  // namespace

extern "C" {

// Returns 0 on success, -1 on invalid arguments.
//   row, col, elabel, vlabel : host CSR by source (elabel / vlabel may be NULL)
//   dir                      : 0 out-edges, 1 in-edges, 2 both
//   levels                   : int32[(k+1)*n], row i = canonical block of every vertex at level i
//   counts                   : int64[k+1], number of blocks per level
//   levels_computed          : last level actually refined (levels after it are copies)
//   initial                  : optional int32[n]; when given, P_0 is the partition
//                              it induces (equal values = same block) instead of the
//                              label partition -- refinement of an arbitrary starting
//                              partition (the relational coarsest partition setting,
//                              Def. "rel-coar-par-prob", stratified to k rounds).
//   subject                  : the subject part of the key (Def. "cse": v ~s v').
//                              0: the vertex's own block at the previous level
//                              (stratified k-bisimulation, Section 3); 1: T (no
//                              condition); 2: equal vertex labels (the paper's OC
//                              type cluster); 3: id (the vertex itself).  With
//                              1..3 the levels are the chained CSE^i = (~s, ~p,
//                              CSE^{i-1}) of Def. "chaining-parameterization",
//                              CSE^0 = P_0, ~p = id with edge labels, T without.
//                              Those levels need not refine each other, so early
//                              stop compares whole levels instead of counts.
int oracle_refine_cse(int64_t n, int64_t m, const int64_t* row, const int32_t* col,
                      const int32_t* elabel, const int32_t* vlabel, int dir,
                      int use_vertex_labels, int use_edge_labels, int subject, int k, int early_stop,
                      const int32_t* initial,
                      int32_t* levels, int64_t* counts, int* levels_computed) {
    if (n < 0 || m < 0 || k < 0 || dir < 0 || dir > 2 || subject < 0 || subject > 3) return -1;
    if (n > 0 && (!row || !levels || !counts)) return -1;
    if (m > 0 && !col) return -1;
    if (n > 0 && (row[0] != 0 || row[n] != m)) return -1;
    for (int64_t v = 0; v < n; ++v)
        if (row[v + 1] < row[v]) return -1;
    for (int64_t e = 0; e < m; ++e)
        if (col[e] < 0 || col[e] >= n) return -1;

    const int32_t* lab = use_edge_labels ? elabel : nullptr;
    EdgeLists outL, inL;
    if (dir == 0 || dir == 2) outL = out_lists(n, row, col, lab);
    if (dir == 1 || dir == 2) inL = in_lists(n, row, col, lab);

    // Level 0.
    {
        std::map<int32_t, int32_t> ids;
        for (int64_t v = 0; v < n; ++v) {
            int32_t label = initial ? initial[v] : ((use_vertex_labels && vlabel) ? vlabel[v] : 0);
            std::map<int32_t, int32_t>::iterator it = ids.find(label);
            if (it == ids.end()) it = ids.insert(std::make_pair(label, (int32_t)ids.size())).first;
            levels[v] = it->second;
        }
        counts[0] = (int64_t)ids.size();
    }
    if (levels_computed) *levels_computed = 0;

    for (int i = 1; i <= k; ++i) {
        const int32_t* prev = levels + (size_t)(i - 1) * (size_t)n;
        int32_t* cur = levels + (size_t)i * (size_t)n;
        std::map<Key, int32_t> ids;
        for (int64_t v = 0; v < n; ++v) {
            std::vector<Pair> sig;
            if (dir == 0 || dir == 2)
                for (size_t t = 0; t < outL.adj[(size_t)v].size(); ++t)
                    sig.push_back(Pair(0, outL.adj[(size_t)v][t].second, prev[outL.adj[(size_t)v][t].first]));
            if (dir == 1 || dir == 2)
                for (size_t t = 0; t < inL.adj[(size_t)v].size(); ++t)
                    sig.push_back(Pair(1, inL.adj[(size_t)v][t].second, prev[inL.adj[(size_t)v][t].first]));
            std::sort(sig.begin(), sig.end());
            sig.erase(std::unique(sig.begin(), sig.end()), sig.end());
            int32_t s = prev[v];
            if (subject == 1) s = 0;
            if (subject == 2) s = vlabel ? vlabel[v] : 0;
            if (subject == 3) s = (int32_t)v;
            Key key(s, sig);
            std::map<Key, int32_t>::iterator it = ids.find(key);
            if (it == ids.end()) it = ids.insert(std::make_pair(key, (int32_t)ids.size())).first;
            cur[v] = it->second;
        }
        counts[i] = (int64_t)ids.size();
        if (levels_computed) *levels_computed = i;
        const bool same = subject == 0 ? counts[i] == counts[i - 1]
                                       : std::memcmp(cur, prev, sizeof(int32_t) * (size_t)n) == 0;
        if (early_stop && same) {
            for (int j = i + 1; j <= k; ++j) {
                std::memcpy(levels + (size_t)j * (size_t)n, cur, sizeof(int32_t) * (size_t)n);
                counts[j] = counts[i];
            }
            break;
        }
    }
    return 0;
}

int oracle_refine_init(int64_t n, int64_t m, const int64_t* row, const int32_t* col,
                       const int32_t* elabel, const int32_t* vlabel, int dir,
                       int use_vertex_labels, int use_edge_labels, int k, int early_stop,
                       const int32_t* initial,
                       int32_t* levels, int64_t* counts, int* levels_computed) {
    return oracle_refine_cse(n, m, row, col, elabel, vlabel, dir, use_vertex_labels, use_edge_labels, 0, k,
                             early_stop, initial, levels, counts, levels_computed);
}

int oracle_refine(int64_t n, int64_t m, const int64_t* row, const int32_t* col,
                  const int32_t* elabel, const int32_t* vlabel, int dir,
                  int use_vertex_labels, int use_edge_labels, int k, int early_stop,
                  int32_t* levels, int64_t* counts, int* levels_computed) {
    return oracle_refine_init(n, m, row, col, elabel, vlabel, dir, use_vertex_labels,
                              use_edge_labels, k, early_stop, nullptr, levels, counts,
                              levels_computed);
}

// Summary graph of a partition (Sec. "Graph Summaries for Bisimulation": one
// summary vertex per block, a labelled summary edge from block b to block c
// when the vertices of b have an edge with that label into c).  Every graph
// edge v -> w with label l yields the triple (src_level[x], l or 0, dst_level[y])
// where x -> y is the edge in the processed direction (out: x = v, y = w; in:
// x = w, y = v); the output lists each distinct triple once, in the order of
// its first occurrence in the edge list (sources ascending, then CSR order).
// With src_level = P_i and dst_level = P_{i-1} of a stratified refinement this
// is the paper's layer of summary edges between the two levels; with both the
// same partition it is the quotient graph.  Returns the number of triples, or
// -1 for a direction other than out (0) or in (1).
int64_t oracle_summary(int64_t n, const int64_t* row, const int32_t* col, const int32_t* elabel, int dir,
                       int use_edge_labels, const int32_t* src_level, const int32_t* dst_level,
                       int32_t* out_src, int32_t* out_label, int32_t* out_dst) {
    if (dir != 0 && dir != 1) return -1;
    std::set<std::tuple<int32_t, int32_t, int32_t>> seen;
    int64_t count = 0;
    for (int64_t v = 0; v < n; ++v) {
        for (int64_t e = row[v]; e < row[v + 1]; ++e) {
            const int64_t w = col[e];
            const int64_t x = dir == 0 ? v : w;
            const int64_t y = dir == 0 ? w : v;
            const int32_t l = (use_edge_labels && elabel) ? elabel[e] : 0;
            const std::tuple<int32_t, int32_t, int32_t> t(src_level[x], l, dst_level[y]);
            if (seen.insert(t).second) {
                out_src[count] = std::get<0>(t);
                out_label[count] = std::get<1>(t);
                out_dst[count] = std::get<2>(t);
                ++count;
            }
        }
    }
    return count;
}

}  // extern "C"
