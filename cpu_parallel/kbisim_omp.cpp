// Multi-core CPU k-bisimulation: a comparison baseline for the GPU library,
// using every host core through OpenMP.  It computes what the paper's
// Alg. 1 computes (Section 4.1; signature of Def. "signature", equivalences
// of Defs. "edge-labeled-fw-bisimulation" and "vertex-labeled-bw-bisimulation"),
// with the same readings as the library: the key of a vertex is its own block
// at level i-1 plus the SET of (direction, edge label, neighbour's block at
// level i-1) over its edges in the chosen direction(s); blocks are numbered by
// the rank of their smallest member.
//
// One round, data-parallel in three steps:
//   1. every vertex builds its signature (gather, sort, drop duplicates) into
//      its own run of a flat array, and a 64-bit digest of it;
//   2. a parallel sort of the vertices by (own block, digest, size, pairs,
//      vertex id) brings equal keys together, compared in full, so the first
//      vertex of every group of equal keys is the group's smallest member;
//   3. those first vertices are marked, a prefix count over vertex ids ranks
//      them, and every vertex takes its group's rank.
// The digest only orders the sort; equality is decided by the pairs
// themselves, so the result never depends on it.
#include <omp.h>
#include <parallel/algorithm>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <vector>

namespace {

struct Csr {
    std::vector<int64_t> row;
    std::vector<int32_t> col;  // neighbour | direction bit 31
    std::vector<int32_t> lab;
};

// Processed edge lists: out-edges, in-edges (transpose) or both, the
// direction in bit 31 of the neighbour word (0 = out, 1 = in).
Csr processed(int64_t n, int64_t m, const int64_t* row, const int32_t* col, const int32_t* lab, int dir) {
    Csr c;
    const bool out = dir == 0 || dir == 2, in = dir == 1 || dir == 2;
    std::vector<int64_t> indeg((size_t)n + 1, 0);
    if (in)
        for (int64_t e = 0; e < m; ++e) ++indeg[(size_t)col[e] + 1];
    c.row.assign((size_t)n + 1, 0);
    for (int64_t v = 0; v < n; ++v)
        c.row[(size_t)v + 1] = c.row[(size_t)v] + (out ? row[v + 1] - row[v] : 0) + (in ? indeg[(size_t)v + 1] : 0);
    c.col.resize((size_t)c.row[(size_t)n]);
    c.lab.resize((size_t)c.row[(size_t)n]);
    std::vector<int64_t> cur(c.row.begin(), c.row.end() - 1);
    if (out) {
#pragma omp parallel for schedule(dynamic, 4096)
        for (int64_t v = 0; v < n; ++v) {
            int64_t w = cur[(size_t)v];
            for (int64_t e = row[v]; e < row[v + 1]; ++e, ++w) {
                c.col[(size_t)w] = col[e];
                c.lab[(size_t)w] = lab ? lab[e] : 0;
            }
            cur[(size_t)v] = w;
        }
    }
    if (in) {
        for (int64_t v = 0; v < n; ++v)
            for (int64_t e = row[v]; e < row[v + 1]; ++e) {
                const int64_t w = cur[(size_t)col[e]]++;
                c.col[(size_t)w] = (int32_t)((uint32_t)v | 0x80000000u);
                c.lab[(size_t)w] = lab ? lab[e] : 0;
            }
    }
    return c;
}

uint64_t mix(uint64_t x) {  // SplitMix64 output function (Steele, Lea & Flood, OOPSLA 2014)
    x ^= x >> 30;
    x *= 0xbf58476d1ce4e5b9ULL;
    x ^= x >> 27;
    x *= 0x94d049bb133111ebULL;
    return x ^ (x >> 31);
}

// Canonical ids from groups of equal keys: `order` sorted so equal keys are
// adjacent and each group starts with its smallest vertex; same(a, b) tells
// whether two vertices have equal keys.  Returns the number of blocks.
template <class Same>
int64_t assign(int64_t n, const std::vector<int32_t>& order, Same same, int32_t* out) {
    std::vector<uint8_t> first((size_t)n, 0);
    std::vector<int32_t> head((size_t)n);  // head of the group at every position
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) first[(size_t)j] = j == 0 || !same(order[(size_t)j - 1], order[(size_t)j]);
    // group heads: a parallel pass per chunk, then carried across chunks
    const int T = omp_get_max_threads();
    std::vector<int32_t> carry((size_t)T + 1, -1);
#pragma omp parallel num_threads(T)
    {
        const int t = omp_get_thread_num();
        const int64_t a = n * t / T, b = n * (t + 1) / T;
        int32_t h = -1;
        for (int64_t j = a; j < b; ++j) {
            if (first[(size_t)j]) h = (int32_t)j;
            head[(size_t)j] = h;
        }
        carry[(size_t)t + 1] = h;
#pragma omp barrier
#pragma omp single
        for (int u = 1; u <= T; ++u)
            if (carry[(size_t)u] < 0) carry[(size_t)u] = carry[(size_t)u - 1];
        for (int64_t j = a; j < b && head[(size_t)j] < 0; ++j) head[(size_t)j] = carry[(size_t)t];
    }
    // ranks of the minima (the group heads) in vertex-id order
    std::vector<uint8_t> is_min((size_t)n, 0);
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j)
        if (first[(size_t)j]) is_min[(size_t)order[(size_t)j]] = 1;
    std::vector<int32_t> rank((size_t)n);
    std::vector<int64_t> part((size_t)T + 1, 0);
#pragma omp parallel num_threads(T)
    {
        const int t = omp_get_thread_num();
        const int64_t a = n * t / T, b = n * (t + 1) / T;
        int64_t c = 0;
        for (int64_t v = a; v < b; ++v) c += is_min[(size_t)v];
        part[(size_t)t + 1] = c;
#pragma omp barrier
#pragma omp single
        for (int u = 1; u <= T; ++u) part[(size_t)u] += part[(size_t)u - 1];
        int64_t r = part[(size_t)t];
        for (int64_t v = a; v < b; ++v) {
            rank[(size_t)v] = (int32_t)r;
            r += is_min[(size_t)v];
        }
    }
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; ++j) out[order[(size_t)j]] = rank[(size_t)order[(size_t)head[(size_t)j]]];
    return part[(size_t)T];
}

}  // namespace

extern "C" {

int cpu_parallel_threads(void) { return omp_get_max_threads(); }

// Levels 0..k into levels[(k+1)*n], counts[k+1], *levels_computed; same
// contract as the library's kb_refine with early stop on or off.
int cpu_parallel_refine(int64_t n, int64_t m, const int64_t* row, const int32_t* col, const int32_t* elabel,
                        const int32_t* vlabel, int dir, int use_vertex_labels, int use_edge_labels, int k,
                        int early_stop, int32_t* levels, int64_t* counts, int* levels_computed) {
    if (n < 0 || m < 0 || k < 0 || dir < 0 || dir > 2) return 1;
    *levels_computed = 0;
    if (n == 0) {
        for (int i = 0; i <= k; ++i) counts[i] = 0;
        return 0;
    }
    const Csr c = processed(n, m, row, col, use_edge_labels ? elabel : nullptr, dir);
    std::vector<int32_t> order((size_t)n);
    // level 0: vertex labels (or one block)
    {
        std::vector<int32_t> key((size_t)n, 0);
        if (use_vertex_labels && vlabel) std::copy(vlabel, vlabel + n, key.begin());
        std::iota(order.begin(), order.end(), 0);
        __gnu_parallel::sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
            return key[(size_t)a] != key[(size_t)b] ? key[(size_t)a] < key[(size_t)b] : a < b;
        });
        counts[0] = assign(n, order, [&](int32_t a, int32_t b) { return key[(size_t)a] == key[(size_t)b]; }, levels);
    }
    std::vector<uint64_t> sig((size_t)c.row[(size_t)n]);
    std::vector<int32_t> cnt((size_t)n);
    std::vector<uint64_t> dig((size_t)n);
    for (int i = 1; i <= k; ++i) {
        const int32_t* prev = levels + (size_t)(i - 1) * (size_t)n;
        int32_t* cur = levels + (size_t)i * (size_t)n;
#pragma omp parallel for schedule(dynamic, 2048)
        for (int64_t v = 0; v < n; ++v) {
            uint64_t* s = sig.data() + c.row[(size_t)v];
            const int64_t d = c.row[(size_t)v + 1] - c.row[(size_t)v];
            for (int64_t j = 0; j < d; ++j) {
                const uint32_t w = (uint32_t)c.col[(size_t)(c.row[(size_t)v] + j)];
                s[j] = ((uint64_t)(uint32_t)c.lab[(size_t)(c.row[(size_t)v] + j)] << 32) | (w & 0x80000000u) |
                       (uint32_t)prev[w & 0x7fffffffu];
            }
            std::sort(s, s + d);
            const int64_t u = std::unique(s, s + d) - s;
            cnt[(size_t)v] = (int32_t)u;
            uint64_t h = mix((uint64_t)u + 0x9e3779b97f4a7c15ULL);
            for (int64_t j = 0; j < u; ++j) h = mix(h ^ s[j]);
            dig[(size_t)v] = h;
        }
        auto less = [&](int32_t a, int32_t b) {
            if (prev[a] != prev[b]) return prev[a] < prev[b];
            if (dig[(size_t)a] != dig[(size_t)b]) return dig[(size_t)a] < dig[(size_t)b];
            if (cnt[(size_t)a] != cnt[(size_t)b]) return cnt[(size_t)a] < cnt[(size_t)b];
            const int r = std::memcmp(sig.data() + c.row[(size_t)a], sig.data() + c.row[(size_t)b],
                                      sizeof(uint64_t) * (size_t)cnt[(size_t)a]);
            if (r != 0) {
                // lexicographic on the words (memcmp's byte order only has to be a total order)
                return r < 0;
            }
            return a < b;
        };
        auto same = [&](int32_t a, int32_t b) {
            return prev[a] == prev[b] && dig[(size_t)a] == dig[(size_t)b] && cnt[(size_t)a] == cnt[(size_t)b] &&
                   std::memcmp(sig.data() + c.row[(size_t)a], sig.data() + c.row[(size_t)b],
                               sizeof(uint64_t) * (size_t)cnt[(size_t)a]) == 0;
        };
        std::iota(order.begin(), order.end(), 0);
        __gnu_parallel::sort(order.begin(), order.end(), less);
        counts[i] = assign(n, order, same, cur);
        *levels_computed = i;
        if (early_stop && counts[i] == counts[i - 1]) {
            for (int j = i + 1; j <= k; ++j) {
                std::memcpy(levels + (size_t)j * (size_t)n, cur, sizeof(int32_t) * (size_t)n);
                counts[j] = counts[i];
            }
            break;
        }
    }
    return 0;
}

}  // extern "C"
