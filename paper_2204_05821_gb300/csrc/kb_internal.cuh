// Internal declarations of the GB300 k-bisimulation library: tile geometry,
// device-side parameter blocks, hashing and pair packing, and the host-side
// launchers implemented in kb_kernels.cu / kb_setup.cu.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kbisim.h"

namespace kb {

// ---------------------------------------------------------------- geometry
// Vertices with more than hub_threshold edges (at most kMaxHubThreshold) are
// hubs, split into chunks of RoundParams::hub_chunk edges (256, 512 or 1024);
// medium vertices keep their pairs in one shared-memory set of 2 x
// kMaxHubThreshold entries.
constexpr int kMaxHubThreshold = 1024;
constexpr int kDefaultHubThreshold = kMaxHubThreshold;
constexpr int kDefaultHubChunk = 512;   // edges per hub-chunk CTA
constexpr int kMaxHubChunk = 1024;
constexpr int kHubThreads = 128;        // threads of a hub-chunk CTA
static_assert(kMaxHubChunk < 65536, "a chunk's edge count is packed in 16 bits");
// Medium vertices up to this degree take a warp each, larger ones a CTA
// (RoundParams::med_split, at most kMaxMedSplit).
constexpr int kMaxMedSplit = 256;
constexpr int kDefaultMedSplit = kMaxMedSplit;
constexpr int kHubFinalThreads = 256;
constexpr int kProbeLimit = 1 << 22;  // bound on block-table probes per vertex
constexpr int kSmallDegree = 32;      // vertices with at most this many edges take the warp kernel
constexpr int kDefaultWarpVerts = 128;

constexpr uint64_t kEmptyPair = ~0ull;  // block field 0x7fffffff never occurs (n <= 2^31-2)

// bits of Counters::err
enum : int32_t { kErrTableFull = 1, kErrInvalid = 2, kErrStage = 4, kErrHubSet = 8 };

struct Counters {
    int32_t err;
    int32_t diff;   // set when two compared levels differ (launch_levels_differ)
    int64_t count;  // blocks at the level just assigned
    int64_t frozen; // vertices frozen for the next round (launch_freeze_clean)
    int64_t med_on; // medium vertices that refine next round (launch_count_refining)
    int64_t hub_on; // hubs that refine next round (launch_count_refining)
    int64_t moved;  // re-keyed vertices whose smallest block member changed (renumbering)
    // vertices re-keyed this round and their edges in the processed
    // direction, per kernel family: small, medium, hub
    int64_t keyed_v[3];
    int64_t keyed_e[3];
    int32_t dense_bad;  // a level-0 key outside [0, kDenseLabels) (launch_dense_labels)
};

// Everything one refinement round reads and writes.
struct RoundParams {
    int64_t n;
    const int64_t* row;   // [n+1] CSR of the processed direction
    const int32_t* col;   // [m_proc] neighbour; bit 31 set for in-edges
    const int32_t* lab;   // [m_proc] edge label or nullptr (all labels 0)
    const int32_t* prev;  // [n] previous level (vertex labels at level 0)
    // Locality order (optional).  perm[v] is v's position in an order that puts
    // often-gathered vertices first; col then holds positions instead of ids and
    // gat holds the previous level in that order, each block named by its
    // smallest member instead of its rank (gat[perm[v]] = smallest member of
    // v's block; any injective naming of blocks gives the same partition), so
    // the per-edge gather of neighbour blocks hits a compact, cache-resident
    // head, and the renumbering rewrites gat only where a block's smallest
    // member changed.  perm == nullptr: col holds ids and the gather reads prev.
    const int32_t* perm;
    int32_t* gat;
    // Generic CSE rounds (Def. "cse"): the subject part of every key, one class
    // id (< n) per vertex; nullptr keys by the own previous block (stratified
    // bisimulation).
    const int32_t* own_key;
    // Incremental refinement (kb_refine_update): only vertices with their bit
    // set in vmask are re-keyed; every other vertex keeps its old grouping at
    // this level: keep_old is the level's old row and kmin[b] the smallest
    // such vertex of old block b.  nullptr when every vertex is re-keyed.
    const uint32_t* vmask;
    const int32_t* keep_old;
    const uint32_t* kmin;
    // Frozen blocks (stratified rounds, whose keys hold the own previous block):
    // a block that cannot change this round, because it has one member (a
    // vertex alone in its previous block stays alone) or because all its
    // members have no edges and it was formed by a signature round (their keys
    // are then (own block, empty set) alike).  Bit v of frozen: v is skipped by
    // the round kernels; frozen_min holds the minima of frozen blocks and
    // starts the round's bitmap of minima; a skipped vertex that is not a
    // minimum keeps its slot_of entry of the round that formed its block.  The
    // renumbering sets bit b of shared for every block minimum b that another
    // vertex points to.  All nullptr when every vertex is re-keyed.
    const uint32_t* frozen;
    const uint32_t* frozen_min;
    uint32_t* shared;
    // Clean blocks (with frozen blocks).  minof[v] is the smallest member of
    // v's block whenever v is not that member; the renumbering writes it for
    // every re-keyed vertex, and a frozen vertex keeps it.  moved (when set)
    // receives bit v for every re-keyed vertex whose smallest block member
    // changed this round (read against bitmap_prev, the previous level's block
    // minima, and minof), counted in ctr->moved; under the locality order the
    // bit goes to v's position, which is what the neighbour ids hold.
    uint32_t* minof;
    uint32_t* moved;
    int32_t hub_threshold;
    int32_t small_max;    // largest degree of the small-vertex kernel (<= kSmallDegree, <= hub_threshold)
    int32_t warp_verts;   // vertices per warp task of the small-vertex kernel
    int32_t hub_chunk;    // edges per hub-chunk CTA: 256, 512 or 1024
    int32_t med_split;    // medium vertices up to this degree take a warp, larger a CTA (1..kMaxMedSplit)
    int32_t hash_mode;
    uint32_t epoch;       // 1..255, tags this round's table entries
    uint64_t* table;      // [mask+1] block table
    uint64_t mask;
    int32_t* slot_of;     // [n] table slot of every vertex; 0x80000000|own for an empty signature
    uint64_t* emin;       // [n] smallest vertex with an empty signature per own block:
                          //     (ehigh << 32) | vertex, ehigh decreasing from round to round
    uint32_t ehigh;
    uint32_t* bitmap;     // [n/32+1] bit v set iff v is the smallest member of its block
    Counters* ctr;
    // medium vertices (small_max < degree <= hub_threshold), processed by the tile kernel
    const int32_t* med_v;
    int64_t n_med;
    // hubs (vertices with more than hub_threshold edges)
    int32_t n_hubs;
    const int32_t* hub_v;          // [n_hubs] ascending
    const int64_t* hub_chunk_off;  // [n_hubs+1]
    const int32_t* chunk_hub;      // [total chunks] hub index of every chunk
    const uint64_t* chunk_ext;     // [total chunks] (first edge << 16) | edges of every chunk
    const int64_t* hub_set_off;    // [n_hubs+1] open-addressing set per hub (hub_set_capacity slots)
    uint64_t* hub_sets;
    uint64_t* hub_acc;  // [n_hubs] sum of pair mixes over unique pairs
    uint32_t* hub_cnt;  // [n_hubs] unique pairs
    // several graphs at once (batched refinement, serving); all null for one graph
    const int32_t* vgraph;     // [n] graph of every vertex
    const uint8_t* gactive;    // [G] the graph refines this round (else it keeps its partition)
    const int64_t* voff;       // [G+1] first vertex of every graph
    int32_t n_graphs;
    const uint8_t* gmode;      // [G] 1: the graph computes its level 0 this round (serving), or nullptr
    const int32_t* vlab;       // [n] vertex labels read by graphs in level-0 mode, or nullptr (all 0)
    const uint32_t* bitmap_prev;  // block minima of the previous level (batched: kept by inactive graphs)
    const uint32_t* gbase_prev;   // [G+1] rank of every graph's first vertex at the previous level
    uint32_t* gbase_cur;          // [G+1] the same at this level (written by the renumbering)
};

__host__ __device__ __forceinline__ bool batched(const RoundParams& p) { return p.vgraph != nullptr; }

// The subject part of vertex v's key in a signature round.
__host__ __device__ __forceinline__ int32_t own_of(const RoundParams& p, int64_t v) {
    return p.own_key ? p.own_key[v] : p.prev[v];
}

// The array the per-edge gather reads through col (see RoundParams::perm).
__host__ __device__ __forceinline__ const int32_t* gather_base(const RoundParams& p) {
    return p.perm ? p.gat : p.prev;
}

// The previous block of neighbour word w (bit 31: direction).
__device__ __forceinline__ int32_t gather_block(const RoundParams& p, int32_t w) {
    return __ldg(gather_base(p) + (w & 0x7fffffff));
}

// ---------------------------------------------------------------- hashing
// SplitMix64 output function (Steele, Lea & Flood, "Fast splittable
// pseudorandom number generators", OOPSLA 2014): a bijective 64-bit mixer.
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t x) {
    x ^= x >> 30;
    x *= 0xbf58476d1ce4e5b9ULL;
    x ^= x >> 27;
    x *= 0x94d049bb133111ebULL;
    x ^= x >> 31;
    return x;
}

// A signature pair (direction d, edge label l, neighbour block b) as one
// 64-bit word: label in bits 63..32, d in bit 31, b in bits 30..0.
__device__ __forceinline__ uint64_t pack_pair(int32_t label, uint32_t col_word, int32_t block) {
    return ((uint64_t)(uint32_t)label << 32) | (uint64_t)(col_word & 0x80000000u) | (uint64_t)(uint32_t)block;
}

__device__ __forceinline__ uint64_t pair_mix(uint64_t p) { return mix64(p ^ 0x9e3779b97f4a7c15ULL); }

// A hub's global dedup set: 1.5 x its degree (at most two thirds full), any
// size, home slot by multiply-shift range reduction of the pair mix.
__host__ __device__ __forceinline__ int64_t hub_set_capacity(int64_t degree) {
    const int64_t c = degree + degree / 2 + 4;
    return c < 64 ? 64 : (c & ~(int64_t)3);
}

__device__ __forceinline__ uint64_t hub_set_home(uint64_t pr, uint64_t cap) {
    return __umul64hi(pair_mix(pr), cap);
}

// Slot of (local vertex j, pair p) in a shared dedup set.
__device__ __forceinline__ uint32_t set_slot(uint64_t p, uint32_t j) {
    return (uint32_t)(mix64(p + 0x632be59bd9b4e019ULL * (uint64_t)(j + 1)) >> 20);
}

// Hash of a vertex key (own previous block, signature set).  The set enters
// through an order-independent sum of pair mixes over its distinct pairs and
// its size.  hash_mode 1 keeps only the own block (forces collisions).
__device__ __forceinline__ uint64_t vertex_hash(int32_t own, uint32_t cnt, uint64_t acc, int mode) {
    uint64_t base = mix64(((uint64_t)(uint32_t)own << 32) ^ 0x5851f42d4c957f2dULL);
    if (mode == 1) return base;
    return mix64(base ^ mix64(acc + 0xd6e8feb86659fd93ULL * ((uint64_t)cnt + 1)));
}

__device__ __forceinline__ uint32_t table_hi(uint64_t h, uint32_t epoch) {
    return (epoch << 24) | (uint32_t)(h >> 40);
}

// ---------------------------------------------------------------- launchers
// Signature rounds (kb_kernels.cu).  The round's bitmap of block minima starts
// as p.frozen_min (or empty).
void launch_clear_round(const RoundParams& p, cudaStream_t s);
// Empty the hub sets of the hubs that refine this round.
void launch_clear_hub_sets(const RoundParams& p, int64_t total_slots, cudaStream_t s);
// Clean blocks (RoundParams::minof).  After the renumbering of level i
// (`level`, whose minima are in p.bitmap, moved vertices in `moved`): mark =
// blocks of level i holding a vertex with an edge to a moved vertex (bit =
// level-i id; a vertex above max_scan edges counts as such).  Only vertices
// that are neither alone in their block (bitmap & ~shared) nor edgeless are
// scanned, and nothing when more than an eighth of the vertices moved.
// stable_count >= 0: the pass does nothing when this round's count equals it
// (a stable round under early stop is the last one).
void launch_dirty_blocks(const RoundParams& p, const uint32_t* edgeless, const uint32_t* moved, const int32_t* level,
                         int32_t max_scan, uint32_t* mark, cudaStream_t s, int64_t stable_count = -1);
// After the renumbering (single-graph stratified rounds): the frozen blocks
// of the next round.  A vertex is frozen when it is alone in its block (a
// minimum in bitmap that no other vertex marked in shared), edgeless
// (edgeless != null: from the first signature round on, a block holding an
// edgeless vertex holds only edgeless vertices with one previous block), or
// in a level-i block without a mark bit (mark != null, unless more than an
// eighth of the vertices moved).  frozen_min receives the minima of frozen
// blocks; shared keeps exactly their marks; ctr->frozen counts the frozen
// vertices.
// Serving (vgraph, gmode given): the vertices of graphs that computed their
// level 0 in this step are not frozen by the edgeless rule.
void launch_freeze_clean(int64_t n, const uint32_t* bitmap, uint32_t* shared, const uint32_t* edgeless,
                         const int32_t* level, const uint32_t* mark, uint32_t* frozen, uint32_t* frozen_min,
                         Counters* ctr, cudaStream_t s, const int32_t* vgraph = nullptr,
                         const uint8_t* gmode = nullptr, int64_t stable_count = -1);
// Clear bits a..b-1 of a bitmap.
void launch_clear_bits(uint32_t* words, int64_t a, int64_t b, cudaStream_t s);
// The vertices this round re-keys (not in p.frozen) and their edges, per
// kernel family, into ctr->keyed_v / keyed_e (work accounting only).
void launch_round_work(const RoundParams& p, cudaStream_t s);
// After launch_freeze_clean: the medium vertices and hubs that are not frozen, into
// ctr->med_on and ctr->hub_on (their kernels are skipped when none refine).
void launch_count_refining(const RoundParams& p, const uint32_t* frozen, Counters* ctr, cudaStream_t s);
// Bit v set iff v has no edges in the processed CSR.
void launch_edgeless_bits(int64_t n, const int64_t* row, uint32_t* bits, cudaStream_t s);
// compact: windows are packed from the vertices that refine (worth it when
// many are frozen), else from consecutive vertices.
void launch_small_round(const RoundParams& p, bool level0, bool compact, cudaStream_t s);
void launch_medium_round(const RoundParams& p, cudaStream_t s);  // kb_medium.cu
// Per-device kernel attributes (shared-memory carveouts); call once per device
// before the first launch and outside any stream capture.
void set_medium_kernel_attributes();
void launch_hub_chunk(const RoundParams& p, int64_t total_chunks, cudaStream_t s);
void launch_hub_final(const RoundParams& p, cudaStream_t s);
// Canonical renumbering: prefix of block minima, then ids.
// rank: (n/32 + 2) words, rank[w] = (minima before word w, minima bits of word w).
// stable_count >= 0 (frozen-block rounds under early stop): a round whose
// count equals it copies the previous level (it is the last round).
void launch_renumber(const RoundParams& p, uint2* rank, uint32_t* scan_tmp, int32_t* out, cudaStream_t s,
                     int64_t stable_count = -1);
size_t scan_tmp_words(int64_t n_items);
// Level 0 of one graph whose keys (vertex labels, or a starting partition)
// are all in [0, kDenseLabels): the label partition straight from each
// label's smallest vertex, without the block table.  launch_dense_labels
// lowers lmin[label] (all ones for an unused label) to the label's smallest
// vertex and sets ctr->dense_bad if some key lies outside the range (the
// caller then takes the general path).  launch_dense_level0 then writes what
// the general level-0 pass writes: the minima bitmap and the shared-block
// marks of p, the rank words, ctr->count, the level (out), minof and the
// locality order's copy gat.  lpair: kDenseLabels (minimum, id) words of scratch.
constexpr int kDenseLabels = 8192;
void launch_dense_labels(int64_t n, const int32_t* key, uint32_t* lmin, Counters* ctr, cudaStream_t s);
void launch_dense_level0(const RoundParams& p, const int32_t* key, const uint32_t* lmin, uint2* lpair, uint2* rank,
                         uint32_t* scan_tmp, int32_t* out, cudaStream_t s);
void launch_fill_i32(int32_t* out, int64_t n, int32_t value, cudaStream_t s);
// Batched runs: inactive graphs keep the block minima of the previous level.
void launch_carry_minima(const RoundParams& p, cudaStream_t s);
// Batched runs: per-graph stop test after round `round` (count unchanged with
// early stop, or the graph's own k reached) -> gactive cleared, glast set.
void launch_graph_stop(const RoundParams& p, int round, const int32_t* k_per_graph, const uint8_t* early,
                       uint8_t* gactive, int32_t* glast, int32_t* sticky_err, cudaStream_t s);
// Batched runs: row -= gbase[graph of v] (union-global ids to graph-local ids).
void launch_localize(int32_t* row, int64_t n, const int32_t* vgraph, const uint32_t* gbase, cudaStream_t s);
// vgraph[v] = graph owning v
void launch_vertex_graph(const int64_t* voff, int32_t G, int64_t n, int32_t* vgraph, cudaStream_t s);

// Setup (kb_setup.cu)
void launch_validate(int64_t n, int64_t m, const int64_t* row, const int32_t* col, Counters* ctr,
                     cudaStream_t s);
// in-degree histogram: deg[w] += 1 per edge (deg must be zeroed)
void launch_in_degree(int64_t m, const int32_t* col, int64_t* deg, cudaStream_t s);
// exclusive prefix of n int64 values into out[0..n] (out[n] = total); in and out may alias
void launch_scan_i64(const int64_t* in, int64_t n, int64_t* out, int64_t* tmp, cudaStream_t s);
size_t scan_i64_tmp(int64_t n);
// Build the processed CSR for IN (include_out = 0) or BOTH (include_out = 1):
//   row_p[v] = (include_out ? row[v] : 0) + in_prefix[v]
void launch_build_csr(int64_t n, int64_t m, const int64_t* row, const int32_t* col, const int32_t* lab,
                      const int64_t* in_prefix, int include_out, int64_t* row_p, int32_t* col_p,
                      int32_t* lab_p, int64_t* cursor, cudaStream_t s);
// Compact the vertices with more than thr edges (unordered) into out_v with
// their degrees in out_deg; count in *n_out.
void launch_find_hubs(int64_t n, const int64_t* row, int32_t thr, int32_t* out_v, int64_t* out_deg,
                      int32_t* n_out, cudaStream_t s);
// Append the vertices with lo < degree <= hi to out (order within a warp
// preserved); count in *n_out.
void launch_chunk_ext(int64_t chunks, const int32_t* chunk_hub, const int32_t* hub_v, const int64_t* chunk_off,
                      const int64_t* row, int32_t chunk, uint64_t* out, cudaStream_t s);
void launch_locality_order(int64_t n, int64_t m, const int32_t* col, uint32_t* cnt, unsigned long long* hist,
                           int32_t* perm, cudaStream_t s);
void launch_remap_cols(int64_t m, const int32_t* col, const int32_t* perm, int32_t* out, cudaStream_t s);
// Rank of every set bit of a bitmap: prefix[w] = set bits before word w, the
// total in ctr->count (kb_kernels.cu).
void launch_bitmap_rank(const uint32_t* bitmap, int64_t nw, uint32_t* scan_tmp, uint32_t* prefix, Counters* ctr,
                        cudaStream_t s);
// Summary graph (kb_summary.cu)
struct SummaryParams {
    int64_t n, m;
    const int64_t* row;         // [n+1] the caller's out-edge CSR
    const int32_t* col;         // [m]
    const int32_t* lab;         // [m] or nullptr (every label reads 0)
    int32_t dir;                // 0: x = source, y = target; 1: reversed
    const int32_t* lsrc;        // [n] block of x
    const int32_t* ldst;        // [n] block of y
    unsigned long long* table;  // [2 * cap] 16-byte slots; both words zero = empty
    unsigned long long* first;  // [cap] smallest edge index of the slot's triple
    uint64_t mask;              // cap - 1
    uint32_t* bitmap;           // [m/32+1] edges that are first occurrences
    Counters* ctr;
};
void launch_summary_insert(const SummaryParams& q, cudaStream_t s);
void launch_summary_mark(const SummaryParams& q, cudaStream_t s);
void launch_summary_emit(const SummaryParams& q, const uint32_t* prefix, int32_t* out_src, int32_t* out_label,
                         int32_t* out_dst, cudaStream_t s);
// fill out[i] = i (kb_kernels.cu)
void launch_iota_i32(int32_t* out, int64_t n, cudaStream_t s);
// ctr->diff |= (a != b) over n entries (kb_kernels.cu)
void launch_levels_differ(const int32_t* a, const int32_t* b, int64_t n, Counters* ctr, cudaStream_t s);
// Incremental refinement (kb_update.cu)
void launch_dirty_from_moved(int64_t n, int64_t m, const int64_t* row, const int32_t* col, const uint32_t* moved,
                             uint32_t* dirty, cudaStream_t s);
void launch_or_words(int64_t nw, const uint32_t* a, const uint32_t* b, uint32_t* out, cudaStream_t s);
void launch_work_set(int64_t n, const int32_t* prev, const uint32_t* dirty, uint8_t* flag, uint32_t* wmask,
                     unsigned long long* count, cudaStream_t s);
void launch_keep_min(int64_t n, const uint32_t* wmask, const int32_t* old, uint32_t* kmin, cudaStream_t s);
void launch_keep_bits(int64_t n, const uint32_t* wmask, const int32_t* old, const uint32_t* kmin, uint32_t* bitmap,
                      cudaStream_t s);
void launch_moved(int64_t n, const uint32_t* wmask, const int32_t* old, const int32_t* cur, int32_t* ranges,
                  uint32_t* moved, cudaStream_t s);
void launch_check_ids(int64_t n, const int32_t* a, Counters* ctr, cudaStream_t s);
// *out += vertices in the blocks of `level` that hold a vertex of ids
// (touched: a zeroed bitmap of n bits; ids and level values in [0, n)).
void launch_touched_size(int64_t n, int64_t count, const int32_t* ids, const int32_t* level, uint32_t* touched,
                         unsigned long long* out, cudaStream_t s);
// *out += set bits of words[0..nw) (kb_kernels.cu)
void launch_count_bits(const uint32_t* words, int64_t nw, int64_t* out, cudaStream_t s);
void launch_set_bits(int64_t n, int64_t count, const int32_t* ids, uint32_t* bits, Counters* ctr, cudaStream_t s);
void launch_classify(int64_t n, const int64_t* row, int32_t lo, int32_t hi, int32_t* out, int64_t* n_out,
                     cudaStream_t s);
// Copy row src of the level store to the rows [first, last] of levels.
void launch_copy_rows(int32_t* levels, int64_t n, int src, int first, int last, cudaStream_t s);

// ---- serving arena (kb_serve.cu)
// Copy vertices [src_vbase, src_vbase+n] and edges [src_ebase, src_ebase+m)
// of a CSR into an arena at dst_vbase / dst_ebase, rebasing row offsets and
// neighbour ids (the in-edge bit of a neighbour id is kept).  Labels may be
// null (written as 0).  When sB and dB are given, block ids move too, as
// sB - b_sub + b_add.
struct PlaceArgs {
    const int64_t* srow;
    const int32_t* scol;
    const int32_t* slab;
    const int32_t* svlab;
    const int32_t* sB;
    int64_t* drow;
    int32_t* dcol;
    int32_t* dlab;
    int32_t* dvlab;
    int32_t* dB;
    int64_t n, m;
    int64_t src_vbase, dst_vbase, src_ebase, dst_ebase;
    uint32_t b_sub, b_add;
};
void launch_place(const PlaceArgs& a, cudaStream_t s);
// For every arena vertex whose graph g has slot_row[g] >= 0:
// slot_levels[g][slot_row[g] * slot_n[g] + (v - voff[g])] = B[v] - gbase[g].
void launch_emit(int64_t n, const int32_t* vgraph, const int32_t* B, const uint32_t* gbase, int32_t* const* slot_levels,
                 const int32_t* slot_row, const int64_t* slot_n, const int64_t* voff, cudaStream_t s);

}  // namespace kb
