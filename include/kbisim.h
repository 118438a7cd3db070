/*
 * kbisim.h -- C ABI of the GB300 stratified k-bisimulation library.
 *
 * The library partitions the vertices of a labelled directed graph into the
 * blocks of its stratified k-bisimulation, for every level 0..k, by signature
 * refinement (paper Section 4.1, Alg. 1, with the signature of Def.
 * "signature" and the equivalences of Defs. "fw-bisim", "bw-bisim",
 * "edge-labeled-fw-bisimulation" and "vertex-labeled-bw-bisimulation"):
 *
 *   level 0   P_0 = vertices grouped by vertex label (or {V} without labels);
 *   level i   u, v share a block iff they shared one at level i-1 and
 *             { (d, edge label, block_{i-1}(w)) : edges (v, w) in direction d }
 *             is the same set for both.
 *
 * Every level is returned with canonical block ids: the blocks of a level are
 * numbered 0, 1, 2, ... by increasing smallest member vertex id.  Results are
 * exact integers and do not depend on hashing, table size, thread timing or
 * batch composition.
 *
 * Conventions for every call:
 *   - Every pointer documented "device" must point to memory of the context's
 *     device; "host" pointers to ordinary host memory.  The caller owns all
 *     inputs and outputs and keeps them alive until the call returns.
 *   - Calls run on the context's stream.  Calls that return counts on the
 *     host synchronise that stream before returning; all others are
 *     asynchronous.
 *   - No call throws, aborts or traps.  Errors are returned as kb_status; a
 *     human-readable message for the last error is kb_last_error(ctx).
 *   - Vertex ids and block ids are int32, so n <= 2^31 - 2.  Edge offsets are
 *     int64.
 */
#ifndef KBISIM_H_
#define KBISIM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    KB_OK = 0,
    KB_ERR_INVALID_ARG = 1,   /* bad sizes, null pointers, non-monotone offsets, ids out of range */
    KB_ERR_OOM = 2,           /* device allocation failed or caller workspace too small */
    KB_ERR_TABLE_FULL = 3,    /* a key needed more than 2^22 probes of the block table; nothing is
                                 retried.  The table holds n / load_factor slots, so this needs a
                                 clustered hash, e.g. hash_mode 1 on a previous block with millions
                                 of distinct signatures */
    KB_ERR_TIMEOUT = 4,       /* a bounded device wait gave up */
    KB_ERR_CUDA = 5,          /* a CUDA runtime call failed */
    KB_ERR_DEVICE_CHECK = 6,  /* a device-side consistency check failed */
    KB_ERR_NOT_FOUND = 7      /* unknown server ticket */
} kb_status;

typedef enum { KB_DIR_OUT = 0, KB_DIR_IN = 1, KB_DIR_BOTH = 2 } kb_direction;

/* A graph in out-edge CSR form.  All arrays are DEVICE pointers owned by the
 * caller (for kb_refine_host: HOST pointers).
 *   n               number of vertices, 0 <= n <= 2^31 - 2
 *   m               number of edges, 0 <= m <= 2^45 (KB_ERR_INVALID_ARG beyond)
 *   row_offsets     int64[n+1], row_offsets[0] = 0, non-decreasing, row_offsets[n] = m;
 *                   the out-edges of v are row_offsets[v] .. row_offsets[v+1]-1
 *   col_indices     int32[m], target of each edge, 0 <= target < n (self loops and
 *                   parallel edges allowed: a multigraph)
 *   edge_labels     int32[m] or NULL; one label per edge, any int32 value.  The paper
 *                   maps edges to label SETS (Def. "multi-relational-labeled-property-
 *                   graph"); a caller interns each set to one int32.
 *   vertex_labels   int32[n] or NULL; one label per vertex, any int32 value. */
typedef struct {
    int64_t n;
    int64_t m;
    const int64_t* row_offsets;
    const int32_t* col_indices;
    const int32_t* edge_labels;
    const int32_t* vertex_labels;
} kb_graph;

/* Refinement options.  Start from kb_options_default() (or a preset) and
 * change fields; zero in a tuning field means "library default".
 *   direction          out-edges (forward), in-edges (backward) or both
 *   use_vertex_labels  level 0 groups by vertex label (else P_0 = {V})
 *   use_edge_labels    pairs carry the edge label (else every label reads 0)
 *   early_stop         stop once a round keeps the block count (paper Alg. 1, the
 *                      count test); later levels are then copies
 *   load_factor        block-table load factor in (0, 0.9]; 0 -> 0.5 (the table has
 *                      a power of two of slots, at most 2^31: above 2^30 vertices it
 *                      is fuller than asked)
 *   hub_threshold      vertices with more edges than this (in the chosen direction)
 *                      take the multi-CTA hub path; 0 -> default 1024; at most 1024
 *   hash_mode          0: full 64-bit signature hash.  1: weak hash of the previous
 *                      block only, which forces collisions (tests the full
 *                      signature compare); results are identical in both modes
 *   validate           1: check offsets and ids on the device before refining
 *   small_task_vertices vertices each warp of the small-vertex kernel takes per task
 *                      (tile size); 0 -> default 128, else 32..65536
 *   hub_chunk_edges    edges of one hub that one CTA dedups in shared memory before
 *                      merging into the hub's global set (tile size of the hub
 *                      path); 0 -> default 512, else 256, 512 or 1024
 *   medium_split       medium vertices (above small_max_degree edges, at most
 *                      hub_threshold) with at most this many edges take a warp each,
 *                      larger ones a CTA each; 0 -> default 256, else 1..256
 *   small_max_degree   vertices with at most this many edges take the small-vertex
 *                      (warp-per-task) kernel; 0 -> default 32, else 1..32 (and at
 *                      most hub_threshold)
 *                      The five tuning fields above, load_factor and hub_threshold,
 *                      when 0, take the values kb_autotune cached for the call's size
 *                      class, else the defaults.  None of them changes any result.
 *   reorder            internal locality order for the per-edge gather of neighbour
 *                      blocks: vertices are ranked by how often they are gathered
 *                      (sampled in-degree of the processed direction) and the
 *                      library works on a copy of the neighbour ids in that order.
 *                      Costs one pass over the edges and 4 B x (m + 2n) of workspace
 *                      per call; results are identical either way.
 *                      0 -> automatic: on for prepared graphs (kb_graph_prepare)
 *                      with at least 2^22 processed edges, where its cost is paid
 *                      once; for kb_refine only with that many edges and at least
 *                      24 rounds (its cost, about one round, is paid per call),
 *                      1 -> off, 2 -> on (single-graph calls; batched and served
 *                      refinement never reorder)
 *   subject            the subject part of every key, v ~s v' of Def. "cse" (complex
 *                      schema element, Sec. "Graph Summaries for Bisimulation"):
 *                      KB_SUBJECT_PREVIOUS (0): the own block at the previous level,
 *                      i.e. stratified k-bisimulation (Defs. of Sec. 3);
 *                      KB_SUBJECT_ALL (1): T, no condition; KB_SUBJECT_LABEL (2):
 *                      equal vertex labels (the OC type cluster; all equal when
 *                      vertex_labels is NULL); KB_SUBJECT_ID (3): id, the vertex itself.
 *                      With 1..3 level i is the chained CSE^i = (~s, ~p, CSE^{i-1})
 *                      (Def. "chaining-parameterization") with CSE^0 = level 0 (labels
 *                      or {V} per use_vertex_labels, or kb_refine_from's start) and ~p
 *                      = id with edge labels, T without; e.g. Eq. (gsm:schaetzle) is
 *                      (T, id, T)^k: KB_SUBJECT_ALL, edge labels, no vertex labels, out;
 *                      Eq. (gsm:kaushik) is ((OC, T, OC)^-1)^k: KB_SUBJECT_LABEL, vertex
 *                      labels, no edge labels, in.  Such levels need not refine one
 *                      another: early stop then compares whole levels (one extra pass).
 *                      Single-graph calls only (KB_ERR_INVALID_ARG in batched, served
 *                      and allocation-free refinement).
 *   rekey_all          0 (default): single-graph stratified rounds (subject
 *                      KB_SUBJECT_PREVIOUS) skip the blocks that cannot change, since
 *                      keys hold the own previous block: a block of one vertex stays
 *                      one vertex; a block formed by a round from vertices without
 *                      edges (keys (own block, empty set)) stays as it is; and a
 *                      block none of whose members has an edge into a block of the
 *                      previous level that the last round split keeps its members
 *                      (their signatures are the previous ones with blocks renamed
 *                      one to one); such vertices keep their block without being
 *                      re-keyed.
 *                      1: re-key every vertex every round.  Results are identical
 *                      either way. */
typedef struct {
    int32_t direction;
    int32_t use_vertex_labels;
    int32_t use_edge_labels;
    int32_t early_stop;
    float load_factor;
    int32_t hub_threshold;
    int32_t hash_mode;
    int32_t validate;
    int32_t small_task_vertices;
    int32_t reorder;
    int32_t subject;
    int32_t rekey_all;
    int32_t hub_chunk_edges;
    int32_t medium_split;
    int32_t small_max_degree;
    int32_t reserved[1];
} kb_options;

enum { KB_SUBJECT_PREVIOUS = 0, KB_SUBJECT_ALL = 1, KB_SUBJECT_LABEL = 2, KB_SUBJECT_ID = 3 };

typedef struct kb_context kb_context;

/* Defaults: OUT, vertex and edge labels on, early stop on, validate on. */
kb_options kb_options_default(void);
/* Schaetzle et al. preset (paper eq. "gsm:schaetzle", Def. "edge-labeled-fw-
 * bisimulation"): OUT edges, edge labels, no vertex labels. */
kb_options kb_options_schaetzle(void);
/* Kaushik et al. preset (paper eq. "gsm:kaushik", Def. "vertex-labeled-bw-
 * bisimulation"): IN edges, vertex labels, no edge labels. */
kb_options kb_options_kaushik(void);

const char* kb_status_string(kb_status status);

/* Create a context on `device` bound to `stream` (a cudaStream_t; NULL = the
 * legacy default stream).  The context caches device scratch between calls. */
kb_status kb_create(kb_context** ctx, int device, void* stream);
kb_status kb_destroy(kb_context* ctx);
const char* kb_last_error(const kb_context* ctx);

/* Bytes of device scratch that kb_refine / kb_refine_from need for this graph
 * and these options (reads row_offsets on the device; synchronises). */
kb_status kb_workspace_size(kb_context* ctx, const kb_graph* g, const kb_options* opt, int k,
                            size_t* bytes);

/* Use caller-owned device memory as scratch (e.g. a torch tensor).  The
 * buffer must stay alive while calls that use it run.  ptr = NULL reverts to
 * library-allocated scratch.  Calls fail with KB_ERR_OOM if it is too small. */
kb_status kb_set_workspace(kb_context* ctx, void* device_ptr, size_t bytes);

/* Refine levels 0..k.
 *   levels           DEVICE int32[(k+1)*n]; row i (levels + i*n) receives the
 *                    canonical block id of every vertex at level i
 *   counts           HOST int64[k+1]; counts[i] = number of blocks at level i
 *   levels_computed  HOST, may be NULL; the last level actually refined (< k when
 *                    early_stop found a stable partition; rows after it are copies)
 * Synchronises the stream once per round to read the block count, and once
 * more at level 0 when it has keys (vertex labels or a starting partition): a
 * range check decides whether they all lie in [0, 8192), which takes a path
 * without the block table. */
kb_status kb_refine(kb_context* ctx, const kb_graph* g, const kb_options* opt, int k,
                    int32_t* levels, int64_t* counts, int* levels_computed);

/* Resume from a known level (refinement depends only on the graph and the
 * previous level).  start is DEVICE int32[n] holding any partition (equal
 * values = same block); row i_start of `levels` receives its canonical
 * renumbering and rows i_start+1..k the refined levels.  Rows below i_start
 * are left untouched; counts[0..i_start-1] likewise.  With i_start = 0 this
 * refines an arbitrary starting partition instead of the label partition. */
kb_status kb_refine_from(kb_context* ctx, const kb_graph* g, const kb_options* opt,
                         const int32_t* start, int i_start, int k, int32_t* levels,
                         int64_t* counts, int* levels_computed);

/* ---- Prepared graphs ---------------------------------------------------------
 * Every refinement call on a graph first derives per-graph structures from
 * it: validation, the processed CSR (in-edges for KB_DIR_IN / KB_DIR_BOTH),
 * the degree classes (list of medium vertices), the hub plan (chunks and the
 * layout of the per-hub sets), the bits of edgeless vertices and, when on,
 * the locality order (vertices ranked by how often they are gathered, with
 * the neighbour ids rewritten to those ranks).  None of them depends on the
 * levels, so Alg. 1's rounds (Sec. 4.1) can run on them any number of times.
 * kb_graph_prepare builds them once, in device memory of the prepared graph's
 * own; kb_refine_prepared is kb_refine without that per-call work.
 *   g, opt    as for kb_refine.  The graph fields of opt are fixed here:
 *             direction, use_edge_labels, hub_threshold, small_max_degree,
 *             hub_chunk_edges, reorder and validate (checked once, here).
 *             reorder 0 (automatic) turns the locality order on for at least
 *             2^22 processed edges, since its cost is paid once (it costs about
 *             as much as one round and saves part of every round's gather).
 *   out       receives the prepared graph.  It refers to g's arrays, which must
 *             stay alive and unchanged until kb_graph_release.  It can be used
 *             by any context on the same device, by one call at a time.
 * Errors as kb_refine (KB_ERR_INVALID_ARG for malformed CSR with validate,
 * KB_ERR_OOM when its buffers do not fit).  Synchronises. */
typedef struct kb_prepared kb_prepared;
kb_status kb_graph_prepare(kb_context* ctx, const kb_graph* g, const kb_options* opt, kb_prepared** out);
/* Free a prepared graph's device memory (NULL is accepted). */
kb_status kb_graph_release(kb_prepared* pg);

typedef struct {
    size_t device_bytes;     /* device memory the prepared graph holds */
    int64_t n_hubs;          /* vertices above the hub threshold */
    int64_t n_hub_chunks;    /* hub-chunk CTAs of a round that keys every hub */
    int64_t n_medium;        /* medium vertices */
    int32_t reorder;         /* 1: locality order on */
    int32_t hub_threshold;
    int32_t small_max_degree;
    int32_t hub_chunk_edges;
    float build_ms;          /* host time of kb_graph_prepare */
    int32_t reserved[3];
} kb_prepared_info;
kb_status kb_prepared_get_info(const kb_prepared* pg, kb_prepared_info* info);

/* kb_refine on a prepared graph: levels, counts and levels_computed exactly as
 * kb_refine of the same graph and options gives them.  opt->direction and
 * opt->use_edge_labels must equal those of kb_graph_prepare
 * (KB_ERR_INVALID_ARG otherwise); its other graph fields are ignored (the
 * prepared values apply).  The per-call fields apply: use_vertex_labels,
 * early_stop, load_factor, hash_mode, small_task_vertices, medium_split,
 * subject, rekey_all. */
kb_status kb_refine_prepared(kb_context* ctx, const kb_prepared* pg, const kb_options* opt, int k,
                             int32_t* levels, int64_t* counts, int* levels_computed);

/* Full (unstratified) bisimulation: refine until a round leaves the partition
 * unchanged, as Schaetzle et al. do (Sec. "Bisimulation Variants": they iterate
 * until no further change instead of stopping after k rounds), keeping only
 * the last two levels instead of k+1 rows.  With an initial partition this is
 * the coarsest stable refinement of P_0 (Def. "relational coarsest partition
 * problem", Sec. "Native Kaushik et al. Algorithm"), here for the direction and
 * labels of `opt`.
 *   initial      DEVICE int32[n] or NULL; starting partition (equal values = same
 *                block).  NULL: vertex labels (opt->use_vertex_labels) or {V}.
 *   max_rounds   upper bound on rounds (>= 0); stops earlier when stable
 *   final_level  DEVICE int32[n], caller-owned; the last partition, canonical ids
 *   count        HOST; blocks of final_level
 *   rounds       HOST; rounds run (a stable run's last round reproduced its input)
 *   stable       HOST, may be NULL; 1 when a round found the partition stable
 *                (always when n == 0), 0 when max_rounds ran out first
 * opt->early_stop is ignored (the run always stops at stability).  Uses 8 B x n
 * of library scratch besides the refinement workspace.  Synchronises. */
kb_status kb_refine_fixpoint(kb_context* ctx, const kb_graph* g, const kb_options* opt,
                             const int32_t* initial, int max_rounds, int32_t* final_level,
                             int64_t* count, int* rounds, int* stable);

/* Summary graph of a partition pair (Sec. "Graph Summaries for Bisimulation":
 * one summary vertex per block, a labelled edge from block b to block c when
 * the vertices of b have an edge with that label into c).  Every graph edge
 * v -> w with label l gives the triple (src_level[x], l, dst_level[y]), x -> y
 * being the edge in `direction` (out: x = v, y = w; in: x = w, y = v); the
 * output lists each distinct triple once, in order of its first occurrence in
 * the edge list (sources ascending, then CSR order).
 * With src_level = P_i and dst_level = P_{i-1} of one refinement this is the
 * paper's layer of summary edges between the two levels, and then every vertex
 * of b has the edge (its signature over P_{i-1} is its block's); with both the
 * same partition it is the quotient graph (an edge when some vertex has one).
 *   g                  DEVICE CSR as for kb_refine, m < 2^32; ids are validated
 *   direction          KB_DIR_OUT or KB_DIR_IN (call twice for both)
 *   use_edge_labels    0: every label reads 0 (g->edge_labels may be NULL)
 *   src_level, dst_level DEVICE int32[n]: block of every vertex; any int32 values
 *   out_src, out_label, out_dst DEVICE int32[capacity] each, caller-owned
 *   capacity           entries the outputs hold; m always suffices; 0 with NULL
 *                      outputs counts only
 *   count              HOST; the number of summary edges, set also when the
 *                      outputs are too small (then KB_ERR_INVALID_ARG, outputs
 *                      untouched)
 * Scratch: about 24 B x next_pow2(1.25 m) + m/4 B of library-owned device memory,
 * kept for later calls (grow-only) and released by kb_destroy.  Synchronises. */
kb_status kb_summary(kb_context* ctx, const kb_graph* g, int direction, int use_edge_labels,
                     const int32_t* src_level, const int32_t* dst_level, int32_t* out_src,
                     int32_t* out_label, int32_t* out_dst, int64_t capacity, int64_t* count);

/* Incremental refinement after a change of the graph (edges inserted, deleted
 * or relabelled; vertex labels may change too).  The paper leaves incremental
 * k-bisimulation as future work (Sec. "Conclusion and Future Work").  Each
 * round re-keys only a work set -- the vertices of every previous-level block
 * that holds a dirty vertex (changed edge list, block changed at the previous
 * level, or an edge to such a vertex) -- and keeps the old grouping of all
 * others; every level is renumbered canonically, so the output equals
 * kb_refine on the new graph.
 *   g          the NEW graph (DEVICE CSR as for kb_refine)
 *   opt        the options the old levels were computed with (subject must be
 *              KB_SUBJECT_PREVIOUS; the locality order is not used)
 *   changed    DEVICE int32[n_changed]: every vertex whose edge list in the
 *              processed direction changed (out: sources of inserted, deleted or
 *              relabelled edges; in: their targets; both: both ends); duplicates
 *              are fine
 *   levels     DEVICE int32[(k+1)*n], in: kb_refine's levels of the graph before
 *              the change (same n, same options); out: the levels of g
 *   counts, levels_computed  as for kb_refine
 *   work       HOST int64[k+1] or NULL: vertices re-keyed per level (level 0: n)
 * When the first round's work set would exceed a quarter of the vertices (the
 * old level-0 blocks holding changed vertices are that large, as label
 * classes often are), the call runs as kb_refine on g instead, whose frozen
 * blocks then cost less than re-keying whole blocks; work reports n for every
 * computed level.  The result is the same either way.
 * KB_ERR_INVALID_ARG when an old level or a changed id lies outside [0, n).
 * Scratch: about 29 B x n of library-owned device memory.  Synchronises. */
kb_status kb_refine_update(kb_context* ctx, const kb_graph* g, const kb_options* opt, int k,
                           const int32_t* changed, int64_t n_changed, int32_t* levels,
                           int64_t* counts, int* levels_computed, int64_t* work);

/* kb_refine with HOST buffers: g's arrays and `levels` (int32[(k+1)*n]) are host
 * memory (pinned memory copies fastest).  The library copies the graph to the
 * device, refines, and copies every level back.  Synchronises. */
kb_status kb_refine_host(kb_context* ctx, const kb_graph* g, const kb_options* opt, int k,
                         int32_t* levels, int64_t* counts, int* levels_computed);

/* Per-round and per-kernel timing of the last refine call, in milliseconds,
 * measured with CUDA events on the context stream when enabled.
 *   kb_set_timing(ctx, 1) enables event recording (small overhead); 2 also
 *   records the work of every round (kb_get_round_work; one extra pass over
 *   the row offsets per round); 0 disables both.
 *   round_ms[i] for i < n_rounds: device time of refinement round i+1.
 *   kernel_ms[j] / kernel_launches[j] for j < KB_KERNEL_COUNT: summed device time
 *   and launches of each kernel family inside the rounds. */
enum {
    KB_KERNEL_SMALL = 0,       /* warp kernel: vertices with <= 32 edges (signature, dedup, hash, insert) */
    KB_KERNEL_MEDIUM = 1,      /* tile kernel: vertices with 33..hub_threshold edges */
    KB_KERNEL_HUB_CHUNK = 2,   /* hub pairs: chunk dedup + global set insert */
    KB_KERNEL_HUB_FINAL = 3,   /* hub hash + block-table insert */
    KB_KERNEL_RENUMBER = 4,    /* prefix scan of block minima + canonical assignment */
    KB_KERNEL_OTHER = 5,       /* clears, copies */
    KB_KERNEL_COUNT = 6
};
kb_status kb_set_timing(kb_context* ctx, int enable);
kb_status kb_get_timing(const kb_context* ctx, float* round_ms, int max_rounds, int* n_rounds,
                        float* kernel_ms, int64_t* kernel_launches);

/* Work of the rounds of the last kb_refine / kb_refine_from / kb_refine_fixpoint
 * call on this context made with kb_set_timing(ctx, 2): the vertices each
 * round re-keyed and their edges in
 * the processed direction, per kernel family (small: at most 32 edges, medium:
 * up to hub_threshold, hub: more).  Single-graph stratified rounds (subject
 * KB_SUBJECT_PREVIOUS, rekey_all 0) skip the blocks that cannot change: keys
 * hold the own previous block (Sec. 3: i-bisimilar vertices are
 * (i-1)-bisimilar), so a block of one vertex, a block of edgeless vertices
 * formed by a round, and a block none of whose members has an edge to a
 * vertex whose smallest block member the last round changed keep their
 * members without being re-keyed.
 *   vertices, edges  HOST int64[3 * max_rounds] or NULL; entry 3*i + f is round
 *                    i+1 (the first signature round after the starting level),
 *                    family f = 0 small, 1 medium, 2 hub
 *   n_rounds         HOST: rounds recorded */
kb_status kb_get_round_work(const kb_context* ctx, int64_t* vertices, int64_t* edges, int max_rounds,
                            int* n_rounds);

/* Batched refinement of G independent graphs given as one disjoint union.
 *   union_graph            DEVICE CSR over all vertices; edges never cross graphs
 *   graph_vertex_offsets   HOST int64[G+1]; graph j owns vertices
 *                          [off[j], off[j+1]) of the union
 *   k_per_graph            HOST int32[G]; each graph's own k (>= 0)
 *   levels                 DEVICE int32[(k_max+1)*n_total]; row i holds every graph's
 *                          level min(i, its last level) with ids LOCAL to the graph
 *                          (canonical per graph, exactly as a solo kb_refine)
 *   counts                 HOST int64[G*(k_max+1)]; counts[j*(k_max+1)+i]
 *   levels_computed        HOST int32[G] or NULL
 * Rounds run for all active graphs at once: one signature launch per round over
 * the union, the whole k_max-round loop captured once in a CUDA graph and
 * replayed, and a device-side per-graph stop flag (no host sync per round). */
kb_status kb_refine_batch(kb_context* ctx, const kb_graph* union_graph,
                          const int64_t* graph_vertex_offsets, int64_t G,
                          const int32_t* k_per_graph, const kb_options* opt, int32_t* levels,
                          int64_t* counts, int32_t* levels_computed);

/* Autotuner.  Chooses the block-table load factor, the degree-class bounds
 * (hub_threshold, small_max_degree, medium_split) and the tile sizes
 * (small_task_vertices, hub_chunk_edges) by timing the call it is given:
 *   graph_vertex_offsets == NULL: kb_refine of g with `rounds` rounds;
 *   else (HOST int64[G+1], as kb_refine_batch): kb_refine_batch of the union g,
 *        every graph with k = rounds (k_per_graph NULL) or k_per_graph[j].
 * Early stop is off while timing.  A coordinate search starts from the
 * options' values (defaults where 0), tries every value of one field at a time
 * and keeps a value only when it is faster by more than 2%:
 *   load_factor {0.35, 0.5, 0.7}, hub_threshold {256, 512, 1024},
 *   small_max_degree {16, 24, 32}, medium_split {64, 128, 256},
 *   small_task_vertices {64, 128, 256, 512}, hub_chunk_edges {256, 512, 1024};
 * each setting is timed (CUDA events, one warm-up run) as the best of two
 * runs.  The choice is cached in the context under the call's size class
 * (single graph or batch, and log2 of the processed edges per graph); later
 * kb_refine, kb_refine_batch and kb_workspace_size calls whose options leave a
 * field 0 take it from the cached entry of their own class, or of the nearest
 * class of the same kind within a factor of 8.  `out` (HOST, may be NULL)
 * receives the choice, its time and the time with library defaults.
 * Results never depend on these fields.  Synchronises. */
typedef struct {
    float load_factor;
    int32_t hub_threshold;
    int32_t small_task_vertices;
    int32_t hub_chunk_edges;
    int32_t medium_split;
    int32_t small_max_degree;
    float ms;           /* time of the timed call with the chosen values */
    float default_ms;   /* the same with every tuning field at its default */
    int32_t size_class; /* key of the cached entry */
    int32_t reserved[3];
} kb_tuning;
kb_status kb_autotune(kb_context* ctx, const kb_graph* g, const int64_t* graph_vertex_offsets, int64_t G,
                      const int32_t* k_per_graph, const kb_options* opt, int rounds, kb_tuning* out);
/* Forget every cached tuning of the context. */
kb_status kb_clear_tuning(kb_context* ctx);

/* ---- Serving: continuous batching of summarisation requests ----------------
 * A server keeps every admitted request's graph and partitions on the device
 * and advances all of them by one refinement round per kb_server_step: one
 * set of kernel launches covers every in-flight request, whatever its size,
 * direction or k.  Requests that arrive while others run wait until arena
 * space, a request slot and device memory for their level store are free,
 * and are then admitted at the next step (their level 0 is computed in that
 * step alongside the others' rounds).  Results are identical to a solo
 * kb_refine of the same graph and options.
 *   max_vertices / max_edges   arena capacity; a graph's processed edges count
 *                              (2m for KB_DIR_BOTH) must fit max_edges
 *   max_requests               requests in flight at most
 *   memory_budget              device bytes for the per-request level stores
 *                              ((k+1)*n*4 each); 0 = free device memory minus a
 *                              1 GiB reserve, checked at every admission
 *   load_factor, hub_threshold, hash_mode   as in kb_options */
typedef struct {
    int64_t max_vertices;
    int64_t max_edges;
    int32_t max_requests;
    int32_t hub_threshold;
    size_t memory_budget;
    float load_factor;
    int32_t hash_mode;
    int32_t reserved[6];
} kb_server_config;

typedef struct {
    int64_t submitted, completed, running, waiting;
    int64_t steps, compactions;
    double p50_ms, p99_ms, mean_ms;   /* submit-to-completion latency of completed requests */
    double requests_per_s;            /* completed requests / time since the first submit */
    double edge_rounds_per_s;         /* processed edges x rounds of completed requests / same time */
    int64_t failed;                   /* requests rejected at admission (malformed CSR) */
} kb_server_stats;

typedef struct kb_server kb_server;

kb_server_config kb_server_config_default(void);
kb_status kb_server_create(kb_server** server, int device, void* stream, const kb_server_config* cfg);
kb_status kb_server_destroy(kb_server* server);
const char* kb_server_last_error(const kb_server* server);
/* Queue a request.  g holds HOST arrays that the caller keeps alive and
 * unchanged until the request has been admitted (kb_server_poll reports 1, 2
 * or 3): they are copied to the device at admission, not at submission.
 * levels_out is HOST int32[(k+1)*n] or NULL: when given, the levels are
 * written there when the request finishes (no host copy inside the library;
 * keep it alive until kb_server_fetch).  Checked here: sizes, the ends of
 * row_offsets and the arena's capacity; every offset and neighbour id is
 * checked on the device at admission, where a malformed graph fails alone
 * (state 3) without reaching the shared arena.  ticket receives the request's
 * id.  Thread-safe with respect to kb_server_step. */
kb_status kb_server_submit(kb_server* server, const kb_graph* g, const kb_options* opt, int k, int32_t* levels_out,
                           int64_t* ticket);
/* Admit what fits, then run one round for every in-flight request and retire
 * finished ones (their levels are copied to host memory).  running / waiting
 * (may be NULL) receive the request counts after the step. */
kb_status kb_server_step(kb_server* server, int32_t* running, int32_t* waiting);
/* state: 0 waiting, 1 running, 2 done (fetchable), 3 rejected at admission
 * (kb_server_fetch returns KB_ERR_INVALID_ARG and forgets it); KB_ERR_NOT_FOUND
 * if unknown. */
kb_status kb_server_poll(kb_server* server, int64_t ticket, int32_t* state);
/* Copy a finished request's results to HOST buffers (levels int32[(k+1)*n],
 * may be NULL or the levels_out given at submission; counts int64[k+1]) and
 * forget it. */
kb_status kb_server_fetch(kb_server* server, int64_t ticket, int32_t* levels, int64_t* counts,
                          int32_t* levels_computed);
kb_status kb_server_get_stats(kb_server* server, kb_server_stats* stats);

/* ---- One refinement round without device allocation -----------------------
 * The paper has no counterpart to this entry point.  It serves callers that
 * must not allocate device memory, themselves or through the library: an
 * application that reserves all device memory in its own pool at start-up, or
 * a latency-critical thread for which the device-wide synchronisation that
 * cudaMalloc / cudaFree may cause is not acceptable.  It needs no context.
 *
 * Computes level i from level i-1 (one round of the refinement, out-edges):
 *   stream   cudaStream_t to run on (NULL = legacy default stream); the call
 *            synchronises it before returning
 *   g        DEVICE CSR as for kb_refine, with n <= KB_NOALLOC_MAX_VERTICES and
 *            no vertex with more than hub_threshold (default 1024) edges
 *   opt      direction must be KB_DIR_OUT; use_edge_labels, hash_mode,
 *            hub_threshold, small_task_vertices (0 or 32..65536),
 *            medium_split (0..256), small_max_degree (0..32) and validate are
 *            honoured (0 = library default; cached tunings are not consulted)
 *   prev     DEVICE int32[n], canonical ids of level i-1, each in [0, n)
 *   out      DEVICE int32[n], receives the canonical ids of level i
 *   count    HOST, receives the number of blocks of level i
 * Its scratch is one static device array of about 33 MB inside the library,
 * which every device that loads the library keeps until the process exits.
 * The first call on a device looks up the array's device address (and sets
 * the round kernels' shared-memory attributes).  Every call synchronises
 * `stream` and reads results back to the host before returning, so no call
 * can be part of a CUDA-graph capture.
 * Every call shares the array, which keeps the previous call's contents
 * (each call resets what it uses), so calls that overlap on the GPU -- from
 * several streams or threads -- race; the caller must serialise them.
 * Errors: KB_ERR_INVALID_ARG for n above the limit, another direction, a
 * vertex whose degree lies outside [0, hub threshold], an id of prev outside
 * [0, n), a tuning field out of range or (with validate) malformed CSR;
 * `out` is then left untouched.  KB_ERR_CUDA when a runtime call fails. */
#define KB_NOALLOC_MAX_VERTICES 1048576
kb_status kb_refine_round_noalloc(void* stream, const kb_graph* g, const kb_options* opt,
                                  const int32_t* prev, int32_t* out, int64_t* count);

#ifdef __cplusplus
}
#endif

#endif /* KBISIM_H_ */
