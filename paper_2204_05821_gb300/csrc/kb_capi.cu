// Host side of the C ABI declared in include/kbisim.h: contexts, workspace
// planning, the per-round driver loop (paper Alg. 1: rounds 1..k with the
// block-count stop test), host-buffer refinement and timing.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "kb_internal.cuh"

struct kb_context {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string last_error;
    // scratch: caller-provided or library-owned (grow-only)
    void* user_ws = nullptr;
    size_t user_ws_bytes = 0;
    void* own_ws = nullptr;
    size_t own_ws_bytes = 0;
    // small persistent device state
    kb::Counters* d_ctr = nullptr;
    kb::Counters* h_ctr = nullptr;  // pinned
    int32_t* d_hub_n = nullptr;
    int32_t* h_hub_n = nullptr;  // pinned
    int64_t* d_med_n = nullptr;
    int64_t* h_med_n = nullptr;  // pinned
    void* hub_tmp = nullptr;     // unordered hub list during planning
    size_t hub_tmp_bytes = 0;
    void* plan_tmp = nullptr;    // in-degree scratch used by kb_workspace_size
    size_t plan_tmp_bytes = 0;
    // host-buffer refinement staging (library-owned)
    void* stage = nullptr;
    size_t stage_bytes = 0;
    // autotuned values per size class (kb_autotune); plan_graphs is the graph
    // count of the batched call being planned
    std::map<int32_t, kb_tuning> tuned;
    int64_t plan_graphs = 1;
    // batched refinement
    void* batch_ws = nullptr;
    size_t batch_ws_bytes = 0;
    void* tune_buf = nullptr;
    size_t tune_buf_bytes = 0;
    // fixpoint refinement: the last two levels
    void* fix_buf = nullptr;
    size_t fix_buf_bytes = 0;
    // summary graph: triple table, first edges, edge bitmap and its ranks
    void* sum_buf = nullptr;
    size_t sum_buf_bytes = 0;
    // incremental refinement: bitmaps, block flags, kept minima, id ranges
    void* upd_buf = nullptr;
    size_t upd_buf_bytes = 0;
    unsigned long long* d_work = nullptr;  // |W| of the current round
    cudaStream_t cap_stream = nullptr;  // non-default stream used only to capture CUDA graphs
    cudaStream_t copy_stream = nullptr;  // level rows back to the host (kb_refine_host)
    cudaEvent_t row_ev = nullptr;
    // timing: CUDA events per kernel family; with work, also the vertices and
    // edges every round re-keys (one extra pass over the row offsets a round)
    bool timing = false;
    bool work = false;
    std::vector<float> round_ms;
    // per round of the last kb_refine / kb_refine_from / kb_refine_fixpoint
    // call: vertices and processed edges re-keyed by the small, medium and hub
    // kernels
    std::vector<std::array<int64_t, 6>> round_keyed;
    float kernel_ms[KB_KERNEL_COUNT] = {};
    int64_t kernel_launches[KB_KERNEL_COUNT] = {};
    cudaEvent_t ev[2 * 10 + 2] = {};  // pairs for the round timer; the last two time whole calls
};

namespace {

using kb::Counters;

kb_status fail(kb_context* ctx, kb_status st, const char* fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        ctx->last_error = buf;
    }
    return st;
}

#define KB_CUDA(ctx, call)                                                                        \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return fail((ctx), KB_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));     \
    } while (0)

#define KB_TRY(expr)                       \
    do {                                   \
        kb_status s_ = (expr);             \
        if (s_ != KB_OK) return s_;        \
    } while (0)

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

uint64_t next_pow2(uint64_t x) {
    uint64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

// Block-table slots for n vertices at load factor lf: a power of two of at
// least 1024 and at most 2^31, since a vertex's slot index is kept in the 31
// low bits of its slot_of entry (bit 31 marks an empty signature).  Above
// 2^30 vertices the table can thus be fuller than lf asks (it still holds
// every block: n <= 2^31 - 2).
uint64_t table_capacity(int64_t n, float lf) {
    uint64_t cap = next_pow2((uint64_t)((double)std::max<int64_t>(n, 1) / (double)lf) + 1);
    if (cap < 1024) cap = 1024;
    if (cap > ((uint64_t)1 << 31)) cap = (uint64_t)1 << 31;
    return cap;
}

// Device buffers of one refine call, carved from one workspace allocation.
struct Plan {
    int64_t n = 0, m = 0, m_proc = 0;
    int dir = 0;
    bool labels = false;
    int thr = kb::kDefaultHubThreshold;
    int hub_chunk = kb::kDefaultHubChunk;
    int med_split = kb::kDefaultMedSplit;
    int small_max = kb::kSmallDegree;
    int warp_verts = kb::kDefaultWarpVerts;
    int32_t size_class = 0;  // key of the tuning cache
    uint64_t cap = 0;
    bool reorder = false;  // locality order of the gather (RoundParams::perm)
    int subject = 0;       // kb_options::subject (generic CSE rounds when > 0)
    bool freeze = false;   // frozen blocks skip the rounds (RoundParams::frozen)
    bool dense0 = false;   // one graph: level 0 may take the small-label path (launch_dense_level0)
    bool ext_table = false;  // block table and empty-signature minima live outside the workspace
    bool ext_freeze = false;  // frozen-block state lives outside the workspace
    // the per-graph part (processed CSR, degree classes, hub plan, locality
    // order, edgeless bits) lives in a prepared graph's own buffers: layout
    // offsets of that part are relative to them (kb_graph_prepare)
    bool graph_ext = false;
    size_t graph_bytes = 0;
    // hubs (host copies, ascending vertex id)
    std::vector<int32_t> hub_v;
    std::vector<int64_t> chunk_off, set_off;
    std::vector<int32_t> chunk_hub;
    // their sizes (the lists themselves are dropped once on the device)
    size_t n_hubs = 0;
    int64_t n_chunks = 0, set_slots = 0;
    // layout
    size_t o_rowp = 0, o_colp = 0, o_labp = 0, o_cursor = 0, o_inpref = 0, o_i64tmp = 0;
    size_t csr_bytes = 0;
    size_t o_emin = 0, o_med = 0, o_slot = 0, o_table = 0, o_bitmap = 0, o_prefix = 0, o_scan = 0, o_hubv = 0, o_chunk = 0, o_setoff = 0,
           o_chunkhub = 0, o_chunkext = 0, o_perm = 0, o_gat = 0, o_colr = 0, o_hist = 0, o_ownkey = 0, o_acc = 0, o_cnt = 0, o_sets = 0,
           o_frozen = 0, o_fmin = 0, o_edgeless = 0, o_shared = 0, o_minof = 0, o_bm2 = 0, o_moved = 0, o_mark = 0,
           o_dense = 0;
    size_t total = 0;
};

bool needs_in_csr(int dir) { return dir == KB_DIR_IN || dir == KB_DIR_BOTH; }

}  // namespace

// A prepared graph (kb_graph_prepare): the per-graph part of a plan built
// once, in device buffers of its own.
struct kb_prepared {
    int device = 0;
    kb_graph g{};       // the caller's arrays
    int32_t dir = 0;
    int32_t edge_labels = 0;
    Plan P;             // graph_ext layout; host hub lists dropped after upload
    char* csr = nullptr;   // processed CSR (IN / BOTH)
    char* gbuf = nullptr;  // per-graph part
    int64_t n_med = 0;
    float build_ms = 0.f;
    ~kb_prepared() {
        if (!csr && !gbuf) return;
        int cur = 0;
        cudaGetDevice(&cur);
        cudaSetDevice(device);
        cudaFree(csr);
        cudaFree(gbuf);
        cudaSetDevice(cur);
    }
};

namespace {

void layout_csr(Plan& P) {
    size_t off = 0;
    P.csr_bytes = 0;
    if (!needs_in_csr(P.dir)) return;
    auto take = [&](size_t bytes) { size_t o = off; off += align_up(bytes); return o; };
    P.o_rowp = take(sizeof(int64_t) * (size_t)(P.n + 1));
    P.o_colp = take(sizeof(int32_t) * (size_t)P.m_proc);
    P.o_labp = take(P.labels ? sizeof(int32_t) * (size_t)P.m_proc : 0);
    P.o_cursor = take(sizeof(int64_t) * (size_t)(P.n + 1));
    P.o_inpref = take(sizeof(int64_t) * (size_t)(P.n + 1));
    P.o_i64tmp = take(sizeof(int64_t) * kb::scan_i64_tmp(P.n + 1));
    P.csr_bytes = off;
}

// Round buffers.  The per-graph part comes first, at offsets after the CSR
// (or, with graph_ext, from 0 in a buffer of its own: graph_bytes); the
// per-call part follows in the workspace (total).
void layout_round(Plan& P) {
    size_t goff = P.graph_ext ? 0 : P.csr_bytes;
    auto takeg = [&](size_t bytes) { size_t o = goff; goff += align_up(bytes); return o; };
    const int64_t nw = (P.n >> 5) + 1;
    const size_t H = P.n_hubs;
    P.o_med = takeg(sizeof(int32_t) * (size_t)(std::min<int64_t>(P.n, P.m_proc / 2 + 1) + 1));
    P.o_hubv = takeg(sizeof(int32_t) * H);
    P.o_chunk = takeg(sizeof(int64_t) * (H + 1));
    P.o_setoff = takeg(sizeof(int64_t) * (H + 1));
    P.o_chunkhub = takeg(sizeof(int32_t) * (size_t)P.n_chunks);
    P.o_chunkext = takeg(sizeof(uint64_t) * (size_t)P.n_chunks);
    P.o_perm = takeg(P.reorder ? sizeof(int32_t) * (size_t)P.n : 0);
    // a reordered copy of the caller's neighbour ids; the library's own in-edge
    // CSR is reordered in place
    P.o_colr = takeg(P.reorder && !needs_in_csr(P.dir) ? sizeof(int32_t) * (size_t)P.m_proc : 0);
    P.o_hist = takeg(P.reorder ? sizeof(unsigned long long) * 512 : 0);
    P.o_edgeless = takeg((P.freeze || P.graph_ext) ? sizeof(uint32_t) * (size_t)nw : 0);
    P.graph_bytes = P.graph_ext ? goff : 0;
    size_t off = P.graph_ext ? 0 : goff;
    auto take = [&](size_t bytes) { size_t o = off; off += align_up(bytes); return o; };
    P.o_emin = take(P.ext_table ? 0 : sizeof(uint64_t) * (size_t)std::max<int64_t>(P.n, 1));
    P.o_slot = take(sizeof(int32_t) * (size_t)std::max<int64_t>(P.n, 1));
    P.o_table = take(P.ext_table ? 0 : sizeof(uint64_t) * (size_t)P.cap);
    P.o_bitmap = take(sizeof(uint32_t) * (size_t)nw);
    P.o_prefix = take(sizeof(uint2) * (size_t)(nw + 1));
    P.o_scan = take(sizeof(uint32_t) * kb::scan_tmp_words(nw));
    P.o_acc = take(sizeof(uint64_t) * H);
    P.o_cnt = take(sizeof(uint32_t) * H);
    P.o_sets = take(sizeof(uint64_t) * (size_t)P.set_slots);
    P.o_gat = take(P.reorder ? sizeof(int32_t) * (size_t)P.n : 0);
    P.o_ownkey = take(P.subject ? sizeof(int32_t) * (size_t)P.n : 0);
    const bool own_freeze = P.freeze && !P.ext_freeze;
    P.o_frozen = take(own_freeze ? sizeof(uint32_t) * (size_t)nw : 0);
    P.o_fmin = take(own_freeze ? sizeof(uint32_t) * (size_t)nw : 0);
    P.o_shared = take(own_freeze ? sizeof(uint32_t) * (size_t)nw : 0);
    P.o_minof = take(own_freeze ? sizeof(uint32_t) * (size_t)P.n : 0);
    P.o_bm2 = take(P.freeze ? sizeof(uint32_t) * (size_t)nw : 0);
    P.o_moved = take(own_freeze ? sizeof(uint32_t) * (size_t)nw : 0);
    P.o_mark = take(own_freeze ? sizeof(uint32_t) * (size_t)nw : 0);
    P.o_dense = take(P.dense0 ? (sizeof(uint32_t) + sizeof(uint2)) * (size_t)kb::kDenseLabels : 0);
    P.total = off;
}

kb_status check_graph(kb_context* ctx, const kb_graph* g, const kb_options* opt, int k) {
    if (!g || !opt) return fail(ctx, KB_ERR_INVALID_ARG, "graph and options must not be NULL");
    if (g->n < 0 || g->m < 0) return fail(ctx, KB_ERR_INVALID_ARG, "negative n or m");
    if (g->n > 2147483646LL) return fail(ctx, KB_ERR_INVALID_ARG, "n exceeds 2^31-2");
    if (g->m > (1LL << 45)) return fail(ctx, KB_ERR_INVALID_ARG, "m exceeds 2^45");
    if (k < 0) return fail(ctx, KB_ERR_INVALID_ARG, "k must be >= 0");
    if (opt->direction < 0 || opt->direction > 2) return fail(ctx, KB_ERR_INVALID_ARG, "bad direction");
    if (g->n > 0 && !g->row_offsets) return fail(ctx, KB_ERR_INVALID_ARG, "row_offsets is NULL");
    if (g->m > 0 && !g->col_indices) return fail(ctx, KB_ERR_INVALID_ARG, "col_indices is NULL");
    if (g->n == 0 && g->m != 0) return fail(ctx, KB_ERR_INVALID_ARG, "edges without vertices");
    if (opt->load_factor < 0.f || opt->load_factor > 0.9f)
        return fail(ctx, KB_ERR_INVALID_ARG, "load_factor must be in (0, 0.9]");
    if (opt->hub_threshold < 0 || opt->hub_threshold > kb::kMaxHubThreshold)
        return fail(ctx, KB_ERR_INVALID_ARG, "hub_threshold must be in [0, %d]", kb::kMaxHubThreshold);
    if (opt->hash_mode < 0 || opt->hash_mode > 1) return fail(ctx, KB_ERR_INVALID_ARG, "bad hash_mode");
    if (opt->reorder < 0 || opt->reorder > 2) return fail(ctx, KB_ERR_INVALID_ARG, "reorder must be 0, 1 or 2");
    if (opt->subject < 0 || opt->subject > 3) return fail(ctx, KB_ERR_INVALID_ARG, "subject must be 0..3");
    if (opt->small_task_vertices != 0 && (opt->small_task_vertices < 32 || opt->small_task_vertices > 65536))
        return fail(ctx, KB_ERR_INVALID_ARG, "small_task_vertices must be 0 or in [32, 65536]");
    if (opt->hub_chunk_edges != 0 && opt->hub_chunk_edges != 256 && opt->hub_chunk_edges != 512 &&
        opt->hub_chunk_edges != 1024)
        return fail(ctx, KB_ERR_INVALID_ARG, "hub_chunk_edges must be 0, 256, 512 or 1024");
    if (opt->medium_split < 0 || opt->medium_split > kb::kMaxMedSplit)
        return fail(ctx, KB_ERR_INVALID_ARG, "medium_split must be in [0, %d]", kb::kMaxMedSplit);
    if (opt->small_max_degree < 0 || opt->small_max_degree > kb::kSmallDegree)
        return fail(ctx, KB_ERR_INVALID_ARG, "small_max_degree must be in [0, %d]", kb::kSmallDegree);
    if (opt->direction == KB_DIR_BOTH && g->m > (int64_t)1 << 62)
        return fail(ctx, KB_ERR_INVALID_ARG, "too many edges");
    return KB_OK;
}

kb_status ensure_buffer(kb_context* ctx, void** buf, size_t* have, size_t need) {
    if (need <= *have) return KB_OK;
    if (*buf) cudaFree(*buf);
    *buf = nullptr;
    *have = 0;
    if (cudaMalloc(buf, need) != cudaSuccess) {
        cudaGetLastError();
        *buf = nullptr;
        return fail(ctx, KB_ERR_OOM, "cannot allocate %zu bytes of device memory", need);
    }
    *have = need;
    return KB_OK;
}

kb_status read_counters(kb_context* ctx) {
    KB_CUDA(ctx, cudaMemcpyAsync(ctx->h_ctr, ctx->d_ctr, sizeof(Counters), cudaMemcpyDeviceToHost, ctx->stream));
    KB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return KB_OK;
}

kb_status device_error(kb_context* ctx) {
    const int32_t e = ctx->h_ctr->err;
    if (e & kb::kErrInvalid)
        return fail(ctx, KB_ERR_INVALID_ARG, "row_offsets not monotone from 0 to m, or a neighbour id out of [0, n)");
    if (e & kb::kErrTableFull) return fail(ctx, KB_ERR_TABLE_FULL, "block table probe limit reached");
    if (e & (kb::kErrStage | kb::kErrHubSet)) return fail(ctx, KB_ERR_DEVICE_CHECK, "device consistency check failed (%d)", e);
    return KB_OK;
}

// Build the processed CSR (IN / BOTH) into `base` (layout_csr offsets).
kb_status build_processed_csr(kb_context* ctx, const kb_graph* g, Plan& P, char* base) {
    if (!needs_in_csr(P.dir)) return KB_OK;
    int64_t* inpref = reinterpret_cast<int64_t*>(base + P.o_inpref);
    KB_CUDA(ctx, cudaMemsetAsync(inpref, 0, sizeof(int64_t) * (size_t)(P.n + 1), ctx->stream));
    kb::launch_in_degree(P.m, g->col_indices, inpref, ctx->stream);
    kb::launch_scan_i64(inpref, P.n, inpref, reinterpret_cast<int64_t*>(base + P.o_i64tmp), ctx->stream);
    kb::launch_build_csr(P.n, P.m, g->row_offsets, g->col_indices, P.labels ? g->edge_labels : nullptr, inpref,
                         P.dir == KB_DIR_BOTH ? 1 : 0, reinterpret_cast<int64_t*>(base + P.o_rowp),
                         reinterpret_cast<int32_t*>(base + P.o_colp),
                         P.labels ? reinterpret_cast<int32_t*>(base + P.o_labp) : nullptr,
                         reinterpret_cast<int64_t*>(base + P.o_cursor), ctx->stream);
    KB_CUDA(ctx, cudaGetLastError());
    return KB_OK;
}

// Discover hubs of the processed CSR and fill the host side of the plan.
kb_status plan_hubs(kb_context* ctx, Plan& P, const int64_t* row_p) {
    P.hub_v.clear();
    P.chunk_off.assign(1, 0);
    P.set_off.assign(1, 0);
    P.chunk_hub.clear();
    P.n_hubs = 0;
    P.n_chunks = P.set_slots = 0;
    if (P.n == 0 || P.m_proc == 0) return KB_OK;
    const int64_t hmax = std::min<int64_t>(P.n, P.m_proc / (P.thr + 1) + 1);
    const size_t deg_off = align_up(sizeof(int32_t) * (size_t)hmax);
    KB_TRY(ensure_buffer(ctx, &ctx->hub_tmp, &ctx->hub_tmp_bytes, deg_off + sizeof(int64_t) * (size_t)hmax));
    int32_t* d_v = reinterpret_cast<int32_t*>(ctx->hub_tmp);
    int64_t* d_deg = reinterpret_cast<int64_t*>(reinterpret_cast<char*>(ctx->hub_tmp) + deg_off);
    KB_CUDA(ctx, cudaMemsetAsync(ctx->d_hub_n, 0, sizeof(int32_t), ctx->stream));
    kb::launch_find_hubs(P.n, row_p, P.thr, d_v, d_deg, ctx->d_hub_n, ctx->stream);
    KB_CUDA(ctx, cudaGetLastError());
    KB_CUDA(ctx, cudaMemcpyAsync(ctx->h_hub_n, ctx->d_hub_n, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
    KB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    const int32_t H = *ctx->h_hub_n;
    if (H <= 0) return KB_OK;
    if (H > hmax) return fail(ctx, KB_ERR_DEVICE_CHECK, "hub count exceeds bound");
    std::vector<int32_t> hv((size_t)H);
    std::vector<int64_t> hd((size_t)H);
    KB_CUDA(ctx, cudaMemcpy(hv.data(), d_v, sizeof(int32_t) * (size_t)H, cudaMemcpyDeviceToHost));
    KB_CUDA(ctx, cudaMemcpy(hd.data(), d_deg, sizeof(int64_t) * (size_t)H, cudaMemcpyDeviceToHost));
    std::vector<int32_t> order((size_t)H);
    for (int32_t i = 0; i < H; ++i) order[(size_t)i] = i;
    std::sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return hv[(size_t)a] < hv[(size_t)b]; });
    P.hub_v.resize((size_t)H);
    std::vector<int64_t> deg((size_t)H);
    for (int32_t i = 0; i < H; ++i) {
        P.hub_v[(size_t)i] = hv[(size_t)order[(size_t)i]];
        deg[(size_t)i] = hd[(size_t)order[(size_t)i]];
    }
    P.chunk_off.resize((size_t)H + 1);
    P.set_off.resize((size_t)H + 1);
    for (int32_t i = 0; i < H; ++i) {
        const int64_t d = deg[(size_t)i];
        P.chunk_off[(size_t)i + 1] = P.chunk_off[(size_t)i] + (d + P.hub_chunk - 1) / P.hub_chunk;
        P.set_off[(size_t)i + 1] = P.set_off[(size_t)i] + kb::hub_set_capacity(d);
    }
    P.chunk_hub.resize((size_t)P.chunk_off[(size_t)H]);
    for (int32_t i = 0; i < H; ++i)
        for (int64_t c = P.chunk_off[(size_t)i]; c < P.chunk_off[(size_t)i + 1]; ++c) P.chunk_hub[(size_t)c] = i;
    P.n_hubs = (size_t)H;
    P.n_chunks = P.chunk_off[(size_t)H];
    P.set_slots = P.set_off[(size_t)H];
    return KB_OK;
}

// Size class of a call, the key of the tuning cache: single graphs by
// floor(log2) of their processed edges, batches (64 + ...) by floor(log2) of
// the processed edges per graph.
int32_t size_class(int64_t m_proc, int64_t graphs, bool batch) {
    const int64_t per = std::max<int64_t>(1, m_proc / std::max<int64_t>(graphs, 1));
    int32_t c = 0;
    while ((per >> (c + 1)) > 0) ++c;
    return batch ? 64 + c : c;
}

// The cached tuning of class c, else of the nearest class of the same kind
// at most 3 classes (a factor of 8 in edges) away, else nullptr.
const kb_tuning* tuned_for(const kb_context* ctx, int32_t c) {
    const kb_tuning* best = nullptr;
    int32_t dist = 4;
    for (const auto& kv : ctx->tuned) {
        if ((kv.first >= 64) != (c >= 64)) continue;
        const int32_t d = std::abs(kv.first - c);
        if (d < dist) {
            dist = d;
            best = &kv.second;
        }
    }
    return best;
}

int32_t pick_field(int32_t given, int32_t cached, int32_t dflt) { return given ? given : (cached ? cached : dflt); }

// The plan fields a call may choose on a prepared graph: key subject, frozen
// blocks, table size, medium split and warp task size.
void resolve_call_fields(Plan& P, const kb_options* opt, int rounds, bool multi, const kb_tuning* T) {
    P.subject = opt->subject;
    // stratified rounds of one graph or (multi) of batched and served graphs;
    // incremental refinement plans without, and generic CSE keys need not
    // hold the own previous block
    P.freeze = (rounds >= 0 || multi) && P.subject == KB_SUBJECT_PREVIOUS && opt->rekey_all == 0;
    P.dense0 = !multi;
    P.med_split = pick_field(opt->medium_split, T ? T->medium_split : 0, kb::kDefaultMedSplit);
    P.warp_verts = pick_field(opt->small_task_vertices, T ? T->small_task_vertices : 0, kb::kDefaultWarpVerts);
    float lf = opt->load_factor > 0.f ? opt->load_factor : (T ? T->load_factor : 0.f);
    if (!(lf > 0.f)) lf = 0.5f;
    P.cap = table_capacity(P.n, lf);
}

// `rounds`: refinement rounds the call runs (decides the automatic locality
// order); negative for batched and served refinement, which never reorder.
// With P.graph_ext set (building a prepared graph) the automatic locality
// order is on for at least 2^22 processed edges: its cost is paid once.
kb_status make_plan(kb_context* ctx, const kb_graph* g, const kb_options* opt, Plan& P, char** csr_base_out,
                    bool for_query, int rounds, bool multi = false) {
    P.n = g->n;
    P.m = g->m;
    P.dir = opt->direction;
    P.m_proc = P.dir == KB_DIR_BOTH ? 2 * g->m : g->m;
    const bool auto_order = P.graph_ext || rounds >= 24;
    P.reorder = rounds >= 0 && P.n > 0 && P.m_proc > 0 &&
                (opt->reorder == 2 || (opt->reorder == 0 && auto_order && P.m_proc >= ((int64_t)1 << 22)));
    P.labels = opt->use_edge_labels && g->edge_labels != nullptr;
    // tuning fields: the options' value, else the cached tuning of the call's
    // size class, else the library default
    P.size_class = size_class(P.m_proc, multi ? ctx->plan_graphs : 1, multi);
    const kb_tuning* T = tuned_for(ctx, P.size_class);
    P.thr = pick_field(opt->hub_threshold, T ? T->hub_threshold : 0, kb::kDefaultHubThreshold);
    P.hub_chunk = pick_field(opt->hub_chunk_edges, T ? T->hub_chunk_edges : 0, kb::kDefaultHubChunk);
    P.small_max = std::min(pick_field(opt->small_max_degree, T ? T->small_max_degree : 0, kb::kSmallDegree), P.thr);
    resolve_call_fields(P, opt, rounds, multi, T);
    layout_csr(P);
    const int64_t* row_p = g->row_offsets;
    char* csr_base = nullptr;
    if (needs_in_csr(P.dir)) {
        // The processed CSR is needed to find hubs; during a size query it is
        // built in library scratch, otherwise at the head of the workspace.
        if (for_query) {
            KB_TRY(ensure_buffer(ctx, &ctx->plan_tmp, &ctx->plan_tmp_bytes, P.csr_bytes));
            csr_base = reinterpret_cast<char*>(ctx->plan_tmp);
        } else {
            csr_base = *csr_base_out;
        }
        KB_TRY(build_processed_csr(ctx, g, P, csr_base));
        row_p = reinterpret_cast<const int64_t*>(csr_base + P.o_rowp);
    }
    KB_TRY(plan_hubs(ctx, P, row_p));
    layout_round(P);
    return KB_OK;
}

// Acquire a workspace of `bytes`; returns its base.
kb_status acquire_workspace(kb_context* ctx, size_t bytes, char** base) {
    if (ctx->user_ws) {
        if (bytes > ctx->user_ws_bytes)
            return fail(ctx, KB_ERR_OOM, "caller workspace holds %zu bytes, %zu needed", ctx->user_ws_bytes, bytes);
        *base = reinterpret_cast<char*>(ctx->user_ws);
        return KB_OK;
    }
    KB_TRY(ensure_buffer(ctx, &ctx->own_ws, &ctx->own_ws_bytes, std::max<size_t>(bytes, 256)));
    *base = reinterpret_cast<char*>(ctx->own_ws);
    return KB_OK;
}

struct Timer {
    kb_context* ctx;
    int used = 0;
    int fam[10];
    explicit Timer(kb_context* c) : ctx(c) {}
    void begin(int family) {
        if (!ctx->timing || used >= 10) return;
        fam[used] = family;
        cudaEventRecord(ctx->ev[2 * used], ctx->stream);
    }
    void end() {
        if (!ctx->timing || used >= 10) return;
        cudaEventRecord(ctx->ev[2 * used + 1], ctx->stream);
        ++used;
    }
    // after a stream sync
    float collect() {
        float round = 0.f;
        if (!ctx->timing) return 0.f;
        for (int i = 0; i < used; ++i) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ctx->ev[2 * i], ctx->ev[2 * i + 1]);
            ctx->kernel_ms[fam[i]] += ms;
            ctx->kernel_launches[fam[i]] += 1;
            round += ms;
        }
        if (used > 0) {
            float span = 0.f;
            cudaEventElapsedTime(&span, ctx->ev[0], ctx->ev[2 * used - 1]);
            round = span;
        }
        used = 0;
        return round;
    }
};

// Everything one refine call needs on the device: the plan, the bound round
// parameters and the table epoch.
struct Prepared {
    Plan P;
    char* ws = nullptr;  // workspace base (round buffers)
    kb::RoundParams p{};
    uint2* prefix = nullptr;  // rank words of the renumbering (launch_renumber)
    uint32_t* scan_tmp = nullptr;
    int64_t total_chunks = 0;
    size_t set_bytes = 0;
    uint32_t epoch = 0;
    // frozen blocks for the next round and their minima, edgeless vertices
    // (Plan::freeze; RoundParams::frozen)
    uint32_t* frozen = nullptr;
    uint32_t* frozen_min = nullptr;
    uint32_t* edgeless = nullptr;
    // clean blocks (frozen blocks on): the two bitmaps of block minima used in
    // turn (this level's and the previous level's), moved vertices and marked
    // (dirty) blocks; RoundParams::minof
    uint32_t* bm[2] = {nullptr, nullptr};
    int bm_cur = 0;
    uint32_t* moved = nullptr;
    uint32_t* mark = nullptr;
    uint32_t* dense_min = nullptr;  // launch_dense_labels / launch_dense_level0 (Plan::dense0)
    uint2* dense_pair = nullptr;
    bool compact = false;  // small-kernel windows skip frozen vertices (many frozen)
    bool sparse = false;   // fewer than 1/64 of the vertices refine: long warp tasks
    // A caller-held block table (ext_cap slots) and empty-signature minima
    // (at least n entries) that outlive one prepare: they are neither carved
    // from the workspace nor cleared, and the table epoch carries on (the
    // server re-plans its arena at every admission).
    uint64_t* ext_table = nullptr;
    uint64_t ext_cap = 0;
    uint64_t* ext_emin = nullptr;
    // Likewise the frozen-block state (frozen, frozen_min, shared, minof,
    // moved, mark; bitmaps of at least n bits, minof of n entries): kept as it
    // is by prepare, so that blocks stay frozen across a re-plan that moves
    // no vertex (the server's admissions, which append at the arena's tail).
    uint32_t* ext_frozen = nullptr;
    uint32_t* ext_frozen_min = nullptr;
    uint32_t* ext_shared = nullptr;
    uint32_t* ext_minof = nullptr;
    uint32_t* ext_moved = nullptr;
    uint32_t* ext_mark = nullptr;
    bool med_on = true;    // some medium vertex refines this round
    bool hub_on = true;    // some hub refines this round
};

// Bind the per-graph part of a plan into p: the processed CSR (csr: IN /
// BOTH), the hub lists, the locality order and the medium list (gws: graph
// part base).  build: also fill them (hub lists uploaded, chunk extents, the
// locality order, using `count_tmp` (n words) as scratch, the medium list
// and, with `edgeless`, the edgeless bits); else they hold a prepared graph's
// contents.  Synchronises when building.
kb_status bind_graph_part(kb_context* ctx, const kb_graph* g, const Plan& P, char* csr, char* gws, bool build,
                          uint32_t* count_tmp, kb::RoundParams& p, cudaStream_t s) {
    const int64_t n = g->n;
    if (needs_in_csr(P.dir)) {
        p.row = reinterpret_cast<const int64_t*>(csr + P.o_rowp);
        p.col = reinterpret_cast<const int32_t*>(csr + P.o_colp);
        p.lab = P.labels ? reinterpret_cast<const int32_t*>(csr + P.o_labp) : nullptr;
    } else {
        p.row = g->row_offsets;
        p.col = g->col_indices;
        p.lab = P.labels ? g->edge_labels : nullptr;
    }
    const size_t H = P.n_hubs;
    p.n_hubs = (int32_t)H;
    p.hub_v = reinterpret_cast<const int32_t*>(gws + P.o_hubv);
    p.hub_chunk_off = reinterpret_cast<const int64_t*>(gws + P.o_chunk);
    p.hub_set_off = reinterpret_cast<const int64_t*>(gws + P.o_setoff);
    p.chunk_hub = reinterpret_cast<const int32_t*>(gws + P.o_chunkhub);
    p.chunk_ext = reinterpret_cast<const uint64_t*>(gws + P.o_chunkext);
    if (build && H) {
        KB_CUDA(ctx, cudaMemcpyAsync(gws + P.o_hubv, P.hub_v.data(), sizeof(int32_t) * H, cudaMemcpyHostToDevice, s));
        KB_CUDA(ctx, cudaMemcpyAsync(gws + P.o_chunk, P.chunk_off.data(), sizeof(int64_t) * (H + 1),
                                     cudaMemcpyHostToDevice, s));
        KB_CUDA(ctx, cudaMemcpyAsync(gws + P.o_setoff, P.set_off.data(), sizeof(int64_t) * (H + 1),
                                     cudaMemcpyHostToDevice, s));
        KB_CUDA(ctx, cudaMemcpyAsync(gws + P.o_chunkhub, P.chunk_hub.data(), sizeof(int32_t) * P.chunk_hub.size(),
                                     cudaMemcpyHostToDevice, s));
        kb::launch_chunk_ext((int64_t)P.chunk_hub.size(), p.chunk_hub, p.hub_v, p.hub_chunk_off, p.row, P.hub_chunk,
                             reinterpret_cast<uint64_t*>(gws + P.o_chunkext), s);
        KB_CUDA(ctx, cudaGetLastError());
    }
    if (P.reorder) {
        int32_t* perm = reinterpret_cast<int32_t*>(gws + P.o_perm);
        int32_t* colr = needs_in_csr(P.dir) ? const_cast<int32_t*>(p.col) : reinterpret_cast<int32_t*>(gws + P.o_colr);
        if (build) {
            // rank vertices by how often they are gathered and move the
            // neighbour ids to those ranks
            kb::launch_locality_order(n, P.m_proc, p.col, count_tmp,
                                      reinterpret_cast<unsigned long long*>(gws + P.o_hist), perm, s);
            kb::launch_remap_cols(P.m_proc, p.col, perm, colr, s);
            KB_CUDA(ctx, cudaGetLastError());
        }
        p.col = colr;
        p.perm = perm;
    }
    p.med_v = reinterpret_cast<int32_t*>(gws + P.o_med);
    if (build) {
        p.n_med = 0;
        if (g->m > 0) {
            KB_CUDA(ctx, cudaMemsetAsync(ctx->d_med_n, 0, sizeof(int64_t), s));
            kb::launch_classify(n, p.row, p.small_max, P.thr, const_cast<int32_t*>(p.med_v), ctx->d_med_n, s);
            KB_CUDA(ctx, cudaGetLastError());
            KB_CUDA(ctx, cudaMemcpyAsync(ctx->h_med_n, ctx->d_med_n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            KB_CUDA(ctx, cudaStreamSynchronize(s));
            p.n_med = *ctx->h_med_n;
        }
        if (P.freeze || P.graph_ext)  // laid out only then
            kb::launch_edgeless_bits(n, p.row, reinterpret_cast<uint32_t*>(gws + P.o_edgeless), s);
        KB_CUDA(ctx, cudaGetLastError());
    }
    return KB_OK;
}

// Validate, plan, acquire the workspace, bind the round parameters, list the
// medium vertices and reset the per-call state (block table, empty-signature
// minima).  With a prepared graph (pg) only the per-call part is planned and
// reset.  Synchronises.
kb_status prepare(kb_context* ctx, const kb_graph* g, const kb_options* opt, Prepared& R, int rounds,
                  bool multi = false, const kb_prepared* pg = nullptr) {
    cudaStream_t s = ctx->stream;
    const int64_t n = g->n;
    KB_CUDA(ctx, cudaMemsetAsync(ctx->d_ctr, 0, sizeof(Counters), s));
    Plan& P = R.P;
    char* csr = nullptr;
    char* gws = nullptr;
    char* ws = nullptr;
    kb::RoundParams& p = R.p;
    p = kb::RoundParams{};
    p.n = n;
    p.ctr = ctx->d_ctr;
    if (pg) {
        P = pg->P;
        P.ext_table = R.ext_table != nullptr;
        P.ext_freeze = R.ext_frozen != nullptr;
        resolve_call_fields(P, opt, rounds, multi, tuned_for(ctx, P.size_class));
        layout_round(P);
        KB_TRY(acquire_workspace(ctx, P.total, &ws));
        p.small_max = P.small_max;
        csr = pg->csr;
        gws = pg->gbuf;
        KB_TRY(bind_graph_part(ctx, g, P, csr, gws, false, nullptr, p, s));
        p.n_med = pg->n_med;
    } else {
        if (opt->validate) {
            kb::launch_validate(n, g->m, g->row_offsets, g->col_indices, ctx->d_ctr, s);
            KB_CUDA(ctx, cudaGetLastError());
            KB_TRY(read_counters(ctx));
            KB_TRY(device_error(ctx));
        }
        // The processed CSR sits at the head of the workspace, so its size is known
        // before the hub layout.
        Plan probe;
        probe.n = n;
        probe.m = g->m;
        probe.dir = opt->direction;
        probe.m_proc = probe.dir == KB_DIR_BOTH ? 2 * g->m : g->m;
        probe.labels = opt->use_edge_labels && g->edge_labels != nullptr;
        layout_csr(probe);
        char* base = nullptr;
        if (probe.csr_bytes) {
            // The hub layout is not known yet: reserve the CSR part first.  A
            // library-owned workspace keeps its contents when it does not grow.
            if (ctx->user_ws) {
                KB_TRY(acquire_workspace(ctx, probe.csr_bytes, &base));
            } else {
                KB_TRY(ensure_buffer(ctx, &ctx->plan_tmp, &ctx->plan_tmp_bytes, probe.csr_bytes));
                base = reinterpret_cast<char*>(ctx->plan_tmp);
            }
        }
        P.ext_table = R.ext_table != nullptr;
        P.ext_freeze = R.ext_frozen != nullptr;
        KB_TRY(make_plan(ctx, g, opt, P, &base, false, rounds, multi));
        if (ctx->user_ws) {
            KB_TRY(acquire_workspace(ctx, P.total, &ws));
        } else {
            // round buffers live in the owned workspace; the CSR stays in plan_tmp
            const size_t csr_bytes = P.csr_bytes;
            P.csr_bytes = 0;
            layout_round(P);
            P.csr_bytes = csr_bytes;
            KB_TRY(ensure_buffer(ctx, &ctx->own_ws, &ctx->own_ws_bytes, std::max<size_t>(P.total, 256)));
            ws = reinterpret_cast<char*>(ctx->own_ws);
        }
        csr = base;
        gws = ws;
        p.small_max = P.small_max;
        // the slot array serves as the count buffer of the locality order:
        // every round rewrites it
        KB_TRY(bind_graph_part(ctx, g, P, csr, gws, true, reinterpret_cast<uint32_t*>(ws + P.o_slot), p, s));
    }
    R.ws = ws;
    p.hub_threshold = P.thr;
    p.small_max = P.small_max;
    p.warp_verts = P.warp_verts;
    p.hub_chunk = P.hub_chunk;
    p.med_split = P.med_split;
    p.hash_mode = opt->hash_mode;
    p.table = R.ext_table ? R.ext_table : reinterpret_cast<uint64_t*>(ws + P.o_table);
    p.mask = (R.ext_table ? R.ext_cap : P.cap) - 1;
    p.slot_of = reinterpret_cast<int32_t*>(ws + P.o_slot);
    if (R.ext_table) {
        p.emin = R.ext_emin;  // entries of earlier rounds carry a larger round word and lose
    } else {
        p.emin = reinterpret_cast<uint64_t*>(ws + P.o_emin);
        KB_CUDA(ctx, cudaMemsetAsync(p.emin, 0xff, sizeof(uint64_t) * (size_t)n, s));
    }
    p.bitmap = reinterpret_cast<uint32_t*>(ws + P.o_bitmap);
    p.ctr = ctx->d_ctr;
    p.hub_sets = reinterpret_cast<uint64_t*>(ws + P.o_sets);
    p.hub_acc = reinterpret_cast<uint64_t*>(ws + P.o_acc);
    p.hub_cnt = reinterpret_cast<uint32_t*>(ws + P.o_cnt);
    if (P.reorder) p.gat = reinterpret_cast<int32_t*>(ws + P.o_gat);
    R.prefix = reinterpret_cast<uint2*>(ws + P.o_prefix);
    R.scan_tmp = reinterpret_cast<uint32_t*>(ws + P.o_scan);
    if (P.dense0) {
        R.dense_min = reinterpret_cast<uint32_t*>(ws + P.o_dense);
        R.dense_pair = reinterpret_cast<uint2*>(ws + P.o_dense + align_up(sizeof(uint32_t) * kb::kDenseLabels));
    }
    R.total_chunks = P.n_chunks;
    R.set_bytes = sizeof(uint64_t) * (size_t)P.set_slots;
    if (!R.ext_table) {
        KB_CUDA(ctx, cudaMemsetAsync(p.table, 0, sizeof(uint64_t) * (size_t)P.cap, s));
        R.epoch = 0;
    }
    if (P.freeze) {
        R.edgeless = reinterpret_cast<uint32_t*>(gws + P.o_edgeless);
        R.bm[0] = p.bitmap;
        R.bm[1] = reinterpret_cast<uint32_t*>(ws + P.o_bm2);
        R.bm_cur = 0;
        if (R.ext_frozen) {
            // the caller's state, kept as it is
            R.frozen = R.ext_frozen;
            R.frozen_min = R.ext_frozen_min;
            p.shared = R.ext_shared;
            p.minof = R.ext_minof;
            R.moved = R.ext_moved;
            R.mark = R.ext_mark;
        } else {
            // nothing frozen before the starting level; shared starts empty
            const size_t bw = sizeof(uint32_t) * (size_t)((n >> 5) + 1);
            R.frozen = reinterpret_cast<uint32_t*>(ws + P.o_frozen);
            R.frozen_min = reinterpret_cast<uint32_t*>(ws + P.o_fmin);
            p.shared = reinterpret_cast<uint32_t*>(ws + P.o_shared);
            p.minof = reinterpret_cast<uint32_t*>(ws + P.o_minof);
            R.moved = reinterpret_cast<uint32_t*>(ws + P.o_moved);
            R.mark = reinterpret_cast<uint32_t*>(ws + P.o_mark);
            KB_CUDA(ctx, cudaMemsetAsync(R.frozen, 0, bw, s));
            KB_CUDA(ctx, cudaMemsetAsync(R.frozen_min, 0, bw, s));
            KB_CUDA(ctx, cudaMemsetAsync(p.shared, 0, bw, s));
        }
        KB_CUDA(ctx, cudaGetLastError());
    }
    return KB_OK;
}

// Advance the table epoch (entries of other epochs read as empty); the table
// is cleared once every 255 rounds.
kb_status next_epoch(kb_context* ctx, Prepared& R, cudaStream_t s) {
    if (R.epoch == 255) {
        KB_CUDA(ctx, cudaMemsetAsync(R.p.table, 0, sizeof(uint64_t) * (size_t)(R.p.mask + 1), s));
        R.epoch = 0;
    }
    R.p.epoch = ++R.epoch;
    return KB_OK;
}

// Starting level: canonical renumbering of `key` (labels or a given
// partition; all-zero partition when key is NULL in a batched run).
kb_status launch_level0(kb_context* ctx, Prepared& R, const int32_t* key, int32_t* out, cudaStream_t s) {
    KB_TRY(next_epoch(ctx, R, s));
    KB_CUDA(ctx, cudaMemsetAsync(ctx->d_ctr, 0, sizeof(Counters), s));
    KB_CUDA(ctx, cudaMemsetAsync(R.p.bitmap, 0, sizeof(uint32_t) * (size_t)((R.p.n >> 5) + 1), s));
    R.p.prev = key;
    R.p.frozen = nullptr;
    R.p.frozen_min = nullptr;
    // small non-negative keys (one graph): each label's smallest vertex
    // directly; the check for the range costs one host round trip
    bool dense = false;
    if (key && R.dense_min && !kb::batched(R.p) && R.p.n > 0) {
        KB_CUDA(ctx, cudaMemsetAsync(R.dense_min, 0xff, sizeof(uint32_t) * kb::kDenseLabels, s));
        kb::launch_dense_labels(R.p.n, key, R.dense_min, ctx->d_ctr, s);
        KB_TRY(read_counters(ctx));
        dense = ctx->h_ctr->dense_bad == 0;
    }
    if (dense) {
        kb::launch_dense_level0(R.p, key, R.dense_min, R.dense_pair, R.prefix, R.scan_tmp, out, s);
    } else {
        kb::launch_small_round(R.p, true, false, s);
        kb::launch_renumber(R.p, R.prefix, R.scan_tmp, out, s);
    }
    // a starting level may mix edgeless vertices with others in one block:
    // only its singletons are frozen in the first round
    if (R.p.shared) {
        kb::launch_freeze_clean(R.p.n, R.p.bitmap, R.p.shared, nullptr, out, nullptr, R.frozen, R.frozen_min,
                                ctx->d_ctr, s);
        kb::launch_count_refining(R.p, R.frozen, ctx->d_ctr, s);
    }
    KB_CUDA(ctx, cudaGetLastError());
    return KB_OK;
}

// One refinement round up to (not including) the renumbering.
kb_status launch_round_body(kb_context* ctx, Prepared& R, cudaStream_t s, Timer* T) {
    kb::RoundParams& p = R.p;
    // with frozen blocks, the medium and hub kernels run only while some of
    // their vertices refine (after the first rounds, hubs are mostly alone in
    // their blocks)
    const bool med = p.n_med && (!p.frozen || R.med_on);
    const bool hub = p.n_hubs && (!p.frozen || R.hub_on);
    if (T) T->begin(KB_KERNEL_OTHER);
    KB_CUDA(ctx, cudaMemsetAsync(ctx->d_ctr, 0, sizeof(Counters), s));
    kb::launch_clear_round(p, s);
    if (hub && !p.frozen && R.set_bytes) KB_CUDA(ctx, cudaMemsetAsync(p.hub_sets, 0xff, R.set_bytes, s));
    if (T) T->end();
    if (T) T->begin(KB_KERNEL_SMALL);
    if (R.sparse) {
        // few vertices refine: long warp tasks, so that far fewer CTAs set up
        // and flush a join map for a handful of vertices each
        kb::RoundParams q = p;
        q.warp_verts = 4096;
        kb::launch_small_round(q, false, true, s);
    } else {
        kb::launch_small_round(p, false, R.compact, s);
    }
    if (T) T->end();
    if (med) {
        if (T) T->begin(KB_KERNEL_MEDIUM);
        kb::launch_medium_round(p, s);
        if (T) T->end();
    }
    if (hub) {
        if (T) T->begin(KB_KERNEL_HUB_CHUNK);
        if (p.frozen) kb::launch_clear_hub_sets(p, (int64_t)(R.set_bytes / sizeof(uint64_t)), s);
        kb::launch_hub_chunk(p, R.total_chunks, s);
        if (T) T->end();
        if (T) T->begin(KB_KERNEL_HUB_FINAL);
        kb::launch_hub_final(p, s);
        if (T) T->end();
    }
    KB_CUDA(ctx, cudaGetLastError());
    return KB_OK;
}

void reset_timing(kb_context* ctx) {
    ctx->round_ms.clear();
    for (int f = 0; f < KB_KERNEL_COUNT; ++f) {
        ctx->kernel_ms[f] = 0.f;
        ctx->kernel_launches[f] = 0;
    }
}

// Where the levels go: the caller's (k+1) x n array, or (fixpoint mode, levels
// == nullptr) two library buffers used in turn.
struct LevelRows {
    int32_t* levels = nullptr;
    int32_t* ping[2] = {nullptr, nullptr};
    int64_t n = 0;
    // optional host copy of `levels` (kb_refine_host): every row is copied on
    // a second stream as soon as it is final, overlapping the later rounds
    int32_t* host = nullptr;
    int32_t* row(int i) const { return levels ? levels + (size_t)i * (size_t)n : ping[i & 1]; }
};

// Queue the device-to-host copy of rows first..last (final on ctx->stream).
kb_status emit_rows(kb_context* ctx, const LevelRows& rows, int first, int last) {
    if (!rows.host || rows.n == 0 || last < first) return KB_OK;
    KB_CUDA(ctx, cudaEventRecord(ctx->row_ev, ctx->stream));
    KB_CUDA(ctx, cudaStreamWaitEvent(ctx->copy_stream, ctx->row_ev, 0));
    KB_CUDA(ctx, cudaMemcpyAsync(rows.host + (size_t)first * (size_t)rows.n, rows.row(first),
                                 sizeof(int32_t) * (size_t)rows.n * (size_t)(last - first + 1), cudaMemcpyDeviceToHost,
                                 ctx->copy_stream));
    return KB_OK;
}

// Waits for the row copies when leaving refine_core by any path, so no copy
// into the caller's host buffer outlives the call.
struct RowCopyGuard {
    cudaStream_t cs;
    ~RowCopyGuard() {
        if (cs) cudaStreamSynchronize(cs);
    }
};

// The refinement driver shared by kb_refine, kb_refine_from and
// kb_refine_fixpoint.  counts (k+1 entries) may be NULL in fixpoint mode;
// *last_count receives the block count of the last level computed and
// *stopped_stable whether a round reproduced its input partition.
kb_status refine_core(kb_context* ctx, const kb_graph* g, const kb_options* opt, const int32_t* start, int i_start,
                      int k, const LevelRows& rows, int64_t* counts, int* levels_computed, int64_t* last_count,
                      bool* stopped_stable = nullptr, const kb_prepared* pg = nullptr) {
    const int64_t n = g->n;
    const bool fixpoint = rows.levels == nullptr;
    if (levels_computed) *levels_computed = i_start;
    if (stopped_stable) *stopped_stable = false;
    if (n == 0) {
        if (counts)
            for (int i = i_start; i <= k; ++i) counts[i] = 0;
        if (last_count) *last_count = 0;
        return KB_OK;
    }
    cudaStream_t s = ctx->stream;
    ctx->round_keyed.clear();
    RowCopyGuard copies{rows.host ? ctx->copy_stream : nullptr};
    Prepared R;
    KB_TRY(prepare(ctx, g, opt, R, k - i_start, false, pg));
    kb::RoundParams& p = R.p;

    // ---- the subject part of every key (generic CSE rounds)
    if (R.P.subject) {
        int32_t* own = reinterpret_cast<int32_t*>(R.ws + R.P.o_ownkey);
        if (R.P.subject == KB_SUBJECT_ALL || (R.P.subject == KB_SUBJECT_LABEL && !g->vertex_labels)) {
            kb::launch_fill_i32(own, n, 0, s);
        } else if (R.P.subject == KB_SUBJECT_ID) {
            kb::launch_iota_i32(own, n, s);
        } else {
            // label classes with canonical ids < n (the level-0 pass on the labels)
            KB_TRY(launch_level0(ctx, R, g->vertex_labels, own, s));
            KB_TRY(read_counters(ctx));
            KB_TRY(device_error(ctx));
        }
        KB_CUDA(ctx, cudaGetLastError());
    }

    // ---- the starting level
    int32_t* row0 = rows.row(i_start);
    const int32_t* init_key = start ? start : (opt->use_vertex_labels ? g->vertex_labels : nullptr);
    int64_t prev_count = 1;
    if (init_key) {
        KB_TRY(launch_level0(ctx, R, init_key, row0, s));
        KB_TRY(read_counters(ctx));
        KB_TRY(device_error(ctx));
        prev_count = ctx->h_ctr->count;
        R.compact = R.P.freeze && ctx->h_ctr->frozen * 4 > n;
        R.sparse = R.P.freeze && (n - ctx->h_ctr->frozen) * 64 < n;
        R.med_on = ctx->h_ctr->med_on > 0;
        R.hub_on = ctx->h_ctr->hub_on > 0;
    } else {
        kb::launch_fill_i32(row0, n, 0, s);
        if (p.perm) kb::launch_fill_i32(p.gat, n, 0, s);
        if (p.minof) {
            // P_0 = {V}: one block, whose smallest member is vertex 0
            kb::launch_fill_i32(reinterpret_cast<int32_t*>(p.minof), n, 0, s);
            KB_CUDA(ctx, cudaMemsetAsync(p.bitmap, 0, sizeof(uint32_t) * (size_t)((n >> 5) + 1), s));
            kb::launch_fill_i32(reinterpret_cast<int32_t*>(p.bitmap), 1, 1, s);
        }
    }
    if (counts) counts[i_start] = prev_count;
    if (last_count) *last_count = prev_count;
    KB_TRY(emit_rows(ctx, rows, i_start, i_start));

    // ---- refinement rounds
    for (int i = i_start + 1; i <= k; ++i) {
        Timer T(ctx);
        KB_TRY(next_epoch(ctx, R, s));
        p.ehigh = 0xffffffffu - (uint32_t)(i - i_start);
        p.prev = rows.row(i - 1);
        p.own_key = R.P.subject ? reinterpret_cast<const int32_t*>(R.ws + R.P.o_ownkey) : nullptr;
        p.frozen = R.frozen;
        p.frozen_min = R.frozen_min;
        if (p.minof) {
            // the minima of level i-1 stay readable while level i's are built
            p.bitmap_prev = R.bm[R.bm_cur];
            R.bm_cur ^= 1;
            p.bitmap = R.bm[R.bm_cur];
            p.moved = R.moved;
        }
        int32_t* out = rows.row(i);
        KB_TRY(launch_round_body(ctx, R, s, &T));
        if (ctx->work) kb::launch_round_work(p, s);
        T.begin(KB_KERNEL_RENUMBER);
        // under early stop a round that keeps the count is the last one
        const int64_t stable = (opt->early_stop || fixpoint) && !R.P.subject ? prev_count : -1;
        kb::launch_renumber(p, R.prefix, R.scan_tmp, out, s, stable);
        KB_TRY(emit_rows(ctx, rows, i, i));
        // the next round's frozen blocks: singletons; a block formed by this
        // round that holds an edgeless vertex holds only edgeless vertices with
        // one previous block; and clean blocks, none of whose members has an
        // edge to a vertex whose smallest block member this round changed
        if (p.shared) {
            KB_CUDA(ctx, cudaMemsetAsync(R.mark, 0, sizeof(uint32_t) * (size_t)((n >> 5) + 1), s));
            kb::launch_dirty_blocks(p, R.edgeless, R.moved, out, kb::kMaxHubThreshold, R.mark, s, stable);
            kb::launch_freeze_clean(n, p.bitmap, p.shared, R.edgeless, out, R.mark, R.frozen, R.frozen_min,
                                    ctx->d_ctr, s, nullptr, nullptr, stable);
            kb::launch_count_refining(p, R.frozen, ctx->d_ctr, s);
        }
        T.end();
        // CSE levels need not refine each other: compare whole levels
        if (R.P.subject) kb::launch_levels_differ(out, p.prev, n, ctx->d_ctr, s);
        KB_CUDA(ctx, cudaGetLastError());
        KB_TRY(read_counters(ctx));
        if (ctx->work) {
            const Counters& hc = *ctx->h_ctr;
            ctx->round_keyed.push_back(
                {hc.keyed_v[0], hc.keyed_v[1], hc.keyed_v[2], hc.keyed_e[0], hc.keyed_e[1], hc.keyed_e[2]});
        }
        // compacted small-kernel windows pay once a quarter of the vertices are frozen
        R.compact = R.P.freeze && ctx->h_ctr->frozen * 4 > n;
        R.sparse = R.P.freeze && (n - ctx->h_ctr->frozen) * 64 < n;
        R.med_on = ctx->h_ctr->med_on > 0;
        R.hub_on = ctx->h_ctr->hub_on > 0;
        ctx->round_ms.push_back(T.collect());
        KB_TRY(device_error(ctx));
        const int64_t c = ctx->h_ctr->count;
        if (counts) counts[i] = c;
        if (last_count) *last_count = c;
        if (levels_computed) *levels_computed = i;
        const bool unchanged = R.P.subject ? ctx->h_ctr->diff == 0 : c == prev_count;
        if ((opt->early_stop || fixpoint) && unchanged) {
            // stratified levels only split blocks, so an unchanged count means an
            // unchanged partition; generic CSE levels were compared entry by entry
            if (stopped_stable) *stopped_stable = true;
            if (!fixpoint && i < k) {
                kb::launch_copy_rows(rows.levels, n, i, i + 1, k, s);
                KB_TRY(emit_rows(ctx, rows, i + 1, k));
            }
            if (counts)
                for (int j = i + 1; j <= k; ++j) counts[j] = c;
            KB_CUDA(ctx, cudaGetLastError());
            break;
        }
        prev_count = c;
    }
    KB_CUDA(ctx, cudaStreamSynchronize(s));
    return KB_OK;
}

kb_status refine_impl(kb_context* ctx, const kb_graph* g, const kb_options* opt, const int32_t* start, int i_start,
                      int k, int32_t* levels, int64_t* counts, int* levels_computed,
                      const kb_prepared* pg = nullptr, int32_t* host_levels = nullptr);

// Incremental refinement (kb_refine_update): levels holds the levels of the
// graph before the change (same options); each round re-keys only the work set
// and keeps the old grouping elsewhere (see kb_update.cu), then renumbers.
kb_status update_impl(kb_context* ctx, const kb_graph* g, const kb_options* opt, int k, const int32_t* changed,
                      int64_t n_changed, int32_t* levels, int64_t* counts, int* levels_computed, int64_t* work) {
    KB_TRY(check_graph(ctx, g, opt, k));
    if (opt->subject != KB_SUBJECT_PREVIOUS)
        return fail(ctx, KB_ERR_INVALID_ARG, "incremental refinement takes subject = KB_SUBJECT_PREVIOUS only");
    if (!counts) return fail(ctx, KB_ERR_INVALID_ARG, "counts is NULL");
    if (n_changed < 0 || (n_changed > 0 && !changed)) return fail(ctx, KB_ERR_INVALID_ARG, "bad changed list");
    const int64_t n = g->n;
    if (n > 0 && !levels) return fail(ctx, KB_ERR_INVALID_ARG, "levels is NULL");
    KB_CUDA(ctx, cudaSetDevice(ctx->device));
    reset_timing(ctx);
    if (levels_computed) *levels_computed = 0;
    if (n == 0) {
        for (int i = 0; i <= k; ++i) counts[i] = 0;
        if (work)
            for (int i = 0; i <= k; ++i) work[i] = 0;
        return KB_OK;
    }
    cudaStream_t s = ctx->stream;
    auto row = [&](int i) { return levels + (size_t)i * (size_t)n; };

    // scratch: changed, dirty, moved and work-set bitmaps, block flags, kept
    // minima, the old row of the current level, the new level 0, id ranges
    const int64_t nw = (n >> 5) + 1;
    const size_t szb = align_up(sizeof(uint32_t) * (size_t)nw), sz4 = align_up(sizeof(int32_t) * (size_t)n);
    KB_TRY(ensure_buffer(ctx, &ctx->upd_buf, &ctx->upd_buf_bytes, 4 * szb + align_up((size_t)n) + 3 * sz4 + 4 * sz4));
    if (!ctx->d_work && cudaMalloc(reinterpret_cast<void**>(&ctx->d_work), sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, KB_ERR_OOM, "cannot allocate a counter");
    }
    char* b = reinterpret_cast<char*>(ctx->upd_buf);

    // The first round re-keys at least every vertex of an old level-0 block
    // that holds a changed vertex.  When that is over a quarter of the
    // vertices (level-0 blocks are label classes, often huge), recomputing
    // with the frozen blocks of a full refinement costs less than re-keying
    // whole blocks round after round.
    {
        KB_CUDA(ctx, cudaMemsetAsync(ctx->d_ctr, 0, sizeof(Counters), s));
        kb::launch_check_ids(n, row(0), ctx->d_ctr, s);
        uint32_t* scratch = reinterpret_cast<uint32_t*>(b);
        KB_CUDA(ctx, cudaMemsetAsync(scratch, 0, szb, s));
        kb::launch_set_bits(n, n_changed, changed, scratch, ctx->d_ctr, s);
        KB_TRY(read_counters(ctx));
        if (ctx->h_ctr->err & kb::kErrInvalid)
            return fail(ctx, KB_ERR_INVALID_ARG, "old levels or changed vertices hold ids outside [0, n)");
        KB_CUDA(ctx, cudaMemsetAsync(scratch, 0, szb, s));
        KB_CUDA(ctx, cudaMemsetAsync(ctx->d_work, 0, sizeof(unsigned long long), s));
        kb::launch_touched_size(n, n_changed, changed, row(0), scratch, ctx->d_work, s);
        KB_CUDA(ctx, cudaGetLastError());
        unsigned long long w1 = 0;
        KB_CUDA(ctx, cudaMemcpyAsync(&w1, ctx->d_work, sizeof(w1), cudaMemcpyDeviceToHost, s));
        KB_CUDA(ctx, cudaStreamSynchronize(s));
        if ((int64_t)w1 * 4 > n) {
            KB_TRY(refine_impl(ctx, g, opt, nullptr, 0, k, levels, counts, levels_computed));
            if (work) {
                const int lc = levels_computed ? *levels_computed : k;
                for (int i = 0; i <= k; ++i) work[i] = i <= lc ? n : 0;
            }
            return KB_OK;
        }
    }

    Prepared R;
    // no locality order: the dirty pass reads neighbour ids, not ranks
    KB_TRY(prepare(ctx, g, opt, R, -1));
    kb::RoundParams& p = R.p;
    uint32_t* changed_bits = reinterpret_cast<uint32_t*>(b);
    uint32_t* dirty = reinterpret_cast<uint32_t*>(b + szb);
    uint32_t* moved = reinterpret_cast<uint32_t*>(b + 2 * szb);
    uint32_t* wmask = reinterpret_cast<uint32_t*>(b + 3 * szb);
    uint8_t* flag = reinterpret_cast<uint8_t*>(b + 4 * szb);
    char* b2 = b + 4 * szb + align_up((size_t)n);
    uint32_t* kmin = reinterpret_cast<uint32_t*>(b2);
    int32_t* keep = reinterpret_cast<int32_t*>(b2 + sz4);
    int32_t* level0 = reinterpret_cast<int32_t*>(b2 + 2 * sz4);
    int32_t* ranges = reinterpret_cast<int32_t*>(b2 + 3 * sz4);

    // the old levels must be partitions with ids in [0, n); the changed ids too
    KB_CUDA(ctx, cudaMemsetAsync(ctx->d_ctr, 0, sizeof(Counters), s));
    for (int i = 0; i <= k; ++i) kb::launch_check_ids(n, row(i), ctx->d_ctr, s);
    KB_CUDA(ctx, cudaMemsetAsync(changed_bits, 0, szb, s));
    kb::launch_set_bits(n, n_changed, changed, changed_bits, ctx->d_ctr, s);
    KB_CUDA(ctx, cudaGetLastError());
    KB_TRY(read_counters(ctx));
    if (ctx->h_ctr->err & kb::kErrInvalid)
        return fail(ctx, KB_ERR_INVALID_ARG, "old levels or changed vertices hold ids outside [0, n)");

    // level 0 from scratch; its moved vertices start the dirty set
    const int32_t* init_key = opt->use_vertex_labels ? g->vertex_labels : nullptr;
    if (init_key) {
        KB_TRY(launch_level0(ctx, R, init_key, level0, s));
        KB_TRY(read_counters(ctx));
        KB_TRY(device_error(ctx));
        counts[0] = ctx->h_ctr->count;
    } else {
        kb::launch_fill_i32(level0, n, 0, s);
        if (p.perm) kb::launch_fill_i32(p.gat, n, 0, s);
        counts[0] = 1;
    }
    KB_CUDA(ctx, cudaMemsetAsync(wmask, 0xff, szb, s));
    kb::launch_moved(n, wmask, row(0), level0, ranges, moved, s);
    KB_CUDA(ctx, cudaMemcpyAsync(row(0), level0, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s));
    KB_CUDA(ctx, cudaMemsetAsync(ctx->d_ctr, 0, sizeof(Counters), s));
    kb::launch_count_bits(moved, nw, &ctx->d_ctr->moved, s);
    KB_TRY(read_counters(ctx));
    if (work) work[0] = n;

    for (int i = 1; i <= k; ++i) {
        Timer T(ctx);
        // dirty = changed | moved | predecessors of moved; W = their previous-level blocks
        // (the pass over every edge only when some vertex moved)
        const bool any_moved = ctx->h_ctr->moved > 0;
        kb::launch_or_words(nw, changed_bits, moved, dirty, s);
        if (any_moved) kb::launch_dirty_from_moved(n, R.P.m_proc, p.row, p.col, moved, dirty, s);
        KB_CUDA(ctx, cudaMemsetAsync(ctx->d_work, 0, sizeof(unsigned long long), s));
        kb::launch_work_set(n, row(i - 1), dirty, flag, wmask, ctx->d_work, s);
        KB_CUDA(ctx, cudaMemcpyAsync(keep, row(i), sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s));
        kb::launch_keep_min(n, wmask, keep, kmin, s);
        KB_TRY(next_epoch(ctx, R, s));
        p.ehigh = 0xffffffffu - (uint32_t)i;
        p.prev = row(i - 1);
        p.vmask = wmask;
        p.keep_old = keep;
        p.kmin = kmin;
        KB_TRY(launch_round_body(ctx, R, s, &T));
        kb::launch_keep_bits(n, wmask, keep, kmin, p.bitmap, s);
        T.begin(KB_KERNEL_RENUMBER);
        kb::launch_renumber(p, R.prefix, R.scan_tmp, row(i), s);
        T.end();
        kb::launch_moved(n, wmask, keep, row(i), ranges, moved, s);
        kb::launch_count_bits(moved, nw, &ctx->d_ctr->moved, s);
        KB_CUDA(ctx, cudaGetLastError());
        KB_TRY(read_counters(ctx));
        ctx->round_ms.push_back(T.collect());
        KB_TRY(device_error(ctx));
        counts[i] = ctx->h_ctr->count;
        if (work) {
            unsigned long long w = 0;
            KB_CUDA(ctx, cudaMemcpy(&w, ctx->d_work, sizeof(w), cudaMemcpyDeviceToHost));
            work[i] = (int64_t)w;
        }
        if (levels_computed) *levels_computed = i;
        if (opt->early_stop && counts[i] == counts[i - 1]) {
            if (i < k) kb::launch_copy_rows(levels, n, i, i + 1, k, s);
            for (int j = i + 1; j <= k; ++j) {
                counts[j] = counts[i];
                if (work) work[j] = 0;
            }
            KB_CUDA(ctx, cudaGetLastError());
            break;
        }
    }
    p.vmask = nullptr;
    p.keep_old = nullptr;
    p.kmin = nullptr;
    KB_CUDA(ctx, cudaStreamSynchronize(s));
    return KB_OK;
}

kb_status refine_impl(kb_context* ctx, const kb_graph* g, const kb_options* opt, const int32_t* start, int i_start,
                      int k, int32_t* levels, int64_t* counts, int* levels_computed, const kb_prepared* pg,
                      int32_t* host_levels) {
    KB_TRY(check_graph(ctx, g, opt, k));
    if (i_start < 0 || i_start > k) return fail(ctx, KB_ERR_INVALID_ARG, "i_start must be in [0, k]");
    if (!counts) return fail(ctx, KB_ERR_INVALID_ARG, "counts is NULL");
    if (g->n > 0 && !levels) return fail(ctx, KB_ERR_INVALID_ARG, "levels is NULL");
    KB_CUDA(ctx, cudaSetDevice(ctx->device));
    reset_timing(ctx);
    LevelRows rows;
    rows.levels = levels;
    rows.n = g->n;
    rows.host = host_levels;
    if (host_levels && !ctx->copy_stream) {
        KB_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
        KB_CUDA(ctx, cudaEventCreateWithFlags(&ctx->row_ev, cudaEventDisableTiming));
    }
    return refine_core(ctx, g, opt, start, i_start, k, rows, counts, levels_computed, nullptr, nullptr, pg);
}

// Summary graph of (src_level, dst_level): distinct triples in order of first
// occurrence (see kb_summary in kbisim.h).  Scratch is library-owned and
// grow-only (released by kb_destroy), like the refinement workspace.
kb_status summary_impl(kb_context* ctx, const kb_graph* g, int direction, int use_edge_labels,
                       const int32_t* src_level, const int32_t* dst_level, int32_t* out_src, int32_t* out_label,
                       int32_t* out_dst, int64_t capacity, int64_t* count) {
    if (!g || !count) return fail(ctx, KB_ERR_INVALID_ARG, "graph and count must not be NULL");
    if (g->n < 0 || g->m < 0 || g->n > 2147483646LL) return fail(ctx, KB_ERR_INVALID_ARG, "bad n or m");
    if (g->m >= ((int64_t)1 << 32)) return fail(ctx, KB_ERR_INVALID_ARG, "the summary graph takes m < 2^32");
    if (direction != KB_DIR_OUT && direction != KB_DIR_IN)
        return fail(ctx, KB_ERR_INVALID_ARG, "direction must be out or in (call once per direction)");
    if (capacity < 0) return fail(ctx, KB_ERR_INVALID_ARG, "negative capacity");
    if (g->n > 0 && (!g->row_offsets || !src_level || !dst_level))
        return fail(ctx, KB_ERR_INVALID_ARG, "row_offsets and levels must not be NULL");
    if (g->m > 0 && !g->col_indices) return fail(ctx, KB_ERR_INVALID_ARG, "col_indices is NULL");
    if (capacity > 0 && (!out_src || !out_label || !out_dst))
        return fail(ctx, KB_ERR_INVALID_ARG, "output arrays must not be NULL when capacity > 0");
    *count = 0;
    if (g->m == 0) return KB_OK;
    KB_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;
    const int64_t m = g->m;
    const uint64_t cap = std::max<uint64_t>(1024, next_pow2((uint64_t)(m + m / 4 + 64)));
    const int64_t nw = (m >> 5) + 1;
    const size_t sz_table = 16 * (size_t)cap, sz_first = 8 * (size_t)cap, sz_bitmap = 4 * (size_t)nw,
                 sz_prefix = 4 * (size_t)(nw + 1), sz_scan = 4 * kb::scan_tmp_words(nw);
    const size_t total = align_up(sz_table) + align_up(sz_first) + align_up(sz_bitmap) + align_up(sz_prefix) +
                         align_up(sz_scan);
    KB_TRY(ensure_buffer(ctx, &ctx->sum_buf, &ctx->sum_buf_bytes, total));
    char* base = reinterpret_cast<char*>(ctx->sum_buf);
    kb::SummaryParams q{};
    q.n = g->n;
    q.m = m;
    q.row = g->row_offsets;
    q.col = g->col_indices;
    q.lab = use_edge_labels ? g->edge_labels : nullptr;
    q.dir = direction;
    q.lsrc = src_level;
    q.ldst = dst_level;
    size_t off = 0;
    q.table = reinterpret_cast<unsigned long long*>(base + off);
    off += align_up(sz_table);
    q.first = reinterpret_cast<unsigned long long*>(base + off);
    off += align_up(sz_first);
    q.bitmap = reinterpret_cast<uint32_t*>(base + off);
    off += align_up(sz_bitmap);
    uint32_t* prefix = reinterpret_cast<uint32_t*>(base + off);
    off += align_up(sz_prefix);
    uint32_t* scan_tmp = reinterpret_cast<uint32_t*>(base + off);
    q.mask = cap - 1;
    q.ctr = ctx->d_ctr;
    kb_status st = KB_OK;
    auto run = [&]() -> kb_status {
        KB_CUDA(ctx, cudaMemsetAsync(ctx->d_ctr, 0, sizeof(Counters), s));
        KB_CUDA(ctx, cudaMemsetAsync(q.table, 0, sz_table, s));
        KB_CUDA(ctx, cudaMemsetAsync(q.first, 0xff, sz_first, s));
        KB_CUDA(ctx, cudaMemsetAsync(q.bitmap, 0, sz_bitmap, s));
        kb::launch_validate(g->n, m, g->row_offsets, g->col_indices, ctx->d_ctr, s);
        KB_CUDA(ctx, cudaGetLastError());
        KB_TRY(read_counters(ctx));
        KB_TRY(device_error(ctx));
        kb::launch_summary_insert(q, s);
        kb::launch_summary_mark(q, s);
        kb::launch_bitmap_rank(q.bitmap, nw, scan_tmp, prefix, ctx->d_ctr, s);
        KB_CUDA(ctx, cudaGetLastError());
        KB_TRY(read_counters(ctx));
        if (ctx->h_ctr->err & kb::kErrTableFull) return fail(ctx, KB_ERR_TABLE_FULL, "summary table probe limit reached");
        KB_TRY(device_error(ctx));
        *count = ctx->h_ctr->count;
        if (*count > capacity)
            return fail(ctx, KB_ERR_INVALID_ARG, "capacity %lld is below the %lld summary edges", (long long)capacity,
                        (long long)*count);
        kb::launch_summary_emit(q, prefix, out_src, out_label, out_dst, s);
        KB_CUDA(ctx, cudaGetLastError());
        return KB_OK;
    };
    st = run();
    if (cudaStreamSynchronize(s) != cudaSuccess && st == KB_OK) st = fail(ctx, KB_ERR_CUDA, "summary graph failed");
    return st;
}

// Rounds until the partition is stable (or max_rounds), keeping only the
// last two levels.
kb_status fixpoint_impl(kb_context* ctx, const kb_graph* g, const kb_options* opt, const int32_t* initial,
                        int max_rounds, int32_t* final_level, int64_t* count, int* rounds, int* stable) {
    KB_TRY(check_graph(ctx, g, opt, max_rounds));
    if (!count || !rounds) return fail(ctx, KB_ERR_INVALID_ARG, "count and rounds must not be NULL");
    if (g->n > 0 && !final_level) return fail(ctx, KB_ERR_INVALID_ARG, "final_level is NULL");
    KB_CUDA(ctx, cudaSetDevice(ctx->device));
    reset_timing(ctx);
    const int64_t n = g->n;
    LevelRows rows;
    rows.n = n;
    if (n > 0) {
        const size_t half = (sizeof(int32_t) * (size_t)n + 255) & ~(size_t)255;
        KB_TRY(ensure_buffer(ctx, &ctx->fix_buf, &ctx->fix_buf_bytes, 2 * half));
        rows.ping[0] = reinterpret_cast<int32_t*>(ctx->fix_buf);
        rows.ping[1] = reinterpret_cast<int32_t*>(reinterpret_cast<char*>(ctx->fix_buf) + half);
    }
    int last = 0;
    int64_t c = 0;
    bool st = false;
    KB_TRY(refine_core(ctx, g, opt, initial, 0, max_rounds, rows, nullptr, &last, &c, &st));
    *rounds = last;
    *count = c;
    if (stable) *stable = (st || n == 0) ? 1 : 0;
    if (n == 0) return KB_OK;
    KB_CUDA(ctx, cudaMemcpyAsync(final_level, rows.row(last), sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice,
                                 ctx->stream));
    KB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return KB_OK;
}

// Batched refinement of G graphs held as one disjoint union (see
// kb_refine_batch in kbisim.h).  Block ids are union-global while the rounds
// run: the own previous block is part of every key, so vertices of different
// graphs never share a block, and level 0 hashes the graph id into the key.
// Rounds 1..k_max are captured once into a CUDA graph; per-graph stopping is
// decided on the device, so the loop needs no host synchronisation.
kb_status batch_impl(kb_context* ctx, const kb_graph* g, const int64_t* voff_h, int64_t G, const int32_t* k_h,
                     const kb_options* opt, int32_t* levels, int64_t* counts, int32_t* lc_out) {
    if (!g || !opt) return fail(ctx, KB_ERR_INVALID_ARG, "graph and options must not be NULL");
    if (G < 0 || G > (int64_t)1 << 30) return fail(ctx, KB_ERR_INVALID_ARG, "bad graph count");
    if (G > 0 && (!voff_h || !k_h || !counts)) return fail(ctx, KB_ERR_INVALID_ARG, "NULL batch arrays");
    int kmax = 0;
    for (int64_t j = 0; j < G; ++j) {
        if (k_h[j] < 0) return fail(ctx, KB_ERR_INVALID_ARG, "k of graph %lld is negative", (long long)j);
        kmax = std::max(kmax, (int)k_h[j]);
        if (voff_h[j + 1] < voff_h[j]) return fail(ctx, KB_ERR_INVALID_ARG, "graph_vertex_offsets not monotone");
    }
    if (G > 0 && (voff_h[0] != 0 || voff_h[G] != g->n))
        return fail(ctx, KB_ERR_INVALID_ARG, "graph_vertex_offsets must run from 0 to n");
    KB_TRY(check_graph(ctx, g, opt, kmax));
    if (opt->subject != KB_SUBJECT_PREVIOUS)
        return fail(ctx, KB_ERR_INVALID_ARG, "batched refinement takes subject = KB_SUBJECT_PREVIOUS only");
    const int64_t n = g->n;
    if (G == 0) return KB_OK;
    for (int64_t j = 0; j < G * (kmax + 1); ++j) counts[j] = 0;
    if (lc_out)
        for (int64_t j = 0; j < G; ++j) lc_out[j] = 0;
    if (n == 0) return KB_OK;
    if (!levels) return fail(ctx, KB_ERR_INVALID_ARG, "levels is NULL");
    KB_CUDA(ctx, cudaSetDevice(ctx->device));
    reset_timing(ctx);
    cudaStream_t s = ctx->stream;
    Prepared R;
    ctx->plan_graphs = G;
    const kb_status pst = prepare(ctx, g, opt, R, -1, true);
    ctx->plan_graphs = 1;
    KB_TRY(pst);
    kb::RoundParams& p = R.p;

    // batch scratch
    const int64_t nw = (n >> 5) + 1;
    size_t off = 0;
    auto take = [&](size_t b) { size_t o = off; off += align_up(b); return o; };
    const size_t o_vgraph = take(sizeof(int32_t) * (size_t)n);
    const size_t o_voff = take(sizeof(int64_t) * (size_t)(G + 1));
    const size_t o_k = take(sizeof(int32_t) * (size_t)G);
    const size_t o_act = take((size_t)G);
    const size_t o_early = take((size_t)G);
    const size_t o_last = take(sizeof(int32_t) * (size_t)G);
    const size_t o_sticky = take(sizeof(int32_t));
    const size_t o_bases = take(sizeof(uint32_t) * (size_t)(G + 1) * (size_t)(kmax + 1));
    const size_t o_bm2 = take(sizeof(uint32_t) * (size_t)nw);
    KB_TRY(ensure_buffer(ctx, &ctx->batch_ws, &ctx->batch_ws_bytes, off));
    char* b = reinterpret_cast<char*>(ctx->batch_ws);
    int32_t* vgraph = reinterpret_cast<int32_t*>(b + o_vgraph);
    int64_t* voff = reinterpret_cast<int64_t*>(b + o_voff);
    int32_t* kd = reinterpret_cast<int32_t*>(b + o_k);
    uint8_t* gact = reinterpret_cast<uint8_t*>(b + o_act);
    uint8_t* early = reinterpret_cast<uint8_t*>(b + o_early);
    int32_t* glast = reinterpret_cast<int32_t*>(b + o_last);
    int32_t* sticky = reinterpret_cast<int32_t*>(b + o_sticky);
    uint32_t* bases = reinterpret_cast<uint32_t*>(b + o_bases);
    uint32_t* bm_a = p.bitmap;
    uint32_t* bm_b = reinterpret_cast<uint32_t*>(b + o_bm2);
    std::vector<uint8_t> act_h((size_t)G), early_h((size_t)G, (uint8_t)(opt->early_stop ? 1 : 0));
    for (int64_t j = 0; j < G; ++j) act_h[(size_t)j] = k_h[j] > 0 ? 1 : 0;
    KB_CUDA(ctx, cudaMemcpyAsync(voff, voff_h, sizeof(int64_t) * (size_t)(G + 1), cudaMemcpyHostToDevice, s));
    KB_CUDA(ctx, cudaMemcpyAsync(kd, k_h, sizeof(int32_t) * (size_t)G, cudaMemcpyHostToDevice, s));
    KB_CUDA(ctx, cudaMemcpyAsync(gact, act_h.data(), (size_t)G, cudaMemcpyHostToDevice, s));
    KB_CUDA(ctx, cudaMemcpyAsync(early, early_h.data(), (size_t)G, cudaMemcpyHostToDevice, s));
    KB_CUDA(ctx, cudaMemsetAsync(glast, 0, sizeof(int32_t) * (size_t)G, s));
    KB_CUDA(ctx, cudaMemsetAsync(sticky, 0, sizeof(int32_t), s));
    kb::launch_vertex_graph(voff, (int32_t)G, n, vgraph, s);
    p.vgraph = vgraph;
    p.voff = voff;
    p.n_graphs = (int32_t)G;

    // level 0 for every graph: key (graph, label) or (graph) without labels
    p.gactive = nullptr;
    p.gbase_cur = bases;
    KB_TRY(launch_level0(ctx, R, opt->use_vertex_labels ? g->vertex_labels : nullptr, levels, s));
    KB_TRY(read_counters(ctx));
    KB_TRY(device_error(ctx));

    // rounds 1..kmax, captured once
    p.gactive = gact;
    if (kmax > 0) {
        if (!ctx->cap_stream) KB_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
        cudaStream_t cs = ctx->cap_stream;
        KB_CUDA(ctx, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        kb_status st = KB_OK;
        for (int i = 1; i <= kmax && st == KB_OK; ++i) {
            st = next_epoch(ctx, R, cs);
            if (st != KB_OK) break;
            p.ehigh = 0xffffffffu - (uint32_t)i;
            p.prev = levels + (size_t)(i - 1) * (size_t)n;
            p.bitmap = (i & 1) ? bm_b : bm_a;
            p.bitmap_prev = (i & 1) ? bm_a : bm_b;
            p.gbase_prev = bases + (size_t)(i - 1) * (size_t)(G + 1);
            p.gbase_cur = bases + (size_t)i * (size_t)(G + 1);
            // frozen blocks as in a single-graph call (blocks never span
            // graphs); the medium and hub kernels always launch (no host
            // reads inside the captured rounds)
            p.frozen = R.frozen;
            p.frozen_min = R.frozen_min;
            p.moved = R.moved;
            // from round 2 on, windows packed from the vertices that refine
            // (frozen blocks and stopped graphs take no lane)
            R.compact = i >= 2;
            int32_t* out = levels + (size_t)i * (size_t)n;
            st = launch_round_body(ctx, R, cs, nullptr);
            if (st != KB_OK) break;
            kb::launch_carry_minima(p, cs);
            kb::launch_renumber(p, R.prefix, R.scan_tmp, out, cs);
            if (p.shared) {
                if (cudaMemsetAsync(R.mark, 0, sizeof(uint32_t) * (size_t)nw, cs) != cudaSuccess) {
                    st = fail(ctx, KB_ERR_CUDA, "memset failed");
                    break;
                }
                kb::launch_dirty_blocks(p, R.edgeless, R.moved, out, kb::kMaxHubThreshold, R.mark, cs);
                kb::launch_freeze_clean(n, p.bitmap, p.shared, R.edgeless, out, R.mark, R.frozen, R.frozen_min,
                                        ctx->d_ctr, cs);
            }
            kb::launch_graph_stop(p, i, kd, early, gact, glast, sticky, cs);
        }
        cudaGraph_t graph = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(cs, &graph);
        if (st != KB_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (ce != cudaSuccess) return fail(ctx, KB_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(ce));
        cudaGraphExec_t exec = nullptr;
        const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) return fail(ctx, KB_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(ie));
        cudaEvent_t e0 = ctx->ev[20], e1 = ctx->ev[21];
        cudaEventRecord(e0, s);
        const cudaError_t le = cudaGraphLaunch(exec, s);
        cudaEventRecord(e1, s);
        if (le != cudaSuccess) {
            cudaGraphExecDestroy(exec);
            return fail(ctx, KB_ERR_CUDA, "graph launch failed: %s", cudaGetErrorString(le));
        }
        const cudaError_t se = cudaStreamSynchronize(s);
        cudaGraphExecDestroy(exec);
        if (se != cudaSuccess) return fail(ctx, KB_ERR_CUDA, "batched rounds failed: %s", cudaGetErrorString(se));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ctx->round_ms.push_back(ms);
    }
    p.bitmap = bm_a;

    // results: graph-local ids, per-graph counts, last refined level
    std::vector<uint32_t> bases_h((size_t)(G + 1) * (size_t)(kmax + 1));
    int32_t sticky_h = 0;
    KB_CUDA(ctx, cudaMemcpyAsync(bases_h.data(), bases, sizeof(uint32_t) * bases_h.size(), cudaMemcpyDeviceToHost, s));
    KB_CUDA(ctx, cudaMemcpyAsync(&sticky_h, sticky, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    if (lc_out) KB_CUDA(ctx, cudaMemcpyAsync(lc_out, glast, sizeof(int32_t) * (size_t)G, cudaMemcpyDeviceToHost, s));
    for (int i = 0; i <= kmax; ++i)
        kb::launch_localize(levels + (size_t)i * (size_t)n, n, vgraph, bases + (size_t)i * (size_t)(G + 1), s);
    KB_CUDA(ctx, cudaGetLastError());
    KB_CUDA(ctx, cudaStreamSynchronize(s));
    if (sticky_h & kb::kErrTableFull) return fail(ctx, KB_ERR_TABLE_FULL, "block table probe limit reached");
    if (sticky_h) return fail(ctx, KB_ERR_DEVICE_CHECK, "device consistency check failed (%d)", sticky_h);
    for (int64_t j = 0; j < G; ++j)
        for (int i = 0; i <= kmax; ++i) {
            const uint32_t* bi = bases_h.data() + (size_t)i * (size_t)(G + 1);
            counts[j * (kmax + 1) + i] = (int64_t)(bi[j + 1] - bi[j]);
        }
    return KB_OK;
}


// ============================================================================
// Serving: continuous batching over a device arena (see kb_server_* in
// kbisim.h).  Every admitted request owns one graph slot of the arena, in
// arena order; retired slots stay as dead ranges until a compaction packs the
// live ones into the other arena buffer.
// ============================================================================
struct Arena {
    int64_t* row = nullptr;   // [Ncap+1]
    int32_t* col = nullptr;   // [Mcap]
    int32_t* lab = nullptr;   // [Mcap]
    int32_t* vlab = nullptr;  // [Ncap]
    int32_t* B[2] = {nullptr, nullptr};  // [Ncap] current / next level, union-global ids
};

struct ServeRequest {
    int64_t ticket = 0;
    int state = 0;  // 0 waiting, 1 running, 2 done, 3 failed (rejected at admission)
    int64_t n = 0, m = 0, m_proc = 0;
    // the caller's host arrays, read at admission (lab / vlab null when unused)
    const int64_t* row = nullptr;
    const int32_t* col = nullptr;
    const int32_t* lab = nullptr;
    const int32_t* vlab = nullptr;
    kb_options opt;
    int k = 0;
    int slot = -1;
    int round = 0;  // next level to compute (0 = level 0)
    int32_t* d_levels = nullptr;
    size_t level_bytes = 0;
    int32_t* out = nullptr;               // caller's host levels, or null: kept in `levels`
    std::unique_ptr<int32_t[]> levels;    // host copy after completion (when out is null)
    std::vector<int64_t> counts;
    int32_t levels_computed = 0;
    double t_submit = 0, t_done = 0;
    std::string error;
};

struct Slot {
    int64_t ticket = -1;  // -1: dead
    int64_t vbase = 0, n = 0, ebase = 0, m = 0;
};

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

struct kb_server {
    kb_context* ctx = nullptr;
    kb_server_config cfg{};
    std::string last_error;
    std::mutex mu;  // guards queue, requests, stats (submit vs step)
    Arena arena[2];
    int cur = 0;  // active arena buffer
    int bsel = 0;  // which B buffer of the arena holds the current level
    int64_t n_used = 0, m_used = 0;
    std::vector<Slot> slots;
    std::deque<int64_t> waiting;
    std::map<int64_t, ServeRequest> reqs;
    int64_t next_ticket = 1;
    size_t level_bytes_in_use = 0;
    // level stores are reused: freed ones wait in a list per power-of-two size
    std::map<size_t, std::vector<int32_t*>> level_pool;
    // block table and empty-signature minima of the arena, kept across re-plans
    uint64_t* table = nullptr;
    uint64_t table_cap = 0;
    uint64_t* emin = nullptr;
    uint64_t round_counter = 0;  // rounds run; decreasing round words of the minima
    // Frozen-block state of the arena, sized for a full arena and kept across
    // re-plans: frozen vertices, minima of frozen blocks, shared marks,
    // smallest members, moved vertices, dirty blocks, and the two bitmaps of
    // block minima used in turn.
    uint32_t* frz[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    uint32_t* minof = nullptr;
    uint32_t* bitmap1 = nullptr;
    int64_t planned_n = 0;        // arena vertices at the last re-plan
    bool vertices_moved = false;  // a compaction since the last re-plan
    // The last step's minima and smallest members are valid for this step's
    // moved vertices (false after a compaction, which moves vertices and
    // clears the frozen blocks)
    bool history = false;
    // per-slot device arrays (capacity max_requests + dead slots: sized by max_slots)
    int32_t max_slots = 0;
    int32_t* vgraph = nullptr;
    int64_t* voff = nullptr;
    uint8_t* gactive = nullptr;
    uint8_t* gmode = nullptr;
    uint32_t* bases[2] = {nullptr, nullptr};
    uint32_t* bitmap2 = nullptr;
    int32_t** slot_levels = nullptr;
    int32_t* slot_row = nullptr;
    int64_t* slot_n = nullptr;
    std::vector<uint32_t> gbase_host;
    // staging for admission (raw graph, processed CSR for IN / BOTH)
    void* stage = nullptr;
    size_t stage_bytes = 0;
    // round state
    Prepared R;
    bool dirty = true;

    int bmsel = 0;
    uint32_t* bm_ws = nullptr;
    // stats
    double t_first = -1;
    int64_t submitted = 0, completed = 0, failed = 0, steps = 0, compactions = 0;
    double edge_rounds = 0;
    std::vector<double> latencies_ms;
};

namespace {

kb_status sfail(kb_server* sv, kb_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    sv->last_error = buf;
    return st;
}

#define SV_CUDA(sv, call)                                                                            \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess) return sfail((sv), KB_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

#define SV_TRY(sv, expr)                                                     \
    do {                                                                     \
        kb_status s_ = (expr);                                               \
        if (s_ != KB_OK) {                                                   \
            if ((sv)->last_error.empty()) (sv)->last_error = (sv)->ctx->last_error; \
            return s_;                                                       \
        }                                                                    \
    } while (0)

// Copy request r's graph into the arena at the tail as slot `slot`.
kb_status place_request(kb_server* sv, ServeRequest& r, int slot, bool* rejected) {
    *rejected = false;
    kb_context* ctx = sv->ctx;
    cudaStream_t s = ctx->stream;
    Arena& A = sv->arena[sv->cur];
    const int64_t n = r.n, m = r.m, mp = r.m_proc;
    // staging: raw CSR (+ processed CSR for IN / BOTH)
    size_t off = 0;
    auto take = [&](size_t b) { size_t o = off; off += align_up(b); return o; };
    const size_t o_row = take(sizeof(int64_t) * (size_t)(n + 1));
    const size_t o_col = take(sizeof(int32_t) * (size_t)m);
    const size_t o_lab = take(sizeof(int32_t) * (size_t)m);
    const size_t o_vlab = take(sizeof(int32_t) * (size_t)n);
    Plan P;
    P.n = n;
    P.m = m;
    P.dir = r.opt.direction;
    P.m_proc = mp;
    P.labels = r.lab != nullptr;
    layout_csr(P);
    const size_t o_csr = take(P.csr_bytes);
    if (off > sv->stage_bytes) {
        if (sv->stage) cudaFree(sv->stage);
        sv->stage = nullptr;
        sv->stage_bytes = 0;
        if (cudaMalloc(&sv->stage, off) != cudaSuccess) {
            cudaGetLastError();
            return sfail(sv, KB_ERR_OOM, "cannot allocate %zu bytes of staging", off);
        }
        sv->stage_bytes = off;
    }
    char* b = reinterpret_cast<char*>(sv->stage);
    SV_CUDA(sv, cudaMemcpyAsync(b + o_row, r.row, sizeof(int64_t) * (size_t)(n + 1), cudaMemcpyHostToDevice, s));
    if (m) SV_CUDA(sv, cudaMemcpyAsync(b + o_col, r.col, sizeof(int32_t) * (size_t)m, cudaMemcpyHostToDevice, s));
    if (m && P.labels)
        SV_CUDA(sv, cudaMemcpyAsync(b + o_lab, r.lab, sizeof(int32_t) * (size_t)m, cudaMemcpyHostToDevice, s));
    if (r.vlab) SV_CUDA(sv, cudaMemcpyAsync(b + o_vlab, r.vlab, sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, s));
    // the arena is shared: a malformed CSR is checked on the device before it
    // is placed, and the request fails alone
    SV_CUDA(sv, cudaMemsetAsync(ctx->d_ctr, 0, sizeof(Counters), s));
    kb::launch_validate(n, m, reinterpret_cast<const int64_t*>(b + o_row), reinterpret_cast<const int32_t*>(b + o_col),
                        ctx->d_ctr, s);
    SV_CUDA(sv, cudaGetLastError());
    SV_CUDA(sv, cudaMemcpyAsync(ctx->h_ctr, ctx->d_ctr, sizeof(Counters), cudaMemcpyDeviceToHost, s));
    SV_CUDA(sv, cudaStreamSynchronize(s));
    if (ctx->h_ctr->err & kb::kErrInvalid) {
        *rejected = true;
        r.error = "row_offsets not monotone from 0 to m, or a neighbour id out of [0, n)";
        return KB_OK;
    }
    kb::PlaceArgs a{};
    a.srow = reinterpret_cast<const int64_t*>(b + o_row);
    a.scol = reinterpret_cast<const int32_t*>(b + o_col);
    a.slab = P.labels ? reinterpret_cast<const int32_t*>(b + o_lab) : nullptr;
    if (needs_in_csr(P.dir)) {
        kb_graph g{n, m, a.srow, a.scol, a.slab, nullptr};
        char* csr = b + o_csr;
        SV_TRY(sv, build_processed_csr(ctx, &g, P, csr));
        a.srow = reinterpret_cast<const int64_t*>(csr + P.o_rowp);
        a.scol = reinterpret_cast<const int32_t*>(csr + P.o_colp);
        a.slab = P.labels ? reinterpret_cast<const int32_t*>(csr + P.o_labp) : nullptr;
    }
    a.svlab = r.vlab ? reinterpret_cast<const int32_t*>(b + o_vlab) : nullptr;
    a.drow = A.row;
    a.dcol = A.col;
    a.dlab = A.lab;
    a.dvlab = A.vlab;
    a.n = n;
    a.m = mp;
    a.src_vbase = 0;
    a.src_ebase = 0;
    a.dst_vbase = sv->n_used;
    a.dst_ebase = sv->m_used;
    kb::launch_place(a, s);
    SV_CUDA(sv, cudaGetLastError());
    Slot sl;
    sl.ticket = r.ticket;
    sl.vbase = sv->n_used;
    sl.n = n;
    sl.ebase = sv->m_used;
    sl.m = mp;
    if ((int)sv->slots.size() != slot) return sfail(sv, KB_ERR_DEVICE_CHECK, "slot order broken");
    sv->slots.push_back(sl);
    sv->n_used += n;
    sv->m_used += mp;
    r.slot = slot;
    return KB_OK;
}

// Pack the live slots into the other arena buffer.
kb_status compact(kb_server* sv) {
    kb_context* ctx = sv->ctx;
    cudaStream_t s = ctx->stream;
    Arena& S = sv->arena[sv->cur];
    Arena& D = sv->arena[1 - sv->cur];
    std::vector<Slot> live;
    int64_t nv = 0, ne = 0;
    SV_CUDA(sv, cudaMemsetAsync(D.row, 0, sizeof(int64_t), s));
    for (size_t j = 0; j < sv->slots.size(); ++j) {
        const Slot& o = sv->slots[j];
        if (o.ticket < 0) continue;
        kb::PlaceArgs a{};
        a.srow = S.row;
        a.scol = S.col;
        a.slab = S.lab;
        a.svlab = S.vlab;
        a.sB = S.B[sv->bsel];
        a.drow = D.row;
        a.dcol = D.col;
        a.dlab = D.lab;
        a.dvlab = D.vlab;
        a.dB = D.B[0];
        a.n = o.n;
        a.m = o.m;
        a.src_vbase = o.vbase;
        a.src_ebase = o.ebase;
        a.dst_vbase = nv;
        a.dst_ebase = ne;
        a.b_sub = sv->gbase_host.size() > j ? sv->gbase_host[j] : 0u;
        a.b_add = (uint32_t)nv;
        kb::launch_place(a, s);
        Slot ns = o;
        ns.vbase = nv;
        ns.ebase = ne;
        sv->reqs[o.ticket].slot = (int)live.size();
        live.push_back(ns);
        nv += o.n;
        ne += o.m;
    }
    SV_CUDA(sv, cudaGetLastError());
    sv->slots = live;
    sv->n_used = nv;
    sv->m_used = ne;
    sv->cur = 1 - sv->cur;
    sv->bsel = 0;
    sv->gbase_host.clear();
    sv->dirty = true;
    sv->vertices_moved = true;
    ++sv->compactions;
    return KB_OK;
}

size_t free_device_bytes() {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return fr;
}

// Size class of a level store: the next power of two of at least 256 bytes.
size_t level_store_bytes(size_t bytes) {
    size_t b = 256;
    while (b < bytes) b <<= 1;
    return b;
}

// Admit waiting requests in arrival order while they fit.
kb_status admit(kb_server* sv, bool* changed) {
    std::vector<int64_t> admitted;
    while (true) {
        int64_t t;
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            if (sv->waiting.empty()) break;
            t = sv->waiting.front();
        }
        ServeRequest& r = sv->reqs[t];
        int live = 0;
        for (const Slot& sl : sv->slots) live += sl.ticket >= 0;
        if (live >= sv->cfg.max_requests) break;
        const size_t lb = level_store_bytes(sizeof(int32_t) * (size_t)r.n * (size_t)(r.k + 1));
        std::vector<int32_t*>& pooled = sv->level_pool[lb];
        const size_t budget = sv->cfg.memory_budget;
        if (budget) {
            if (sv->level_bytes_in_use + lb > budget) break;
        } else if (pooled.empty()) {
            const size_t fr = free_device_bytes();
            if (fr < lb + ((size_t)1 << 30)) break;
        }
        const bool fits_tail = sv->n_used + r.n <= sv->cfg.max_vertices && sv->m_used + r.m_proc <= sv->cfg.max_edges &&
                               (int)sv->slots.size() < sv->max_slots;
        if (!fits_tail) {
            int64_t ln = 0, lm = 0;
            for (const Slot& sl : sv->slots)
                if (sl.ticket >= 0) {
                    ln += sl.n;
                    lm += sl.m;
                }
            if (ln + r.n > sv->cfg.max_vertices || lm + r.m_proc > sv->cfg.max_edges) break;
            SV_TRY(sv, compact(sv));
        }
        if (!pooled.empty()) {
            r.d_levels = pooled.back();
            pooled.pop_back();
        } else if (cudaMalloc(&r.d_levels, lb) != cudaSuccess) {
            cudaGetLastError();
            r.d_levels = nullptr;
            break;
        }
        r.level_bytes = lb;
        sv->level_bytes_in_use += lb;
        bool rejected = false;
        SV_TRY(sv, place_request(sv, r, (int)sv->slots.size(), &rejected));
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->waiting.pop_front();
        if (rejected) {
            sv->level_pool[lb].push_back(r.d_levels);
            sv->level_bytes_in_use -= lb;
            r.d_levels = nullptr;
            r.state = 3;
            r.row = nullptr;
            ++sv->failed;
            continue;
        }
        r.state = 1;
        r.round = 0;
        r.counts.assign((size_t)r.k + 1, 0);
        r.row = nullptr;  // the caller's graph arrays are no longer read
        r.col = r.lab = r.vlab = nullptr;
        *changed = true;
    }
    return KB_OK;
}

// Finish request r after its last round, in two parts so that every request
// retiring in a step shares one synchronisation: retire_copy queues the copy
// of its levels to the host (the caller's buffer given at submission, else a
// buffer of its own; rows after the last refined level repeat it), and
// retire_finish, after the stream has drained, releases its level store.
kb_status retire_copy(kb_server* sv, ServeRequest& r, int last) {
    cudaStream_t s = sv->ctx->stream;
    const size_t n = (size_t)r.n;
    if (!r.out) {
        r.levels.reset(new (std::nothrow) int32_t[std::max<size_t>(n * (size_t)(r.k + 1), 1)]);
        if (!r.levels) return sfail(sv, KB_ERR_OOM, "cannot allocate host memory for the levels");
    }
    int32_t* dst = r.out ? r.out : r.levels.get();
    if (n) {
        SV_CUDA(sv, cudaMemcpyAsync(dst, r.d_levels, sizeof(int32_t) * n * (size_t)(last + 1), cudaMemcpyDeviceToHost, s));
        for (int j = last + 1; j <= r.k; ++j)
            SV_CUDA(sv, cudaMemcpyAsync(dst + (size_t)j * n, r.d_levels + (size_t)last * n, sizeof(int32_t) * n,
                                        cudaMemcpyDeviceToHost, s));
    }
    return KB_OK;
}

void retire_finish(kb_server* sv, ServeRequest& r, int last) {
    for (int j = last + 1; j <= r.k; ++j) r.counts[(size_t)j] = r.counts[(size_t)last];
    r.levels_computed = last;
    sv->level_pool[r.level_bytes].push_back(r.d_levels);
    r.d_levels = nullptr;
    sv->level_bytes_in_use -= r.level_bytes;
    sv->slots[(size_t)r.slot].ticket = -1;
    r.slot = -1;
    r.t_done = now_s();
    std::lock_guard<std::mutex> lk(sv->mu);
    r.state = 2;
    ++sv->completed;
    sv->latencies_ms.push_back(1000.0 * (r.t_done - r.t_submit));
    sv->edge_rounds += (double)r.m_proc * (double)last;
}

kb_status server_step(kb_server* sv, int32_t* running, int32_t* waiting_out) {
    kb_context* ctx = sv->ctx;
    cudaStream_t s = ctx->stream;
    SV_CUDA(sv, cudaSetDevice(ctx->device));
    bool changed = false;
    SV_TRY(sv, admit(sv, &changed));
    if (changed) sv->dirty = true;
    int live = 0;
    int64_t live_n = 0;
    for (const Slot& sl : sv->slots)
        if (sl.ticket >= 0) {
            ++live;
            live_n += sl.n;
        }
    // every round's kernels span the whole arena, retired ranges included:
    // pack the live requests once the dead ones dominate (cheap under light
    // load, when little is live)
    if (live > 0 && sv->n_used - live_n > 4 * live_n + ((int64_t)1 << 22)) SV_TRY(sv, compact(sv));
    if (live > 0) {
        const int G = (int)sv->slots.size();
        Arena& A = sv->arena[sv->cur];
        kb::RoundParams& p = sv->R.p;
        if (sv->dirty) {
            // re-plan the arena: medium / hub lists, block table, minima
            kb_graph view{sv->n_used, sv->m_used, A.row, A.col, A.lab, nullptr};
            kb_options o = kb_options_default();
            o.validate = 0;
            o.load_factor = sv->cfg.load_factor;
            o.hub_threshold = sv->cfg.hub_threshold;
            o.hash_mode = sv->cfg.hash_mode;
            sv->R.ext_table = sv->table;
            sv->R.ext_cap = sv->table_cap;
            sv->R.ext_emin = sv->emin;
            sv->R.ext_frozen = sv->frz[0];
            sv->R.ext_frozen_min = sv->frz[1];
            sv->R.ext_shared = sv->frz[2];
            sv->R.ext_moved = sv->frz[3];
            sv->R.ext_mark = sv->frz[4];
            sv->R.ext_minof = sv->minof;
            const size_t bw = sizeof(uint32_t) * (size_t)((sv->n_used >> 5) + 1);
            if (sv->vertices_moved) {
                // compacted: vertex ids moved, nothing carries over
                for (int f = 0; f < 3; ++f) SV_CUDA(sv, cudaMemsetAsync(sv->frz[f], 0, bw, s));
                sv->history = false;
                sv->vertices_moved = false;
            } else {
                // admitted at the tail: the new vertices start unfrozen, the
                // others keep their blocks' state; the bits past the last
                // vertex are cleared too (rank scans count whole words)
                const int64_t word_end = ((sv->n_used >> 5) + 1) * 32;
                for (int f = 0; f < 3; ++f) kb::launch_clear_bits(sv->frz[f], sv->planned_n, word_end, s);
            }
            SV_TRY(sv, prepare(ctx, &view, &o, sv->R, -1, true));
            sv->bm_ws = sv->bitmap1;
            sv->planned_n = sv->n_used;
            std::vector<int64_t> voff((size_t)G + 1);
            for (int j = 0; j < G; ++j) voff[(size_t)j] = sv->slots[(size_t)j].vbase;
            voff[(size_t)G] = sv->n_used;
            SV_CUDA(sv, cudaMemcpyAsync(sv->voff, voff.data(), sizeof(int64_t) * (size_t)(G + 1), cudaMemcpyHostToDevice, s));
            kb::launch_vertex_graph(sv->voff, G, sv->n_used, sv->vgraph, s);
            sv->dirty = false;
        }
        // per-slot flags for this step
        std::vector<uint8_t> act((size_t)G), mode((size_t)G);
        std::vector<int32_t*> lev((size_t)G, nullptr);
        std::vector<int32_t> row((size_t)G, -1);
        std::vector<int64_t> sn((size_t)G, 0);
        for (int j = 0; j < G; ++j) {
            const Slot& sl = sv->slots[(size_t)j];
            sn[(size_t)j] = sl.n;
            if (sl.ticket < 0) continue;
            ServeRequest& r = sv->reqs[sl.ticket];
            act[(size_t)j] = 1;
            mode[(size_t)j] = r.round == 0 ? 1 : 0;
            lev[(size_t)j] = r.d_levels;
            row[(size_t)j] = r.round;
        }
        SV_CUDA(sv, cudaMemcpyAsync(sv->gactive, act.data(), (size_t)G, cudaMemcpyHostToDevice, s));
        SV_CUDA(sv, cudaMemcpyAsync(sv->gmode, mode.data(), (size_t)G, cudaMemcpyHostToDevice, s));
        SV_CUDA(sv, cudaMemcpyAsync(sv->slot_levels, lev.data(), sizeof(int32_t*) * (size_t)G, cudaMemcpyHostToDevice, s));
        SV_CUDA(sv, cudaMemcpyAsync(sv->slot_row, row.data(), sizeof(int32_t) * (size_t)G, cudaMemcpyHostToDevice, s));
        SV_CUDA(sv, cudaMemcpyAsync(sv->slot_n, sn.data(), sizeof(int64_t) * (size_t)G, cudaMemcpyHostToDevice, s));
        // one round for everything in flight
        SV_TRY(sv, next_epoch(ctx, sv->R, s));
        p.ehigh = 0xffffffffu - (uint32_t)(++sv->round_counter);
        p.vgraph = sv->vgraph;
        p.voff = sv->voff;
        p.n_graphs = G;
        p.gactive = sv->gactive;
        p.gmode = sv->gmode;
        p.vlab = A.vlab;
        p.prev = A.B[sv->bsel];
        // block-minima bitmaps alternate between the prepared one and the server's own
        p.bitmap = sv->bmsel ? sv->bitmap2 : sv->bm_ws;
        p.bitmap_prev = sv->bmsel ? sv->bm_ws : sv->bitmap2;
        p.gbase_prev = sv->bases[1 - (sv->steps & 1)];
        p.gbase_cur = sv->bases[sv->steps & 1];
        int32_t* out = A.B[1 - sv->bsel];
        // frozen blocks, as in a single-graph call (blocks never span graphs)
        p.frozen = sv->R.frozen;
        p.frozen_min = sv->R.frozen_min;
        p.moved = sv->history ? sv->R.moved : nullptr;
        SV_TRY(sv, launch_round_body(ctx, sv->R, s, nullptr));
        kb::launch_carry_minima(p, s);
        kb::launch_renumber(p, sv->R.prefix, sv->R.scan_tmp, out, s);
        kb::launch_emit(sv->n_used, sv->vgraph, out, p.gbase_cur, sv->slot_levels, sv->slot_row, sv->slot_n, sv->voff, s);
        if (p.shared) {
            const uint32_t* mark = nullptr;
            if (p.moved) {
                SV_CUDA(sv, cudaMemsetAsync(sv->R.mark, 0, sizeof(uint32_t) * (size_t)((sv->n_used >> 5) + 1), s));
                kb::launch_dirty_blocks(p, sv->R.edgeless, sv->R.moved, out, kb::kMaxHubThreshold, sv->R.mark, s);
                mark = sv->R.mark;
            }
            kb::launch_freeze_clean(sv->n_used, p.bitmap, p.shared, sv->R.edgeless, out, mark, sv->R.frozen,
                                    sv->R.frozen_min, ctx->d_ctr, s, sv->vgraph, sv->gmode);
        }
        sv->history = true;
        SV_CUDA(sv, cudaGetLastError());
        sv->gbase_host.assign((size_t)G + 1, 0);
        SV_CUDA(sv, cudaMemcpyAsync(sv->gbase_host.data(), p.gbase_cur, sizeof(uint32_t) * (size_t)(G + 1),
                                    cudaMemcpyDeviceToHost, s));
        SV_CUDA(sv, cudaMemcpyAsync(ctx->h_ctr, ctx->d_ctr, sizeof(Counters), cudaMemcpyDeviceToHost, s));
        SV_CUDA(sv, cudaStreamSynchronize(s));
        if (ctx->h_ctr->err) {
            SV_TRY(sv, device_error(ctx));
        }
        sv->bsel = 1 - sv->bsel;
        sv->bmsel = 1 - sv->bmsel;
        // bookkeeping and retirement (one synchronisation for all copies)
        std::vector<std::pair<ServeRequest*, int>> finished;
        for (int j = 0; j < G; ++j) {
            const Slot sl = sv->slots[(size_t)j];
            if (sl.ticket < 0) continue;
            ServeRequest& r = sv->reqs[sl.ticket];
            const int64_t cnt = (int64_t)(sv->gbase_host[(size_t)j + 1] - sv->gbase_host[(size_t)j]);
            r.counts[(size_t)r.round] = cnt;
            const int done_round = r.round;
            bool done = done_round >= r.k;
            if (done_round > 0 && r.opt.early_stop && cnt == r.counts[(size_t)done_round - 1]) done = true;
            ++r.round;
            if (done) {
                SV_TRY(sv, retire_copy(sv, r, done_round));
                finished.push_back({&r, done_round});
            }
        }
        if (!finished.empty()) {
            SV_CUDA(sv, cudaStreamSynchronize(s));
            for (auto& f : finished) retire_finish(sv, *f.first, f.second);
        }
        ++sv->steps;
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    int run = 0;
    for (const Slot& sl : sv->slots) run += sl.ticket >= 0;
    if (running) *running = run;
    if (waiting_out) *waiting_out = (int32_t)sv->waiting.size();
    return KB_OK;
}
}  // namespace

extern "C" {

kb_options kb_options_default(void) {
    kb_options o;
    std::memset(&o, 0, sizeof(o));
    o.direction = KB_DIR_OUT;
    o.use_vertex_labels = 1;
    o.use_edge_labels = 1;
    o.early_stop = 1;
    o.validate = 1;
    return o;
}

kb_options kb_options_schaetzle(void) {
    kb_options o = kb_options_default();
    o.direction = KB_DIR_OUT;
    o.use_vertex_labels = 0;
    o.use_edge_labels = 1;
    return o;
}

kb_options kb_options_kaushik(void) {
    kb_options o = kb_options_default();
    o.direction = KB_DIR_IN;
    o.use_vertex_labels = 1;
    o.use_edge_labels = 0;
    return o;
}

const char* kb_status_string(kb_status st) {
    switch (st) {
        case KB_OK: return "ok";
        case KB_ERR_INVALID_ARG: return "invalid argument";
        case KB_ERR_OOM: return "out of device memory";
        case KB_ERR_TABLE_FULL: return "block table full";
        case KB_ERR_TIMEOUT: return "device wait timed out";
        case KB_ERR_CUDA: return "CUDA error";
        case KB_ERR_DEVICE_CHECK: return "device consistency check failed";
        case KB_ERR_NOT_FOUND: return "not found";
    }
    return "unknown status";
}

kb_status kb_create(kb_context** out, int device, void* stream) {
    if (!out) return KB_ERR_INVALID_ARG;
    *out = nullptr;
    kb_context* ctx = new (std::nothrow) kb_context();
    if (!ctx) return KB_ERR_OOM;
    ctx->device = device;
    ctx->stream = reinterpret_cast<cudaStream_t>(stream);
    if (cudaSetDevice(device) != cudaSuccess || cudaMalloc(&ctx->d_ctr, sizeof(Counters)) != cudaSuccess ||
        cudaMalloc(&ctx->d_hub_n, sizeof(int32_t)) != cudaSuccess ||
        cudaMalloc(&ctx->d_med_n, sizeof(int64_t)) != cudaSuccess ||
        cudaMallocHost(&ctx->h_med_n, sizeof(int64_t)) != cudaSuccess ||
        cudaMallocHost(&ctx->h_ctr, sizeof(Counters)) != cudaSuccess ||
        cudaMallocHost(&ctx->h_hub_n, sizeof(int32_t)) != cudaSuccess) {
        cudaGetLastError();
        kb_destroy(ctx);
        return KB_ERR_CUDA;
    }
    for (auto& e : ctx->ev) cudaEventCreate(&e);
    kb::set_medium_kernel_attributes();
    cudaGetLastError();
    *out = ctx;
    return KB_OK;
}

kb_status kb_destroy(kb_context* ctx) {
    if (!ctx) return KB_OK;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream); else cudaDeviceSynchronize();
    cudaFree(ctx->d_ctr);
    cudaFree(ctx->d_hub_n);
    cudaFree(ctx->d_med_n);
    cudaFreeHost(ctx->h_med_n);
    cudaFreeHost(ctx->h_ctr);
    cudaFreeHost(ctx->h_hub_n);
    cudaFree(ctx->own_ws);
    cudaFree(ctx->hub_tmp);
    cudaFree(ctx->plan_tmp);
    cudaFree(ctx->stage);
    cudaFree(ctx->batch_ws);
    cudaFree(ctx->tune_buf);
    cudaFree(ctx->fix_buf);
    cudaFree(ctx->sum_buf);
    cudaFree(ctx->upd_buf);
    cudaFree(ctx->d_work);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
    if (ctx->row_ev) cudaEventDestroy(ctx->row_ev);

    for (auto& e : ctx->ev)
        if (e) cudaEventDestroy(e);
    delete ctx;
    return KB_OK;
}

const char* kb_last_error(const kb_context* ctx) { return ctx ? ctx->last_error.c_str() : "no context"; }

kb_status kb_workspace_size(kb_context* ctx, const kb_graph* g, const kb_options* opt, int k, size_t* bytes) {
    if (!ctx || !bytes) return KB_ERR_INVALID_ARG;
    KB_TRY(check_graph(ctx, g, opt, k));
    KB_CUDA(ctx, cudaSetDevice(ctx->device));
    if (g->n == 0) {
        *bytes = 0;
        return KB_OK;
    }
    Plan P;
    char* unused = nullptr;
    KB_TRY(make_plan(ctx, g, opt, P, &unused, true, k));
    *bytes = P.total;
    return KB_OK;
}

kb_status kb_set_workspace(kb_context* ctx, void* ptr, size_t bytes) {
    if (!ctx) return KB_ERR_INVALID_ARG;
    ctx->user_ws = ptr;
    ctx->user_ws_bytes = ptr ? bytes : 0;
    return KB_OK;
}

kb_status kb_refine(kb_context* ctx, const kb_graph* g, const kb_options* opt, int k, int32_t* levels,
                    int64_t* counts, int* levels_computed) {
    if (!ctx) return KB_ERR_INVALID_ARG;
    return refine_impl(ctx, g, opt, nullptr, 0, k, levels, counts, levels_computed);
}

kb_status kb_refine_from(kb_context* ctx, const kb_graph* g, const kb_options* opt, const int32_t* start,
                         int i_start, int k, int32_t* levels, int64_t* counts, int* levels_computed) {
    if (!ctx) return KB_ERR_INVALID_ARG;
    if (!start && g && g->n > 0) return fail(ctx, KB_ERR_INVALID_ARG, "start is NULL");
    return refine_impl(ctx, g, opt, start, i_start, k, levels, counts, levels_computed);
}

kb_status kb_graph_prepare(kb_context* ctx, const kb_graph* g, const kb_options* opt, kb_prepared** out) {
    if (!ctx) return KB_ERR_INVALID_ARG;
    if (!out) return fail(ctx, KB_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    KB_TRY(check_graph(ctx, g, opt, 0));
    KB_CUDA(ctx, cudaSetDevice(ctx->device));
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = ctx->stream;
    std::unique_ptr<kb_prepared> pg(new kb_prepared);
    pg->device = ctx->device;
    pg->g = *g;
    pg->dir = opt->direction;
    pg->edge_labels = opt->use_edge_labels ? 1 : 0;
    const int64_t n = g->n;
    KB_CUDA(ctx, cudaMemsetAsync(ctx->d_ctr, 0, sizeof(Counters), s));
    if (opt->validate && n > 0) {
        kb::launch_validate(n, g->m, g->row_offsets, g->col_indices, ctx->d_ctr, s);
        KB_CUDA(ctx, cudaGetLastError());
        KB_TRY(read_counters(ctx));
        KB_TRY(device_error(ctx));
    }
    Plan& P = pg->P;
    P.graph_ext = true;
    Plan probe;
    probe.n = n;
    probe.m = g->m;
    probe.dir = opt->direction;
    probe.m_proc = probe.dir == KB_DIR_BOTH ? 2 * g->m : g->m;
    probe.labels = opt->use_edge_labels && g->edge_labels != nullptr;
    layout_csr(probe);
    auto alloc = [&](char** ptr, size_t bytes) -> kb_status {
        if (cudaMalloc(reinterpret_cast<void**>(ptr), std::max<size_t>(bytes, 256)) != cudaSuccess) {
            cudaGetLastError();
            *ptr = nullptr;
            return fail(ctx, KB_ERR_OOM, "cannot allocate %zu bytes of device memory", bytes);
        }
        return KB_OK;
    };
    if (probe.csr_bytes) KB_TRY(alloc(&pg->csr, probe.csr_bytes));
    char* base = pg->csr;
    if (n > 0) KB_TRY(make_plan(ctx, g, opt, P, &base, false, 1, false));
    KB_TRY(alloc(&pg->gbuf, P.graph_bytes));
    if (n > 0) {
        char* count_tmp = nullptr;
        if (P.reorder) KB_TRY(alloc(&count_tmp, sizeof(uint32_t) * (size_t)n));
        kb::RoundParams p{};
        p.n = n;
        p.small_max = P.small_max;
        const kb_status st = bind_graph_part(ctx, g, P, pg->csr, pg->gbuf, true,
                                             reinterpret_cast<uint32_t*>(count_tmp), p, s);
        const cudaError_t e = cudaStreamSynchronize(s);
        cudaFree(count_tmp);
        KB_TRY(st);
        if (e != cudaSuccess) return fail(ctx, KB_ERR_CUDA, "prepare: %s", cudaGetErrorString(e));
        pg->n_med = p.n_med;
    }
    // the hub lists are on the device now
    std::vector<int32_t>().swap(P.hub_v);
    std::vector<int64_t>().swap(P.chunk_off);
    std::vector<int64_t>().swap(P.set_off);
    std::vector<int32_t>().swap(P.chunk_hub);
    pg->build_ms = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *out = pg.release();
    return KB_OK;
}

kb_status kb_graph_release(kb_prepared* pg) {
    delete pg;
    return KB_OK;
}

kb_status kb_prepared_get_info(const kb_prepared* pg, kb_prepared_info* info) {
    if (!pg || !info) return KB_ERR_INVALID_ARG;
    std::memset(info, 0, sizeof(*info));
    info->device_bytes = (pg->csr ? pg->P.csr_bytes : 0) + pg->P.graph_bytes;
    info->n_hubs = (int64_t)pg->P.n_hubs;
    info->n_hub_chunks = pg->P.n_chunks;
    info->n_medium = pg->n_med;
    info->reorder = pg->P.reorder ? 1 : 0;
    info->hub_threshold = pg->P.thr;
    info->small_max_degree = pg->P.small_max;
    info->hub_chunk_edges = pg->P.hub_chunk;
    info->build_ms = pg->build_ms;
    return KB_OK;
}

kb_status kb_refine_prepared(kb_context* ctx, const kb_prepared* pg, const kb_options* opt, int k, int32_t* levels,
                             int64_t* counts, int* levels_computed) {
    if (!ctx) return KB_ERR_INVALID_ARG;
    if (!pg || !opt) return fail(ctx, KB_ERR_INVALID_ARG, "prepared graph and options must not be NULL");
    if (pg->device != ctx->device)
        return fail(ctx, KB_ERR_INVALID_ARG, "the graph was prepared on device %d, the context is on %d", pg->device,
                    ctx->device);
    if (opt->direction != pg->dir || (opt->use_edge_labels ? 1 : 0) != pg->edge_labels)
        return fail(ctx, KB_ERR_INVALID_ARG, "direction and use_edge_labels must be those of kb_graph_prepare");
    return refine_impl(ctx, &pg->g, opt, nullptr, 0, k, levels, counts, levels_computed, pg);
}

kb_status kb_refine_update(kb_context* ctx, const kb_graph* g, const kb_options* opt, int k, const int32_t* changed,
                           int64_t n_changed, int32_t* levels, int64_t* counts, int* levels_computed, int64_t* work) {
    if (!ctx) return KB_ERR_INVALID_ARG;
    return update_impl(ctx, g, opt, k, changed, n_changed, levels, counts, levels_computed, work);
}

kb_status kb_summary(kb_context* ctx, const kb_graph* g, int direction, int use_edge_labels,
                     const int32_t* src_level, const int32_t* dst_level, int32_t* out_src, int32_t* out_label,
                     int32_t* out_dst, int64_t capacity, int64_t* count) {
    if (!ctx) return KB_ERR_INVALID_ARG;
    return summary_impl(ctx, g, direction, use_edge_labels, src_level, dst_level, out_src, out_label, out_dst,
                        capacity, count);
}

kb_status kb_refine_fixpoint(kb_context* ctx, const kb_graph* g, const kb_options* opt, const int32_t* initial,
                             int max_rounds, int32_t* final_level, int64_t* count, int* rounds, int* stable) {
    if (!ctx) return KB_ERR_INVALID_ARG;
    return fixpoint_impl(ctx, g, opt, initial, max_rounds, final_level, count, rounds, stable);
}

kb_status kb_refine_host(kb_context* ctx, const kb_graph* g, const kb_options* opt, int k, int32_t* levels,
                         int64_t* counts, int* levels_computed) {
    if (!ctx) return KB_ERR_INVALID_ARG;
    KB_TRY(check_graph(ctx, g, opt, k));
    if (!counts) return fail(ctx, KB_ERR_INVALID_ARG, "counts is NULL");
    if (g->n > 0 && !levels) return fail(ctx, KB_ERR_INVALID_ARG, "levels is NULL");
    KB_CUDA(ctx, cudaSetDevice(ctx->device));
    const int64_t n = g->n, m = g->m;
    const bool el = g->edge_labels && opt->use_edge_labels;
    const bool vl = g->vertex_labels && opt->use_vertex_labels;
    size_t off = 0;
    auto take = [&](size_t b) { size_t o = off; off += align_up(b); return o; };
    const size_t o_row = take(sizeof(int64_t) * (size_t)(n + 1));
    const size_t o_col = take(sizeof(int32_t) * (size_t)m);
    const size_t o_el = take(el ? sizeof(int32_t) * (size_t)m : 0);
    const size_t o_vl = take(vl ? sizeof(int32_t) * (size_t)n : 0);
    const size_t o_lv = take(sizeof(int32_t) * (size_t)n * (size_t)(k + 1));
    KB_TRY(ensure_buffer(ctx, &ctx->stage, &ctx->stage_bytes, std::max<size_t>(off, 256)));
    char* b = reinterpret_cast<char*>(ctx->stage);
    cudaStream_t s = ctx->stream;
    if (n > 0) {
        KB_CUDA(ctx, cudaMemcpyAsync(b + o_row, g->row_offsets, sizeof(int64_t) * (size_t)(n + 1),
                                     cudaMemcpyHostToDevice, s));
    }
    if (m > 0) KB_CUDA(ctx, cudaMemcpyAsync(b + o_col, g->col_indices, sizeof(int32_t) * (size_t)m, cudaMemcpyHostToDevice, s));
    if (el && m > 0) KB_CUDA(ctx, cudaMemcpyAsync(b + o_el, g->edge_labels, sizeof(int32_t) * (size_t)m, cudaMemcpyHostToDevice, s));
    if (vl && n > 0) KB_CUDA(ctx, cudaMemcpyAsync(b + o_vl, g->vertex_labels, sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, s));
    kb_graph dg = *g;
    dg.row_offsets = reinterpret_cast<const int64_t*>(b + o_row);
    dg.col_indices = reinterpret_cast<const int32_t*>(b + o_col);
    dg.edge_labels = el ? reinterpret_cast<const int32_t*>(b + o_el) : nullptr;
    dg.vertex_labels = vl ? reinterpret_cast<const int32_t*>(b + o_vl) : nullptr;
    int32_t* dlev = reinterpret_cast<int32_t*>(b + o_lv);
    // every level row goes back to the host as soon as it is final
    KB_TRY(refine_impl(ctx, &dg, opt, nullptr, 0, k, dlev, counts, levels_computed, nullptr, levels));
    KB_CUDA(ctx, cudaStreamSynchronize(s));
    return KB_OK;
}

kb_status kb_set_timing(kb_context* ctx, int enable) {
    if (!ctx) return KB_ERR_INVALID_ARG;
    if (enable < 0 || enable > 2) return fail(ctx, KB_ERR_INVALID_ARG, "timing mode must be 0, 1 or 2");
    ctx->timing = enable != 0;
    ctx->work = enable == 2;
    return KB_OK;
}

kb_status kb_get_timing(const kb_context* ctx, float* round_ms, int max_rounds, int* n_rounds, float* kernel_ms,
                        int64_t* kernel_launches) {
    if (!ctx) return KB_ERR_INVALID_ARG;
    const int nr = (int)ctx->round_ms.size();
    if (n_rounds) *n_rounds = nr;
    if (round_ms)
        for (int i = 0; i < nr && i < max_rounds; ++i) round_ms[i] = ctx->round_ms[(size_t)i];
    for (int f = 0; f < KB_KERNEL_COUNT; ++f) {
        if (kernel_ms) kernel_ms[f] = ctx->kernel_ms[f];
        if (kernel_launches) kernel_launches[f] = ctx->kernel_launches[f];
    }
    return KB_OK;
}

kb_status kb_get_round_work(const kb_context* ctx, int64_t* vertices, int64_t* edges, int max_rounds,
                            int* n_rounds) {
    if (!ctx) return KB_ERR_INVALID_ARG;
    const int nr = (int)ctx->round_keyed.size();
    if (n_rounds) *n_rounds = nr;
    for (int i = 0; i < nr && i < max_rounds; ++i)
        for (int f = 0; f < 3; ++f) {
            if (vertices) vertices[3 * i + f] = ctx->round_keyed[(size_t)i][(size_t)f];
            if (edges) edges[3 * i + f] = ctx->round_keyed[(size_t)i][(size_t)f + 3];
        }
    return KB_OK;
}

kb_status kb_refine_batch(kb_context* ctx, const kb_graph* union_graph, const int64_t* graph_vertex_offsets,
                          int64_t G, const int32_t* k_per_graph, const kb_options* opt, int32_t* levels,
                          int64_t* counts, int32_t* levels_computed) {
    if (!ctx) return KB_ERR_INVALID_ARG;
    return batch_impl(ctx, union_graph, graph_vertex_offsets, G, k_per_graph, opt, levels, counts, levels_computed);
}

kb_status kb_autotune(kb_context* ctx, const kb_graph* g, const int64_t* voff, int64_t G, const int32_t* k_per_graph,
                      const kb_options* opt, int rounds, kb_tuning* out) {
    if (!ctx) return KB_ERR_INVALID_ARG;
    if (!g || !opt) return fail(ctx, KB_ERR_INVALID_ARG, "graph and options must not be NULL");
    const bool batch = voff != nullptr;
    if (batch && (G < 1 || G > (int64_t)1 << 30)) return fail(ctx, KB_ERR_INVALID_ARG, "bad graph count");
    std::vector<int32_t> ks;
    int kmax = rounds;
    if (batch) {
        ks.assign((size_t)G, rounds);
        if (k_per_graph) {
            kmax = 0;
            for (int64_t j = 0; j < G; ++j) {
                ks[(size_t)j] = k_per_graph[j];
                kmax = std::max(kmax, (int)k_per_graph[j]);
            }
        }
    }
    if (kmax < 1) return fail(ctx, KB_ERR_INVALID_ARG, "the timed call must run at least one round");
    KB_TRY(check_graph(ctx, g, opt, kmax));
    KB_CUDA(ctx, cudaSetDevice(ctx->device));
    const int64_t n = g->n;
    KB_TRY(ensure_buffer(ctx, &ctx->tune_buf, &ctx->tune_buf_bytes,
                         std::max<size_t>(256, sizeof(int32_t) * (size_t)n * (size_t)(kmax + 1))));
    int32_t* lev = reinterpret_cast<int32_t*>(ctx->tune_buf);
    std::vector<int64_t> counts((size_t)(batch ? G : 1) * (size_t)(kmax + 1));
    const int64_t m_proc = opt->direction == KB_DIR_BOTH ? 2 * g->m : g->m;
    const int32_t cls = size_class(m_proc, batch ? G : 1, batch);

    // every tuning field explicit, so no cached tuning is consulted while timing
    kb_options base = *opt;
    base.early_stop = 0;
    base.validate = 0;
    kb_options dflt = base;
    dflt.load_factor = 0.5f;
    dflt.hub_threshold = kb::kDefaultHubThreshold;
    dflt.small_task_vertices = kb::kDefaultWarpVerts;
    dflt.hub_chunk_edges = kb::kDefaultHubChunk;
    dflt.medium_split = kb::kDefaultMedSplit;
    dflt.small_max_degree = kb::kSmallDegree;
    kb_options start = dflt;
    if (base.load_factor > 0.f) start.load_factor = base.load_factor;
    if (base.hub_threshold) start.hub_threshold = base.hub_threshold;
    if (base.small_task_vertices) start.small_task_vertices = base.small_task_vertices;
    if (base.hub_chunk_edges) start.hub_chunk_edges = base.hub_chunk_edges;
    if (base.medium_split) start.medium_split = base.medium_split;
    if (base.small_max_degree) start.small_max_degree = base.small_max_degree;

    // one warm-up run, then the best of two timed runs
    auto timed = [&](const kb_options& t, float* best_ms) -> kb_status {
        float best = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            cudaEvent_t e0 = ctx->ev[20], e1 = ctx->ev[21];
            KB_CUDA(ctx, cudaEventRecord(e0, ctx->stream));
            if (batch)
                KB_TRY(batch_impl(ctx, g, voff, G, ks.data(), &t, lev, counts.data(), nullptr));
            else
                KB_TRY(refine_impl(ctx, g, &t, nullptr, 0, rounds, lev, counts.data(), nullptr));
            KB_CUDA(ctx, cudaEventRecord(e1, ctx->stream));
            KB_CUDA(ctx, cudaEventSynchronize(e1));
            float ms = 0.f;
            KB_CUDA(ctx, cudaEventElapsedTime(&ms, e0, e1));
            if (rep > 0) best = std::min(best, ms);
        }
        *best_ms = best;
        return KB_OK;
    };
    float default_ms = 0.f;
    KB_TRY(timed(dflt, &default_ms));
    float best = default_ms;
    kb_options win = start;
    if (std::memcmp(&start, &dflt, sizeof(kb_options)) != 0) KB_TRY(timed(start, &best));

    // coordinate search, one field at a time
    const float lfs[] = {0.35f, 0.5f, 0.7f};
    const int32_t thrs[] = {256, 512, 1024};
    const int32_t smaxs[] = {16, 24, 32};
    const int32_t splits[] = {64, 128, 256};
    const int32_t wvs[] = {64, 128, 256, 512};
    const int32_t chunks[] = {256, 512, 1024};
    const int n_values[6] = {3, 3, 3, 3, 4, 3};
    for (int axis = 0; axis < 6; ++axis) {
        kb_options center = win;
        for (int c = 0; c < n_values[axis]; ++c) {
            kb_options t = center;
            switch (axis) {
                case 0: t.load_factor = lfs[c]; break;
                case 1: t.hub_threshold = thrs[c]; break;
                case 2: t.small_max_degree = smaxs[c]; break;
                case 3: t.medium_split = splits[c]; break;
                case 4: t.small_task_vertices = wvs[c]; break;
                default: t.hub_chunk_edges = chunks[c]; break;
            }
            if (std::memcmp(&t, &center, sizeof(kb_options)) == 0) continue;  // timed already
            float ms = 0.f;
            KB_TRY(timed(t, &ms));
            if (ms < 0.98f * best) {
                best = ms;
                win = t;
            }
        }
    }
    kb_tuning T;
    std::memset(&T, 0, sizeof(T));
    T.load_factor = win.load_factor;
    T.hub_threshold = win.hub_threshold;
    T.small_task_vertices = win.small_task_vertices;
    T.hub_chunk_edges = win.hub_chunk_edges;
    T.medium_split = win.medium_split;
    T.small_max_degree = win.small_max_degree;
    T.ms = best;
    T.default_ms = default_ms;
    T.size_class = cls;
    ctx->tuned[cls] = T;
    if (out) *out = T;
    return KB_OK;
}

kb_status kb_clear_tuning(kb_context* ctx) {
    if (!ctx) return KB_ERR_INVALID_ARG;
    ctx->tuned.clear();
    return KB_OK;
}


kb_server_config kb_server_config_default(void) {
    kb_server_config c;
    std::memset(&c, 0, sizeof(c));
    c.max_vertices = (int64_t)1 << 26;
    c.max_edges = (int64_t)1 << 28;
    c.max_requests = 256;
    return c;
}

kb_status kb_server_create(kb_server** out, int device, void* stream, const kb_server_config* cfg) {
    if (!out || !cfg) return KB_ERR_INVALID_ARG;
    *out = nullptr;
    if (cfg->max_vertices < 1 || cfg->max_vertices > 2147483646LL || cfg->max_edges < 0 || cfg->max_requests < 1)
        return KB_ERR_INVALID_ARG;
    if (cfg->load_factor < 0.f || cfg->load_factor > 0.9f) return KB_ERR_INVALID_ARG;
    if (cfg->hub_threshold < 0 || cfg->hub_threshold > kb::kMaxHubThreshold) return KB_ERR_INVALID_ARG;
    if (cfg->hash_mode < 0 || cfg->hash_mode > 1) return KB_ERR_INVALID_ARG;
    kb_server* sv = new (std::nothrow) kb_server();
    if (!sv) return KB_ERR_OOM;
    sv->cfg = *cfg;
    sv->max_slots = 4 * cfg->max_requests;
    kb_status st = kb_create(&sv->ctx, device, stream);
    if (st != KB_OK) {
        delete sv;
        return st;
    }
    const int64_t N = cfg->max_vertices, M = std::max<int64_t>(cfg->max_edges, 1), S = sv->max_slots;
    bool ok = true;
    auto alloc = [&](void** ptr, size_t bytes) {
        if (ok && cudaMalloc(ptr, std::max<size_t>(bytes, 16)) != cudaSuccess) {
            cudaGetLastError();
            ok = false;
        }
    };
    for (int a = 0; a < 2; ++a) {
        Arena& A = sv->arena[a];
        alloc((void**)&A.row, sizeof(int64_t) * (size_t)(N + 1));
        alloc((void**)&A.col, sizeof(int32_t) * (size_t)M);
        alloc((void**)&A.lab, sizeof(int32_t) * (size_t)M);
        alloc((void**)&A.vlab, sizeof(int32_t) * (size_t)N);
        alloc((void**)&A.B[0], sizeof(int32_t) * (size_t)N);
        alloc((void**)&A.B[1], sizeof(int32_t) * (size_t)N);
    }
    alloc((void**)&sv->vgraph, sizeof(int32_t) * (size_t)N);
    alloc((void**)&sv->voff, sizeof(int64_t) * (size_t)(S + 1));
    alloc((void**)&sv->gactive, (size_t)S);
    alloc((void**)&sv->gmode, (size_t)S);
    alloc((void**)&sv->bases[0], sizeof(uint32_t) * (size_t)(S + 1));
    alloc((void**)&sv->bases[1], sizeof(uint32_t) * (size_t)(S + 1));
    alloc((void**)&sv->bitmap2, sizeof(uint32_t) * (size_t)((N >> 5) + 1));
    alloc((void**)&sv->slot_levels, sizeof(int32_t*) * (size_t)S);
    alloc((void**)&sv->slot_row, sizeof(int32_t) * (size_t)S);
    alloc((void**)&sv->slot_n, sizeof(int64_t) * (size_t)S);
    // the arena's block table and empty-signature minima, sized for a full arena
    const float lf = cfg->load_factor > 0.f ? cfg->load_factor : 0.5f;
    sv->table_cap = table_capacity(N, lf);
    alloc((void**)&sv->table, sizeof(uint64_t) * (size_t)sv->table_cap);
    alloc((void**)&sv->emin, sizeof(uint64_t) * (size_t)N);
    const size_t bwN = sizeof(uint32_t) * (size_t)((N >> 5) + 1);
    for (int f = 0; f < 5; ++f) alloc((void**)&sv->frz[f], bwN);
    alloc((void**)&sv->minof, sizeof(uint32_t) * (size_t)N);
    alloc((void**)&sv->bitmap1, bwN);
    if (ok) {
        ok = cudaMemset(sv->arena[0].row, 0, sizeof(int64_t)) == cudaSuccess &&
             cudaMemset(sv->arena[1].row, 0, sizeof(int64_t)) == cudaSuccess &&
             cudaMemset(sv->bitmap2, 0, sizeof(uint32_t) * (size_t)((N >> 5) + 1)) == cudaSuccess &&
             cudaMemset(sv->table, 0, sizeof(uint64_t) * (size_t)sv->table_cap) == cudaSuccess &&
             cudaMemset(sv->emin, 0xff, sizeof(uint64_t) * (size_t)N) == cudaSuccess &&
             cudaMemset(sv->frz[0], 0, bwN) == cudaSuccess && cudaMemset(sv->frz[1], 0, bwN) == cudaSuccess &&
             cudaMemset(sv->frz[2], 0, bwN) == cudaSuccess && cudaMemset(sv->bitmap1, 0, bwN) == cudaSuccess;
    }
    if (!ok) {
        kb_server_destroy(sv);
        return KB_ERR_OOM;
    }
    *out = sv;
    return KB_OK;
}

kb_status kb_server_destroy(kb_server* sv) {
    if (!sv) return KB_OK;
    if (sv->ctx) {
        cudaSetDevice(sv->ctx->device);
        if (sv->ctx->stream) cudaStreamSynchronize(sv->ctx->stream); else cudaDeviceSynchronize();
    }
    for (auto& kv : sv->reqs)
        if (kv.second.d_levels) cudaFree(kv.second.d_levels);
    for (auto& kv : sv->level_pool)
        for (int32_t* b : kv.second) cudaFree(b);
    cudaFree(sv->table);
    cudaFree(sv->emin);
    for (int f = 0; f < 5; ++f) cudaFree(sv->frz[f]);
    cudaFree(sv->minof);
    cudaFree(sv->bitmap1);
    for (int a = 0; a < 2; ++a) {
        Arena& A = sv->arena[a];
        cudaFree(A.row);
        cudaFree(A.col);
        cudaFree(A.lab);
        cudaFree(A.vlab);
        cudaFree(A.B[0]);
        cudaFree(A.B[1]);
    }
    cudaFree(sv->vgraph);
    cudaFree(sv->voff);
    cudaFree(sv->gactive);
    cudaFree(sv->gmode);
    cudaFree(sv->bases[0]);
    cudaFree(sv->bases[1]);
    cudaFree(sv->bitmap2);
    cudaFree(sv->slot_levels);
    cudaFree(sv->slot_row);
    cudaFree(sv->slot_n);
    cudaFree(sv->stage);
    kb_destroy(sv->ctx);
    delete sv;
    return KB_OK;
}

const char* kb_server_last_error(const kb_server* sv) { return sv ? sv->last_error.c_str() : "no server"; }

kb_status kb_server_submit(kb_server* sv, const kb_graph* g, const kb_options* opt, int k, int32_t* levels_out,
                           int64_t* ticket) {
    static const int64_t kEmptyRow[1] = {0};
    if (!sv || !ticket) return KB_ERR_INVALID_ARG;
    if (!g || !opt) return sfail(sv, KB_ERR_INVALID_ARG, "graph and options must not be NULL");
    if (opt->subject != KB_SUBJECT_PREVIOUS)
        return sfail(sv, KB_ERR_INVALID_ARG, "served refinement takes subject = KB_SUBJECT_PREVIOUS only");
    if (g->n < 0 || g->m < 0 || k < 0 || opt->direction < 0 || opt->direction > 2)
        return sfail(sv, KB_ERR_INVALID_ARG, "bad request");
    if (g->n > 0 && !g->row_offsets) return sfail(sv, KB_ERR_INVALID_ARG, "row_offsets is NULL");
    if (g->m > 0 && !g->col_indices) return sfail(sv, KB_ERR_INVALID_ARG, "col_indices is NULL");
    if (g->n == 0 && g->m != 0) return sfail(sv, KB_ERR_INVALID_ARG, "edges without vertices");
    const int64_t mp = opt->direction == KB_DIR_BOTH ? 2 * g->m : g->m;
    if (g->n > sv->cfg.max_vertices || mp > sv->cfg.max_edges)
        return sfail(sv, KB_ERR_INVALID_ARG, "request larger than the arena");
    // the ends of the offsets here; every offset and neighbour id is checked
    // on the device at admission, before the graph reaches the shared arena
    if (g->n > 0 && (g->row_offsets[0] != 0 || g->row_offsets[g->n] != g->m))
        return sfail(sv, KB_ERR_INVALID_ARG, "row_offsets must run from 0 to m");
    ServeRequest r;
    r.n = g->n;
    r.m = g->m;
    r.m_proc = mp;
    r.opt = *opt;
    r.k = k;
    r.row = g->n > 0 ? g->row_offsets : kEmptyRow;
    r.col = g->col_indices;
    r.lab = (g->m && g->edge_labels && opt->use_edge_labels) ? g->edge_labels : nullptr;
    r.vlab = (g->n && g->vertex_labels && opt->use_vertex_labels) ? g->vertex_labels : nullptr;
    r.out = levels_out;
    r.t_submit = now_s();
    std::lock_guard<std::mutex> lk(sv->mu);
    r.ticket = sv->next_ticket++;
    *ticket = r.ticket;
    if (sv->t_first < 0) sv->t_first = r.t_submit;
    ++sv->submitted;
    const int64_t t = r.ticket;
    sv->reqs.emplace(t, std::move(r));
    sv->waiting.push_back(t);
    return KB_OK;
}

kb_status kb_server_step(kb_server* sv, int32_t* running, int32_t* waiting) {
    if (!sv) return KB_ERR_INVALID_ARG;
    sv->last_error.clear();
    return server_step(sv, running, waiting);
}

kb_status kb_server_poll(kb_server* sv, int64_t ticket, int32_t* state) {
    if (!sv || !state) return KB_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) return KB_ERR_NOT_FOUND;
    *state = it->second.state;
    return KB_OK;
}

kb_status kb_server_fetch(kb_server* sv, int64_t ticket, int32_t* levels, int64_t* counts, int32_t* levels_computed) {
    if (!sv) return KB_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) return KB_ERR_NOT_FOUND;
    ServeRequest& r = it->second;
    if (r.state == 3) {
        const std::string why = r.error;
        sv->reqs.erase(it);
        return sfail(sv, KB_ERR_INVALID_ARG, "request %lld was rejected at admission: %s", (long long)ticket,
                     why.c_str());
    }
    if (r.state != 2) return sfail(sv, KB_ERR_INVALID_ARG, "request %lld has not finished", (long long)ticket);
    if (levels && r.n) {
        const size_t bytes = sizeof(int32_t) * (size_t)r.n * (size_t)(r.k + 1);
        if (r.out) {
            if (levels != r.out) std::memcpy(levels, r.out, bytes);
        } else {
            std::memcpy(levels, r.levels.get(), bytes);
        }
    }
    if (counts) std::memcpy(counts, r.counts.data(), sizeof(int64_t) * r.counts.size());
    if (levels_computed) *levels_computed = r.levels_computed;
    sv->reqs.erase(it);
    return KB_OK;
}

kb_status kb_server_get_stats(kb_server* sv, kb_server_stats* st) {
    if (!sv || !st) return KB_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(sv->mu);
    std::memset(st, 0, sizeof(*st));
    st->submitted = sv->submitted;
    st->completed = sv->completed;
    st->failed = sv->failed;
    int run = 0;
    for (const Slot& sl : sv->slots) run += sl.ticket >= 0;
    st->running = run;
    st->waiting = (int64_t)sv->waiting.size();
    st->steps = sv->steps;
    st->compactions = sv->compactions;
    if (!sv->latencies_ms.empty()) {
        std::vector<double> l = sv->latencies_ms;
        std::sort(l.begin(), l.end());
        auto pct = [&](double q) {
            const size_t i = (size_t)std::min<double>((double)(l.size() - 1), std::ceil(q * (double)l.size()) - 1);
            return l[i];
        };
        st->p50_ms = pct(0.50);
        st->p99_ms = pct(0.99);
        double sum = 0;
        for (double x : l) sum += x;
        st->mean_ms = sum / (double)l.size();
    }
    const double span = sv->t_first >= 0 ? now_s() - sv->t_first : 0;
    if (span > 0) {
        st->requests_per_s = (double)sv->completed / span;
        st->edge_rounds_per_s = sv->edge_rounds / span;
    }
    return KB_OK;
}

}  // extern "C"
