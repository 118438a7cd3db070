// kb_refine_round_noalloc: one refinement round that allocates no device
// memory.  Its scratch (block table, slot per vertex, empty-signature minima,
// bitmap of block minima and its prefix, medium-vertex list, counters) lives
// in one file-scope device array of fixed size, shared by every call on a
// device and kept until the process exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "kb_internal.cuh"

namespace {

constexpr int64_t kMaxVertices = KB_NOALLOC_MAX_VERTICES;
constexpr uint64_t kTableCap = (uint64_t)2 * kMaxVertices;  // load factor 0.5 at the limit
constexpr size_t kAlign = 256;

constexpr size_t up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }
constexpr int64_t kWords = (kMaxVertices >> 5) + 1;
// layout of the scratch array
constexpr size_t kOffCtr = 0;                                        // kb::Counters
constexpr size_t kOffCounts = kOffCtr + up(sizeof(kb::Counters));    // int64 medium count, int64 oversize count
constexpr size_t kOffTable = kOffCounts + up(2 * sizeof(int64_t));
constexpr size_t kOffSlot = kOffTable + up(sizeof(uint64_t) * kTableCap);
constexpr size_t kOffEmin = kOffSlot + up(sizeof(int32_t) * kMaxVertices);
constexpr size_t kOffBitmap = kOffEmin + up(sizeof(uint64_t) * kMaxVertices);
constexpr size_t kOffPrefix = kOffBitmap + up(sizeof(uint32_t) * kWords);
constexpr size_t kOffScan = kOffPrefix + up(sizeof(uint2) * (kWords + 1));  // rank words
constexpr size_t kScanWords = (size_t)((kWords + 4095) / 4096) + 1;
constexpr size_t kOffMed = kOffScan + up(sizeof(uint32_t) * kScanWords);
constexpr size_t kScratchBytes = kOffMed + up(sizeof(int32_t) * kMaxVertices);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once
// per device; the symbol's host-side name is not a device address).
kb_status scratch_address(int device, unsigned char** out) {
    if (device < 0 || device >= kMaxDevices) return KB_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[device]) {
        void* ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) {
            cudaGetLastError();
            return KB_ERR_CUDA;
        }
        g_scratch_ptr[device] = ptr;
        kb::set_medium_kernel_attributes();  // once per device, on the first call
        cudaGetLastError();
    }
    *out = reinterpret_cast<unsigned char*>(g_scratch_ptr[device]);
    return KB_OK;
}

// Level i-1 must hold ids in [0, n): they index the empty-signature minima.
__global__ void check_prev_kernel(int64_t n, const int32_t* prev, kb::Counters* ctr) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    bool bad = false;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        if (prev[v] < 0 || (int64_t)prev[v] >= n) bad = true;
    if (bad) atomicOr(&ctr->err, kb::kErrInvalid);
}

// Vertices this entry point cannot take: a degree above the hub threshold (no
// hub path here) or a negative one (offsets not monotone, when validation is
// off).  Counted into *bad.
__global__ void check_degree_kernel(int64_t n, const int64_t* row, int32_t thr, unsigned long long* bad) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long c = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const int64_t d = row[v + 1] - row[v];
        if (d < 0 || d > thr) ++c;
    }
    if (c) atomicAdd(bad, c);
}

uint64_t next_pow2(uint64_t x) {
    uint64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

#define NA_CUDA(call)                                  \
    do {                                               \
        if ((call) != cudaSuccess) {                   \
            cudaGetLastError();                        \
            return KB_ERR_CUDA;                        \
        }                                              \
    } while (0)

}  // namespace

extern "C" kb_status kb_refine_round_noalloc(void* stream, const kb_graph* g, const kb_options* opt,
                                             const int32_t* prev, int32_t* out, int64_t* count) {
    if (!g || !opt || !count) return KB_ERR_INVALID_ARG;
    if (g->n < 0 || g->m < 0 || g->n > kMaxVertices) return KB_ERR_INVALID_ARG;
    if (opt->direction != KB_DIR_OUT) return KB_ERR_INVALID_ARG;
    if (opt->subject != KB_SUBJECT_PREVIOUS) return KB_ERR_INVALID_ARG;
    if (opt->hash_mode < 0 || opt->hash_mode > 1) return KB_ERR_INVALID_ARG;
    if (opt->hub_threshold < 0 || opt->hub_threshold > kb::kMaxHubThreshold) return KB_ERR_INVALID_ARG;
    if (opt->small_task_vertices != 0 && (opt->small_task_vertices < 32 || opt->small_task_vertices > 65536))
        return KB_ERR_INVALID_ARG;
    if (opt->medium_split < 0 || opt->medium_split > kb::kMaxMedSplit) return KB_ERR_INVALID_ARG;
    if (opt->small_max_degree < 0 || opt->small_max_degree > kb::kSmallDegree) return KB_ERR_INVALID_ARG;
    if (g->n == 0) {
        *count = 0;
        return KB_OK;
    }
    if (!g->row_offsets || !prev || !out || (g->m > 0 && !g->col_indices)) return KB_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int device = 0;
    NA_CUDA(cudaGetDevice(&device));
    unsigned char* base = nullptr;
    const kb_status st = scratch_address(device, &base);
    if (st != KB_OK) return st;

    const int64_t n = g->n;
    const int32_t thr = opt->hub_threshold > 0 ? opt->hub_threshold : kb::kDefaultHubThreshold;
    const uint64_t cap = std::max<uint64_t>(1024, next_pow2((uint64_t)(2 * n)));
    kb::Counters* ctr = reinterpret_cast<kb::Counters*>(base + kOffCtr);
    int64_t* cnts = reinterpret_cast<int64_t*>(base + kOffCounts);

    kb::RoundParams p{};
    p.n = n;
    p.row = g->row_offsets;
    p.col = g->col_indices;
    p.lab = opt->use_edge_labels ? g->edge_labels : nullptr;
    p.prev = prev;
    p.hub_threshold = thr;
    p.small_max = std::min(opt->small_max_degree > 0 ? opt->small_max_degree : kb::kSmallDegree, thr);
    p.warp_verts = opt->small_task_vertices;
    p.hub_chunk = kb::kDefaultHubChunk;  // no hubs here
    p.med_split = opt->medium_split > 0 ? opt->medium_split : kb::kDefaultMedSplit;
    p.hash_mode = opt->hash_mode;
    p.epoch = 1;
    p.table = reinterpret_cast<uint64_t*>(base + kOffTable);
    p.mask = cap - 1;
    p.slot_of = reinterpret_cast<int32_t*>(base + kOffSlot);
    p.emin = reinterpret_cast<uint64_t*>(base + kOffEmin);
    p.ehigh = 0xfffffffeu;  // emin is reset to all ones below, so this round's entries win
    p.bitmap = reinterpret_cast<uint32_t*>(base + kOffBitmap);
    p.ctr = ctr;
    p.med_v = reinterpret_cast<const int32_t*>(base + kOffMed);
    p.n_hubs = 0;

    // The array keeps the previous call's contents: reset what must start clean.
    NA_CUDA(cudaMemsetAsync(ctr, 0, sizeof(kb::Counters), s));
    NA_CUDA(cudaMemsetAsync(cnts, 0, 2 * sizeof(int64_t), s));
    NA_CUDA(cudaMemsetAsync(p.table, 0, sizeof(uint64_t) * cap, s));
    NA_CUDA(cudaMemsetAsync(p.emin, 0xff, sizeof(uint64_t) * (size_t)n, s));
    NA_CUDA(cudaMemsetAsync(p.bitmap, 0, sizeof(uint32_t) * (size_t)((n >> 5) + 1), s));
    if (opt->validate) kb::launch_validate(n, g->m, g->row_offsets, g->col_indices, ctr, s);
    const unsigned grid = (unsigned)std::min<int64_t>((n + 255) / 256, 1024);
    check_prev_kernel<<<grid, 256, 0, s>>>(n, prev, ctr);
    check_degree_kernel<<<grid, 256, 0, s>>>(n, p.row, thr, reinterpret_cast<unsigned long long*>(&cnts[1]));
    if (g->m > 0)
        kb::launch_classify(n, p.row, p.small_max, thr, reinterpret_cast<int32_t*>(base + kOffMed), &cnts[0], s);
    NA_CUDA(cudaGetLastError());
    int64_t host_cnts[2] = {0, 0};
    kb::Counters host_ctr{};
    NA_CUDA(cudaMemcpyAsync(host_cnts, cnts, sizeof(host_cnts), cudaMemcpyDeviceToHost, s));
    NA_CUDA(cudaMemcpyAsync(&host_ctr, ctr, sizeof(host_ctr), cudaMemcpyDeviceToHost, s));
    NA_CUDA(cudaStreamSynchronize(s));
    if (host_ctr.err & kb::kErrInvalid) return KB_ERR_INVALID_ARG;
    if (host_cnts[1] > 0) return KB_ERR_INVALID_ARG;  // a degree outside [0, hub threshold]
    p.n_med = host_cnts[0];

    kb::launch_small_round(p, false, false, s);
    kb::launch_medium_round(p, s);
    kb::launch_renumber(p, reinterpret_cast<uint2*>(base + kOffPrefix), reinterpret_cast<uint32_t*>(base + kOffScan),
                        out, s);
    NA_CUDA(cudaGetLastError());
    NA_CUDA(cudaMemcpyAsync(&host_ctr, ctr, sizeof(host_ctr), cudaMemcpyDeviceToHost, s));
    NA_CUDA(cudaStreamSynchronize(s));
    if (host_ctr.err & kb::kErrTableFull) return KB_ERR_TABLE_FULL;
    if (host_ctr.err) return KB_ERR_DEVICE_CHECK;
    *count = host_ctr.count;
    return KB_OK;
}
