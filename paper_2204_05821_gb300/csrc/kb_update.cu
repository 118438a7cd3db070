// Incremental refinement after edge insertions and deletions
// (kb_refine_update).  The paper leaves incremental k-bisimulation as future
// work (Sec. "Conclusion and Future Work": one changed edge can change ids in
// every later round).  Here a round re-keys only a work set W and keeps the
// old grouping of every other vertex:
//
//   dirty(i)  = changed edge lists, vertices whose block changed as a set at
//               level i-1 ("moved"), and vertices with an edge to a moved one;
//   W(i)      = every vertex of a level-(i-1) block that holds a dirty vertex.
//
// Keys hold the own previous block, so a level-i block lies inside one
// level-(i-1) block: blocks are either inside W or outside it.  Outside W,
// edge lists, neighbour blocks and own blocks are unchanged as sets, so two
// such vertices are equivalent now exactly when they were before.  Every
// level is then renumbered canonically in full.
#include <cuda_runtime.h>

#include "kb_device.cuh"
#include "kb_internal.cuh"

namespace kb {
namespace {

constexpr int kT = 256;
constexpr int kPer = 4;
constexpr int kTile = kT * kPer;

__device__ __forceinline__ bool bit(const uint32_t* b, int64_t v) { return (b[v >> 5] >> (v & 31)) & 1u; }

__device__ __forceinline__ int64_t source_in(const int64_t* row, int64_t lo, int64_t hi, int64_t e) {
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (row[mid] <= e) lo = mid; else hi = mid - 1;
    }
    return lo;
}

int grid_of(int64_t items, int threads) {
    const int64_t b = (items + threads - 1) / threads;
    return (int)(b < 1 ? 1 : (b > 152 * 64 ? 152 * 64 : b));
}

// dirty[v] |= moved[y] over every edge v -> y of the processed CSR, in tiles of
// consecutive edges (two binary searches give a tile's source range).
__global__ void __launch_bounds__(kT) dirty_from_moved_kernel(int64_t n, int64_t m, const int64_t* row,
                                                              const int32_t* col, const uint32_t* moved,
                                                              uint32_t* dirty) {
    __shared__ int64_t s_v[2];
    const int64_t tiles = (m + kTile - 1) / kTile;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int64_t e0 = t * kTile;
        const int64_t e1 = min(m, e0 + kTile) - 1;
        __syncthreads();
        if (threadIdx.x < 2) s_v[threadIdx.x] = source_in(row, 0, n - 1, threadIdx.x ? e1 : e0);
        __syncthreads();
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
            const int64_t e = e0 + u * kT + threadIdx.x;
            if (e >= m || !bit(moved, col[e] & 0x7fffffff)) continue;
            const int64_t v = source_in(row, s_v[0], s_v[1], e);
            atomicOr(&dirty[v >> 5], 1u << (v & 31));
        }
    }
}

__global__ void or_words_kernel(int64_t nw, const uint32_t* a, const uint32_t* b, uint32_t* out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nw; i += stride) out[i] = a[i] | b[i];
}

// flag[b] = 1 for every level-(i-1) block b holding a dirty vertex
__global__ void flag_blocks_kernel(int64_t n, const int32_t* prev, const uint32_t* dirty, uint8_t* flag) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        if (bit(dirty, v)) flag[prev[v]] = 1;
}

// W = vertices of flagged blocks, one bitmap word per warp; |W| into count
__global__ void work_set_kernel(int64_t n, const int32_t* prev, const uint8_t* flag, uint32_t* wmask,
                                unsigned long long* count) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
        const int64_t v = base + threadIdx.x;  // blockDim is a multiple of 32: a warp covers one word
        const bool in = v < n && flag[prev[v]];
        const unsigned b = __ballot_sync(kFull, in);
        if ((threadIdx.x & 31) == 0 && (v >> 5) <= ((n - 1) >> 5)) {
            wmask[v >> 5] = b;
            if (b) atomicAdd(count, (unsigned long long)__popc(b));
        }
    }
}

// kmin[b] = smallest vertex outside W of old block b
__global__ void keep_min_kernel(int64_t n, const uint32_t* wmask, const int32_t* old, uint32_t* kmin) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        if (!bit(wmask, v)) atomicMin(&kmin[old[v]], (uint32_t)v);
}

// the kept blocks' smallest members into the bitmap of block minima
__global__ void keep_bits_kernel(int64_t n, const uint32_t* wmask, const int32_t* old, const uint32_t* kmin,
                                 uint32_t* bitmap) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
        const int64_t v = base + threadIdx.x;
        const bool mn = v < n && !bit(wmask, v) && kmin[old[v]] == (uint32_t)v;
        const unsigned b = __ballot_sync(kFull, mn);
        if ((threadIdx.x & 31) == 0 && b) atomicOr(&bitmap[v >> 5], b);
    }
}

// per old block the range of new ids, per new block the range of old ids (W only)
__global__ void moved_scatter_kernel(int64_t n, const uint32_t* wmask, const int32_t* old, const int32_t* cur,
                                     int32_t* om_lo, int32_t* om_hi, int32_t* nm_lo, int32_t* nm_hi) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        if (!bit(wmask, v)) continue;
        const int32_t a = old[v], b = cur[v];
        atomicMin(&om_lo[a], b);
        atomicMax(&om_hi[a], b);
        atomicMin(&nm_lo[b], a);
        atomicMax(&nm_hi[b], a);
    }
}

// moved: a vertex of W whose old block split or whose new block merged
__global__ void moved_mark_kernel(int64_t n, const uint32_t* wmask, const int32_t* old, const int32_t* cur,
                                  const int32_t* om_lo, const int32_t* om_hi, const int32_t* nm_lo,
                                  const int32_t* nm_hi, uint32_t* moved) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
        const int64_t v = base + threadIdx.x;
        bool mv = false;
        if (v < n && bit(wmask, v)) {
            const int32_t a = old[v], b = cur[v];
            mv = om_lo[a] != om_hi[a] || nm_lo[b] != nm_hi[b];
        }
        const unsigned w = __ballot_sync(kFull, mv);
        if ((threadIdx.x & 31) == 0 && (v >> 5) <= ((n - 1) >> 5)) moved[v >> 5] = w;
    }
}

__global__ void check_ids_kernel(int64_t n, const int32_t* a, Counters* ctr) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    bool bad = false;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        bad |= a[v] < 0 || (int64_t)a[v] >= n;
    if (__any_sync(kFull, bad) && (threadIdx.x & 31) == 0) atomicOr(&ctr->err, kErrInvalid);
}

__global__ void set_bits_kernel(int64_t n, int64_t count, const int32_t* ids, uint32_t* bits, Counters* ctr) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
        const int32_t v = ids[i];
        if (v < 0 || (int64_t)v >= n) {
            atomicOr(&ctr->err, kErrInvalid);
            continue;
        }
        atomicOr(&bits[v >> 5], 1u << (v & 31));
    }
}

// Blocks of `level` holding a vertex of ids[0..count) into touched (ids and
// level values already checked to lie in [0, n)).
__global__ void touch_blocks_kernel(int64_t count, const int32_t* ids, const int32_t* level, uint32_t* touched) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
        const int32_t b = level[ids[i]];
        atomicOr(&touched[b >> 5], 1u << (b & 31));
    }
}

// *out += vertices whose block of `level` is touched.
__global__ void __launch_bounds__(256) touched_size_kernel(int64_t n, const int32_t* level, const uint32_t* touched,
                                                            unsigned long long* out) {
    __shared__ unsigned long long s_sum[8];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long c = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const int32_t b = level[v];
        c += (touched[b >> 5] >> (b & 31)) & 1u;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) s_sum[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < 8; ++w) t += s_sum[w];
        if (t) atomicAdd(out, t);
    }
}

}  // namespace

void launch_dirty_from_moved(int64_t n, int64_t m, const int64_t* row, const int32_t* col, const uint32_t* moved,
                             uint32_t* dirty, cudaStream_t s) {
    if (n <= 0 || m <= 0) return;
    const int64_t tiles = (m + kTile - 1) / kTile;
    dirty_from_moved_kernel<<<grid_of(tiles * kT, kT), kT, 0, s>>>(n, m, row, col, moved, dirty);
}

void launch_or_words(int64_t nw, const uint32_t* a, const uint32_t* b, uint32_t* out, cudaStream_t s) {
    if (nw > 0) or_words_kernel<<<grid_of(nw, 256), 256, 0, s>>>(nw, a, b, out);
}

void launch_work_set(int64_t n, const int32_t* prev, const uint32_t* dirty, uint8_t* flag, uint32_t* wmask,
                     unsigned long long* count, cudaStream_t s) {
    if (n <= 0) return;
    cudaMemsetAsync(flag, 0, (size_t)n, s);
    flag_blocks_kernel<<<grid_of(n, 256), 256, 0, s>>>(n, prev, dirty, flag);
    work_set_kernel<<<grid_of(n, 256), 256, 0, s>>>(n, prev, flag, wmask, count);
}

void launch_keep_min(int64_t n, const uint32_t* wmask, const int32_t* old, uint32_t* kmin, cudaStream_t s) {
    if (n <= 0) return;
    cudaMemsetAsync(kmin, 0xff, sizeof(uint32_t) * (size_t)n, s);
    keep_min_kernel<<<grid_of(n, 256), 256, 0, s>>>(n, wmask, old, kmin);
}

void launch_keep_bits(int64_t n, const uint32_t* wmask, const int32_t* old, const uint32_t* kmin, uint32_t* bitmap,
                      cudaStream_t s) {
    if (n > 0) keep_bits_kernel<<<grid_of(n, 256), 256, 0, s>>>(n, wmask, old, kmin, bitmap);
}

void launch_moved(int64_t n, const uint32_t* wmask, const int32_t* old, const int32_t* cur, int32_t* ranges,
                  uint32_t* moved, cudaStream_t s) {
    if (n <= 0) return;
    int32_t* om_lo = ranges;
    int32_t* om_hi = ranges + n;
    int32_t* nm_lo = ranges + 2 * n;
    int32_t* nm_hi = ranges + 3 * n;
    launch_fill_i32(om_lo, n, 0x7fffffff, s);
    launch_fill_i32(om_hi, n, -1, s);
    launch_fill_i32(nm_lo, n, 0x7fffffff, s);
    launch_fill_i32(nm_hi, n, -1, s);
    moved_scatter_kernel<<<grid_of(n, 256), 256, 0, s>>>(n, wmask, old, cur, om_lo, om_hi, nm_lo, nm_hi);
    moved_mark_kernel<<<grid_of(n, 256), 256, 0, s>>>(n, wmask, old, cur, om_lo, om_hi, nm_lo, nm_hi, moved);
}

void launch_check_ids(int64_t n, const int32_t* a, Counters* ctr, cudaStream_t s) {
    if (n > 0) check_ids_kernel<<<grid_of(n, 256), 256, 0, s>>>(n, a, ctr);
}

void launch_set_bits(int64_t n, int64_t count, const int32_t* ids, uint32_t* bits, Counters* ctr, cudaStream_t s) {
    if (count > 0) set_bits_kernel<<<grid_of(count, 256), 256, 0, s>>>(n, count, ids, bits, ctr);
}

void launch_touched_size(int64_t n, int64_t count, const int32_t* ids, const int32_t* level, uint32_t* touched,
                         unsigned long long* out, cudaStream_t s) {
    if (count > 0) touch_blocks_kernel<<<grid_of(count, 256), 256, 0, s>>>(count, ids, level, touched);
    const int g = grid_of(n, 256) < 1216 ? grid_of(n, 256) : 1216;
    if (n > 0) touched_size_kernel<<<g, 256, 0, s>>>(n, level, touched, out);
}

}  // namespace kb
