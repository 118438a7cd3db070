// Summary graph of a partition pair (Sec. "Graph Summaries for Bisimulation":
// one summary vertex per block, a labelled summary edge from block b to block c
// when the vertices of b have an edge with that label into c).
//
// Every edge v -> w with label l gives the triple (lsrc[x], l, ldst[y]), with
// x -> y the edge in the processed direction.  The distinct triples are found
// with one open-addressing table of 16-byte slots claimed by a 128-bit CAS (the
// triple itself is the key, so no compare against a representative is
// needed); each slot also keeps its smallest edge index.  Output order is
// first occurrence in the edge list: the first edges are marked in an edge
// bitmap, ranked by a popcount prefix scan, and every first edge writes its
// triple at its rank.
//
//   insert  CTA tiles of kSumTile consecutive edges: two binary searches give
//           the tile's source range, every edge finds its source inside it;
//           lanes of a warp holding the same triple elect the lowest (its edge
//           comes first) to probe the table, so repeated triples cost one
//           atomic per warp;
//   mark    one bit per occupied slot, at its first edge;
//   emit    the edges again, in order: every first occurrence re-derives its
//           triple and writes it at its rank (consecutive writes per warp).
#include <cuda_runtime.h>

#include "kb_device.cuh"
#include "kb_internal.cuh"

namespace kb {
namespace {

constexpr int kSumThreads = 256;
constexpr int kSumPer = 4;
constexpr int kSumTile = kSumThreads * kSumPer;

// Atomic 128-bit compare-and-swap of a 16-byte aligned slot (lo at the lower
// address); returns the slot's previous contents.
__device__ __forceinline__ void cas128(unsigned long long* slot, unsigned long long clo, unsigned long long chi,
                                       unsigned long long nlo, unsigned long long nhi, unsigned long long* olo,
                                       unsigned long long* ohi) {
    asm volatile(
        "{\n\t.reg .b128 d, c, n;\n\t"
        "mov.b128 c, {%2, %3};\n\t"
        "mov.b128 n, {%4, %5};\n\t"
        "atom.global.cas.b128 d, [%6], c, n;\n\t"
        "mov.b128 {%0, %1}, d;\n\t}"
        : "=l"(*olo), "=l"(*ohi)
        : "l"(clo), "l"(chi), "l"(nlo), "l"(nhi), "l"(slot)
        : "memory");
}

// The source of edge e among vertices [lo, hi]: row[v] <= e < row[v + 1].
__device__ __forceinline__ int64_t source_in(const int64_t* row, int64_t lo, int64_t hi, int64_t e) {
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (row[mid] <= e) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(kSumThreads) summary_insert_kernel(const SummaryParams q) {
    __shared__ int64_t s_v[2];
    const int lane = threadIdx.x & 31;
    const int64_t tiles = (q.m + kSumTile - 1) / kSumTile;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int64_t e0 = t * kSumTile;
        const int64_t e1 = min(q.m, e0 + kSumTile) - 1;
        __syncthreads();  // s_v of the previous tile is no longer read
        if (threadIdx.x < 2) s_v[threadIdx.x] = source_in(q.row, 0, q.n - 1, threadIdx.x ? e1 : e0);
        __syncthreads();
        const int64_t vlo = s_v[0], vhi = s_v[1];
#pragma unroll
        for (int u = 0; u < kSumPer; ++u) {
            const int64_t e = e0 + u * kSumThreads + threadIdx.x;
            const bool ok = e < q.m;
            unsigned long long lo = 0, hi = 0;
            if (ok) {
                const int64_t v = source_in(q.row, vlo, vhi, e);
                const int64_t w = q.col[e];
                const int64_t x = q.dir == 0 ? v : w;
                const int64_t y = q.dir == 0 ? w : v;
                const uint32_t l = q.lab ? (uint32_t)q.lab[e] : 0u;
                lo = ((unsigned long long)l << 32) | (uint32_t)q.lsrc[x];
                hi = (1ull << 32) | (uint32_t)q.ldst[y];  // bit 32 marks an occupied slot
            }
            // lanes with the same triple: the lowest one (smallest edge) inserts
            const unsigned grp = __match_any_sync(kFull, lo) & __match_any_sync(kFull, hi);
            if (!ok || lane != __ffs(grp) - 1) continue;
            uint64_t pos = mix64(lo ^ mix64(hi ^ 0x2545f4914f6cdd1dULL)) & q.mask;
            bool placed = false;
            for (int it = 0; it < kProbeLimit; ++it) {
                unsigned long long olo, ohi;
                cas128(q.table + 2 * pos, 0ull, 0ull, lo, hi, &olo, &ohi);
                if ((olo == 0ull && ohi == 0ull) || (olo == lo && ohi == hi)) {
                    placed = true;
                    break;
                }
                pos = (pos + 1) & q.mask;
            }
            if (!placed) {
                set_error(q.ctr, kErrTableFull);
                continue;
            }
            unsigned long long* f = q.first + pos;
            if ((unsigned long long)e < *reinterpret_cast<volatile unsigned long long*>(f))
                atomicMin(f, (unsigned long long)e);
        }
    }
}

__global__ void summary_mark_kernel(const SummaryParams q) {
    const int64_t cap = (int64_t)q.mask + 1;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cap; i += stride) {
        if (q.table[2 * i + 1] == 0ull) continue;
        const unsigned long long e = q.first[i];
        if (e >= (unsigned long long)q.m) {  // only after a reported table overflow
            set_error(q.ctr, kErrTableFull);
            continue;
        }
        atomicOr(&q.bitmap[e >> 5], 1u << (e & 31));
    }
}

// Walks the edges again in their order: a first occurrence re-derives its
// triple and writes it at its rank, so a warp's writes are consecutive.
__global__ void __launch_bounds__(kSumThreads) summary_emit_kernel(const SummaryParams q, const uint32_t* prefix,
                                                                   int32_t* out_src, int32_t* out_label,
                                                                   int32_t* out_dst) {
    __shared__ int64_t s_v[2];
    const int lane = threadIdx.x & 31;
    const int64_t tiles = (q.m + kSumTile - 1) / kSumTile;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int64_t e0 = t * kSumTile;
        const int64_t e1 = min(q.m, e0 + kSumTile) - 1;
        __syncthreads();
        if (threadIdx.x < 2) s_v[threadIdx.x] = source_in(q.row, 0, q.n - 1, threadIdx.x ? e1 : e0);
        __syncthreads();
        const int64_t vlo = s_v[0], vhi = s_v[1];
#pragma unroll
        for (int u = 0; u < kSumPer; ++u) {
            const int64_t e = e0 + u * kSumThreads + threadIdx.x;
            if (e >= q.m) continue;
            const uint32_t w = q.bitmap[e >> 5];
            if (!((w >> lane) & 1u)) continue;  // e & 31 == lane: tiles and warps are 32-aligned
            const int64_t v = source_in(q.row, vlo, vhi, e);
            const int64_t y0 = q.col[e];
            const int64_t x = q.dir == 0 ? v : y0;
            const int64_t y = q.dir == 0 ? y0 : v;
            const uint32_t r = prefix[e >> 5] + (uint32_t)__popc(w & ((1u << lane) - 1u));
            out_src[r] = q.lsrc[x];
            out_label[r] = q.lab ? q.lab[e] : 0;
            out_dst[r] = q.ldst[y];
        }
    }
}

int grid_of(int64_t items, int threads) {
    const int64_t b = (items + threads - 1) / threads;
    return (int)(b < 1 ? 1 : (b > 152 * 64 ? 152 * 64 : b));
}

}  // namespace

void launch_summary_insert(const SummaryParams& q, cudaStream_t s) {
    if (q.m <= 0) return;
    const int64_t tiles = (q.m + kSumTile - 1) / kSumTile;
    summary_insert_kernel<<<grid_of(tiles * kSumThreads, kSumThreads), kSumThreads, 0, s>>>(q);
}

void launch_summary_mark(const SummaryParams& q, cudaStream_t s) {
    summary_mark_kernel<<<grid_of((int64_t)q.mask + 1, 256), 256, 0, s>>>(q);
}

void launch_summary_emit(const SummaryParams& q, const uint32_t* prefix, int32_t* out_src, int32_t* out_label,
                         int32_t* out_dst, cudaStream_t s) {
    if (q.m <= 0) return;
    const int64_t tiles = (q.m + kSumTile - 1) / kSumTile;
    summary_emit_kernel<<<grid_of(tiles * kSumThreads, kSumThreads), kSumThreads, 0, s>>>(q, prefix, out_src,
                                                                                       out_label, out_dst);
}

}  // namespace kb
