// Device helpers of the serving arena: placing a request's CSR (and moving
// it during compaction) with vertex and edge ids rebased, and writing every
// running request's new level, in its own graph-local ids, to its level store.
#include <cuda_runtime.h>

#include "kb_internal.cuh"

namespace kb {
namespace {

int grid_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152 * 16) b = 152 * 16;
    return (int)b;
}

__global__ void place_vertices_kernel(const PlaceArgs a) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= a.n; i += stride) {
        a.drow[a.dst_vbase + i] = a.srow[a.src_vbase + i] - a.src_ebase + a.dst_ebase;
        if (i == a.n) continue;
        a.dvlab[a.dst_vbase + i] = a.svlab ? a.svlab[a.src_vbase + i] : 0;
        if (a.sB && a.dB) a.dB[a.dst_vbase + i] = (int32_t)((uint32_t)a.sB[a.src_vbase + i] - a.b_sub + a.b_add);
    }
}

__global__ void place_edges_kernel(const PlaceArgs a) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < a.m; j += stride) {
        const uint32_t c = (uint32_t)a.scol[a.src_ebase + j];
        const uint32_t w = (c & 0x7fffffffu) - (uint32_t)a.src_vbase + (uint32_t)a.dst_vbase;
        a.dcol[a.dst_ebase + j] = (int32_t)((c & 0x80000000u) | w);
        a.dlab[a.dst_ebase + j] = a.slab ? a.slab[a.src_ebase + j] : 0;
    }
}

__global__ void emit_kernel(int64_t n, const int32_t* vgraph, const int32_t* B, const uint32_t* gbase,
                            int32_t* const* slot_levels, const int32_t* slot_row, const int64_t* slot_n,
                            const int64_t* voff) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const int32_t g = vgraph[v];
        const int32_t r = slot_row[g];
        if (r < 0) continue;
        const int64_t local = v - voff[g];
        slot_levels[g][(int64_t)r * slot_n[g] + local] = (int32_t)((uint32_t)B[v] - gbase[g]);
    }
}

}  // namespace

void launch_place(const PlaceArgs& a, cudaStream_t s) {
    place_vertices_kernel<<<grid_for(a.n + 1, 256), 256, 0, s>>>(a);
    if (a.m > 0) place_edges_kernel<<<grid_for(a.m, 256), 256, 0, s>>>(a);
}

void launch_emit(int64_t n, const int32_t* vgraph, const int32_t* B, const uint32_t* gbase, int32_t* const* slot_levels,
                 const int32_t* slot_row, const int64_t* slot_n, const int64_t* voff, cudaStream_t s) {
    if (n <= 0) return;
    emit_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, vgraph, B, gbase, slot_levels, slot_row, slot_n, voff);
}

}  // namespace kb
