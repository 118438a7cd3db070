// Per-call setup kernels: input validation, the in-edge / both-direction CSR
// the backward and two-sided equivalences read (paper Defs. "bw-bisim" and
// "vertex-labeled-bw-bisimulation" use in-neighbours, N^-(v) of Section 3.1),
// hub discovery, an int64 prefix scan and level-row copies.
#include <cuda_runtime.h>

#include "kb_internal.cuh"

namespace kb {
namespace {

constexpr uint32_t kFull = 0xffffffffu;

int grid_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (int)b;
}

__global__ void validate_kernel(int64_t n, int64_t m, const int64_t* row, const int32_t* col, Counters* ctr) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool bad = false;
    if (t0 == 0 && (row[0] != 0 || row[n] != m)) bad = true;
    for (int64_t v = t0; v < n; v += stride)
        if (row[v + 1] < row[v]) bad = true;
    for (int64_t e = t0; e < m; e += stride) {
        const int32_t w = col[e];
        if (w < 0 || (int64_t)w >= n) bad = true;
    }
    if (__any_sync(kFull, bad) && (threadIdx.x & 31) == 0) atomicOr(&ctr->err, kErrInvalid);
}

__global__ void in_degree_kernel(int64_t m, const int32_t* col, int64_t* deg) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride)
        atomicAdd(reinterpret_cast<unsigned long long*>(&deg[col[e]]), 1ull);
}

// Source vertex of edge e: the largest v with row[v] <= e.
__device__ __forceinline__ int64_t edge_source(const int64_t* row, int64_t n, int64_t e) {
    int64_t lo = 0, hi = n;  // row[lo] <= e < row[hi]
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (row[mid] <= e) lo = mid; else hi = mid;
    }
    return lo;
}

__global__ void rows_kernel(int64_t n, const int64_t* row, const int64_t* in_prefix, int include_out,
                            int64_t* row_p, int64_t* cursor) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v <= n; v += stride) {
        const int64_t r = (include_out ? row[v] : 0) + in_prefix[v];
        row_p[v] = r;
        if (v < n) cursor[v] = r + (include_out ? row[v + 1] - row[v] : 0);
    }
}

__global__ void place_edges_kernel(int64_t n, int64_t m, const int64_t* row, const int32_t* col, const int32_t* lab,
                                   int include_out, const int64_t* row_p, int32_t* col_p, int32_t* lab_p,
                                   int64_t* cursor) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        const int64_t v = edge_source(row, n, e);
        const int32_t w = col[e];
        const int32_t l = lab ? lab[e] : 0;
        if (include_out) {
            const int64_t q = row_p[v] + (e - row[v]);
            col_p[q] = w;
            if (lab_p) lab_p[q] = l;
        }
        const int64_t q = (int64_t)atomicAdd(reinterpret_cast<unsigned long long*>(&cursor[w]), 1ull);
        col_p[q] = (int32_t)((uint32_t)v | 0x80000000u);
        if (lab_p) lab_p[q] = l;
    }
}

__global__ void find_hubs_kernel(int64_t n, const int64_t* row, int32_t thr, int32_t* out_v, int64_t* out_deg,
                                 int32_t* n_out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const int64_t d = row[v + 1] - row[v];
        if (d > thr) {
            const int32_t i = atomicAdd(n_out, 1);
            out_v[i] = (int32_t)v;
            out_deg[i] = d;
        }
    }
}

// Extent of every hub chunk, packed as (first edge << 16) | edge count, so a
// chunk CTA reads one word instead of a chain of four dependent loads.
__global__ void chunk_ext_kernel(int64_t chunks, const int32_t* chunk_hub, const int32_t* hub_v,
                                 const int64_t* chunk_off, const int64_t* row, int32_t chunk, uint64_t* out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < chunks; c += stride) {
        const int32_t h = chunk_hub[c];
        const int32_t v = hub_v[h];
        const int64_t e0 = row[v] + (c - chunk_off[h]) * (int64_t)chunk;
        const int64_t len = min((int64_t)chunk, row[(int64_t)v + 1] - e0);
        out[c] = ((uint64_t)e0 << 16) | (uint64_t)len;
    }
}

// ---- locality order (see RoundParams::perm)
// How often each vertex is gathered: its occurrences in the processed col,
// counted over runs of 32 edges taken every `stride` edges (all edges when
// stride == 32).
__global__ void count_targets_kernel(int64_t m, const int32_t* col, int64_t stride, uint32_t* cnt) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t runs = (m + stride - 1) / stride;
    for (int64_t r = warp; r < runs; r += nwarps) {
        const int64_t e = r * stride + lane;
        if (e < m) atomicAdd(&cnt[col[e] & 0x7fffffff], 1u);
    }
}

// 256 classes, about 8 per octave of the count; class 0 = never gathered.
__device__ __forceinline__ int hot_class(uint32_t c) {
    if (c == 0) return 0;
    const int e = 31 - __clz(c);
    const int frac = e >= 3 ? (int)((c >> (e - 3)) & 7u) : (int)((c << (3 - e)) & 7u);
    return min(255, 1 + e * 8 + frac);
}

__global__ void class_hist_kernel(int64_t n, const uint32_t* cnt, unsigned long long* hist) {
    __shared__ uint32_t h[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        atomicAdd(&h[hot_class(cnt[v])], 1u);
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += blockDim.x)
        if (h[i]) atomicAdd(&hist[i], (unsigned long long)h[i]);
}

// cursor[k] = vertices in classes above k (hotter classes come first).
__global__ void class_base_kernel(const unsigned long long* hist, unsigned long long* cursor) {
    __shared__ unsigned long long s[256];
    const int k = threadIdx.x;
    s[k] = hist[k];
    __syncthreads();
    if (k == 0) {
        unsigned long long run = 0;
        for (int j = 255; j >= 0; --j) {
            const unsigned long long c = s[j];
            s[j] = run;
            run += c;
        }
    }
    __syncthreads();
    cursor[k] = s[k];
}

// perm[v] = position of v in the class order; one atomic per class and warp.
__global__ void class_scatter_kernel(int64_t n, const uint32_t* cnt, unsigned long long* cursor, int32_t* perm) {
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x; b < n; b += stride) {
        const int64_t v = b + threadIdx.x;
        const bool ok = v < n;
        const int k = ok ? hot_class(cnt[v]) : 256 + lane;  // lanes past the end match nobody
        const unsigned grp = __match_any_sync(kFull, k);
        const int leader = __ffs(grp) - 1;
        unsigned long long base = 0;
        if (ok && lane == leader) base = atomicAdd(&cursor[k], (unsigned long long)__popc(grp));
        base = __shfl_sync(kFull, base, leader);
        if (ok) perm[v] = (int32_t)(base + __popc(grp & ((1u << lane) - 1u)));
    }
}

// Neighbour ids -> positions in the order, keeping the direction bit.
__global__ void remap_cols_kernel(int64_t m, const int32_t* col, const int32_t* perm, int32_t* out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
        const int32_t w = col[e];
        out[e] = (int32_t)((uint32_t)perm[w & 0x7fffffff] | ((uint32_t)w & 0x80000000u));
    }
}

__global__ void classify_kernel(int64_t n, const int64_t* row, int32_t lo, int32_t hi, int32_t* out,
                                unsigned long long* n_out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
        const int64_t v = base + threadIdx.x;
        bool take = false;
        if (v < n) {
            const int64_t d = row[v + 1] - row[v];
            take = d > lo && d <= hi;
        }
        const unsigned b = __ballot_sync(kFull, take);
        if (!b) continue;
        unsigned long long pos = 0;
        if (lane == 0) pos = atomicAdd(n_out, (unsigned long long)__popc(b));
        pos = __shfl_sync(kFull, pos, 0);
        if (take) out[pos + __popc(b & ((1u << lane) - 1u))] = (int32_t)v;
    }
}

// ---- int64 exclusive scan (reduce, scan of block sums, down-sweep)
constexpr int kT = 1024;
constexpr int kItems = 4;
constexpr int kTile = kT * kItems;

__device__ __forceinline__ int64_t block_exscan_i64(int64_t x, int64_t* tmp, int64_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) tmp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int64_t w = tmp[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(kFull, w, o);
            if (lane >= o) w += y;
        }
        tmp[lane] = w;
    }
    __syncthreads();
    const int64_t base = warp > 0 ? tmp[warp - 1] : 0;
    *total = tmp[31];
    __syncthreads();
    return base + incl - x;
}

__global__ void __launch_bounds__(kT) scan_reduce_kernel(const int64_t* in, int64_t n, int64_t* sums) {
    __shared__ int64_t tmp[32];
    const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kItems;
    int64_t s = 0;
#pragma unroll
    for (int u = 0; u < kItems; ++u)
        if (base + u < n) s += in[base + u];
    int64_t total;
    block_exscan_i64(s, tmp, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kT) scan_sums_kernel(int64_t* sums, int64_t nb) {
    __shared__ int64_t tmp[32];
    int64_t carry = 0;
    for (int64_t b = 0; b < nb; b += kT) {
        const int64_t i = b + threadIdx.x;
        const int64_t x = i < nb ? sums[i] : 0;
        int64_t total;
        const int64_t ex = block_exscan_i64(x, tmp, &total);
        if (i < nb) sums[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) sums[nb] = carry;
}

__global__ void __launch_bounds__(kT) scan_down_kernel(const int64_t* in, int64_t n, const int64_t* sums,
                                                        int64_t* out) {
    __shared__ int64_t tmp[32];
    const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kItems;
    int64_t c[kItems];
    int64_t s = 0;
#pragma unroll
    for (int u = 0; u < kItems; ++u) {
        c[u] = base + u < n ? in[base + u] : 0;
        s += c[u];
    }
    int64_t total;
    int64_t ex = block_exscan_i64(s, tmp, &total) + sums[blockIdx.x];
    __syncthreads();  // every thread has read its inputs before any output is written (in may alias out)
#pragma unroll
    for (int u = 0; u < kItems; ++u) {
        if (base + u < n) out[base + u] = ex;
        ex += c[u];
    }
}

__global__ void write_total_kernel(const int64_t* sums, int64_t nb, int64_t* out, int64_t n) { out[n] = sums[nb]; }

}  // namespace

void launch_validate(int64_t n, int64_t m, const int64_t* row, const int32_t* col, Counters* ctr, cudaStream_t s) {
    validate_kernel<<<grid_for(n > m ? n : m, 256), 256, 0, s>>>(n, m, row, col, ctr);
}

void launch_in_degree(int64_t m, const int32_t* col, int64_t* deg, cudaStream_t s) {
    if (m <= 0) return;
    in_degree_kernel<<<grid_for(m, 256), 256, 0, s>>>(m, col, deg);
}

size_t scan_i64_tmp(int64_t n) { return (size_t)((n + kTile - 1) / kTile) + 2; }

void launch_scan_i64(const int64_t* in, int64_t n, int64_t* out, int64_t* tmp, cudaStream_t s) {
    const int64_t nb = (n + kTile - 1) / kTile;
    if (nb > 0) scan_reduce_kernel<<<(unsigned)nb, kT, 0, s>>>(in, n, tmp);
    scan_sums_kernel<<<1, kT, 0, s>>>(tmp, nb);
    if (nb > 0) scan_down_kernel<<<(unsigned)nb, kT, 0, s>>>(in, n, tmp, out);
    write_total_kernel<<<1, 1, 0, s>>>(tmp, nb, out, n);
}

void launch_build_csr(int64_t n, int64_t m, const int64_t* row, const int32_t* col, const int32_t* lab,
                      const int64_t* in_prefix, int include_out, int64_t* row_p, int32_t* col_p, int32_t* lab_p,
                      int64_t* cursor, cudaStream_t s) {
    rows_kernel<<<grid_for(n + 1, 256), 256, 0, s>>>(n, row, in_prefix, include_out, row_p, cursor);
    if (m > 0)
        place_edges_kernel<<<grid_for(m, 256), 256, 0, s>>>(n, m, row, col, lab, include_out, row_p, col_p, lab_p,
                                                            cursor);
}

void launch_find_hubs(int64_t n, const int64_t* row, int32_t thr, int32_t* out_v, int64_t* out_deg, int32_t* n_out,
                      cudaStream_t s) {
    if (n <= 0) return;
    find_hubs_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, row, thr, out_v, out_deg, n_out);
}

void launch_chunk_ext(int64_t chunks, const int32_t* chunk_hub, const int32_t* hub_v, const int64_t* chunk_off,
                      const int64_t* row, int32_t chunk, uint64_t* out, cudaStream_t s) {
    if (chunks <= 0) return;
    chunk_ext_kernel<<<grid_for(chunks, 256), 256, 0, s>>>(chunks, chunk_hub, hub_v, chunk_off, row, chunk, out);
}

void launch_locality_order(int64_t n, int64_t m, const int32_t* col, uint32_t* cnt, unsigned long long* hist,
                           int32_t* perm, cudaStream_t s) {
    if (n <= 0) return;
    cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * (size_t)n, s);
    cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * 512, s);
    if (m > 0) {
        // every edge up to 2^26 edges, then one run of 32 in every 256
        const int64_t stride = m <= ((int64_t)1 << 26) ? 32 : 256;
        const int64_t runs = (m + stride - 1) / stride;
        count_targets_kernel<<<grid_for(runs * 32, 256), 256, 0, s>>>(m, col, stride, cnt);
    }
    class_hist_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, cnt, hist);
    class_base_kernel<<<1, 256, 0, s>>>(hist, hist + 256);
    class_scatter_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, cnt, hist + 256, perm);
}

void launch_remap_cols(int64_t m, const int32_t* col, const int32_t* perm, int32_t* out, cudaStream_t s) {
    if (m <= 0) return;
    remap_cols_kernel<<<grid_for(m, 256), 256, 0, s>>>(m, col, perm, out);
}

void launch_classify(int64_t n, const int64_t* row, int32_t lo, int32_t hi, int32_t* out, int64_t* n_out,
                     cudaStream_t s) {
    if (n <= 0) return;
    classify_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, row, lo, hi, out,
                                                     reinterpret_cast<unsigned long long*>(n_out));
}

void launch_copy_rows(int32_t* levels, int64_t n, int src, int first, int last, cudaStream_t s) {
    for (int r = first; r <= last; ++r)
        if (r != src)
            cudaMemcpyAsync(levels + (size_t)r * (size_t)n, levels + (size_t)src * (size_t)n,
                            sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s);
}

}  // namespace kb
