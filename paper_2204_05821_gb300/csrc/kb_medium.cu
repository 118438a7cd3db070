// Warp kernels for the medium vertices (small_max < degree <= hub_threshold).
//
// One warp takes one vertex at a time and never waits on the rest of its CTA,
// so the memory latencies of different warps overlap freely:
//   * the vertex's (direction, edge label, previous block of neighbour) pairs
//     go into a warp-private open-addressing set in shared memory (the pairs
//     themselves, inserted with a 64-bit shared CAS), sized to the next power
//     of two >= 2 x degree; a pair that is already present is a duplicate
//     (set semantics, Def. "signature"), a new one is summed into the
//     order-independent hash;
//   * neighbour ids and labels of the next batch of edges are loaded before
//     the current batch's gathered blocks are consumed;
//   * lane 0 probes the block table; on a tag match the warp re-derives the
//     representative's pairs from the CSR and looks each one up in the set,
//     marking hits in a bitmap: the signatures are equal when every pair of
//     the representative is found and the distinct pairs hit number exactly
//     the vertex's own count.
//
// Two kernels share the medium-vertex list, each skipping the other's
// vertices: degrees up to RoundParams::med_split (at most 256) take a warp
// each (512-entry sets, 4 warps per CTA); larger degrees, up to 1024, take a
// CTA of 128 threads each (one 2048-entry set).
#include <cuda_runtime.h>

#include <algorithm>

#include "kb_device.cuh"
#include "kb_internal.cuh"

namespace kb {
namespace {

constexpr int kMedSplit = kMaxMedSplit;  // largest degree the warp kernel's set holds
constexpr int kMedTask = 32;    // list entries per warp task (one per lane)
constexpr int kMedCtaThreads = 128;  // threads per vertex of the second class
static_assert(kMaxHubThreshold <= 1024, "the second class holds degrees up to 1024");

// Home slot of a pair in a vertex's shared set: bits of the same mix that
// enters the hash sum, so each new pair costs one mix.
__device__ __forceinline__ uint32_t med_slot(uint64_t pm, uint32_t cmask) { return (uint32_t)(pm >> 24) & cmask; }

template <int kCap, int kWarps>
__global__ void __launch_bounds__(kWarps * 32) medium_round_kernel(const RoundParams p, int32_t dlo, int32_t dhi) {
    __shared__ uint64_t s_set[kWarps][kCap];
    __shared__ uint32_t s_mark[kWarps][kCap / 32];
    constexpr int U = 4;  // edges per lane and batch

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t* set = s_set[warp];
    uint32_t* mark = s_mark[warp];
    const int64_t t0 = ((int64_t)blockIdx.x * kWarps + warp) * kMedTask;
    if (t0 >= p.n_med) return;  // uniform over the warp
    const int nt = (int)min((int64_t)kMedTask, p.n_med - t0);

    // the task's vertices, row offsets and own blocks, loaded at once
    int32_t tv = 0, town = 0;
    int64_t trs = 0, tre = 0;
    bool take = false;
    if (lane < nt) {
        tv = p.med_v[t0 + lane];
        trs = p.row[tv];
        tre = p.row[(int64_t)tv + 1];
        town = own_of(p, tv);
        const int64_t d = tre - trs;
        take = d > dlo && d <= dhi && vertex_refines(p, tv);
    }
    unsigned todo = __ballot_sync(kFull, take);

    while (todo) {
        const int j = __ffs(todo) - 1;
        todo &= todo - 1;
        const int32_t v = __shfl_sync(kFull, tv, j);
        const int32_t own = __shfl_sync(kFull, town, j);
        const int64_t rs = __shfl_sync(kFull, trs, j);
        const int64_t re = __shfl_sync(kFull, tre, j);
        const int d = (int)(re - rs);
        int c = 64;
        while (c < 2 * d) c <<= 1;
        if (c > kCap) {  // cannot happen: dhi <= kCap / 2
            if (lane == 0) set_error(p.ctr, kErrStage);
            continue;
        }
        const uint32_t cmask = (uint32_t)c - 1u;
        for (int i = lane; i < c; i += 32) set[i] = kEmptyPair;
        __syncwarp();

        uint64_t acc = 0;
        uint32_t cnt = 0;
        int32_t w[U], l[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t e = rs + u * 32 + lane;
            w[u] = 0;
            l[u] = 0;
            if (e < re) {
                w[u] = __ldcs(p.col + e);
                l[u] = p.lab ? __ldcs(p.lab + e) : 0;
            }
        }
        for (int64_t e0 = rs; e0 < re; e0 += 32 * U) {
            int32_t b[U];
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (e0 + u * 32 + lane < re) b[u] = gather_block(p, w[u]);
            // the next batch's neighbours and labels, issued before the gather is consumed
            int32_t w2[U], l2[U];
            const int64_t e1 = e0 + 32 * U;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t e = e1 + u * 32 + lane;
                w2[u] = 0;
                l2[u] = 0;
                if (e < re) {
                    w2[u] = __ldcs(p.col + e);
                    l2[u] = p.lab ? __ldcs(p.lab + e) : 0;
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (e0 + u * 32 + lane >= re) continue;
                const uint64_t pr = pack_pair(l[u], (uint32_t)w[u], b[u]);
                const uint64_t pm = pair_mix(pr);
                uint32_t slot = med_slot(pm, cmask);
                while (true) {
                    const unsigned long long old = atomicCAS(reinterpret_cast<unsigned long long*>(set + slot),
                                                             (unsigned long long)kEmptyPair, (unsigned long long)pr);
                    if (old == (unsigned long long)kEmptyPair) {
                        acc += pm;
                        ++cnt;
                        break;
                    }
                    if (old == (unsigned long long)pr) break;
                    slot = (slot + 1) & cmask;
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                w[u] = w2[u];
                l[u] = l2[u];
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            acc += __shfl_xor_sync(kFull, (unsigned long long)acc, o);
            cnt += __shfl_xor_sync(kFull, cnt, o);
        }
        __syncwarp();

        // find or insert, with the full signature compare on every tag match
        const uint64_t h = vertex_hash(own, cnt, acc, p.hash_mode);
        uint64_t pos = h & p.mask;
        const uint32_t hi = table_hi(h, p.epoch);
        while (true) {
            int r = 0;
            uint32_t rep = 0;
            if (lane == 0) r = probe_table(p, &pos, hi, (uint32_t)v, &rep);
            r = __shfl_sync(kFull, r, 0);
            if (r == 0) break;
            if (r == 2) {
                if (lane == 0) set_error(p.ctr, kErrTableFull);
                break;
            }
            rep = __shfl_sync(kFull, rep, 0);
            pos = __shfl_sync(kFull, (unsigned long long)pos, 0);
            bool ok = same_graph(p, rep, v) && own_of(p, rep) == own;
            if (ok) {
                for (int i = lane; i < c / 32; i += 32) mark[i] = 0u;
                __syncwarp();
                const int64_t rb = p.row[rep], rend = p.row[(int64_t)rep + 1];
                uint32_t nf = 0;
                for (int64_t e0 = rb; e0 < rend && ok; e0 += 32) {
                    const int64_t e = e0 + lane;
                    bool found = true;
                    if (e < rend) {
                        const int32_t ww = __ldg(p.col + e);
                        const int32_t ll = p.lab ? __ldg(p.lab + e) : 0;
                        const uint64_t pr = pack_pair(ll, (uint32_t)ww, gather_block(p, ww));
                        uint32_t slot = med_slot(pair_mix(pr), cmask);
                        found = false;
                        while (true) {
                            const uint64_t cur = set[slot];
                            if (cur == kEmptyPair) break;
                            if (cur == pr) {
                                const uint32_t bit = 1u << (slot & 31);
                                const uint32_t old = atomicOr(&mark[slot >> 5], bit);
                                if (!(old & bit)) ++nf;
                                found = true;
                                break;
                            }
                            slot = (slot + 1) & cmask;
                        }
                    }
                    ok = __all_sync(kFull, found);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) nf += __shfl_xor_sync(kFull, nf, o);
                ok = ok && nf == cnt;
                __syncwarp();
            }
            if (ok) {
                if (lane == 0) join_slot(p, pos, hi, (uint32_t)v);
                break;
            }
            pos = (pos + 1) & p.mask;
        }
        __syncwarp();  // the set is rebuilt for the next vertex
    }
}

// The same for degrees up to 1024, one CTA per vertex: its kThreads threads
// share one set, so a 2048-entry set costs 16 KB per CTA instead of per warp
// and the SM keeps many more warps in flight.
template <int kCap, int kThreads>
__global__ void __launch_bounds__(kThreads) medium_cta_kernel(const RoundParams p, int32_t dlo, int32_t dhi) {
    constexpr int U = 4;
    constexpr int W = kThreads / 32;
    __shared__ uint64_t s_set[kCap];
    __shared__ uint32_t s_mark[kCap / 32];
    __shared__ int32_t s_v[kMedTask], s_own[kMedTask];
    __shared__ int64_t s_rs[kMedTask], s_re[kMedTask];
    __shared__ unsigned long long s_acc[W];
    __shared__ uint32_t s_cnt[W];
    __shared__ unsigned s_todo;
    __shared__ int s_r, s_nf;
    __shared__ uint32_t s_rep;
    __shared__ unsigned long long s_pos;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t t0 = (int64_t)blockIdx.x * kMedTask;
    if (t0 >= p.n_med) return;  // uniform over the CTA
    if (warp == 0) {
        const int nt = (int)min((int64_t)kMedTask, p.n_med - t0);
        bool take = false;
        if (lane < nt) {
            const int32_t v = p.med_v[t0 + lane];
            const int64_t rs = p.row[v], re = p.row[(int64_t)v + 1];
            s_v[lane] = v;
            s_rs[lane] = rs;
            s_re[lane] = re;
            s_own[lane] = own_of(p, v);
            take = re - rs > dlo && re - rs <= dhi && vertex_refines(p, v);
        }
        const unsigned todo = __ballot_sync(kFull, take);
        if (lane == 0) s_todo = todo;
    }
    __syncthreads();
    unsigned todo = s_todo;
    while (todo) {
        const int j = __ffs(todo) - 1;
        todo &= todo - 1;
        const int32_t v = s_v[j], own = s_own[j];
        const int64_t rs = s_rs[j], re = s_re[j];
        const int d = (int)(re - rs);
        int c = 64;
        while (c < 2 * d) c <<= 1;
        if (c > kCap) {  // cannot happen: dhi <= kCap / 2
            if (tid == 0) set_error(p.ctr, kErrStage);
            continue;
        }
        const uint32_t cmask = (uint32_t)c - 1u;
        for (int i = tid; i < c; i += kThreads) s_set[i] = kEmptyPair;
        __syncthreads();

        uint64_t acc = 0;
        uint32_t cnt = 0;
        int32_t w[U], l[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t e = rs + u * kThreads + tid;
            w[u] = 0;
            l[u] = 0;
            if (e < re) {
                w[u] = __ldcs(p.col + e);
                l[u] = p.lab ? __ldcs(p.lab + e) : 0;
            }
        }
        for (int64_t e0 = rs; e0 < re; e0 += kThreads * U) {
            int32_t b[U];
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (e0 + u * kThreads + tid < re) b[u] = gather_block(p, w[u]);
            int32_t w2[U], l2[U];
            const int64_t e1 = e0 + kThreads * U;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t e = e1 + u * kThreads + tid;
                w2[u] = 0;
                l2[u] = 0;
                if (e < re) {
                    w2[u] = __ldcs(p.col + e);
                    l2[u] = p.lab ? __ldcs(p.lab + e) : 0;
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (e0 + u * kThreads + tid >= re) continue;
                const uint64_t pr = pack_pair(l[u], (uint32_t)w[u], b[u]);
                const uint64_t pm = pair_mix(pr);
                uint32_t slot = med_slot(pm, cmask);
                while (true) {
                    const unsigned long long old = atomicCAS(reinterpret_cast<unsigned long long*>(s_set + slot),
                                                             (unsigned long long)kEmptyPair, (unsigned long long)pr);
                    if (old == (unsigned long long)kEmptyPair) {
                        acc += pm;
                        ++cnt;
                        break;
                    }
                    if (old == (unsigned long long)pr) break;
                    slot = (slot + 1) & cmask;
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                w[u] = w2[u];
                l[u] = l2[u];
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            acc += __shfl_xor_sync(kFull, (unsigned long long)acc, o);
            cnt += __shfl_xor_sync(kFull, cnt, o);
        }
        if (lane == 0) {
            s_acc[warp] = acc;
            s_cnt[warp] = cnt;
        }
        __syncthreads();
        acc = 0;
        cnt = 0;
#pragma unroll
        for (int i = 0; i < W; ++i) {
            acc += s_acc[i];
            cnt += s_cnt[i];
        }

        // find or insert, with the full signature compare on every tag match
        const uint64_t h = vertex_hash(own, cnt, acc, p.hash_mode);
        const uint32_t hi = table_hi(h, p.epoch);
        if (tid == 0) s_pos = h & p.mask;
        while (true) {
            if (tid == 0) {
                uint64_t pos = s_pos;
                uint32_t rep = 0;
                s_r = probe_table(p, &pos, hi, (uint32_t)v, &rep);
                s_pos = pos;
                s_rep = rep;
                s_nf = 0;
            }
            __syncthreads();
            const int r = s_r;
            if (r == 0) break;
            if (r == 2) {
                if (tid == 0) set_error(p.ctr, kErrTableFull);
                break;
            }
            const uint32_t rep = s_rep;
            bool ok = same_graph(p, rep, v) && own_of(p, rep) == own;
            if (ok) {
                for (int i = tid; i < c / 32; i += kThreads) s_mark[i] = 0u;
                __syncthreads();
                const int64_t rb = p.row[rep], rend = p.row[(int64_t)rep + 1];
                int nf = 0;
                for (int64_t e0 = rb; e0 < rend; e0 += kThreads) {
                    const int64_t e = e0 + tid;
                    bool found = true;
                    if (e < rend) {
                        const int32_t ww = __ldg(p.col + e);
                        const int32_t ll = p.lab ? __ldg(p.lab + e) : 0;
                        const uint64_t pr = pack_pair(ll, (uint32_t)ww, gather_block(p, ww));
                        uint32_t slot = med_slot(pair_mix(pr), cmask);
                        found = false;
                        while (true) {
                            const uint64_t cur = s_set[slot];
                            if (cur == kEmptyPair) break;
                            if (cur == pr) {
                                const uint32_t bit = 1u << (slot & 31);
                                const uint32_t old = atomicOr(&s_mark[slot >> 5], bit);
                                if (!(old & bit)) ++nf;
                                found = true;
                                break;
                            }
                            slot = (slot + 1) & cmask;
                        }
                    }
                    if (!__syncthreads_and(found)) {
                        ok = false;
                        break;
                    }
                }
                if (nf) atomicAdd(&s_nf, nf);
                __syncthreads();
                ok = ok && (uint32_t)s_nf == cnt;
            }
            if (ok) {
                if (tid == 0) join_slot(p, s_pos, hi, (uint32_t)v);
                break;
            }
            if (tid == 0) s_pos = (s_pos + 1) & p.mask;
            __syncthreads();
        }
        __syncthreads();  // the set is rebuilt for the next vertex
    }
}

}  // namespace

// The CTA kernel's 17.5 KB set per CTA would let the SM give nearly all of its
// L1 to shared memory (12 CTAs by registers); at 60% of the maximum carveout 7
// CTAs run and the rest stays L1, which the kernel's many outstanding random
// loads need (2e9-edge graph: 8.2 -> 6.5 ms per round for the medium class).
void set_medium_kernel_attributes() {
    cudaFuncSetAttribute(medium_cta_kernel<2 * kMaxHubThreshold, kMedCtaThreads>,
                         cudaFuncAttributePreferredSharedMemoryCarveout, 60);
}

void launch_medium_round(const RoundParams& p, cudaStream_t s) {
    if (p.n_med <= 0) return;
    const int64_t tasks = (p.n_med + kMedTask - 1) / kMedTask;
    const int32_t thr = std::min(p.hub_threshold, (int32_t)kMaxHubThreshold);
    const int32_t split = std::min(std::max(p.med_split, 1), (int32_t)kMedSplit);
    if (p.small_max < split) {
        constexpr int kW = 4;
        medium_round_kernel<2 * kMedSplit, kW>
            <<<(unsigned)((tasks + kW - 1) / kW), kW * 32, 0, s>>>(p, p.small_max, std::min(thr, split));
    }
    if (thr > split)
        medium_cta_kernel<2 * kMaxHubThreshold, kMedCtaThreads>
            <<<(unsigned)tasks, kMedCtaThreads, 0, s>>>(p, std::max(p.small_max, split), thr);
}

}  // namespace kb
