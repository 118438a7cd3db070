// Warp kernel for the vertices with at most 32 edges in the processed
// direction (the large majority of vertices in power-law graphs), and for
// level 0 (no edges; the key is the vertex label or a starting partition).
//
// One warp packs consecutive small vertices into its 32 lanes, one edge per
// lane, so loads of neighbour ids and labels stay coalesced.  Everything after
// the loads stays in registers:
//   * duplicate pairs of a vertex (set semantics, Def. "signature") are found
//     with two __match_any_sync calls, on the pair and on the owning vertex;
//   * per-vertex counts and pair-mix sums come from one warp scan;
//   * the full signature compare against a table representative (which is
//     itself a small vertex: larger ones enter the table after this kernel)
//     runs on every lane at once: each lane re-derives its representative's
//     pairs and looks each up among its own vertex's pairs, which the warp
//     parks in a 256-byte shared buffer; equality needs every pair of each
//     side found on the other.
// No block-level barriers: occupancy hides the latency of the gather, the
// table probes and the compares.
#include <cuda_runtime.h>

#include "kb_device.cuh"
#include "kb_internal.cuh"

namespace kb {
namespace {

constexpr int kSmallThreads = 256;

__device__ __forceinline__ uint64_t shfl64(uint64_t x, int src) {
    return __shfl_sync(kFull, (unsigned long long)x, src);
}

template <bool kLevel0>
__global__ void __launch_bounds__(kSmallThreads) small_round_kernel(const RoundParams p) {
    __shared__ uint64_t s_pairs[kSmallThreads];
    const int lane = threadIdx.x & 31;
    uint64_t* wpairs = s_pairs + (threadIdx.x & ~31);
    const int64_t warp = ((int64_t)blockIdx.x * kSmallThreads + threadIdx.x) >> 5;
    const int64_t vb = warp * p.warp_verts;
    if (vb >= p.n) return;
    const int64_t ve = min(p.n, vb + p.warp_verts);

    for (int64_t v0 = vb; v0 < ve;) {
        const int nvw = (int)min((int64_t)32, ve - v0);
        const int64_t v = v0 + lane;
        int cd = 0;
        bool small = false;
        int64_t a = 0;
        int32_t own = 0;
        bool l0 = kLevel0;
        if (lane < nvw && vertex_active(p, v)) {
            if (!kLevel0 && vertex_level0(p, v)) {
                l0 = true;
                own = p.vlab ? p.vlab[v] : 0;
                small = true;
            } else if (kLevel0) {
                own = p.prev ? p.prev[v] : 0;
                small = true;
            } else {
                own = p.prev ? p.prev[v] : 0;
                a = p.row[v];
                const int64_t d = p.row[v + 1] - a;
                small = d <= p.small_max;
                cd = small ? (int)d : 0;
            }
        }
        // pack whole vertices while their edges fit in 32 lanes
        int incl = cd;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
        }
        const unsigned fit = __ballot_sync(kFull, lane < nvw && incl <= 32);
        const int nfit = __popc(fit);  // incl is non-decreasing, so the fitting lanes are 0..nfit-1
        const int E = __shfl_sync(kFull, incl, nfit - 1);
        const int start = incl - cd;

        uint64_t pr = 0;
        int j = 0;
        uint64_t c = 0;
        uint32_t cu = 0;
        if (!kLevel0) {
            const bool owns = lane < nfit && cd > 0;
            const unsigned heads = __reduce_or_sync(kFull, owns ? (1u << start) : 0u);
            const unsigned has_e = __ballot_sync(kFull, owns);
            if (lane < E) {
                const unsigned upto = lane == 31 ? kFull : ((2u << lane) - 1u);
                j = (int)__fns(has_e, 0, __popc(heads & upto));
            }
            const int64_t aj = __shfl_sync(kFull, (long long)a, j);
            const int sj = __shfl_sync(kFull, start, j);
            if (lane < E) {
                const int64_t e = aj + (lane - sj);
                const int32_t w = __ldcs(p.col + e);
                const int32_t l = p.lab ? __ldcs(p.lab + e) : 0;
                pr = pack_pair(l, (uint32_t)w, __ldg(p.prev + (w & 0x7fffffff)));
                const unsigned act = E == 32 ? kFull : ((1u << E) - 1u);
                const unsigned m = __match_any_sync(act, (unsigned long long)pr) & __match_any_sync(act, (unsigned)j);
                if (__ffs(m) - 1 == lane) {
                    c = pair_mix(pr);
                    cu = 1;
                }
            }
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint64_t c2 = shfl64(c, lane >= o ? lane - o : lane);
                const uint32_t u2 = __shfl_sync(kFull, cu, lane >= o ? lane - o : lane);
                if (lane >= o) {
                    c += c2;
                    cu += u2;
                }
            }
        }
        const int src_end = max(start + cd - 1, 0), src_pre = max(start - 1, 0);
        const uint64_t c_end = shfl64(c, src_end), c_pre = shfl64(c, src_pre);
        const uint32_t u_end = __shfl_sync(kFull, cu, src_end), u_pre = __shfl_sync(kFull, cu, src_pre);
        uint64_t acc = 0;
        uint32_t cnt = 0;
        if (cd > 0) {
            acc = c_end - (start > 0 ? c_pre : 0ull);
            cnt = u_end - (start > 0 ? u_pre : 0u);
        }

        bool pending = lane < nfit && small;
        uint64_t pos = 0;
        uint32_t hi = 0, rep = 0;
        if (pending) {
            if (!l0 && cd == 0) {
                join_empty(p, own, (uint32_t)v);
                pending = false;
            } else {
                // at level 0 of a multi-graph run the key is (graph, label)
                const uint32_t c2 = (l0 && batched(p)) ? (uint32_t)p.vgraph[v] : cnt;
                const uint64_t h = vertex_hash(own, c2, acc, p.hash_mode);
                pos = h & p.mask;
                hi = table_hi(h, p.epoch);
            }
        }
        if (!kLevel0) {
            __syncwarp();
            wpairs[lane] = pr;  // lanes >= E hold unused values
            __syncwarp();
        }
        const unsigned vmask = cd >= 32 ? kFull : ((1u << cd) - 1u);
        while (__any_sync(kFull, pending)) {
            if (!pending) continue;
            const int r = probe_table(p, &pos, hi, (uint32_t)v, &rep);
            if (r == 0) {
                pending = false;
                continue;
            }
            if (r == 2) {
                set_error(p.ctr, kErrTableFull);
                pending = false;
                continue;
            }
            // full signature compare with the representative, on this lane
            bool eq = same_graph(p, rep, v);
            if (eq) {
                const int32_t* keys = (l0 && !kLevel0) ? p.vlab : p.prev;
                eq = (keys ? __ldg(keys + rep) : 0) == own;
            }
            if (!l0 && eq) {
                const int64_t rb = p.row[rep], re = p.row[(int64_t)rep + 1];
                unsigned vfound = 0;
                for (int64_t e0 = rb; e0 < re && eq; e0 += 4) {
                    uint64_t x[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        x[u] = 0;
                        if (e0 + u < re) {
                            const int32_t w = __ldg(p.col + e0 + u);
                            const int32_t l = p.lab ? __ldg(p.lab + e0 + u) : 0;
                            x[u] = pack_pair(l, (uint32_t)w, __ldg(p.prev + (w & 0x7fffffff)));
                        }
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        if (e0 + u >= re) break;
                        bool found = false;
                        for (int t = 0; t < cd; ++t) {
                            if (wpairs[start + t] == x[u]) {
                                vfound |= 1u << t;
                                found = true;
                            }
                        }
                        if (!found) eq = false;
                    }
                }
                if (vfound != vmask) eq = false;
            }
            if (eq) {
                join_slot(p, pos, hi, (uint32_t)v);
                pending = false;
            } else {
                pos = (pos + 1) & p.mask;
            }
        }
        v0 += nfit;
    }
}

}  // namespace

void launch_small_round(const RoundParams& p, bool level0, cudaStream_t s) {
    if (p.n <= 0) return;
    const int64_t wv = p.warp_verts > 0 ? p.warp_verts : kDefaultWarpVerts;
    const int64_t warps = (p.n + wv - 1) / wv;
    const int64_t blocks = (warps * 32 + kSmallThreads - 1) / kSmallThreads;
    RoundParams q = p;
    q.warp_verts = (int32_t)wv;
    if (level0)
        small_round_kernel<true><<<(unsigned)blocks, kSmallThreads, 0, s>>>(q);
    else
        small_round_kernel<false><<<(unsigned)blocks, kSmallThreads, 0, s>>>(q);
}

}  // namespace kb
