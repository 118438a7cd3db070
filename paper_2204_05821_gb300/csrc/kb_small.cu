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
//
// Hot keys.  In power-law graphs millions of vertices share a key (all
// edgeless vertices with the same label, all vertices with one edge to the
// same hub block), and a global atomic per vertex on the same word serialises.
// So joins are aggregated per CTA: a shared map keyed by the table slot (or by
// the own block of an empty signature) keeps the smallest joining vertex, and
// the CTA applies one global atomicMin per key when it finishes.  New-block
// owners toggle their minimum bits once per window (one atomicXor per bitmap
// word).  The XOR toggling of block minima is order independent, so the
// aggregation leaves the result unchanged.
#include <cuda_runtime.h>

#include "kb_device.cuh"
#include "kb_internal.cuh"

namespace kb {
namespace {

constexpr int kSmallThreads = 256;
#ifndef KB_SMALL_MIN_BLOCKS
#define KB_SMALL_MIN_BLOCKS 6  // caps registers at 40: 48 warps per SM (a few bytes spill)
#endif
constexpr int kSmallWarps = kSmallThreads / 32;
// Joins a CTA can aggregate (1 x its vertices at the default task size; a
// join that finds no room goes to global memory at once).  The map is kept
// small on purpose: shared memory comes out of the SM's L1, and the L1 also
// tracks the kernel's many outstanding random loads.
#ifndef KB_MAP_CAP
#define KB_MAP_CAP 1024
#endif
constexpr int kMapCap = KB_MAP_CAP;
constexpr uint64_t kMapEmpty = ~0ull;
constexpr uint64_t kEmptyKeyBit = 1ull << 63;  // map key of an empty-signature join: bit 63 | own

__device__ __forceinline__ uint64_t shfl64(uint64_t x, int src) {
    return __shfl_sync(kFull, (unsigned long long)x, src);
}

struct JoinMap {
    uint64_t key[kMapCap];
    uint32_t hi[kMapCap];
    uint32_t vmin[kMapCap];
};

// Record that v joins `key`; false when the map has no room (the caller then
// joins globally right away).
__device__ __forceinline__ bool map_join(JoinMap& M, uint64_t key, uint32_t hi, uint32_t v) {
    uint32_t slot = (uint32_t)(mix64(key) >> 32) & (kMapCap - 1);
    for (int t = 0; t < 32; ++t) {
        uint64_t cur = M.key[slot];
        if (cur == kMapEmpty) {
            cur = atomicCAS(reinterpret_cast<unsigned long long*>(&M.key[slot]), (unsigned long long)kMapEmpty,
                            (unsigned long long)key);
            if (cur == kMapEmpty) {
                M.hi[slot] = hi;
                cur = key;
            }
        }
        if (cur == key) {
            atomicMin(&M.vmin[slot], v);
            return true;
        }
        slot = (slot + 1) & (kMapCap - 1);
    }
    return false;
}

// Global atomicMin of a CTA's smallest joining vertex, with minimum toggles.
// A block's minimum only decreases during a round, so a read that finds it at
// or below v makes the atomic (and its toggles) a no-op, and it is skipped:
// hot keys would otherwise take one serialised atomic per CTA.
__device__ __forceinline__ void flush_join(const RoundParams& p, uint64_t key, uint32_t hi, uint32_t v) {
    if (key & kEmptyKeyBit) {
        const int32_t own = (int32_t)(uint32_t)key;
        const uint64_t want = ((uint64_t)p.ehigh << 32) | v;
        const uint64_t seen = volatile_load(&p.emin[own]);
        if ((uint32_t)(seen >> 32) == p.ehigh && (uint32_t)seen <= v) return;  // minima only decrease
        const uint64_t old = atomicMin(reinterpret_cast<unsigned long long*>(&p.emin[own]), (unsigned long long)want);
        if ((uint32_t)(old >> 32) != p.ehigh) {
            toggle_min(p.bitmap, v);
        } else if (v < (uint32_t)old) {
            toggle_min(p.bitmap, v);
            toggle_min(p.bitmap, (uint32_t)old);
        }
    } else {
        const uint64_t want = ((uint64_t)hi << 32) | v;
        const uint64_t seen = volatile_load(&p.table[key]);
        if ((uint32_t)(seen >> 32) == hi && (uint32_t)seen <= v) return;  // minima only decrease
        const uint64_t old = atomicMin(reinterpret_cast<unsigned long long*>(&p.table[key]), (unsigned long long)want);
        if (v < (uint32_t)old) {
            toggle_min(p.bitmap, v);
            toggle_min(p.bitmap, (uint32_t)old);
        }
    }
}

template <bool kLevel0, bool kCompact>
__global__ void __launch_bounds__(kSmallThreads, KB_SMALL_MIN_BLOCKS) small_round_kernel(const RoundParams p) {
    __shared__ uint64_t s_pairs[kSmallThreads];
    __shared__ JoinMap M;
    __shared__ unsigned long long s_l0[kLevel0 ? 256 : 1];
    const int lane = threadIdx.x & 31;
    uint64_t* wpairs = s_pairs + (threadIdx.x & ~31);
    for (int i = threadIdx.x; i < kMapCap; i += kSmallThreads) {
        M.key[i] = kMapEmpty;
        M.vmin[i] = 0xffffffffu;
    }
    if (kLevel0)
        for (int i = threadIdx.x; i < 256; i += kSmallThreads) s_l0[i] = ~0ull;
    __syncthreads();

    const int64_t cta_base = (int64_t)blockIdx.x * kSmallWarps * p.warp_verts;
    const int64_t vb = cta_base + (int64_t)(threadIdx.x >> 5) * p.warp_verts;
    const int64_t ve = min(p.n, vb + p.warp_verts);

    // A window holds up to 32 vertices of the task, one per lane: consecutive
    // ones, or (kCompact, when many vertices are frozen) the next ones that
    // refine this round among the next kLook, so that frozen and inactive
    // vertices take no lane.  The next window is picked, and its row offsets
    // and own blocks loaded, while the current one works (its start is known
    // once the current one is packed).
    constexpr int kLook = kCompact ? 128 : 32;
    const int span = (int)(ve - vb);  // task vertices (at most 65536)
    // next window: this lane's vertex as an offset from vb (-1: none), and
    // packed: vertices picked (bits 0..5), more than 32 candidates in the span
    // (bit 6), offset of the first vertex after the span (bits 7..)
    int pf_off = -1;
    int pf_win = 0;
    int64_t pf_a = 0;
    int32_t pf_d = 0, pf_own = 0;
    auto pick = [&](int c) {
        if (!kCompact) {  // the next 32 vertices
            pf_off = c + lane < span ? c + lane : -1;
        } else {  // the next 32 that refine, among the next kLook
            unsigned bk[kLook / 32];
#pragma unroll
            for (int k = 0; k < kLook / 32; ++k) {
                const int u = c + 32 * k + lane;
                bk[k] = __ballot_sync(kFull, u < span && vertex_active(p, vb + u) && !vertex_frozen(p, vb + u));
            }
            int rem = lane, total = 0;
            pf_off = -1;
#pragma unroll
            for (int k = 0; k < kLook / 32; ++k) {
                const int ck = __popc(bk[k]);
                if (pf_off < 0 && rem < ck) pf_off = c + 32 * k + __fns(bk[k], 0, rem + 1);
                if (pf_off < 0) rem -= ck;
                total += ck;
            }
            pf_win = min(total, 32) | (total > 32 ? 64 : 0) | (min(span, c + kLook) << 7);
        }
        if (pf_off >= 0) {
            const int64_t pv = vb + pf_off;
            pf_own = (!kLevel0 && p.own_key) ? p.own_key[pv] : (p.prev ? p.prev[pv] : 0);
            if (!kLevel0) {
                pf_a = p.row[pv];
                pf_d = (int32_t)min(p.row[pv + 1] - pf_a, (int64_t)0x7fffffff);
            }
        }
    };
    pick(0);
    for (int wc = 0; wc < span;) {
        const int64_t v0 = vb + wc;  // first vertex of a window of consecutive vertices (not kCompact)
        const int nvw = kCompact ? pf_win & 63 : min(span - wc, 32);
        const int64_t v = kCompact ? vb + pf_off : v0 + lane;  // meaningful for lanes < nvw
        if (kCompact && nvw == 0) {  // nothing to key in this span
            wc = pf_win >> 7;
            if (wc < span) pick(wc);
            continue;
        }
        const bool more = (pf_win & 64) != 0;
        const int span_end = pf_win >> 7;
        int cd = 0;
        bool small = false;
        int64_t a = 0;
        int32_t own = 0;
        bool l0 = kLevel0;
        const int64_t cur_a = pf_a;
        const int32_t cur_d = pf_d, cur_own = pf_own;
        if (lane < nvw && (kCompact || (vertex_active(p, v) && !vertex_frozen(p, v)))) {
            if (!kLevel0 && vertex_level0(p, v)) {
                l0 = true;
                own = p.vlab ? p.vlab[v] : 0;
                small = true;
            } else if (kLevel0) {
                own = cur_own;
                small = true;
            } else {
                own = cur_own;
                a = cur_a;
                small = cur_d <= p.small_max;
                cd = small ? cur_d : 0;
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
        // the next window starts at the first vertex that did not fit, else
        // after the last one picked, else after the span
        if (!kCompact) {
            wc += nfit;
        } else {
            const int o_nf = __shfl_sync(kFull, pf_off, nfit < 32 ? nfit : 31);
            const int o_last = __shfl_sync(kFull, pf_off, 31);
            wc = nfit < nvw ? o_nf : (more ? o_last + 1 : span_end);
        }
        if (wc < span) pick(wc);

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
                pr = pack_pair(l, (uint32_t)w, gather_block(p, w));
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
        bool inserted = false;
        uint64_t pos = 0;
        uint32_t hi = 0, rep = 0;
        if (pending) {
            if (!l0 && cd == 0) {
                // (own block, empty set): grouped by the own block exactly
                const uint64_t key = kEmptyKeyBit | (uint32_t)own;
                if (!map_join(M, key, 0u, (uint32_t)v)) flush_join(p, key, 0u, (uint32_t)v);
                p.slot_of[v] = (int32_t)(0x80000000u | (uint32_t)own);
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
        // Level 0 of one graph: the key is the label alone, so a slot that a
        // lane of this CTA found (or claimed) for a label serves later lanes
        // with the same label without a probe or a compare (a direct-mapped
        // cache of (label, slot) words).
        uint32_t l0c = 0;
        bool resolved = false;
        if (kLevel0 && !batched(p)) {
            l0c = ((uint32_t)own * 2654435761u) >> 24;
            if (pending) {
                const unsigned long long e = s_l0[l0c];
                if (e != ~0ull && (uint32_t)(e >> 32) == (uint32_t)own) {
                    pos = (uint32_t)e;
                    if (!map_join(M, pos, hi, (uint32_t)v)) flush_join(p, pos, hi, (uint32_t)v);
                    p.slot_of[v] = (int32_t)pos;
                    pending = false;
                }
            }
        }
        const unsigned vmask = cd >= 32 ? kFull : ((1u << cd) - 1u);
        while (__any_sync(kFull, pending)) {
            if (!pending) continue;
            const int r = probe_table(p, &pos, hi, (uint32_t)v, &rep, false);
            if (r == 0) {
                inserted = true;
                pending = false;
                continue;
            }
            if (r == 2) {
                set_error(p.ctr, kErrTableFull);
                pending = false;
                continue;
            }
            // full signature compare with the representative, on this lane;
            // its key and its row offsets are loaded together
            const int32_t* keys = (l0 && !kLevel0) ? p.vlab : ((!kLevel0 && p.own_key) ? p.own_key : p.prev);
            const int32_t rkey = keys ? __ldg(keys + rep) : 0;
            int64_t rb = 0, re = 0;
            if (!l0) {
                rb = p.row[rep];
                re = p.row[(int64_t)rep + 1];
            }
            bool eq = same_graph(p, rep, v) && rkey == own;
            if (!l0 && eq) {
                unsigned vfound = 0;
                for (int64_t e0 = rb; e0 < re && eq; e0 += 4) {
                    uint64_t x[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        x[u] = 0;
                        if (e0 + u < re) {
                            const int32_t w = __ldg(p.col + e0 + u);
                            const int32_t l = p.lab ? __ldg(p.lab + e0 + u) : 0;
                            x[u] = pack_pair(l, (uint32_t)w, gather_block(p, w));
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
                if (!map_join(M, pos, hi, (uint32_t)v)) flush_join(p, pos, hi, (uint32_t)v);
                p.slot_of[v] = (int32_t)pos;
                pending = false;
                resolved = true;
            } else {
                pos = (pos + 1) & p.mask;
            }
        }
        if (kLevel0 && !batched(p) && (resolved || inserted))
            s_l0[l0c] = ((unsigned long long)(uint32_t)own << 32) | (uint32_t)pos;
        // new-block owners of this window: one atomicXor per bitmap word (the
        // window's vertices lie in at most kLook / 32 + 1 words)
        if (!kCompact) {
            const uint32_t sh = (uint32_t)(v0 & 31);
            const int64_t w0 = v0 >> 5;
            const bool in0 = (v >> 5) == w0;
            const unsigned m0 = __ballot_sync(kFull, inserted && in0);
            const unsigned m1 = __ballot_sync(kFull, inserted && !in0);
            if (lane == 0) {
                if (m0) atomicXor(&p.bitmap[w0], m0 << sh);
                if (m1) atomicXor(&p.bitmap[w0 + 1], m1 >> (32 - sh));
            }
        } else {
            unsigned todo = __ballot_sync(kFull, inserted);
            while (todo) {
                const int64_t w = __shfl_sync(kFull, (long long)(v >> 5), __ffs(todo) - 1);
                const bool mine = inserted && (v >> 5) == w;
                const unsigned bits = __reduce_or_sync(kFull, mine ? 1u << (v & 31) : 0u);
                if (lane == 0) atomicXor(&p.bitmap[w], bits);
                todo &= ~__ballot_sync(kFull, mine);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kMapCap; i += kSmallThreads) {
        const uint64_t key = M.key[i];
        if (key != kMapEmpty) flush_join(p, key, M.hi[i], M.vmin[i]);
    }
}

}  // namespace

void launch_small_round(const RoundParams& p, bool level0, bool compact, cudaStream_t s) {
    if (p.n <= 0) return;
    const int64_t wv = p.warp_verts > 0 ? p.warp_verts : kDefaultWarpVerts;
    const int64_t per_cta = wv * kSmallWarps;
    const int64_t blocks = (p.n + per_cta - 1) / per_cta;
    RoundParams q = p;
    q.warp_verts = (int32_t)wv;
    if (level0)
        small_round_kernel<true, false><<<(unsigned)blocks, kSmallThreads, 0, s>>>(q);
    else if (compact)
        small_round_kernel<false, true><<<(unsigned)blocks, kSmallThreads, 0, s>>>(q);
    else
        small_round_kernel<false, false><<<(unsigned)blocks, kSmallThreads, 0, s>>>(q);
}

}  // namespace kb
