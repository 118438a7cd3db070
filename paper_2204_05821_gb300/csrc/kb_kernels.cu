// Refinement-round kernels of the GB300 k-bisimulation library.
//
// One round (paper Alg. 1, one pass of the loop; Def. "signature"):
//   1. kb_small.cu / kb_medium.cu: every non-hub vertex gathers its (direction,
//      edge label, previous block of neighbour) pairs, drops duplicates, hashes
//      (own previous block, pair set) and finds or inserts its key in the
//      block table.  A hash match is accepted only after the full signature
//      compare (the paper's implementations trust the hash; Section 4.3 notes
//      BRS is only correct while hashes do not collide).
//   2. hub_chunk_kernel / hub_final_kernel: the same for vertices with more
//      than hub_threshold edges, split over many CTAs.
//   3. renumber: the block table keeps the smallest member of every block; a
//      bitmap marks those minima, its prefix count gives every block its
//      canonical id (rank of its smallest member).
//   4. freeze (stratified single-graph rounds): blocks that cannot change in
//      the next round -- one member, or formed by a round from edgeless
//      vertices -- are skipped by steps 1-2 there and keep their minima.
#include <cuda_runtime.h>

#include "kb_device.cuh"
#include "kb_internal.cuh"

namespace kb {
namespace {

// ----------------------------------------------------------------------------
// Hub chunks: kChunk edges of one hub per CTA.  Chunk-local dedup in shared
// memory, then the chunk's distinct pairs go into the hub's global set; pairs
// new to the hub (the CAS that placed them found the slot empty) are counted
// and summed into its hash.
// ----------------------------------------------------------------------------
template <int kChunk>
__global__ void __launch_bounds__(kHubThreads) hub_chunk_kernel(const RoundParams p) {
    constexpr int kHubSetCap = 2 * kChunk;  // the chunk's shared dedup set
    __shared__ uint64_t s_pair[kChunk];
    __shared__ uint64_t s_new[kChunk];
    __shared__ uint32_t s_set[kHubSetCap];
    __shared__ int s_nuniq, s_nnew;
    __shared__ uint64_t s_accsum;

    const int tid = threadIdx.x;
    const int64_t c = blockIdx.x;
    // every thread reads the chunk's hub and packed extent (one broadcast word each)
    const int h = p.chunk_hub[c];
    const uint64_t ext = p.chunk_ext[c];
    const int64_t e0 = (int64_t)(ext >> 16);
    const int E = (int)(ext & 0xffffu);
    if ((batched(p) || p.vmask || p.frozen) && !vertex_refines(p, p.hub_v[h])) return;  // uniform over the CTA
    if (tid == 0) {
        s_nuniq = 0;
        s_nnew = 0;
        s_accsum = 0ull;
    }
    for (int i = tid; i < kHubSetCap; i += kHubThreads) s_set[i] = 0u;

    for (int base = 0; base < E; base += 4 * kHubThreads) {
        int32_t w[4], l[4], b[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int le = base + u * kHubThreads + tid;
            if (le < E) {
                w[u] = __ldcs(p.col + e0 + le);
                l[u] = p.lab ? __ldcs(p.lab + e0 + le) : 0;
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int le = base + u * kHubThreads + tid;
            if (le < E) b[u] = gather_block(p, w[u]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int le = base + u * kHubThreads + tid;
            if (le < E) s_pair[le] = pack_pair(l[u], (uint32_t)w[u], b[u]);
        }
    }
    __syncthreads();

    // chunk-local distinct pairs, compacted into s_new with one shared atomic per warp
    for (int base = 0; base < E; base += kHubThreads) {
        const int le = base + tid;
        bool isu = false;
        uint64_t pr = 0;
        if (le < E) {
            pr = s_pair[le];
            uint32_t slot = set_slot(pr, 0u) & (kHubSetCap - 1);
            while (true) {
                uint32_t cur = s_set[slot];
                if (cur == 0u) {
                    const uint32_t old = atomicCAS(&s_set[slot], 0u, (uint32_t)(le + 1));
                    if (old == 0u) {
                        isu = true;
                        break;
                    }
                    cur = old;
                }
                if (s_pair[(int)cur - 1] == pr) break;
                slot = (slot + 1) & (kHubSetCap - 1);
            }
        }
        const unsigned b = __ballot_sync(kFull, isu);
        int wbase = 0;
        if ((tid & 31) == 0 && b) wbase = atomicAdd(&s_nuniq, __popc(b));
        wbase = __shfl_sync(kFull, wbase, 0);
        if (isu) s_new[wbase + __popc(b & ((1u << (tid & 31)) - 1u))] = pr;
    }
    __syncthreads();

    // insert into the hub's global set
    const int nu = s_nuniq;
    uint64_t* gset = p.hub_sets + p.hub_set_off[h];
    const uint64_t gcap = (uint64_t)(p.hub_set_off[h + 1] - p.hub_set_off[h]);
    uint64_t lacc = 0;
    uint32_t lnew = 0;
    // Up to kChunk / kHubThreads pairs per thread: the first probe of every
    // pair is a CAS issued before waiting on any, then the rare collisions are
    // finished one by one.
    constexpr int kPer = kChunk / kHubThreads;
    uint64_t prs[kPer], slots[kPer], olds[kPer];
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
        const int i = tid + u * kHubThreads;
        if (i < nu) {
            prs[u] = s_new[i];
            slots[u] = hub_set_home(prs[u], gcap);
            olds[u] = atomicCAS(reinterpret_cast<unsigned long long*>(&gset[slots[u]]),
                                (unsigned long long)kEmptyPair, (unsigned long long)prs[u]);
        }
    }
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
        const int i = tid + u * kHubThreads;
        if (i >= nu) continue;
        const uint64_t pr = prs[u];
        uint64_t slot = slots[u], old = olds[u];
        bool placed = false;
        for (uint64_t t = 0; t < gcap; ++t) {
            if (old == kEmptyPair) {
                lacc += pair_mix(pr);
                ++lnew;
                placed = true;
                break;
            }
            if (old == pr) {
                placed = true;
                break;
            }
            slot = slot + 1 == gcap ? 0 : slot + 1;
            old = atomicCAS(reinterpret_cast<unsigned long long*>(&gset[slot]), (unsigned long long)kEmptyPair,
                            (unsigned long long)pr);
        }
        // sets hold 1.5 x the hub's degree: a pair that finds no slot means
        // corrupted sets (reported as a device check failure)
        if (!placed) set_error(p.ctr, kErrHubSet);
    }
    // CTA sums of the pairs new to the hub: hash and count
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lacc += __shfl_xor_sync(kFull, lacc, o);
        lnew += __shfl_xor_sync(kFull, lnew, o);
    }
    if ((tid & 31) == 0 && lnew) {
        atomicAdd(reinterpret_cast<unsigned long long*>(&s_accsum), (unsigned long long)lacc);
        atomicAdd(&s_nnew, (int)lnew);
    }
    __syncthreads();
    if (tid == 0 && s_nnew) {
        atomicAdd(&p.hub_cnt[h], (uint32_t)s_nnew);
        atomicAdd(reinterpret_cast<unsigned long long*>(&p.hub_acc[h]), (unsigned long long)s_accsum);
    }
}

__device__ __forceinline__ bool hub_set_contains(const uint64_t* gset, uint64_t gcap, uint64_t pr) {
    uint64_t slot = hub_set_home(pr, gcap);
    for (uint64_t t = 0; t < gcap; ++t) {
        const uint64_t cur = gset[slot];
        if (cur == pr) return true;
        if (cur == kEmptyPair) return false;
        slot = slot + 1 == gcap ? 0 : slot + 1;
    }
    return false;
}

// ----------------------------------------------------------------------------
// Hub keys: one CTA per hub finds or inserts the hub's key, comparing the full
// signature against the representative of any slot with a matching tag.
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(kHubFinalThreads) hub_final_kernel(const RoundParams p) {
    __shared__ uint64_t s_pair[kMaxHubThreshold];
    __shared__ uint32_t s_set[2 * kMaxHubThreshold];
    __shared__ int s_kind;
    __shared__ uint32_t s_rep;
    __shared__ uint64_t s_pos;
    __shared__ int s_ok, s_cnt_r;

    const int tid = threadIdx.x;
    const int h = blockIdx.x;
    const int32_t v = p.hub_v[h];
    if (!vertex_refines(p, v)) return;
    const int32_t own = own_of(p, v);
    const uint32_t cnt = p.hub_cnt[h];
    const uint64_t hv = vertex_hash(own, cnt, p.hub_acc[h], p.hash_mode);
    const uint32_t hi = table_hi(hv, p.epoch);
    const uint64_t* gset = p.hub_sets + p.hub_set_off[h];
    const uint64_t gcap = (uint64_t)(p.hub_set_off[h + 1] - p.hub_set_off[h]);
    if (tid == 0) s_pos = hv & p.mask;

    for (int iter = 0; iter < kProbeLimit; ++iter) {
        __syncthreads();
        if (tid == 0) {
            uint64_t pos = s_pos;
            uint32_t rep = 0;
            s_kind = probe_table(p, &pos, hi, (uint32_t)v, &rep);
            s_pos = pos;
            s_rep = rep;
            s_ok = 1;
            s_cnt_r = 0;
        }
        __syncthreads();
        const int kind = s_kind;
        if (kind == 0) return;
        if (kind == 2) {
            if (tid == 0) set_error(p.ctr, kErrTableFull);
            return;
        }
        const uint32_t r = s_rep;
        bool ok = same_graph(p, r, v) && (own_of(p, r) == own);
        const int64_t rb = p.row[r], re = p.row[r + 1];
        if (ok && re - rb > p.hub_threshold) {
            // representative is a hub: compare distinct counts, then look its
            // distinct pairs (the filled slots of its set) up in our set
            int lo = 0, hi2 = p.n_hubs;
            while (hi2 - lo > 1) { int mid = (lo + hi2) >> 1; if (p.hub_v[mid] <= (int32_t)r) lo = mid; else hi2 = mid; }
            const uint32_t cnt_r = p.hub_cnt[lo];
            ok = (cnt_r == cnt);
            if (ok) {
                // its set holds exactly its distinct pairs (and empty slots)
                const uint64_t* rset = p.hub_sets + p.hub_set_off[lo];
                const int64_t rcap = p.hub_set_off[lo + 1] - p.hub_set_off[lo];
                bool all = true;
                for (int64_t i = tid; i < rcap && all; i += kHubFinalThreads) {
                    const uint64_t pr = rset[i];
                    if (pr != kEmptyPair && !hub_set_contains(gset, gcap, pr)) all = false;
                }
                if (!all) s_ok = 0;
            } else if (tid == 0) {
                s_ok = 0;
            }
        } else if (ok) {
            // representative is a small vertex: derive its pairs, count its
            // distinct pairs in shared memory and look each up in our set
            const int d = (int)(re - rb);
            for (int i = tid; i < 2 * kMaxHubThreshold; i += kHubFinalThreads) s_set[i] = 0u;
            __syncthreads();
            bool all = true;
            for (int i = tid; i < d; i += kHubFinalThreads) {
                const int32_t w = __ldg(p.col + rb + i);
                const int32_t l = p.lab ? __ldg(p.lab + rb + i) : 0;
                const uint64_t pr = pack_pair(l, (uint32_t)w, gather_block(p, w));
                s_pair[i] = pr;
                if (!hub_set_contains(gset, gcap, pr)) all = false;
            }
            __syncthreads();
            for (int i = tid; i < d; i += kHubFinalThreads) {
                const uint64_t pr = s_pair[i];
                uint32_t slot = set_slot(pr, 0u) & (2 * kMaxHubThreshold - 1);
                while (true) {
                    uint32_t cur = s_set[slot];
                    if (cur == 0u) {
                        const uint32_t old = atomicCAS(&s_set[slot], 0u, (uint32_t)(i + 1));
                        if (old == 0u) { atomicAdd(&s_cnt_r, 1); break; }
                        cur = old;
                    }
                    if (s_pair[(int)cur - 1] == pr) break;
                    slot = (slot + 1) & (2 * kMaxHubThreshold - 1);
                }
            }
            if (!all) s_ok = 0;
            __syncthreads();
            if (tid == 0 && (uint32_t)s_cnt_r != cnt) s_ok = 0;
        } else if (tid == 0) {
            s_ok = 0;
        }
        __syncthreads();
        if (tid == 0) {
            if (s_ok) {
                join_slot(p, s_pos, hi, (uint32_t)v);
                s_kind = 0;
            } else {
                s_pos = (s_pos + 1) & p.mask;
            }
        }
        __syncthreads();
        if (s_kind == 0) return;
    }
    if (tid == 0) set_error(p.ctr, kErrTableFull);
}

// ----------------------------------------------------------------------------
// Canonical renumbering
// ----------------------------------------------------------------------------
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ uint32_t block_sum_u32(uint32_t x, uint32_t* tmp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    if (lane == 0) tmp[warp] = x;
    __syncthreads();
    uint32_t t = 0;
    if (warp == 0) {
        t = lane < (int)(blockDim.x >> 5) ? tmp[lane] : 0u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(kFull, t, o);
    }
    __syncthreads();
    return t;
}

// exclusive scan of one value per thread (blockDim = kScanThreads)
__device__ __forceinline__ uint32_t block_exscan_u32(uint32_t x, uint32_t* tmp, uint32_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) tmp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = tmp[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(kFull, w, o);
            if (lane >= o) w += y;
        }
        tmp[lane] = w;
    }
    __syncthreads();
    const uint32_t base = warp > 0 ? tmp[warp - 1] : 0u;
    *total = tmp[31];
    __syncthreads();
    return base + incl - x;
}

__global__ void __launch_bounds__(kScanThreads) popc_reduce_kernel(const uint32_t* bitmap, int64_t nw,
                                                                  uint32_t* block_sums) {
    __shared__ uint32_t tmp[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    uint32_t s = 0;
#pragma unroll
    for (int u = 0; u < kScanItems; ++u) {
        const int64_t i = base + (int64_t)u * kScanThreads + threadIdx.x;
        if (i < nw) s += __popc(bitmap[i]);
    }
    s = block_sum_u32(s, tmp);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kScanThreads) scan_block_sums_kernel(uint32_t* block_sums, int64_t nb,
                                                                      Counters* ctr) {
    __shared__ uint32_t tmp[32];
    uint32_t carry = 0;
    for (int64_t base = 0; base < nb; base += kScanThreads) {
        const int64_t i = base + threadIdx.x;
        const uint32_t x = i < nb ? block_sums[i] : 0u;
        uint32_t total;
        const uint32_t ex = block_exscan_u32(x, tmp, &total);
        if (i < nb) block_sums[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) ctr->count = (int64_t)carry;
}

// prefix[w] = set bits before word w; with rank given instead, rank[w] =
// (prefix[w], bitmap[w]), so a rank lookup is one 8-byte load.
__global__ void __launch_bounds__(kScanThreads) popc_scan_kernel(const uint32_t* bitmap, int64_t nw,
                                                                const uint32_t* block_sums, uint32_t* prefix,
                                                                uint2* rank) {
    __shared__ uint32_t tmp[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t w[kScanItems], c[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int u = 0; u < kScanItems; ++u) {
        const int64_t i = base + u;
        w[u] = i < nw ? bitmap[i] : 0u;
        c[u] = (uint32_t)__popc(w[u]);
        s += c[u];
    }
    uint32_t total;
    uint32_t ex = block_exscan_u32(s, tmp, &total) + block_sums[blockIdx.x];
#pragma unroll
    for (int u = 0; u < kScanItems; ++u) {
        const int64_t i = base + u;
        if (i < nw) {
            if (rank)
                rank[i] = make_uint2(ex, w[u]);
            else
                prefix[i] = ex;
        }
        ex += c[u];
    }
}

// Shared-block marks (RoundParams::shared) go through a small direct-mapped
// cache of the minima this CTA marked already: a block with millions of
// members (all edgeless vertices with one label) would otherwise send one
// atomic per member to a single word.
constexpr int kMarkCache = 1024;
constexpr uint32_t kNoMark = 0xffffffffu;

__global__ void __launch_bounds__(256) assign_kernel(const RoundParams p, const uint2* rank, int32_t* out) {
    __shared__ uint32_t s_mark[kMarkCache];
    if (p.shared) {
        for (int i = threadIdx.x; i < kMarkCache; i += blockDim.x) s_mark[i] = kNoMark;
        __syncthreads();
    }
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < p.n; v += stride) {
        uint32_t mn = (uint32_t)v;
        uint32_t mark = kNoMark;
        if (!vertex_active(p, v)) {
            if (!p.vmask) {  // a batched graph that stopped: its ids shift with the graphs before it
                // (batched runs never use the locality order)
                const int32_t g = p.vgraph[v];
                out[v] = (int32_t)((uint32_t)p.prev[v] - p.gbase_prev[g] + p.gbase_cur[g]);
                continue;
            }
            mn = p.kmin[p.keep_old[v]];  // incremental: the smallest kept member of its old block
            if ((int64_t)mn >= p.n) mn = (uint32_t)v;
        } else if (!((p.bitmap[v >> 5] >> (v & 31)) & 1u)) {
            const uint32_t sl = (uint32_t)p.slot_of[v];
            if (sl & 0x80000000u)
                mn = (uint32_t)p.emin[(sl & 0x7fffffffu) % (uint32_t)p.n];
            else
                mn = (uint32_t)(p.table[(uint64_t)sl & p.mask] & 0xffffffffu);
            if ((int64_t)mn >= p.n) mn = (uint32_t)v;  // only after a reported device error
            mark = mn;  // v is not the minimum: its block has another member
        }
        const uint2 rw = rank[mn >> 5];
        const int32_t b = (int32_t)(rw.x + __popc(rw.y & ((1u << (mn & 31)) - 1u)));
        out[v] = b;
        if (p.perm) p.gat[p.perm[v]] = (int32_t)mn;  // the block by its smallest member
        if (p.shared) {
            // one lane per distinct minimum in the warp, then the CTA's cache,
            // then an L2 read: an atomic on a bit already set costs far more
            // than the read (batched and incremental runs, which leave the
            // loop early above, have no shared marks)
            const unsigned grp = __match_any_sync(__activemask(), mark);
            if (mark != kNoMark && (int)(threadIdx.x & 31) == __ffs(grp) - 1) {
                const uint32_t c = (mark * 2654435761u) >> 22;
                if (s_mark[c] != mark) {
                    s_mark[c] = mark;
                    const uint32_t bit = 1u << (mark & 31);
                    if (!(__ldcg(p.shared + (mark >> 5)) & bit)) atomicOr(&p.shared[mark >> 5], bit);
                }
            }
        }
    }
}

// The round kept the block count: blocks only split, so it kept every block
// and its ids are the previous level's.  Under early stop it is the last
// round, and nothing else of it is needed.  (Apart from assign_frozen_kernel,
// whose registers bound its occupancy.)
__global__ void __launch_bounds__(256) stable_copy_kernel(const RoundParams p, int32_t* out, int64_t stable_count) {
    if (p.ctr->count != stable_count) return;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t done = 0;
    if (((reinterpret_cast<uintptr_t>(p.prev) | reinterpret_cast<uintptr_t>(out)) & 15) == 0) {
        const int64_t n4 = p.n >> 2;  // 16-byte copies while both rows allow them
        const int4* src = reinterpret_cast<const int4*>(p.prev);
        int4* dst = reinterpret_cast<int4*>(out);
        for (int64_t i = t; i < n4; i += stride) dst[i] = __ldcs(src + i);
        done = n4 << 2;
    }
    for (int64_t v = done + t; v < p.n; v += stride) out[v] = p.prev[v];
}

// Canonical ids of a stratified round with frozen blocks (RoundParams::minof;
// one graph, or several at once): assign_kernel's work with every lane of a warp on one
// bitmap word (a warp-uniform loop), so that the moved vertices (re-keyed
// vertices whose smallest block member changed: v itself or minof[v] at the
// previous level, read before minof[v] is rewritten) leave as one word per
// warp.  Frozen vertices keep minof, and their blocks keep their shared marks
// (the freeze pass carries them over), so only re-keyed vertices mark.  moved
// may be null (the starting level).
__global__ void __launch_bounds__(256) assign_frozen_kernel(const RoundParams p, const uint2* rank, int32_t* out,
                                                             uint32_t* moved, int64_t stable_count) {
    __shared__ uint32_t s_mark[kMarkCache];
    // a round that kept the block count is copied by stable_copy_kernel
    if (stable_count >= 0 && p.ctr->count == stable_count) return;
    for (int i = threadIdx.x; i < kMarkCache; i += blockDim.x) s_mark[i] = kNoMark;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < p.n; base += stride) {
        const int64_t v = base + lane;
        bool mv = false;
        uint32_t mark = kNoMark;
        if (v < p.n && !vertex_active(p, v)) {
            // a batched graph that stopped: its ids shift with the graphs before it
            const int32_t g = p.vgraph[v];
            out[v] = (int32_t)((uint32_t)p.prev[v] - p.gbase_prev[g] + p.gbase_cur[g]);
        } else if (v < p.n) {
            const bool fz = vertex_frozen(p, v);
            uint32_t mn = (uint32_t)v;
            if (!((p.bitmap[v >> 5] >> (v & 31)) & 1u)) {
                if (fz) {
                    mn = p.minof[v];  // a frozen block keeps its members and smallest member
                } else {
                    const uint32_t sl = (uint32_t)p.slot_of[v];
                    if (sl & 0x80000000u)
                        mn = (uint32_t)p.emin[(sl & 0x7fffffffu) % (uint32_t)p.n];
                    else
                        mn = (uint32_t)(p.table[(uint64_t)sl & p.mask] & 0xffffffffu);
                    mark = mn;  // v is not the minimum: its block has another member
                }
                if ((int64_t)mn >= p.n) {  // only after a reported device error
                    mn = (uint32_t)v;
                    mark = kNoMark;
                }
            }
            const uint2 rw = rank[mn >> 5];
            const int32_t b = (int32_t)(rw.x + __popc(rw.y & ((1u << (mn & 31)) - 1u)));
            out[v] = b;
            if (!fz) {
                // a graph that computed its level 0 here has no previous level
                bool new_min = true;
                if (moved && !vertex_level0(p, v)) {
                    const uint32_t pm = ((p.bitmap_prev[v >> 5] >> (v & 31)) & 1u) ? (uint32_t)v : p.minof[v];
                    mv = pm != mn;
                    new_min = mv;
                }
                // the locality order's copy of the level names every block by
                // its smallest member, which only moved vertices change (a
                // frozen block keeps its members and its smallest member)
                if (p.perm && new_min) p.gat[p.perm[v]] = (int32_t)mn;
                if (mn != (uint32_t)v) p.minof[v] = mn;
            }
        }
        // one lane per distinct minimum in the warp, then the CTA's cache,
        // then an L2 read: an atomic on a bit already set costs far more
        // than the read
        const unsigned grp = __match_any_sync(kFull, mark);
        if (mark != kNoMark && lane == __ffs(grp) - 1) {
            const uint32_t c = (mark * 2654435761u) >> 22;
            if (s_mark[c] != mark) {
                s_mark[c] = mark;
                const uint32_t bit = 1u << (mark & 31);
                if (!(__ldcg(p.shared + (mark >> 5)) & bit)) atomicOr(&p.shared[mark >> 5], bit);
            }
        }
        if (moved) {
            const unsigned w = __ballot_sync(kFull, mv);
            if (p.perm) {
                if (mv) atomicOr(&moved[p.perm[v] >> 5], 1u << (p.perm[v] & 31));
            } else if (lane == 0) {
                moved[base >> 5] = w;
            }
        }
    }
}

// Vertices of bitmap word w that are neither alone in their block nor
// edgeless (and exist).
__device__ __forceinline__ uint32_t candidate_word(const uint32_t* bitmap, const uint32_t* shared,
                                                   const uint32_t* edgeless, int64_t w, int64_t n) {
    uint32_t c = ~(bitmap[w] & ~shared[w]);
    if (edgeless) c &= ~edgeless[w];
    const int64_t first = w * 32;
    if (first + 32 > n) c &= n > first ? ((1u << (uint32_t)(n - first)) - 1u) : 0u;
    return c;
}

// A warp takes 32 consecutive bitmap words (1024 vertices) and deals their
// candidate vertices (candidate_word) to its lanes, 32 at a time: *v receives
// the vertex of rank r among them, or -1.  excl / c are this lane's word's
// exclusive candidate prefix and candidate bits.
__device__ __forceinline__ int64_t dealt_vertex(int64_t w0, uint32_t excl, uint32_t c, int r, int total) {
    int src = 0;
#pragma unroll
    for (int j = 1; j < 32; ++j)
        if ((int)__shfl_sync(kFull, excl, j) <= r) src = j;
    const uint32_t cs = __shfl_sync(kFull, c, src);
    const uint32_t es = __shfl_sync(kFull, excl, src);
    if (r >= total) return -1;
    return (w0 + src) * 32 + (int64_t)__fns(cs, 0, r - (int)es + 1);
}

// A level-i block X can split in the next round only if one of its members
// has an edge to a vertex whose smallest block member changed this round.
// For X to split, two members u, v with equal signatures over level i-1 must
// differ over level i: u has an edge (label l) into a level-i part C of some
// level-(i-1) block B, and v has its label-l edges into B only outside C, in
// another part C'.  So B split, and C or C' lacks B's smallest member: the
// members of that part changed smallest member, and u or v has an edge to
// one of them.  Mark (bit = level-i id) the blocks that hold such a member; a
// vertex with more than max_scan edges marks its block unread.  When more
// than an eighth of the vertices moved, nothing is scanned: the freeze pass
// then takes every block as marked.
__device__ __forceinline__ bool few_moved(const RoundParams& p) { return p.ctr->moved * 8 <= p.n; }

__global__ void __launch_bounds__(256) dirty_blocks_kernel(const RoundParams p, const uint32_t* edgeless,
                                                            const uint32_t* moved, const int32_t* level,
                                                            int32_t max_scan, uint32_t* mark, int64_t stable_count) {
    if (!few_moved(p)) return;
    if (stable_count >= 0 && p.ctr->count == stable_count) return;  // the last round: nothing follows
    const int lane = threadIdx.x & 31;
    const int64_t nw = (p.n >> 5) + 1;
    const int64_t w0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32;
    if (w0 >= nw) return;  // uniform over the warp
    const uint32_t c = w0 + lane < nw ? candidate_word(p.bitmap, p.shared, edgeless, w0 + lane, p.n) : 0u;
    uint32_t incl = __popc(c);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    const int total = (int)__shfl_sync(kFull, incl, 31);
    const uint32_t excl = incl - __popc(c);
    for (int t = 0; t < total; t += 32) {
        const int64_t v = dealt_vertex(w0, excl, c, t + lane, total);
        if (v < 0 || !vertex_active(p, v)) continue;
        const int64_t a = p.row[v], e_end = p.row[v + 1];
        // a graph that computed its level 0 here has no history: all dirty
        bool dirty = e_end - a > max_scan || vertex_level0(p, v);
        for (int64_t e0 = a; e0 < e_end && !dirty; e0 += 4) {
            int32_t w[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) w[u] = e0 + u < e_end ? (__ldg(p.col + e0 + u) & 0x7fffffff) : -1;
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (w[u] >= 0 && ((moved[w[u] >> 5] >> (w[u] & 31)) & 1u)) dirty = true;
        }
        if (dirty) {
            const uint32_t b = (uint32_t)level[v];
            const uint32_t mb = 1u << (b & 31);
            if (!(__ldcg(mark + (b >> 5)) & mb)) atomicOr(&mark[b >> 5], mb);
        }
    }
}

// The frozen blocks of the next round: a vertex is frozen when it is alone in
// its block (a minimum that no other vertex marked shared), edgeless
// (edgeless != null), or in a level-i block without a mark bit (mark != null
// and no more than an eighth of the vertices moved).  frozen_min holds the
// minima of frozen blocks, and the shared marks of exactly those minima are
// kept for the next round (their blocks keep their members; the others are
// marked afresh).  A warp takes 32 bitmap words and deals the candidates
// whose block it must look up to its lanes, as dirty_blocks_kernel does.
__global__ void __launch_bounds__(256) freeze_clean_kernel(int64_t n, const uint32_t* bitmap, uint32_t* shared,
                                                            const uint32_t* edgeless, const int32_t* level,
                                                            const uint32_t* mark, uint32_t* frozen,
                                                            uint32_t* frozen_min, Counters* ctr, const int32_t* vgraph,
                                                            const uint8_t* gmode, int64_t stable_count) {
    __shared__ uint32_t s_clean[8][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t nw = (n >> 5) + 1;
    const int64_t w0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + warp) * 32;
    if (w0 >= nw) return;  // uniform over the warp
    if (stable_count >= 0 && ctr->count == stable_count) return;  // the last round: nothing follows
    if (mark && ctr->moved * 8 > n) mark = nullptr;  // the dirty pass scanned nothing
    const int64_t w = w0 + lane;
    uint32_t b = 0, sh = 0, e = 0, c = 0;
    if (w < nw) {
        b = bitmap[w];
        sh = shared[w];
        e = edgeless ? edgeless[w] : 0u;
        c = mark ? candidate_word(bitmap, shared, edgeless, w, n) : 0u;
    }
    if (gmode && edgeless) {
        // serving: a graph that computed its level 0 in this step has not had
        // its edgeless blocks formed by a round yet
        for (int j = 0; j < 32; ++j) {
            const uint32_t ej = __shfl_sync(kFull, e, j);
            const int64_t vj = (w0 + j) * 32 + lane;
            const bool lvl0 = vj < n && ((ej >> lane) & 1u) && gmode[vgraph[vj]] == 1;
            const uint32_t drop = __ballot_sync(kFull, lvl0);
            if (lane == j) {
                e &= ~drop;
                // their blocks are looked up (and marked dirty) instead; without
                // marks nothing but singletons is frozen
                if (mark) c |= drop & ~(b & ~sh);
            }
        }
    }
    s_clean[warp][lane] = 0u;
    __syncwarp();
    uint32_t incl = __popc(c);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    const int total = (int)__shfl_sync(kFull, incl, 31);
    const uint32_t excl = incl - __popc(c);
    for (int t = 0; t < total; t += 32) {
        const int64_t v = dealt_vertex(w0, excl, c, t + lane, total);
        if (v < 0) continue;
        const uint32_t l = (uint32_t)level[v];
        if (!((mark[l >> 5] >> (l & 31)) & 1u)) atomicOr(&s_clean[warp][(v >> 5) - w0], 1u << (v & 31));
    }
    __syncwarp();
    if (w < nw) {
        // no bit past the last vertex survives (rank scans count whole words)
        const uint32_t valid = w * 32 + 32 <= n ? 0xffffffffu : (n > w * 32 ? (1u << (uint32_t)(n - w * 32)) - 1u : 0u);
        const uint32_t single = b & ~sh & valid;
        const uint32_t cl = s_clean[warp][lane];
        const uint32_t fz = single | (e & valid) | cl;
        const uint32_t fm = single | (b & (e | cl) & valid);
        frozen[w] = fz;
        frozen_min[w] = fm;
        shared[w] = sh & fm;
    }
}

// The vertices a round re-keys (those not in frozen; all when frozen is null)
// and their processed edges, per kernel family: small (at most small_max
// edges), medium, hub (more than thr edges).
__global__ void __launch_bounds__(256) round_work_kernel(int64_t n, const int64_t* row, const uint32_t* frozen,
                                                          int32_t small_max, int32_t thr, Counters* ctr) {
    __shared__ unsigned long long s_sum[6][8];
    unsigned long long c[6] = {0, 0, 0, 0, 0, 0};
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        if (frozen && ((frozen[v >> 5] >> (v & 31)) & 1u)) continue;
        const int64_t d = row[v + 1] - row[v];
        const int f = d <= small_max ? 0 : (d > thr ? 2 : 1);
        c[f] += 1;
        c[3 + f] += (unsigned long long)d;
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c[k] += __shfl_xor_sync(kFull, c[k], o);
        if ((threadIdx.x & 31) == 0) s_sum[k][threadIdx.x >> 5] = c[k];
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        unsigned long long t = 0;
        for (int w = 0; w < 8; ++w) t += s_sum[threadIdx.x][w];
        int64_t* dst = threadIdx.x < 3 ? &ctr->keyed_v[threadIdx.x] : &ctr->keyed_e[threadIdx.x - 3];
        if (t) atomicAdd(reinterpret_cast<unsigned long long*>(dst), t);
    }
}

// Clear bits a..b-1 of a bitmap (partial words at the ends keep their other bits).
__global__ void clear_bits_kernel(uint32_t* words, int64_t a, int64_t b) {
    const int64_t w0 = a >> 5, w1 = (b - 1) >> 5;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t w = w0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w <= w1; w += stride) {
        uint32_t keep = 0u;
        if (w == w0 && (a & 31)) keep |= (1u << (a & 31)) - 1u;
        if (w == w1 && (b & 31)) keep |= ~((1u << (b & 31)) - 1u);
        words[w] &= keep;
    }
}

// *out += set bits of words[0..nw): a few hundred atomics in all
__global__ void __launch_bounds__(256) count_bits_kernel(const uint32_t* words, int64_t nw, int64_t* out) {
    __shared__ unsigned long long s_sum[8];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long c = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nw; i += stride) c += __popc(words[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
    if ((threadIdx.x & 31) == 0) s_sum[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < 8; ++w) t += s_sum[w];
        if (t) atomicAdd(reinterpret_cast<unsigned long long*>(out), t);
    }
}

__global__ void count_refining_kernel(const int32_t* med_v, int64_t n_med, const int32_t* hub_v, int64_t n_hubs,
                                      const uint32_t* frozen, Counters* ctr) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long cm = 0, ch = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_med + n_hubs; i += stride) {
        const int32_t v = i < n_med ? med_v[i] : hub_v[i - n_med];
        const bool on = !((frozen[v >> 5] >> (v & 31)) & 1u);
        if (i < n_med) cm += on; else ch += on;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        cm += __shfl_xor_sync(kFull, cm, o);
        ch += __shfl_xor_sync(kFull, ch, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (cm) atomicAdd(reinterpret_cast<unsigned long long*>(&ctr->med_on), cm);
        if (ch) atomicAdd(reinterpret_cast<unsigned long long*>(&ctr->hub_on), ch);
    }
}

__global__ void edgeless_bits_kernel(int64_t n, const int64_t* row, uint32_t* bits) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
        const int64_t v = base + threadIdx.x;  // blockDim is a multiple of 32: a warp covers one word
        const bool e = v < n && row[v + 1] == row[v];
        const unsigned w = __ballot_sync(kFull, e);
        if ((threadIdx.x & 31) == 0 && (v >> 5) <= (n >> 5)) bits[v >> 5] = w;
    }
}

// Refill the sets of the hubs that refine this round with the empty pair, in
// tiles of kClearTile consecutive slots of all sets together (one hub's set
// can hold 10^8 slots; large tiles keep the per-tile search for the first hub
// rare).  Sets hold at least 64 slots, so a tile overlaps at most
// kClearTile / 64 + 1 hubs; they start at multiples of 4 slots, so a 16-byte
// store never straddles two sets.
constexpr int kClearTile = 65536;
constexpr int kClearHubs = kClearTile / 64 + 1;

__global__ void __launch_bounds__(256) clear_hub_sets_kernel(const RoundParams p) {
    __shared__ int s_h0;
    __shared__ int64_t s_end[kClearHubs];
    __shared__ uint8_t s_ref[kClearHubs];
    const int64_t total = p.hub_set_off[p.n_hubs];
    const int64_t t0 = (int64_t)blockIdx.x * kClearTile;
    const int64_t t1 = min(total, t0 + kClearTile);
    if (threadIdx.x == 0) {
        int lo = 0, hi = p.n_hubs - 1;  // first hub whose set ends after t0
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (p.hub_set_off[mid + 1] > t0) hi = mid; else lo = mid + 1;
        }
        s_h0 = lo;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kClearHubs; i += blockDim.x) {
        const int h = s_h0 + i;
        const bool in = h < p.n_hubs && p.hub_set_off[h] < t1;
        s_end[i] = in ? p.hub_set_off[h + 1] : t1;
        s_ref[i] = in && vertex_refines(p, p.hub_v[h]);
        if (!in) break;  // later entries keep their stale values: the walk below stops at this one
    }
    __syncthreads();
    ulonglong2* sets2 = reinterpret_cast<ulonglong2*>(p.hub_sets);
    const ulonglong2 e = make_ulonglong2(kEmptyPair, kEmptyPair);
    int j = 0;
    for (int64_t s = t0 + 2 * threadIdx.x; s < t1; s += 2 * blockDim.x) {
        while (j < kClearHubs - 1 && s_end[j] <= s) ++j;
        if (s_ref[j]) sets2[s >> 1] = e;
    }
}

// ----------------------------------------------------------------------------
// Level 0 over small labels.  A shared minimum is read before the atomicMin
// that would lower it: after a label's first members, a CTA's later (larger)
// vertices leave its minimum alone.
// ----------------------------------------------------------------------------
constexpr int kDenseThreads = 512;

__device__ __forceinline__ void see_label(uint32_t* s_min, int64_t v, int32_t l, bool& bad) {
    if ((uint32_t)l >= (uint32_t)kDenseLabels) {
        bad = true;
        return;
    }
    if ((uint32_t)v < s_min[l]) atomicMin(&s_min[l], (uint32_t)v);
}

__global__ void __launch_bounds__(kDenseThreads) dense_label_min_kernel(int64_t n, const int32_t* key, uint32_t* lmin,
                                                                         Counters* ctr) {
    __shared__ uint32_t s_min[kDenseLabels];
    for (int i = threadIdx.x; i < kDenseLabels; i += blockDim.x) s_min[i] = 0xffffffffu;
    __syncthreads();
    bool bad = false;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t done = 0;
    if ((reinterpret_cast<uintptr_t>(key) & 15) == 0) {
        const int64_t n4 = n >> 2;  // four keys per 16-byte load
        const int4* k4 = reinterpret_cast<const int4*>(key);
        for (int64_t i = t; i < n4; i += stride) {
            const int4 q = __ldcs(k4 + i);
            see_label(s_min, 4 * i, q.x, bad);
            see_label(s_min, 4 * i + 1, q.y, bad);
            see_label(s_min, 4 * i + 2, q.z, bad);
            see_label(s_min, 4 * i + 3, q.w, bad);
        }
        done = n4 << 2;
    }
    for (int64_t v = done + t; v < n; v += stride) see_label(s_min, v, __ldcs(key + v), bad);
    if (bad) atomicOr(&ctr->dense_bad, 1);
    __syncthreads();
    for (int i = threadIdx.x; i < kDenseLabels; i += blockDim.x)
        if (s_min[i] != 0xffffffffu) atomicMin(&lmin[i], s_min[i]);
}

// Every used label's smallest vertex is a block minimum.
__global__ void dense_mark_kernel(const RoundParams p, const uint32_t* lmin) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= kDenseLabels) return;
    const uint32_t m = lmin[l];
    if (m != 0xffffffffu) atomicOr(&p.bitmap[m >> 5], 1u << (m & 31));
}

// (smallest vertex, canonical id) of every used label
__global__ void dense_ids_kernel(const uint32_t* lmin, const uint2* rank, uint2* lpair) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= kDenseLabels) return;
    const uint32_t m = lmin[l];
    uint32_t id = 0u;
    if (m != 0xffffffffu) {
        const uint2 rw = rank[m >> 5];
        id = rw.x + __popc(rw.y & ((1u << (m & 31)) - 1u));
    }
    lpair[l] = make_uint2(m, id);
}

// The level, minof, the locality order's copy and the shared-block marks (a
// block is shared when a vertex other than its smallest member has its label;
// each CTA marks a label once).  The 64 KB label table stays in L1.
__global__ void __launch_bounds__(256) dense_assign_kernel(const RoundParams p, const int32_t* key,
                                                           const uint2* lpair, int32_t* out) {
    __shared__ uint32_t s_marked[kDenseLabels / 32];
    for (int i = threadIdx.x; i < kDenseLabels / 32; i += blockDim.x) s_marked[i] = 0u;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < p.n; v += stride) {
        const uint32_t l = (uint32_t)__ldcs(key + v);
        if (l >= (uint32_t)kDenseLabels) {  // the keys changed since they were checked
            set_error(p.ctr, kErrInvalid);
            continue;
        }
        const uint2 e = __ldg(lpair + l);
        const uint32_t mn = e.x;
        out[v] = (int32_t)e.y;
        if (p.perm) p.gat[p.perm[v]] = (int32_t)mn;  // the block by its smallest member
        if (mn != (uint32_t)v) {
            if (p.minof) p.minof[v] = mn;
            const uint32_t bit = 1u << (l & 31);
            if (p.shared && !(s_marked[l >> 5] & bit) && !(atomicOr(&s_marked[l >> 5], bit) & bit))
                atomicOr(&p.shared[mn >> 5], 1u << (mn & 31));
        }
    }
}

// rank of every graph's first vertex (the first vertex of a graph is always
// the smallest member of its block)
__global__ void graph_base_kernel(const RoundParams p, const uint2* rank) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g > p.n_graphs) return;
    const int64_t x = p.voff[g];
    uint32_t r;
    if (x >= p.n) {
        r = rank[(p.n >> 5) + 1].x;
    } else {
        const uint2 rw = rank[x >> 5];
        r = rw.x + __popc(rw.y & ((1u << (x & 31)) - 1u));
    }
    p.gbase_cur[g] = r;
}

__global__ void carry_minima_kernel(const RoundParams p) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < p.n; base += stride) {
        const int64_t v = base + threadIdx.x;  // blockDim is a multiple of 32: a warp covers one bitmap word
        const bool keep = v < p.n && !vertex_active(p, v) && ((p.bitmap_prev[v >> 5] >> (v & 31)) & 1u);
        const unsigned b = __ballot_sync(kFull, keep);
        if ((threadIdx.x & 31) == 0 && b) atomicOr(&p.bitmap[v >> 5], b);
    }
}

__global__ void graph_stop_kernel(const RoundParams p, int round, const int32_t* k_per_graph, const uint8_t* early,
                                  uint8_t* gactive, int32_t* glast, int32_t* sticky_err) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g == 0 && p.ctr->err) atomicOr(sticky_err, p.ctr->err);
    if (g >= p.n_graphs || !gactive[g]) return;
    const uint32_t cur = p.gbase_cur[g + 1] - p.gbase_cur[g];
    const uint32_t prv = p.gbase_prev[g + 1] - p.gbase_prev[g];
    glast[g] = round;
    if ((early[g] && cur == prv) || round >= k_per_graph[g]) gactive[g] = 0;
}

__global__ void localize_kernel(int32_t* row, int64_t n, const int32_t* vgraph, const uint32_t* gbase) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        row[v] = (int32_t)((uint32_t)row[v] - gbase[vgraph[v]]);
}

__global__ void vertex_graph_kernel(const int64_t* voff, int32_t G, int64_t n, int32_t* vgraph) {
    const int g = blockIdx.x;
    if (g >= G) return;
    for (int64_t v = voff[g] + threadIdx.x; v < voff[g + 1]; v += blockDim.x) vgraph[v] = g;
}

__global__ void write_total_kernel(uint2* rank, int64_t nw, const Counters* ctr) {
    rank[nw] = make_uint2((uint32_t)ctr->count, 0u);
}

__global__ void fill_i32_kernel(int32_t* out, int64_t n, int32_t value) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) out[i] = value;
}

__global__ void iota_i32_kernel(int32_t* out, int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) out[i] = (int32_t)i;
}

__global__ void levels_differ_kernel(const int32_t* a, const int32_t* b, int64_t n, Counters* ctr) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    bool d = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) d |= a[i] != b[i];
    if (__any_sync(kFull, d) && (threadIdx.x & 31) == 0) atomicOr(&ctr->diff, 1);
}

int grid_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152 * 64) b = 152 * 64;
    return (int)b;
}

}  // namespace

void launch_clear_round(const RoundParams& p, cudaStream_t s) {
    const size_t bytes = sizeof(uint32_t) * (size_t)((p.n >> 5) + 1);
    if (p.frozen_min)
        cudaMemcpyAsync(p.bitmap, p.frozen_min, bytes, cudaMemcpyDeviceToDevice, s);
    else
        cudaMemsetAsync(p.bitmap, 0, bytes, s);
    if (p.n_hubs > 0) {
        cudaMemsetAsync(p.hub_acc, 0, sizeof(uint64_t) * (size_t)p.n_hubs, s);
        cudaMemsetAsync(p.hub_cnt, 0, sizeof(uint32_t) * (size_t)p.n_hubs, s);
    }
}

void launch_clear_hub_sets(const RoundParams& p, int64_t total_slots, cudaStream_t s) {
    if (p.n_hubs <= 0 || total_slots <= 0) return;
    clear_hub_sets_kernel<<<(unsigned)((total_slots + kClearTile - 1) / kClearTile), 256, 0, s>>>(p);
}

void launch_dirty_blocks(const RoundParams& p, const uint32_t* edgeless, const uint32_t* moved, const int32_t* level,
                         int32_t max_scan, uint32_t* mark, cudaStream_t s, int64_t stable_count) {
    if (p.n <= 0) return;
    const int64_t warps = ((p.n >> 5) + 1 + 31) / 32;  // 32 bitmap words each
    dirty_blocks_kernel<<<(unsigned)((warps + 7) / 8), 256, 0, s>>>(p, edgeless, moved, level, max_scan, mark,
                                                                     stable_count);
}

void launch_freeze_clean(int64_t n, const uint32_t* bitmap, uint32_t* shared, const uint32_t* edgeless,
                         const int32_t* level, const uint32_t* mark, uint32_t* frozen, uint32_t* frozen_min,
                         Counters* ctr, cudaStream_t s, const int32_t* vgraph, const uint8_t* gmode,
                         int64_t stable_count) {
    if (n <= 0) return;
    const int64_t warps = ((n >> 5) + 1 + 31) / 32;  // 32 bitmap words each
    freeze_clean_kernel<<<(unsigned)((warps + 7) / 8), 256, 0, s>>>(n, bitmap, shared, edgeless, level, mark, frozen,
                                                                     frozen_min, ctr, vgraph, gmode, stable_count);
    const int64_t nw = (n >> 5) + 1;
    count_bits_kernel<<<grid_for(nw, 256) < 1216 ? grid_for(nw, 256) : 1216, 256, 0, s>>>(frozen, nw, &ctr->frozen);
}

void launch_round_work(const RoundParams& p, cudaStream_t s) {
    if (p.n <= 0) return;
    const int g = grid_for(p.n, 256) < 1216 ? grid_for(p.n, 256) : 1216;
    round_work_kernel<<<g, 256, 0, s>>>(p.n, p.row, p.frozen, p.small_max, p.hub_threshold, p.ctr);
}

void launch_count_bits(const uint32_t* words, int64_t nw, int64_t* out, cudaStream_t s) {
    if (nw <= 0) return;
    count_bits_kernel<<<grid_for(nw, 256) < 1216 ? grid_for(nw, 256) : 1216, 256, 0, s>>>(words, nw, out);
}

void launch_clear_bits(uint32_t* words, int64_t a, int64_t b, cudaStream_t s) {
    if (b <= a) return;
    const int64_t w0 = a >> 5, w1 = (b - 1) >> 5;
    clear_bits_kernel<<<grid_for(w1 - w0 + 1, 256), 256, 0, s>>>(words, a, b);
}

void launch_count_refining(const RoundParams& p, const uint32_t* frozen, Counters* ctr, cudaStream_t s) {
    const int64_t items = p.n_med + p.n_hubs;
    if (items > 0)
        count_refining_kernel<<<grid_for(items, 256), 256, 0, s>>>(p.med_v, p.n_med, p.hub_v, p.n_hubs, frozen, ctr);
}

void launch_edgeless_bits(int64_t n, const int64_t* row, uint32_t* bits, cudaStream_t s) {
    if (n > 0) edgeless_bits_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, row, bits);
}

void launch_hub_chunk(const RoundParams& p, int64_t total_chunks, cudaStream_t s) {
    if (p.n_hubs <= 0 || total_chunks <= 0) return;
    if (p.hub_chunk == 256)
        hub_chunk_kernel<256><<<(unsigned)total_chunks, kHubThreads, 0, s>>>(p);
    else if (p.hub_chunk == 1024)
        hub_chunk_kernel<1024><<<(unsigned)total_chunks, kHubThreads, 0, s>>>(p);
    else
        hub_chunk_kernel<kDefaultHubChunk><<<(unsigned)total_chunks, kHubThreads, 0, s>>>(p);
}

void launch_hub_final(const RoundParams& p, cudaStream_t s) {
    if (p.n_hubs <= 0) return;
    hub_final_kernel<<<(unsigned)p.n_hubs, kHubFinalThreads, 0, s>>>(p);
}

size_t scan_tmp_words(int64_t n_items) { return (size_t)((n_items + kScanTile - 1) / kScanTile) + 1; }

void launch_bitmap_rank(const uint32_t* bitmap, int64_t nw, uint32_t* scan_tmp, uint32_t* prefix, Counters* ctr,
                        cudaStream_t s) {
    const int64_t nb = (nw + kScanTile - 1) / kScanTile;
    popc_reduce_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(bitmap, nw, scan_tmp);
    scan_block_sums_kernel<<<1, kScanThreads, 0, s>>>(scan_tmp, nb, ctr);
    popc_scan_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(bitmap, nw, scan_tmp, prefix, nullptr);
}

void launch_renumber(const RoundParams& p, uint2* rank, uint32_t* scan_tmp, int32_t* out, cudaStream_t s,
                     int64_t stable_count) {
    const int64_t nw = (p.n >> 5) + 1;
    const int64_t nb = (nw + kScanTile - 1) / kScanTile;
    popc_reduce_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(p.bitmap, nw, scan_tmp);
    scan_block_sums_kernel<<<1, kScanThreads, 0, s>>>(scan_tmp, nb, p.ctr);
    popc_scan_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(p.bitmap, nw, scan_tmp, nullptr, rank);
    if (batched(p)) {
        // rank[nw] (one past the last word) is not written by the scan: the
        // total sits in the counters, and graph_base_kernel reads it there
        // for a graph that starts at n.
        write_total_kernel<<<1, 1, 0, s>>>(rank, nw, p.ctr);
        graph_base_kernel<<<(p.n_graphs + 1 + 255) / 256, 256, 0, s>>>(p, rank);
    }
    if (p.minof) {
        if (p.moved && p.perm) cudaMemsetAsync(p.moved, 0, sizeof(uint32_t) * (size_t)nw, s);
        if (p.n > 0 && stable_count >= 0)
            stable_copy_kernel<<<grid_for(p.n, 256) < 1216 ? grid_for(p.n, 256) : 1216, 256, 0, s>>>(p, out,
                                                                                                 stable_count);
        if (p.n > 0) assign_frozen_kernel<<<grid_for(p.n, 256), 256, 0, s>>>(p, rank, out, p.moved, stable_count);
        if (p.moved) count_bits_kernel<<<grid_for(nw, 256) < 1216 ? grid_for(nw, 256) : 1216, 256, 0, s>>>(
            p.moved, nw, &p.ctr->moved);
        return;
    }
    if (p.n > 0) assign_kernel<<<grid_for(p.n, 256), 256, 0, s>>>(p, rank, out);
}

void launch_dense_labels(int64_t n, const int32_t* key, uint32_t* lmin, Counters* ctr, cudaStream_t s) {
    if (n <= 0) return;
    int64_t grid = (n + kDenseThreads - 1) / kDenseThreads;
    if (grid > 152 * 4) grid = 152 * 4;  // each CTA flushes its label table once
    dense_label_min_kernel<<<(unsigned)grid, kDenseThreads, 0, s>>>(n, key, lmin, ctr);
}

void launch_dense_level0(const RoundParams& p, const int32_t* key, const uint32_t* lmin, uint2* lpair, uint2* rank,
                         uint32_t* scan_tmp, int32_t* out, cudaStream_t s) {
    if (p.n <= 0) return;
    const int64_t nw = (p.n >> 5) + 1;
    const int64_t nb = (nw + kScanTile - 1) / kScanTile;
    dense_mark_kernel<<<(kDenseLabels + 255) / 256, 256, 0, s>>>(p, lmin);
    popc_reduce_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(p.bitmap, nw, scan_tmp);
    scan_block_sums_kernel<<<1, kScanThreads, 0, s>>>(scan_tmp, nb, p.ctr);
    popc_scan_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(p.bitmap, nw, scan_tmp, nullptr, rank);
    dense_ids_kernel<<<(kDenseLabels + 255) / 256, 256, 0, s>>>(lmin, rank, lpair);
    dense_assign_kernel<<<grid_for(p.n, 256), 256, 0, s>>>(p, key, lpair, out);
}

void launch_carry_minima(const RoundParams& p, cudaStream_t s) {
    if (p.n <= 0) return;
    carry_minima_kernel<<<grid_for(p.n, 256), 256, 0, s>>>(p);
}

void launch_graph_stop(const RoundParams& p, int round, const int32_t* k_per_graph, const uint8_t* early,
                       uint8_t* gactive, int32_t* glast, int32_t* sticky_err, cudaStream_t s) {
    if (p.n_graphs <= 0) return;
    graph_stop_kernel<<<(p.n_graphs + 255) / 256, 256, 0, s>>>(p, round, k_per_graph, early, gactive, glast,
                                                                sticky_err);
}

void launch_localize(int32_t* row, int64_t n, const int32_t* vgraph, const uint32_t* gbase, cudaStream_t s) {
    if (n <= 0) return;
    localize_kernel<<<grid_for(n, 256), 256, 0, s>>>(row, n, vgraph, gbase);
}

void launch_vertex_graph(const int64_t* voff, int32_t G, int64_t n, int32_t* vgraph, cudaStream_t s) {
    if (G <= 0) return;
    vertex_graph_kernel<<<(unsigned)G, 256, 0, s>>>(voff, G, n, vgraph);
}

void launch_iota_i32(int32_t* out, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    iota_i32_kernel<<<grid_for(n, 256), 256, 0, s>>>(out, n);
}

void launch_levels_differ(const int32_t* a, const int32_t* b, int64_t n, Counters* ctr, cudaStream_t s) {
    if (n <= 0) return;
    levels_differ_kernel<<<grid_for(n, 256), 256, 0, s>>>(a, b, n, ctr);
}

void launch_fill_i32(int32_t* out, int64_t n, int32_t value, cudaStream_t s) {
    if (n <= 0) return;
    fill_i32_kernel<<<grid_for(n, 256), 256, 0, s>>>(out, n, value);
}

}  // namespace kb
