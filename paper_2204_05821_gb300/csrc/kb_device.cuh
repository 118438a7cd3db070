// Device helpers shared by the round kernels: the block-table protocol
// (probe, insert, join) and the bitmap of block minima.
#pragma once

#include "kb_internal.cuh"

namespace kb {

constexpr uint32_t kFull = 0xffffffffu;

__device__ __forceinline__ void set_error(Counters* c, int32_t bit) { atomicOr(&c->err, bit); }

__device__ __forceinline__ uint64_t volatile_load(const uint64_t* p) {
    return *reinterpret_cast<const volatile uint64_t*>(p);
}

// Toggle membership of v in the set of block minima.  Every vertex that ever
// becomes the minimum of its slot is toggled on once and off once when a
// smaller member replaces it, so the final bitmap holds exactly the minima,
// whatever order the toggles land in.
__device__ __forceinline__ void toggle_min(uint32_t* bitmap, uint32_t v) {
    atomicXor(&bitmap[v >> 5], 1u << (v & 31));
}

// Join slot `pos` (same epoch and tag as ours) with vertex v.
__device__ __forceinline__ void join_slot(const RoundParams& p, uint64_t pos, uint32_t hi, uint32_t v) {
    const uint64_t want = ((uint64_t)hi << 32) | v;
    const uint64_t old = atomicMin(reinterpret_cast<unsigned long long*>(&p.table[pos]),
                                   (unsigned long long)want);
    const uint32_t prev_min = (uint32_t)old;
    if (v < prev_min) {
        toggle_min(p.bitmap, v);
        toggle_min(p.bitmap, prev_min);
    }
    p.slot_of[v] = (int32_t)pos;
}

__device__ __forceinline__ bool vertex_active(const RoundParams& p, int64_t v) {
    if (p.vmask && !((p.vmask[v >> 5] >> (v & 31)) & 1u)) return false;
    return !p.gactive || p.gactive[p.vgraph[v]];
}

// A graph in level-0 mode (serving: admitted this step) keys its vertices by
// (graph, label) and ignores its edges.
__device__ __forceinline__ bool vertex_level0(const RoundParams& p, int64_t v) {
    return p.gmode && p.gmode[p.vgraph[v]] == 1;
}

// In a frozen block (RoundParams::frozen): it keeps its previous block.
__device__ __forceinline__ bool vertex_frozen(const RoundParams& p, int64_t v) {
    return p.frozen && ((__ldg(p.frozen + (v >> 5)) >> (v & 31)) & 1u);
}

// Active and refining by signature (not in level-0 mode, not frozen).
__device__ __forceinline__ bool vertex_refines(const RoundParams& p, int64_t v) {
    return vertex_active(p, v) && !vertex_level0(p, v) && !vertex_frozen(p, v);
}

// In multi-graph runs a representative must belong to the same graph.
__device__ __forceinline__ bool same_graph(const RoundParams& p, int64_t a, int64_t b) {
    return !p.vgraph || p.vgraph[a] == p.vgraph[b];
}

// A vertex without edges in the processed direction has the key (own block,
// empty set): it is grouped by its own block exactly, without hashing or a
// signature compare.  emin[own] keeps the smallest such vertex of this round;
// entries of earlier rounds carry a larger high word and lose every atomicMin.
__device__ __forceinline__ void join_empty(const RoundParams& p, int32_t own, uint32_t v) {
    const uint64_t want = ((uint64_t)p.ehigh << 32) | v;
    const uint64_t old = atomicMin(reinterpret_cast<unsigned long long*>(&p.emin[own]), (unsigned long long)want);
    if ((uint32_t)(old >> 32) != p.ehigh) {
        toggle_min(p.bitmap, v);
    } else if (v < (uint32_t)old) {
        toggle_min(p.bitmap, v);
        toggle_min(p.bitmap, (uint32_t)old);
    }
    p.slot_of[v] = (int32_t)(0x80000000u | (uint32_t)own);
}

// Probe the block table from *pos.  Returns 0 when v inserted a new key,
// 1 with *rep set when a slot with our tag was found (a signature compare
// decides), 2 when the probe limit was hit.
__device__ __forceinline__ int probe_table(const RoundParams& p, uint64_t* pos_io, uint32_t hi, uint32_t v,
                                           uint32_t* rep, bool toggle = true) {
    uint64_t pos = *pos_io;
    for (int it = 0; it < kProbeLimit; ++it) {
        uint64_t cur = volatile_load(&p.table[pos]);
        if ((uint32_t)(cur >> 56) != p.epoch) {
            const uint64_t want = ((uint64_t)hi << 32) | v;
            const uint64_t old = atomicCAS(reinterpret_cast<unsigned long long*>(&p.table[pos]),
                                           (unsigned long long)cur, (unsigned long long)want);
            if (old == cur) {
                p.slot_of[v] = (int32_t)pos;
                if (toggle) toggle_min(p.bitmap, v);
                *pos_io = pos;
                return 0;
            }
            cur = old;
            if ((uint32_t)(cur >> 56) != p.epoch) continue;
        }
        if ((uint32_t)(cur >> 32) == hi) {
            *rep = (uint32_t)cur;
            *pos_io = pos;
            return 1;
        }
        pos = (pos + 1) & p.mask;
    }
    return 2;
}


}  // namespace kb
