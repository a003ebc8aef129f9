// walk.cuh -- warp-cooperative neighbour walk over the implicit hierarchy.
//
// The paper's GPU loops avoid per-thread neighbour buffers by walking the tree
// and interacting in chunks of N_chunk = 32 neighbours (Sec. 2.4, Sec. 3).
// Here one warp owns a group of up to 32 Morton-consecutive particles and
// walks the hierarchy once for the whole group: each step pops up to four
// nodes and tests their 32 children in parallel (one child per lane) against
// the group's bounding box; accepted leaves are queued and turned into tiles
// of 32 candidate particles, which the caller culls, stages in shared memory
// and interacts in batches of 32 -- the warp-wide descendant of N_chunk.
#pragma once

#include "common.cuh"

namespace sph {

constexpr int kStack = 384;     // see the bound below
constexpr int kStackPop4 = 192; // pop four nodes per step only while sp <= this
constexpr int kLeafQ = 64;      // ring buffer; a step adds <= 32 leaves to <= 3 pending

// Stack bound: a pop-4 step starts from sp <= 192 and ends at sp <= 220. In
// the pop-1 regime the entries above that base form a depth-first stack of at
// most 7 pending siblings per level below the base entry, so sp stays below
// 220 + 8 * kMaxLev = 316 < kStack.

// Group bounding box (absolute integer coordinates; a Morton-contiguous run of
// one box never wraps), its centre R and half extents E in box units.
struct GroupBox {
    uint32_t lo[3], hi[3], R[3];
    float E[3];
    float Emax;
};

__device__ __forceinline__ void group_box(uint4 X, bool valid, double s, GroupBox& g) {
    uint32_t v[3] = {X.x, X.y, X.z};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        g.lo[a] = warp_min(valid ? v[a] : 0xffffffffu);
        g.hi[a] = warp_max(valid ? v[a] : 0u);
        uint32_t ext = g.hi[a] - g.lo[a];
        g.R[a] = g.lo[a] + (ext >> 1);
        g.E[a] = (float)((double)((ext >> 1) + 2u) * s);
    }
    g.Emax = fmaxf(g.E[0], fmaxf(g.E[1], g.E[2]));
}

// Node test: periodic gap between the group box and a node box below radius
// Rint (integer units, already padded by the caller).
__device__ __forceinline__ bool node_near(const GroupBox& g, uint4 nlo, uint4 nhi, float Rint) {
    float gx = periodic_gap(g.lo[0], g.hi[0], nlo.x, nhi.x);
    float gy = periodic_gap(g.lo[1], g.hi[1], nlo.y, nhi.y);
    float gz = periodic_gap(g.lo[2], g.hi[2], nlo.z, nhi.z);
    return gx * gx + gy * gy + gz * gz < Rint * Rint;
}

// Walk the hierarchy of box B for one warp. `test(level, global_node)` is the
// per-lane child test; `tile(p)` is called by all lanes with one candidate
// particle per lane (sorted index, or -1), up to four leaves per call.
template <class Test, class Tile>
__device__ __forceinline__ void walk_box(const BoxDesc& B, int* stack, int* leafq, Test&& test,
                                         Tile&& tile) {
    const unsigned lane = lane_id();
    const unsigned lt = (1u << lane) - 1u;
    int sp = 0, qh = 0, qt = 0;
    const int nlev = B.nlev;
    if (nlev == 1) {
        if (lane == 0) leafq[0] = (int)B.off;
        qt = 1;
    } else {
        if (lane == 0) stack[0] = (nlev - 1) << 27;
        sp = 1;
    }
    __syncwarp();
    const long long pend = B.off + B.n;
    while (sp > 0 || qt > qh) {
        if (sp > 0) {
            int npop = sp <= kStackPop4 ? min(sp, 4) : 1;
            int slot = (int)(lane >> 3), c = (int)(lane & 7u);
            int enc = slot < npop ? stack[sp - 1 - slot] : 0;
            __syncwarp();
            sp -= npop;
            int lev = enc >> 27, t = enc & ((1 << 27) - 1);
            int cl = lev - 1, ct = t * kFan + c;
            bool ok = slot < npop && cl >= 0 && ct < B.lvl_n[max(cl, 0)];
            bool pass = ok && test(cl, B.lvl_off[cl] + ct);
            bool isleaf = pass && cl == 0;
            bool isint = pass && cl > 0;
            unsigned ml = __ballot_sync(0xffffffffu, isleaf);
            unsigned mi = __ballot_sync(0xffffffffu, isint);
            if (isleaf) leafq[(qt + __popc(ml & lt)) & (kLeafQ - 1)] = (int)(B.off + (long long)ct * kLeaf);
            if (isint) stack[sp + __popc(mi & lt)] = (cl << 27) | ct;
            qt += __popc(ml);
            sp += __popc(mi);
            __syncwarp();
        }
        while (qt - qh >= 4 || (sp == 0 && qt > qh)) {
            int nt = min(qt - qh, 4);
            int slot = (int)(lane >> 3), c = (int)(lane & 7u);
            int p = -1;
            if (slot < nt) {
                int p0 = leafq[(qh + slot) & (kLeafQ - 1)];
                if ((long long)p0 + c < pend) p = p0 + c;
            }
            __syncwarp();
            qh += nt;
            tile(p);
        }
    }
}

}  // namespace sph
