#pragma once
// wpp.cuh -- shared device code of the default path's density and force kernels.
//
// Member-parallel kernels (k_density_mp, k_force_mp): a warp takes a group of up
// to 8 active particles of one aligned run of sorted particles (a leaf-parent
// node by default), walks the hierarchy once for the group, and tests each
// candidate load against every member at once; the members' near or pair lists
// are then evaluated with several lanes per member. What they cannot take (groups
// of one, overflowing lists) goes to the one-particle kernels described next.
//
// One-particle kernels (k_density_wpp, k_force_wpp): work is handed out in
// chunks of up to 8 Morton-consecutive active particles.
// Those of one leaf-parent node form a group: the warp walks the hierarchy
// once for the whole group (popping up to four nodes per step, one child per
// lane) and keeps the group's leaf list in shared memory. Each particle then
// takes its own leaf list from the group's by the same node test its own walk
// would make, and is processed by the whole warp: its candidates are tested 32
// at a time, one per lane (lanes 8k..8k+7 on the eight particles of a leaf, a
// coalesced 128-byte load), and the pairs in its neighbour set are compacted
// by ballot into a warp-wide hit buffer whose pair terms are evaluated 32 at a
// time. Every step therefore runs with (nearly) all lanes busy, whatever the
// lengths of the neighbour lists of nearby particles. Per-lane FP32 partial
// sums are folded across the warp with error-free (TwoSum) transformations,
// so the result is deterministic and carries the compensation of the fold.
//
// Density keeps the pairs within 1.04 h of one walk (the "near list") across
// the h iterations (safeguarded Newton on N^(1/3), FP32) and walks again only
// when h leaves the walk radius. The neighbour predicate is the exact one,
// (double)D2 < (h 2^32/L)^2, decided in FP64 only inside a thin band around
// the FP32 radius test.
//
// Neighbour lists: a density call records each active particle's neighbour
// set at its final h. When every particle was active (or with
// SPH_PARTIAL_LISTS), the transpose adds each particle's partners with
// h_i <= r_ij < h_j, and the force pass then reads its pairs from the two lists
// (k_force_list) instead of walking; the walks serve the particles, or calls,
// the lists cannot.
#include <algorithm>

#include "internal.cuh"

namespace sph {

constexpr int kWppWarps = 4;
constexpr int kWppThreads = kWppWarps * 32;
// Register budgets: force, 8 resident blocks (32 warps, 64 registers) or 6 (24
// warps, 80 registers); density, 5 (20 warps, 96 registers: its shared memory
// holds 5 blocks per SM) or 4 (16 warps, 128 registers). The launch takes the
// one matching blocks_per_sm; the autotuner picks between them per pass.
constexpr int kWppDensityBps = 5;
constexpr int kWppDensityMaxBps = 5;
constexpr int kWppLeftBps = 6;   // the one-particle density kernel over the leftovers: 80 registers
constexpr int kWppFmBps = 6;     // the member-parallel force walk: 80 registers
constexpr int kWppForceBps = 8;
constexpr int kWppMaxBps = 16;
constexpr int kWppStack = 256;       // see the bound below
constexpr int kWppPop4 = 96;         // pop four nodes per step only while sp <= this
constexpr int kWppPop8 = 96;         // group walk: pop eight nodes per step only while sp <= this
constexpr int kWppLeaves = 128;      // leaf list per warp; a step adds <= 32
constexpr int kWppHits = 64;         // hit buffer per warp; drained at >= 32
constexpr int kWppNear = 128;        // density: pairs within the walk radius, kept across h iterations
constexpr int kWppGrpLeaves = 448;   // leaf list of a group walk, shared by the group's particles
constexpr int kWppGrpSpan = 64;      // default group span: one leaf-parent node (kLeaf * kFan particles)
constexpr float kWppWalkR = 1.04f;   // default walk radius of the density pass (times the starting h)

// Stack bound: a pop-4 step starts from sp <= 96 and ends at sp <= 92 + 32 =
// 124; a pop-8 step of the group walk ends at sp <= 88 + 64 = 152. Above that,
// in the pop-1 regime, the entries above the base form a depth-first stack
// with at most 7 pending siblings per level, so sp stays below
// 152 + 8 * kMaxLev = 248 < kWppStack.

struct WppSmem {
    int glf[kWppGrpLeaves];  // group walk: leaves within reach of at least one particle of the group
                             // (bit 31: "wide" for the group, see WppGroupGeom)
    int stk[kWppStack];
    int lid[kWppLeaves];     // leaf index within the box; bit 31 = "wide" (exact separations)
    float4 lof[kWppLeaves];  // leaf centre - particle (box units), h-independent rounding bound
    union {
        struct {
            float2 d[kWppNear];  // density: (r^2, m) of the near list, or the hit buffer
            int j[kWppNear];     // density: the near list's neighbour indices
        } n;
        float4 f[kWppHits];      // force: hit buffer (dx, dy, dz, neighbour index bits)
    } hit;
};

struct WppArgs {
    const BoxDesc* boxes;
    int n_boxes;
    const int32_t* act;
    const uint32_t* count_ptr;   // active count (device)
    unsigned* queue;
    int chunk;                   // consecutive active particles per queue grab
    const uint4* posm;
    const float4* posf;
    const int32_t* perm;
    const uint4* node_c;
    const float4* node_e;
    const uint4* node_lo;
    const uint4* node_hi;
    // density
    float* h;
    float* rho;
    float* omega;
    int32_t* n_ngb;
    uint8_t* flags;
    double n_target, n_tol;
    int max_iter;
    int guess_h, fixed_h;
    float walk_r;                // density: near-list radius / h (see kWppWalkR)
    int grp_shift;               // log2 of the group span (a group stays within an aligned run of
                                 // 2^grp_shift sorted particles)
    // force
    const float4* fvel;
    const float4* fthermo;
    const float4* fposh;         // per force call: leaf-relative position, h
    const float4* fvm;           // per force call: v, m
    float* acc;
    float* dudt;
    float* vsig;
    float alpha;
    unsigned long long* hash;
    Counters* ctr;
    // neighbour lists (NULL: not recorded / not used)
    int32_t* nbr;                // pool of list_pool entries
    int32_t* nbr_off;
    int32_t* nbr_n;
    int32_t* ext;                // n segments of kExtCap entries, ascending per particle
    uint32_t* ext_n;             // extra partners per particle; kExtUnusable: not usable
    uint4* list_xh;              // the lists' particle data: integer position, bits of the h they were made with
    unsigned* list_st;           // see kListSt
    // density: velocity divergence and curl (NULL: not asked)
    const float4* vpack;         // sorted (v, m)
    float* divv;
    float* curlv;
    // force: Balsara factors (sorted order; NULL: no switch), or (factor,
    // viscosity parameter) pairs for per-particle viscosity
    const float* fbal;
    const float2* fvisc;
    // force: conduction (sorted (u, kappa); NULL: no conduction) and its output (caller order)
    const float2* fcond;
    float* dudt_cond;
    int32_t* fb_list;
    long long list_pool;
    int list_chunk;              // pool entries a warp reserves at a time
    int n_total;                 // particles in the grid
    // force walk after a list pass: the particles the lists could not serve
    // (fb_act, *fb_count) when the lists are valid, else the whole active set
    const int32_t* fb_act;
    const unsigned* fb_count;
    // density, member-parallel path: near-list indices, kMpMembers x kMpCap per persistent warp
    int32_t* mp_j;
    // density: the particles the member-parallel kernel leaves to the one-particle kernel
    int32_t* left;
    unsigned* left_n;
    // lists of a partial active set: the active flag per sorted particle, the
    // far-partner scratch (kMpMembers x kMpFar per warp), and the generation
    // stamp per particle (a list serves only if its stamp is the current one)
    const uint8_t* flagp;
    int32_t* mp_x;
    uint32_t* list_ep;
};

// The recorded lists can serve this force call: none of the recorded lists
// is missing or has incomplete extra partners, and h is unchanged. (Whether a
// particle's own list is from the last density call is its list_ep stamp.)
__device__ __forceinline__ bool wpp_lists_valid(const unsigned* st) {
    return st[1] == 0u && st[2] == 0u;
}

__device__ __forceinline__ int wpp_box(const BoxDesc* boxes, int nb, long long p) {
    int lo = 0, hi = nb - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (boxes[mid].off <= p) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Error-free (TwoSum) fold of two per-lane sums across the warp: after one
// exchange lanes 0-15 carry the first and 16-31 the second; every lane ends
// with both compensated totals (sa - ca, sb - cb). Both orders of a TwoSum
// are exact, so the result does not depend on which lane adds which.
__device__ __forceinline__ void wpp_fold2(float a, float b, float& sa, float& ca, float& sb, float& cb) {
    const unsigned lane = lane_id();
    const bool lo16 = lane < 16u;
    float s = lo16 ? a : b, c = 0.f;
    const float o = __shfl_xor_sync(0xffffffffu, lo16 ? b : a, 16);
    {
        const float t = __fadd_rn(s, o);
        const float bp = __fsub_rn(t, s);
        c = __fsub_rn(0.f, __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(o, bp)));
        s = t;
    }
#pragma unroll
    for (int k = 8; k > 0; k >>= 1) {
        const float s2 = __shfl_xor_sync(0xffffffffu, s, k), c2 = __shfl_xor_sync(0xffffffffu, c, k);
        const float t = __fadd_rn(s, s2);
        const float bp = __fsub_rn(t, s);
        const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(s2, bp));
        s = t;
        c = __fsub_rn(__fadd_rn(c, c2), e);
    }
    sa = __shfl_sync(0xffffffffu, s, 0);
    ca = __shfl_sync(0xffffffffu, c, 0);
    sb = __shfl_sync(0xffffffffu, s, 16);
    cb = __shfl_sync(0xffffffffu, c, 16);
}

// The same error-free fold for four per-lane sums at once, halving the
// values a lane carries at the first two levels (lanes 0-15 keep the first
// two sums, 16-31 the last two; then each half keeps one). Returns, in lanes
// 8c..8c+7, sum c as one correctly rounded s - c.
__device__ __forceinline__ float wpp_fold4(float x, float y, float z, float u) {
    const unsigned lane = lane_id();
    auto two_sum = [](float& s, float& c, float s2, float c2) {
        const float t = __fadd_rn(s, s2);
        const float bp = __fsub_rn(t, s);
        const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(s2, bp));
        s = t;
        c = __fsub_rn(__fadd_rn(c, c2), e);
    };
    const bool lo16 = lane < 16u;
    // level 16: keep (x, y) or (z, u)
    float s1 = lo16 ? x : z, s2 = lo16 ? y : u, c1 = 0.f, c2 = 0.f;
    {
        const float o1 = __shfl_xor_sync(0xffffffffu, lo16 ? z : x, 16);
        const float o2 = __shfl_xor_sync(0xffffffffu, lo16 ? u : y, 16);
        two_sum(s1, c1, o1, 0.f);
        two_sum(s2, c2, o2, 0.f);
    }
    // level 8: keep the first or the second of the pair
    const bool lo8 = (lane & 8u) == 0u;
    float s = lo8 ? s1 : s2, c = lo8 ? c1 : c2;
    {
        const float os = __shfl_xor_sync(0xffffffffu, lo8 ? s2 : s1, 8);
        const float oc = __shfl_xor_sync(0xffffffffu, lo8 ? c2 : c1, 8);
        two_sum(s, c, os, oc);
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {
        const float os = __shfl_xor_sync(0xffffffffu, s, o), oc = __shfl_xor_sync(0xffffffffu, c, o);
        two_sum(s, c, os, oc);
    }
    return __fsub_rn(s, c);
}

// The same error-free fold of four per-lane sums within each aligned octet of
// lanes (eight lanes per particle): lanes with bit 2 clear keep the first two
// sums and the others the last two, then bit 1 picks one of the pair. Returns,
// in lanes 2c and 2c + 1 of the octet, sum c as one correctly rounded s - c.
__device__ __forceinline__ float wpp_fold4_oct(float x, float y, float z, float u) {
    const unsigned lane = lane_id();
    auto two_sum = [](float& s, float& c, float s2, float c2) {
        const float t = __fadd_rn(s, s2);
        const float bp = __fsub_rn(t, s);
        const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(s2, bp));
        s = t;
        c = __fsub_rn(__fadd_rn(c, c2), e);
    };
    const bool lo4 = (lane & 4u) == 0u;
    float s1 = lo4 ? x : z, s2 = lo4 ? y : u, c1 = 0.f, c2 = 0.f;
    {
        const float o1 = __shfl_xor_sync(0xffffffffu, lo4 ? z : x, 4);
        const float o2 = __shfl_xor_sync(0xffffffffu, lo4 ? u : y, 4);
        two_sum(s1, c1, o1, 0.f);
        two_sum(s2, c2, o2, 0.f);
    }
    const bool lo2 = (lane & 2u) == 0u;
    float s = lo2 ? s1 : s2, c = lo2 ? c1 : c2;
    {
        const float os = __shfl_xor_sync(0xffffffffu, lo2 ? s2 : s1, 2);
        const float oc = __shfl_xor_sync(0xffffffffu, lo2 ? c2 : c1, 2);
        two_sum(s, c, os, oc);
    }
    {
        const float os = __shfl_xor_sync(0xffffffffu, s, 1), oc = __shfl_xor_sync(0xffffffffu, c, 1);
        two_sum(s, c, os, oc);
    }
    return __fsub_rn(s, c);
}

// Error-free fold of one per-lane sum within each aligned octet of lanes;
// every lane of the octet ends with the total rounded once.
__device__ __forceinline__ float wpp_fold1_oct(float x) {
    float s = x, c = 0.f;
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {
        const float s2 = __shfl_xor_sync(0xffffffffu, s, o), c2 = __shfl_xor_sync(0xffffffffu, c, o);
        const float t = __fadd_rn(s, s2);
        const float bp = __fsub_rn(t, s);
        const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(s2, bp));
        s = t;
        c = __fsub_rn(__fadd_rn(c, c2), e);
    }
    return __fsub_rn(s, c);
}

// (h 2^32 / L)^2 in FP64, the right-hand side of the exact neighbour
// predicate. Out of line so that the compiler cannot hoist the FP64 division
// out of the rare band branches onto every evaluation: with one particle per
// warp each FP64 instruction costs a full warp slot of the narrow FP64 pipe.
// Without the division when L is a power of two: then h 2^32 / L = h S
// exactly (S = 2^32 / L is a power of two), a product in place of a
// division's instruction sequence; the value is the same.
static __device__ __noinline__ double wpp_hh(float h, const BoxDesc& B) {
    const double Hd = B.pow2 ? (double)h * B.S : (double)h * 4294967296.0 / B.L;
    return Hd * Hd;
}

// Node test: periodic distance from the particle to the node box below R
// (the slack covers the FP32 rounding of the centre offset).
__device__ __forceinline__ bool wpp_near(float dx, float dy, float dz, float4 e, float R) {
    const float gx = fmaxf(fabsf(dx) - e.x, 0.f), gy = fmaxf(fabsf(dy) - e.y, 0.f),
                gz = fmaxf(fabsf(dz) - e.z, 0.f);
    const float Rt = R * (1.f + 3.0517578125e-05f) + 2.384185791015625e-07f * (fabsf(dx) + fabsf(dy) + fabsf(dz));
    return gx * gx + gy * gy + gz * gz < Rt * Rt;
}

// The walk of one particle. Pushes leaves (with their offsets and bounds) to
// the shared leaf list; when the list cannot take another step's leaves it
// calls flush() (which must empty it) and marks the list incomplete.
// radius(e) is the test radius for a node with extents/h_max e; it also
// enters a leaf's "wide" test (a leaf whose extent plus radius nears half the
// box takes exact integer separations instead of centre offsets).
template <class Radius, class Flush>
__device__ __forceinline__ void wpp_walk(WppSmem& sm, const BoxDesc& B, const uint4* __restrict__ node_c,
                                         const float4* __restrict__ node_e, uint4 Xi, float sf, int& nlf,
                                         bool& complete, Radius&& radius, Flush&& flush) {
    const unsigned lane = lane_id();
    const unsigned lt = (1u << lane) - 1u;
    const float rel = 9.5367431640625e-07f;  // 2^-20
    const float wideL = B.wideL;
    int sp = 0;
    if (B.nlev == 1) {
        // a single leaf: the whole box
        if (lane == 0) {
            const uint4 C = node_c[B.lvl_off[0]];
            const float4 E = node_e[B.lvl_off[0]];
            const float ox = (float)(int)(C.x - Xi.x) * sf, oy = (float)(int)(C.y - Xi.y) * sf,
                        oz = (float)(int)(C.z - Xi.z) * sf;
            const bool wide = 2.f * (E.x + E.y + E.z) + radius(E) >= wideL;
            sm.lid[nlf] = wide ? (int)0x80000000u : 0;
            sm.lof[nlf] = make_float4(ox, oy, oz, rel * (4.f * (E.x + E.y + E.z) + 2.f * (fabsf(ox) + fabsf(oy) + fabsf(oz))));
        }
        ++nlf;
        __syncwarp();
        return;
    }
    if (lane == 0) sm.stk[0] = (B.nlev - 1) << 27;
    sp = 1;
    __syncwarp();
    while (sp > 0) {
        if (nlf > kWppLeaves - 32) {
            flush();
            complete = false;
        }
        const int npop = sp <= kWppPop4 ? min(sp, 4) : 1;
        const int slot = (int)(lane >> 3), c = (int)(lane & 7u);
        const int enc = slot < npop ? sm.stk[sp - 1 - slot] : 0;
        __syncwarp();
        sp -= npop;
        const int lev = enc >> 27, t = enc & ((1 << 27) - 1);
        const int cl = lev - 1, ct = t * kFan + c;
        const bool ok = slot < npop && ct < B.lvl_n[max(cl, 0)];
        bool pass = false;
        float dx = 0.f, dy = 0.f, dz = 0.f;
        float4 E = make_float4(0.f, 0.f, 0.f, 0.f);
        if (ok) {
            const int nd = B.lvl_off[cl] + ct;
            const uint4 C = node_c[nd];
            E = node_e[nd];
            dx = (float)(int)(C.x - Xi.x) * sf;
            dy = (float)(int)(C.y - Xi.y) * sf;
            dz = (float)(int)(C.z - Xi.z) * sf;
            pass = wpp_near(dx, dy, dz, E, radius(E));
        }
        const bool isleaf = pass && cl == 0, isint = pass && cl > 0;
        const unsigned ml = __ballot_sync(0xffffffffu, isleaf);
        const unsigned mi = __ballot_sync(0xffffffffu, isint);
        if (isleaf) {
            const int li = nlf + __popc(ml & lt);
            const bool wide = 2.f * (E.x + E.y + E.z) + radius(E) >= wideL;
            sm.lid[li] = ct | (wide ? (int)0x80000000u : 0);
            sm.lof[li] = make_float4(dx, dy, dz, rel * (4.f * (E.x + E.y + E.z) + 2.f * (fabsf(dx) + fabsf(dy) + fabsf(dz))));
        }
        if (isint) sm.stk[sp + __popc(mi & lt)] = (cl << 27) | ct;
        nlf += __popc(ml);
        sp += __popc(mi);
        __syncwarp();
    }
}

// A group: the leading run of the remaining active particles act[t..t1) that
// lie in the box and the aligned run of 2^shift sorted particles (by default
// kWppGrpSpan: the leaf-parent node) of act[t]. Lane l < n holds member l's
// sorted index in p (other lanes: -1).
struct WppGroup {
    int n;
    int p;
    int box;
};

__device__ __forceinline__ WppGroup wpp_group(const BoxDesc* boxes, int nb, const int32_t* act, int t, int t1,
                                              int shift) {
    const unsigned lane = lane_id();
    const int rem = t1 - t;
    int pl = -1, bl = 0;
    if ((int)lane < rem) {
        pl = act[t + lane];
        if (nb > 1) bl = wpp_box(boxes, nb, pl);
    }
    const int p0 = __shfl_sync(0xffffffffu, pl, 0), b0 = __shfl_sync(0xffffffffu, bl, 0);
    const long long off = boxes[b0].off;
    const bool same = (int)lane < rem && bl == b0 && ((pl - off) >> shift) == ((p0 - off) >> shift);
    const unsigned m = __ballot_sync(0xffffffffu, same);
    WppGroup g;
    g.n = __ffs(~m) - 1;   // rem <= 8, so ~m has a set bit
    g.p = (int)lane < g.n ? pl : -1;
    g.box = b0;
    return g;
}

// One walk of the hierarchy for a whole group (sm: any shared-memory block
// with a leaf list glf[kWppGrpLeaves] and a stack stk[kWppStack]), whose members' integer
// positions lie within hx[a] (integer units, per axis) of the integer centre
// Gc; eg = hx * (L/2^32), rounded up. A node passes when its box comes within
// radius(E) of the group's box. This holds whenever the node passes the test
// of any member (wpp_near at that member's position, with a radius no larger
// than the group's): per axis, a member's periodic offset from the node is at
// least the group centre's minus hx, in every periodic image. The slack
// (2^-14 of R plus 2^-20 of the offsets and extents) covers the FP32 rounding
// of both tests. Leaves go to sm.glf; returns their number, or -1 when they
// would not fit (the members then walk alone).
// Geometry of a group and of its leaf list: the integer centre Gc, the
// half-extents eg (box units, rounded up) of the members' box around it, and,
// over the listed leaves, the largest bound eb on the FP32 rounding error of
// a separation (leaf centre - Gc) + (particle - leaf centre) - (member - Gc);
// a listed leaf is marked wide (bit 31) when that form may not be the minimum
// image for every member.
struct WppGroupGeom {
    uint4 Gc;
    float egx, egy, egz;
    float eb;
};

template <class SM, class Radius>
__device__ __forceinline__ int wpp_group_walk(SM& sm, const BoxDesc& B, const uint4* __restrict__ node_c,
                                              const float4* __restrict__ node_e, WppGroupGeom& gg, float sf,
                                              Radius&& radius) {
    const unsigned lane = lane_id();
    const unsigned lt = (1u << lane) - 1u;
    const uint4 Gc = gg.Gc;
    const float egx = gg.egx, egy = gg.egy, egz = gg.egz;
    const float egs = egx + egy + egz;
    const float rel = 9.5367431640625e-07f;  // 2^-20
    float eb = 0.f;
    int ngl = 0;
    if (lane == 0) sm.stk[0] = (B.nlev - 1) << 27;
    int sp = 1;
    __syncwarp();
    // One child test of the walk: pass/leaf/internal for child c of node enc.
    auto test = [&](int enc, int c, bool live, int& ct, bool& isleaf, bool& isint) {
        const int lev = enc >> 27, t = enc & ((1 << 27) - 1);
        const int cl = lev - 1;
        ct = t * kFan + c;
        const bool ok = live && ct < B.lvl_n[max(cl, 0)];
        bool pass = false;
        if (ok) {
            const int nd = B.lvl_off[cl] + ct;
            const uint4 C = node_c[nd];
            const float4 E = node_e[nd];
            const float dx = (float)(int)(C.x - Gc.x) * sf, dy = (float)(int)(C.y - Gc.y) * sf,
                        dz = (float)(int)(C.z - Gc.z) * sf;
            const float gx = fmaxf(fabsf(dx) - E.x - egx, 0.f), gy = fmaxf(fabsf(dy) - E.y - egy, 0.f),
                        gz = fmaxf(fabsf(dz) - E.z - egz, 0.f);
            const float Rt = radius(E) * (1.f + 6.103515625e-05f) +
                             9.5367431640625e-07f * (fabsf(dx) + fabsf(dy) + fabsf(dz) + E.x + E.y + E.z + egs);
            pass = gx * gx + gy * gy + gz * gz < Rt * Rt;
            if (pass && cl == 0) {
                const bool wide = 2.f * (E.x + E.y + E.z + egs) + radius(E) >= B.wideL;
                ct |= wide ? (int)0x80000000u : 0;
                if (!wide)
                    eb = fmaxf(eb, rel * (4.f * (E.x + E.y + E.z) + 2.f * (fabsf(dx) + fabsf(dy) + fabsf(dz))));
            }
        }
        isleaf = pass && cl == 0;
        isint = pass && cl > 0;
    };
    // Up to eight nodes per step while the stack is shallow (two children per
    // lane, their loads in flight together), one node per step beyond.
    while (sp > 0) {
        if (ngl > kWppGrpLeaves - 64) return -1;
        const int npop = sp <= kWppPop8 ? min(sp, 8) : 1;
        const int slot = (int)(lane >> 3), c = (int)(lane & 7u);
        const int encA = slot < npop ? sm.stk[sp - 1 - slot] : 0;
        const int encB = slot + 4 < npop ? sm.stk[sp - 5 - slot] : 0;
        __syncwarp();
        sp -= npop;
        int ctA, ctB;
        bool leafA, intA, leafB, intB;
        test(encA, c, slot < npop, ctA, leafA, intA);
        test(encB, c, slot + 4 < npop, ctB, leafB, intB);
        const int clA = (encA >> 27) - 1, clB = (encB >> 27) - 1;
        const unsigned mlA = __ballot_sync(0xffffffffu, leafA), miA = __ballot_sync(0xffffffffu, intA);
        const unsigned mlB = __ballot_sync(0xffffffffu, leafB), miB = __ballot_sync(0xffffffffu, intB);
        if (leafA) sm.glf[ngl + __popc(mlA & lt)] = ctA;
        if (intA) sm.stk[sp + __popc(miA & lt)] = (clA << 27) | ctA;
        ngl += __popc(mlA);
        sp += __popc(miA);
        if (leafB) sm.glf[ngl + __popc(mlB & lt)] = ctB;
        if (intB) sm.stk[sp + __popc(miB & lt)] = (clB << 27) | ctB;
        ngl += __popc(mlB);
        sp += __popc(miB);
        __syncwarp();
    }
    gg.eb = warp_max(eb) + rel * 2.f * egs;
    return ngl;
}

// Group geometry from the members' integer positions (lanes with `valid`),
// then the group walk. Returns -1 (no shared list) when the group spans a
// quarter of the box or more on some axis.
template <class SM, class Radius>
__device__ __forceinline__ int wpp_group_leaves(SM& sm, const BoxDesc& B, const uint4* __restrict__ node_c,
                                                const float4* __restrict__ node_e, uint4 Xl, bool valid, float sf,
                                                Radius&& radius, WppGroupGeom& gg) {
    const unsigned X0x = __shfl_sync(0xffffffffu, Xl.x, 0), X0y = __shfl_sync(0xffffffffu, Xl.y, 0),
                   X0z = __shfl_sync(0xffffffffu, Xl.z, 0);
    const int dx = valid ? (int)(Xl.x - X0x) : 0, dy = valid ? (int)(Xl.y - X0y) : 0,
              dz = valid ? (int)(Xl.z - X0z) : 0;
    const int lox = warp_min(dx), loy = warp_min(dy), loz = warp_min(dz);
    const long long ex = (long long)warp_max(dx) - lox, ey = (long long)warp_max(dy) - loy,
                    ez = (long long)warp_max(dz) - loz;
    if (ex >= (1ll << 30) || ey >= (1ll << 30) || ez >= (1ll << 30)) return -1;
    gg.Gc.x = X0x + (unsigned)(lox + (int)(ex >> 1));
    gg.Gc.y = X0y + (unsigned)(loy + (int)(ey >> 1));
    gg.Gc.z = X0z + (unsigned)(loz + (int)(ez >> 1));
    gg.Gc.w = 0u;
    const float up = 1.f + 9.5367431640625e-07f;
    gg.egx = (float)((ex + 1) >> 1) * sf * up;
    gg.egy = (float)((ey + 1) >> 1) * sf * up;
    gg.egz = (float)((ez + 1) >> 1) * sf * up;
    return wpp_group_walk(sm, B, node_c, node_e, gg, sf, radius);
}
template <class Radius>
__device__ __forceinline__ int wpp_group_leaves(WppSmem& sm, const BoxDesc& B, const uint4* __restrict__ node_c,
                                                const float4* __restrict__ node_e, uint4 Xl, bool valid, float sf,
                                                Radius&& radius) {
    WppGroupGeom gg;
    return wpp_group_leaves(sm, B, node_c, node_e, Xl, valid, sf, radius, gg);
}

// A member's own leaf list from the group's: the leaves of sm.glf that pass
// the member's node test, pushed exactly as wpp_walk pushes them (same test,
// same entries), so the member sees the leaf set of its own walk.
template <class Radius, class Flush>
__device__ __forceinline__ void wpp_filter(WppSmem& sm, int ngl, const BoxDesc& B, const uint4* __restrict__ node_c,
                                           const float4* __restrict__ node_e, uint4 Xi, float sf, int& nlf,
                                           bool& complete, Radius&& radius, Flush&& flush) {
    const unsigned lane = lane_id();
    const unsigned lt = (1u << lane) - 1u;
    const float rel = 9.5367431640625e-07f;  // 2^-20
    const float wideL = B.wideL;
    for (int base = 0; base < ngl; base += 32) {
        if (nlf > kWppLeaves - 32) {
            flush();
            complete = false;
        }
        const int k = base + (int)lane;
        bool pass = false;
        int ct = 0;
        float dx = 0.f, dy = 0.f, dz = 0.f;
        float4 E = make_float4(0.f, 0.f, 0.f, 0.f);
        if (k < ngl) {
            ct = sm.glf[k] & 0x7fffffff;
            const int nd = B.lvl_off[0] + ct;
            const uint4 C = node_c[nd];
            E = node_e[nd];
            dx = (float)(int)(C.x - Xi.x) * sf;
            dy = (float)(int)(C.y - Xi.y) * sf;
            dz = (float)(int)(C.z - Xi.z) * sf;
            pass = wpp_near(dx, dy, dz, E, radius(E));
        }
        const unsigned ml = __ballot_sync(0xffffffffu, pass);
        if (pass) {
            const int li = nlf + __popc(ml & lt);
            const bool wide = 2.f * (E.x + E.y + E.z) + radius(E) >= wideL;
            sm.lid[li] = ct | (wide ? (int)0x80000000u : 0);
            sm.lof[li] = make_float4(dx, dy, dz, rel * (4.f * (E.x + E.y + E.z) + 2.f * (fabsf(dx) + fabsf(dy) + fabsf(dz))));
        }
        nlf += __popc(ml);
        __syncwarp();
    }
}

__device__ __forceinline__ float hinv_cube(float h) {
    const float r = 1.f / h;
    return r * r * r;
}

__device__ __forceinline__ float wpp_guess_h(const BoxDesc& B, const uint4* node_lo, const uint4* node_hi,
                                             long long p, double s, double n_target) {
    double best = 0.25 * B.L;
    const int top = B.nlev > 1 ? 1 : 0;
    for (int lev = 0; lev <= top; ++lev) {
        const long long span = lev ? (long long)kLeaf * kFan : kLeaf;
        const long long t = (p - B.off) / span;
        const uint4 lo = node_lo[B.lvl_off[lev] + t], hi = node_hi[B.lvl_off[lev] + t];
        const double cnt = (double)min(span, B.n - t * span);
        const double V = ((double)(hi.x - lo.x) + 1.0) * ((double)(hi.y - lo.y) + 1.0) *
                         ((double)(hi.z - lo.z) + 1.0) * s * s * s;
        best = fmin(best, cbrt(3.0 * n_target * V / (4.0 * 3.141592653589793 * cnt)));
    }
    return (float)best;
}

// Bracketed, safeguarded step of the smoothing-length solve (the rule of the
// other paths): Newton on N^(1/3) - N_t^(1/3), bisection when the step leaves
// the bracket or does not halve. Everything is FP32 here: a warp works on one
// particle, so each FP64 instruction would cost a full warp slot of the narrow
// FP64 pipe per particle. Only the sign of f is used. Returns false when h
// cannot move (the bracket is one float wide, or an error bit was set).
__device__ __forceinline__ bool wpp_h_update(float& h, float f, float N, float dN, float n_target, float capu,
                                             float& blo, float& bhi, float& dold, unsigned& st) {
    if (f < 0.f) blo = h; else bhi = h;
    const float step = dN > 0.f ? 3.f * N * (1.f - cbrtf(n_target / N)) / dN : NAN;
    float hn = h - step;
    if (isinf(bhi)) {
        if (h >= capu) {
            st |= ST_H_TOO_LARGE;
            return false;
        }
        if (!(hn > h)) hn = 2.f * h;
        hn = fminf(hn, fminf(capu, 8.f * h));
    } else if (!(hn > blo && hn < bhi) || !(fabsf(step) <= 0.5f * dold)) {
        hn = 0.5f * (blo + bhi);
    }
    dold = fabsf(hn - h);
    if (!(hn > blo) || (!isinf(bhi) && !(hn < bhi))) {
        const float mid = 0.5f * (blo + bhi);
        hn = (mid > blo && mid < bhi) ? mid : h;
    }
    if (hn == h) return false;
    h = hn;
    return true;
}

// The particle-i constants of the force pair terms.
struct WppForceI {
    float vx, vy, vz;
    float hinv, rho, A, c, norm;   // norm = 8/(pi h^4)
    float f;                       // Balsara factor (1 without the switch)
    float u, kap;                  // conduction: u and conductivity (unused without it)
    float al;                      // own viscosity parameter (VISC = 2 only)
};

// Viscosity variants of the force pair term: kViscScalar, one alpha for every
// pair; kViscBalsara, alpha (f_i + f_j)/2; kViscPerParticle, per-particle
// alpha, (alpha_i + alpha_j)/2 (f_i + f_j)/2, f = 1 without the switch.
constexpr int kViscScalar = 0, kViscBalsara = 1, kViscPerParticle = 2;

// One force pair term, Gadget-2 grad-h form with signal-velocity viscosity,
// added to i's per-lane sums. (dx, dy, dz) = x_j - x_i; vj = (v_j, m_j);
// thj = (rho_j, A_j, c_j, 1/h_j); bj = (f_j, alpha_j): j's Balsara factor
// (VISC >= 1) and viscosity parameter (VISC = 2), see kViscScalar.
// COND adds the conduction term m_j/(rho_i rho_j) 4 k_i k_j/(k_i + k_j)
// (u_i - u_j) Fbar_ij to Sc, with cj = (u_j, kappa_j).
template <int VISC, bool COND>
__device__ __forceinline__ void wpp_force_pair(const WppForceI& I, float dx, float dy, float dz, float4 vj, float4 thj,
                                               float2 bj, float2 cj, float alpha, float& Sx, float& Sy, float& Sz,
                                               float& Su, float& Sc, float& vsmax) {
    const float kNorm = (float)(8.0 / 3.141592653589793);
    const float r2 = dx * dx + dy * dy + dz * dz;
    if (r2 <= 0.f) {  // coincident: no direction, no force
        vsmax = fmaxf(vsmax, I.c + thj.z);
        return;
    }
    const float rinv = rsqrtf(r2), r = r2 * rinv;
    float w_, dwi, dwj;
    spline<float>(r * I.hinv, w_, dwi);
    spline<float>(r * thj.w, w_, dwj);
    const float hinvj = thj.w;
    const float Fi = I.norm * dwi * rinv;
    const float Fj = kNorm * hinvj * hinvj * hinvj * hinvj * dwj * rinv;
    const float vr = -((I.vx - vj.x) * dx + (I.vy - vj.y) * dy + (I.vz - vj.z) * dz);
    const float wij = vr * rinv;
    const float vs = I.c + thj.z - 3.f * wij;
    vsmax = fmaxf(vsmax, vs);
    // Pi_ij = -(alpha/2) v_sig w_ij / rho_bar, rho_bar = (rho_i + rho_j)/2
    const float aij = VISC == kViscPerParticle ? 0.5f * (I.al + bj.y) : alpha;
    float PI = wij < 0.f ? __fdividef(-aij * vs * wij, I.rho + thj.x) : 0.f;
    if (VISC != kViscScalar) PI *= 0.5f * (I.f + bj.x);
    const float Fbar = 0.5f * (Fi + Fj);
    const float mj = vj.w;
    if (COND) {
        const float ks = I.kap + cj.y;
        const float kij = ks > 0.f ? __fdividef(4.f * I.kap * cj.y, ks) : 0.f;
        Sc += __fdividef(mj, I.rho * thj.x) * kij * (I.u - cj.x) * Fbar;
    }
    const float coef = mj * (I.A * Fi + thj.y * Fj + PI * Fbar);
    Sx += coef * dx;
    Sy += coef * dy;
    Sz += coef * dz;
    Su += mj * vr * (I.A * Fi + 0.5f * PI * Fbar);
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------

// SPH_TIME_KERNELS: an event pair around a span of launches on stream s.
struct WppSpan {
    cudaEvent_t a = nullptr;
    int kind = 0;
};

static inline cudaError_t span_begin(sph_ctx* ctx, int timed, int kind, cudaStream_t s, WppSpan& sp) {
    sp.kind = kind;
    if (!timed) return cudaSuccess;
    sp.a = timing_event(ctx);
    if (!sp.a) return cudaErrorMemoryAllocation;
    return cudaEventRecord(sp.a, s);
}

static inline cudaError_t span_end(sph_ctx* ctx, const WppSpan& sp, cudaStream_t s) {
    if (!sp.a) return cudaSuccess;
    cudaEvent_t b = timing_event(ctx);
    if (!b) return cudaErrorMemoryAllocation;
    cudaEventRecord(b, s);
    ctx->timed.push_back({sp.a, b, sp.kind});
    return cudaSuccess;
}

// Persistent grid and the number of consecutive active particles a warp takes
// per queue grab (several for locality in L1, fewer when the set is small so
// that every warp gets work).
static inline void wpp_shape(sph_ctx* ctx, int bps, int64_t n_active, int& blocks, int& chunk) {
    const int b = std::min(bps, std::min(kWppMaxBps, kMpWarpsPerSm / kWppWarps));
    const long long warps_needed = std::max<long long>(1, n_active);
    const long long want_blocks = (warps_needed + kWppWarps - 1) / kWppWarps;
    blocks = (int)std::max<long long>(1, std::min<long long>((long long)ctx->sm_count * b, want_blocks));
    const long long warps = (long long)blocks * kWppWarps;
    chunk = (int)std::max<long long>(1, std::min<long long>(kMpMembers, n_active / (warps * 4)));
}

// log2 of a group span (0: the default kWppGrpSpan)
static inline int wpp_grp_shift(int span) {
    int s = 0;
    while ((1 << s) < (span > 0 ? span : kWppGrpSpan)) ++s;
    return s;
}

static inline WppArgs wpp_common(sph_ctx* ctx, const sph_grid* g, unsigned* queue) {
    WppArgs c = {};
    c.boxes = g->boxes;
    c.n_boxes = g->n_boxes;
    c.act = g->act;
    c.count_ptr = g->scan + g->n;
    c.queue = queue;
    c.posm = g->posm;
    c.posf = g->posf;
    c.perm = g->perm;
    c.node_c = g->node_c;
    c.node_e = g->node_e;
    c.node_lo = g->node_lo;
    c.node_hi = g->node_hi;
    c.ctr = ctx->counters;
    c.n_total = (int)g->n;
    c.grp_shift = 6;   // kWppGrpSpan
    return c;
}


// The member-parallel kernels pay when there are enough groups to fill the
// GPU (a warp per group of up to 8: at least 16 warps per SM) and active
// particles are not too sparse to share leaves (at least 1 in 256 active).
// Measured on 10M clustered particles with time-bin active sets: 1% active
// (100k) runs faster in groups, 0.1% (10k) slower.
static inline bool wpp_groups_pay(const sph_ctx* ctx, int64_t n_active, int64_t n) {
    return n_active >= (int64_t)kMpMembers * 16 * ctx->sm_count && n_active * 256 >= n;
}

// Grid of a warp-per-particle helper kernel over n particles (256 threads).
static inline int helper_blocks(sph_ctx* ctx, int64_t n) {
    return (int)std::max<long long>(1, std::min<long long>((long long)ctx->sm_count * 8, (n + 7) / 8));
}

}  // namespace sph
