// wpp.cu -- warp-per-particle density and force kernels (the default path).
//
// Work is handed out in chunks of up to 8 Morton-consecutive active particles.
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
// set at its final h. When every particle was active, the transpose adds each
// particle's partners with h_i <= r_ij < h_j, and the force pass then reads
// its pairs from the two lists (k_force_list) instead of walking; the walk
// (k_force_wpp) serves the particles, or calls, the lists cannot.
#include <algorithm>

#include "internal.cuh"

namespace sph {

constexpr int kWppWarps = 4;
constexpr int kWppThreads = kWppWarps * 32;
// Register budgets: 8 resident blocks (32 warps, 64 registers) or 6 (24 warps,
// 80 registers); the launch takes the one matching blocks_per_sm. The
// autotuner picks between them per pass.
constexpr int kWppDensityBps = 8;
constexpr int kWppForceBps = 8;
constexpr int kWppMaxBps = 16;
constexpr int kWppStack = 256;       // see the bound below
constexpr int kWppPop4 = 96;         // pop four nodes per step only while sp <= this
constexpr int kWppLeaves = 128;      // leaf list per warp; a step adds <= 32
constexpr int kWppHits = 64;         // hit buffer per warp; drained at >= 32
constexpr int kWppNear = 128;        // density: pairs within the walk radius, kept across h iterations
constexpr int kWppGrpLeaves = 384;   // leaf list of a group walk, shared by the group's particles
constexpr int kWppGrpSpan = 64;      // a group never leaves one leaf-parent node (kLeaf * kFan particles)
constexpr float kWppWalkR = 1.04f;   // density walks at 1.04 h so that later iterations reuse the list

// Stack bound: a pop-4 step starts from sp <= 96 and ends at sp <= 92 + 32 =
// 124. Above that, in the pop-1 regime, the entries above the base form a
// depth-first stack with at most 7 pending siblings per level, so sp stays
// below 124 + 8 * kMaxLev = 220 < kWppStack.

struct WppSmem {
    int stk[kWppStack];
    int glf[kWppGrpLeaves];  // group walk: leaves within reach of at least one particle of the group
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
    const int32_t* ext;          // pool of ext_pool entries, ascending per particle
    const uint32_t* ext_off;     // n + 1
    const uint32_t* ext_n;       // nonzero: the particle's extra partners are not usable
    float* list_h;
    unsigned* list_st;           // see kListSt
    // density: velocity divergence and curl (NULL: not asked)
    const float4* vpack;         // sorted (v, m)
    float* divv;
    float* curlv;
    // force: Balsara factors (sorted order; NULL: no switch)
    const float* fbal;
    // force: conduction (sorted (u, kappa); NULL: no conduction) and its output (caller order)
    const float2* fcond;
    float* dudt_cond;
    int32_t* fb_list;
    long long list_pool;
    int list_chunk;              // pool entries a warp reserves at a time
    unsigned ext_pool;
    int n_total;                 // particles in the grid
    // force walk after a list pass: the particles the lists could not serve
    // (fb_act, *fb_count) when the lists are valid, else the whole active set
    const int32_t* fb_act;
    const unsigned* fb_count;
};

// The recorded lists can serve this force call: every particle's list was
// written by the last density call, none is missing, and h is unchanged.
__device__ __forceinline__ bool wpp_lists_valid(const unsigned* st, int n) {
    return st[0] == (unsigned)n && st[1] == 0u && st[2] == 0u;
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

// (h 2^32 / L)^2 in FP64, the right-hand side of the exact neighbour
// predicate. Out of line so that the compiler cannot hoist the FP64 division
// out of the rare band branches onto every evaluation: with one particle per
// warp each FP64 instruction costs a full warp slot of the narrow FP64 pipe.
__device__ __noinline__ double wpp_hh(float h, double L) {
    const double Hd = (double)h * 4294967296.0 / L;
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
// lie in the box and the leaf-parent node (kWppGrpSpan sorted particles) of
// act[t]. Lane l < n holds member l's sorted index in p (other lanes: -1).
struct WppGroup {
    int n;
    int p;
    int box;
};

__device__ __forceinline__ WppGroup wpp_group(const BoxDesc* boxes, int nb, const int32_t* act, int t, int t1) {
    const unsigned lane = lane_id();
    const int rem = t1 - t;
    int pl = -1, bl = 0;
    if ((int)lane < rem) {
        pl = act[t + lane];
        if (nb > 1) bl = wpp_box(boxes, nb, pl);
    }
    const int p0 = __shfl_sync(0xffffffffu, pl, 0), b0 = __shfl_sync(0xffffffffu, bl, 0);
    const long long off = boxes[b0].off;
    const bool same = (int)lane < rem && bl == b0 && (pl - off) / kWppGrpSpan == (p0 - off) / kWppGrpSpan;
    const unsigned m = __ballot_sync(0xffffffffu, same);
    WppGroup g;
    g.n = __ffs(~m) - 1;   // rem <= 8, so ~m has a set bit
    g.p = (int)lane < g.n ? pl : -1;
    g.box = b0;
    return g;
}

// One walk of the hierarchy for a whole group, whose members' integer
// positions lie within hx[a] (integer units, per axis) of the integer centre
// Gc; eg = hx * (L/2^32), rounded up. A node passes when its box comes within
// radius(E) of the group's box. This holds whenever the node passes the test
// of any member (wpp_near at that member's position, with a radius no larger
// than the group's): per axis, a member's periodic offset from the node is at
// least the group centre's minus hx, in every periodic image. The slack
// (2^-14 of R plus 2^-20 of the offsets and extents) covers the FP32 rounding
// of both tests. Leaves go to sm.glf; returns their number, or -1 when they
// would not fit (the members then walk alone).
template <class Radius>
__device__ __forceinline__ int wpp_group_walk(WppSmem& sm, const BoxDesc& B, const uint4* __restrict__ node_c,
                                              const float4* __restrict__ node_e, uint4 Gc, float egx, float egy,
                                              float egz, float sf, Radius&& radius) {
    const unsigned lane = lane_id();
    const unsigned lt = (1u << lane) - 1u;
    const float egs = egx + egy + egz;
    int ngl = 0;
    if (lane == 0) sm.stk[0] = (B.nlev - 1) << 27;
    int sp = 1;
    __syncwarp();
    while (sp > 0) {
        if (ngl > kWppGrpLeaves - 32) return -1;
        const int npop = sp <= kWppPop4 ? min(sp, 4) : 1;
        const int slot = (int)(lane >> 3), c = (int)(lane & 7u);
        const int enc = slot < npop ? sm.stk[sp - 1 - slot] : 0;
        __syncwarp();
        sp -= npop;
        const int lev = enc >> 27, t = enc & ((1 << 27) - 1);
        const int cl = lev - 1, ct = t * kFan + c;
        const bool ok = slot < npop && ct < B.lvl_n[max(cl, 0)];
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
        }
        const bool isleaf = pass && cl == 0, isint = pass && cl > 0;
        const unsigned ml = __ballot_sync(0xffffffffu, isleaf);
        const unsigned mi = __ballot_sync(0xffffffffu, isint);
        if (isleaf) sm.glf[ngl + __popc(ml & lt)] = ct;
        if (isint) sm.stk[sp + __popc(mi & lt)] = (cl << 27) | ct;
        ngl += __popc(ml);
        sp += __popc(mi);
        __syncwarp();
    }
    return ngl;
}

// Group geometry from the members' integer positions (lanes with `valid`),
// then the group walk. Returns -1 (no shared list) when the group spans a
// quarter of the box or more on some axis.
template <class Radius>
__device__ __forceinline__ int wpp_group_leaves(WppSmem& sm, const BoxDesc& B, const uint4* __restrict__ node_c,
                                                const float4* __restrict__ node_e, uint4 Xl, bool valid, float sf,
                                                Radius&& radius) {
    const unsigned X0x = __shfl_sync(0xffffffffu, Xl.x, 0), X0y = __shfl_sync(0xffffffffu, Xl.y, 0),
                   X0z = __shfl_sync(0xffffffffu, Xl.z, 0);
    const int dx = valid ? (int)(Xl.x - X0x) : 0, dy = valid ? (int)(Xl.y - X0y) : 0,
              dz = valid ? (int)(Xl.z - X0z) : 0;
    const int lox = warp_min(dx), loy = warp_min(dy), loz = warp_min(dz);
    const long long ex = (long long)warp_max(dx) - lox, ey = (long long)warp_max(dy) - loy,
                    ez = (long long)warp_max(dz) - loz;
    if (ex >= (1ll << 30) || ey >= (1ll << 30) || ez >= (1ll << 30)) return -1;
    uint4 Gc;
    Gc.x = X0x + (unsigned)(lox + (int)(ex >> 1));
    Gc.y = X0y + (unsigned)(loy + (int)(ey >> 1));
    Gc.z = X0z + (unsigned)(loz + (int)(ez >> 1));
    Gc.w = 0u;
    const float up = 1.f + 9.5367431640625e-07f;
    const float egx = (float)((ex + 1) >> 1) * sf * up, egy = (float)((ey + 1) >> 1) * sf * up,
                egz = (float)((ez + 1) >> 1) * sf * up;
    return wpp_group_walk(sm, B, node_c, node_e, Gc, egx, egy, egz, sf, radius);
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
            ct = sm.glf[k];
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
};

// One force pair term, Gadget-2 grad-h form with signal-velocity viscosity,
// added to i's per-lane sums. (dx, dy, dz) = x_j - x_i; vj = (v_j, m_j);
// thj = (rho_j, A_j, c_j, 1/h_j); fj = j's Balsara factor (1 without the
// switch: BAL = false leaves Pi_ij alone; BAL = true multiplies it by (f_i + f_j)/2).
// COND adds the conduction term m_j/(rho_i rho_j) 4 k_i k_j/(k_i + k_j)
// (u_i - u_j) Fbar_ij to Sc, with cj = (u_j, kappa_j).
template <bool BAL, bool COND>
__device__ __forceinline__ void wpp_force_pair(const WppForceI& I, float dx, float dy, float dz, float4 vj, float4 thj,
                                               float fj, float2 cj, float alpha, float& Sx, float& Sy, float& Sz,
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
    float PI = wij < 0.f ? __fdividef(-alpha * vs * wij, I.rho + thj.x) : 0.f;
    if (BAL) PI *= 0.5f * (I.f + fj);
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
// Density
// ---------------------------------------------------------------------------

template <bool HASH, int MINB, bool DIVCURL>
__global__ void __launch_bounds__(kWppThreads, MINB) k_density_wpp(WppArgs a) {
    __shared__ WppSmem smem[kWppWarps];
    WppSmem& sm = smem[threadIdx.x >> 5];
    const unsigned lane = lane_id();
    const unsigned lt = (1u << lane) - 1u;
    const float rel = 9.5367431640625e-07f;  // 2^-20
    const float nt = (float)a.n_target, nt3 = 3.f * nt, tol3 = 3.f * (float)a.n_tol;
    const int cnt = (int)*a.count_ptr;
    unsigned c_pairs = 0, c_evals = 0, c_tests = 0, c_status = 0, c_lists = 0;   // per warp (32-bit suffices)
    long long ch_next = 0, ch_end = 0;   // the warp's current chunk of the neighbour-list pool
    for (;;) {
        int t0 = 0;
        if (lane == 0) t0 = (int)atomicAdd(a.queue, (unsigned)a.chunk);
        t0 = __shfl_sync(0xffffffffu, t0, 0);
        if (t0 >= cnt) break;
        const int t1 = min(t0 + a.chunk, cnt);
        for (int t = t0; t < t1;) {
            const WppGroup G = wpp_group(a.boxes, a.n_boxes, a.act, t, t1);
            t += G.n;
            const BoxDesc& B = a.boxes[G.box];
            const float sf = B.sf;
            const int off = (int)B.off, pend = (int)(B.off + B.n);
            // members' start h, one per lane, then one shared walk for the group
            // (radius: the largest first walk radius of its members)
            uint4 Xl = make_uint4(0u, 0u, 0u, 0u);
            int ol = 0;
            float hl = 0.f;
            if (G.p >= 0) {
                Xl = a.posm[G.p];
                ol = a.perm[G.p];
                hl = a.h[ol];
                if (a.guess_h || !(hl > 0.f) || !isfinite(hl))
                    hl = wpp_guess_h(B, a.node_lo, a.node_hi, G.p, ldexp(B.L, -32), a.n_target);
            }
            int ngl = -1;
            if (G.n >= 2 && B.nlev > 1) {
                const float Rg = warp_max(a.fixed_h ? hl : hl * kWppWalkR);
                ngl = wpp_group_leaves(sm, B, a.node_c, a.node_e, Xl, G.p >= 0, sf, [&](float4) { return Rg; });
            }
            for (int m = 0; m < G.n; ++m) {
                const int p = __shfl_sync(0xffffffffu, G.p, m);
                const uint4 Xi = make_uint4(__shfl_sync(0xffffffffu, Xl.x, m), __shfl_sync(0xffffffffu, Xl.y, m),
                                            __shfl_sync(0xffffffffu, Xl.z, m), __shfl_sync(0xffffffffu, Xl.w, m));
                const int oi = __shfl_sync(0xffffffffu, ol, m);
                float h = __shfl_sync(0xffffffffu, hl, m);
                bool first = true;   // the first walk takes the group's leaf list
                float blo = 0.f, bhi = INFINITY, dold = INFINITY;
                unsigned st = 0;
                int nlf = 0, nnear = 0;
                bool complete = false;   // the leaf list holds every leaf within Rw
                bool near_ok = false;    // the near list holds every pair within Rw
                float Rw = 0.f, ebmax = 0.f;
                // per-lane partial sums (a lane holds ~1/32 of the pairs; the fold
                // across lanes is error-free, so no per-lane compensation is needed)
                float Sw, Sdw, Smw, Smdw;
                int nn;
                unsigned long long hs;
                for (int it = 0;; ++it) {
                    Sw = Sdw = Smw = Smdw = 0.f;
                    nn = 0;
                    hs = 0;
                    const float hinv = 1.f / h;
                    double HH = -1.0;
                    int nh = 0;
                    auto exact_in = [&](int q) {
                        if (HH < 0.0) HH = wpp_hh(h, B.L);
                        return exact_pred(exact_d2(Xi, a.posm[q]), HH);
                    };
                    auto term = [&](float r2, float m) {
                        const float qq = (r2 > 0.f ? r2 * rsqrtf(r2) : 0.f) * hinv;
                        float w, dw;
                        spline<float>(qq, w, dw);
                        const float qdw = qq * dw;
                        Sw += w;
                        Sdw += qdw;
                        Smw += m * w;
                        Smdw += m * qdw;
                    };
                    // fallback evaluation: pair terms of hits [0, k) of the buffer
                    auto drain = [&](int k) {
                        __syncwarp();
                        if ((int)lane < k) term(sm.hit.n.d[lane].x, sm.hit.n.d[lane].y);
                        __syncwarp();
                    };
                    // Tests the candidates of leaf list entries [0, nlf), 32 per
                    // step. near == false: pairs within h go to the hit buffer and
                    // are evaluated at this h. near == true: pairs within the walk
                    // radius Rw go to the near list (capacity kWppNear).
                    auto process = [&](bool near) {
                        const float R = near ? Rw : h;
                        for (int base = 0; base < nlf; base += 4) {
                            // li <= 127 < kWppLeaves: entries past nlf are stale but in
                            // bounds; lanes without a candidate read particle p itself
                            const int li = base + (int)(lane >> 3);
                            const int id = sm.lid[li];
                            const float4 o = sm.lof[li];
                            const int qq = off + (id & 0x7fffffff) * kLeaf + (int)(lane & 7u);
                            const bool cand = li < nlf && qq < pend;
                            const int q = cand ? qq : p;
                            const float4 f = __ldg(a.posf + q);
                            float dx = o.x + f.x, dy = o.y + f.y, dz = o.z + f.z, m = f.w;
                            if (__any_sync(0xffffffffu, cand && id < 0)) {
                                if (cand && id < 0) {   // wide leaf: exact integer separations
                                    const uint4 Xj = a.posm[q];
                                    dx = (float)(int)(Xj.x - Xi.x) * sf;
                                    dy = (float)(int)(Xj.y - Xi.y) * sf;
                                    dz = (float)(int)(Xj.z - Xi.z) * sf;
                                    m = __uint_as_float(Xj.w);
                                }
                            }
                            const float r2 = dx * dx + dy * dy + dz * dz;
                            const float eL = o.w + 2.f * rel * R;
                            const float tR = R + eL;
                            bool in = cand && r2 < tR * tR * (1.f + 4.f * rel);
                            if (!near) {
                                // kept pairs of the near list take the exact test when evaluated
                                const float sR = fmaxf(R - eL, 0.f);
                                const bool band = in && !(r2 < sR * sR * (1.f - 4.f * rel));
                                if (__any_sync(0xffffffffu, band)) {
                                    if (band) in = exact_in(q);
                                }
                            }
                            c_tests += __popc(__ballot_sync(0xffffffffu, cand));
                            const unsigned hm = __ballot_sync(0xffffffffu, in);
                            if (near) {
                                if (in) {
                                    const int k = nnear + __popc(hm & lt);
                                    if (k < kWppNear) {
                                        sm.hit.n.d[k] = make_float2(r2, m);
                                        sm.hit.n.j[k] = q;
                                    }
                                }
                                nnear += __popc(hm);
                                continue;
                            }
                            if (in) {
                                sm.hit.n.d[nh + __popc(hm & lt)] = make_float2(r2, m);
                                if (q != p) {
                                    ++nn;
                                    if (HASH) hs += splitmix64((unsigned long long)a.perm[q]);
                                }
                            }
                            nh += __popc(hm);
                            if (nh >= 32) {
                                drain(32);
                                nh -= 32;
                                if ((int)lane < nh) sm.hit.n.d[lane] = sm.hit.n.d[32 + lane];
                                __syncwarp();
                            }
                        }
                        __syncwarp();
                    };
                    const bool rewalk = !complete || !(h <= Rw * 0.99999f);
                    if (rewalk) {
                        Rw = a.fixed_h ? h : h * kWppWalkR;
                        nlf = 0;
                        nnear = 0;
                        complete = true;
                        // a walk that overflows the leaf list evaluates its leaves at h as it goes
                        if (first && ngl >= 0)
                            wpp_filter(sm, ngl, B, a.node_c, a.node_e, Xi, sf, nlf, complete,
                                       [&](float4) { return Rw; }, [&]() { process(false); nlf = 0; });
                        else
                            wpp_walk(sm, B, a.node_c, a.node_e, Xi, sf, nlf, complete, [&](float4) { return Rw; },
                                     [&]() { process(false); nlf = 0; });
                        first = false;
                        near_ok = false;
                        if (complete) {
                            float eb = 0.f;
                            for (int k = (int)lane; k < nlf; k += 32) eb = fmaxf(eb, sm.lof[k].w);
                            ebmax = warp_max(eb);
                            process(true);
                            near_ok = nnear <= kWppNear;
                        }
                    }
                    if (near_ok) {
                        // every pair within Rw is in the near list: the exact test at h
                        const float eL = ebmax + 2.f * rel * h;
                        const float hi2 = (h + eL) * (h + eL) * (1.f + 4.f * rel);
                        const float lo2 = h > eL ? (h - eL) * (h - eL) * (1.f - 4.f * rel) : 0.f;
                        for (int k = (int)lane; k < nnear; k += 32) {
                            const float2 e = sm.hit.n.d[k];
                            if (e.x < hi2) {
                                const int q = sm.hit.n.j[k];
                                if (e.x < lo2 || exact_in(q)) {
                                    term(e.x, e.y);
                                    if (q != p) {
                                        ++nn;
                                        if (HASH) hs += splitmix64((unsigned long long)a.perm[q]);
                                    }
                                }
                            }
                        }
                    } else {
                        process(false);
                        drain(nh);
                    }
                    ++c_evals;
                    float Cw, Cdw;
                    wpp_fold2(Sw, Sdw, Sw, Cw, Sdw, Cdw);
                    // 3 (N_eff - N_t) = (32 S - 3 N_t) - 32 C: the scalings by 32 are exact
                    const float f3 = __fsub_rn(__fsub_rn(32.f * Sw, nt3), 32.f * Cw);
                    bool done = false;
                    if (a.fixed_h || fabsf(f3) <= tol3) {
                        done = true;
                    } else if (it >= a.max_iter) {
                        done = true;
                        st |= ST_NOT_CONVERGED;
                    } else {
                        const float N = (32.f / 3.f) * __fsub_rn(Sw, Cw);
                        const float dN = -(32.f / 3.f) * __fsub_rn(Sdw, Cdw) / h;
                        if (!wpp_h_update(h, f3, N, dN, nt, B.capu, blo, bhi, dold, st)) done = true;
                    }
                    if (done) break;
                }
                float Cmw, Cmdw;
                wpp_fold2(Smw, Smdw, Smw, Cmw, Smdw, Cmdw);
                nn = warp_sum(nn);
                if (HASH) hs = warp_sum(hs);
                if (a.nbr || DIVCURL) {
                    // Enumerate the neighbour set {j != i : r_ij < h_i} at the final h
                    // again, with the same exact predicate, from the near list, the leaf
                    // list, or a fresh walk, whichever the final evaluation relied on:
                    // - to record it for the force pass (nn entries, reserved from the
                    //   warp's chunk of the list pool);
                    // - to sum the velocity divergence and curl over it.
                    int loff = -1;
                    if (a.nbr) {
                        if (nn > a.list_chunk) {
                            unsigned long long o = 0;
                            if (lane == 0) o = atomicAdd(reinterpret_cast<unsigned long long*>(a.list_st + 4),
                                                         (unsigned long long)nn);
                            o = __shfl_sync(0xffffffffu, o, 0);
                            if ((long long)o + nn <= a.list_pool) loff = (int)o;
                        } else {
                            if (ch_next + nn > ch_end) {
                                unsigned long long o = 0;
                                if (lane == 0) o = atomicAdd(reinterpret_cast<unsigned long long*>(a.list_st + 4),
                                                             (unsigned long long)a.list_chunk);
                                o = __shfl_sync(0xffffffffu, o, 0);
                                ch_next = (long long)o;
                                ch_end = ch_next + a.list_chunk;
                            }
                            if (ch_next + nn <= a.list_pool) loff = (int)ch_next;
                            ch_next += nn;
                        }
                    }
                    const bool rec = loff >= 0 && nn > 0;
                    // per-lane sums of m_j w'(q)/r (v_ij . r_ij) and (v_ij x r_ij)
                    float Dd = 0.f, Dx = 0.f, Dy = 0.f, Dz = 0.f;
                    if (rec || DIVCURL) {
                        int32_t* dst = rec ? a.nbr + loff : nullptr;
                        int pos = 0;
                        double HHf = -1.0;
                        const float hinv = 1.f / h;
                        const float4 vi = DIVCURL ? a.vpack[p] : make_float4(0.f, 0.f, 0.f, 0.f);
                        auto exact_f = [&](int q) {
                            if (HHf < 0.0) HHf = wpp_hh(h, B.L);
                            return exact_pred(exact_d2(Xi, a.posm[q]), HHf);
                        };
                        // d = x_j - x_i; r_ij = -d, v_ij = v_i - v_j
                        auto vterm = [&](float dx, float dy, float dz, int q) {
                            const float r2 = dx * dx + dy * dy + dz * dz;
                            if (!(r2 > 0.f)) return;   // coincident: no direction
                            const float rinv = rsqrtf(r2);
                            float w_, dw;
                            spline<float>(r2 * rinv * hinv, w_, dw);
                            const float4 vj = __ldg(a.vpack + q);
                            const float g = vj.w * dw * rinv;
                            const float vx = vi.x - vj.x, vy = vi.y - vj.y, vz = vi.z - vj.z;
                            Dd -= g * (vx * dx + vy * dy + vz * dz);
                            Dx -= g * (vy * dz - vz * dy);
                            Dy -= g * (vz * dx - vx * dz);
                            Dz -= g * (vx * dy - vy * dx);
                        };
                        auto put = [&](bool in, int q, float dx, float dy, float dz) {
                            if (DIVCURL && in) vterm(dx, dy, dz, q);
                            if (rec) {
                                const unsigned hm = __ballot_sync(0xffffffffu, in);
                                if (in) {
                                    const int k = pos + __popc(hm & lt);
                                    if (k < nn) dst[k] = q;
                                }
                                pos += __popc(hm);
                            }
                        };
                        if (near_ok) {
                            const float eL = ebmax + 2.f * rel * h;
                            const float hi2 = (h + eL) * (h + eL) * (1.f + 4.f * rel);
                            const float lo2 = h > eL ? (h - eL) * (h - eL) * (1.f - 4.f * rel) : 0.f;
                            for (int k0 = 0; k0 < nnear; k0 += 32) {
                                const int k = k0 + (int)lane;
                                bool in = false;
                                int q = p;
                                float dx = 0.f, dy = 0.f, dz = 0.f;
                                if (k < nnear) {
                                    const float r2 = sm.hit.n.d[k].x;
                                    q = sm.hit.n.j[k];
                                    in = q != p && r2 < hi2 && (r2 < lo2 || exact_f(q));
                                    if (DIVCURL && in) {
                                        const uint4 Xj = a.posm[q];
                                        dx = (float)(int)(Xj.x - Xi.x) * sf;
                                        dy = (float)(int)(Xj.y - Xi.y) * sf;
                                        dz = (float)(int)(Xj.z - Xi.z) * sf;
                                    }
                                }
                                put(in, q, dx, dy, dz);
                            }
                        } else {
                            // the candidates of the leaf list at h, as process(false) tests them
                            auto record = [&]() {
                                for (int base = 0; base < nlf; base += 4) {
                                    const int li = base + (int)(lane >> 3);
                                    const int id = sm.lid[li];
                                    const float4 o = sm.lof[li];
                                    const int qq = off + (id & 0x7fffffff) * kLeaf + (int)(lane & 7u);
                                    const bool cand = li < nlf && qq < pend;
                                    const int q = cand ? qq : p;
                                    const float4 f = __ldg(a.posf + q);
                                    float dx = o.x + f.x, dy = o.y + f.y, dz = o.z + f.z;
                                    if (__any_sync(0xffffffffu, cand && id < 0)) {
                                        if (cand && id < 0) {
                                            const uint4 Xj = a.posm[q];
                                            dx = (float)(int)(Xj.x - Xi.x) * sf;
                                            dy = (float)(int)(Xj.y - Xi.y) * sf;
                                            dz = (float)(int)(Xj.z - Xi.z) * sf;
                                        }
                                    }
                                    const float r2 = dx * dx + dy * dy + dz * dz;
                                    const float eL = o.w + 2.f * rel * h;
                                    const float tR = h + eL, sR = fmaxf(h - eL, 0.f);
                                    bool in = cand && q != p && r2 < tR * tR * (1.f + 4.f * rel);
                                    const bool band = in && !(r2 < sR * sR * (1.f - 4.f * rel));
                                    if (__any_sync(0xffffffffu, band)) {
                                        if (band) in = exact_f(q);
                                    }
                                    put(in, q, dx, dy, dz);
                                }
                            };
                            if (!complete) {
                                nlf = 0;
                                complete = true;
                                wpp_walk(sm, B, a.node_c, a.node_e, Xi, sf, nlf, complete, [&](float4) { return h; },
                                         [&]() { record(); nlf = 0; });
                            }
                            record();
                        }
                        if (rec && pos != nn) loff = -1;   // cannot happen: the same predicate counted nn
                    }
                    if (a.nbr) {
                        if (lane == 0) {
                            a.nbr_off[p] = loff >= 0 ? loff : 0;
                            a.nbr_n[p] = loff >= 0 ? nn : -1;
                            a.list_h[p] = h;
                        }
                        ++c_lists;
                    }
                    if (DIVCURL) {
                        // div = -(1/rho) sum m v_ij . grad W, curl = |(1/rho) sum m v_ij x grad W|,
                        // grad_i W = 8/(pi h^4) w'(q) r_ij / r
                        const float fs = wpp_fold4(Dd, Dx, Dy, Dz);
                        const float sd = __shfl_sync(0xffffffffu, fs, 0), sx = __shfl_sync(0xffffffffu, fs, 8),
                                    sy = __shfl_sync(0xffffffffu, fs, 16), sz = __shfl_sync(0xffffffffu, fs, 24);
                        if (lane == 0) {
                            const float hinv = 1.f / h;
                            const float rho = 2.5464790894703255f * __fsub_rn(Smw, Cmw) * hinv_cube(h);
                            const float nr = 2.5464790894703255f * hinv_cube(h) * hinv / rho;
                            a.divv[oi] = -nr * sd;
                            a.curlv[oi] = nr * sqrtf(sx * sx + sy * sy + sz * sz);
                        }
                    }
                }
                if (lane == 0) {
                    const float smw = __fsub_rn(Smw, Cmw), smdw = __fsub_rn(Smdw, Cmdw);
                    a.h[oi] = h;
                    a.rho[oi] = 2.5464790894703255f * smw * hinv_cube(h);   // 8/(pi h^3) sum m w
                    a.omega[oi] = smdw != 0.f ? -3.f * smw / smdw : 1.f;
                    a.n_ngb[oi] = nn;
                    a.flags[oi] = (uint8_t)st;
                    if (HASH) a.hash[oi] = hs;
                    c_pairs += (unsigned)nn;
                    c_status |= st;
                }
                __syncwarp();
            }
        }
    }
    const unsigned long long all_tests = c_tests;   // counted warp-uniformly
    if (lane == 0) {
        if (a.nbr && c_lists) atomicAdd(&a.list_st[0], c_lists);
        atomicAdd(&a.ctr->density_pairs, (unsigned long long)c_pairs);
        atomicAdd(&a.ctr->density_evals, (unsigned long long)c_evals);
        atomicAdd(&a.ctr->pair_tests, all_tests);
        if (c_status) atomicOr(&a.ctr->status, c_status);
    }
}

// ---------------------------------------------------------------------------
// Force
// ---------------------------------------------------------------------------

template <bool HASH, int MINB, bool BAL, bool COND>
__global__ void __launch_bounds__(kWppThreads, MINB) k_force_wpp(WppArgs a) {
    __shared__ WppSmem smem[kWppWarps];
    WppSmem& sm = smem[threadIdx.x >> 5];
    const unsigned lane = lane_id();
    const unsigned lt = (1u << lane) - 1u;
    const float rel = 9.5367431640625e-07f;
    const float elo = 1.f - 4.f * rel, ehi = 1.f + 4.f * rel;
    const float kNorm = (float)(8.0 / 3.141592653589793);
    const float alpha = a.alpha;
    // after a list pass: only the particles the lists could not serve, one per
    // queue grab (walked alone), unless the lists could not serve the call
    const int32_t* act = a.act;
    int cnt = (int)*a.count_ptr, chunk = a.chunk;
    if (a.fb_act && wpp_lists_valid(a.list_st, a.n_total)) {
        act = a.fb_act;
        cnt = (int)*a.fb_count;
        chunk = 1;
    }
    unsigned long long c_pairs = 0, c_tests = 0;   // lane 0's per-warp totals
    for (;;) {
        int t0 = 0;
        if (lane == 0) t0 = (int)atomicAdd(a.queue, (unsigned)chunk);
        t0 = __shfl_sync(0xffffffffu, t0, 0);
        if (t0 >= cnt) break;
        const int t1 = min(t0 + chunk, cnt);
        for (int t = t0; t < t1;) {
            const WppGroup G = wpp_group(a.boxes, a.n_boxes, act, t, t1);
            t += G.n;
            const BoxDesc& B = a.boxes[G.box];
            const float sf = B.sf;
            const int off = (int)B.off, pend = (int)(B.off + B.n);
            // one shared walk for the group (radius: the largest member h)
            uint4 Xl = make_uint4(0u, 0u, 0u, 0u);
            float hl = 0.f;
            if (G.p >= 0) {
                Xl = a.posm[G.p];
                hl = a.fvel[G.p].w;
            }
            int ngl = -1;
            if (G.n >= 2 && B.nlev > 1) {
                const float hg = warp_max(hl);
                ngl = wpp_group_leaves(sm, B, a.node_c, a.node_e, Xl, G.p >= 0, sf,
                                       [&](float4 e) { return fmaxf(hg, e.w); });
            }
            for (int m = 0; m < G.n; ++m) {
                const int p = __shfl_sync(0xffffffffu, G.p, m);
                const uint4 Xi = make_uint4(__shfl_sync(0xffffffffu, Xl.x, m), __shfl_sync(0xffffffffu, Xl.y, m),
                                            __shfl_sync(0xffffffffu, Xl.z, m), __shfl_sync(0xffffffffu, Xl.w, m));
                const float hi = __shfl_sync(0xffffffffu, hl, m);
                const int oi = a.perm[p];
                const float4 vi = a.fvm[p];
                const float4 thi = a.fthermo[p];
                const float2 ci = COND ? a.fcond[p] : make_float2(0.f, 0.f);
                const WppForceI I = {vi.x, vi.y, vi.z, thi.w, thi.x, thi.y, thi.z,
                                     kNorm * thi.w * thi.w * thi.w * thi.w, BAL ? a.fbal[p] : 1.f, ci.x, ci.y};
                // i side of the band test: h_i (1 +- 2^-19) (the leaf's rounding bound is added per leaf)
                const float hiP = hi * (1.f + 2.f * rel), hiM = hi * (1.f - 2.f * rel);
                double HHi = -1.0;
                float Sx = 0.f, Sy = 0.f, Sz = 0.f, Su = 0.f, Sc = 0.f, vsmax = 0.f;   // per-lane partial sums
                int np = 0, nh = 0, nlf = 0;
                unsigned tests = 0;
                bool complete = true;
                unsigned long long hs = 0;
                // pair terms of hit-buffer entries [0, k), one per lane
                auto drain = [&](int k) {
                    __syncwarp();
                    if ((int)lane < k) {
                        const float4 e = sm.hit.f[lane];
                        const int q = __float_as_int(e.w);
                        wpp_force_pair<BAL, COND>(I, e.x, e.y, e.z, __ldg(a.fvm + q), __ldg(a.fthermo + q),
                                                  BAL ? __ldg(a.fbal + q) : 1.f,
                                                  COND ? __ldg(a.fcond + q) : make_float2(0.f, 0.f), alpha, Sx, Sy,
                                                  Sz, Su, Sc, vsmax);
                    }
                    __syncwarp();
                };
                // Tests the candidates of leaf list entries [0, nlf), 32 per step
                // (lanes 8k..8k+7: the particles of the step's k-th leaf). A pair
                // is in the set when r < h_i or r < h_j; r^2 is tested in FP32
                // against each radius widened and narrowed by the leaf's rounding
                // bound, and only pairs inside that thin band take the exact
                // integer/FP64 predicate.
                auto process = [&]() {
                    for (int base = 0; base < nlf; base += 4) {
                        // li <= 127 < kWppLeaves: entries past nlf are stale but in
                        // bounds; lanes without a candidate read particle p itself
                        const int li = base + (int)(lane >> 3);
                        const int id = sm.lid[li];
                        const float4 o = sm.lof[li];
                        const int qq = off + (id & 0x7fffffff) * kLeaf + (int)(lane & 7u);
                        const bool cand = li < nlf && qq < pend;
                        const int q = cand ? qq : p;
                        const bool ok = cand && q != p;
                        const float4 f = __ldg(a.fposh + q);
                        float dx = o.x + f.x, dy = o.y + f.y, dz = o.z + f.z;
                        if (__any_sync(0xffffffffu, ok && id < 0)) {
                            if (ok && id < 0) {   // wide leaf: exact integer separations
                                const uint4 Xj = a.posm[q];
                                dx = (float)(int)(Xj.x - Xi.x) * sf;
                                dy = (float)(int)(Xj.y - Xi.y) * sf;
                                dz = (float)(int)(Xj.z - Xi.z) * sf;
                            }
                        }
                        const float r2 = dx * dx + dy * dy + dz * dz;
                        const float si = fmaxf(hiM - o.w, 0.f), sj = fmaxf(fmaf(f.w, 1.f - 2.f * rel, -o.w), 0.f);
                        bool in = ok && (r2 < si * si * elo || r2 < sj * sj * elo);
                        const float ti = hiP + o.w, tj = fmaf(f.w, 1.f + 2.f * rel, o.w);
                        const bool mi = r2 < ti * ti * ehi, mj = r2 < tj * tj * ehi;
                        const bool band = ok && !in && (mi || mj);
                        if (__any_sync(0xffffffffu, band)) {
                            if (band) {
                                const unsigned long long D2 = exact_d2(Xi, a.posm[q]);
                                if (mi) {
                                    if (HHi < 0.0) HHi = wpp_hh(hi, B.L);
                                    in = exact_pred(D2, HHi);
                                }
                                if (!in && mj) in = exact_pred(D2, wpp_hh(f.w, B.L));
                            }
                        }
                        tests += __popc(__ballot_sync(0xffffffffu, cand));
                        const unsigned hm = __ballot_sync(0xffffffffu, in);
                        if (in) {
                            sm.hit.f[nh + __popc(hm & lt)] = make_float4(dx, dy, dz, __int_as_float(q));
                            if (HASH) hs += splitmix64((unsigned long long)a.perm[q]);
                        }
                        np += __popc(hm);
                        nh += __popc(hm);
                        if (nh >= 32) {
                            drain(32);
                            nh -= 32;
                            if ((int)lane < nh) sm.hit.f[lane] = sm.hit.f[32 + lane];
                            __syncwarp();
                        }
                    }
                };
                if (ngl >= 0)
                    wpp_filter(sm, ngl, B, a.node_c, a.node_e, Xi, sf, nlf, complete,
                               [&](float4 e) { return fmaxf(hi, e.w); }, [&]() { process(); nlf = 0; });
                else
                    wpp_walk(sm, B, a.node_c, a.node_e, Xi, sf, nlf, complete, [&](float4 e) { return fmaxf(hi, e.w); },
                             [&]() { process(); nlf = 0; });
                process();
                drain(nh);
                // fold the per-lane sums: lanes 0-7 end with acc.x, 8-15 acc.y,
                // 16-23 acc.z, 24-31 du/dt
                const float fs = wpp_fold4(Sx, Sy, Sz, Su);
                vsmax = warp_max(vsmax);
                if (HASH) hs = warp_sum(hs);
                if ((lane & 7u) == 0u) {
                    const int comp = (int)(lane >> 3);
                    if (comp < 3) a.acc[3 * (size_t)oi + comp] = fs;
                    else a.dudt[oi] = fs;
                }
                if (COND) {
                    float cs, cc, z0, z1;
                    wpp_fold2(Sc, 0.f, cs, cc, z0, z1);
                    if (lane == 0) a.dudt_cond[oi] = __fsub_rn(cs, cc);
                }
                if (lane == 0) {
                    a.vsig[oi] = vsmax;
                    if (HASH) a.hash[oi] = hs;
                    c_pairs += (unsigned long long)np;
                    c_tests += tests;
                }
                __syncwarp();
            }
        }
    }
    if (lane == 0) {
        atomicAdd(&a.ctr->force_pairs, c_pairs);
        atomicAdd(&a.ctr->pair_tests, c_tests);
    }
}

// ---------------------------------------------------------------------------
// Neighbour lists reused by the force pass
// ---------------------------------------------------------------------------
//
// The force pair set of i is {j != i : r_ij < h_i} U {j : r_ij < h_j}. An
// all-active density pass records the first part per particle (its neighbour
// list at the converged h). The second part, minus what the first already
// holds, is the transpose: j is an extra partner of i when i is on j's list
// and r_ij >= h_i. k_list_ext scatters those, k_list_sort puts each extra list
// in ascending order (the scatter's order depends on scheduling; the sorted
// order makes the force sums deterministic), and k_force_list evaluates the
// pair terms straight from the two lists: no walk and no candidate tests.

// Warp per particle j: every i on j's list with r_ij >= h_i gets j as an
// extra partner (possible only if h_i < h_j, which is tested first). "r_ij <
// h_i" is the exact predicate, decided in FP32 outside a band of 2^-20 around
// h_i^2 and in FP64 inside it. COUNT = true counts each i's extra partners in
// ext_n and marks the list entries that make one in nbr_x; COUNT = false
// places the marked pairs in i's segment [ext_off[i], ext_off[i+1]) of
// ext_raw (scatter order; ext_n counts down to 0).
template <bool COUNT>
__global__ void __launch_bounds__(256) k_list_ext(const BoxDesc* __restrict__ boxes, int nb, int n,
                                                  const uint4* __restrict__ posm, const int32_t* __restrict__ nbr,
                                                  const int32_t* __restrict__ nbr_off,
                                                  const int32_t* __restrict__ nbr_n, uint8_t* __restrict__ nbr_x,
                                                  const float* __restrict__ list_h, uint32_t* __restrict__ ext_n,
                                                  const uint32_t* __restrict__ ext_off, int32_t* __restrict__ ext_raw,
                                                  unsigned ext_pool, unsigned* list_st) {
    const unsigned lane = lane_id();
    const int warps = gridDim.x * (blockDim.x >> 5);
    const float band = 9.5367431640625e-07f;  // 2^-20
    for (int j = blockIdx.x * (blockDim.x >> 5) + (int)(threadIdx.x >> 5); j < n; j += warps) {
        const int cnt = nbr_n[j];
        if (cnt < 0) {   // j's list is missing: the extra lists cannot be completed
            if (COUNT && lane == 0) atomicOr(&list_st[1], 1u);
            continue;
        }
        const int off = nbr_off[j];
        const int32_t* lj = nbr + off;
        if (COUNT) {
            const BoxDesc& B = boxes[nb == 1 ? 0 : wpp_box(boxes, nb, j)];
            const float Hs = (float)(4294967296.0 / B.L);   // integer units per box unit
            const uint4 Xj = posm[j];
            const float hj = list_h[j];
            auto decide = [&](int i, float hi, uint4 Xi) {
                bool x = false;
                if (hi < hj) {
                    const unsigned long long D2 = exact_d2(Xi, Xj);
                    const float d2 = __ull2float_rn(D2), Hi = hi * Hs, H2 = Hi * Hi;
                    if (d2 > H2 * (1.f + band)) x = true;
                    else if (!(d2 < H2 * (1.f - band))) x = !exact_pred(D2, wpp_hh(hi, B.L));
                }
                return x;
            };
            // two entries per lane per step (k and k + 32), their gathers issued together
            for (int k = (int)lane; k < cnt; k += 64) {
                const int k1 = k + 32;
                const bool two = k1 < cnt;
                const int i0 = lj[k], i1 = two ? lj[k1] : i0;
                const float h0 = list_h[i0], h1 = list_h[i1];
                const uint4 X0 = h0 < hj ? posm[i0] : Xj, X1 = (two && h1 < hj) ? posm[i1] : Xj;
                const bool x0 = decide(i0, h0, X0);
                nbr_x[off + k] = x0 ? 1 : 0;
                if (x0) atomicAdd(&ext_n[i0], 1u);
                if (two) {
                    const bool x1 = decide(i1, h1, X1);
                    nbr_x[off + k1] = x1 ? 1 : 0;
                    if (x1) atomicAdd(&ext_n[i1], 1u);
                }
            }
        } else {
            for (int k = (int)lane; k < cnt; k += 32) {
                if (!nbr_x[off + k]) continue;
                const int i = lj[k];
                if (ext_off[i + 1] <= ext_pool) {
                    const unsigned pos = atomicSub(&ext_n[i], 1u) - 1u;
                    ext_raw[ext_off[i] + pos] = j;
                }
            }
        }
    }
}

// Warp per particle: its extra partners (distinct indices) in ascending
// order. Up to 64 entries: each placed at its rank (registers); up to
// kSortMax: a bitonic sort in shared memory; longer segments (and segments
// that did not fit the pool) are marked in ext_n (nonzero), and the force
// pass walks for those particles.
constexpr int kSortMax = 1024;

__global__ void __launch_bounds__(256) k_list_sort(int n, const uint32_t* __restrict__ ext_off, unsigned ext_pool,
                                                   const int32_t* __restrict__ ext_raw, int32_t* __restrict__ ext,
                                                   uint32_t* __restrict__ ext_n) {
    __shared__ int buf[8][kSortMax];
    int* sb = buf[threadIdx.x >> 5];
    const unsigned lane = lane_id();
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int i = blockIdx.x * (blockDim.x >> 5) + (int)(threadIdx.x >> 5); i < n; i += warps) {
        const unsigned b = ext_off[i], e = ext_off[i + 1];
        if (e > ext_pool || e == b) continue;
        const int c = (int)(e - b);
        const int32_t* src = ext_raw + b;
        int32_t* dst = ext + b;
        if (c <= 64) {
            const int v0 = (int)lane < c ? src[lane] : 0x7fffffff;
            const int v1 = (int)lane + 32 < c ? src[lane + 32] : 0x7fffffff;
            int r0 = 0, r1 = 0;
            const int c0 = min(c, 32);
            for (int k = 0; k < c0; ++k) {
                const int x = __shfl_sync(0xffffffffu, v0, k);
                r0 += x < v0;
                r1 += x < v1;
            }
            for (int k = 32; k < c; ++k) {
                const int x = __shfl_sync(0xffffffffu, v1, k - 32);
                r0 += x < v0;
                r1 += x < v1;
            }
            if ((int)lane < c) dst[r0] = v0;
            if ((int)lane + 32 < c) dst[r1] = v1;
        } else if (c <= kSortMax) {
            int P = 128;
            while (P < c) P <<= 1;
            for (int k = (int)lane; k < P; k += 32) sb[k] = k < c ? src[k] : 0x7fffffff;
            __syncwarp();
            for (int size = 2; size <= P; size <<= 1) {
                for (int stride = size >> 1; stride > 0; stride >>= 1) {
                    for (int t = (int)lane; t < (P >> 1); t += 32) {
                        const int lo = ((t & ~(stride - 1)) << 1) | (t & (stride - 1));
                        const int hi = lo + stride;
                        const int x = sb[lo], y = sb[hi];
                        if ((x > y) == ((lo & size) == 0)) {
                            sb[lo] = y;
                            sb[hi] = x;
                        }
                    }
                    __syncwarp();
                }
            }
            for (int k = (int)lane; k < c; k += 32) dst[k] = sb[k];
            __syncwarp();
        } else if (lane == 0) {
            ext_n[i] = 1u;   // too long to sort here: walked by the force pass
        }
    }
}

// Force pass from the recorded lists: warp per active particle, pairs 32 at a
// time (the neighbour list, then the extra partners), the same pair terms and
// fold as k_force_wpp. If the lists cannot serve the call at all the kernel
// does nothing and the walk that follows takes the whole active set;
// particles whose own lists did not fit go to fb_list for that walk.
template <bool HASH, bool BAL, bool COND>
__global__ void __launch_bounds__(128) k_force_list(WppArgs a) {
    if (!wpp_lists_valid(a.list_st, a.n_total)) return;
    const unsigned lane = lane_id();
    const int warps = gridDim.x * (blockDim.x >> 5);
    const int cnt = (int)*a.count_ptr;
    const float kNorm = (float)(8.0 / 3.141592653589793);
    unsigned long long c_pairs = 0;   // per warp, lane-uniform
    for (int t = blockIdx.x * (blockDim.x >> 5) + (int)(threadIdx.x >> 5); t < cnt; t += warps) {
        const int p = a.act[t];
        const int cn = a.nbr_n[p];
        const unsigned e0 = a.ext_off[p], e1 = a.ext_off[p + 1];
        if (cn < 0 || e1 > a.ext_pool || a.ext_n[p] != 0u) {
            if (lane == 0) a.fb_list[atomicAdd(&a.list_st[3], 1u)] = p;
            continue;
        }
        const BoxDesc& B = a.boxes[a.n_boxes == 1 ? 0 : wpp_box(a.boxes, a.n_boxes, p)];
        const float sf = B.sf;
        const uint4 Xi = a.posm[p];
        const int oi = a.perm[p];
        const float4 vi = a.fvm[p];
        const float4 thi = a.fthermo[p];
        const float2 ci = COND ? a.fcond[p] : make_float2(0.f, 0.f);
        const WppForceI I = {vi.x, vi.y, vi.z, thi.w, thi.x, thi.y, thi.z, kNorm * thi.w * thi.w * thi.w * thi.w,
                             BAL ? a.fbal[p] : 1.f, ci.x, ci.y};
        float Sx = 0.f, Sy = 0.f, Sz = 0.f, Su = 0.f, Sc = 0.f, vsmax = 0.f;
        unsigned long long hs = 0;
        const int tot = cn + (int)(e1 - e0);
        const int32_t* ln = a.nbr + a.nbr_off[p];
        const int32_t* le = a.ext + e0;
        // two pairs per lane per step (k and k + 32), their loads issued together;
        // each lane still sums its pairs in the order k, k + 32, k + 64, ...
        for (int k = (int)lane; k < tot; k += 64) {
            const int k1 = k + 32;
            const bool two = k1 < tot;
            const int q0 = k < cn ? ln[k] : le[k - cn];
            const int q1 = two ? (k1 < cn ? ln[k1] : le[k1 - cn]) : q0;
            const uint4 X0 = a.posm[q0], X1 = a.posm[q1];
            const float4 v0 = __ldg(a.fvm + q0), v1 = __ldg(a.fvm + q1);
            const float4 t0 = __ldg(a.fthermo + q0), t1 = __ldg(a.fthermo + q1);
            const float b0 = BAL ? __ldg(a.fbal + q0) : 1.f, b1 = BAL ? __ldg(a.fbal + q1) : 1.f;
            const float2 c0 = COND ? __ldg(a.fcond + q0) : make_float2(0.f, 0.f);
            const float2 c1 = COND ? __ldg(a.fcond + q1) : make_float2(0.f, 0.f);
            wpp_force_pair<BAL, COND>(I, (float)(int)(X0.x - Xi.x) * sf, (float)(int)(X0.y - Xi.y) * sf,
                                      (float)(int)(X0.z - Xi.z) * sf, v0, t0, b0, c0, a.alpha, Sx, Sy, Sz, Su, Sc,
                                      vsmax);
            if (HASH) hs += splitmix64((unsigned long long)a.perm[q0]);
            if (two) {
                wpp_force_pair<BAL, COND>(I, (float)(int)(X1.x - Xi.x) * sf, (float)(int)(X1.y - Xi.y) * sf,
                                          (float)(int)(X1.z - Xi.z) * sf, v1, t1, b1, c1, a.alpha, Sx, Sy, Sz, Su, Sc,
                                          vsmax);
                if (HASH) hs += splitmix64((unsigned long long)a.perm[q1]);
            }
        }
        const float fs = wpp_fold4(Sx, Sy, Sz, Su);
        vsmax = warp_max(vsmax);
        if (HASH) hs = warp_sum(hs);
        if ((lane & 7u) == 0u) {
            const int comp = (int)(lane >> 3);
            if (comp < 3) a.acc[3 * (size_t)oi + comp] = fs;
            else a.dudt[oi] = fs;
        }
        if (COND) {
            float cs, cc, z0, z1;
            wpp_fold2(Sc, 0.f, cs, cc, z0, z1);
            if (lane == 0) a.dudt_cond[oi] = __fsub_rn(cs, cc);
        }
        if (lane == 0) {
            a.vsig[oi] = vsmax;
            if (HASH) a.hash[oi] = hs;
        }
        c_pairs += (unsigned long long)tot;
    }
    if (lane == 0 && c_pairs) atomicAdd(&a.ctr->force_pairs, c_pairs);
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------

// SPH_TIME_KERNELS: an event pair around a span of launches on stream s.
struct WppSpan {
    cudaEvent_t a = nullptr;
    int kind = 0;
};

static cudaError_t span_begin(sph_ctx* ctx, int timed, int kind, cudaStream_t s, WppSpan& sp) {
    sp.kind = kind;
    if (!timed) return cudaSuccess;
    sp.a = timing_event(ctx);
    if (!sp.a) return cudaErrorMemoryAllocation;
    return cudaEventRecord(sp.a, s);
}

static cudaError_t span_end(sph_ctx* ctx, const WppSpan& sp, cudaStream_t s) {
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
static void wpp_shape(sph_ctx* ctx, int bps, int64_t n_active, int& blocks, int& chunk) {
    const int b = std::min(bps, kWppMaxBps);
    const long long warps_needed = std::max<long long>(1, n_active);
    const long long want_blocks = (warps_needed + kWppWarps - 1) / kWppWarps;
    blocks = (int)std::max<long long>(1, std::min<long long>((long long)ctx->sm_count * b, want_blocks));
    const long long warps = (long long)blocks * kWppWarps;
    chunk = (int)std::max<long long>(1, std::min<long long>(8, n_active / (warps * 4)));
}

static WppArgs wpp_common(sph_ctx* ctx, const sph_grid* g, unsigned* queue) {
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
    return c;
}

// Sorted (v, m) for the density pass's velocity divergence and curl.
__global__ void k_vel_pack(int n, const int32_t* __restrict__ perm, const float* __restrict__ vel,
                           const float4* __restrict__ posf, float4* __restrict__ vm) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const size_t o = (size_t)perm[p];
    vm[p] = make_float4(vel[3 * o], vel[3 * o + 1], vel[3 * o + 2], posf[p].w);
}

// Grid of a warp-per-particle helper kernel over n particles (256 threads).
static int helper_blocks(sph_ctx* ctx, int64_t n) {
    return (int)std::max<long long>(1, std::min<long long>((long long)ctx->sm_count * 8, (n + 7) / 8));
}

// Kernel variants of the force pass: hash output, register budget, Balsara's
// switch, conduction.
template <bool H, bool BAL, bool COND>
static void launch_fl(int blocks, cudaStream_t s, const WppArgs& c) {
    k_force_list<H, BAL, COND><<<blocks, 128, 0, s>>>(c);
}
static void launch_force_list(bool hash, bool bal, bool cond, int blocks, cudaStream_t s, const WppArgs& c) {
    if (hash) {
        if (bal) cond ? launch_fl<true, true, true>(blocks, s, c) : launch_fl<true, true, false>(blocks, s, c);
        else cond ? launch_fl<true, false, true>(blocks, s, c) : launch_fl<true, false, false>(blocks, s, c);
    } else {
        if (bal) cond ? launch_fl<false, true, true>(blocks, s, c) : launch_fl<false, true, false>(blocks, s, c);
        else cond ? launch_fl<false, false, true>(blocks, s, c) : launch_fl<false, false, false>(blocks, s, c);
    }
}
template <bool H, int M>
static void launch_fw(bool bal, bool cond, int blocks, cudaStream_t s, const WppArgs& c) {
    if (bal) {
        if (cond) k_force_wpp<H, M, true, true><<<blocks, kWppThreads, 0, s>>>(c);
        else k_force_wpp<H, M, true, false><<<blocks, kWppThreads, 0, s>>>(c);
    } else {
        if (cond) k_force_wpp<H, M, false, true><<<blocks, kWppThreads, 0, s>>>(c);
        else k_force_wpp<H, M, false, false><<<blocks, kWppThreads, 0, s>>>(c);
    }
}
static void launch_force_walk(bool hash, bool six, bool bal, bool cond, int blocks, cudaStream_t s,
                              const WppArgs& c) {
    if (six) hash ? launch_fw<true, 6>(bal, cond, blocks, s, c) : launch_fw<false, 6>(bal, cond, blocks, s, c);
    else hash ? launch_fw<true, 8>(bal, cond, blocks, s, c) : launch_fw<false, 8>(bal, cond, blocks, s, c);
}

cudaError_t launch_density_wpp(sph_ctx* ctx, const DensityLaunch& a, int64_t n_active, cudaStream_t s) {
    sph_grid* g = const_cast<sph_grid*>(a.g);
    cudaError_t e = cudaMemsetAsync(ctx->queue + 2, 0, sizeof(unsigned), s);
    if (e) return e;
    WppArgs c = wpp_common(ctx, g, ctx->queue + 2);
    int blocks = 0;
    const int bps = a.blocks_per_sm > 0 ? a.blocks_per_sm : kWppDensityBps;
    wpp_shape(ctx, bps, n_active, blocks, c.chunk);
    c.h = a.h;
    c.rho = a.rho;
    c.omega = a.omega;
    c.n_ngb = a.n_ngb;
    c.flags = a.flags;
    c.hash = a.hash;
    c.n_target = a.n_target;
    c.n_tol = a.n_tol;
    c.max_iter = a.max_iter;
    c.guess_h = a.guess_h;
    c.fixed_h = a.fixed_h;
    if (a.divv) {
        k_vel_pack<<<(int)((g->n + 255) / 256), 256, 0, s>>>((int)g->n, g->perm, a.vel, g->posf, g->fvm);
        ++ctx->launches;
        c.vpack = g->fvm;
        c.divv = a.divv;
        c.curlv = a.curlv;
    }
    // Neighbour lists: recorded when the active count can cover all particles.
    // They serve a force call only if every particle was in fact active
    // (checked on the device: lists written == n); a call on a smaller active
    // set leaves them unusable.
    const bool full = g->nbr != nullptr && n_active == g->n;
    if (full) {
        c.nbr = g->nbr;
        c.nbr_off = g->nbr_off;
        c.nbr_n = g->nbr_n;
        c.list_h = g->list_h;
        c.list_st = g->list_st;
        c.list_pool = g->list_pool;
        // chunks small enough that every warp's first reservations fit in a quarter of the pool
        const long long warps = (long long)blocks * kWppWarps;
        c.list_chunk = (int)std::max<long long>(32, std::min<long long>(kListChunk, g->list_pool / (4 * warps)));
        if ((e = cudaMemsetAsync(g->list_st, 0, sizeof(unsigned) * kListSt, s))) return e;
    }
    WppSpan sp;
    if ((e = span_begin(ctx, a.time_kernels, 0, s, sp))) return e;
    const bool dc = a.divv != nullptr;
    auto kd = bps <= 6 ? (a.hash ? (dc ? k_density_wpp<true, 6, true> : k_density_wpp<true, 6, false>)
                                 : (dc ? k_density_wpp<false, 6, true> : k_density_wpp<false, 6, false>))
                       : (a.hash ? (dc ? k_density_wpp<true, 8, true> : k_density_wpp<true, 8, false>)
                                 : (dc ? k_density_wpp<false, 8, true> : k_density_wpp<false, 8, false>));
    kd<<<blocks, kWppThreads, 0, s>>>(c);
    ++ctx->launches;
    // SPH_TIME_KERNELS times the density kernel alone; the list build follows
    if ((e = span_end(ctx, sp, s))) return e;
    if (full) {
        const int n = (int)g->n, hb = helper_blocks(ctx, n);
        const unsigned ep = (unsigned)g->ext_pool;
        if ((e = cudaMemsetAsync(g->ext_n, 0, sizeof(uint32_t) * n, s))) return e;
        k_list_ext<true><<<hb, 256, 0, s>>>(g->boxes, g->n_boxes, n, g->posm, g->nbr, g->nbr_off, g->nbr_n, g->nbr_x,
                                            g->list_h, g->ext_n, g->ext_off, g->ext_raw, ep, g->list_st);
        scan_exclusive<uint32_t>(g->ext_n, n, g->ext_off, g->scan_tmp, s, &ctx->launches);
        k_list_ext<false><<<hb, 256, 0, s>>>(g->boxes, g->n_boxes, n, g->posm, g->nbr, g->nbr_off, g->nbr_n, g->nbr_x,
                                             g->list_h, g->ext_n, g->ext_off, g->ext_raw, ep, g->list_st);
        k_list_sort<<<hb, 256, 0, s>>>(n, g->ext_off, ep, g->ext_raw, g->ext, g->ext_n);
        ctx->launches += 3;
    }
    g->lists_full = full;
    return cudaGetLastError();
}

cudaError_t launch_force_wpp(sph_ctx* ctx, const ForceLaunch& a, int64_t n_active, cudaStream_t s) {
    sph_grid* g = const_cast<sph_grid*>(a.g);
    cudaError_t e;
    const bool lists = g->nbr != nullptr && g->lists_full;
    if (lists && (e = cudaMemsetAsync(g->list_st + 2, 0, 2 * sizeof(unsigned), s))) return e;
    force_pack(g, a.vel, a.u, a.h, a.rho, a.omega, (float)a.gamma, s, lists ? g->list_h : nullptr,
               lists ? g->list_st + 2 : nullptr, a.divv, a.curlv, a.kappa);
    ++ctx->launches;
    if ((e = cudaMemsetAsync(ctx->queue + 3, 0, sizeof(unsigned), s))) return e;
    WppArgs c = wpp_common(ctx, g, ctx->queue + 3);
    int blocks = 0;
    const int bps = a.blocks_per_sm > 0 ? a.blocks_per_sm : kWppForceBps;
    wpp_shape(ctx, bps, n_active, blocks, c.chunk);
    c.fvel = g->fvel;
    c.fthermo = g->fthermo;
    c.fposh = g->fposh;
    c.fvm = g->fvm;
    c.acc = a.acc;
    c.dudt = a.dudt;
    c.vsig = a.vsig;
    c.alpha = (float)a.alpha;
    c.hash = a.hash;
    c.fbal = a.divv ? g->fbal : nullptr;
    c.fcond = a.kappa ? g->fcond : nullptr;
    c.dudt_cond = a.dudt_cond;
    WppSpan sp;
    if ((e = span_begin(ctx, a.time_kernels, 1, s, sp))) return e;
    if (lists) {
        // pairs from the recorded lists; the walk that follows takes the
        // particles they cannot serve (usually none), or every active particle
        // if the lists cannot serve this call
        c.nbr = g->nbr;
        c.nbr_off = g->nbr_off;
        c.nbr_n = g->nbr_n;
        c.ext = g->ext;
        c.ext_off = g->ext_off;
        c.ext_n = g->ext_n;
        c.ext_pool = (unsigned)g->ext_pool;
        c.list_st = g->list_st;
        c.fb_list = g->fb_list;
        const int lb = (int)std::max<long long>(
            1, std::min<long long>((long long)ctx->sm_count * 16, (n_active + 3) / 4));
        launch_force_list(a.hash != nullptr, c.fbal != nullptr, c.fcond != nullptr, lb, s, c);
        ++ctx->launches;
        c.fb_act = g->fb_list;
        c.fb_count = g->list_st + 3;
    }
    launch_force_walk(a.hash != nullptr, bps <= 6, c.fbal != nullptr, c.fcond != nullptr, blocks, s, c);
    ++ctx->launches;
    if ((e = span_end(ctx, sp, s))) return e;
    return cudaGetLastError();
}

}  // namespace sph
