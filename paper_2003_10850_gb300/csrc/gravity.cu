// gravity.cu -- short-range gravity of the TreePM split by a Barnes-Hut walk.
//
// The paper's code computes short-range gravity by Barnes-Hut: particles
// interact with distant tree nodes as point masses chosen by an opening
// criterion, and the interactions happen inside the walk (Sec. 1, Sec. 3).
// Long-range gravity (the particle mesh) is not part of this pass.
//
// The tree is the grid's hierarchy (a leaf is 8 consecutive Morton-sorted
// particles, a node 8 consecutive nodes of the level below). Its node boxes are
// exact integer boxes, so every decision of the walk is taken in exact integer
// arithmetic on coarse coordinates (integer coordinates >> 8), with no
// FP64 on the per-node or per-pair path:
//   D2 = sum_a G_a^2, G_a the periodic gap between X_i and the box on axis a;
//   F2 = sum_a F_a^2, F_a the periodic distance to the far side, rounded up;
//   L2 = l^2, l the box's largest side;  RCi = ceil((r_cut 2^24 / L)^2);
//   P = rint(theta^2 2^16).
// The root is always opened; a child of an opened node is skipped if
// D2 >= RCi, taken as its monopole if P > 0, D2 > 0, F2 < RCi, L2 <= D2 and
// 2^16 L2 <= P D2, and opened otherwise (a leaf: its particles one by one,
// each if its coarse distance is below RCi). D2 < RCi <= 2^44 and P <= 2^16
// keep the products below 2^60.
//
// One warp per active particle: each step pops up to four opened nodes and
// tests their children one per lane; opened leaves gather in a shared list
// whose particles are tested four leaves at a time (lanes 8k..8k+7 on leaf
// k). Accepted nodes and particles inside the cutoff are compacted by ballot
// into a per-warp interaction buffer that is evaluated 32 entries at a time,
// so the pair terms run with every lane busy. The pair term is
//   a_i += G m_j K(r) (x_j - x_i),  K(r) = M(r/h_s) g(r) / r^3,
// M the spline softening's mass fraction, g(r) = erfc(r/2r_s) + r/(r_s sqrt(pi))
// exp(-r^2/4r_s^2) the short-range factor (erfc to 1.5e-7, see grav_K).
#include <cmath>

#include "wpp.cuh"

namespace sph {

constexpr int kGravStack = 256;   // see the bound below
constexpr int kGravLeaves = 64;   // opened leaves waiting; <= 3 + 32 at any time
constexpr int kGravHits = 64;     // interactions waiting; <= 31 + 32 at any time

// Stack bound: a pop-4 step starts at sp <= 96 and pushes <= 32 children; in
// the pop-1 regime a step pushes <= 8 children of the node it pops, so the
// stack grows by at most 7 per level of depth-first descent:
// sp <= 124 + 7 kMaxLev < kGravStack.

struct GravArgs {
    const BoxDesc* boxes;
    int n_boxes;
    const int32_t* act;
    const uint32_t* count_ptr;
    unsigned* queue;
    const uint4* posm;
    const int32_t* perm;
    const uint4* node_lo;
    const uint4* node_hi;
    const uint4* node_c;
    const float4* node_m;   // centre of mass - node centre (box units), mass
    const unsigned long long* box_rci;   // per box: RCi
    float* acc;
    int32_t* n_nodes;
    int32_t* n_pairs;
    Counters* ctr;
    float G;
    unsigned long long P;    // rint(theta^2 2^16)
    float hs, inv_hs;        // softening radius (0: none)
    float inv2rs;            // 1 / (2 r_s); r_s <= 0: 0
};

// Leaf moments: mass and centre of mass relative to the node centre.
__global__ void k_grav_leaf_moments(const uint4* __restrict__ posm, const BoxDesc* __restrict__ boxes,
                                    const uint4* __restrict__ nc, float4* __restrict__ nm) {
    const BoxDesc& B = boxes[blockIdx.y];
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= B.lvl_n[0]) return;
    const long long p0 = B.off + (long long)t * kLeaf, p1 = min(p0 + kLeaf, B.off + B.n);
    const int nd = B.lvl_off[0] + t;
    const uint4 c = nc[nd];
    float M = 0.f, sx = 0.f, sy = 0.f, sz = 0.f;
    for (long long p = p0; p < p1; ++p) {
        const uint4 x = posm[p];
        const float m = __uint_as_float(x.w);
        M += m;
        sx = fmaf(m, (float)(int)(x.x - c.x), sx);
        sy = fmaf(m, (float)(int)(x.y - c.y), sy);
        sz = fmaf(m, (float)(int)(x.z - c.z), sz);
    }
    const float s = M > 0.f ? B.sf / M : 0.f;
    nm[nd] = make_float4(sx * s, sy * s, sz * s, M);
}

// Node moments from the children's (level lev >= 1).
__global__ void k_grav_node_moments(int lev, const BoxDesc* __restrict__ boxes, const uint4* __restrict__ nc,
                                    float4* __restrict__ nm) {
    const BoxDesc& B = boxes[blockIdx.y];
    if (lev >= B.nlev) return;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= B.lvl_n[lev]) return;
    const int c0 = t * kFan, c1 = min(c0 + kFan, B.lvl_n[lev - 1]);
    const int nd = B.lvl_off[lev] + t;
    const uint4 c = nc[nd];
    const float sf = B.sf;
    float M = 0.f, sx = 0.f, sy = 0.f, sz = 0.f;
    for (int k = c0; k < c1; ++k) {
        const int ch = B.lvl_off[lev - 1] + k;
        const float4 q = nm[ch];
        const uint4 cc = nc[ch];
        M += q.w;
        sx = fmaf(q.w, fmaf((float)(int)(cc.x - c.x), sf, q.x), sx);
        sy = fmaf(q.w, fmaf((float)(int)(cc.y - c.y), sf, q.y), sy);
        sz = fmaf(q.w, fmaf((float)(int)(cc.z - c.z), sf, q.z), sz);
    }
    const float s = M > 0.f ? 1.f / M : 0.f;
    nm[nd] = make_float4(sx * s, sy * s, sz * s, M);
}

// RCi = ceil((r_cut 2^24 / L)^2) of each box (FP64, then exact).
__global__ void k_grav_box_rc(const BoxDesc* __restrict__ boxes, int nb, double r_cut,
                              unsigned long long* __restrict__ rci) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const double rcu = r_cut / boxes[b].L * 16777216.0;
    rci[b] = (unsigned long long)ceil(rcu * rcu);
}

// M(q) g(r) / r^3 for r^2 = r2 > 0, and r.
// The split factor g = erfc(x) + (2/sqrt(pi)) x e^{-x^2}, x = r / (2 r_s), takes
// erfc from Abramowitz & Stegun 7.1.26 (Hastings' rational approximation,
// |error| <= 1.5e-7): erfc(x) = t (a1 + t (a2 + t (a3 + t (a4 + t a5)))) e^{-x^2},
// t = 1 / (1 + p x), so that both terms share one exponential.
__device__ __forceinline__ float grav_K(const GravArgs& a, float r2, float& r) {
    r = r2 * rsqrtf(r2);
    float Mq = 1.f;
    if (r < a.hs) {   // mass fraction of the cubic spline (support 1) inside q
        const float q = r * a.inv_hs, q2 = q * q, q3 = q2 * q;
        Mq = q <= 0.5f ? q3 * fmaf(q2, fmaf(32.f, q, -192.f / 5.f), 32.f / 3.f)
                       : fmaf(q3, fmaf(q, fmaf(q, fmaf(-32.f / 3.f, q, 192.f / 5.f), -48.f), 64.f / 3.f),
                              -1.f / 15.f);
    }
    float g = 1.f;
    if (a.inv2rs > 0.f) {
        const float x = r * a.inv2rs;
        const float t = __fdividef(1.f, fmaf(0.3275911f, x, 1.f));
        const float poly =
            t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, 1.061405429f, -1.453152027f), 1.421413741f), -0.284496736f),
                     0.254829592f);
        g = __expf(-x * x) * fmaf(1.1283791671f, x, poly);   // 2 / sqrt(pi) = 1.1283791671
    }
    return __fdividef(Mq * g, r2 * r);   // r^3 stays far inside the normal range
}

// One axis of the exact coarse box geometry: squared gap, squared far-side
// distance (rounded up) and coarse side.
__device__ __forceinline__ void grav_axis(unsigned x, unsigned lo, unsigned hi, unsigned long long& D2,
                                          unsigned long long& F2, unsigned& l) {
    unsigned gap = 0u, far;
    if (x < lo || x > hi) {
        const unsigned g1 = lo - x, g2 = x - hi;   // both ways round the periodic axis
        gap = min(g1, g2);
        far = gap + (hi - lo);
    } else {
        far = max(x - lo, hi - x);
    }
    const unsigned g = gap >> 8, f = (unsigned)(((unsigned long long)far + 255ull) >> 8);
    D2 += (unsigned long long)g * g;
    F2 += (unsigned long long)f * f;
    l = max(l, (hi - lo) >> 8);
}

// Exact coarse geometry of a node box seen from X: D2 (gap), F2 (far side,
// rounded up), L2 (largest side squared), per the rules above.
__device__ __forceinline__ void grav_box(uint4 X, uint4 lo, uint4 hi, unsigned long long& D2,
                                         unsigned long long& F2, unsigned long long& L2) {
    D2 = F2 = 0ull;
    unsigned l = 0u;
    grav_axis(X.x, lo.x, hi.x, D2, F2, l);
    grav_axis(X.y, lo.y, hi.y, D2, F2, l);
    grav_axis(X.z, lo.z, hi.z, D2, F2, l);
    L2 = (unsigned long long)l * l;
}

__global__ void __launch_bounds__(kWppThreads) k_gravity(GravArgs a) {
    __shared__ int stk_all[kWppWarps][kGravStack];
    __shared__ int lf_all[kWppWarps][kGravLeaves];
    __shared__ float4 hb_all[kWppWarps][kGravHits];
    const int w = threadIdx.x >> 5;
    int* stk = stk_all[w];
    int* lf = lf_all[w];
    float4* hb = hb_all[w];
    const unsigned lane = lane_id();
    const unsigned lt = (1u << lane) - 1u;
    const int cnt = (int)*a.count_ptr;
    unsigned long long c_nodes = 0, c_pairs = 0;
    for (;;) {
        int t = 0;
        if (lane == 0) t = (int)atomicAdd(a.queue, 1u);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= cnt) break;
        const int p = a.act[t];
        const int bi = a.n_boxes == 1 ? 0 : wpp_box(a.boxes, a.n_boxes, p);
        const BoxDesc& B = a.boxes[bi];
        const float sf = B.sf;
        const unsigned long long RCi = a.box_rci[bi];
        const uint4 Xi = a.posm[p];
        float ax = 0.f, ay = 0.f, az = 0.f, sc = 0.f;
        int nn = 0, np = 0;
        int sp = 0, nl = 0, nh = 0;
        const int top = B.nlev - 1;
        if (top == 0) {
            nl = 1;
            if (lane == 0) lf[0] = 0;
        } else if (lane == 0) {
            stk[0] = (int)((unsigned)top << 28);
            sp = 1;
        }
        sp = __shfl_sync(0xffffffffu, sp, 0);
        __syncwarp();
        // One loop with one site for each kind of step, in this priority:
        // evaluate 32 buffered interactions (or the last few once the walk is
        // done), test the particles of four opened leaves (or the last few),
        // test the children of up to four opened nodes. The buffer holds <= 31
        // entries before a test step adds <= 32; the leaf list <= 3 before a
        // node step adds <= 32.
        for (;;) {
            const bool walk_done = sp == 0 && nl == 0;
            if (nh >= 32 || (walk_done && nh > 0)) {
                const int k = min(nh, 32);
                if ((int)lane < k) {
                    const float4 h = hb[lane];
                    const float r2 = h.x * h.x + h.y * h.y + h.z * h.z;
                    if (r2 > 0.f) {
                        float r;
                        const float f = a.G * h.w * grav_K(a, r2, r);
                        ax = fmaf(f, h.x, ax);
                        ay = fmaf(f, h.y, ay);
                        az = fmaf(f, h.z, az);
                        sc = fmaf(fabsf(f), r, sc);
                    }
                }
                nh -= k;   // <= 31 left: move hb[32..nh+32) down
                const float4 v = (int)lane < nh ? hb[lane + 32] : make_float4(0.f, 0.f, 0.f, 0.f);
                __syncwarp();
                if ((int)lane < nh) hb[lane] = v;
                __syncwarp();
                continue;
            }
            if (walk_done) break;
            bool take = false;
            float4 e = make_float4(0.f, 0.f, 0.f, 0.f);
            if (nl >= 4 || (sp == 0 && nl > 0)) {
                // the particles of leaves lf[0..k), lanes 8s..8s+7 on leaf s
                const int k = min(nl, 4);
                const int s = (int)(lane >> 3);
                if (s < k) {
                    const long long q = B.off + (long long)lf[s] * kLeaf + (lane & 7u);
                    if (q < B.off + B.n && q != p) {
                        const uint4 Xq = a.posm[q];
                        const int dx = (int)(Xq.x - Xi.x), dy = (int)(Xq.y - Xi.y), dz = (int)(Xq.z - Xi.z);
                        const unsigned gx = (unsigned)abs(dx) >> 8, gy = (unsigned)abs(dy) >> 8,
                                       gz = (unsigned)abs(dz) >> 8;
                        const unsigned long long D2 = (unsigned long long)gx * gx + (unsigned long long)gy * gy +
                                                      (unsigned long long)gz * gz;
                        if (D2 < RCi) {
                            ++np;
                            take = true;
                            e = make_float4((float)dx * sf, (float)dy * sf, (float)dz * sf, __uint_as_float(Xq.w));
                        }
                    }
                }
                nl -= k;   // <= 31 left: move lf[k..nl+k) down
                const int v = (int)lane < nl ? lf[lane + k] : 0;
                __syncwarp();
                if ((int)lane < nl) lf[lane] = v;
            } else {
                // the children of up to four opened nodes, one per lane
                const int npop = sp <= 96 ? min(4, sp) : 1;
                const int slot = (int)(lane >> 3);
                int lev = -1, child = -1;
                if (slot < npop) {
                    const unsigned en = (unsigned)stk[sp - 1 - slot];
                    const int k = (int)(en >> 28), tt = (int)(en & 0x0fffffffu);
                    const int c = tt * kFan + (int)(lane & 7u);
                    if (c < B.lvl_n[k - 1]) {
                        lev = k - 1;
                        child = c;
                    }
                }
                __syncwarp();
                sp -= npop;
                bool push = false, leaf = false;
                if (child >= 0) {
                    const int nd = B.lvl_off[lev] + child;
                    unsigned long long D2, F2, L2;
                    grav_box(Xi, a.node_lo[nd], a.node_hi[nd], D2, F2, L2);
                    if (D2 < RCi) {
                        if (a.P > 0ull && D2 > 0ull && F2 < RCi && L2 <= D2 && (L2 << 16) <= a.P * D2) {
                            ++nn;
                            take = true;
                            const float4 m = a.node_m[nd];
                            const uint4 c = a.node_c[nd];
                            e = make_float4(fmaf((float)(int)(c.x - Xi.x), sf, m.x),
                                            fmaf((float)(int)(c.y - Xi.y), sf, m.y),
                                            fmaf((float)(int)(c.z - Xi.z), sf, m.z), m.w);
                        } else if (lev == 0) {
                            leaf = true;
                        } else {
                            push = true;
                        }
                    }
                }
                const unsigned bp = __ballot_sync(0xffffffffu, push), bl = __ballot_sync(0xffffffffu, leaf);
                if (push) stk[sp + __popc(bp & lt)] = (int)(((unsigned)lev << 28) | (unsigned)child);
                if (leaf) lf[nl + __popc(bl & lt)] = child;
                sp += __popc(bp);
                nl += __popc(bl);
            }
            // append this step's interactions to the buffer
            const unsigned bt = __ballot_sync(0xffffffffu, take);
            if (take) hb[nh + __popc(bt & lt)] = e;
            nh += __popc(bt);
            __syncwarp();
        }
        const float fs = wpp_fold4(ax, ay, az, sc);
        nn = warp_sum(nn);
        np = warp_sum(np);
        const int oi = a.perm[p];
        if ((lane & 7u) == 0u && (lane >> 3) < 3u) a.acc[3 * (size_t)oi + (lane >> 3)] = fs;
        if (lane == 0) {
            if (a.n_nodes) a.n_nodes[oi] = nn;
            if (a.n_pairs) a.n_pairs[oi] = np;
        }
        c_nodes += (unsigned long long)nn;
        c_pairs += (unsigned long long)np;
    }
    if (lane == 0 && (c_nodes | c_pairs)) {
        atomicAdd(&a.ctr->grav_nodes, c_nodes);
        atomicAdd(&a.ctr->grav_pairs, c_pairs);
    }
}

// ---------------------------------------------------------------------------
// Shared walk for a group of up to 8 active particles of one leaf-parent node
// ---------------------------------------------------------------------------
//
// The members' integer positions lie in a box G (per axis an interval of
// span < 2^30 starting at glo). For a node, bounds over G decide it for every
// member at once, with the per-member rule's outcome:
//   D2_G = sum_a (gap_a(G) >> 8)^2 <= every member's D2 (the gap from the
//          interval to the node box: 0 if they overlap, else the smaller of
//          the ends' gaps, since a point's gap has no interior minimum off the
//          box);
//   F2_G = sum_a ceil(far_a(G) / 256)^2 >= every member's F2 (a point's far
//          distance max(x - lo, hi - x), continued by gap + side off the box,
//          is convex on any interval that does not hold the point (lo + hi)/2
//          + 2^31 where the nearest image switches, so its largest value is at
//          an end; an interval that holds it gets no group decision).
// D2_G >= RCi skips the node for all; the accept test on (D2_G, F2_G) accepts
// it for all (D2 >= D2_G and F2 <= F2_G keep every inequality, and F2 < RCi
// implies D2 < RCi). Other nodes are decided member by member with the exact
// rule; the members that open a node carry on with it as a member mask. A
// particle of an opened leaf is taken for every member of the leaf's mask
// when its largest coarse distance to the interval is inside the cutoff,
// dropped when the smallest is not, and tested member by member otherwise.
// Interactions are buffered with their member masks and evaluated by lanes
// 4m..4m+3 for member m, from exact integer separations (a node entry adds
// its centre-of-mass offset), so every count and term is the one-particle
// kernel's.
constexpr int kGgMembers = 8;

struct GravGroupSmem {
    int stk[kGravStack];
    unsigned char stm[kGravStack];   // member mask of each stacked node
    int lf[kGravLeaves];
    unsigned short lfm[kGravLeaves]; // member mask of each opened leaf; bit 8: every particle of it
                                     // lies inside the cutoff of every member (no tests needed)
    uint4 hA[kGravHits];    // integer anchor (particle position or node centre), mass bits
    float4 hB[kGravHits];   // offset from the anchor (box units: a node's centre of mass)
    int hq[kGravHits];      // particle index (-1: a node)
    int hm[kGravHits];      // member mask
    uint4 mX[kGgMembers];   // member integer positions
};

// One axis of a point's exact coarse geometry against [lo, hi]: raw gap and
// far distance (the rule of grav_axis before the coarse shift).
__device__ __forceinline__ void grav_axis_raw(unsigned x, unsigned lo, unsigned hi, unsigned& gap, unsigned& far) {
    if (x < lo || x > hi) {
        gap = min(lo - x, x - hi);
        far = gap + (hi - lo);
    } else {
        gap = 0u;
        far = max(x - lo, hi - x);
    }
}

// The group bounds of one axis (interval [e1, e1 + span]): adds to D2_G and
// F2_G; `ok` cleared when the interval holds the switching point of the
// nearest image, where the far bound would not hold.
__device__ __forceinline__ void grav_axis_group(unsigned e1, unsigned span, unsigned lo, unsigned hi,
                                                unsigned long long& D2, unsigned long long& F2, unsigned& l,
                                                bool& ok) {
    unsigned g1, f1, g2, f2;
    grav_axis_raw(e1, lo, hi, g1, f1);
    grav_axis_raw(e1 + span, lo, hi, g2, f2);
    const bool overlap = g1 == 0u || g2 == 0u || (lo - e1) <= span;
    const unsigned gap = overlap ? 0u : min(g1, g2);
    const unsigned sw = lo + ((hi - lo) >> 1) + 0x80000000u;
    if ((sw - e1) <= span) ok = false;
    const unsigned far = max(f1, f2);
    const unsigned g = gap >> 8, f = (unsigned)(((unsigned long long)far + 255ull) >> 8);
    D2 += (unsigned long long)g * g;
    F2 += (unsigned long long)f * f;
    l = max(l, (hi - lo) >> 8);
}

// The monopole rule of the walk (see the top of the file).
__device__ __forceinline__ bool grav_accept(unsigned long long P, unsigned long long D2, unsigned long long F2,
                                            unsigned long long L2, unsigned long long RCi) {
    return P > 0ull && D2 > 0ull && F2 < RCi && L2 <= D2 && (L2 << 16) <= P * D2;
}

// Largest and smallest coarse distance (>> 8) on one axis from x to the
// points of the interval [e1, e1 + span] (|x - y| is convex along the
// interval: the largest is at an end, the smallest 0 inside, else at an end).
__device__ __forceinline__ void grav_axis_pt(unsigned x, unsigned e1, unsigned span, unsigned& hi_, unsigned& lo_) {
    const unsigned a1 = (unsigned)abs((int)(x - e1)), a2 = (unsigned)abs((int)(x - (e1 + span)));
    hi_ = max(a1, a2) >> 8;
    lo_ = (x - e1) <= span ? 0u : (min(a1, a2) >> 8);
}

// Error-free (TwoSum) fold of two per-lane sums over aligned quads of lanes;
// every lane of the quad ends with both totals, rounded once.
__device__ __forceinline__ void grav_fold_quad2(float& s1, float& s2) {
    auto two_sum = [](float& s, float& c, float s2_, float c2_) {
        const float t = __fadd_rn(s, s2_);
        const float bp = __fsub_rn(t, s);
        const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(s2_, bp));
        s = t;
        c = __fsub_rn(__fadd_rn(c, c2_), e);
    };
    float c1 = 0.f, c2 = 0.f;
#pragma unroll
    for (int o = 1; o <= 2; o <<= 1) {
        const float a1 = __shfl_xor_sync(0xffffffffu, s1, o), b1 = __shfl_xor_sync(0xffffffffu, c1, o);
        const float a2 = __shfl_xor_sync(0xffffffffu, s2, o), b2 = __shfl_xor_sync(0xffffffffu, c2, o);
        two_sum(s1, c1, a1, b1);
        two_sum(s2, c2, a2, b2);
    }
    s1 = __fsub_rn(s1, c1);
    s2 = __fsub_rn(s2, c2);
}

__global__ void __launch_bounds__(kWppThreads) k_gravity_group(GravArgs a) {
    __shared__ GravGroupSmem smem[kWppWarps];
    GravGroupSmem& sm = smem[threadIdx.x >> 5];
    const unsigned lane = lane_id();
    const unsigned lt = (1u << lane) - 1u;
    const int cnt = (int)*a.count_ptr;
    const int mm = (int)(lane >> 2), sub = (int)(lane & 3u);   // evaluation: lane (member, quarter)
    unsigned long long c_nodes = 0, c_pairs = 0;
    for (;;) {
        int t0 = 0;
        if (lane == 0) t0 = (int)atomicAdd(a.queue, (unsigned)kGgMembers);
        t0 = __shfl_sync(0xffffffffu, t0, 0);
        if (t0 >= cnt) break;
        const int t1 = min(t0 + kGgMembers, cnt);
        for (int t = t0; t < t1;) {
            const WppGroup G = wpp_group(a.boxes, a.n_boxes, a.act, t, t1, 6);
            t += G.n;
            const BoxDesc& B = a.boxes[G.box];
            const float sf = B.sf;
            const unsigned long long RCi = a.box_rci[G.box];
            const unsigned full = (1u << G.n) - 1u;
            // members: lane l < G.n holds member l; the group's interval per axis
            uint4 Xl = make_uint4(0u, 0u, 0u, 0u);
            if (G.p >= 0) Xl = a.posm[G.p];
            if ((int)lane < kGgMembers) sm.mX[lane] = Xl;
            const unsigned X0x = __shfl_sync(0xffffffffu, Xl.x, 0), X0y = __shfl_sync(0xffffffffu, Xl.y, 0),
                           X0z = __shfl_sync(0xffffffffu, Xl.z, 0);
            const bool mv = G.p >= 0;
            const int dx0 = mv ? (int)(Xl.x - X0x) : 0, dy0 = mv ? (int)(Xl.y - X0y) : 0,
                      dz0 = mv ? (int)(Xl.z - X0z) : 0;
            const int lox = warp_min(dx0), loy = warp_min(dy0), loz = warp_min(dz0);
            const long long sxl = (long long)warp_max(dx0) - lox, syl = (long long)warp_max(dy0) - loy,
                            szl = (long long)warp_max(dz0) - loz;
            // a group spanning a quarter of the box or more takes no group decision
            const bool gok = sxl < (1ll << 30) && syl < (1ll << 30) && szl < (1ll << 30);
            const unsigned gex = X0x + (unsigned)lox, gey = X0y + (unsigned)loy, gez = X0z + (unsigned)loz;
            const unsigned spx = (unsigned)sxl, spy = (unsigned)syl, spz = (unsigned)szl;
            // the evaluation lanes' member
            const uint4 Xm = make_uint4(__shfl_sync(0xffffffffu, Xl.x, mm), __shfl_sync(0xffffffffu, Xl.y, mm),
                                        __shfl_sync(0xffffffffu, Xl.z, mm), 0u);
            const int pmm = __shfl_sync(0xffffffffu, G.p, mm);
            const bool mlive = mm < G.n;
            float ax = 0.f, ay = 0.f, az = 0.f, sc = 0.f;
            int nn = 0, np = 0;
            int sp = 0, nl = 0, nh = 0;
            const int top = B.nlev - 1;
            if (top == 0) {
                nl = 1;
                if (lane == 0) {
                    sm.lf[0] = 0;
                    sm.lfm[0] = (unsigned short)full;
                }
            } else {
                if (lane == 0) {
                    sm.stk[0] = (int)((unsigned)top << 28);
                    sm.stm[0] = (unsigned char)full;
                }
                sp = 1;
            }
            __syncwarp();
            // The one-particle kernel's loop: evaluate 32 buffered interactions (or
            // the last few once the walk is done), test the particles of four
            // opened leaves (or the last few), test the children of up to four
            // opened nodes; with a member mask on every node, leaf and entry.
            for (;;) {
                const bool walk_done = sp == 0 && nl == 0;
                if (nh >= 32 || (walk_done && nh > 0)) {
                    const int k = min(nh, 32);
#pragma unroll 2
                    for (int jj = 0; jj < 8; ++jj) {
                        const int c = sub + 4 * jj;
                        if (c < k && mlive && ((sm.hm[c] >> mm) & 1) && sm.hq[c] != pmm) {
                            const uint4 A = sm.hA[c];
                            const float4 Bo = sm.hB[c];
                            if (sm.hq[c] < 0) ++nn; else ++np;
                            const float ex = fmaf((float)(int)(A.x - Xm.x), sf, Bo.x),
                                        ey = fmaf((float)(int)(A.y - Xm.y), sf, Bo.y),
                                        ez = fmaf((float)(int)(A.z - Xm.z), sf, Bo.z);
                            const float r2 = ex * ex + ey * ey + ez * ez;
                            if (r2 > 0.f) {
                                float r;
                                const float f = a.G * __uint_as_float(A.w) * grav_K(a, r2, r);
                                ax = fmaf(f, ex, ax);
                                ay = fmaf(f, ey, ay);
                                az = fmaf(f, ez, az);
                                sc = fmaf(fabsf(f), r, sc);
                            }
                        }
                    }
                    __syncwarp();
                    nh -= k;   // <= 31 left: move entries [32, nh + 32) down
                    uint4 vA = make_uint4(0u, 0u, 0u, 0u);
                    float4 vB = make_float4(0.f, 0.f, 0.f, 0.f);
                    int vq = 0, vm = 0;
                    if ((int)lane < nh) {
                        vA = sm.hA[lane + 32];
                        vB = sm.hB[lane + 32];
                        vq = sm.hq[lane + 32];
                        vm = sm.hm[lane + 32];
                    }
                    __syncwarp();
                    if ((int)lane < nh) {
                        sm.hA[lane] = vA;
                        sm.hB[lane] = vB;
                        sm.hq[lane] = vq;
                        sm.hm[lane] = vm;
                    }
                    __syncwarp();
                    continue;
                }
                if (walk_done) break;
                unsigned emask = 0u;   // members taking this lane's interaction
                uint4 eA = make_uint4(0u, 0u, 0u, 0u);
                float4 eB = make_float4(0.f, 0.f, 0.f, 0.f);
                int eq = -1;
                if (nl >= 4 || (sp == 0 && nl > 0)) {
                    // the particles of leaves lf[0..k), lanes 8s..8s+7 on leaf s
                    const int k = min(nl, 4);
                    const int s = (int)(lane >> 3);
                    if (s < k) {
                        const unsigned M = sm.lfm[s] & 0xffu;
                        const bool allin = (sm.lfm[s] >> 8) != 0u;
                        const long long q = B.off + (long long)sm.lf[s] * kLeaf + (lane & 7u);
                        if (q < B.off + B.n) {
                            const uint4 Xq = a.posm[q];
                            bool decided = false;
                            if (allin) {
                                decided = true;
                                emask = M;
                            } else if (gok) {
                                unsigned hx, lx, hy, ly, hz, lz;
                                grav_axis_pt(Xq.x, gex, spx, hx, lx);
                                grav_axis_pt(Xq.y, gey, spy, hy, ly);
                                grav_axis_pt(Xq.z, gez, spz, hz, lz);
                                const unsigned long long U = (unsigned long long)hx * hx +
                                                             (unsigned long long)hy * hy +
                                                             (unsigned long long)hz * hz;
                                const unsigned long long Lw = (unsigned long long)lx * lx +
                                                              (unsigned long long)ly * ly +
                                                              (unsigned long long)lz * lz;
                                if (Lw >= RCi) {
                                    decided = true;
                                } else if (U < RCi) {
                                    decided = true;
                                    emask = M;
                                }
                            }
                            if (!decided) {
                                for (unsigned r = M; r; r &= r - 1u) {
                                    const int m = __ffs(r) - 1;
                                    const uint4 Y = sm.mX[m];
                                    const unsigned gx = (unsigned)abs((int)(Xq.x - Y.x)) >> 8,
                                                   gy = (unsigned)abs((int)(Xq.y - Y.y)) >> 8,
                                                   gz = (unsigned)abs((int)(Xq.z - Y.z)) >> 8;
                                    const unsigned long long D2 = (unsigned long long)gx * gx +
                                                                  (unsigned long long)gy * gy +
                                                                  (unsigned long long)gz * gz;
                                    if (D2 < RCi) emask |= 1u << m;
                                }
                            }
                            eA = Xq;
                            eq = (int)q;
                        }
                    }
                    nl -= k;   // <= 31 left: move lf[k..nl+k) down
                    const int v = (int)lane < nl ? sm.lf[lane + k] : 0;
                    const unsigned short vm = (int)lane < nl ? sm.lfm[lane + k] : (unsigned short)0;
                    __syncwarp();
                    if ((int)lane < nl) {
                        sm.lf[lane] = v;
                        sm.lfm[lane] = vm;
                    }
                } else {
                    // the children of up to four opened nodes, one per lane
                    const int npop = sp <= 96 ? min(4, sp) : 1;
                    const int slot = (int)(lane >> 3);
                    int lev = -1, child = -1;
                    unsigned M = 0u;
                    if (slot < npop) {
                        const unsigned en = (unsigned)sm.stk[sp - 1 - slot];
                        M = sm.stm[sp - 1 - slot];
                        const int k = (int)(en >> 28), tt = (int)(en & 0x0fffffffu);
                        const int c = tt * kFan + (int)(lane & 7u);
                        if (c < B.lvl_n[k - 1]) {
                            lev = k - 1;
                            child = c;
                        }
                    }
                    __syncwarp();
                    sp -= npop;
                    unsigned om = 0u;   // members that open the child
                    bool allin = false; // an opened leaf wholly inside every member's cutoff
                    if (child >= 0) {
                        const int nd = B.lvl_off[lev] + child;
                        const uint4 lo = a.node_lo[nd], hi = a.node_hi[nd];
                        bool decided = false;
                        if (gok) {
                            unsigned long long D2 = 0ull, F2 = 0ull;
                            unsigned l = 0u;
                            bool ok = true;
                            grav_axis_group(gex, spx, lo.x, hi.x, D2, F2, l, ok);
                            grav_axis_group(gey, spy, lo.y, hi.y, D2, F2, l, ok);
                            grav_axis_group(gez, spz, lo.z, hi.z, D2, F2, l, ok);
                            if (D2 >= RCi) {
                                decided = true;
                            } else if (ok && grav_accept(a.P, D2, F2, (unsigned long long)l * l, RCi)) {
                                decided = true;
                                emask = M;
                            }
                            // a point of the box is no farther from a member than the box's
                            // far side, so F2_G < RCi puts every particle inside the cutoff
                            allin = ok && F2 < RCi;
                        }
                        if (!decided) {
                            for (unsigned r = M; r; r &= r - 1u) {
                                const int m = __ffs(r) - 1;
                                unsigned long long D2, F2, L2;
                                grav_box(sm.mX[m], lo, hi, D2, F2, L2);
                                if (D2 < RCi) {
                                    if (grav_accept(a.P, D2, F2, L2, RCi)) emask |= 1u << m;
                                    else om |= 1u << m;
                                }
                            }
                        }
                        if (emask) {
                            const float4 nm = a.node_m[nd];
                            eA = a.node_c[nd];
                            eA.w = __float_as_uint(nm.w);
                            eB = make_float4(nm.x, nm.y, nm.z, 0.f);
                        }
                    }
                    const bool push = om != 0u && lev > 0, leaf = om != 0u && lev == 0;
                    const unsigned bp = __ballot_sync(0xffffffffu, push), bl = __ballot_sync(0xffffffffu, leaf);
                    if (push) {
                        const int o = sp + __popc(bp & lt);
                        sm.stk[o] = (int)(((unsigned)lev << 28) | (unsigned)child);
                        sm.stm[o] = (unsigned char)om;
                    }
                    if (leaf) {
                        const int o = nl + __popc(bl & lt);
                        sm.lf[o] = child;
                        sm.lfm[o] = (unsigned short)(om | (allin ? 0x100u : 0u));
                    }
                    sp += __popc(bp);
                    nl += __popc(bl);
                }
                // append this step's interactions to the buffer
                const bool take = emask != 0u;
                const unsigned bt = __ballot_sync(0xffffffffu, take);
                if (take) {
                    const int o = nh + __popc(bt & lt);
                    sm.hA[o] = eA;
                    sm.hB[o] = eB;
                    sm.hq[o] = eq;
                    sm.hm[o] = (int)emask;
                }
                nh += __popc(bt);
                __syncwarp();
            }
            // per member: fold its quad's sums, write its outputs
            grav_fold_quad2(ax, ay);
            grav_fold_quad2(az, sc);
            nn += __shfl_xor_sync(0xffffffffu, nn, 1);
            nn += __shfl_xor_sync(0xffffffffu, nn, 2);
            np += __shfl_xor_sync(0xffffffffu, np, 1);
            np += __shfl_xor_sync(0xffffffffu, np, 2);
            if (mlive) {
                const int oi = a.perm[pmm];
                if (sub < 3) a.acc[3 * (size_t)oi + sub] = sub == 0 ? ax : (sub == 1 ? ay : az);
                if (sub == 3) {
                    if (a.n_nodes) a.n_nodes[oi] = nn;
                    if (a.n_pairs) a.n_pairs[oi] = np;
                }
                if (sub == 0) {
                    c_nodes += (unsigned long long)nn;
                    c_pairs += (unsigned long long)np;
                }
            }
            __syncwarp();
        }
    }
    c_nodes = warp_sum(c_nodes);
    c_pairs = warp_sum(c_pairs);
    if (lane == 0 && (c_nodes | c_pairs)) {
        atomicAdd(&a.ctr->grav_nodes, c_nodes);
        atomicAdd(&a.ctr->grav_pairs, c_pairs);
    }
}

cudaError_t launch_gravity(sph_ctx* ctx, const GravityLaunch& L, int64_t n_active, cudaStream_t s) {
    sph_grid* g = const_cast<sph_grid*>(L.g);
    const int nb = g->n_boxes;
    dim3 lg((g->max_leaves + 127) / 128, nb);
    k_grav_leaf_moments<<<lg, 128, 0, s>>>(g->posm, g->boxes, g->node_c, g->node_m);
    ++ctx->launches;
    for (int lev = 1; lev < g->max_lev; ++lev) {
        dim3 ng((g->lvl_max[lev] + 127) / 128, nb);
        k_grav_node_moments<<<ng, 128, 0, s>>>(lev, g->boxes, g->node_c, g->node_m);
        ++ctx->launches;
    }
    k_grav_box_rc<<<(nb + 127) / 128, 128, 0, s>>>(g->boxes, nb, L.r_cut, g->box_rci);
    ++ctx->launches;
    cudaError_t e = cudaMemsetAsync(ctx->queue + 4, 0, sizeof(unsigned), s);
    if (e) return e;
    GravArgs a = {};
    a.boxes = g->boxes;
    a.n_boxes = nb;
    a.act = g->act;
    a.count_ptr = g->scan + g->n;
    a.queue = ctx->queue + 4;
    a.posm = g->posm;
    a.perm = g->perm;
    a.node_lo = g->node_lo;
    a.node_hi = g->node_hi;
    a.node_c = g->node_c;
    a.node_m = g->node_m;
    a.box_rci = g->box_rci;
    a.acc = L.acc;
    a.n_nodes = L.n_nodes;
    a.n_pairs = L.n_pairs;
    a.ctr = ctx->counters;
    a.G = (float)L.G;
    a.P = (unsigned long long)std::rint(L.theta * L.theta * 65536.0);
    a.hs = (float)L.h_soft;
    a.inv_hs = L.h_soft > 0.0 ? (float)(1.0 / L.h_soft) : 0.f;
    a.inv2rs = L.r_split > 0.0 ? (float)(0.5 / L.r_split) : 0.f;
    if (wpp_groups_pay(ctx, n_active, g->n)) {
        // groups of up to 8 particles of a leaf-parent node share one walk
        const long long want = (n_active + kGgMembers * kWppWarps - 1) / (kGgMembers * kWppWarps);
        const int blocks = (int)std::max<long long>(1, std::min<long long>((long long)ctx->sm_count * 8, want));
        k_gravity_group<<<blocks, kWppThreads, 0, s>>>(a);
    } else {
        const long long want = (n_active + kWppWarps - 1) / kWppWarps;
        const int blocks = (int)std::max<long long>(1, std::min<long long>((long long)ctx->sm_count * 8, want));
        k_gravity<<<blocks, kWppThreads, 0, s>>>(a);
    }
    ++ctx->launches;
    return cudaGetLastError();
}

}  // namespace sph
