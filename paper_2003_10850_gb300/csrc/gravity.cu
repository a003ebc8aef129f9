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
    const long long want = (n_active + kWppWarps - 1) / kWppWarps;
    const int blocks = (int)std::max<long long>(1, std::min<long long>((long long)ctx->sm_count * 8, want));
    k_gravity<<<blocks, kWppThreads, 0, s>>>(a);
    ++ctx->launches;
    return cudaGetLastError();
}

}  // namespace sph
