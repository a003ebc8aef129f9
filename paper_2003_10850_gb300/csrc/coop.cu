// coop.cu -- warp-cooperative density and force kernels (the default path).
//
// One warp per group of <= 32 Morton-consecutive active particles. The warp
// walks the hierarchy once for the group with a shared depth-first stack of
// (node, lane mask) entries: every lane tests each child of a popped node
// against its OWN sphere, and a ballot decides whether the child is pushed
// (internal) or appended to the lists of the lanes that need it (leaf). The
// node data are broadcast loads and the walk has no divergence. Each lane then
// runs through its own compacted leaf list (the candidate set of exactly its
// own sphere, as a per-particle walk would find), testing the leaf's particles
// and appending the pairs in the set to a per-lane hit buffer; the pair terms
// are evaluated from the hit buffers in uniform loops. Versus one thread per
// particle walking alone, node tests are shared by the warp and both the walk
// and the pair evaluation run with (nearly) all lanes active.
//
// Density iterates h per lane (FP64 bracket, as in tpp.cu), re-walking with
// only the unconverged lanes in the root mask. FP32 pair terms with per-batch
// Kahan compensation; exact neighbour predicate in a thin band, as elsewhere.
#include <algorithm>

#include "internal.cuh"

namespace sph {

constexpr int kCoopWarps = 3;
constexpr int kCoopMinBlocks = 8;  // register budget for 24 resident warps per SM
constexpr int kCStack = 96;   // depth-first: <= 7 pending siblings per level + 1
constexpr int kLL = 16;       // leaves per lane per chunk
constexpr int kLCache = 64;   // leaves per lane remembered between density iterations
constexpr int kCoopMaxBps = 16;
constexpr float kWalkR = 1.06f;  // density walks cover 1.06 h so later iterations can reuse them
constexpr int kHB = 16;       // buffered hits per lane (a leaf adds <= 8)

// Per-warp shared memory: the walk stack, the per-lane leaf lists and the
// per-lane hit buffers ((r^2, m) for density, the neighbour's index for force),
// ~6.9 KB per warp.
struct CoopSmem {
    uint4 nc[kFan];     // children of the popped node, staged by one coalesced load
    float4 ne[kFan];
    int stk[kCStack];
    unsigned stm[kCStack];
    int leaves[kLL][32];
    union {
        float2 d[kHB][32];
        int f[kHB][32];
    } hits;
};

struct CoopArgs {
    const BoxDesc* boxes;
    const Group* groups;
    const int* n_groups;
    unsigned* queue;
    const int32_t* act;
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
    int* lcache;        // per persistent warp: kLCache x 32 leaf indices of the last walk
    // force
    const float4* fvel;
    const float4* fthermo;
    float* acc;
    float* dudt;
    float* vsig;
    float alpha;
    unsigned long long* hash;
    Counters* ctr;
};

__device__ __forceinline__ bool coop_near(uint4 c, float4 e, uint4 X, float sf, float R) {
    const float dx = (float)(int)(c.x - X.x) * sf, dy = (float)(int)(c.y - X.y) * sf,
                dz = (float)(int)(c.z - X.z) * sf;
    const float gx = fmaxf(fabsf(dx) - e.x, 0.f), gy = fmaxf(fabsf(dy) - e.y, 0.f),
                gz = fmaxf(fabsf(dz) - e.z, 0.f);
    const float Rt = R * (1.f + 3.0517578125e-05f) + 2.384185791015625e-07f * (fabsf(dx) + fabsf(dy) + fabsf(dz)) +
                     4.f * sf;
    return gx * gx + gy * gy + gz * gz < Rt * Rt;
}

// The cooperative walk. `walk_mask` = lanes that take part; `radius(e)` gives
// the calling lane's test radius for a node with extents/h_max e; `leaf(t)`
// processes leaf t of the box for the calling lane (called by each lane on its
// own leaves, all lanes in lockstep over the list index); `drain()` is called
// by all lanes after each chunk of leaves (to flush hit buffers).
template <class Radius, class Leaf, class Drain>
__device__ __forceinline__ void coop_walk(CoopSmem& sm, const BoxDesc& B, const uint4* __restrict__ node_c,
                                          const float4* __restrict__ node_e, uint4 X, float sf, unsigned walk_mask,
                                          Radius&& radius, Leaf&& leaf, Drain&& drain) {
    const unsigned lane = lane_id();
    const bool mine = (walk_mask >> lane) & 1u;
    int sp = 0, cnt = 0;
    if (B.nlev == 1) {
        if (mine) { sm.leaves[0][lane] = 0; cnt = 1; }
    } else {
        if (lane == 0) { sm.stk[0] = (B.nlev - 1) << 27; sm.stm[0] = walk_mask; }
        sp = 1;
    }
    __syncwarp();
    for (;;) {
        // walk until some lane's list is nearly full or the stack is empty
        while (sp > 0) {
            if (__any_sync(0xffffffffu, cnt > kLL - 8)) break;
            const int enc = sm.stk[sp - 1];
            const unsigned M = sm.stm[sp - 1];
            __syncwarp();
            --sp;
            const int lev = enc >> 27, t = enc & ((1 << 27) - 1);
            const int cl = lev - 1;
            const int c0 = t * kFan, c1 = min(c0 + kFan, B.lvl_n[cl]);
            const int base = B.lvl_off[cl];
            const bool in = (M >> lane) & 1u;
            // lanes 0-7 fetch the children's centres, lanes 8-15 their extents:
            // one load per lane instead of a dependent load pair per child test
            const int nch = c1 - c0;
            if (lane < (unsigned)nch) sm.nc[lane] = node_c[base + c0 + lane];
            else if (lane >= 8u && lane - 8u < (unsigned)nch) sm.ne[lane - 8] = node_e[base + c0 + lane - 8];
            __syncwarp();
            for (int c = c0; c < c1; ++c) {
                const uint4 nc = sm.nc[c - c0];
                const float4 ne = sm.ne[c - c0];
                const bool pass = in && coop_near(nc, ne, X, sf, radius(ne));
                const unsigned Mc = __ballot_sync(0xffffffffu, pass);
                if (!Mc) continue;
                if (cl == 0) {
                    if (pass) sm.leaves[cnt++][lane] = c;
                } else {
                    if (lane == 0) { sm.stk[sp] = (cl << 27) | c; sm.stm[sp] = Mc; }
                    ++sp;
                }
            }
            __syncwarp();
        }
        // every lane processes its own list, in lockstep over the list index
        const int mx = warp_max(cnt);
        __syncwarp();
        for (int k = 0; k < mx; ++k) {
            const int lt = k < cnt ? sm.leaves[k][lane] : -1;
            leaf(lt);
        }
        drain();
        cnt = 0;
        __syncwarp();
        if (sp == 0) break;
    }
}

__device__ __forceinline__ float coop_guess_h(const BoxDesc& B, const uint4* node_lo, const uint4* node_hi,
                                              long long p, double s, double n_target) {
    double best = 0.25 * B.L;
    const int top = B.nlev > 1 ? 1 : 0;
    for (int lev = 0; lev <= top; ++lev) {
        long long span = lev ? (long long)kLeaf * kFan : kLeaf;
        long long t = (p - B.off) / span;
        uint4 lo = node_lo[B.lvl_off[lev] + t], hi = node_hi[B.lvl_off[lev] + t];
        double cnt = (double)min(span, B.n - t * span);
        double V = ((double)(hi.x - lo.x) + 1.0) * ((double)(hi.y - lo.y) + 1.0) * ((double)(hi.z - lo.z) + 1.0) *
                   s * s * s;
        best = fmin(best, cbrt(3.0 * n_target * V / (4.0 * 3.141592653589793 * cnt)));
    }
    return (float)best;
}

// same bracketed, safeguarded step as tpp.cu's h_update
__device__ __forceinline__ bool coop_h_update(float& h, double f, float N, float dN, float n_target, double cap,
                                              double& blo, double& bhi, float& dold, unsigned& st) {
    if (f < 0) blo = h; else bhi = h;
    float step = dN > 0.f ? 3.f * N * (1.f - cbrtf(n_target / N)) / dN : NAN;
    double hn = (double)h - (double)step;
    if (isinf(bhi)) {
        if ((double)h >= cap) {
            st |= ST_H_TOO_LARGE;
            return false;
        }
        if (!(hn > (double)h)) hn = 2.0 * (double)h;
        hn = fmin(hn, fmin(cap, 8.0 * (double)h));
    } else if (!(hn > blo && hn < bhi) || !(fabsf(step) <= 0.5f * dold)) {
        hn = 0.5 * (blo + bhi);
    }
    dold = fabsf((float)(hn - (double)h));
    float hf = (float)hn;
    if (!(hf > (float)blo) || (!isinf(bhi) && !(hf < (float)bhi))) {
        const float mid = (float)(0.5 * (blo + bhi));
        hf = (mid > (float)blo && mid < (float)bhi) ? mid : h;
    }
    if (hf == h) return false;
    h = hf;
    return true;
}

// ---------------------------------------------------------------------------
// Density
// ---------------------------------------------------------------------------

template <bool HASH>
__global__ void __launch_bounds__(kCoopWarps * 32, kCoopMinBlocks) k_density_coop(CoopArgs a) {
    __shared__ CoopSmem smem[kCoopWarps];
    CoopSmem& sm = smem[threadIdx.x >> 5];
    const unsigned lane = lane_id();
    const float rel = 9.5367431640625e-07f;  // 2^-20
    const int ng = *a.n_groups;
    unsigned long long c_pairs = 0, c_evals = 0, c_tests = 0, c_groups = 0;
    unsigned c_status = 0;
    for (;;) {
        int gi = 0;
        if (lane == 0) gi = (int)atomicAdd(a.queue, 1u);
        gi = __shfl_sync(0xffffffffu, gi, 0);
        if (gi >= ng) break;
        const Group G = a.groups[gi];
        const BoxDesc& B = a.boxes[G.box];
        const double L = B.L, s = ldexp(L, -32);
        const float sf = (float)s;
        const bool valid = (int)lane < G.count;
        const int p = valid ? a.act[G.first + lane] : 0;
        const uint4 Xi = valid ? a.posm[p] : make_uint4(0, 0, 0, 0);
        const int oi = valid ? a.perm[p] : 0;
        float h = valid ? a.h[oi] : 1.f;
        if (valid && (a.guess_h || !(h > 0.f) || !isfinite(h))) h = coop_guess_h(B, a.node_lo, a.node_hi, p, s, a.n_target);
        const double cap = 0.5 * L * (1.0 - 1e-9);
        double blo = 0.0, bhi = INFINITY;
        float dold = INFINITY;
        unsigned st = 0;
        bool conv = !valid;
        float Sw = 0.f, Cw = 0.f, Sdw = 0.f, Cdw = 0.f, Smw = 0.f, Cmw = 0.f, Smdw = 0.f, Cmdw = 0.f;
        int nn = 0;
        unsigned long long hs = 0;
        // Leaves of the last walk (radius Rw = 1.06 h), per lane: the h iteration
        // re-tests their particles while h stays below Rw instead of walking again.
        int* lc = a.lcache + (size_t)(blockIdx.x * kCoopWarps + (threadIdx.x >> 5)) * (kLCache * 32);
        int ncache = 0;
        float Rw = 0.f;
        for (int it = 0;; ++it) {
            const unsigned wm = __ballot_sync(0xffffffffu, !conv);
            if (!wm) break;
            const bool rewalk = __any_sync(0xffffffffu, !conv && (ncache > kLCache || !(h <= Rw * 0.99999f)));
            const float hinv = 1.f / h;
            double HH = -1.0;
            if (!conv) {
                Sw = Cw = Sdw = Cdw = Smw = Cmw = Smdw = Cmdw = 0.f;
                nn = 0;
                hs = 0;
            }
            int nh = 0;
            unsigned long long tests = 0;
            auto drain = [&]() {
                const int mx = warp_max(nh);
                float pw = 0.f, pdw = 0.f, pmw = 0.f, pmdw = 0.f;
                for (int k = 0; k < mx; ++k) {
                    if (k < nh) {
                        const float2 e = sm.hits.d[k][lane];
                        const float qq = (e.x > 0.f ? e.x * rsqrtf(e.x) : 0.f) * hinv;
                        float w, dw;
                        spline<float>(qq, w, dw);
                        const float qdw = qq * dw;
                        pw += w;
                        pdw += qdw;
                        pmw += e.y * w;
                        pmdw += e.y * qdw;
                    }
                }
                if (!conv) {
                    kahan_add(Sw, Cw, pw);
                    kahan_add(Sdw, Cdw, pdw);
                    kahan_add(Smw, Cmw, pmw);
                    kahan_add(Smdw, Cmdw, pmdw);
                }
                nh = 0;
                __syncwarp();
            };
            auto leaf = [&](int lt) {
                if (__any_sync(0xffffffffu, nh > kHB - 8)) drain();
                if (lt < 0) return;
                if (rewalk) {
                    if (ncache < kLCache) lc[ncache * 32 + lane] = lt;
                    ++ncache;
                }
                const int nd = B.lvl_off[0] + lt;
                const uint4 C = a.node_c[nd];
                const float4 E = a.node_e[nd];
                const long long q0 = B.off + (long long)lt * kLeaf, q1 = min(q0 + kLeaf, B.off + B.n);
                const bool wide = 2.f * (E.x + E.y + E.z) + h >= 0.45f * (float)L;
                const float ox = (float)(int)(C.x - Xi.x) * sf, oy = (float)(int)(C.y - Xi.y) * sf,
                            oz = (float)(int)(C.z - Xi.z) * sf;
                const float eL = rel * (4.f * (E.x + E.y + E.z) + 2.f * (fabsf(ox) + fabsf(oy) + fabsf(oz)) + 2.f * h);
                const float lo2 = h > eL ? (h - eL) * (h - eL) * (1.f - 4.f * rel) : 0.f;
                const float hi2 = (h + eL) * (h + eL) * (1.f + 4.f * rel);
                for (long long q = q0; q < q1; ++q) {
                    float dx, dy, dz, m;
                    if (!wide) {
                        const float4 f = a.posf[q];
                        dx = ox + f.x; dy = oy + f.y; dz = oz + f.z; m = f.w;
                    } else {
                        const uint4 Xj = a.posm[q];
                        dx = (float)(int)(Xj.x - Xi.x) * sf; dy = (float)(int)(Xj.y - Xi.y) * sf;
                        dz = (float)(int)(Xj.z - Xi.z) * sf; m = __uint_as_float(Xj.w);
                    }
                    const float r2 = dx * dx + dy * dy + dz * dz;
                    if (r2 < hi2) {
                        bool in = r2 < lo2;
                        if (!in) {
                            if (HH < 0.0) {
                                const double Hd = (double)h * 4294967296.0 / L;
                                HH = Hd * Hd;
                            }
                            in = exact_pred(exact_d2(Xi, a.posm[q]), HH);
                        }
                        if (in) {
                            sm.hits.d[nh++][lane] = make_float2(r2, m);
                            if (q != p) {
                                ++nn;
                                if (HASH) hs += splitmix64((unsigned long long)a.perm[q]);
                            }
                        }
                    }
                }
                tests += (unsigned long long)(q1 - q0);
            };
            if (rewalk) {
                if (!conv) {
                    ncache = 0;
                    Rw = h * kWalkR;
                }
                coop_walk(sm, B, a.node_c, a.node_e, Xi, sf, wm, [&](float4) { return Rw; }, leaf, drain);
            } else {
                // the lanes' leaves within their last walk radius, from the list
                const int mx = warp_max(conv ? 0 : ncache);
                for (int k = 0; k < mx; ++k) leaf(!conv && k < ncache ? lc[k * 32 + lane] : -1);
                drain();
            }
            c_tests += tests;
            if (!conv) {
                ++c_evals;
                const double f = (32.0 / 3.0) * ((double)Sw - (double)Cw) - a.n_target;
                if (a.fixed_h || fabs(f) <= a.n_tol) {
                    conv = true;
                } else if (it >= a.max_iter) {
                    conv = true;
                    st |= ST_NOT_CONVERGED;
                } else {
                    const float N = (32.f / 3.f) * (Sw - Cw);
                    const float dN = -(32.f / 3.f) * (Sdw - Cdw) / h;
                    if (!coop_h_update(h, f, N, dN, (float)a.n_target, cap, blo, bhi, dold, st)) conv = true;
                }
            }
        }
        if (valid) {
            const double smw = (double)Smw - (double)Cmw, smdw = (double)Smdw - (double)Cmdw, hd = (double)h;
            a.h[oi] = h;
            a.rho[oi] = (float)(8.0 / (3.141592653589793 * hd * hd * hd) * smw);
            a.omega[oi] = (float)(smdw != 0.0 ? -3.0 * smw / smdw : 1.0);
            a.n_ngb[oi] = nn;
            a.flags[oi] = (uint8_t)st;
            if (HASH) a.hash[oi] = hs;
            c_pairs += (unsigned long long)nn;
            c_status |= st;
        }
        ++c_groups;
    }
    c_pairs = warp_sum(c_pairs);
    c_evals = warp_sum(c_evals);
    c_tests = warp_sum(c_tests);
    c_status = __reduce_or_sync(0xffffffffu, c_status);
    if (lane == 0) {
        atomicAdd(&a.ctr->density_pairs, c_pairs);
        atomicAdd(&a.ctr->density_evals, c_evals);
        atomicAdd(&a.ctr->pair_tests, c_tests);
        atomicAdd(&a.ctr->groups, c_groups);
        if (c_status) atomicOr(&a.ctr->status, c_status);
    }
}

// ---------------------------------------------------------------------------
// Force
// ---------------------------------------------------------------------------

template <bool HASH>
__global__ void __launch_bounds__(kCoopWarps * 32, kCoopMinBlocks) k_force_coop(CoopArgs a) {
    __shared__ CoopSmem smem[kCoopWarps];
    CoopSmem& sm = smem[threadIdx.x >> 5];
    const unsigned lane = lane_id();
    const float rel = 9.5367431640625e-07f;
    const float elo = 1.f - 4.f * rel, ehi = 1.f + 4.f * rel;
    const float kNorm = (float)(8.0 / 3.141592653589793);
    const float alpha = a.alpha;
    const int ng = *a.n_groups;
    unsigned long long c_pairs = 0, c_tests = 0, c_groups = 0;
    for (;;) {
        int gi = 0;
        if (lane == 0) gi = (int)atomicAdd(a.queue, 1u);
        gi = __shfl_sync(0xffffffffu, gi, 0);
        if (gi >= ng) break;
        const Group G = a.groups[gi];
        const BoxDesc& B = a.boxes[G.box];
        const double L = B.L, s = ldexp(L, -32);
        const float sf = (float)s;
        const bool valid = (int)lane < G.count;
        const int p = valid ? a.act[G.first + lane] : 0;
        const uint4 Xi = valid ? a.posm[p] : make_uint4(0, 0, 0, 0);
        const int oi = valid ? a.perm[p] : 0;
        const float4 vi = a.fvel[p];
        const float4 thi = a.fthermo[p];
        const float hi = vi.w, hinvi = thi.w, rhoi = thi.x, Ai = thi.y, ci = thi.z;
        const float normi = kNorm * hinvi * hinvi * hinvi * hinvi;
        double HHi = -1.0;
        float Sx = 0.f, Cx = 0.f, Sy = 0.f, Cy = 0.f, Sz = 0.f, Cz = 0.f, Su = 0.f, Cu = 0.f, vsmax = 0.f;
        int np = 0, nh = 0;
        unsigned long long hs = 0, tests = 0;
        auto drain = [&]() {
            const int mx = warp_max(nh);
            float pax = 0.f, pay = 0.f, paz = 0.f, pdu = 0.f;
            for (int k = 0; k < mx; ++k) {
                if (k >= nh) continue;
                const int q = sm.hits.f[k][lane];
                const uint4 Xj = a.posm[q];
                // d = x_j - x_i from the exact integer separation
                const float dx = (float)(int)(Xj.x - Xi.x) * sf, dy = (float)(int)(Xj.y - Xi.y) * sf,
                            dz = (float)(int)(Xj.z - Xi.z) * sf;
                const float r2 = dx * dx + dy * dy + dz * dz;
                const float4 vj = a.fvel[q];
                const float4 thj = a.fthermo[q];
                const float mj = __uint_as_float(Xj.w);
                if (r2 <= 0.f) {
                    vsmax = fmaxf(vsmax, ci + thj.z);
                    continue;
                }
                const float rinv = rsqrtf(r2), r = r2 * rinv;
                float w_, dwi, dwj;
                spline<float>(r * hinvi, w_, dwi);
                spline<float>(r * thj.w, w_, dwj);
                const float hinvj = thj.w;
                const float Fi = normi * dwi * rinv;
                const float Fj = kNorm * hinvj * hinvj * hinvj * hinvj * dwj * rinv;
                const float vr = -((vi.x - vj.x) * dx + (vi.y - vj.y) * dy + (vi.z - vj.z) * dz);
                const float wij = vr * rinv;
                const float vs = ci + thj.z - 3.f * wij;
                vsmax = fmaxf(vsmax, vs);
                const float PI = wij < 0.f ? -alpha * vs * wij / (rhoi + thj.x) : 0.f;
                const float Fbar = 0.5f * (Fi + Fj);
                const float coef = mj * (Ai * Fi + thj.y * Fj + PI * Fbar);
                pax += coef * dx;
                pay += coef * dy;
                paz += coef * dz;
                pdu += mj * vr * (Ai * Fi + 0.5f * PI * Fbar);
            }
            kahan_add(Sx, Cx, pax);
            kahan_add(Sy, Cy, pay);
            kahan_add(Sz, Cz, paz);
            kahan_add(Su, Cu, pdu);
            nh = 0;
            __syncwarp();
        };
        auto leaf = [&](int lt) {
            if (__any_sync(0xffffffffu, nh > kHB - 8)) drain();
            if (lt < 0) return;
            const int nd = B.lvl_off[0] + lt;
            const uint4 C = a.node_c[nd];
            const float4 E = a.node_e[nd];
            const long long q0 = B.off + (long long)lt * kLeaf, q1 = min(q0 + kLeaf, B.off + B.n);
            const bool wide = 2.f * (E.x + E.y + E.z) + fmaxf(hi, E.w) >= 0.45f * (float)L;
            const float ox = (float)(int)(C.x - Xi.x) * sf, oy = (float)(int)(C.y - Xi.y) * sf,
                        oz = (float)(int)(C.z - Xi.z) * sf;
            const float eL = rel * (4.f * (E.x + E.y + E.z) + 2.f * (fabsf(ox) + fabsf(oy) + fabsf(oz)));
            const float ei = eL + 2.f * rel * hi;
            const float lo2i = hi > ei ? (hi - ei) * (hi - ei) * elo : 0.f;
            const float hi2i = (hi + ei) * (hi + ei) * ehi;
            for (long long q = q0; q < q1; ++q) {
                if (q == p) continue;
                float dx, dy, dz;
                if (!wide) {
                    const float4 f = a.posf[q];
                    dx = ox + f.x; dy = oy + f.y; dz = oz + f.z;
                } else {
                    const uint4 Xj = a.posm[q];
                    dx = (float)(int)(Xj.x - Xi.x) * sf; dy = (float)(int)(Xj.y - Xi.y) * sf;
                    dz = (float)(int)(Xj.z - Xi.z) * sf;
                }
                const float r2 = dx * dx + dy * dy + dz * dz;
                const float hj = a.fvel[q].w;
                const float ej = eL + 2.f * rel * hj;
                const bool mi = r2 < hi2i, mj = r2 < (hj + ej) * (hj + ej) * ehi;
                if (!(mi || mj)) continue;
                bool in = r2 < lo2i || r2 < (hj > ej ? (hj - ej) * (hj - ej) * elo : 0.f);
                if (!in) {
                    const unsigned long long D2 = exact_d2(Xi, a.posm[q]);
                    if (HHi < 0.0) {
                        const double Hd = (double)hi * 4294967296.0 / L;
                        HHi = Hd * Hd;
                    }
                    const double Hj = (double)hj * 4294967296.0 / L;
                    in = (mi && exact_pred(D2, HHi)) || (mj && exact_pred(D2, Hj * Hj));
                }
                if (!in) continue;
                ++np;
                if (HASH) hs += splitmix64((unsigned long long)a.perm[q]);
                sm.hits.f[nh++][lane] = (int)q;
            }
            tests += (unsigned long long)(q1 - q0);
        };
        const unsigned wm = __ballot_sync(0xffffffffu, valid);
        coop_walk(sm, B, a.node_c, a.node_e, Xi, sf, wm, [&](float4 e) { return fmaxf(hi, e.w); }, leaf, drain);
        if (valid) {
            a.acc[3 * (size_t)oi] = (float)((double)Sx - (double)Cx);
            a.acc[3 * (size_t)oi + 1] = (float)((double)Sy - (double)Cy);
            a.acc[3 * (size_t)oi + 2] = (float)((double)Sz - (double)Cz);
            a.dudt[oi] = (float)((double)Su - (double)Cu);   // final accumulation in FP64
            a.vsig[oi] = vsmax;
            if (HASH) a.hash[oi] = hs;
            c_pairs += (unsigned long long)np;
            c_tests += tests;
        }
        ++c_groups;
    }
    c_pairs = warp_sum(c_pairs);
    c_tests = warp_sum(c_tests);
    if (lane == 0) {
        atomicAdd(&a.ctr->force_pairs, c_pairs);
        atomicAdd(&a.ctr->pair_tests, c_tests);
        atomicAdd(&a.ctr->groups, c_groups);
    }
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------

template <typename Kern>
static cudaError_t coop_launch(sph_ctx* ctx, Kern k, const CoopArgs& args, int bps, int kind, int timed,
                               cudaStream_t s) {
    const int blocks = ctx->sm_count * std::min(bps > 0 ? bps : kCoopMinBlocks, kCoopMaxBps);
    cudaEvent_t ea = nullptr, eb = nullptr;
    if (timed) {
        ea = timing_event(ctx);
        eb = timing_event(ctx);
        if (!ea || !eb) return cudaErrorMemoryAllocation;
        cudaEventRecord(ea, s);
    }
    k<<<blocks, kCoopWarps * 32, 0, s>>>(args);
    ++ctx->launches;
    if (timed) {
        cudaEventRecord(eb, s);
        ctx->timed.push_back({ea, eb, kind});
    }
    return cudaGetLastError();
}

static CoopArgs coop_common(sph_ctx* ctx, const sph_grid* g, unsigned* queue) {
    CoopArgs c = {};
    c.boxes = g->boxes;
    c.groups = g->groups;
    c.n_groups = g->n_groups;
    c.queue = queue;
    c.act = g->act;
    c.posm = g->posm;
    c.posf = g->posf;
    c.perm = g->perm;
    c.node_c = g->node_c;
    c.node_e = g->node_e;
    c.node_lo = g->node_lo;
    c.node_hi = g->node_hi;
    c.ctr = ctx->counters;
    return c;
}

cudaError_t launch_density_coop(sph_ctx* ctx, const DensityLaunch& a, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(ctx->queue + 2, 0, sizeof(unsigned), s);
    if (e) return e;
    CoopArgs c = coop_common(ctx, a.g, ctx->queue + 2);
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
    c.lcache = a.g->lcache;
    return a.hash ? coop_launch(ctx, k_density_coop<true>, c, a.blocks_per_sm, 0, a.time_kernels, s)
                  : coop_launch(ctx, k_density_coop<false>, c, a.blocks_per_sm, 0, a.time_kernels, s);
}

cudaError_t launch_force_coop(sph_ctx* ctx, const ForceLaunch& a, cudaStream_t s) {
    force_pack(a.g, a.vel, a.u, a.h, a.rho, a.omega, (float)a.gamma, s);
    ++ctx->launches;
    cudaError_t e = cudaMemsetAsync(ctx->queue + 3, 0, sizeof(unsigned), s);
    if (e) return e;
    CoopArgs c = coop_common(ctx, a.g, ctx->queue + 3);
    c.fvel = a.g->fvel;
    c.fthermo = a.g->fthermo;
    c.acc = a.acc;
    c.dudt = a.dudt;
    c.vsig = a.vsig;
    c.alpha = (float)a.alpha;
    c.hash = a.hash;
    return a.hash ? coop_launch(ctx, k_force_coop<true>, c, a.blocks_per_sm, 1, a.time_kernels, s)
                  : coop_launch(ctx, k_force_coop<false>, c, a.blocks_per_sm, 1, a.time_kernels, s);
}

}  // namespace sph
