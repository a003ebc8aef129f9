// wpp.cu -- warp-per-particle density and force kernels.
//
// One warp per active particle. The warp walks the hierarchy for its particle
// alone, popping up to four nodes per step and testing their children one per
// lane, and keeps the particle's leaf list (with each leaf's centre offset and
// rounding bound) in shared memory. The candidates of that list are then
// tested 32 at a time, one per lane (lanes 8k..8k+7 on the eight particles of
// the k-th leaf of the step, a coalesced 128-byte load), and the pairs in the
// neighbour set are compacted by ballot into a warp-wide hit buffer whose
// pair terms are evaluated 32 at a time, one per lane. Every step therefore
// runs with (nearly) all lanes busy, whatever the lengths of the neighbour
// lists of nearby particles. Per-lane partial sums are compensated (Kahan) and
// folded across the warp with an error-free (TwoSum) butterfly, so the result
// is deterministic and carries the compensation of a sequential sum.
//
// Density keeps the leaf list of a walk at 1.06 h across the h iterations
// (Newton on N^(1/3) with an FP64 bracket, as in the other paths) and walks
// again only when h leaves the walk radius. The neighbour predicate is the
// exact one ((double)D2 < (h 2^32/L)^2) inside a thin band around the FP32
// radius test, as elsewhere.
#include <algorithm>

#include "internal.cuh"

namespace sph {

constexpr int kWppWarps = 4;
constexpr int kWppThreads = kWppWarps * 32;
// Register budgets: 8 resident blocks (32 warps, 64 registers) or 6 (24 warps,
// 80 registers); the launch takes the one matching blocks_per_sm. Defaults
// (measured, 10M clustered): 8 for both passes.
constexpr int kWppDensityBps = 8;
constexpr int kWppForceBps = 8;
constexpr int kWppMaxBps = 16;
constexpr int kWppStack = 256;       // see the bound below
constexpr int kWppPop4 = 96;         // pop four nodes per step only while sp <= this
constexpr int kWppLeaves = 128;      // leaf list per warp; a step adds <= 32
constexpr int kWppHits = 64;         // hit buffer per warp; drained at >= 32
constexpr int kWppNear = 128;        // density: pairs within the walk radius, kept across h iterations
constexpr float kWppWalkR = 1.06f;   // density walks at 1.06 h so that later iterations reuse the list

// Stack bound: a pop-4 step starts from sp <= 96 and ends at sp <= 92 + 32 =
// 124. Above that, in the pop-1 regime, the entries above the base form a
// depth-first stack with at most 7 pending siblings per level, so sp stays
// below 124 + 8 * kMaxLev = 220 < kWppStack.

struct WppSmem {
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
    // force
    const float4* fvel;
    const float4* fthermo;
    const float4* fposh;         // per force call: leaf-relative position, h
    float* acc;
    float* dudt;
    float* vsig;
    float alpha;
    unsigned long long* hash;
    Counters* ctr;
};

__device__ __forceinline__ int wpp_box(const BoxDesc* boxes, int nb, long long p) {
    int lo = 0, hi = nb - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (boxes[mid].off <= p) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Error-free fold of per-lane compensated sums (value = s - c) across the
// warp: TwoSum of the two partial sums, the rounding error moved into c.
// Every lane ends with the same (s, c): both orders of a TwoSum are exact.
__device__ __forceinline__ void wpp_fold(float& s, float& c) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float s2 = __shfl_xor_sync(0xffffffffu, s, o), c2 = __shfl_xor_sync(0xffffffffu, c, o);
        const float t = __fadd_rn(s, s2);
        const float bp = __fsub_rn(t, s);
        const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(s2, bp));
        s = t;
        c = __fsub_rn(__fadd_rn(c, c2), e);
    }
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

// Candidates per lane per step of the candidate loop: the loads of WPP_TILES
// tiles of 32 are issued before any of them is used.
#ifndef WPP_TILES
#define WPP_TILES 1
#endif
constexpr int kWppU = WPP_TILES;

// ---------------------------------------------------------------------------
// Density
// ---------------------------------------------------------------------------

template <bool HASH, int MINB>
__global__ void __launch_bounds__(kWppThreads, MINB) k_density_wpp(WppArgs a) {
    __shared__ WppSmem smem[kWppWarps];
    WppSmem& sm = smem[threadIdx.x >> 5];
    const unsigned lane = lane_id();
    const unsigned lt = (1u << lane) - 1u;
    const float rel = 9.5367431640625e-07f;  // 2^-20
    const float nt = (float)a.n_target, nt3 = 3.f * nt, tol3 = 3.f * (float)a.n_tol;
    const int cnt = (int)*a.count_ptr;
    unsigned c_pairs = 0, c_evals = 0, c_tests = 0, c_status = 0;   // per warp (32-bit suffices)
    for (;;) {
        int t0 = 0;
        if (lane == 0) t0 = (int)atomicAdd(a.queue, (unsigned)a.chunk);
        t0 = __shfl_sync(0xffffffffu, t0, 0);
        if (t0 >= cnt) break;
        const int t1 = min(t0 + a.chunk, cnt);
        for (int t = t0; t < t1; ++t) {
            const int p = a.act[t];
            const BoxDesc& B = a.boxes[a.n_boxes == 1 ? 0 : wpp_box(a.boxes, a.n_boxes, p)];
            const float sf = B.sf;
            const int off = (int)B.off, pend = (int)(B.off + B.n);
            const uint4 Xi = a.posm[p];
            const int oi = a.perm[p];
            float h = a.h[oi];
            if (a.guess_h || !(h > 0.f) || !isfinite(h))
                h = wpp_guess_h(B, a.node_lo, a.node_hi, p, ldexp(B.L, -32), a.n_target);
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
                        const int li = base + (int)(lane >> 3);
                        bool in = false;
                        float r2 = 0.f, m = 0.f;
                        int q = -1;
                        if (li < nlf) {
                            const int id = sm.lid[li];
                            const float4 o = sm.lof[li];
                            q = off + (id & 0x7fffffff) * kLeaf + (int)(lane & 7u);
                            if (q < pend) {
                                float dx, dy, dz;
                                if (id >= 0) {
                                    const float4 f = __ldg(a.posf + q);
                                    dx = o.x + f.x; dy = o.y + f.y; dz = o.z + f.z; m = f.w;
                                } else {
                                    const uint4 Xj = a.posm[q];
                                    dx = (float)(int)(Xj.x - Xi.x) * sf; dy = (float)(int)(Xj.y - Xi.y) * sf;
                                    dz = (float)(int)(Xj.z - Xi.z) * sf; m = __uint_as_float(Xj.w);
                                }
                                r2 = dx * dx + dy * dy + dz * dz;
                                const float eL = o.w + 2.f * rel * R;
                                const float hi2 = (R + eL) * (R + eL) * (1.f + 4.f * rel);
                                if (r2 < hi2) {
                                    if (near) {
                                        in = true;   // kept: the exact test at h is made when evaluating
                                    } else {
                                        const float lo2 = R > eL ? (R - eL) * (R - eL) * (1.f - 4.f * rel) : 0.f;
                                        in = r2 < lo2 || exact_in(q);
                                    }
                                }
                                ++c_tests;
                            } else {
                                q = -1;
                            }
                        }
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
                        __syncwarp();
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
                    wpp_walk(sm, B, a.node_c, a.node_e, Xi, sf, nlf, complete, [&](float4) { return Rw; },
                             [&]() { process(false); nlf = 0; });
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
                float Cw = 0.f, Cdw = 0.f;
                wpp_fold(Sw, Cw);
                wpp_fold(Sdw, Cdw);
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
            float Cmw = 0.f, Cmdw = 0.f;
            wpp_fold(Smw, Cmw);
            wpp_fold(Smdw, Cmdw);
            nn = warp_sum(nn);
            if (HASH) hs = warp_sum(hs);
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
    const unsigned long long all_tests = warp_sum((unsigned long long)c_tests);
    if (lane == 0) {
        atomicAdd(&a.ctr->density_pairs, (unsigned long long)c_pairs);
        atomicAdd(&a.ctr->density_evals, (unsigned long long)c_evals);
        atomicAdd(&a.ctr->pair_tests, all_tests);
        if (c_status) atomicOr(&a.ctr->status, c_status);
    }
}

// ---------------------------------------------------------------------------
// Force
// ---------------------------------------------------------------------------

template <bool HASH, int MINB>
__global__ void __launch_bounds__(kWppThreads, MINB) k_force_wpp(WppArgs a) {
    __shared__ WppSmem smem[kWppWarps];
    WppSmem& sm = smem[threadIdx.x >> 5];
    const unsigned lane = lane_id();
    const unsigned lt = (1u << lane) - 1u;
    const float rel = 9.5367431640625e-07f;
    const float elo = 1.f - 4.f * rel, ehi = 1.f + 4.f * rel;
    const float kNorm = (float)(8.0 / 3.141592653589793);
    const float alpha = a.alpha;
    const int cnt = (int)*a.count_ptr;
    unsigned long long c_pairs = 0, c_tests = 0;   // lane 0's per-warp totals
    for (;;) {
        int t0 = 0;
        if (lane == 0) t0 = (int)atomicAdd(a.queue, (unsigned)a.chunk);
        t0 = __shfl_sync(0xffffffffu, t0, 0);
        if (t0 >= cnt) break;
        const int t1 = min(t0 + a.chunk, cnt);
        for (int t = t0; t < t1; ++t) {
            const int p = a.act[t];
            const BoxDesc& B = a.boxes[a.n_boxes == 1 ? 0 : wpp_box(a.boxes, a.n_boxes, p)];
            const float sf = B.sf;
            const int off = (int)B.off, pend = (int)(B.off + B.n);
            const uint4 Xi = a.posm[p];
            const int oi = a.perm[p];
            const float4 vi = a.fvel[p];
            const float4 thi = a.fthermo[p];
            const float hi = vi.w, hinvi = thi.w, rhoi = thi.x, Ai = thi.y, ci = thi.z;
            const float normi = kNorm * hinvi * hinvi * hinvi * hinvi;
            double HHi = -1.0;
            float Sx = 0.f, Sy = 0.f, Sz = 0.f, Su = 0.f, vsmax = 0.f;   // per-lane partial sums
            int np = 0, nh = 0, nlf = 0;
            unsigned tests = 0;
            bool complete = true;
            unsigned long long hs = 0;
            auto drain = [&](int k) {
                if ((int)lane < k) {
                    const float4 e = sm.hit.f[lane];
                    const int q = __float_as_int(e.w);
                    const float dx = e.x, dy = e.y, dz = e.z;
                    const float r2 = dx * dx + dy * dy + dz * dz;
                    const float4 vj = __ldg(a.fvel + q);
                    const float4 thj = __ldg(a.fthermo + q);
                    const float mj = __ldg(&a.posf[q].w);
                    if (r2 <= 0.f) {  // coincident: no direction, no force
                        vsmax = fmaxf(vsmax, ci + thj.z);
                    } else {
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
                        Sx += coef * dx;
                        Sy += coef * dy;
                        Sz += coef * dz;
                        Su += mj * vr * (Ai * Fi + 0.5f * PI * Fbar);
                    }
                }
                __syncwarp();
            };
            auto process = [&]() {
                for (int base = 0; base < nlf; base += 4 * kWppU) {
                    int q[kWppU], id[kWppU];
                    float4 o[kWppU], f[kWppU];
#pragma unroll
                    for (int u = 0; u < kWppU; ++u) {
                        const int li = base + 4 * u + (int)(lane >> 3);
                        q[u] = -1;
                        id[u] = 0;
                        if (li < nlf) {
                            id[u] = sm.lid[li];
                            o[u] = sm.lof[li];
                            const int qq = off + (id[u] & 0x7fffffff) * kLeaf + (int)(lane & 7u);
                            if (qq < pend) {
                                q[u] = qq;
                                ++tests;
                            }
                        }
                    }
#pragma unroll
                    for (int u = 0; u < kWppU; ++u)
                        if (q[u] >= 0) f[u] = __ldg(a.fposh + q[u]);
#pragma unroll
                    for (int u = 0; u < kWppU; ++u) {
                        bool in = false;
                        float dx = 0.f, dy = 0.f, dz = 0.f;
                        if (q[u] >= 0 && q[u] != p) {
                            const float hj = f[u].w;
                            if (id[u] >= 0) {
                                dx = o[u].x + f[u].x; dy = o[u].y + f[u].y; dz = o[u].z + f[u].z;
                            } else {
                                const uint4 Xj = a.posm[q[u]];
                                dx = (float)(int)(Xj.x - Xi.x) * sf; dy = (float)(int)(Xj.y - Xi.y) * sf;
                                dz = (float)(int)(Xj.z - Xi.z) * sf;
                            }
                            const float r2 = dx * dx + dy * dy + dz * dz;
                            const float ei = o[u].w + 2.f * rel * hi, ej = o[u].w + 2.f * rel * hj;
                            const bool mi = r2 < (hi + ei) * (hi + ei) * ehi, mjb = r2 < (hj + ej) * (hj + ej) * ehi;
                            if (mi || mjb) {
                                in = r2 < (hi > ei ? (hi - ei) * (hi - ei) * elo : 0.f) ||
                                     r2 < (hj > ej ? (hj - ej) * (hj - ej) * elo : 0.f);
                                if (!in) {
                                    const unsigned long long D2 = exact_d2(Xi, a.posm[q[u]]);
                                    if (HHi < 0.0) HHi = wpp_hh(hi, B.L);
                                    in = (mi && exact_pred(D2, HHi)) || (mjb && exact_pred(D2, wpp_hh(hj, B.L)));
                                }
                            }
                        }
                        const unsigned hm = __ballot_sync(0xffffffffu, in);
                        if (in) {
                            sm.hit.f[nh + __popc(hm & lt)] = make_float4(dx, dy, dz, __int_as_float(q[u]));
                            ++np;
                            if (HASH) hs += splitmix64((unsigned long long)a.perm[q[u]]);
                        }
                        nh += __popc(hm);
                        __syncwarp();
                        if (nh >= 32) {
                            drain(32);
                            nh -= 32;
                            if ((int)lane < nh) sm.hit.f[lane] = sm.hit.f[32 + lane];
                            __syncwarp();
                        }
                    }
                }
            };
            wpp_walk(sm, B, a.node_c, a.node_e, Xi, sf, nlf, complete, [&](float4 e) { return fmaxf(hi, e.w); },
                     [&]() { process(); nlf = 0; });
            process();
            drain(nh);
            float Cx = 0.f, Cy = 0.f, Cz = 0.f, Cu = 0.f;
            wpp_fold(Sx, Cx);
            wpp_fold(Sy, Cy);
            wpp_fold(Sz, Cz);
            wpp_fold(Su, Cu);
            vsmax = warp_max(vsmax);
            np = warp_sum(np);
            if (HASH) hs = warp_sum(hs);
            tests = warp_sum(tests);
            if (lane == 0) {
                // each compensated pair folds with one correctly rounded subtraction
                a.acc[3 * (size_t)oi] = __fsub_rn(Sx, Cx);
                a.acc[3 * (size_t)oi + 1] = __fsub_rn(Sy, Cy);
                a.acc[3 * (size_t)oi + 2] = __fsub_rn(Sz, Cz);
                a.dudt[oi] = __fsub_rn(Su, Cu);
                a.vsig[oi] = vsmax;
                if (HASH) a.hash[oi] = hs;
                c_pairs += (unsigned long long)np;
                c_tests += tests;
            }
            __syncwarp();
        }
    }
    if (lane == 0) {
        atomicAdd(&a.ctr->force_pairs, c_pairs);
        atomicAdd(&a.ctr->pair_tests, c_tests);
    }
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------

template <typename Kern>
static cudaError_t wpp_launch(sph_ctx* ctx, Kern k, const WppArgs& args, int blocks, int kind, int timed,
                              cudaStream_t s) {
    cudaEvent_t ea = nullptr, eb = nullptr;
    if (timed) {
        ea = timing_event(ctx);
        eb = timing_event(ctx);
        if (!ea || !eb) return cudaErrorMemoryAllocation;
        cudaEventRecord(ea, s);
    }
    k<<<blocks, kWppThreads, 0, s>>>(args);
    ++ctx->launches;
    if (timed) {
        cudaEventRecord(eb, s);
        ctx->timed.push_back({ea, eb, kind});
    }
    return cudaGetLastError();
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
    return c;
}

cudaError_t launch_density_wpp(sph_ctx* ctx, const DensityLaunch& a, int64_t n_active, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(ctx->queue + 2, 0, sizeof(unsigned), s);
    if (e) return e;
    WppArgs c = wpp_common(ctx, a.g, ctx->queue + 2);
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
    if (bps <= 6)
        return a.hash ? wpp_launch(ctx, k_density_wpp<true, 6>, c, blocks, 0, a.time_kernels, s)
                      : wpp_launch(ctx, k_density_wpp<false, 6>, c, blocks, 0, a.time_kernels, s);
    return a.hash ? wpp_launch(ctx, k_density_wpp<true, 8>, c, blocks, 0, a.time_kernels, s)
                  : wpp_launch(ctx, k_density_wpp<false, 8>, c, blocks, 0, a.time_kernels, s);
}

cudaError_t launch_force_wpp(sph_ctx* ctx, const ForceLaunch& a, int64_t n_active, cudaStream_t s) {
    force_pack(a.g, a.vel, a.u, a.h, a.rho, a.omega, (float)a.gamma, s);
    ++ctx->launches;
    cudaError_t e = cudaMemsetAsync(ctx->queue + 3, 0, sizeof(unsigned), s);
    if (e) return e;
    WppArgs c = wpp_common(ctx, a.g, ctx->queue + 3);
    int blocks = 0;
    const int bps = a.blocks_per_sm > 0 ? a.blocks_per_sm : kWppForceBps;
    wpp_shape(ctx, bps, n_active, blocks, c.chunk);
    c.fvel = a.g->fvel;
    c.fthermo = a.g->fthermo;
    c.fposh = a.g->fposh;
    c.acc = a.acc;
    c.dudt = a.dudt;
    c.vsig = a.vsig;
    c.alpha = (float)a.alpha;
    c.hash = a.hash;
    if (bps <= 6)
        return a.hash ? wpp_launch(ctx, k_force_wpp<true, 6>, c, blocks, 1, a.time_kernels, s)
                      : wpp_launch(ctx, k_force_wpp<false, 6>, c, blocks, 1, a.time_kernels, s);
    return a.hash ? wpp_launch(ctx, k_force_wpp<true, 8>, c, blocks, 1, a.time_kernels, s)
                  : wpp_launch(ctx, k_force_wpp<false, 8>, c, blocks, 1, a.time_kernels, s);
}

}  // namespace sph
